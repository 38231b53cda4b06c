// pct_raster.cu -- the NEO phantom raster x_true (Sec. II-A): RSP of every
// voxel by its centre point, the mean of its 2^dim corner points, or the
// weighted-area average over S^dim sub-sample midpoints; regions painted in
// order (the last region containing a point gives its RSP).
//
// Definition (FP64): point p_a = o_a + k_a h_a (k_a = index, or index + 1/2
// for the centre); p lies in region r when sum_a ((p_a - c_a) / a_a)^2 <= 1,
// summed over the axes in order; a corner raster sums the corners' RSP in
// corner order (bit a of the corner number = +1 along axis a) and scales by
// 1 / 2^dim; the result is rounded once to FP32.
//
// GB300 form: a block rasterises a tile of voxels.  Adjacent voxels share
// corners, so the tile's (TX+1)(TY+1)(TZ+1) corner points are classified once
// into shared memory (about 1.1 - 1.5 tests per voxel instead of 4 or 8).
// Each point test runs in FP32 with a bound on its distance to the FP64
// definition's q; only points within that bound of an ellipse's surface are
// tested again in FP64, exactly as defined.  The corner sums stay FP64 in the
// definition's order.  Output bit for bit equal to the definition.
#include "pct_kernels.cuh"

namespace pct {

namespace {

constexpr int kTX = 32;

template <int DIM>
struct Tile {
  static constexpr int TX = kTX, TY = DIM == 3 ? 8 : 16, TZ = DIM == 3 ? 4 : 1;
  static constexpr int CX = TX + 1, CY = TY + 1, CZ = DIM == 3 ? TZ + 1 : 1;
  static constexpr int NC = CX * CY * CZ;
};

// region r contains p: the FP64 definition
__device__ __forceinline__ bool inside_f64(const PhantomDev& ph, int r, int axes, const double p[3]) {
  double q = 0.0;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    if (a >= axes) break;
    const double d = (p[a] - ph.c[r][a]) / ph.a[r][a];
    q = q + d * d;
  }
  return q <= 1.0;
}

// The last region containing p (-1: none).  q in FP32 differs from the real
// q by at most 2^-19 sum_a B_a^2, B_a = (|p_a| + |c_a|) / a_a (rounding of p,
// c and 1/a to FP32, the difference, product, square and sum); the FP64 q by
// at most 2^-50 of that.  Outside 2^-16 sum B_a^2 of 1 both decide alike.
__device__ __forceinline__ int region_of(const PhantomDev& ph, int axes, const double p[3]) {
  float pf[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) pf[a] = (float)p[a];
  for (int r = ph.n_regions - 1; r >= 0; --r) {
    float q = 0.f, bnd = 0.f;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      if (a >= axes) break;
      const float ra = (float)ph.ra[r][a];
      const float d = (pf[a] - (float)ph.c[r][a]) * ra;
      const float B = (fabsf(pf[a]) + fabsf((float)ph.c[r][a])) * ra;
      q = fmaf(d, d, q);
      bnd = fmaf(B, B, bnd);
    }
    const float e = 1.52587890625e-05f * bnd;  // 2^-16
    bool in;
    if (q < 1.f - e)
      in = true;
    else if (q > 1.f + e)
      in = false;
    else
      in = inside_f64(ph, r, axes, p);
    if (in) return r;
  }
  return -1;
}

}  // namespace

// x_true of one tile of voxels per block (corner or centre raster)
template <int DIM>
__global__ void __launch_bounds__(256) k_raster_tile(PhantomDev ph, float* __restrict__ x) {
  using T = Tile<DIM>;
  __shared__ double crd[T::CX + T::CY + T::CZ];  // corner coordinates along each axis
  __shared__ signed char reg[T::NC];
  const GridDev& g = ph.g;
  const int axes = (DIM == 3 && ph.kind == PCT_ELLIPSOID) ? 3 : 2;
  // tile of this block (1D grid: any grid shape the phantom accepts fits)
  const long long ntx = (g.n[0] + T::TX - 1) / T::TX, nty = (g.n[1] + T::TY - 1) / T::TY;
  const long long tb = blockIdx.x;
  const int i0 = (int)(tb % ntx) * T::TX, j0 = (int)((tb / ntx) % nty) * T::TY, k0 = (int)(tb / (ntx * nty)) * T::TZ;
  const bool corner = ph.raster == PCT_RASTER_CORNER;
  const double off = corner ? 0.0 : 0.5;
  for (int t = threadIdx.x; t < T::CX + T::CY + T::CZ; t += blockDim.x) {
    const int a = t < T::CX ? 0 : (t < T::CX + T::CY ? 1 : 2);
    const int k = t - (a == 0 ? 0 : (a == 1 ? T::CX : T::CX + T::CY)) + (a == 0 ? i0 : (a == 1 ? j0 : k0));
    crd[t] = a < DIM ? g.o[a] + ((double)k + off) * g.h[a] : 0.0;
  }
  __syncthreads();
  if (corner) {
    for (int c = threadIdx.x; c < T::NC; c += blockDim.x) {
      const int ci = c % T::CX, cj = (c / T::CX) % T::CY, ck = c / (T::CX * T::CY);
      const double p[3] = {crd[ci], crd[T::CX + cj], DIM == 3 ? crd[T::CX + T::CY + ck] : 0.0};
      const bool live = i0 + ci <= g.n[0] && j0 + cj <= g.n[1] && (DIM == 2 || k0 + ck <= g.n[2]);
      reg[c] = (signed char)(live ? region_of(ph, axes, p) : -1);
    }
    __syncthreads();
  }
  constexpr int NV = T::TX * T::TY * T::TZ;
  for (int v = threadIdx.x; v < NV; v += blockDim.x) {
    const int vi = v % T::TX, vj = (v / T::TX) % T::TY, vk = v / (T::TX * T::TY);
    const int ix = i0 + vi, iy = j0 + vj, iz = k0 + vk;
    if (ix >= g.n[0] || iy >= g.n[1] || (DIM == 3 && iz >= g.n[2])) continue;
    double val;
    if (corner) {
      constexpr int nc = DIM == 3 ? 8 : 4;
      double sum = 0.0;
#pragma unroll
      for (int c = 0; c < nc; ++c) {
        const int r = reg[(vi + (c & 1)) + T::CX * ((vj + ((c >> 1) & 1)) + T::CY * (DIM == 3 ? vk + ((c >> 2) & 1) : 0))];
        sum = sum + (r >= 0 ? ph.rsp[r] : 0.0);
      }
      val = sum * (1.0 / (double)nc);
    } else {
      const double p[3] = {crd[vi], crd[T::CX + vj], DIM == 3 ? crd[T::CX + T::CY + vk] : 0.0};
      const int r = region_of(ph, axes, p);
      val = r >= 0 ? ph.rsp[r] : 0.0;
    }
    x[ix + (long long)g.n[0] * (iy + (long long)g.n[1] * (DIM == 3 ? iz : 0))] = (float)val;
  }
}

// Weighted-area raster: thread per voxel, S^dim sub-sample midpoints, each
// classified by region_of; x = (sum_r rsp_r count_r) / S^dim in FP64, the
// regions in order (the counts are exact, so the result is the definition's).
template <int DIM>
__global__ void __launch_bounds__(256) k_raster_area(PhantomDev ph, float* __restrict__ x, long long nvox) {
  __shared__ double u[64];                   // (k + 1/2) / S
  __shared__ int cnt[kMaxRegions][256];      // per thread: sub-samples per region
  const int S = ph.area_s;
  for (int k = threadIdx.x; k < S; k += blockDim.x) u[k] = ((double)k + 0.5) / (double)S;
  for (int r = 0; r < ph.n_regions; ++r) cnt[r][threadIdx.x] = 0;
  __syncthreads();
  const long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (j >= nvox) return;
  const GridDev& g = ph.g;
  const int axes = (DIM == 3 && ph.kind == PCT_ELLIPSOID) ? 3 : 2;
  const int ix = (int)(j % g.n[0]);
  const long long q = j / g.n[0];
  const int iy = (int)(q % g.n[1]);
  const int iz = DIM == 3 ? (int)(q / g.n[1]) : 0;
  double p[3] = {0.0, 0.0, 0.0};
  for (int kz = 0; kz < (DIM == 3 ? S : 1); ++kz) {
    if (DIM == 3) p[2] = g.o[2] + ((double)iz + u[kz]) * g.h[2];
    for (int ky = 0; ky < S; ++ky) {
      p[1] = g.o[1] + ((double)iy + u[ky]) * g.h[1];
      for (int kx = 0; kx < S; ++kx) {
        p[0] = g.o[0] + ((double)ix + u[kx]) * g.h[0];
        const int r = region_of(ph, axes, p);
        if (r >= 0) ++cnt[r][threadIdx.x];
      }
    }
  }
  const double nsub = (double)S * (double)S * (DIM == 3 ? (double)S : 1.0);
  double sum = 0.0;
  for (int r = 0; r < ph.n_regions; ++r) sum = sum + ph.rsp[r] * (double)cnt[r][threadIdx.x];
  x[j] = (float)(sum / nsub);
}

void launch_raster(const PhantomDev& ph, float* x, long long nvox, cudaStream_t st) {
  if (nvox <= 0) return;
  const GridDev& g = ph.g;
  if (ph.raster == PCT_RASTER_AREA) {
    const unsigned blocks = (unsigned)((nvox + 255) / 256);
    if (g.dim == 3)
      k_raster_area<3><<<blocks, 256, 0, st>>>(ph, x, nvox);
    else
      k_raster_area<2><<<blocks, 256, 0, st>>>(ph, x, nvox);
    return;
  }
  if (g.dim == 3) {
    using T = Tile<3>;
    const long long tiles = (long long)((g.n[0] + T::TX - 1) / T::TX) * ((g.n[1] + T::TY - 1) / T::TY) *
                            ((g.n[2] + T::TZ - 1) / T::TZ);
    k_raster_tile<3><<<(unsigned)tiles, 256, 0, st>>>(ph, x);
  } else {
    using T = Tile<2>;
    const long long tiles = (long long)((g.n[0] + T::TX - 1) / T::TX) * ((g.n[1] + T::TY - 1) / T::TY);
    k_raster_tile<2><<<(unsigned)tiles, 256, 0, st>>>(ph, x);
  }
}

}  // namespace pct
