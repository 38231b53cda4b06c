// pct_f64.cu -- all-FP64 form of the simulation kernels: per-proton path +
// traversal count and fill (Sec. II-B, II-C) and the matrix-free projectors
// (Ax, A^T r).
//
// One thread per proton; every floating-point step is the FP64 definition.
// This is the comparison form for PCT_PREC_MIXED and the exact fallback's
// reference; it is FP64-pipe bound on GB300 (FP64 runs at about 1/70 of
// the FP32 rate there).
#include "pct_kernels.cuh"

namespace pct {

// ---------------------------------------------------------------------------
// Sinks of merged entries
// ---------------------------------------------------------------------------
struct CountSink {
  long long n;
  __device__ void put(int, double) { ++n; }
  __device__ void pend(int) {}
};

struct FillSinkF64 {
  int* col;
  float* val;
  const float* x;
  long long pos, end;  // next position, the end of the row's range (stores stay inside)
  double b;
  bool constant;
  float hconst;
  __device__ void put(int c, double len) {
    if (pos < end) {
      col[pos] = c;
      val[pos] = constant ? hconst : (float)len;
    }
    ++pos;
    b = b + len * (double)__ldg(x + c);
  }
  __device__ void pend(int) {}
};

template <class Sink>
__device__ __forceinline__ void walk_path_f64(const SimDev& S, const PathF64& p, Sink& sink) {
  RowMerge<double> mg;
  mg.init();
  double Va[3], Vb[3];
  path_vertex(S, p, 0, Va);
  for (int q = 0; q + 1 < p.nv; ++q) {
    path_vertex(S, p, q + 1, Vb);
    mg.seg_begin();
    SegF64 sg;
    if (seg_setup_f64(S.ph.g, Va, Vb, sg)) seg_walk_f64(S.ph.g, sg, mg, sink);
    mg.seg_end();
#pragma unroll
    for (int a = 0; a < 3; ++a) Va[a] = Vb[a];
  }
  mg.finish(sink);
}

__global__ void k_count_f64(SimDev S, long long row0, long long n, long long* __restrict__ counts) {
  long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= n) return;
  PathF64 p = path_setup(S, row0 + i);
  CountSink cs{0};
  walk_path_f64(S, p, cs);
  counts[i] = cs.n;
}

__global__ void k_fill_f64(SimDev S, long long row0, long long n, const long long* __restrict__ row_ptr,
                           const float* __restrict__ x, int* __restrict__ col, float* __restrict__ val,
                           float* __restrict__ b) {
  long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= n) return;
  long long row = row0 + i;
  PathF64 p = path_setup(S, row);
  FillSinkF64 fs;
  fs.col = col;
  fs.val = val;
  fs.x = x;
  fs.pos = row_ptr[i];
  fs.end = row_ptr[i + 1];
  fs.b = 0.0;
  fs.constant = (S.md.chord == PCT_CHORD_CONSTANT);
  fs.hconst = (float)S.ph.g.h[0];
  walk_path_f64(S, p, fs);
  if (fs.pos != fs.end) note_row_mismatch(S);
  double bb = fs.b;
  if (S.md.noise == PCT_NOISE_GAUSS_REL) bb = bb * (1.0 + S.md.noise_rel * p.z_noise);
  b[i] = (float)bb;
}

// matrix-free forward: y_i = sum len * x_j with FP64 lengths
struct DotSinkF64 {
  const float* x;
  double acc;
  __device__ void put(int c, double len) { acc = acc + len * (double)__ldg(x + c); }
  __device__ void pend(int) {}
};

__global__ void k_mf_forward_f64(SimDev S, long long row0, long long n, const float* __restrict__ x,
                                 float* __restrict__ y) {
  long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= n) return;
  PathF64 p = path_setup(S, row0 + i);
  DotSinkF64 ds{x, 0.0};
  walk_path_f64(S, p, ds);
  y[i] = (float)ds.acc;
}

struct ScatterSinkF64 {
  float* g;
  float r;
  // plain `red` with no memory clobber (nothing in the kernel reads g)
  __device__ void put(int c, double len) {
    asm volatile("red.global.add.f32 [%0], %1;" ::"l"(g + c), "f"((float)len * r));
  }
  __device__ void pend(int) {}
};

__global__ void k_mf_adjoint_f64(SimDev S, long long row0, long long n, const float* __restrict__ r,
                                 float* __restrict__ g) {
  long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= n) return;
  float ri = r[i];
  if (ri == 0.0f) return;
  PathF64 p = path_setup(S, row0 + i);
  ScatterSinkF64 ss{g, ri};
  walk_path_f64(S, p, ss);
}

void launch_count_f64(const SimDev& S, long long row0, long long n, long long* counts, cudaStream_t st) {
  if (n <= 0) return;
  int threads = 128;
  k_count_f64<<<(unsigned)((n + threads - 1) / threads), threads, 0, st>>>(S, row0, n, counts);
}

void launch_fill_f64(const SimDev& S, long long row0, long long n, const long long* row_ptr,
                     const float* x, int* col, float* val, float* b, cudaStream_t st) {
  if (n <= 0) return;
  int threads = 128;
  k_fill_f64<<<(unsigned)((n + threads - 1) / threads), threads, 0, st>>>(S, row0, n, row_ptr, x, col,
                                                                          val, b);
}

void launch_mf_forward_f64(const SimDev& S, long long row0, long long n, const float* x, float* y,
                           cudaStream_t st) {
  if (n <= 0) return;
  int threads = 128;
  k_mf_forward_f64<<<(unsigned)((n + threads - 1) / threads), threads, 0, st>>>(S, row0, n, x, y);
}

void launch_mf_adjoint_f64(const SimDev& S, long long row0, long long n, const float* r, float* g,
                           cudaStream_t st) {
  if (n <= 0) return;
  int threads = 128;
  k_mf_adjoint_f64<<<(unsigned)((n + threads - 1) / threads), threads, 0, st>>>(S, row0, n, r, g);
}

}  // namespace pct
