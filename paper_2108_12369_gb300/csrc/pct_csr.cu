// pct_csr.cu -- projectors on an explicit CSR A (Sec. II, A x = b):
// y = A x (one warp per row, coalesced col/val reads, FP32 accumulation)
// and g += A^T r (one warp per row, FP32 atomics on g).  Both are HBM-bound
// at 8 bytes per nonzero.
#include "pct_kernels.cuh"

namespace pct {

// Entries are taken 256 per warp and round: each lane issues its eight col /
// val loads (streamed with an evict-first hint, so that x keeps its place in
// the L2), then its eight x gathers, before the first product needs one
// (NEO-2 forward 57.5 -> 59.4 % of measured HBM against four per lane).
constexpr int kCsrUnroll = 8;

__global__ void k_csr_forward(const long long* __restrict__ row_ptr, const int* __restrict__ col,
                              const float* __restrict__ val, long long row0, long long n,
                              const float* __restrict__ x, float* __restrict__ y) {
  long long w = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
  int lane = threadIdx.x & 31;
  if (w >= n) return;
  long long r = row0 + w;
  long long beg = row_ptr[r], end = row_ptr[r + 1];
  float acc = 0.0f;
  for (long long e0 = beg + lane; e0 < end; e0 += 32 * kCsrUnroll) {
    int c[kCsrUnroll];
    float v[kCsrUnroll], xv[kCsrUnroll];
#pragma unroll
    for (int u = 0; u < kCsrUnroll; ++u) {
      const long long e = e0 + 32 * u;
      c[u] = e < end ? __ldcs(col + e) : -1;
      v[u] = e < end ? __ldcs(val + e) : 0.0f;
    }
#pragma unroll
    for (int u = 0; u < kCsrUnroll; ++u) xv[u] = c[u] >= 0 ? __ldg(x + c[u]) : 0.0f;
#pragma unroll
    for (int u = 0; u < kCsrUnroll; ++u)
      if (c[u] >= 0) acc = fmaf(v[u], xv[u], acc);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  if (lane == 0) y[w] = acc;
}

__global__ void k_csr_adjoint(const long long* __restrict__ row_ptr, const int* __restrict__ col,
                              const float* __restrict__ val, long long row0, long long n,
                              const float* __restrict__ r, float* __restrict__ g) {
  long long w = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
  int lane = threadIdx.x & 31;
  if (w >= n) return;
  float ri = r[w];
  if (ri == 0.0f) return;
  long long rr = row0 + w;
  long long beg = row_ptr[rr], end = row_ptr[rr + 1];
  // plain `red` with no memory clobber (nothing here reads g): the next
  // entries' col / val loads may be issued ahead of it
  for (long long e0 = beg + lane; e0 < end; e0 += 32 * kCsrUnroll) {
    int c[kCsrUnroll];
    float v[kCsrUnroll];
#pragma unroll
    for (int u = 0; u < kCsrUnroll; ++u) {
      const long long e = e0 + 32 * u;
      c[u] = e < end ? __ldcs(col + e) : -1;
      v[u] = e < end ? __ldcs(val + e) : 0.0f;
    }
#pragma unroll
    for (int u = 0; u < kCsrUnroll; ++u)
      if (c[u] >= 0) asm volatile("red.global.add.f32 [%0], %1;" ::"l"(g + c[u]), "f"(v[u] * ri));
  }
}

void launch_csr_forward(const long long* row_ptr, const int* col, const float* val, long long row0,
                        long long n, const float* x, float* y, cudaStream_t st) {
  if (n <= 0) return;
  long long threads = n * 32;
  k_csr_forward<<<(unsigned)((threads + 255) / 256), 256, 0, st>>>(row_ptr, col, val, row0, n, x, y);
}

void launch_csr_adjoint(const long long* row_ptr, const int* col, const float* val, long long row0,
                        long long n, const float* r, float* g, cudaStream_t st) {
  if (n <= 0) return;
  long long threads = n * 32;
  k_csr_adjoint<<<(unsigned)((threads + 255) / 256), 256, 0, st>>>(row_ptr, col, val, row0, n, r, g);
}

}  // namespace pct
