// pct_sap.cu -- string-averaging projections (Sec. II-D, SAP; Censor et al.),
// the paper's reconstruction algorithm, on an explicit CSR A.
//
// One iteration: every string t (rows t, t + M, t + 2M, ... in increasing
// order) starts from the current x and projects its rows one after another,
//   y <- y + lambda (b_i - <a_i, y>) / ||a_i||^2 a_i,
// then x <- sum_t w_t y_t.  The rows of a string depend on each other (each
// projection reads what the previous one wrote), the strings do not: one block
// per string, each with its own copy of y in the workspace (M x n_cols
// floats; the copies of a 2D problem fit in L2), rows in order, the block's
// threads spread over the row's entries.  Per row: gather y at the row's
// columns (L2, bypassing L1 so that the previous row's reductions are seen),
// block sums of a_ij y_j and a_ij^2, then reductions y_j += c a_ij at L2
// (duplicate columns of a row both apply).  The next row's entries are
// prefetched into L2 while the current row is projected.  The averaging
// kernel sums the M copies in FP64 and writes x and, for the next iteration,
// every copy.
#include "pct_kernels.cuh"

namespace pct {

__global__ void k_sap_init(const float* __restrict__ x, float* __restrict__ Y, int M, long long n) {
  const long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (j >= n) return;
  const float v = x[j];
  for (int t = 0; t < M; ++t) Y[(long long)t * n + j] = v;
}

// threads per string: about one per entry of the paper's rows (NEO-2: 239
// entries per row; 14.1 / 12.3 / 18.6 ms per iteration at 128 / 256 / 64)
constexpr int kSapThreads = 256;

__global__ void __launch_bounds__(kSapThreads) k_sap_strings(const long long* __restrict__ row_ptr,
                                                             const int* __restrict__ col,
                                                             const float* __restrict__ val,
                                                             const float* __restrict__ b, long long n_rows, int M,
                                                             float lambda, float* Y, long long n) {
  __shared__ float part[2][kSapThreads / 32];  // the warps' sums of a_ij y_j and a_ij^2
  const int t = blockIdx.x;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  float* y = Y + (long long)t * n;
  long long i = t;
  long long r0 = i < n_rows ? row_ptr[i] : 0, r1 = i < n_rows ? row_ptr[i + 1] : 0;
  for (; i < n_rows; i += M) {
    // the next row of the string: its row pointers now, its entries into L2
    const long long in = i + M;
    long long n0 = 0, n1 = 0;
    if (in < n_rows) {
      n0 = row_ptr[in];
      n1 = row_ptr[in + 1];
      for (long long p = (n0 & ~31LL) + 32LL * tid; p < n1; p += 32LL * kSapThreads) {
        asm volatile("prefetch.global.L2 [%0];" ::"l"(col + p));
        asm volatile("prefetch.global.L2 [%0];" ::"l"(val + p));
      }
    }
    float dot = 0.f, nrm = 0.f;
#pragma unroll 2
    for (long long e = r0 + tid; e < r1; e += kSapThreads) {
      const int c = __ldg(col + e);
      const float v = __ldg(val + e);
      dot = fmaf(v, __ldcg(y + c), dot);
      nrm = fmaf(v, v, nrm);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      dot += __shfl_xor_sync(0xffffffffu, dot, o);
      nrm += __shfl_xor_sync(0xffffffffu, nrm, o);
    }
    if (lane == 0) {
      part[0][wid] = dot;
      part[1][wid] = nrm;
    }
    __syncthreads();
    // every thread forms the same sums in the same order
    dot = part[0][0];
    nrm = part[1][0];
#pragma unroll
    for (int w = 1; w < kSapThreads / 32; ++w) {
      dot += part[0][w];
      nrm += part[1][w];
    }
    if (nrm > 0.f) {
      const float c = __fdiv_rn(lambda * (__ldg(b + i) - dot), nrm);
      for (long long e = r0 + tid; e < r1; e += kSapThreads)
        asm volatile("red.global.add.f32 [%0], %1;" ::"l"(y + __ldg(col + e)), "f"(c * __ldg(val + e)) : "memory");
    }
    // this row's reductions are ordered before the next row's gathers (both
    // at L2), and every thread has read `part` before it is written again
    __threadfence_block();
    __syncthreads();
    r0 = n0;
    r1 = n1;
  }
}

// x = sum_t w_t Y_t (FP64 sum); refill = the copies start the next iteration from x
__global__ void k_sap_average(float* __restrict__ Y, const double* __restrict__ w, int M, long long n,
                              float* __restrict__ x, int refill) {
  const long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (j >= n) return;
  double s = 0.0;
  for (int t = 0; t < M; ++t) s = fma(w[t], (double)Y[(long long)t * n + j], s);
  const float v = (float)s;
  x[j] = v;
  if (refill)
    for (int t = 0; t < M; ++t) Y[(long long)t * n + j] = v;
}

size_t sap_workspace_bytes(long long n_cols, int M) {
  return (((size_t)M * sizeof(double) + 255) & ~(size_t)255) + (size_t)M * (size_t)n_cols * sizeof(float);
}

void launch_sap(const long long* row_ptr, const int* col, const float* val, const float* b, long long n_rows,
                long long n_cols, int M, const double* w_dev, float lambda, int iterations, float* x, void* ws,
                cudaStream_t st) {
  if (iterations <= 0 || n_cols <= 0) return;
  float* Y = (float*)((char*)ws + (((size_t)M * sizeof(double) + 255) & ~(size_t)255));
  const unsigned blocks = (unsigned)((n_cols + 255) / 256);
  k_sap_init<<<blocks, 256, 0, st>>>(x, Y, M, n_cols);
  for (int it = 0; it < iterations; ++it) {
    if (n_rows > 0)
      k_sap_strings<<<(unsigned)M, kSapThreads, 0, st>>>(row_ptr, col, val, b, n_rows, M, lambda, Y, n_cols);
    k_sap_average<<<blocks, 256, 0, st>>>(Y, w_dev, M, n_cols, x, it + 1 < iterations);
  }
}

}  // namespace pct
