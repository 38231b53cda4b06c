// pct_scan.cu -- row pointers of the CSR (Sec. II-C, Fig. 3): exclusive
// scan of the per-row entry counts into int64 (nnz exceeds 2^31 on the
// head-size workloads).  Three passes over kScanTile-row tiles: tile sums,
// a scan of the tile sums, and the in-tile scan plus the tile's offset.
#include "pct_kernels.cuh"

namespace pct {

constexpr int kScanThreads = 256;
constexpr int kPerThread = kScanTile / kScanThreads;  // 16

long long scan_partials_needed(long long n) { return (n + kScanTile - 1) / kScanTile + 1; }

// tile sums of v[0..n)
__global__ void k_tile_sums(const long long* __restrict__ v, long long n, long long* __restrict__ partial) {
  __shared__ long long warp_sum[kScanThreads / 32];
  long long base = (long long)blockIdx.x * kScanTile;
  long long s = 0;
#pragma unroll
  for (int q = 0; q < kPerThread; ++q) {
    long long i = base + (long long)q * kScanThreads + threadIdx.x;
    if (i < n) s += v[i];
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) warp_sum[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x < 32) {
    long long t = (threadIdx.x < kScanThreads / 32) ? warp_sum[threadIdx.x] : 0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
    if (threadIdx.x == 0) partial[blockIdx.x] = t;
  }
}

// exclusive scan of partial[0..nt) in place, one block
__global__ void k_scan_partials(long long* __restrict__ partial, long long nt) {
  __shared__ long long warp_tot[32];
  __shared__ long long carry_s;
  if (threadIdx.x == 0) carry_s = 0;
  __syncthreads();
  for (long long base = 0; base < nt; base += blockDim.x) {
    long long i = base + threadIdx.x;
    long long v = (i < nt) ? partial[i] : 0;
    long long x = v;
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      long long y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) warp_tot[w] = x;
    __syncthreads();
    if (w == 0) {
      int nw = blockDim.x >> 5;
      long long t = (lane < nw) ? warp_tot[lane] : 0;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        long long y = __shfl_up_sync(0xffffffffu, t, o);
        if (lane >= o) t += y;
      }
      if (lane < nw) warp_tot[lane] = t;
    }
    __syncthreads();
    long long carry = carry_s;
    long long incl = x + (w > 0 ? warp_tot[w - 1] : 0);
    if (i < nt) partial[i] = carry + incl - v;
    __syncthreads();
    if (threadIdx.x == blockDim.x - 1) carry_s = carry + incl;
    __syncthreads();
  }
}

// in-tile inclusive scan of v[0..n) plus the tile's exclusive offset
__global__ void k_tile_scan(long long* __restrict__ v, long long n, const long long* __restrict__ partial) {
  __shared__ long long warp_tot[kScanThreads / 32];
  long long base = (long long)blockIdx.x * kScanTile + (long long)threadIdx.x * kPerThread;
  long long loc[kPerThread];
  long long s = 0;
#pragma unroll
  for (int q = 0; q < kPerThread; ++q) {
    long long i = base + q;
    s += (i < n) ? v[i] : 0;
    loc[q] = s;
  }
  int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  long long x = s;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    long long y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) warp_tot[w] = x;
  __syncthreads();
  if (w == 0) {
    long long t = (lane < kScanThreads / 32) ? warp_tot[lane] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      long long y = __shfl_up_sync(0xffffffffu, t, o);
      if (lane >= o) t += y;
    }
    if (lane < kScanThreads / 32) warp_tot[lane] = t;
  }
  __syncthreads();
  long long off = partial[blockIdx.x] + (x - s) + (w > 0 ? warp_tot[w - 1] : 0);
#pragma unroll
  for (int q = 0; q < kPerThread; ++q) {
    long long i = base + q;
    if (i < n) v[i] = off + loc[q];
  }
}

void launch_scan_rowptr(long long* row_ptr, long long n, long long* partial, cudaStream_t st) {
  cudaMemsetAsync(row_ptr, 0, sizeof(long long), st);
  if (n <= 0) return;
  long long nt = (n + kScanTile - 1) / kScanTile;
  k_tile_sums<<<(unsigned)nt, kScanThreads, 0, st>>>(row_ptr + 1, n, partial);
  k_scan_partials<<<1, 1024, 0, st>>>(partial, nt);
  k_tile_scan<<<(unsigned)nt, kScanThreads, 0, st>>>(row_ptr + 1, n, partial);
}

}  // namespace pct
