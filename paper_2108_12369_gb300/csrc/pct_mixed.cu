// pct_mixed.cu -- PCT_PREC_MIXED kernels.
//   count: FP64 path set-up once per proton (the definition), kept as row
//          records (FP64 for exact decisions, double-float for the set-up);
//          warp-cooperative set-up of every segment -> entries per row and
//          compact segment records.
//   fill:  warp-cooperative placement of every crossing from the segment
//          records -> col / val in path order, FP32 Kahan-compensated WEPL
//          per lane summed in double-float, noise factor.
//   batch: one persistent launch of either phase over many simulations.
//   projectors: matrix-free y = A x / g += A^T r with the per-lane walker.
#include <cstdint>

#include "pct_kernels.cuh"
#include "pct_coop.cuh"

namespace pct {


// this warp's part of the block's dynamic shared memory
template <class SM>
__device__ __forceinline__ SM& warp_smem() {
  extern __shared__ __align__(16) unsigned char coop_dyn[];
  return reinterpret_cast<SM*>(coop_dyn)[threadIdx.x >> 5];
}

// dynamic shared memory of a 128-thread count / fill block (rows of up to
// CAP segments)
template <int DIM, bool kFill, int CAP, bool LEAN = false>
constexpr size_t coop_bytes() {
  return kFill ? 4 * sizeof(FillSmem<DIM, CAP, LEAN>) : 4 * sizeof(CoopSmem<DIM, CAP>);
}

// the smaller layout: rows of up to kSegSmall segments on grids whose
// straight lines cross at most 1536 planes (rows then stay well below
// kRowCrossSmall crossings; longer ones take the walker all the same)
bool small_cap(int seg_stride, const GridDev& g) {
  const int planes = g.n[0] + g.n[1] + (g.dim == 3 ? g.n[2] : 0);
  return seg_stride <= kSegSmall && planes <= 1536;
}

// rows one block handles at most (the batch's work items take 64 - 256)
constexpr int kBlockRowsMax = 256;

// Path phase of one block of nr consecutive rows starting at row0 (128
// threads, thread t takes rows row0 + t, + 128, ...): the FP64 path of each
// row (the definition), kept with its double-float copy as row records.  The
// kernel is bound by the FP64 pipe; the rows' lead segments are set up by a
// kernel of their own (lead_block), whose FP32 work would otherwise raise
// this kernel's registers (126 -> 204) and halve its occupancy.  The
// arguments may live in parameter space (one launch per simulation) or in
// global memory (the batch kernel).
template <int DIM>
__device__ __forceinline__ void path_block(const SimDev& S, const MixArgs& M, const SimDev* Sg, const GridDF* gdg,
                                           long long n, long long row0, int nr = 128) {
  for (int t = threadIdx.x; t < nr; t += blockDim.x) {
  const long long i = row0 + t;
  if (i < n) {
    PathF64 p = path_setup<DIM>(S, i);
    M.r64[i] = p;  // exact decisions read the FP64 path back from here
    float fac = (S.md.noise == PCT_NOISE_GAUSS_REL) ? (float)(1.0 + S.md.noise_rel * p.z_noise) : 1.0f;
    RowDF r;
    make_rowdf<DIM>(p, S.R, fac, r);
    M.rdf[i] = r;
  }
  }
}

// The lead-in and lead-out segments (vertices 0 -> 1 and nv-2 -> nv-1) of
// rows [row0, row0 + nr) set up, thread per row, after the path phase (the
// count's table reads them).
template <int DIM>
__device__ __forceinline__ void lead_block(const SimDev& S, const MixArgs& M, const SimDev* Sg, const GridDF* gdg,
                                           long long n, long long row0, int nr) {
  for (int t = threadIdx.x; t < nr; t += blockDim.x) {
    const long long i = row0 + t;
    if (i >= n) break;
    const RowDF& r = M.rdf[i];
    SegP<DIM>* lead = lead_rec<DIM>(M, i);
    df Va[3], Vb[3];
    vertex_df<DIM>(r, M.tab, M.R, 0, Va);
    vertex_df<DIM>(r, M.tab, M.R, 1, Vb);
    lead[0] = seg_prepare<DIM>(S.ph.g, M.gd, Sg, gdg, Va, Vb, r.mag, ExactRef{Sg, M.r64 + i, 0});
    if (r.nv > 2) {
      vertex_df<DIM>(r, M.tab, M.R, r.nv - 2, Va);
      vertex_df<DIM>(r, M.tab, M.R, r.nv - 1, Vb);
      lead[1] = seg_prepare<DIM>(S.ph.g, M.gd, Sg, gdg, Va, Vb, r.mag, ExactRef{Sg, M.r64 + i, r.nv - 2});
    }
  }
}

// The block's 128 rows are handed out one at a time to whichever warp is
// free (rows differ in length; a static split leaves warps idle while the
// block's slowest warp finishes).  All 128 threads call; the counter starts
// at `first`, the rows the warps took before the call (one each).
__device__ __forceinline__ int next_row_of_block(int* take) {
  int k = 0;
  if ((threadIdx.x & 31) == 0) k = atomicAdd(take, 1);
  return __shfl_sync(0xffffffffu, k, 0);
}

// Count phase of a block of nr rows: each warp counts one row at a time.
template <int DIM, int CAP>
__device__ __forceinline__ void rows_block(const SimDev& S, const MixArgs& M, const SimDev* Sg, const GridDF* gdg,
                                           long long n, long long row0, long long* __restrict__ counts,
                                           int nr = 128) {
  CoopSmem<DIM, CAP>& sm = warp_smem<CoopSmem<DIM, CAP>>();
  __shared__ int take, n_walk;
  __shared__ unsigned char walk[kBlockRowsMax];  // rows the cooperative count declined
  if (threadIdx.x == 0) {
    take = 4;
    n_walk = 0;
  }
  __syncthreads();
  for (int k = threadIdx.x >> 5; k < nr && row0 + k < n; k = next_row_of_block(&take))
    if (!coop_count_row<DIM>(S, M, Sg, gdg, row0 + k, sm, counts) && (threadIdx.x & 31) == 0)
      walk[atomicAdd(&n_walk, 1)] = (unsigned char)k;
  // the declined rows after all others: the walker's out-of-line call stays
  // out of the cooperative loop (a call there makes the register allocator
  // keep the loop's state in local memory)
  __syncthreads();
  for (int q = threadIdx.x >> 5; q < n_walk; q += 4) count_row_walk<DIM>(Sg, M, row0 + walk[q], counts);
}

// count blocks resident per SM (64 -> 56 registers a thread: 3D head count
// -3 %, NEO-2 -3 % against 8 blocks)
constexpr int kCountBlocksPerSm = 9;

// The count of one simulation runs as three kernels: the FP64 path set-up
// (lane per row), the lead segments' set-up (lane per row) and the
// warp-cooperative count (warp per row), so that each kernel's code stays
// small enough for the instruction caches and the FP64 kernel keeps its
// occupancy.
template <int DIM>
__global__ void __launch_bounds__(128) k_path_mixed(SimDev S, MixArgs M, const SimDev* Sg, const GridDF* gdg,
                                                    long long n) {
  path_block<DIM>(S, M, Sg, gdg, n, (long long)blockIdx.x * blockDim.x);
}

template <int DIM>
__global__ void __launch_bounds__(128) k_lead_mixed(SimDev S, MixArgs M, const SimDev* Sg, const GridDF* gdg,
                                                    long long n) {
  lead_block<DIM>(S, M, Sg, gdg, n, (long long)blockIdx.x * blockDim.x, blockDim.x);
}

template <int DIM, int CAP>
__global__ void __launch_bounds__(128, kCountBlocksPerSm) k_count_mixed(SimDev S, MixArgs M, const SimDev* Sg, const GridDF* gdg,
                                                     long long n, long long* __restrict__ counts) {
  rows_block<DIM, CAP>(S, M, Sg, gdg, n, (long long)blockIdx.x * blockDim.x, counts);
}

// One block of nr consecutive rows starting at row0 (fill phase): each
// warp writes one row at a time; pf = 1 prefetches the next row's segment
// records into L2 while a row is written.
template <int DIM, int CAP, bool LEAN>
__device__ __forceinline__ void fill_block(const SimDev& S, const MixArgs& M, const SimDev* Sg, const GridDF* gdg,
                                           long long n, long long row0, const long long* __restrict__ row_ptr,
                                           const float* __restrict__ x, int* __restrict__ col,
                                           float* __restrict__ val, float* __restrict__ b, int nr = 128,
                                           int pf = 1) {
  FillSmem<DIM, CAP, LEAN>& sm = warp_smem<FillSmem<DIM, CAP, LEAN>>();
  const int lane = threadIdx.x & 31;
  const int lines = (M.seg_stride * (int)sizeof(SegG<DIM>) + 127) / 128;
  __shared__ int take, n_walk;
  __shared__ unsigned char walk[kBlockRowsMax];  // rows the cooperative fill declined
  if (threadIdx.x == 0) {
    take = 4;
    n_walk = 0;
  }
  __syncthreads();
  int k = threadIdx.x >> 5;
  while (k < nr && row0 + k < n) {
    const long long row = row0 + k;
    const int kn = next_row_of_block(&take);
    // the next row's segment records into L2 while this row is written
    if (!LEAN && pf && kn < nr && row0 + kn < n) {
      const long long rn = row0 + kn;
      const char* nx = (const char*)((const SegG<DIM>*)M.segg + rn * (long long)M.seg_stride);
      if (lane < lines) asm volatile("prefetch.global.L2 [%0];" ::"l"(nx + 128 * lane));
      if (lane == 31) asm volatile("prefetch.global.L2 [%0];" ::"l"(M.rdf + rn));
    }
    if (!coop_fill_row<DIM>(S, M, Sg, gdg, row, sm, row_ptr, x, col, val, b) && lane == 0)
      walk[atomicAdd(&n_walk, 1)] = (unsigned char)k;
    k = kn;
  }
  // the declined rows after all others (their out-of-line walker call stays
  // out of the cooperative loop)
  __syncthreads();
  for (int q = threadIdx.x >> 5; q < n_walk; q += 4) fill_row_walk<DIM>(Sg, M, row0 + walk[q], row_ptr, x, col, val, b);
}

// 3D rows are shorter (fewer crossings per segment): more resident blocks
// pay off there (3D head fill: 8 blocks per SM -5 % against 7, 9 blocks a
// further -1 %, 10 blocks +22 %), 7 in 2D (NEO-2 fill +2 % at 8, no change
// at 9).  The lean form's larger shared layout holds it to 8.
template <int DIM, bool LEAN = false>
constexpr int fill_blocks_per_sm() {
  return DIM == 3 ? (LEAN ? 8 : 9) : 7;
}

template <int DIM, int CAP, bool LEAN>
__global__ void __launch_bounds__(128, fill_blocks_per_sm<DIM, LEAN>()) k_fill_mixed(SimDev S, MixArgs M, const SimDev* Sg, const GridDF* gdg,
                                                    long long n, const long long* __restrict__ row_ptr,
                                                    const float* __restrict__ x, int* __restrict__ col,
                                                    float* __restrict__ val, float* __restrict__ b) {
  fill_block<DIM, CAP, LEAN>(S, M, Sg, gdg, n, (long long)blockIdx.x * blockDim.x, row_ptr, x, col, val, b);
}

// rows [row_begin, n) only (a kernel of its own, so that the whole fill
// keeps its first row at compile-time zero)
template <int DIM, int CAP, bool LEAN>
__global__ void __launch_bounds__(128, fill_blocks_per_sm<DIM, LEAN>()) k_fill_mixed_range(SimDev S, MixArgs M, const SimDev* Sg,
                                                          const GridDF* gdg, long long n,
                                                          const long long* __restrict__ row_ptr,
                                                          const float* __restrict__ x, int* __restrict__ col,
                                                          float* __restrict__ val, float* __restrict__ b,
                                                          long long row_begin) {
  fill_block<DIM, CAP, LEAN>(S, M, Sg, gdg, n, row_begin + (long long)blockIdx.x * blockDim.x, row_ptr, x, col, val, b);
}

// ---------------------------------------------------------------------------
// Batch: one persistent launch over the work items (instance, block of 128
// rows) of many heterogeneous simulations.  A block takes the next item from
// a device counter; items are independent, so nothing ever waits.
// ---------------------------------------------------------------------------
__device__ __forceinline__ int batch_find(const BatchInst* __restrict__ B, int n_inst, int phase, long long item) {
  int lo = 0, hi = n_inst - 1;  // last instance whose first item is <= item
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (B[mid].item0[phase] <= item)
      lo = mid;
    else
      hi = mid - 1;
  }
  return lo;
}

// phases: 0 path set-up, 1 count, 2 fill (the launch bounds follow the
// per-simulation kernels of each phase)
template <int kPhase, int DIM, int CAP, bool LEAN>
__global__ void __launch_bounds__(128, kPhase == 0 ? 1 : (kPhase == 1 ? kCountBlocksPerSm : fill_blocks_per_sm<DIM, LEAN>()))
    k_batch(const BatchInst* __restrict__ B, int n_inst, long long first, long long last,
            unsigned long long* next, int nr, int pf) {
  __shared__ long long item_s;
  for (;;) {
    __syncthreads();
    if (threadIdx.x == 0) item_s = first + (long long)atomicAdd(next, 1ULL);
    __syncthreads();
    const long long item = item_s;
    if (item >= last) return;
    const BatchInst& I = B[batch_find(B, n_inst, kPhase, item)];
    const long long row0 = (item - I.item0[kPhase]) * nr;
    if constexpr (kPhase == 2)
      fill_block<DIM, CAP, LEAN>(I.S, I.M, &I.S, &I.M.gd, I.n, row0, I.row_ptr, I.x, I.col, I.val, I.b, nr, pf);
    else if constexpr (kPhase == 1)
      rows_block<DIM, CAP>(I.S, I.M, &I.S, &I.M.gd, I.n, row0, I.row_ptr_w + 1, nr);
    else {
      path_block<DIM>(I.S, I.M, &I.S, &I.M.gd, I.n, row0, nr);
      lead_block<DIM>(I.S, I.M, &I.S, &I.M.gd, I.n, row0, nr);  // (each thread reads its own rows' records)
    }
  }
}

// opt in to more than 48 KB of dynamic shared memory where a kernel needs it
template <class Kern>
static void smem_attr(Kern k, size_t bytes) {
  if (bytes > 48 * 1024) cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

template <int kPhase, int DIM, int CAP, bool LEAN>
static size_t batch_smem() {
  return kPhase == 0 ? 0 : coop_bytes<DIM, kPhase == 2, CAP, LEAN>();
}

template <int kPhase, int DIM, int CAP, bool LEAN = false>
static int blocks_per_sm() {
  int nb = 0;
  smem_attr(k_batch<kPhase, DIM, CAP, LEAN>, batch_smem<kPhase, DIM, CAP, LEAN>());
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_batch<kPhase, DIM, CAP, LEAN>, 128,
                                                batch_smem<kPhase, DIM, CAP, LEAN>());
  return nb > 0 ? nb : 1;
}

// (the path phase has no shared memory: one capacity serves every batch)
// (the path phase has no shared memory: one capacity serves every batch;
// the count phase reads the lean flag from each instance's arguments)
int batch_blocks_per_sm(int phase, int dim, bool small, bool lean) {
  if (phase == 0) return dim == 2 ? blocks_per_sm<0, 2, kSegMax>() : blocks_per_sm<0, 3, kSegMax>();
  if (phase == 1) {
    if (small) return dim == 2 ? blocks_per_sm<1, 2, kSegSmall>() : blocks_per_sm<1, 3, kSegSmall>();
    return dim == 2 ? blocks_per_sm<1, 2, kSegMax>() : blocks_per_sm<1, 3, kSegMax>();
  }
  if (lean) {
    if (small) return dim == 2 ? blocks_per_sm<2, 2, kSegSmall, true>() : blocks_per_sm<2, 3, kSegSmall, true>();
    return dim == 2 ? blocks_per_sm<2, 2, kSegMax, true>() : blocks_per_sm<2, 3, kSegMax, true>();
  }
  if (small) return dim == 2 ? blocks_per_sm<2, 2, kSegSmall>() : blocks_per_sm<2, 3, kSegSmall>();
  return dim == 2 ? blocks_per_sm<2, 2, kSegMax>() : blocks_per_sm<2, 3, kSegMax>();
}

template <int kPhase, int DIM, int CAP, bool LEAN>
static void launch_phase(const BatchInst* B, int n_inst, long long first, long long last, unsigned long long* next,
                         int grid, int nr, int pf, cudaStream_t st) {
  smem_attr(k_batch<kPhase, DIM, CAP, LEAN>, batch_smem<kPhase, DIM, CAP, LEAN>());
  k_batch<kPhase, DIM, CAP, LEAN><<<grid, 128, batch_smem<kPhase, DIM, CAP, LEAN>(), st>>>(B, n_inst, first, last,
                                                                                          next, nr, pf);
}

template <int kPhase, int DIM>
static void launch_phase_cap(bool small, bool lean, const BatchInst* B, int n_inst, long long first, long long last,
                             unsigned long long* next, int grid, int nr, int pf, cudaStream_t st) {
  if (kPhase == 2 && lean) {
    if (small)
      launch_phase<kPhase, DIM, kSegSmall, true>(B, n_inst, first, last, next, grid, nr, pf, st);
    else
      launch_phase<kPhase, DIM, kSegMax, true>(B, n_inst, first, last, next, grid, nr, pf, st);
  } else if (kPhase == 0 || !small) {
    launch_phase<kPhase, DIM, kSegMax, false>(B, n_inst, first, last, next, grid, nr, pf, st);
  } else {
    launch_phase<kPhase, DIM, kSegSmall, false>(B, n_inst, first, last, next, grid, nr, pf, st);
  }
}

void launch_batch(int phase, int dim, bool small, bool lean, const BatchInst* B, int n_inst, long long first,
                  long long last, unsigned long long* next, int grid, int nr, int pf, cudaStream_t st) {
  cudaMemsetAsync(next, 0, sizeof(unsigned long long), st);
  if (last <= first || n_inst <= 0) return;
  nr = nr < 32 ? 32 : (nr > kBlockRowsMax ? kBlockRowsMax : nr);
  if (phase == 0 && dim == 2) launch_phase_cap<0, 2>(small, lean, B, n_inst, first, last, next, grid, nr, pf, st);
  if (phase == 0 && dim == 3) launch_phase_cap<0, 3>(small, lean, B, n_inst, first, last, next, grid, nr, pf, st);
  if (phase == 1 && dim == 2) launch_phase_cap<1, 2>(small, lean, B, n_inst, first, last, next, grid, nr, pf, st);
  if (phase == 1 && dim == 3) launch_phase_cap<1, 3>(small, lean, B, n_inst, first, last, next, grid, nr, pf, st);
  if (phase == 2 && dim == 2) launch_phase_cap<2, 2>(small, lean, B, n_inst, first, last, next, grid, nr, pf, st);
  if (phase == 2 && dim == 3) launch_phase_cap<2, 3>(small, lean, B, n_inst, first, last, next, grid, nr, pf, st);
}

// ---------------------------------------------------------------------------
// Matrix-free projectors (rows recomputed, nothing stored): y_i = <a_i, x>
// or g += a_i r_i, for rows [row_base, row_base + n).  Same paths, same
// decisions and the same FP32 lengths as the fill.
// ---------------------------------------------------------------------------
struct DotSinkM {
  const float* x;
  float sum, comp;
  float xpend;
  __device__ void pend(int c) { xpend = __ldg(x + c); }
  __device__ void put(int, float len) {
    float y = len * xpend - comp;
    float t = sum + y;
    comp = (t - sum) - y;
    sum = t;
  }
};

// The reduction is issued as a plain `red` with no memory clobber: nothing
// in the kernel reads g, and the compiler may then keep the row's records
// (read from global memory) in registers across it instead of re-reading
// them after every entry.
struct ScatterSinkM {
  float* g;
  float r;
  __device__ void put(int c, float len) {
    asm volatile("red.global.add.f32 [%0], %1;" ::"l"(g + c), "f"(len * r));
  }
  __device__ void pend(int) {}
};

template <int DIM, bool kAdjoint>
__device__ __forceinline__ void proj_block(const SimDev& S, const MixArgs& M, const SimDev* Sg, const GridDF* gdg,
                                           long long n, long long row0, long long row_base,
                                           const float* __restrict__ in, float* __restrict__ out) {
  long long i = row0 + threadIdx.x;
  int key = -1;
  if (i < n && (!kAdjoint || in[i] != 0.0f)) {
    PathF64 p = path_setup<DIM>(S, row_base + i);
    M.r64[i] = p;
    RowDF r;
    make_rowdf<DIM>(p, S.R, 1.0f, r);
    M.rdf[i] = r;
    key = nv_key(p.nv);
  } else if (i < n && !kAdjoint) {
    key = -1;
  }
  __threadfence_block();
  long long row = regroup_rows(i, key);
  const bool live = row >= 0;
  if constexpr (kAdjoint) {
    ScatterSinkM sk{out, live ? in[row] : 0.f};
    walk_row_df<DIM, true>(S, M, Sg, gdg, M.rdf[live ? row : 0], M.r64 + (live ? row : 0), live, sk);
  } else {
    DotSinkM sk{in, 0.f, 0.f, 0.f};
    walk_row_df<DIM, true>(S, M, Sg, gdg, M.rdf[live ? row : 0], M.r64 + (live ? row : 0), live, sk);
    if (live) out[row] = sk.sum;
  }
}

template <int DIM, bool kAdjoint>
__global__ void __launch_bounds__(128) k_proj_mixed(SimDev S, MixArgs M, const SimDev* Sg, const GridDF* gdg,
                                                    long long n, long long row_base, const float* __restrict__ in,
                                                    float* __restrict__ out) {
  proj_block<DIM, kAdjoint>(S, M, Sg, gdg, n, (long long)blockIdx.x * blockDim.x, row_base, in, out);
}

static df split_host(double v) {
  float hi = (float)v;
  return df{hi, (float)(v - (double)hi)};
}

MixArgs mix_args(const SimDev& S, long long n, const void* tab, void* rec, bool lean) {
  MixArgs M;
  for (int a = 0; a < 3; ++a) {
    M.gd.o[a] = split_host(S.ph.g.o[a]);
    M.gd.h[a] = split_host(S.ph.g.h[a]);
    M.gd.of[a] = (float)S.ph.g.o[a];
    M.gd.rh[a] = (float)(1.0 / S.ph.g.h[a]);
  }
  M.R = split_host(S.R);
  M.tab = (const BasisDF*)tab;
  size_t rows = (size_t)(n > 0 ? n : 1);
  const size_t o64 = (rows * sizeof(RowDF) + 255) & ~(size_t)255;
  const size_t olead = o64 + ((rows * sizeof(PathF64) + 255) & ~(size_t)255);
  const size_t osegg = olead + ((2 * rows * sizeof(SegP<3>) + 255) & ~(size_t)255);
  M.rdf = (RowDF*)rec;
  M.r64 = (PathF64*)((char*)rec + o64);
  M.lead = (char*)rec + olead;
  M.segg = lean ? nullptr : (char*)rec + osegg;
  M.rflag = lean ? (unsigned char*)rec + osegg : nullptr;  // (the segment records' place)
  M.seg_stride = seg_stride_of(S.md.model, S.md.K);
  return M;
}

void fill_basis_df(const double* s, const double* h10, const double* h11, int n, void* host_out) {
  BasisDF* t = (BasisDF*)host_out;
  for (int j = 0; j < n; ++j) {
    t[j].s = split_host(s[j]);
    t[j].h10 = split_host(h10[j]);
    t[j].h11 = split_host(h11[j]);
    t[j].pad = df{0.f, 0.f};
  }
}

size_t basis_df_bytes(int n) { return sizeof(BasisDF) * (size_t)n; }

size_t mixed_args_bytes() { return ((sizeof(SimDev) + 255) & ~(size_t)255) + sizeof(GridDF); }

// the kernel arguments, also copied to global memory for the out-of-line
// exact comparisons (the copies are staged before cudaMemcpyAsync returns)
static void args_at(void* args, const SimDev** Sg, const GridDF** gdg) {
  char* base = (char*)args;
  *Sg = (const SimDev*)base;
  *gdg = (const GridDF*)(base + ((sizeof(SimDev) + 255) & ~(size_t)255));
}

static bool upload_args(const SimDev& S, const MixArgs& M, void* args, cudaStream_t st, const SimDev** Sg,
                        const GridDF** gdg) {
  char* base = (char*)args;
  size_t off = (sizeof(SimDev) + 255) & ~(size_t)255;
  args_at(args, Sg, gdg);
  return cudaMemcpyAsync(base, &S, sizeof(SimDev), cudaMemcpyHostToDevice, st) == cudaSuccess &&
         cudaMemcpyAsync(base + off, &M.gd, sizeof(GridDF), cudaMemcpyHostToDevice, st) == cudaSuccess;
}

// the count / fill kernels for rows of up to kSegSmall (small) or kSegMax segments
template <int DIM>
static void launch_count_cap(bool small, unsigned blocks, const SimDev& S, const MixArgs& M, const SimDev* Sg,
                             const GridDF* gdg, long long n, long long* counts, cudaStream_t st) {
  if (small) {
    smem_attr(k_count_mixed<DIM, kSegSmall>, coop_bytes<DIM, false, kSegSmall>());
    k_count_mixed<DIM, kSegSmall><<<blocks, 128, coop_bytes<DIM, false, kSegSmall>(), st>>>(S, M, Sg, gdg, n, counts);
  } else {
    smem_attr(k_count_mixed<DIM, kSegMax>, coop_bytes<DIM, false, kSegMax>());
    k_count_mixed<DIM, kSegMax><<<blocks, 128, coop_bytes<DIM, false, kSegMax>(), st>>>(S, M, Sg, gdg, n, counts);
  }
}

template <int DIM, int CAP, bool LEAN>
static void launch_fill_lean(bool whole, unsigned blocks, const SimDev& S, const MixArgs& M, const SimDev* Sg,
                             const GridDF* gdg, long long n, long long row_end, long long row_begin,
                             const long long* row_ptr, const float* x, int* col, float* val, float* b,
                             cudaStream_t st) {
  const size_t sm = coop_bytes<DIM, true, CAP, LEAN>();
  if (whole) {
    smem_attr(k_fill_mixed<DIM, CAP, LEAN>, sm);
    k_fill_mixed<DIM, CAP, LEAN><<<blocks, 128, sm, st>>>(S, M, Sg, gdg, n, row_ptr, x, col, val, b);
  } else {
    smem_attr(k_fill_mixed_range<DIM, CAP, LEAN>, sm);
    k_fill_mixed_range<DIM, CAP, LEAN><<<blocks, 128, sm, st>>>(S, M, Sg, gdg, row_end, row_ptr, x, col, val, b,
                                                                 row_begin);
  }
}

template <int DIM, int CAP>
static void launch_fill_cap(bool whole, unsigned blocks, const SimDev& S, const MixArgs& M, const SimDev* Sg,
                            const GridDF* gdg, long long n, long long row_end, long long row_begin,
                            const long long* row_ptr, const float* x, int* col, float* val, float* b,
                            cudaStream_t st) {
  if (M.rflag)
    launch_fill_lean<DIM, CAP, true>(whole, blocks, S, M, Sg, gdg, n, row_end, row_begin, row_ptr, x, col, val, b,
                                     st);
  else
    launch_fill_lean<DIM, CAP, false>(whole, blocks, S, M, Sg, gdg, n, row_end, row_begin, row_ptr, x, col, val, b,
                                      st);
}

void launch_count_mixed(const SimDev& S, const void* tab, long long n, void* rec, long long* counts, void* args,
                        cudaStream_t st, bool lean) {
  if (n <= 0) return;
  MixArgs M = mix_args(S, n, tab, rec, lean);
  const SimDev* Sg;
  const GridDF* gdg;
  if (!upload_args(S, M, args, st, &Sg, &gdg)) return;
  int threads = 128;
  unsigned blocks = (unsigned)((n + threads - 1) / threads);
  const bool small = small_cap(M.seg_stride, S.ph.g);
  if (S.ph.g.dim == 2) {
    k_path_mixed<2><<<blocks, threads, 0, st>>>(S, M, Sg, gdg, n);
    k_lead_mixed<2><<<blocks, threads, 0, st>>>(S, M, Sg, gdg, n);
    launch_count_cap<2>(small, blocks, S, M, Sg, gdg, n, counts, st);
  } else {
    k_path_mixed<3><<<blocks, threads, 0, st>>>(S, M, Sg, gdg, n);
    k_lead_mixed<3><<<blocks, threads, 0, st>>>(S, M, Sg, gdg, n);
    launch_count_cap<3>(small, blocks, S, M, Sg, gdg, n, counts, st);
  }
}

void launch_fill_mixed(const SimDev& S, const void* tab, long long n, const void* rec, const long long* row_ptr,
                       const float* x, int* col, float* val, float* b, void* args, cudaStream_t st,
                       long long row_begin, long long row_end, long long nz0, bool upload, bool lean) {
  if (row_end < 0) row_end = n;
  if (n <= 0 || row_end <= row_begin) return;
  MixArgs M = mix_args(S, n, tab, (void*)rec, lean);
  const SimDev* Sg;
  const GridDF* gdg;
  if (upload) {
    if (!upload_args(S, M, args, st, &Sg, &gdg)) return;
  } else {
    args_at(args, &Sg, &gdg);
  }
  int threads = 128;
  unsigned blocks = (unsigned)((row_end - row_begin + threads - 1) / threads);
  const bool whole = row_begin == 0 && row_end == n && nz0 == 0;
  // a block of rows into staging buffers: the kernels address col / val by
  // CSR position and b by row, so the bases move back by the block's first
  // position / row (address arithmetic on the host; every address the
  // kernels form lies inside the staging buffers)
  col = (int*)((uintptr_t)col - sizeof(int) * (uintptr_t)nz0);
  val = (float*)((uintptr_t)val - sizeof(float) * (uintptr_t)nz0);
  b = (float*)((uintptr_t)b - sizeof(float) * (uintptr_t)row_begin);
  const bool small = small_cap(M.seg_stride, S.ph.g);
  if (S.ph.g.dim == 2) {
    if (small)
      launch_fill_cap<2, kSegSmall>(whole, blocks, S, M, Sg, gdg, n, row_end, row_begin, row_ptr, x, col, val, b, st);
    else
      launch_fill_cap<2, kSegMax>(whole, blocks, S, M, Sg, gdg, n, row_end, row_begin, row_ptr, x, col, val, b, st);
  } else {
    if (small)
      launch_fill_cap<3, kSegSmall>(whole, blocks, S, M, Sg, gdg, n, row_end, row_begin, row_ptr, x, col, val, b, st);
    else
      launch_fill_cap<3, kSegMax>(whole, blocks, S, M, Sg, gdg, n, row_end, row_begin, row_ptr, x, col, val, b, st);
  }
}

void launch_proj_mixed(bool adjoint, const SimDev& S, const void* tab, long long row_base, long long n, void* rec,
                       const float* in, float* out, void* args, cudaStream_t st, bool lean) {
  if (n <= 0) return;
  MixArgs M = mix_args(S, n, tab, rec, lean);
  const SimDev* Sg;
  const GridDF* gdg;
  if (!upload_args(S, M, args, st, &Sg, &gdg)) return;
  int threads = 128;
  unsigned blocks = (unsigned)((n + threads - 1) / threads);
  if (S.ph.g.dim == 2) {
    if (adjoint)
      k_proj_mixed<2, true><<<blocks, threads, 0, st>>>(S, M, Sg, gdg, n, row_base, in, out);
    else
      k_proj_mixed<2, false><<<blocks, threads, 0, st>>>(S, M, Sg, gdg, n, row_base, in, out);
  } else {
    if (adjoint)
      k_proj_mixed<3, true><<<blocks, threads, 0, st>>>(S, M, Sg, gdg, n, row_base, in, out);
    else
      k_proj_mixed<3, false><<<blocks, threads, 0, st>>>(S, M, Sg, gdg, n, row_base, in, out);
  }
}

int seg_stride_of(int model, int K) {
  const int nseg = model == PCT_PATH_SPLINE ? K + 2 : (model == PCT_PATH_STRAIGHT_MCS ? 3 : 1);
  return nseg < 1 ? 1 : (nseg > kSegMax ? kSegMax : nseg);
}

size_t mixed_record_size(long long rows, int dim, int model, int K, bool lean) {
  size_t r = (size_t)(rows > 0 ? rows : 1);
  const size_t seg = dim == 3 ? sizeof(SegG<3>) : sizeof(SegG<2>);
  // lean form: one flag byte per row in place of the segment records
  const size_t last = lean ? r : r * (size_t)seg_stride_of(model, K) * seg;
  return ((r * sizeof(RowDF) + 255) & ~(size_t)255) + ((r * sizeof(PathF64) + 255) & ~(size_t)255) +
         ((2 * r * sizeof(SegP<3>) + 255) & ~(size_t)255) + last + 256;
}

}  // namespace pct
