// pct_mixed.cu -- PCT_PREC_MIXED kernels.
//   count: FP64 path set-up once per proton (the definition), kept as two row
//          records (FP64 for exact decisions, double-float for the walk);
//          double-float certified traversal -> entries per row.
//   fill:  double-float traversal from the record -> col / val in path order,
//          FP32 Kahan-compensated WEPL, noise factor.
#include "pct_kernels.cuh"
#include "pct_mixed.cuh"

namespace pct {


// feeds FP64-walked entries into the FP32 row merge
template <class M>
struct MergeToF32 {
  M* mg;
  template <class Sink>
  __device__ void emit(int col, double len, Sink& sink) {
    mg->emit(col, (float)len, sink);
  }
};

// Finished entries of a row.  The count kernel only counts them.  The fill
// kernel stages them per lane in shared memory ([k][33] layout: lanes write
// and read conflict-free) and the warp writes each lane's run with
// coalesced stores; segments walked in FP64 write straight to global.
struct CountSinkM {
  static constexpr bool kStaged = false;
  long long n;
  template <class L>
  __device__ void put(int, L) {
    ++n;
  }
  __device__ void pend(int) {}
};

constexpr int kChunk = 32;     // walk steps between two flushes
constexpr int kRingPitch = 33;

struct FillSinkR {
  static constexpr bool kStaged = true;
  int* colb;        // this warp's staging, [kChunk][kRingPitch]
  float* valb;
  int n, lane;      // staged entries of this lane
  int* col;
  float* val;
  long long pos;    // next global position of this lane's row
  bool direct;
  const float* x;
  float xpend;      // x_true of the pending voxel, loaded a step ahead
  float sum, comp;  // Kahan-compensated WEPL
  bool constant;
  float hconst;
  __device__ void pend(int c) { xpend = __ldg(x + c); }
  __device__ void put(int c, float len) {
    const float v = constant ? hconst : len;
    if (direct) {
      col[pos] = c;
      val[pos] = v;
      ++pos;
    } else {
      colb[n * kRingPitch + lane] = c;
      valb[n * kRingPitch + lane] = v;
      ++n;
    }
    float y = len * xpend - comp;
    float t = sum + y;
    comp = (t - sum) - y;
    sum = t;
  }
  // warp-cooperative: every lane's staged run goes to its row
  __device__ void flush() {
    unsigned todo = __ballot_sync(0xffffffffu, n > 0);
    while (todo) {
      const int L = __ffs(todo) - 1;
      todo &= todo - 1;
      const int nL = __shfl_sync(0xffffffffu, n, L);
      const long long pL = __shfl_sync(0xffffffffu, pos, L);
      if (lane < nL) {
        col[pL + lane] = colb[lane * kRingPitch + L];
        val[pL + lane] = valb[lane * kRingPitch + L];
      }
    }
    pos += n;
    n = 0;
    __syncwarp();
  }
};

// all segments of one row.  The segment loop runs to the warp's largest
// vertex count so that the lanes set up segment q together; walks advance
// in chunks of kChunk entries, after which the fill kernel flushes.
template <int DIM, bool kLengths, class Sink>
__device__ __forceinline__ void walk_row_df(const SimDev& S, const MixArgs& M, const SimDev* Sg, const GridDF* gdg,
                                            const RowDF& r, const PathF64* p64, bool live_row, Sink& sink) {
  // r refers to the row record in global memory: its fields are re-read per
  // segment (L1 hits) instead of occupying ~40 registers for the whole row
  const GridDev& g = S.ph.g;
  const float mag = live_row ? r.mag : 0.f;
  RowMerge<float> mg;
  mg.init();
  MergeToF32<RowMerge<float>> m64{&mg};
  const int nv = live_row ? r.nv : 0;
  const int nv_max = __reduce_max_sync(0xffffffffu, nv);
  df Va[3], Vb[3];
  if (nv > 0) vertex_df<DIM>(r, M.tab, M.R, 0, Va);
  for (int q = 0; q + 1 < nv_max; ++q) {
    const bool act = q + 1 < nv;
    int res = 0;
    SegDF sg;
    Walk32 w;
    ExactRef ends{Sg, p64, q};
    if (act) {
      vertex_df<DIM>(r, M.tab, M.R, q + 1, Vb);
      mg.seg_begin();
      res = 1;
      if (!seg_setup_fast<DIM>(g, M.gd, Va, Vb, mag, sg, w)) {
        res = seg_setup_df<DIM>(g, M.gd, Va, Vb, mag, sg, ends);
        if (res == 1) walk_from_df<DIM>(sg, w);
      }
    }
    // segments whose direction cannot be certified are walked in FP64
    const bool f64seg = act && res == 2;
    if (__any_sync(0xffffffffu, f64seg)) {
      if constexpr (Sink::kStaged) sink.flush();
      if (f64seg) {
        if constexpr (Sink::kStaged) sink.direct = true;
        double P[3], Q[3];
        path_vertex(*Sg, *p64, q, P);
        path_vertex(*Sg, *p64, q + 1, Q);
        SegF64 s64;
        if (seg_setup_f64(g, P, Q, s64)) seg_walk_f64(g, s64, m64, sink);
        if constexpr (Sink::kStaged) sink.direct = false;
      }
    }
    const bool walking = act && res == 1;
    Lean<DIM> L;
    const float seglen = sg.L;
    if (walking) lean_begin<DIM>(g, sg, w, q, L);
    if constexpr (kLengths) {
      while (__any_sync(0xffffffffu, walking && !L.done)) {
#pragma unroll 1
        for (int c = 0; c < kChunk; ++c) {
          if (walking && !L.done) {
            const int vc = L.col;
            const float l = lean_step<DIM>(L, r, M.tab, M.R, M.gd, g, mag, ends);
            mg.emit(vc, l * seglen, sink);
          }
        }
        if constexpr (Sink::kStaged) sink.flush();
      }
    } else {
      if (walking) {
        while (!L.done) {
          const int vc = L.col;
          lean_step<DIM>(L, r, M.tab, M.R, M.gd, g, mag, ends);
          mg.emit(vc, 0.f, sink);
        }
      }
    }
    if (act) {
      mg.seg_end();
#pragma unroll
      for (int a = 0; a < DIM; ++a) Va[a] = Vb[a];
    }
  }
  if (nv > 0) mg.finish(sink);
  if constexpr (Sink::kStaged) sink.flush();
}

// Rows of one block are regrouped by vertex count (path kind) so that each
// warp walks rows with the same number of segments.  Returns the row this
// thread processes (or -1).  key: 0, 1, 2 for 2, 4, more vertices.
__device__ __forceinline__ long long regroup_rows(long long row, int key) {
  __shared__ int cnt[3];
  __shared__ int perm[128];
  if (threadIdx.x < 3) cnt[threadIdx.x] = 0;
  __syncthreads();
  int slot = -1;
  if (key >= 0) slot = atomicAdd(&cnt[key], 1);
  __syncthreads();
  if (key >= 0) {
    int base = (key > 0 ? cnt[0] : 0) + (key > 1 ? cnt[1] : 0);
    perm[base + slot] = threadIdx.x;
  }
  int total = cnt[0] + cnt[1] + cnt[2];
  __syncthreads();
  long long block0 = row - threadIdx.x;
  return (threadIdx.x < total) ? block0 + perm[threadIdx.x] : -1;
}

__device__ __forceinline__ int nv_key(int nv) { return nv <= 2 ? 0 : (nv <= 4 ? 1 : 2); }

// One block of 128 consecutive rows starting at row0 (count phase).  The
// arguments may live in parameter space (one launch per simulation) or in
// global memory (the batch kernel).
template <int DIM>
__device__ __forceinline__ void count_block(const SimDev& S, const MixArgs& M, const SimDev* Sg, const GridDF* gdg,
                                            long long n, long long row0, long long* __restrict__ counts) {
  long long i = row0 + threadIdx.x;
  int key = -1;
  if (i < n) {
    PathF64 p = path_setup(S, i);
    M.r64[i] = p;  // exact decisions read the FP64 path back from here
    float fac = (S.md.noise == PCT_NOISE_GAUSS_REL) ? (float)(1.0 + S.md.noise_rel * p.z_noise) : 1.0f;
    RowDF r;
    make_rowdf<DIM>(p, S.R, fac, r);
    M.rdf[i] = r;
    key = nv_key(p.nv);
  }
  __threadfence_block();
  long long row = regroup_rows(i, key);
  const bool live = row >= 0;
  CountSinkM cs{0};
  walk_row_df<DIM, false>(S, M, Sg, gdg, M.rdf[live ? row : 0], M.r64 + (live ? row : 0), live, cs);
  if (live) counts[row] = cs.n;
}

template <int DIM>
__global__ void __launch_bounds__(128) k_count_mixed(SimDev S, MixArgs M, const SimDev* Sg, const GridDF* gdg,
                                                     long long n, long long* __restrict__ counts) {
  count_block<DIM>(S, M, Sg, gdg, n, (long long)blockIdx.x * blockDim.x, counts);
}

// One block of 128 consecutive rows starting at row0 (fill phase).
template <int DIM>
__device__ __forceinline__ void fill_block(const SimDev& S, const MixArgs& M, const SimDev* Sg, const GridDF* gdg,
                                           long long n, long long row0, const long long* __restrict__ row_ptr,
                                           const float* __restrict__ x, int* __restrict__ col,
                                           float* __restrict__ val, float* __restrict__ b) {
  long long i = row0 + threadIdx.x;
  int key = (i < n) ? nv_key(M.rdf[i].nv) : -1;
  long long row = regroup_rows(i, key);
  const bool live = row >= 0;
  const RowDF& r = M.rdf[live ? row : 0];
  __shared__ int colb[4][kChunk * kRingPitch];
  __shared__ float valb[4][kChunk * kRingPitch];
  const int wid = threadIdx.x >> 5;
  FillSinkR fs;
  fs.colb = colb[wid];
  fs.valb = valb[wid];
  fs.n = 0;
  fs.lane = threadIdx.x & 31;
  fs.col = col;
  fs.val = val;
  fs.pos = live ? row_ptr[row] : 0;
  fs.direct = false;
  fs.x = x;
  fs.xpend = 0.f;
  fs.sum = 0.f;
  fs.comp = 0.f;
  fs.constant = S.md.chord == PCT_CHORD_CONSTANT;
  fs.hconst = (float)S.ph.g.h[0];
  walk_row_df<DIM, true>(S, M, Sg, gdg, r, M.r64 + (live ? row : 0), live, fs);
  if (live) b[row] = fs.sum * r.fac;
}

template <int DIM>
__global__ void __launch_bounds__(128) k_fill_mixed(SimDev S, MixArgs M, const SimDev* Sg, const GridDF* gdg,
                                                    long long n, const long long* __restrict__ row_ptr,
                                                    const float* __restrict__ x, int* __restrict__ col,
                                                    float* __restrict__ val, float* __restrict__ b) {
  fill_block<DIM>(S, M, Sg, gdg, n, (long long)blockIdx.x * blockDim.x, row_ptr, x, col, val, b);
}

// ---------------------------------------------------------------------------
// Batch: one persistent launch over the work items (instance, block of 128
// rows) of many heterogeneous simulations.  A block takes the next item from
// a device counter; items are independent, so nothing ever waits.
// ---------------------------------------------------------------------------
__device__ __forceinline__ int batch_find(const BatchInst* __restrict__ B, int n_inst, long long item) {
  int lo = 0, hi = n_inst - 1;  // last instance whose first item is <= item
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (B[mid].item0 <= item)
      lo = mid;
    else
      hi = mid - 1;
  }
  return lo;
}

template <bool kFill, int DIM>
__global__ void __launch_bounds__(128) k_batch(const BatchInst* __restrict__ B, int n_inst, long long first,
                                               long long last, unsigned long long* next) {
  __shared__ long long item_s;
  for (;;) {
    __syncthreads();
    if (threadIdx.x == 0) item_s = first + (long long)atomicAdd(next, 1ULL);
    __syncthreads();
    const long long item = item_s;
    if (item >= last) return;
    const BatchInst& I = B[batch_find(B, n_inst, item)];
    const long long row0 = (item - I.item0) * 128;
    if (kFill)
      fill_block<DIM>(I.S, I.M, &I.S, &I.M.gd, I.n, row0, I.row_ptr, I.x, I.col, I.val, I.b);
    else
      count_block<DIM>(I.S, I.M, &I.S, &I.M.gd, I.n, row0, I.row_ptr_w + 1);
  }
}

int batch_blocks_per_sm(bool fill, int dim) {
  int nb = 0;
  if (fill && dim == 2) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_batch<true, 2>, 128, 0);
  if (fill && dim == 3) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_batch<true, 3>, 128, 0);
  if (!fill && dim == 2) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_batch<false, 2>, 128, 0);
  if (!fill && dim == 3) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_batch<false, 3>, 128, 0);
  return nb > 0 ? nb : 1;
}

void launch_batch(bool fill, int dim, const BatchInst* B, int n_inst, long long first, long long last,
                  unsigned long long* next, int grid, cudaStream_t st) {
  cudaMemsetAsync(next, 0, sizeof(unsigned long long), st);
  if (last <= first || n_inst <= 0) return;
  if (fill && dim == 2) k_batch<true, 2><<<grid, 128, 0, st>>>(B, n_inst, first, last, next);
  if (fill && dim == 3) k_batch<true, 3><<<grid, 128, 0, st>>>(B, n_inst, first, last, next);
  if (!fill && dim == 2) k_batch<false, 2><<<grid, 128, 0, st>>>(B, n_inst, first, last, next);
  if (!fill && dim == 3) k_batch<false, 3><<<grid, 128, 0, st>>>(B, n_inst, first, last, next);
}

// ---------------------------------------------------------------------------
// Matrix-free projectors (rows recomputed, nothing stored): y_i = <a_i, x>
// or g += a_i r_i, for rows [row_base, row_base + n).  Same paths, same
// decisions and the same FP32 lengths as the fill.
// ---------------------------------------------------------------------------
struct DotSinkM {
  static constexpr bool kStaged = false;
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

struct ScatterSinkM {
  static constexpr bool kStaged = false;
  float* g;
  float r;
  __device__ void put(int c, float len) { atomicAdd(g + c, len * r); }
  __device__ void pend(int) {}
};

template <int DIM, bool kAdjoint>
__device__ __forceinline__ void proj_block(const SimDev& S, const MixArgs& M, const SimDev* Sg, const GridDF* gdg,
                                           long long n, long long row0, long long row_base,
                                           const float* __restrict__ in, float* __restrict__ out) {
  long long i = row0 + threadIdx.x;
  int key = -1;
  if (i < n && (!kAdjoint || in[i] != 0.0f)) {
    PathF64 p = path_setup(S, row_base + i);
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

MixArgs mix_args(const SimDev& S, long long n, const void* tab, void* rec) {
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
  M.rdf = (RowDF*)rec;
  M.r64 = (PathF64*)((char*)rec + ((rows * sizeof(RowDF) + 255) & ~(size_t)255));
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
static bool upload_args(const SimDev& S, const MixArgs& M, void* args, cudaStream_t st, const SimDev** Sg,
                        const GridDF** gdg) {
  char* base = (char*)args;
  size_t off = (sizeof(SimDev) + 255) & ~(size_t)255;
  *Sg = (const SimDev*)base;
  *gdg = (const GridDF*)(base + off);
  return cudaMemcpyAsync(base, &S, sizeof(SimDev), cudaMemcpyHostToDevice, st) == cudaSuccess &&
         cudaMemcpyAsync(base + off, &M.gd, sizeof(GridDF), cudaMemcpyHostToDevice, st) == cudaSuccess;
}

void launch_count_mixed(const SimDev& S, const void* tab, long long n, void* rec, long long* counts, void* args,
                        cudaStream_t st) {
  if (n <= 0) return;
  MixArgs M = mix_args(S, n, tab, rec);
  const SimDev* Sg;
  const GridDF* gdg;
  if (!upload_args(S, M, args, st, &Sg, &gdg)) return;
  int threads = 128;
  unsigned blocks = (unsigned)((n + threads - 1) / threads);
  if (S.ph.g.dim == 2)
    k_count_mixed<2><<<blocks, threads, 0, st>>>(S, M, Sg, gdg, n, counts);
  else
    k_count_mixed<3><<<blocks, threads, 0, st>>>(S, M, Sg, gdg, n, counts);
}

void launch_fill_mixed(const SimDev& S, const void* tab, long long n, const void* rec, const long long* row_ptr,
                       const float* x, int* col, float* val, float* b, void* args, cudaStream_t st) {
  if (n <= 0) return;
  MixArgs M = mix_args(S, n, tab, (void*)rec);
  const SimDev* Sg;
  const GridDF* gdg;
  if (!upload_args(S, M, args, st, &Sg, &gdg)) return;
  int threads = 128;
  unsigned blocks = (unsigned)((n + threads - 1) / threads);
  if (S.ph.g.dim == 2)
    k_fill_mixed<2><<<blocks, threads, 0, st>>>(S, M, Sg, gdg, n, row_ptr, x, col, val, b);
  else
    k_fill_mixed<3><<<blocks, threads, 0, st>>>(S, M, Sg, gdg, n, row_ptr, x, col, val, b);
}

void launch_proj_mixed(bool adjoint, const SimDev& S, const void* tab, long long row_base, long long n, void* rec,
                       const float* in, float* out, void* args, cudaStream_t st) {
  if (n <= 0) return;
  MixArgs M = mix_args(S, n, tab, rec);
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

size_t mixed_record_size(long long rows) {
  size_t r = (size_t)(rows > 0 ? rows : 1);
  return ((r * sizeof(RowDF) + 255) & ~(size_t)255) + r * sizeof(PathF64) + 256;
}

}  // namespace pct
