// pct_mixed.cu -- PCT_PREC_MIXED kernels.
//   count: FP64 path set-up once per proton (the definition), kept as two row
//          records (FP64 for exact decisions, double-float for the walk);
//          double-float certified traversal -> entries per row.
//   fill:  double-float traversal from the record -> col / val in path order,
//          FP32 Kahan-compensated WEPL, noise factor.
#include "pct_kernels.cuh"
#include "pct_mixed.cuh"

namespace pct {

struct MixArgs {
  GridDF gd;
  df R;                 // lead length, double-float
  const BasisDF* tab;   // [K + 1]
  RowDF* rdf;           // [rows]
  PathF64* r64;         // [rows]
};

// exact endpoints of segment q of a path (for the on-demand FP64 decisions)
struct EndsF64 {
  const SimDev* S;
  const PathF64* p;
  int q;
  __device__ void operator()(double P[3], double Q[3]) const {
    path_vertex(*S, *p, q, P);
    path_vertex(*S, *p, q + 1, Q);
  }
};

// feeds FP64-walked entries into the FP32 row merge
template <class M>
struct MergeToF32 {
  M* mg;
  template <class Sink>
  __device__ void emit(int col, double len, Sink& sink) {
    mg->emit(col, (float)len, sink);
  }
};

struct CountSinkM {
  long long n;
  template <class L>
  __device__ void put(int, L) {
    ++n;
  }
};

struct FillSinkM {
  int* col;
  float* val;
  const float* x;
  long long pos;
  float sum, comp;  // Kahan-compensated WEPL
  bool constant;
  float hconst;
  __device__ void put(int c, float len) {
    col[pos] = c;
    val[pos] = constant ? hconst : len;
    ++pos;
    float y = len * __ldg(x + c) - comp;
    float t = sum + y;
    comp = (t - sum) - y;
    sum = t;
  }
};

// all segments of one row; kLengths selects fill (true) or count (false)
template <int DIM, bool kLengths, class Sink>
__device__ __forceinline__ void walk_row_df(const SimDev& S, const MixArgs& M, const RowDF& r, const PathF64* p64,
                                            Sink& sink) {
  const GridDev& g = S.ph.g;
  RowMerge<float> mg;
  mg.init();
  MergeToF32<RowMerge<float>> m64{&mg};
  df Va[3], Vb[3];
  vertex_df<DIM>(r, M.tab, M.R, 0, Va);
  for (int q = 0; q + 1 < r.nv; ++q) {
    vertex_df<DIM>(r, M.tab, M.R, q + 1, Vb);
    mg.seg_begin();
    SegDF sg;
    EndsF64 ends{&S, p64, q};
    int res = seg_setup_df<DIM>(g, M.gd, Va, Vb, r.mag, sg, ends);
    if (res == 1) {
      walk_df<DIM, kLengths>(g, sg, mg, sink, ends);
    } else if (res == 2) {
      double P[3], Q[3];
      ends(P, Q);
      SegF64 s64;
      if (seg_setup_f64(g, P, Q, s64)) seg_walk_f64(g, s64, m64, sink);
    }
    mg.seg_end();
#pragma unroll
    for (int a = 0; a < DIM; ++a) Va[a] = Vb[a];
  }
  mg.finish(sink);
}

template <int DIM>
__global__ void __launch_bounds__(128) k_count_mixed(SimDev S, MixArgs M, long long n,
                                                     long long* __restrict__ counts) {
  long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= n) return;
  RowDF r;
  {
    PathF64 p = path_setup(S, i);
    M.r64[i] = p;  // exact decisions read the FP64 path back from here
    float fac = (S.md.noise == PCT_NOISE_GAUSS_REL) ? (float)(1.0 + S.md.noise_rel * p.z_noise) : 1.0f;
    make_rowdf<DIM>(p, S.R, fac, r);
  }
  M.rdf[i] = r;
  CountSinkM cs{0};
  walk_row_df<DIM, false>(S, M, r, M.r64 + i, cs);
  counts[i] = cs.n;
}

template <int DIM>
__global__ void __launch_bounds__(128) k_fill_mixed(SimDev S, MixArgs M, long long n,
                                                    const long long* __restrict__ row_ptr,
                                                    const float* __restrict__ x, int* __restrict__ col,
                                                    float* __restrict__ val, float* __restrict__ b) {
  long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const RowDF r = M.rdf[i];
  FillSinkM fs{col, val, x, row_ptr[i], 0.f, 0.f, S.md.chord == PCT_CHORD_CONSTANT, (float)S.ph.g.h[0]};
  walk_row_df<DIM, true>(S, M, r, M.r64 + i, fs);
  b[i] = fs.sum * r.fac;
}

static df split_host(double v) {
  float hi = (float)v;
  return df{hi, (float)(v - (double)hi)};
}

static MixArgs mix_args(const SimDev& S, long long n, const void* tab, void* rec) {
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

void launch_count_mixed(const SimDev& S, const void* tab, long long n, void* rec, long long* counts,
                        cudaStream_t st) {
  if (n <= 0) return;
  MixArgs M = mix_args(S, n, tab, rec);
  int threads = 128;
  unsigned blocks = (unsigned)((n + threads - 1) / threads);
  if (S.ph.g.dim == 2)
    k_count_mixed<2><<<blocks, threads, 0, st>>>(S, M, n, counts);
  else
    k_count_mixed<3><<<blocks, threads, 0, st>>>(S, M, n, counts);
}

void launch_fill_mixed(const SimDev& S, const void* tab, long long n, const void* rec, const long long* row_ptr,
                       const float* x, int* col, float* val, float* b, cudaStream_t st) {
  if (n <= 0) return;
  MixArgs M = mix_args(S, n, tab, (void*)rec);
  int threads = 128;
  unsigned blocks = (unsigned)((n + threads - 1) / threads);
  if (S.ph.g.dim == 2)
    k_fill_mixed<2><<<blocks, threads, 0, st>>>(S, M, n, row_ptr, x, col, val, b);
  else
    k_fill_mixed<3><<<blocks, threads, 0, st>>>(S, M, n, row_ptr, x, col, val, b);
}

size_t mixed_record_size(long long rows) {
  size_t r = (size_t)(rows > 0 ? rows : 1);
  return ((r * sizeof(RowDF) + 255) & ~(size_t)255) + r * sizeof(PathF64) + 256;
}

}  // namespace pct
