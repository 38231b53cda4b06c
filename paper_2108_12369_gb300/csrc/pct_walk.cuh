// pct_walk.cuh -- the per-lane walker of PCT_PREC_MIXED: one thread steps
// through one row's segments crossing by crossing (lean FP32 stepper, exact
// decisions where its bounds cannot decide, FP64 walk of segments whose
// direction cannot be certified).  The matrix-free projectors use it for
// every row; the count and fill kernels for the rows the warp-cooperative
// form hands over.
#pragma once
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

// Finished entries of a row go to a sink: put(col, len) in path order,
// pend(col) one step before (lets a sink start loading what put() needs).
struct CountSinkM {
  long long n;
  template <class L>
  __device__ void put(int, L) {
    ++n;
  }
  __device__ void pend(int) {}
};

// All segments of one row.  The segment loop runs to the warp's largest
// vertex count so that the lanes set up segment q together.
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
    if (f64seg) {
      double P[3], Q[3];
      path_vertex(*Sg, *p64, q, P);
      path_vertex(*Sg, *p64, q + 1, Q);
      SegF64 s64;
      if (seg_setup_f64(g, P, Q, s64)) seg_walk_f64(g, s64, m64, sink);
    }
    const bool walking = act && res == 1;
    Lean<DIM> L;
    const float seglen = sg.L;
    if (walking) lean_begin<DIM>(g, sg, w, q, L);
    if constexpr (kLengths) {
      if (walking) {
        while (!L.done) {
          const int vc = L.col;
          const float l = lean_step<DIM>(L, r, M.tab, M.R, M.gd, g, mag, ends);
          mg.emit(vc, l * seglen, sink);
        }
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

}  // namespace pct
