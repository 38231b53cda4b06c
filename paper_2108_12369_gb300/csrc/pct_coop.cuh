// pct_coop.cuh -- warp-cooperative traversal of one row (PCT_PREC_MIXED).
//
// The per-lane walker (walk_row_df) steps through a row one crossing at a
// time: every step waits for the previous one.  Here a warp works on one
// row at a time and every crossing is placed on its own:
//  - count: the row's segments are set up in double-float exactly as for
//    the per-lane walker (one segment per lane); each axis' number of
//    crossings inside a segment follows from one certified comparison of the
//    plane nearest the segment's end with that end.  Per-segment counts,
//    merges and prefix sums give the row's entry count; a compact record per
//    segment is kept for the fill;
//  - fill: the row's crossings are spread over the lanes.  Plane i of axis a
//    (counted from the segment's start voxel) is crossing number
//    i + sum_b n_b of its segment, where n_b, the number of axis-b crossings
//    before it, follows from one certified comparison with the nearest
//    axis-b plane.  The voxel it enters is the start voxel moved by i + 1
//    planes along a and n_b planes along every other axis b; the next
//    crossing (the first of a's next plane and every other axis' first plane
//    after it) ends the entry, which the lane writes at its CSR position.
// Where the FP32 bounds cannot decide, the FP64 definition does (out of
// line).  Decisions, voxel indices, lengths and merges are those of the
// per-lane walker.  Rows with an exact tie between crossings of different
// axes, a segment that needs the FP64 walk, more segments than the warp's
// shared-memory capacity (kSegMax at most) or more crossings than it holds
// (kRowCross at most) are handed to the per-lane walker (lane 0 of the warp); the count marks
// them for the fill.
#pragma once
#include "pct_walk.cuh"

namespace pct {

constexpr int kRowIrregular = 1 << 8;  // record 0 of a row: the row goes to the per-lane walker
constexpr int kMergeBit = 1 << 7;      // segment's first entry continues the previous one

// Summary of one set-up segment.  Crossing i of axis a lies at offset
// fmaf(i, hv[a], ph0[a]) from the segment's grid entry, within
// cb[a] + 8u * offset of the FP64 definition's value.
template <int DIM>
struct alignas(16) SegP {
  float ph0[DIM], hv[DIM], cb[DIM], rhv[DIM];
  float send, eend, L, first;  // end offset and its bound, |Q - P|, first entry's length
  int kn[DIM], cnt[DIM];       // next plane index, crossings counted before the end
  int col0, out_k, misc;       // misc: status | (out_ax + 1) << 2 | negative steps << 4
};

constexpr int kStMiss = 0, kStRegular = 1, kStIrregular = 2;

template <int DIM>
__device__ __forceinline__ SegP<DIM> seg_status_only(int status) {
  SegP<DIM> o;
#pragma unroll
  for (int a = 0; a < DIM; ++a) {
    o.ph0[a] = 0.f;
    o.hv[a] = 1.f;
    o.cb[a] = 0.f;
    o.rhv[a] = 1.f;
    o.kn[a] = 0;
    o.cnt[a] = 0;
  }
  o.send = 0.f;
  o.eend = 0.f;
  o.L = 0.f;
  o.first = 0.f;
  o.col0 = 0;
  o.out_k = 0;
  o.misc = status;
  return o;
}

constexpr float kFar = 3e30f;  // offset of an inert axis' planes (never crossed)

// Summary of a set-up segment: per-axis phases and bounds, and the number
// of each axis' planes strictly before the segment's end (the exit plane of
// the exit axis by index, every other axis by one certified comparison).
// A crossing's nearest plane on another axis b is found from its offset
// divided by hv[b]; the guards keep every offset that enters such a
// quotient within 1/64 plane spacing of the FP64 definition's value, so the
// rounded quotient is one of the two planes around the crossing and one
// certified comparison settles which side it is on.
template <int DIM>
__device__ __forceinline__ SegP<DIM> seg_summary(const GridDev& g, const SegDF& sg, const Walk32& w, ExactRef ends) {
  SegP<DIM> o;
  int col = 0, stride = 1, neg = 0;
#pragma unroll
  for (int a = 0; a < DIM; ++a) {
    const bool inert = (sg.inert >> a) & 1u;
    o.ph0[a] = inert ? kFar : w.ph0[a];
    o.hv[a] = inert ? kFar : w.hv[a];
    o.cb[a] = inert ? 0.f : fmaf(8.f * kU32, w.ph0[a] + w.hv[a], w.e0[a]);
    o.rhv[a] = inert ? 0.f : __frcp_rn(w.hv[a]);
    o.kn[a] = sg.kn[a];
    col += sg.idx[a] * stride;
    stride *= g.n[a];
    if (sg.step[a] < 0) neg |= 1 << a;
  }
  o.send = w.send;
  o.eend = w.esend;
  o.L = sg.L;
  o.col0 = col;
  o.out_k = sg.out.k;
  bool ok = true;
  float fmin = w.send, ecr = 0.f;
#pragma unroll
  for (int a = 0; a < DIM; ++a) {
    int c = 0;
    if ((sg.inert >> a) & 1u) {
      c = 0;
    } else if (sg.out.ax == a) {
      c = (sg.out.k - sg.kn[a]) * sg.step[a];
    } else {
      ok = ok && o.hv[a] >= 64.f * (fmaf(8.f * kU32, w.send + 2.f * o.hv[a], o.cb[a]) + w.esend);
      const float jf = fminf(fmaxf(rintf((w.send - o.ph0[a]) * o.rhv[a]), -1.f), 1e6f);
      const float pj = fmaf(jf, o.hv[a], o.ph0[a]);
      const float d = w.send - pj;
      const float e = fmaf(8.f * kU32, fabsf(pj), o.cb[a]) + w.esend;
      const int j = (int)jf;
      if (d > e)
        c = j + 1;
      else if (d < -e)
        c = j;
      else
        c = (exact_cmp(ends, a, sg.kn[a] + sg.step[a] * j, sg.out.ax, sg.out.k) < 0) ? j + 1 : j;
    }
    c = c < 0 ? 0 : c;
    o.cnt[a] = c;
    if (c > 0) {
      fmin = fminf(fmin, o.ph0[a]);
      ecr = fmaxf(ecr, fmaf(8.f * kU32, w.send, o.cb[a]));  // bound of this axis' crossings
    }
  }
  // every other axis' planes near any crossing
#pragma unroll
  for (int b = 0; b < DIM; ++b)
    if (!((sg.inert >> b) & 1u)) ok = ok && o.hv[b] >= 64.f * (ecr + fmaf(8.f * kU32, w.send + 2.f * o.hv[b], o.cb[b]));
  if (!ok) return seg_status_only<DIM>(kStIrregular);
  o.first = fmaxf(fmin, 0.f) * sg.L;
  o.misc = kStRegular | ((sg.out.ax + 1) << 2) | (neg << 4);
  return o;
}

struct DF3 {
  df v[3];
};

// grid entry / exit in double-float (segments with an end outside the grid
// or near a plane): out of line, it is rare inside a row
template <int DIM>
static __device__ __noinline__ SegP<DIM> prepare_slow(const SimDev* Sg, const GridDF* gdg, DF3 P, DF3 Q, float mag,
                                                      ExactRef ends) {
  SegDF sg;
  Walk32 w;
  const int res = seg_setup_df<DIM, true>(Sg->ph.g, *gdg, P.v, Q.v, mag, sg, ends);
  if (res == 0) return seg_status_only<DIM>(kStMiss);
  if (res != 1) return seg_status_only<DIM>(kStIrregular);
  walk_from_df<DIM>(sg, w);
  return seg_summary<DIM>(Sg->ph.g, sg, w, ends);
}

template <int DIM>
__device__ __forceinline__ SegP<DIM> seg_prepare(const GridDev& g, const GridDF& gd, const SimDev* Sg,
                                                 const GridDF* gdg, const df (&P)[3], const df (&Q)[3], float mag,
                                                 ExactRef ends) {
  SegDF sg;
  Walk32 w;
  if (seg_setup_fast<DIM>(g, gd, P, Q, mag, sg, w)) return seg_summary<DIM>(g, sg, w, ends);
  DF3 p3, q3;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    p3.v[a] = (a < DIM) ? P[a] : df{0.f, 0.f};
    q3.v[a] = (a < DIM) ? Q[a] : df{0.f, 0.f};
  }
  return prepare_slow<DIM>(Sg, gdg, p3, q3, mag, ends);
}

// lead segments (vertex 0 -> 1 and nv-2 -> nv-1), two records per row
template <int DIM>
__device__ __forceinline__ SegP<DIM>* lead_rec(const MixArgs& M, long long row) {
  return (SegP<DIM>*)M.lead + 2 * row;
}

// ---------------------------------------------------------------------------
// Compact segment record.  The count kernel writes one per segment (row
// stride: the model's largest segment count); the fill reads them instead
// of setting the segments up again.  Words (DIM = 2 | 3):
//   ph0[DIM] hv[DIM] cb[DIM] send L first col0 misc cnt (u16 pairs) ebase tail
// ebase: the segment's first entry within the row; tail: the length the
// first entries of the following segments add to its last entry when they
// continue its voxel (merges across polyline joints).
// ---------------------------------------------------------------------------
template <int DIM>
struct SegW {
  static constexpr int PH0 = 0, HV = DIM, CB = 2 * DIM, SEND = 3 * DIM, L = 3 * DIM + 1, FIRST = 3 * DIM + 2,
                       COL0 = 3 * DIM + 3, MISC = 3 * DIM + 4, CNT = 3 * DIM + 5, EBASE = CNT + (DIM + 1) / 2,
                       TAIL = EBASE + 1, NV = (TAIL + 4) / 4;  // int4 per record
};

template <int DIM>
struct alignas(16) SegG {
  int4 v[SegW<DIM>::NV];
};

// the record as registers
template <int DIM>
struct SegR {
  int w[4 * SegW<DIM>::NV];
  __device__ float f(int k) const { return __int_as_float(w[k]); }
  __device__ int cnt(int a) const {
    const int x = w[SegW<DIM>::CNT + (a >> 1)];
    return (a & 1) ? (int)((unsigned)x >> 16) : (x & 0xffff);
  }
  __device__ int C() const {
    int c = 0;
#pragma unroll
    for (int a = 0; a < DIM; ++a) c += cnt(a);
    return c;
  }
};

template <int DIM>
__device__ __forceinline__ SegR<DIM> load_seg(const SegG<DIM>& g) {
  SegR<DIM> r;
#pragma unroll
  for (int q = 0; q < SegW<DIM>::NV; ++q) {
    const int4 v = g.v[q];
    r.w[4 * q] = v.x;
    r.w[4 * q + 1] = v.y;
    r.w[4 * q + 2] = v.z;
    r.w[4 * q + 3] = v.w;
  }
  return r;
}

template <int DIM>
__device__ __forceinline__ void store_rec(SegG<DIM>& g, const SegR<DIM>& r) {
#pragma unroll
  for (int q = 0; q < SegW<DIM>::NV; ++q) g.v[q] = make_int4(r.w[4 * q], r.w[4 * q + 1], r.w[4 * q + 2], r.w[4 * q + 3]);
}

template <int DIM>
__device__ __forceinline__ SegR<DIM> pack_seg(const SegP<DIM>& p) {
  using W = SegW<DIM>;
  SegR<DIM> r;
#pragma unroll
  for (int k = 0; k < 4 * W::NV; ++k) r.w[k] = 0;
#pragma unroll
  for (int a = 0; a < DIM; ++a) {
    r.w[W::PH0 + a] = __float_as_int(p.ph0[a]);
    r.w[W::HV + a] = __float_as_int(p.hv[a]);
    r.w[W::CB + a] = __float_as_int(p.cb[a]);
    r.w[W::CNT + (a >> 1)] |= (a & 1) ? (p.cnt[a] << 16) : p.cnt[a];
  }
  r.w[W::SEND] = __float_as_int(p.send);
  r.w[W::L] = __float_as_int(p.L);
  r.w[W::FIRST] = __float_as_int(p.first);
  r.w[W::COL0] = p.col0;
  r.w[W::MISC] = p.misc;
  return r;
}

constexpr int kSegMax = 64;     // segments of one row handled cooperatively (at most)
constexpr int kSegSmall = 36;   // the smaller per-warp capacity (splines of up to 34 pieces)
constexpr int kRowCross = 4096; // crossings of one row handled cooperatively

constexpr int kQueue = 32;  // crossings per pass left to the exact path
// the smaller per-warp layout (kSegSmall segments) also holds fewer crossings
// and queue entries: rows beyond them take the per-lane walker
constexpr int kRowCrossSmall = 2048;
constexpr int kQueueSmall = 16;

// Count: the row's segment records plus the crossing enumeration, for rows
// of up to CAP segments (a smaller CAP leaves more of the SM's on-chip
// memory to the L1 cache)
template <int DIM, int CAP = kSegMax>
struct CoopSmem {
  static constexpr int kCap = CAP;
  static constexpr int kCross = CAP <= kSegSmall ? kRowCrossSmall : kRowCross;
  static constexpr int kQ = CAP <= kSegSmall ? kQueueSmall : kQueue;
  SegG<DIM> tab[CAP];
  unsigned bits[kCross / 32 + 4];  // segment starts among the row's crossings
  unsigned char ord[CAP];             // k-th segment with crossings
  int aux[CAP];                       // first position of each segment in the current pass
  int q[kQ];                          // crossings (segment | ordinal << 8) left to the exact path
  int qn;
  __device__ int cnt(int s, int a) const {
    const int w = reinterpret_cast<const int*>(&tab[s])[SegW<DIM>::CNT + (a >> 1)];
    return (a & 1) ? (int)((unsigned)w >> 16) : (w & 0xffff);
  }
};

// Fill: the records expanded into per-field arrays (no unpacking per crossing)
template <int DIM, int CAP = kSegMax, bool LEAN = false>
struct FillSmem {
  static constexpr int kCap = CAP;
  static constexpr bool kLean = LEAN;
  SegG<DIM> tab[LEAN ? CAP : 1];  // lean form: the row's segment table, rebuilt here
  static constexpr int kCross = CAP <= kSegSmall ? kRowCrossSmall : kRowCross;
  static constexpr int kQ = CAP <= kSegSmall ? kQueueSmall : kQueue;
  float4 ax[DIM][CAP];  // per axis: ph0, hv, 1 / hv, cb
  int4 cn[CAP];         // crossings per axis (x, y, z), column of the start voxel (w)
  int4 dc[CAP];         // signed column step per axis (x, y, z), first entry's CSR slot + 1 (w)
  float4 sf[CAP];       // send, L, merged tail of the last entry, first entry's length
  int misc[CAP];
  // the two passes' positions (fill_plan): per pass the bitmap of run
  // starts and the run -> segment map; per segment its first position in
  // the axis-0, axis-1 and axis-2 groups
  unsigned bits[kCross / 32 + 4];
  unsigned bits1[kCross / 32 + 4];
  unsigned char ord[CAP];
  unsigned char ord1[2 * CAP];  // a segment can start a run in each of pass 1's two groups
  int aux[CAP];
  int aux1[CAP];
  int aux2[CAP];
  int q[kQ];
  int qn;
  __device__ int cnt(int s, int a) const { return a == 0 ? cn[s].x : (a == 1 ? cn[s].y : cn[s].z); }
};

template <int DIM>
__device__ __forceinline__ int dcol_of(const int (&stride)[3], int misc, int a) {
  int r = stride[0];
#pragma unroll
  for (int b = 1; b < DIM; ++b)
    if (a == b) r = stride[b];
  return ((misc >> (4 + a)) & 1) ? -r : r;
}

// plane index of ordinal k of axis a (counted from the segment's start
// voxel, recovered from its column index)
template <int DIM>
__device__ __forceinline__ int plane_of(const GridDev& g, int col0, int misc, int a, int k) {
  int q = col0, idx = 0;
#pragma unroll
  for (int b = 0; b < DIM; ++b) {
    const int i = (b < DIM - 1) ? q % g.n[b] : q;
    if (b == a) idx = i;
    if (b < DIM - 1) q /= g.n[b];
  }
  const bool neg = (misc >> (4 + a)) & 1;
  return neg ? idx - k : idx + 1 + k;
}

// warp-wide exclusive prefix sum of v; *total receives the sum
__device__ __forceinline__ int warp_excl_scan(int v, int lane, int* total) {
  int x = v;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    int y = __shfl_up_sync(0xffffffffu, x, d);
    if (lane >= d) x += y;
  }
  *total = __shfl_sync(0xffffffffu, x, 31);
  return x - v;
}

// segment of crossing position p in round p0 (positions p0 .. p0 + 31 lie in
// bitmap word p0 / 32); ordbase counts the starts of earlier rounds
__device__ __forceinline__ int seg_at(const unsigned* bits, const unsigned char* ord, int p0, int lane, int& ordbase) {
  const unsigned word = bits[p0 >> 5];
  const int k = ordbase + __popc(word & (0xffffffffu >> (31 - lane))) - 1;
  ordbase += __popc(word);
  return ord[k < 0 ? 0 : k];
}

struct Kahan {
  float sum, comp;
  __device__ void add(float v) {
    float y = v - comp;
    float t = sum + y;
    comp = (t - sum) - y;
    sum = t;
  }
};

// Direct-write sink for rows handed to the per-lane walker (one live lane).
struct FillSinkD {
  int* col;
  float* val;
  long long pos, end;  // next position and the end of the row's range
  const float* x;
  float xpend;
  Kahan k;
  bool constant;
  float hconst;
  __device__ void pend(int c) { xpend = __ldg(x + c); }
  __device__ void put(int c, float len) {
    if (pos < end) {
      col[pos] = c;
      val[pos] = constant ? hconst : len;
    }
    ++pos;
    k.add(len * xpend);
  }
};

// A row the cooperative form does not take, walked by lane 0 with the
// per-lane walker (all lanes call: the walker's segment loop is warp-wide).
// Out of line so that its registers and code stay off the common path.
template <int DIM, bool kFill>
static __device__ __noinline__ void walk_row_lane0(const SimDev* Sg, MixArgs M, long long row,
                                                   long long* __restrict__ counts, long long rowstart,
                                                   long long rowend, const float* __restrict__ x,
                                                   int* __restrict__ col, float* __restrict__ val,
                                                   float* __restrict__ b) {
  const int lane = threadIdx.x & 31;
  const SimDev& S = *Sg;
  const RowDF& r = M.rdf[row];
  const PathF64* p64 = M.r64 + row;
  if constexpr (kFill) {
    FillSinkD fs;
    fs.col = col;
    fs.val = val;
    fs.pos = rowstart;
    fs.end = rowend;
    fs.x = x;
    fs.xpend = 0.f;
    fs.k = Kahan{0.f, 0.f};
    fs.constant = S.md.chord == PCT_CHORD_CONSTANT;
    fs.hconst = (float)S.ph.g.h[0];
    walk_row_df<DIM, true>(S, M, Sg, nullptr, r, p64, lane == 0, fs);
    if (lane == 0) {
      b[row] = fs.k.sum * r.fac;
      if (fs.pos != fs.end) note_row_mismatch(S);
    }
  } else {
    CountSinkM cs{0};
    walk_row_df<DIM, false>(S, M, Sg, nullptr, r, p64, lane == 0, cs);
    if (lane == 0) {
      counts[row] = cs.n;
      if (M.rflag) {
        M.rflag[row] = 1;  // lean form: the row flag
      } else {
        SegG<DIM>* rec = (SegG<DIM>*)M.segg + row * (long long)M.seg_stride;
        reinterpret_cast<int*>(rec)[SegW<DIM>::MISC] = kRowIrregular;
      }
    }
  }
  __syncwarp();
}

// One crossing's view of its segment: the crossing's own axis first, the
// other axes after it in increasing order (selects only, no indexing).
template <int DIM>
struct Axes {
  float p0[DIM], h[DIM], c[DIM];  // phase, spacing and bound constant per axis
  int n[DIM], dc[DIM], ax[DIM];   // crossings, column step, original axis
};

struct Cross {
  int rank;   // position among the segment's crossings
  int colv;   // voxel entered
  float nv;   // offset of the next crossing (the segment's end after the last)
  bool last;
};

// Crossing i of axis A (known at compile time) from the fill's arrays:
// ax[c] = (ph0, hv, 1/hv, cb), cn = (crossings per axis, start column),
// dc = (signed column steps, -).  Decisions from the FP32 bounds; *unsure
// where they cannot decide (the crossing then goes to cross_exact).  The
// next crossing is the first of: this axis' next plane, every other axis'
// first plane after the crossing.
template <int DIM, int A>
__device__ __forceinline__ Cross cross_x(const float4 (&ax)[DIM], const int4& cn, const int4& dc, float send, int i,
                                         float& ph, bool& unsure) {
  const int na = A == 0 ? cn.x : (A == 1 ? cn.y : cn.z);
  const int da = A == 0 ? dc.x : (A == 1 ? dc.y : dc.z);
  Cross o;
  ph = fmaf((float)i, ax[A].y, ax[A].x);
  o.rank = i;
  o.colv = cn.w + (i + 1) * da;
  bool has = i + 1 < na;
  float vm = fmaf((float)(i + 1), ax[A].y, ax[A].x), cm = ax[A].w;
#pragma unroll
  for (int c = 0; c < DIM; ++c) {
    if (c == A) continue;
    const int nc = c == 0 ? cn.x : (c == 1 ? cn.y : cn.z);
    const int dcc = c == 0 ? dc.x : (c == 1 ? dc.y : dc.z);
    const float jf = rintf((ph - ax[c].x) * ax[c].z);
    const float pb = fmaf(jf, ax[c].y, ax[c].x);
    const float d = ph - pb;
    const int j = (int)jf;
    unsure = unsure || (j >= 0 && j < nc && !(fabsf(d) > fmaf(8.f * kU32, ph + fabsf(pb), ax[A].w + ax[c].w)));
    int nb = j + (d > 0.f ? 1 : 0);
    nb = nb < 0 ? 0 : (nb > nc ? nc : nb);
    o.rank += nb;
    o.colv += nb * dcc;
    const float v = fmaf((float)nb, ax[c].y, ax[c].x);
    const bool hv_ = nb < nc;
    const float d2 = v - vm;
    unsure = unsure || (hv_ && has && !(fabsf(d2) > fmaf(8.f * kU32, v + vm, ax[c].w + cm)));
    const bool take = hv_ && (!has || d2 < 0.f);
    vm = take ? v : vm;
    cm = take ? ax[c].w : cm;
    has = has || hv_;
  }
  o.last = !has;
  o.nv = has ? vm : send;
  return o;
}

// The same crossing with every decision exact: FP64 comparisons where the
// FP32 bounds cannot decide (a few crossings per thousand rows).
template <int DIM>
static __device__ __noinline__ Cross cross_exact(const SimDev* Sg, const PathF64* p64, int s, Axes<DIM> X, int i,
                                                 int col0, int misc, float send) {
  const GridDev& g = Sg->ph.g;
  const ExactRef ref{Sg, p64, s};
  Cross o;
  const float ph = fmaf((float)i, X.h[0], X.p0[0]);
  const int a = X.ax[0];
  o.rank = i;
  o.colv = col0 + (i + 1) * X.dc[0];
  int mk = i + 1 < X.n[0] ? 0 : -1, mi = i + 1;
  float vm = fmaf((float)(i + 1), X.h[0], X.p0[0]), cm = X.c[0];
  for (int k = 1; k < DIM; ++k) {
    const int c = X.ax[k];
    const float jf = rintf(__fdividef(ph - X.p0[k], X.h[k]));
    const float pb = fmaf(jf, X.h[k], X.p0[k]);
    const float d = ph - pb;
    const float e = fmaf(8.f * kU32, ph + fabsf(pb), X.c[0] + X.c[k]);
    const int j = (int)jf;
    int nb;
    if (d > e || j < 0 || j >= X.n[k])
      nb = d > 0.f ? j + 1 : j;
    else if (d < -e)
      nb = j;
    else
      nb = exact_cmp(ref, a, plane_of<DIM>(g, col0, misc, a, i), c, plane_of<DIM>(g, col0, misc, c, j)) > 0 ? j + 1
                                                                                                              : j;
    nb = nb < 0 ? 0 : (nb > X.n[k] ? X.n[k] : nb);
    o.rank += nb;
    o.colv += nb * X.dc[k];
    if (nb < X.n[k]) {
      const float v = fmaf((float)nb, X.h[k], X.p0[k]);
      bool take = mk < 0;
      if (!take) {
        const float d2 = v - vm;
        const float e2 = fmaf(8.f * kU32, v + vm, X.c[k] + cm);
        if (d2 < -e2)
          take = true;
        else if (!(d2 > e2))
          take = exact_cmp(ref, c, plane_of<DIM>(g, col0, misc, c, nb), X.ax[mk],
                           plane_of<DIM>(g, col0, misc, X.ax[mk], mi)) < 0;
      }
      if (take) {
        mk = k;
        mi = nb;
        vm = v;
        cm = X.c[k];
      }
    }
  }
  o.last = mk < 0;
  o.nv = mk < 0 ? send : vm;
  return o;
}

// field a of a record's per-axis group k0 (selects, no indexing)
template <int DIM>
__device__ __forceinline__ float rec_f(const SegR<DIM>& R, int k0, int a) {
  return a == 0 ? R.f(k0) : (a == 1 || DIM == 2 ? R.f(k0 + 1) : R.f(k0 + DIM - 1));
}

// exact tie of crossing i of axis u with the nearest plane of axis v
template <int DIM>
static __device__ __noinline__ bool tie_exact(const SimDev* Sg, const PathF64* p64, int s, const SegG<DIM>* rec, int u,
                                              int v, int i) {
  using W = SegW<DIM>;
  const SegR<DIM> R = load_seg<DIM>(*rec);
  const float ph = fmaf((float)i, rec_f<DIM>(R, W::HV, u), rec_f<DIM>(R, W::PH0, u));
  const float jf = rintf(__fdividef(ph - rec_f<DIM>(R, W::PH0, v), rec_f<DIM>(R, W::HV, v)));
  const int j = (int)jf;
  if (j < 0 || j >= R.cnt(v)) return false;
  const GridDev& g = Sg->ph.g;
  const int col0 = R.w[W::COL0], misc = R.w[W::MISC];
  return exact_cmp(ExactRef{Sg, p64, s}, u, plane_of<DIM>(g, col0, misc, u, i), v, plane_of<DIM>(g, col0, misc, v, j)) ==
         0;
}

// marks the runs of segments sa = 2 lane and sb = sa + 1 (na and nb items
// from positions ba and bb) in bits and their segments in ord, from run k0
// on; returns k0 + the number of runs marked
__device__ __forceinline__ unsigned mark_pair(unsigned* bits, unsigned char* ord, unsigned k0, int na, int nb, int ba,
                                              int bb, int sa, unsigned lt) {
  const unsigned bal_a = __ballot_sync(0xffffffffu, na > 0), bal_b = __ballot_sync(0xffffffffu, nb > 0);
  const unsigned r = k0 + __popc(bal_a & lt) + __popc(bal_b & lt);
  if (na > 0) {
    atomicOr(bits + (ba >> 5), 1u << (ba & 31));
    ord[r] = (unsigned char)sa;
  }
  if (nb > 0) {
    atomicOr(bits + (bb >> 5), 1u << (bb & 31));
    ord[r + (na > 0 ? 1 : 0)] = (unsigned char)(sa + 1);
  }
  return k0 + __popc(bal_a) + __popc(bal_b);
}

// Exact ties between crossings of different axes, every pair of axes in one
// pass.  A tie is a crossing of each axis of the pair at the same point, so
// it is found from either side: for each pair the pass takes the crossings
// of the axis with fewer of them in the segment, each against the nearest
// plane of the other axis.  FP32 bounds settle almost all; the crossings
// they cannot settle are queued and decided by the FP64 definition after
// the pass (no call in the loop); *overflow when the queue was full.
template <int DIM, class SM>
__device__ __forceinline__ void tie_pass(SM& sm, int nseg, int lane, const SimDev* Sg, const PathF64* p64, bool& tie,
                                         bool& overflow) {
  using W = SegW<DIM>;
  // positions: one lane per two segments (2 lane, 2 lane + 1), one scan
  const int sa = 2 * lane;
  int n[2] = {0, 0};
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const int s = sa + h;
    if (s < nseg) {
      const int n0 = sm.cnt(s, 0), n1 = sm.cnt(s, 1);
      n[h] = min(n0, n1);
      if constexpr (DIM > 2) {
        const int n2 = sm.cnt(s, 2);
        n[h] += min(n0, n2) + min(n1, n2);
      }
    }
  }
  int tot;
  const int ba = warp_excl_scan(n[0] + n[1], lane, &tot), bb = ba + n[0];
  if (sa < nseg) sm.aux[sa] = ba;
  if (sa + 1 < nseg) sm.aux[sa + 1] = bb;
  for (int w = lane; w < tot / 32 + 1; w += 32) sm.bits[w] = 0u;
  if (lane == 0) sm.qn = 0;
  __syncwarp();
  mark_pair(sm.bits, sm.ord, 0u, n[0], n[1], ba, bb, sa, (1u << lane) - 1u);
  __syncwarp();
  int ordbase = 0;
  for (int p0 = 0; p0 < tot; p0 += 32) {
    const int s = seg_at(sm.bits, sm.ord, p0, lane, ordbase);
    const int p = p0 + lane;
    if (p < tot) {
      const int* wi = reinterpret_cast<const int*>(&sm.tab[s]);
      const float* wf = reinterpret_cast<const float*>(wi);
      const int c01 = wi[W::CNT];
      const int n0 = c01 & 0xffff, n1 = (int)((unsigned)c01 >> 16);
      int i = p - sm.aux[s];
      // the pair (c, a) of item i: (0, 1), then (0, 2) and (1, 2)
      int a = 1, c = 0, na = n1, nc = n0;
      if constexpr (DIM > 2) {
        const int n2 = wi[W::CNT + 1] & 0xffff;
        const int m01 = min(n0, n1);
        if (i >= m01) {
          i -= m01;
          a = 2;
          na = n2;
          const int m02 = min(n0, n2);
          if (i >= m02) {
            i -= m02;
            c = 1;
            nc = n1;
          }
        }
      }
      const bool first_a = na <= nc;
      const int u = first_a ? a : c, v = first_a ? c : a, nv = first_a ? nc : na;
      const float ph = fmaf((float)i, wf[W::HV + u], wf[W::PH0 + u]);
      const float p0v = wf[W::PH0 + v], hv = wf[W::HV + v];
      const float jf = rintf(__fdividef(ph - p0v, hv));
      const float pb = fmaf(jf, hv, p0v);
      const int j = (int)jf;
      if (j >= 0 && j < nv && !(fabsf(ph - pb) > fmaf(8.f * kU32, ph + fabsf(pb), wf[W::CB + u] + wf[W::CB + v]))) {
        const int k = atomicAdd(&sm.qn, 1);
        if (k < SM::kQ)
          sm.q[k] = s | (u << 8) | (v << 10) | (i << 12);
        else
          overflow = true;
      }
    }
  }
  __syncwarp();
  const int nq = min(sm.qn, SM::kQ);
  for (int k = lane; k < nq; k += 32) {
    const int e = sm.q[k], s = e & 0xff;
    tie = tie || tie_exact<DIM>(Sg, p64, s, &sm.tab[s], (e >> 8) & 3, (e >> 10) & 3, e >> 12);
  }
  __syncwarp();
}

// per-row output of the fill
struct FillOut {
  int* col;  // the row's first CSR position
  float* val;
  int len;   // entries of the row
  const float* x;
  int nvox;
  bool constant;
  float hconst;
};

// segment s of the fill's arrays as the exact path's view (axis A first)
template <int DIM, class SM>
__device__ __forceinline__ Axes<DIM> fill_axes(const SM& sm, int s, int a) {
  float p0[DIM], h[DIM], c[DIM];
  int n[DIM], d[DIM];
  const int4 cn = sm.cn[s], dc = sm.dc[s];
#pragma unroll
  for (int k = 0; k < DIM; ++k) {
    const float4 v = sm.ax[k][s];
    p0[k] = v.x;
    h[k] = v.y;
    c[k] = v.w;
    n[k] = k == 0 ? cn.x : (k == 1 ? cn.y : cn.z);
    d[k] = k == 0 ? dc.x : (k == 1 ? dc.y : dc.z);
  }
  int order[DIM];
  if constexpr (DIM == 2) {
    order[0] = a;
    order[1] = 1 - a;
  } else {
    order[0] = a;
    order[1] = a == 0 ? 1 : 0;
    order[2] = a == 2 ? 1 : 2;
  }
  Axes<DIM> X;
#pragma unroll
  for (int k = 0; k < DIM; ++k) {
    X.p0[k] = pick<DIM>(p0, order[k]);
    X.h[k] = pick<DIM>(h, order[k]);
    X.c[k] = pick<DIM>(c, order[k]);
    X.n[k] = pick<DIM>(n, order[k]);
    X.dc[k] = pick<DIM>(d, order[k]);
    X.ax[k] = order[k];
  }
  return X;
}

// one entry: write it; returns its voxel's x_true (loaded, not yet used)
__device__ __forceinline__ float put_entry_x(const FillOut& F, int o, int c, float v) {
  if (o < F.len) {
    F.col[o] = c;
    F.val[o] = F.constant ? F.hconst : v;
  }
  return __ldg(F.x + ((unsigned)c < (unsigned)F.nvox ? c : 0));
}

// one entry: write it and add its WEPL term
__device__ __forceinline__ void put_entry(const FillOut& F, int o, int c, float v, Kahan& wk) {
  if (o < F.len) {
    F.col[o] = c;
    F.val[o] = F.constant ? F.hconst : v;
  }
  wk.add(v * __ldg(F.x + ((unsigned)c < (unsigned)F.nvox ? c : 0)));
}

// The fill's two passes over a row: pass 0 takes the axis-0 crossings of the
// row's segments in order; pass 1 the axis-1 crossings and, in 3D, after all
// of them the axis-2 crossings (a few per row on paths that run across the
// slices), so that these fill axis 1's last round instead of a round of
// their own.  fill_plan sets up both passes' positions at once: one lane per
// two segments (2 lane, 2 lane + 1), one warp scan for the axis-0 and axis-1
// counts together (low and high 16 bits; every total is at most kCross <
// 2^16, so no field carries into the other) and one for axis 2.
struct FillPlan {
  int tot0, tot1, tot;  // pass 0's positions; pass 1's axis-1 and all positions
};

template <int DIM, class SM>
__device__ __forceinline__ FillPlan fill_plan(SM& sm, int nseg, int lane) {
  const int sa = 2 * lane, sb = sa + 1;
  int4 ca = make_int4(0, 0, 0, 0), cb = ca;
  if (sa < nseg) ca = sm.cn[sa];
  if (sb < nseg) cb = sm.cn[sb];
  int t01, t2 = 0;
  const int pa = ca.x | (ca.y << 16);
  const int e01 = warp_excl_scan(pa + (cb.x | (cb.y << 16)), lane, &t01);
  int e2 = 0;
  if constexpr (DIM > 2) e2 = warp_excl_scan(ca.z + cb.z, lane, &t2);
  FillPlan P;
  P.tot0 = t01 & 0xffff;
  P.tot1 = t01 >> 16;
  P.tot = P.tot1 + t2;
  const int b0a = e01 & 0xffff, b1a = e01 >> 16, b2a = P.tot1 + e2;
  const int b0b = b0a + ca.x, b1b = b1a + ca.y, b2b = b2a + ca.z;
  if (sa < nseg) {
    sm.aux[sa] = b0a;
    sm.aux1[sa] = b1a;
    sm.aux2[sa] = b2a;
  }
  if (sb < nseg) {
    sm.aux[sb] = b0b;
    sm.aux1[sb] = b1b;
    sm.aux2[sb] = b2b;
  }
  const int w0 = P.tot0 / 32 + 1, w1 = P.tot / 32 + 1;
  for (int w = lane; w < w0; w += 32) sm.bits[w] = 0u;
  for (int w = lane; w < w1; w += 32) sm.bits1[w] = 0u;
  __syncwarp();
  const unsigned lt = (1u << lane) - 1u;
  mark_pair(sm.bits, sm.ord, 0u, ca.x, cb.x, b0a, b0b, sa, lt);
  const unsigned k1 = mark_pair(sm.bits1, sm.ord1, 0u, ca.y, cb.y, b1a, b1b, sa, lt);
  if constexpr (DIM > 2) mark_pair(sm.bits1, sm.ord1, k1, ca.z, cb.z, b2a, b2b, sa, lt);
  __syncwarp();
  return P;
}

// One pass: positions [0, tot1) are crossings of axis A1 (first position of
// segment s: aux1[s]), [tot1, tot) crossings of axis A2 (aux2[s]; none when
// A2 < 0).  One entry per crossing, written at its CSR position.  Crossings
// the FP32 bounds cannot settle are queued and redone exactly after the pass
// (no call in the loop); *overflow when the queue was full.
template <int DIM, int A1, int A2, class SM>
__device__ __forceinline__ void fill_pass(SM& sm, int tot1, int tot, const int* aux1, const int* aux2,
                                          const unsigned* bits, const unsigned char* ord, int lane, const SimDev* Sg,
                                          const PathF64* p64, const FillOut& F, Kahan& wk, bool& overflow) {
  constexpr int B = A2 < 0 ? A1 : A2;
  if (lane == 0) sm.qn = 0;
  __syncwarp();
  int ordbase = 0;
  // a round's x_true load is consumed one round later, so that it overlaps
  // the next round's work
  float pv = 0.f, px = 0.f;
  for (int p0 = 0; p0 < tot; p0 += 32) {
    const int s = seg_at(bits, ord, p0, lane, ordbase);
    const int p = p0 + lane;
    float v = 0.f, xv = 0.f;
    if (p < tot) {
      float4 ax[DIM];
#pragma unroll
      for (int c = 0; c < DIM; ++c) ax[c] = sm.ax[c][s];
      const int4 cn = sm.cn[s], dc = sm.dc[s];
      const float4 sf = sm.sf[s];
      const bool second = A2 >= 0 && p >= tot1;
      const int i = p - (second ? aux2[s] : aux1[s]);
      bool unsure = false;
      float ph;
      Cross cr;
      if (!second)
        cr = cross_x<DIM, A1>(ax, cn, dc, sf.x, i, ph, unsure);
      else
        cr = cross_x<DIM, B>(ax, cn, dc, sf.x, i, ph, unsure);
      if (!unsure) {
        v = fmaf(fmaxf(cr.nv - ph, 0.f), sf.y, cr.last ? sf.z : 0.f);
        xv = put_entry_x(F, dc.w + cr.rank, cr.colv, v);
      } else {
        const int k = atomicAdd(&sm.qn, 1);
        if (k < SM::kQ)
          sm.q[k] = s | ((second ? B : A1) << 8) | (i << 10);
        else
          overflow = true;
      }
    }
    wk.add(pv * px);
    pv = v;
    px = xv;
  }
  wk.add(pv * px);
  __syncwarp();
  const int nq = min(sm.qn, SM::kQ);
  for (int k = lane; k < nq; k += 32) {
    const int s = sm.q[k] & 0xff, a = (sm.q[k] >> 8) & 3, i = sm.q[k] >> 10;
    const float4 sf = sm.sf[s];
    const float4 axa = sm.ax[a][s];
    const float ph = fmaf((float)i, axa.y, axa.x);
    const Cross cr = cross_exact<DIM>(Sg, p64, s, fill_axes<DIM>(sm, s, a), i, sm.cn[s].w, sm.misc[s], sf.x);
    const float v = fmaf(fmaxf(cr.nv - ph, 0.f), sf.y, cr.last ? sf.z : 0.f);
    put_entry(F, sm.dc[s].w + cr.rank, cr.colv, v, wk);
  }
  __syncwarp();
}

// ---------------------------------------------------------------------------
// Count: one row, the whole warp.  Sets up the interior segments (one per
// lane), forms the per-segment counts, merges and prefix sums, looks for
// exact ties between crossings of different axes, writes the compact
// segment records and the row's entry count.
// ---------------------------------------------------------------------------
// Steps 1-2 of the count, shared with the lean fill: the row's segment table
// in tab[0..nseg) -- lead segments from the path kernel, interior ones set up
// here (one per lane) -- with each segment's merge bit, first CSR slot within
// the row and merged tail.  *totE receives the row's entry count.  Returns
// false where the cooperative form cannot take the row (a segment it cannot
// set up, more than kCross crossings).
template <int DIM, int kCross>
__device__ __forceinline__ bool row_table(const SimDev& S, const MixArgs& M, const SimDev* Sg, const GridDF* gdg,
                                          long long row, int nseg, SegG<DIM>* tab, int* totE) {
  using W = SegW<DIM>;
  const int lane = threadIdx.x & 31;
  const GridDev& g = S.ph.g;
  const RowDF& r = M.rdf[row];
  const int stride[3] = {1, g.n[0], g.n[0] * (DIM > 2 ? g.n[1] : 1)};
  const PathF64* p64 = M.r64 + row;
  // 1. segment table: lead segments from the pre-pass, interior ones here
  const SegP<DIM>* lead = lead_rec<DIM>(M, row);
  if (lane < 2 && (lane == 0 || nseg > 1)) {
    const SegP<DIM> p = lead[lane];
    const int s = lane == 0 ? 0 : nseg - 1;
    store_rec<DIM>(tab[s], pack_seg<DIM>(p));
  }
  const int nint = nseg - 2;
  const float mag = r.mag;
  for (int base = 0; base < nint; base += 32) {
    const int j = base + lane;
    df V[3], Vn[3];
    if (j <= nint) vertex_df<DIM>(r, M.tab, M.R, 1 + j, V);
#pragma unroll
    for (int a = 0; a < DIM; ++a) {
      Vn[a].hi = __shfl_down_sync(0xffffffffu, V[a].hi, 1);
      Vn[a].lo = __shfl_down_sync(0xffffffffu, V[a].lo, 1);
    }
    if (lane == 31 && j < nint) vertex_df<DIM>(r, M.tab, M.R, 2 + j, Vn);
    if (j < nint) {
      const SegP<DIM> p = seg_prepare<DIM>(g, M.gd, Sg, gdg, V, Vn, mag, ExactRef{Sg, p64, 1 + j});
      store_rec<DIM>(tab[1 + j], pack_seg<DIM>(p));
    }
  }
  __syncwarp();

  // 2. per-segment crossings, merges, entries; prefix sums
  int bad = 0, merge[2] = {0, 0}, Cs[2] = {0, 0}, Es[2] = {0, 0};
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const int s = lane + 32 * h;
    if (s < nseg) {
      const SegR<DIM> R = load_seg<DIM>(tab[s]);
      const int st = R.w[W::MISC] & 3;
      int m = 0;
      if (s > 0 && st == kStRegular) {
        const SegR<DIM> Q = load_seg<DIM>(tab[s - 1]);
        if ((Q.w[W::MISC] & 3) == kStRegular) {
          int colx = Q.w[W::COL0];
#pragma unroll
          for (int a = 0; a < DIM; ++a) colx += Q.cnt(a) * dcol_of<DIM>(stride, Q.w[W::MISC], a);
          m = colx == R.w[W::COL0];
        }
      }
      Cs[h] = R.C();
      Es[h] = (st == kStRegular) ? Cs[h] + 1 - m : 0;
      merge[h] = m;
      bad |= st == kStIrregular;
    }
  }
  int t0, t1, eb[2];
  const int totC = __reduce_add_sync(0xffffffffu, Cs[0] + Cs[1]);
  eb[0] = warp_excl_scan(Es[0], lane, &t0);
  eb[1] = warp_excl_scan(Es[1], lane, &t1) + t0;
  *totE = t0 + t1;
  bad |= totC > kCross;
  const bool irregular = __any_sync(0xffffffffu, bad) != 0;
  __syncwarp();
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const int s = lane + 32 * h;
    if (s < nseg) {
      int* ws = reinterpret_cast<int*>(&tab[s]);
      if (merge[h]) ws[W::MISC] |= kMergeBit;
      ws[W::EBASE] = eb[h];
    }
  }
  __syncwarp();
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const int s = lane + 32 * h;
    if (s < nseg) {
      float t = 0.f;
      for (int u = s + 1; u < nseg; ++u) {
        const int* wu = reinterpret_cast<const int*>(&tab[u]);
        if (!(wu[W::MISC] & kMergeBit)) break;
        t = t + __int_as_float(wu[W::FIRST]);
        const int c01 = wu[W::CNT];
        if ((c01 & 0xffff) + ((unsigned)c01 >> 16) + (DIM > 2 ? wu[W::CNT + 1] & 0xffff : 0) > 0) break;
      }
      reinterpret_cast<int*>(&tab[s])[W::TAIL] = __float_as_int(t);
    }
  }
  __syncwarp();
  return !irregular;
}

template <int DIM, class SM>
__device__ __forceinline__ bool coop_count_row(const SimDev& S, const MixArgs& M, const SimDev* Sg, const GridDF* gdg,
                                               long long row, SM& sm, long long* __restrict__ counts) {
  using W = SegW<DIM>;
  const int lane = threadIdx.x & 31;
  const RowDF& r = M.rdf[row];
  const int nseg = r.nv - 1;
  const PathF64* p64 = M.r64 + row;
  bool irregular = nseg > SM::kCap || nseg < 1 || nseg > M.seg_stride;
  if (!irregular) {
    int totE = 0;
    irregular = !row_table<DIM, SM::kCross>(S, M, Sg, gdg, row, nseg, sm.tab, &totE);

    // 3. exact ties between crossings of different axes
    if (!irregular) {
      bool tie = false, overflow = false;
      tie_pass<DIM>(sm, nseg, lane, Sg, p64, tie, overflow);
      irregular = __any_sync(0xffffffffu, tie || overflow) != 0;
    }
    if (!irregular) {
      if (M.rflag) {
        // lean form: no segment records, the fill rebuilds the table
        if (lane == 0) M.rflag[row] = 0;
      } else {
        SegG<DIM>* dst = (SegG<DIM>*)M.segg + row * (long long)M.seg_stride;
        const int4* src = reinterpret_cast<const int4*>(sm.tab);
        int4* d4 = reinterpret_cast<int4*>(dst);
        for (int q = lane; q < nseg * W::NV; q += 32) d4[q] = src[q];
      }
      if (lane == 0) counts[row] = totE;
      __syncwarp();
      return true;
    }
  }
  __syncwarp();
  return false;  // the caller walks it (count_row_walk)
}

// a row the cooperative count declined: the per-lane walker counts it and
// marks it for the fill
template <int DIM>
__device__ __forceinline__ void count_row_walk(const SimDev* Sg, const MixArgs& M, long long row,
                                               long long* __restrict__ counts) {
  walk_row_lane0<DIM, false>(Sg, M, row, counts, 0, 0, nullptr, nullptr, nullptr, nullptr);
}

// ---------------------------------------------------------------------------
// Fill: one row, the whole warp, from the count's segment records.  Each
// lane takes one crossing: its position in the segment, the voxel it
// enters and the next crossing (own axis' next plane or another axis' first
// plane after it, certified like the position) give one entry, written at
// its CSR position; entry 0 of every segment comes from the segment's lane.
// ---------------------------------------------------------------------------
template <int DIM, class SM>
__device__ __forceinline__ bool coop_fill_row(const SimDev& S, const MixArgs& M, const SimDev* Sg, const GridDF* gdg,
                                              long long row, SM& sm, const long long* __restrict__ row_ptr,
                                              const float* __restrict__ x, int* __restrict__ col,
                                              float* __restrict__ val, float* __restrict__ b) {
  using W = SegW<DIM>;
  const int lane = threadIdx.x & 31;
  const GridDev& g = S.ph.g;
  const RowDF& r = M.rdf[row];
  const int nseg = r.nv - 1;
  const long long rowstart = row_ptr[row], rowend = row_ptr[row + 1];
  const SegG<DIM>* rec;
  bool irregular = nseg > SM::kCap || nseg < 1 || nseg > M.seg_stride;
  if constexpr (SM::kLean) {
    // lean form: the count left only the row flag; the segment table is
    // rebuilt in shared memory by the count's own code (same records)
    rec = sm.tab;
    if (!irregular) irregular = M.rflag[row] != 0;
    if (!irregular) {
      int totE;
      row_table<DIM, SM::kCross>(S, M, Sg, gdg, row, nseg, sm.tab, &totE);
    }
  } else {
    rec = (const SegG<DIM>*)M.segg + row * (long long)M.seg_stride;
    if (!irregular) irregular = (reinterpret_cast<const int*>(rec)[W::MISC] & kRowIrregular) != 0;
  }
  if (!irregular) {
    const int stride[3] = {1, g.n[0], g.n[0] * (DIM > 2 ? g.n[1] : 1)};
    // 1. the row's records, expanded: one segment per lane
    int Cs[2] = {0, 0};
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int s = lane + 32 * h;
      if (s < nseg) {
        const SegR<DIM> R = load_seg<DIM>(rec[s]);
        const int misc = R.w[W::MISC];
        int n[3] = {0, 0, 0}, d[3] = {0, 0, 0};
#pragma unroll
        for (int c = 0; c < DIM; ++c) {
          const float hv = R.f(W::HV + c);
          sm.ax[c][s] = make_float4(R.f(W::PH0 + c), hv, hv >= kFar ? 0.f : __frcp_rn(hv), R.f(W::CB + c));
          n[c] = R.cnt(c);
          d[c] = ((misc >> (4 + c)) & 1) ? -stride[c] : stride[c];
        }
        Cs[h] = n[0] + n[1] + n[2];
        sm.cn[s] = make_int4(n[0], n[1], n[2], R.w[W::COL0]);
        sm.dc[s] = make_int4(d[0], d[1], d[2], R.w[W::EBASE] + ((misc & kMergeBit) ? 0 : 1));
        sm.sf[s] = make_float4(R.f(W::SEND), R.f(W::L), R.f(W::TAIL), R.f(W::FIRST));
        sm.misc[s] = misc;
      }
    }
    __syncwarp();
    const int totC = __reduce_add_sync(0xffffffffu, Cs[0] + Cs[1]);
    if (totC <= SM::kCross) {
      Kahan wk{0.f, 0.f};
      FillOut F;
      F.col = col + rowstart;
      F.val = val + rowstart;
      F.len = (int)(rowend - rowstart);
      F.x = x;
      F.nvox = g.n[0] * g.n[1] * (DIM > 2 ? g.n[2] : 1);
      F.constant = S.md.chord == PCT_CHORD_CONSTANT;
      F.hconst = (float)g.h[0];
      const PathF64* p64 = M.r64 + row;
      bool overflow = false;
      const FillPlan P = fill_plan<DIM>(sm, nseg, lane);
      fill_pass<DIM, 0, -1>(sm, P.tot0, P.tot0, sm.aux, sm.aux, sm.bits, sm.ord, lane, Sg, p64, F, wk, overflow);
      fill_pass<DIM, 1, (DIM > 2 ? 2 : -1)>(sm, P.tot1, P.tot, sm.aux1, sm.aux2, sm.bits1, sm.ord1, lane, Sg, p64, F,
                                              wk, overflow);
      // 2. entry 0 of every segment that does not continue the previous one
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int s = lane + 32 * h;
        if (s < nseg) {
          const int misc = sm.misc[s];
          if ((misc & 3) == kStRegular && !(misc & kMergeBit)) {
            const int4 cn = sm.cn[s];
            const float4 sf = sm.sf[s];
            const float v = sf.w + (cn.x + cn.y + cn.z == 0 ? sf.z : 0.f);
            put_entry(F, sm.dc[s].w - 1, cn.w, v, wk);
          }
        }
      }
      if (!__any_sync(0xffffffffu, overflow)) {
        // the lanes' Kahan partials, summed as double-float
        df sum = two_sum(wk.sum, -wk.comp);
#pragma unroll
        for (int d = 16; d > 0; d >>= 1) {
          df o{__shfl_xor_sync(0xffffffffu, sum.hi, d), __shfl_xor_sync(0xffffffffu, sum.lo, d)};
          sum = df_add(sum, o);
        }
        if (lane == 0) b[row] = (sum.hi + sum.lo) * r.fac;
        // entries written against row_ptr's range: the last segment's first
        // slot in the row plus its entries (each crossing, and its first
        // entry unless it continues the previous segment)
        if (lane == 0) {
          const int misc = sm.misc[nseg - 1];
          const int4 cn = sm.cn[nseg - 1];
          const int first = (misc & kMergeBit) ? 0 : 1;
          const int e = (misc & 3) == kStRegular ? cn.x + cn.y + cn.z + first : 0;
          if (sm.dc[nseg - 1].w - first + e != F.len) note_row_mismatch(S);
        }
        __syncwarp();
        return true;
      }
    }
  }
  __syncwarp();
  return false;  // the caller walks it (fill_row_walk)
}

// a row the cooperative fill declined (marked by the count, beyond the
// layout, or a queue overflow): the per-lane walker writes all of it again
template <int DIM>
__device__ __forceinline__ void fill_row_walk(const SimDev* Sg, const MixArgs& M, long long row,
                                              const long long* __restrict__ row_ptr, const float* __restrict__ x,
                                              int* __restrict__ col, float* __restrict__ val,
                                              float* __restrict__ b) {
  walk_row_lane0<DIM, true>(Sg, M, row, nullptr, row_ptr[row], row_ptr[row + 1], x, col, val, b);
}

}  // namespace pct
