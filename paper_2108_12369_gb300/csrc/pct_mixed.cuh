// pct_mixed.cuh -- FP32 form of the path and traversal with certified
// decisions (PCT_PREC_MIXED).
//
// GB300 runs FP64 at about 1/70 of its FP32 rate.  The FP64 definition
// (pct_device.cuh) is reproduced here with double-float arithmetic: each
// real number is an unevaluated sum hi + lo of two FP32 values (Dekker's
// error-free transformations, with FMA), good to about 2^-44 relative.
//  - Polyline vertices are formed as V = P0 + s D + h10 (m0 - D) + h11 (m1 - D)
//    with D = P1 - P0, the Hermite sum of the definition rearranged into
//    small, well-conditioned terms (the rearrangement is exact in reals).
//  - Every traversal decision (next plane, ties, grid entry / exit, start
//    voxel) compares two crossing parameters sigma.  The double-float values
//    carry a rigorous bound on their distance to the FP64 definition's
//    values; when the difference exceeds the bounds its sign is the FP64
//    sign, otherwise (in practice only at exact ties) both FP64 values are
//    evaluated from the row's FP64 record and compared.
//  - Entry lengths are double-float differences of crossing parameters
//    times the FP32 segment length: accurate to ~1e-9 mm regardless of how
//    shallowly the path crosses a plane.
//  - A segment whose direction sign cannot be certified is walked in FP64.
// Voxel indices and row pointers therefore equal the FP64 definition's.
// Everything is templated on the dimension so that per-axis state lives in
// registers (axis selection uses selects, never dynamic indexing).
#pragma once
#include "pct_device.cuh"

namespace pct {

// ---------------------------------------------------------------------------
// double-float arithmetic (requires that a*b+c is never contracted, which
// the -fmad=false build guarantees; FMAs are explicit)
// ---------------------------------------------------------------------------
struct df {
  float hi, lo;
};

__device__ __forceinline__ df quick_two_sum(float a, float b) {  // |a| >= |b|
  float s = a + b;
  float e = b - (s - a);
  return df{s, e};
}
__device__ __forceinline__ df two_sum(float a, float b) {
  float s = a + b;
  float bb = s - a;
  float e = (a - (s - bb)) + (b - bb);
  return df{s, e};
}
// |error| <= 2^-44 (|a| + |b|)
__device__ __forceinline__ df df_add(df a, df b) {
  df s = two_sum(a.hi, b.hi);
  s.lo = s.lo + (a.lo + b.lo);
  return quick_two_sum(s.hi, s.lo);
}
__device__ __forceinline__ df df_neg(df a) { return df{-a.hi, -a.lo}; }
__device__ __forceinline__ df df_sub(df a, df b) { return df_add(a, df_neg(b)); }
// |error| <= 2^-44 |a b|
__device__ __forceinline__ df df_mul(df a, df b) {
  float p = a.hi * b.hi;
  float e = fmaf(a.hi, b.hi, -p);
  e = fmaf(a.hi, b.lo, e);
  e = fmaf(a.lo, b.hi, e);
  return quick_two_sum(p, e);
}
__device__ __forceinline__ df df_mul_f(df a, float b) {
  float p = a.hi * b;
  float e = fmaf(a.hi, b, -p);
  e = fmaf(a.lo, b, e);
  return quick_two_sum(p, e);
}
// 1 / d by one Newton step from the FP32 reciprocal; |error| <= 2^-43 |1/d|
__device__ __forceinline__ df df_recip(df d) {
  float r = __frcp_rn(d.hi);
  df dr = df_mul_f(d, r);                  // ~ 1
  df e = df_sub(df{1.0f, 0.0f}, dr);       // 1 - d r, small
  return df_add(df{r, 0.0f}, df_mul_f(e, r));
}
__device__ __forceinline__ float df_to_f(df a) { return a.hi + a.lo; }

// FP64 -> double-float with integer operations only (no FP64 pipe):
// hi = RN32(d), lo = RN32(d - hi).  Values below 2^-74 in magnitude lose lo
// (error below 2^-98), values below 2^-103 become 0.
__device__ __forceinline__ df split_d(double d) {
  unsigned long long b = (unsigned long long)__double_as_longlong(d);
  int e = (int)((b >> 52) & 0x7ff);
  if (e < 920) return df{0.0f, 0.0f};
  bool neg = (b >> 63) != 0;
  unsigned long long mant = (b & 0xFFFFFFFFFFFFFULL) | (1ULL << 52);
  unsigned long long top = mant >> 29;
  unsigned long long rem = mant & ((1ULL << 29) - 1);
  if (rem > (1ULL << 28) || (rem == (1ULL << 28) && (top & 1ULL))) top += 1;
  long long diff = (long long)mant - (long long)(top << 29);  // |diff| <= 2^28
  // scale factors 2^(e - 1046) and 2^(e - 1075) as floats
  float s_hi = __int_as_float((e - 1046 + 127) << 23);
  float hi = (float)top * s_hi;
  float lo = 0.0f;
  if (e >= 949) lo = (float)diff * __int_as_float((e - 1075 + 127) << 23);
  if (neg) {
    hi = -hi;
    lo = -lo;
  }
  return df{hi, lo};
}

constexpr float kEps44 = 5.684342e-14f;  // 2^-44

// ---------------------------------------------------------------------------
// Row records.  The count kernel forms the FP64 path (the definition) once
// per proton and leaves it, plus a double-float copy of the quantities the
// vertices are built from, for the fill kernel.
// ---------------------------------------------------------------------------
struct alignas(16) RowDF {
  df P0[3];  // kind 0: A
  df Dl[3];  // P1 - P0
  df u0[3];  // m0 - (P1 - P0)
  df u1[3];  // m1 - (P1 - P0)
  df g0[3];
  df g1[3];
  int kind, nv;
  float fac;  // noise factor 1 + noise_rel z (1 without noise)
  float mag;  // max |coordinate| of the polyline's vertices (for bounds)
};

// the Hermite basis at s = j / K as double-float: (s, h10, h11)
struct alignas(16) BasisDF {
  df s, h10, h11;
  df pad;
};

struct GridDF {
  df o[3], h[3];
  float of[3], rh[3];
};

template <int DIM, class T>
__device__ __forceinline__ T pick(const T (&v)[3], int ax) {
  T r = v[0];
#pragma unroll
  for (int a = 1; a < DIM; ++a)
    if (ax == a) r = v[a];
  return r;
}

template <int DIM>
__device__ __forceinline__ void make_rowdf(const PathF64& p, double R, float fac, RowDF& r) {
  r.kind = p.kind;
  r.nv = p.nv;
  r.fac = fac;
  float mag = 0.f;
#pragma unroll
  for (int a = 0; a < DIM; ++a) {
    if (p.kind == 0) {
      r.P0[a] = split_d(p.A[a]);
      r.g0[a] = split_d(p.g0[a]);
      mag = fmaxf(mag, fabsf((float)p.A[a]) + (float)R * fabsf((float)p.g0[a]));
    } else {
      double D = p.P1[a] - p.P0[a];
      r.P0[a] = split_d(p.P0[a]);
      r.Dl[a] = split_d(D);
      r.g0[a] = split_d(p.g0[a]);
      r.g1[a] = split_d(p.g1[a]);
      if (p.kind == 2) {
        r.u0[a] = split_d(p.m0[a] - D);
        r.u1[a] = split_d(p.m1[a] - D);
      }
      float m = fmaxf(fabsf((float)p.P0[a]) + (float)R * fabsf((float)p.g0[a]),
                      fabsf((float)p.P1[a]) + (float)R * fabsf((float)p.g1[a]));
      if (p.kind == 2) m = fmaxf(m, fabsf((float)p.P0[a]) + fabsf((float)D) + fabsf((float)p.m0[a]) +
                                        fabsf((float)p.m1[a]));
      mag = fmaxf(mag, m);
    }
  }
  r.mag = mag;
}

// vertex q of the polyline in double-float (within 2^-40 mag of the FP64 vertex)
template <int DIM>
__device__ __forceinline__ void vertex_df(const RowDF& r, const BasisDF* tab, df Rdf, int q, df (&V)[3]) {
  if (r.kind == 0) {
    df s = (q == 0) ? df_neg(Rdf) : Rdf;
#pragma unroll
    for (int a = 0; a < DIM; ++a) V[a] = df_add(r.P0[a], df_mul(s, r.g0[a]));
    return;
  }
  if (q == 0) {
#pragma unroll
    for (int a = 0; a < DIM; ++a) V[a] = df_sub(r.P0[a], df_mul(Rdf, r.g0[a]));
  } else if (q == 1) {
#pragma unroll
    for (int a = 0; a < DIM; ++a) V[a] = r.P0[a];
  } else if (q == r.nv - 2) {
#pragma unroll
    for (int a = 0; a < DIM; ++a) V[a] = df_add(r.P0[a], r.Dl[a]);
  } else if (q == r.nv - 1) {
#pragma unroll
    for (int a = 0; a < DIM; ++a) V[a] = df_add(df_add(r.P0[a], r.Dl[a]), df_mul(Rdf, r.g1[a]));
  } else {
    BasisDF B = tab[q - 1];
#pragma unroll
    for (int a = 0; a < DIM; ++a)
      V[a] = df_add(df_add(r.P0[a], df_mul(B.s, r.Dl[a])),
                    df_add(df_mul(B.h10, r.u0[a]), df_mul(B.h11, r.u1[a])));
  }
}

// ---------------------------------------------------------------------------
// One segment in double-float with certified decisions
// ---------------------------------------------------------------------------
// An event is plane k of axis ax (0..2), or ax = -1 for the constant k (0 or 1).
struct Ev {
  int ax, k;
};

struct SegDF {
  df P[3];       // start vertex
  df inv[3];     // 1 / D
  df dl[3];      // h / D
  df sn[3];      // sigma of each axis' next plane
  float E0[3], E1[3];  // bound on |sigma~ - sigma| = E0 + E1 |sigma|
  float L;       // |Q - P|
  int idx[3], kn[3], step[3];
  Ev in, out;
  df s_in, s_out;
  // exact data, built on demand
  bool have_ex;
  double ex_dl[3], ex_s0[3];
};

template <int DIM>
__device__ __forceinline__ df plane_df(const GridDF& gd, int a, int k) {
  return df_add(gd.o[a], df_mul_f(gd.h[a], (float)k));
}

// sigma of plane k of axis a: (X_k - P_a) / D_a
template <int DIM>
__device__ __forceinline__ df sigma_df(const SegDF& s, const GridDF& gd, int a, int k) {
  return df_mul(df_sub(plane_df<DIM>(gd, a, k), s.P[a]), s.inv[a]);
}

template <int DIM>
__device__ __forceinline__ df ev_df(const SegDF& s, const GridDF& gd, Ev e) {
  if (e.ax < 0) return df{(float)e.k, 0.0f};
  df r = sigma_df<DIM>(s, gd, 0, e.k);
#pragma unroll
  for (int a = 1; a < DIM; ++a)
    if (e.ax == a) r = sigma_df<DIM>(s, gd, a, e.k);
  return r;
}

template <int DIM, class Ends>
__device__ __forceinline__ void make_exact(const GridDev& g, SegDF& s, const Ends& ends) {
  if (s.have_ex) return;
  double P[3], Q[3];
  ends(P, Q);
#pragma unroll
  for (int a = 0; a < DIM; ++a) {
    double D = Q[a] - P[a];
    double inv = 1.0 / D;
    s.ex_dl[a] = g.h[a] * inv;
    s.ex_s0[a] = (g.o[a] - P[a]) * inv;
  }
  s.have_ex = true;
}

template <int DIM>
__device__ __forceinline__ double ev_f64(const SegDF& s, Ev e) {
  return e.ax < 0 ? (double)e.k : fma((double)e.k, pick<DIM>(s.ex_dl, e.ax), pick<DIM>(s.ex_s0, e.ax));
}

// exact sign of sigma(e1) - sigma(e2) given their double-float values
template <int DIM, class Ends>
__device__ __forceinline__ int cmp_vals(const GridDev& g, SegDF& s, Ev e1, df v1, Ev e2, df v2, const Ends& ends) {
  if (e1.ax == e2.ax && e1.k == e2.k) return 0;
  if (e1.ax < 0 && e2.ax < 0) return e1.k < e2.k ? -1 : (e1.k > e2.k ? 1 : 0);
  float d = (v1.hi - v2.hi) + (v1.lo - v2.lo);
  float m = (e1.ax < 0 ? 0.f : fmaf(pick<DIM>(s.E1, e1.ax), fabsf(v1.hi), pick<DIM>(s.E0, e1.ax))) +
            (e2.ax < 0 ? 0.f : fmaf(pick<DIM>(s.E1, e2.ax), fabsf(v2.hi), pick<DIM>(s.E0, e2.ax)));
  if (d < -m) return -1;
  if (d > m) return 1;
  make_exact<DIM>(g, s, ends);
  double x1 = ev_f64<DIM>(s, e1), x2 = ev_f64<DIM>(s, e2);
  return x1 < x2 ? -1 : (x1 > x2 ? 1 : 0);
}

template <int DIM, class Ends>
__device__ __forceinline__ int cmp_ev(const GridDev& g, const GridDF& gd, SegDF& s, Ev e1, Ev e2, const Ends& ends) {
  return cmp_vals<DIM>(g, s, e1, ev_df<DIM>(s, gd, e1), e2, ev_df<DIM>(s, gd, e2), ends);
}

// Set-up.  Returns 0: the segment misses the grid; 1: ready for walk_df;
// 2: the sign of some axis' extent cannot be certified (walk it in FP64).
template <int DIM, class Ends>
__device__ __forceinline__ int seg_setup_df(const GridDev& g, const GridDF& gd, const df (&P)[3], const df (&Q)[3],
                                            float mag, SegDF& s, const Ends& ends) {
  s.have_ex = false;
  float L2 = 0.f;
  // |V~ - V| <= eV for every vertex (double-float vertex formation, FP64 rounding)
  const float eV = 64.f * kEps44 * mag;
#pragma unroll
  for (int a = 0; a < DIM; ++a) {
    df D = df_sub(Q[a], P[a]);
    float Dh = df_to_f(D);
    if (!(fabsf(Dh) > 4.f * eV + 4.f * kEps44 * fabsf(Dh))) return 2;
    L2 = fmaf(Dh, Dh, L2);
    s.P[a] = P[a];
    s.inv[a] = df_recip(D);
    s.dl[a] = df_mul(gd.h[a], s.inv[a]);
    s.step[a] = Dh > 0.f ? 1 : -1;
    // |sigma~ - sigma| for planes 0..n_a, with X = o + k h:
    //   double-float evaluation  < 2^-42 (|o| + n h + |P|) / |D| + 2^-42 |sigma|
    //   vertices within eV       < eV / |D| + |sigma| 2 eV / |D|
    //   D's own evaluation       < |sigma| 2^-43 mag / |D|
    //   FP64 definition          < 2^-50 (n h + |o - P|) / |D| + 2^-53 |sigma|
    // all times 4 (written as E0 + E1 |sigma|), plus the accumulated error of
    // the incremental steps sigma += dl (< 2^-44 (|sigma| + |dl|) each).
    float mx = (float)g.n[a] * fabsf(gd.h[a].hi) + fabsf(gd.o[a].hi) + fabsf(P[a].hi);
    s.E0[a] = 4.f * (16.f * kEps44 * mx + eV) / fabsf(Dh);
    s.E1[a] = 4.f * (16.f * kEps44 + (2.f * eV + 2.f * kEps44 * mag) / fabsf(Dh));
    s.E0[a] += (float)(g.n[a] + 2) * 2.f * kEps44 * (fabsf(s.dl[a].hi) + 2.f);
  }
  s.L = sqrtf(L2);
  // entry: the largest of 0 and every axis' first plane; exit: the smallest
  // of 1 and every axis' last plane
  s.in = Ev{-1, 0};
  s.out = Ev{-1, 1};
  df vin{0.f, 0.f}, vout{1.f, 0.f};
#pragma unroll
  for (int a = 0; a < DIM; ++a) {
    Ev lo{a, s.step[a] > 0 ? 0 : g.n[a]};
    Ev hi{a, s.step[a] > 0 ? g.n[a] : 0};
    df vlo = sigma_df<DIM>(s, gd, a, lo.k), vhi = sigma_df<DIM>(s, gd, a, hi.k);
    if (cmp_vals<DIM>(g, s, lo, vlo, s.in, vin, ends) > 0) {
      s.in = lo;
      vin = vlo;
    }
    if (cmp_vals<DIM>(g, s, hi, vhi, s.out, vout, ends) < 0) {
      s.out = hi;
      vout = vhi;
    }
  }
  if (cmp_vals<DIM>(g, s, s.in, vin, s.out, vout, ends) >= 0) return 0;
  s.s_in = vin;
  s.s_out = vout;
  // start voxel: (planes with sigma <= s_in) - 1, or n - that count
  const float sin_f = df_to_f(vin);
#pragma unroll
  for (int a = 0; a < DIM; ++a) {
    const int n = g.n[a];
    int i;
    if (s.in.ax == a) {
      i = s.step[a] > 0 ? 0 : n - 1;
    } else {
      df x = df_add(P[a], df_mul_f(df_sub(Q[a], P[a]), sin_f));
      float u = floorf((df_to_f(x) - gd.of[a]) * gd.rh[a]);
      i = (u < 0.f) ? 0 : (u > (float)(n - 1) ? n - 1 : (int)u);
      if (s.step[a] > 0) {
        while (i + 1 <= n - 1 && cmp_vals<DIM>(g, s, Ev{a, i + 1}, sigma_df<DIM>(s, gd, a, i + 1), s.in, vin, ends) <= 0) ++i;
        while (i > 0 && cmp_vals<DIM>(g, s, Ev{a, i}, sigma_df<DIM>(s, gd, a, i), s.in, vin, ends) > 0) --i;
      } else {
        while (i > 0 && cmp_vals<DIM>(g, s, Ev{a, i}, sigma_df<DIM>(s, gd, a, i), s.in, vin, ends) <= 0) --i;
        while (i < n - 1 && cmp_vals<DIM>(g, s, Ev{a, i + 1}, sigma_df<DIM>(s, gd, a, i + 1), s.in, vin, ends) > 0) ++i;
      }
    }
    s.idx[a] = i;
    s.kn[a] = s.step[a] > 0 ? i + 1 : i;
    s.sn[a] = sigma_df<DIM>(s, gd, a, s.kn[a]);
  }
  return 1;
}

// Walk a set-up segment, emitting (voxel, length) in path order.
template <int DIM, bool kLengths, class Merge, class Sink, class Ends>
__device__ __forceinline__ void walk_df(const GridDev& g, SegDF& s, Merge& mg, Sink& sink, const Ends& ends) {
  Ev cur = s.in;
  df vcur = s.s_in;
  const int stride1 = g.n[0], stride2 = g.n[0] * g.n[1];
  int col = s.idx[0] + stride1 * s.idx[1] + (DIM == 3 ? stride2 * s.idx[2] : 0);
  int guard = g.n[0] + g.n[1] + (DIM == 3 ? g.n[2] : 0) + 2;
  while (guard-- > 0) {
    // axis (or axes, on an exact tie) whose next plane comes first
    int m = 0;
    unsigned mask = 1u;
    df vm = s.sn[0];
#pragma unroll
    for (int a = 1; a < DIM; ++a) {
      int r = cmp_vals<DIM>(g, s, Ev{a, s.kn[a]}, s.sn[a], Ev{m, pick<DIM>(s.kn, m)}, vm, ends);
      if (r < 0) {
        m = a;
        mask = 1u << a;
        vm = s.sn[a];
      } else if (r == 0) {
        mask |= 1u << a;
      }
    }
    const int km = pick<DIM>(s.kn, m);
    bool final;
    if (s.out.ax >= 0 && (mask >> s.out.ax & 1u) && pick<DIM>(s.kn, s.out.ax) == s.out.k)
      final = true;  // the step crosses the exit plane itself
    else
      final = cmp_vals<DIM>(g, s, Ev{m, km}, vm, s.out, s.s_out, ends) >= 0;
    float len = 0.f;
    if (kLengths) {
      df vend = final ? s.s_out : vm;
      len = fmaxf(df_to_f(df_sub(vend, vcur)), 0.f) * s.L;
    }
    mg.emit(col, len, sink);
    if (final) break;
    cur = Ev{m, km};
    vcur = vm;
#pragma unroll
    for (int a = 0; a < DIM; ++a) {
      if (mask >> a & 1u) {
        s.idx[a] += s.step[a];
        s.kn[a] += s.step[a];
        col += s.step[a] * (a == 0 ? 1 : (a == 1 ? stride1 : stride2));
        s.sn[a] = df_add(s.sn[a], s.step[a] > 0 ? s.dl[a] : df_neg(s.dl[a]));
      }
    }
  }
}

}  // namespace pct
