// pct_api.cu -- the C ABI of include/pct.h: argument checks, workspace
// layout, host-side tables (angle cos/sin from the host libm, Hermite basis)
// and the launch sequences.  Host code here is compiled without FMA
// contraction so that its tables equal the definition bit for bit.
#include <cmath>
#include <cstdarg>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include <algorithm>
#include <map>
#include <mutex>

#include "pct_kernels.cuh"
#include "pct_mixed.cuh"

using namespace pct;

namespace {

thread_local std::string g_err;

pct_status fail(pct_status st, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_err = buf;
  return st;
}

pct_status cuda_check(const char* what) {
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail(PCT_ECUDA, "%s: %s", what, cudaGetErrorString(e));
  return PCT_OK;
}

bool finite_pos(double v) { return std::isfinite(v) && v > 0.0; }

size_t align256(size_t v) { return (v + 255) & ~(size_t)255; }

}  // namespace

struct pct_phantom {
  pct_phantom_desc desc;
  pct_region regions[PCT_MAX_REGIONS];
  PhantomDev dev;
  long long nvox;
};

// ---------------------------------------------------------------------------
// phantom
// ---------------------------------------------------------------------------
extern "C" pct_status pct_phantom_create(const pct_phantom_desc* d, pct_phantom** out) {
  if (!d || !out) return fail(PCT_EINVAL, "pct_phantom_create: NULL argument");
  *out = nullptr;
  if (d->dim != 2 && d->dim != 3) return fail(PCT_EINVAL, "dim must be 2 or 3 (got %d)", d->dim);
  if (d->kind != PCT_ELLIPSOID && d->kind != PCT_EXTRUDED) return fail(PCT_EINVAL, "bad phantom kind %d", d->kind);
  if (d->raster != PCT_RASTER_CENTER && d->raster != PCT_RASTER_CORNER && d->raster != PCT_RASTER_AREA)
    return fail(PCT_EINVAL, "bad raster option %d", d->raster);
  if (d->raster == PCT_RASTER_AREA && (d->area_samples < 1 || d->area_samples > 64))
    return fail(PCT_EINVAL, "area_samples = %d outside 1..64", d->area_samples);
  long long nvox = 1;
  for (int a = 0; a < d->dim; ++a) {
    if (d->n[a] < 1) return fail(PCT_EINVAL, "n[%d] = %d must be >= 1", a, d->n[a]);
    if (!finite_pos(d->h[a])) return fail(PCT_EINVAL, "h[%d] must be finite and > 0", a);
    nvox *= d->n[a];
    if (nvox >= (1LL << 31)) return fail(PCT_EINVAL, "grid has >= 2^31 voxels");
  }
  if (d->n_regions < 1 || d->n_regions > PCT_MAX_REGIONS)
    return fail(PCT_EINVAL, "n_regions = %d outside 1..%d", d->n_regions, PCT_MAX_REGIONS);
  if (!d->regions) return fail(PCT_EINVAL, "regions is NULL");
  for (int r = 0; r < d->n_regions; ++r) {
    const pct_region& R = d->regions[r];
    int axes = (d->dim == 3) ? 3 : 2;
    for (int a = 0; a < axes; ++a) {
      if (!finite_pos(R.a[a])) return fail(PCT_EINVAL, "region %d semi-axis %d must be finite and > 0", r, a);
      if (!std::isfinite(R.c[a])) return fail(PCT_EINVAL, "region %d centre must be finite", r);
    }
    if (!std::isfinite(R.rsp)) return fail(PCT_EINVAL, "region %d RSP must be finite", r);
  }
  pct_phantom* ph = new (std::nothrow) pct_phantom;
  if (!ph) return fail(PCT_ENOMEM, "out of host memory");
  memset(ph, 0, sizeof(*ph));
  ph->desc = *d;
  memcpy(ph->regions, d->regions, sizeof(pct_region) * d->n_regions);
  ph->desc.regions = ph->regions;
  for (int a = d->dim; a < 3; ++a) {
    ph->desc.n[a] = 1;
    ph->desc.h[a] = 1.0;
  }
  ph->nvox = nvox;
  PhantomDev& pd = ph->dev;
  pd.g.dim = d->dim;
  for (int a = 0; a < 3; ++a) {
    pd.g.n[a] = ph->desc.n[a];
    pd.g.h[a] = ph->desc.h[a];
    pd.g.o[a] = -0.5 * ((double)pd.g.n[a] * pd.g.h[a]);
  }
  pd.kind = d->kind;
  pd.raster = d->raster;
  pd.area_s = d->raster == PCT_RASTER_AREA ? d->area_samples : 1;
  pd.n_regions = d->n_regions;
  for (int r = 0; r < d->n_regions; ++r) {
    for (int a = 0; a < 3; ++a) {
      pd.c[r][a] = ph->regions[r].c[a];
      double ax = (a < d->dim) ? ph->regions[r].a[a] : 1.0;
      if (!(ax > 0.0)) ax = 1.0;
      pd.a[r][a] = ax;
      pd.ra[r][a] = 1.0 / ax;
    }
    pd.rsp[r] = ph->regions[r].rsp;
  }
  *out = ph;
  return PCT_OK;
}

extern "C" pct_status pct_phantom_destroy(pct_phantom* ph) {
  delete ph;
  return PCT_OK;
}

extern "C" int64_t pct_phantom_nvox(const pct_phantom* ph) { return ph ? ph->nvox : -1; }

extern "C" pct_status pct_phantom_rasterize(const pct_phantom* ph, float* x, void* stream) {
  if (!ph || !x) return fail(PCT_EINVAL, "pct_phantom_rasterize: NULL argument");
  launch_raster(ph->dev, x, ph->nvox, (cudaStream_t)stream);
  return cuda_check("raster launch");
}

// ---------------------------------------------------------------------------
// geometry, workspace, tables
// ---------------------------------------------------------------------------
namespace {

struct Layout {
  size_t status, cs, basis, basis32, partial, args, rec, total;
  long long rows;
  int K;
};

pct_status check_geometry(const pct_phantom* ph, const pct_geometry* g, int precision) {
  if (!ph || !g) return fail(PCT_EINVAL, "NULL phantom or geometry");
  if (precision != PCT_PREC_MIXED && precision != PCT_PREC_F64 && precision != PCT_PREC_MIXED_LEAN)
    return fail(PCT_EINVAL, "bad precision %d", precision);
  if (g->n_angles < 0 || g->paths_per_angle < 0) return fail(PCT_EINVAL, "negative angle or path count");
  if (g->n_angles > 0 && !g->angles_rad) return fail(PCT_EINVAL, "angles_rad is NULL");
  for (int k = 0; k < g->n_angles; ++k)
    if (!std::isfinite(g->angles_rad[k])) return fail(PCT_EINVAL, "angle %d is not finite", k);
  long long rows = (long long)g->n_angles * g->paths_per_angle;
  if (g->paths_per_angle > 0 && rows / g->paths_per_angle != g->n_angles) return fail(PCT_EINVAL, "row count overflows");
  if (rows > (1LL << 40)) return fail(PCT_EINVAL, "more than 2^40 rows");
  if (g->first_row < 0 || g->first_row > (1LL << 62) - rows)
    return fail(PCT_EINVAL, "first_row = %lld outside [0, 2^62 - rows]", (long long)g->first_row);
  const pct_path_model& m = g->model;
  if (m.model < PCT_PATH_STRAIGHT || m.model > PCT_PATH_SPLINE) return fail(PCT_EINVAL, "bad path model %d", m.model);
  if (m.chord != PCT_CHORD_EXACT && m.chord != PCT_CHORD_CONSTANT) return fail(PCT_EINVAL, "bad chord option %d", m.chord);
  if (m.noise != PCT_NOISE_NONE && m.noise != PCT_NOISE_GAUSS_REL) return fail(PCT_EINVAL, "bad noise option %d", m.noise);
  if (m.model == PCT_PATH_SPLINE && (m.spline_segments < 1 || m.spline_segments > PCT_MAX_SPLINE_SEGMENTS))
    return fail(PCT_EINVAL, "spline_segments = %d outside 1..%d", m.spline_segments, PCT_MAX_SPLINE_SEGMENTS);
  for (int q = 0; q < 2; ++q)
    if (!std::isfinite(m.t_range[q]) || !std::isfinite(m.v_range[q])) return fail(PCT_EINVAL, "entry ranges must be finite");
  if (m.t_range[0] > m.t_range[1] || m.v_range[0] > m.v_range[1]) return fail(PCT_EINVAL, "entry range lo > hi");
  const double sig[4] = {m.sigma_lat, m.sigma_in, m.sigma_out, m.noise_rel};
  for (double s : sig)
    if (!std::isfinite(s) || s < 0.0) return fail(PCT_EINVAL, "sigmas must be finite and >= 0");
  if (!std::isfinite(m.rho) || m.rho < -1.0 || m.rho > 1.0) return fail(PCT_EINVAL, "rho must lie in [-1, 1]");
  if (m.mcs != PCT_MCS_FIXED && m.mcs != PCT_MCS_HIGHLAND) return fail(PCT_EINVAL, "bad mcs option %d", m.mcs);
  if (m.mcs == PCT_MCS_HIGHLAND && !(finite_pos(m.beam_mev) && finite_pos(m.x0_mm)))
    return fail(PCT_EINVAL, "Highland widths need beam_mev > 0 and x0_mm > 0");
  return PCT_OK;
}

// rec_rows >= 0 sizes the row records for that many rows (projector chunks)
Layout layout_of(const pct_phantom* ph, const pct_geometry* g, int precision, long long rec_rows = -1) {
  Layout L;
  L.rows = (long long)g->n_angles * g->paths_per_angle;
  L.K = (g->model.model == PCT_PATH_SPLINE) ? g->model.spline_segments : 1;
  size_t off = 0;
  L.status = off;  // first: the same place in the workspace for every geometry
  off = align256(off + 2 * sizeof(unsigned long long));
  L.cs = off;
  off = align256(off + sizeof(double2) * (size_t)(g->n_angles > 0 ? g->n_angles : 1));
  L.basis = off;
  off = align256(off + sizeof(Basis4) * (size_t)(L.K + 1));
  L.basis32 = off;
  off = align256(off + basis_df_bytes(L.K + 1));
  L.partial = off;
  off = align256(off + sizeof(long long) * (size_t)scan_partials_needed(L.rows));
  L.args = off;
  off = align256(off + mixed_args_bytes());
  L.rec = off;
  if (precision != PCT_PREC_F64)
    off = align256(off + mixed_record_size(rec_rows >= 0 ? rec_rows : L.rows, ph ? ph->desc.dim : 3, g->model.model,
                                           g->model.spline_segments, precision == PCT_PREC_MIXED_LEAN));
  L.total = off;
  return L;
}

// the simulation's kernel arguments; uploads the angle and basis tables
pct_status make_sim(const pct_phantom* ph, const pct_geometry* g, int precision, void* ws, size_t ws_bytes,
                    cudaStream_t st, SimDev& S, Layout& L, long long rec_rows = -1) {
  pct_status rc = check_geometry(ph, g, precision);
  if (rc != PCT_OK) return rc;
  L = layout_of(ph, g, precision, rec_rows);
  if (!ws || ws_bytes < L.total)
    return fail(PCT_ENOMEM, "workspace of %zu bytes is smaller than the %zu needed", ws_bytes, L.total);
  memset(&S, 0, sizeof(S));
  S.ph = ph->dev;
  const pct_path_model& m = g->model;
  S.md.model = m.model;
  S.md.chord = m.chord;
  S.md.K = L.K;
  S.md.noise = m.noise;
  S.md.t_lo = m.t_range[0];
  S.md.t_hi = m.t_range[1];
  S.md.v_lo = m.v_range[0];
  S.md.v_hi = m.v_range[1];
  S.md.t_span = m.t_range[1] - m.t_range[0];
  S.md.v_span = m.v_range[1] - m.v_range[0];
  S.md.sigma_lat = m.sigma_lat;
  S.md.sigma_in = m.sigma_in;
  S.md.sigma_out = m.sigma_out;
  S.md.rho = m.rho;
  S.md.rho_c = std::sqrt(1.0 - m.rho * m.rho);
  S.md.noise_rel = m.noise_rel;
  // Highland / PDG constants (host FP64, the expressions of the definition):
  // E = T + m_p, (pc)^2 = T (T + 2 m_p), beta c p = (pc)^2 / E, beta^2 = (pc)^2 / E^2
  S.md.mcs = m.mcs;
  if (m.mcs == PCT_MCS_HIGHLAND) {
    const double mp = 938.272088;  // proton mass, MeV (PDG)
    const double E = m.beam_mev + mp;
    const double pc2 = m.beam_mev * (m.beam_mev + 2.0 * mp);
    S.md.hl_k = 13.6 / (pc2 / E);
    S.md.hl_x0 = m.x0_mm;
    S.md.hl_beta2 = pc2 / (E * E);
    S.md.hl_s3 = 1.0 / std::sqrt(3.0);
    S.md.hl_rho = 0.5 * std::sqrt(3.0);
    S.md.hl_rho_c = std::sqrt(1.0 - S.md.hl_rho * S.md.hl_rho);
  }
  S.n_angles = g->n_angles;
  S.P = g->paths_per_angle;
  S.seed = g->seed;
  S.stream = g->stream_id;
  S.first_row = g->first_row;
  double diag2 = 0.0;
  for (int a = 0; a < ph->dev.g.dim; ++a) {
    double w = (double)ph->dev.g.n[a] * ph->dev.g.h[a];
    diag2 = diag2 + w * w;
  }
  S.R = 2.0 * std::sqrt(diag2);
  char* base = (char*)ws;
  S.cs = (const double2*)(base + L.cs);
  S.basis = (const Basis4*)(base + L.basis);
  S.status = (unsigned long long*)(base + L.status);

  std::vector<double2> cs((size_t)(g->n_angles > 0 ? g->n_angles : 1));
  for (int k = 0; k < g->n_angles; ++k) {
    cs[k].x = std::cos(g->angles_rad[k]);
    cs[k].y = std::sin(g->angles_rad[k]);
  }
  std::vector<Basis4> bs((size_t)L.K + 1);
  for (int j = 0; j <= L.K; ++j) {
    double sp = (double)j / (double)L.K;
    double s2 = sp * sp;
    double s3 = s2 * sp;
    bs[j].h00 = (2.0 * s3 - 3.0 * s2) + 1.0;
    bs[j].h10 = (s3 - 2.0 * s2) + sp;
    bs[j].h01 = 3.0 * s2 - 2.0 * s3;
    bs[j].h11 = s3 - s2;
  }
  std::vector<double> sj((size_t)L.K + 1), h10((size_t)L.K + 1), h11((size_t)L.K + 1);
  for (int j = 0; j <= L.K; ++j) {
    sj[j] = (double)j / (double)L.K;
    h10[j] = bs[j].h10;
    h11[j] = bs[j].h11;
  }
  std::vector<char> bf(basis_df_bytes(L.K + 1));
  fill_basis_df(sj.data(), h10.data(), h11.data(), L.K + 1, bf.data());
  // the host vectors are pageable: the copies return once they are staged
  if (cudaMemcpyAsync(base + L.cs, cs.data(), sizeof(double2) * cs.size(), cudaMemcpyHostToDevice, st) != cudaSuccess ||
      cudaMemcpyAsync(base + L.basis, bs.data(), sizeof(Basis4) * bs.size(), cudaMemcpyHostToDevice, st) != cudaSuccess ||
      cudaMemcpyAsync(base + L.basis32, bf.data(), bf.size(), cudaMemcpyHostToDevice, st) != cudaSuccess)
    return cuda_check("table upload");
  return PCT_OK;
}

}  // namespace

extern "C" pct_status pct_simulate_workspace_size(const pct_phantom* ph, const pct_geometry* g, int32_t precision,
                                                  size_t* bytes) {
  if (!bytes) return fail(PCT_EINVAL, "bytes is NULL");
  pct_status rc = check_geometry(ph, g, precision);
  if (rc != PCT_OK) return rc;
  *bytes = layout_of(ph, g, precision).total;
  return PCT_OK;
}

extern "C" pct_status pct_simulate_count(const pct_phantom* ph, const pct_geometry* g, int32_t precision, void* ws,
                                         size_t ws_bytes, int64_t* row_ptr, void* stream) {
  cudaStream_t st = (cudaStream_t)stream;
  SimDev S;
  Layout L;
  pct_status rc = make_sim(ph, g, precision, ws, ws_bytes, st, S, L);
  if (rc != PCT_OK) return rc;
  if (!row_ptr) return fail(PCT_EINVAL, "row_ptr is NULL");
  long long* rp = (long long*)row_ptr;
  if (cudaMemsetAsync(S.status, 0, sizeof(unsigned long long), st) != cudaSuccess) return cuda_check("count");
  if (precision == PCT_PREC_F64)
    launch_count_f64(S, 0, L.rows, rp + 1, st);
  else
    launch_count_mixed(S, (const char*)ws + L.basis32, L.rows, (char*)ws + L.rec, rp + 1, (char*)ws + L.args, st,
                       precision == PCT_PREC_MIXED_LEAN);
  if ((rc = cuda_check("count launch")) != PCT_OK) return rc;
  launch_scan_rowptr(rp, L.rows, (long long*)((char*)ws + L.partial), st);
  return cuda_check("scan launch");
}

extern "C" pct_status pct_simulate_fill(const pct_phantom* ph, const pct_geometry* g, int32_t precision, void* ws,
                                        size_t ws_bytes, const int64_t* row_ptr, const float* x, int32_t* col,
                                        float* val, float* b, void* stream) {
  cudaStream_t st = (cudaStream_t)stream;
  SimDev S;
  Layout L;
  pct_status rc = make_sim(ph, g, precision, ws, ws_bytes, st, S, L);
  if (rc != PCT_OK) return rc;
  if (L.rows > 0 && (!row_ptr || !x || !b)) return fail(PCT_EINVAL, "NULL row_ptr, x_true or b");
  const long long* rp = (const long long*)row_ptr;
  if (precision == PCT_PREC_F64)
    launch_fill_f64(S, 0, L.rows, rp, x, (int*)col, val, b, st);
  else
    launch_fill_mixed(S, (const char*)ws + L.basis32, L.rows, (const char*)ws + L.rec, rp, x, (int*)col, val, b,
                      (char*)ws + L.args, st, 0, -1, 0, true, precision == PCT_PREC_MIXED_LEAN);
  return cuda_check("fill launch");
}

namespace {

// rows whose fill disagreed with row_ptr since the last count (synchronises st)
pct_status read_mismatch(const void* ws, cudaStream_t st, unsigned long long* rows) {
  *rows = 0;
  if (cudaMemcpyAsync(rows, ws, sizeof(unsigned long long), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return cuda_check("reading the fill's row check");
  return PCT_OK;
}

pct_status mismatch_error(const char* what, unsigned long long rows) {
  return fail(PCT_EINVAL,
              "%s: %llu rows received a different number of entries than row_ptr gives them (row_ptr is not the "
              "count of these arguments and workspace)",
              what, rows);
}

// Device -> host streaming of filled rows: the rows are filled block by
// block into two device staging halves; a block's copies to the host (col
// on one stream, val and b on another: two copy engines move the block at
// once) overlap the fill of the next block, and a half is refilled only
// after both its copies.  Blocks continue across calls of rows(), so one
// HostStream serves the blocks of several simulations in turn.
struct HostStream {
  cudaStream_t st = nullptr, cs[2] = {nullptr, nullptr};
  cudaEvent_t ev_fill[2] = {nullptr, nullptr}, ev_copy[2][2] = {{nullptr, nullptr}, {nullptr, nullptr}};
  char* base = nullptr;
  long long half = 0, E = 0, Rb = 0, k = 0;  // k: staging blocks issued so far (half k & 1 next)
  bool ok = true;

  // each half: E col entries, E val entries, E / 16 b values (E a multiple of 64)
  pct_status init(cudaStream_t s, void* staging, size_t staging_bytes) {
    st = s;
    base = (char*)staging;
    half = (long long)(staging_bytes / 2) & ~255LL;
    E = (long long)((double)half / 8.25) & ~63LL;
    Rb = E / 16;
    if (E < 64) return fail(PCT_EINVAL, "staging buffer of %zu bytes is too small", staging_bytes);
    ok = cudaStreamCreateWithFlags(&cs[0], cudaStreamNonBlocking) == cudaSuccess &&
         cudaStreamCreateWithFlags(&cs[1], cudaStreamNonBlocking) == cudaSuccess;
    for (int h = 0; ok && h < 2; ++h)
      ok = cudaEventCreateWithFlags(&ev_fill[h], cudaEventDisableTiming) == cudaSuccess &&
           cudaEventCreateWithFlags(&ev_copy[h][0], cudaEventDisableTiming) == cudaSuccess &&
           cudaEventCreateWithFlags(&ev_copy[h][1], cudaEventDisableTiming) == cudaSuccess;
    return ok ? PCT_OK : cuda_check("host streaming: streams / events");
  }

  // rows [0, rows) of S (row pointers rp_dev on the device, the same values
  // in rph on the host) into col_host / val_host (at the rows' first entry)
  // and b_host (at their first row)
  pct_status rows(const SimDev& S, const Layout& L, void* ws, int precision, long long rows, const long long* rp_dev,
                  const long long* rph, const float* x, int32_t* col_host, float* val_host, float* b_host) {
    long long r0 = 0;
    bool first = true;
    while (ok && r0 < rows) {
      const long long nz0 = rph[r0];
      // the longest block from r0 whose entries and rows fit one half
      long long r1 = (long long)(std::upper_bound(rph + r0, rph + rows + 1, nz0 + E) - rph) - 1;
      r1 = std::min(std::min(r1, r0 + Rb), rows);
      if (r1 <= r0)
        return fail(PCT_EINVAL, "staging buffer cannot hold row %lld (%lld entries)", r0, rph[r0 + 1] - nz0);
      const long long nz1 = rph[r1];
      const int h = (int)(k & 1);
      int* col_s = (int*)(base + h * half);
      float* val_s = (float*)(base + h * half + 4 * E);
      float* b_s = (float*)(base + h * half + 8 * E);
      if (k >= 2)
        ok = cudaStreamWaitEvent(st, ev_copy[h][0], 0) == cudaSuccess &&
             cudaStreamWaitEvent(st, ev_copy[h][1], 0) == cudaSuccess;
      if (!ok) break;  // never refill a half whose copies may still be running
      if (precision == PCT_PREC_F64)  // col / val by CSR position: bases moved back by nz0 (host arithmetic)
        launch_fill_f64(S, r0, r1 - r0, rp_dev + r0, x, (int*)((uintptr_t)col_s - sizeof(int) * (uintptr_t)nz0),
                        (float*)((uintptr_t)val_s - sizeof(float) * (uintptr_t)nz0), b_s, st);
      else
        launch_fill_mixed(S, (const char*)ws + L.basis32, L.rows, (const char*)ws + L.rec, rp_dev, x, col_s, val_s,
                          b_s, (char*)ws + L.args, st, r0, r1, nz0, first, precision == PCT_PREC_MIXED_LEAN);
      first = false;
      ok = ok && cudaGetLastError() == cudaSuccess && cudaEventRecord(ev_fill[h], st) == cudaSuccess &&
           cudaStreamWaitEvent(cs[0], ev_fill[h], 0) == cudaSuccess &&
           cudaStreamWaitEvent(cs[1], ev_fill[h], 0) == cudaSuccess;
      if (ok && nz1 > nz0)
        ok = cudaMemcpyAsync(col_host + nz0, col_s, 4 * (size_t)(nz1 - nz0), cudaMemcpyDeviceToHost, cs[0]) ==
                 cudaSuccess &&
             cudaMemcpyAsync(val_host + nz0, val_s, 4 * (size_t)(nz1 - nz0), cudaMemcpyDeviceToHost, cs[1]) ==
                 cudaSuccess;
      ok = ok &&
           cudaMemcpyAsync(b_host + r0, b_s, 4 * (size_t)(r1 - r0), cudaMemcpyDeviceToHost, cs[1]) == cudaSuccess &&
           cudaEventRecord(ev_copy[h][0], cs[0]) == cudaSuccess && cudaEventRecord(ev_copy[h][1], cs[1]) == cudaSuccess;
      ++k;
      r0 = r1;
    }
    return ok ? PCT_OK : PCT_ECUDA;
  }

  // waits for every copy and fill; the CUDA error, if any
  pct_status finish(const char* what) {
    ok = ok && (!cs[0] || cudaStreamSynchronize(cs[0]) == cudaSuccess) &&
         (!cs[1] || cudaStreamSynchronize(cs[1]) == cudaSuccess) && cudaStreamSynchronize(st) == cudaSuccess;
    if (ok) return PCT_OK;
    const pct_status e = cuda_check(what);
    return e != PCT_OK ? e : fail(PCT_ECUDA, "%s: a CUDA call failed", what);
  }

  ~HostStream() {
    for (int c = 0; c < 2; ++c)
      if (cs[c]) cudaStreamSynchronize(cs[c]);
    if (st) cudaStreamSynchronize(st);
    for (int h = 0; h < 2; ++h) {
      if (ev_fill[h]) cudaEventDestroy(ev_fill[h]);
      for (int c = 0; c < 2; ++c)
        if (ev_copy[h][c]) cudaEventDestroy(ev_copy[h][c]);
    }
    for (int c = 0; c < 2; ++c)
      if (cs[c]) cudaStreamDestroy(cs[c]);
  }
};

}  // namespace

// Phase 2 into host memory: the rows go through the staging halves as
// HostStream describes.
extern "C" pct_status pct_simulate_fill_host(const pct_phantom* ph, const pct_geometry* g, int32_t precision,
                                             void* ws, size_t ws_bytes, const int64_t* row_ptr_dev,
                                             const float* x, void* staging, size_t staging_bytes,
                                             int64_t* row_ptr_host, int32_t* col_host, float* val_host,
                                             float* b_host, void* stream) {
  cudaStream_t st = (cudaStream_t)stream;
  // argument checks first (host only)
  pct_status rc = check_geometry(ph, g, precision);
  if (rc != PCT_OK) return rc;
  const long long rows = layout_of(ph, g, precision).rows;
  if (!row_ptr_dev || !row_ptr_host) return fail(PCT_EINVAL, "pct_simulate_fill_host: NULL row pointers");
  if (rows > 0 && (!x || !b_host || !staging)) return fail(PCT_EINVAL, "pct_simulate_fill_host: NULL argument");
  if ((uintptr_t)staging % 256 != 0) return fail(PCT_EINVAL, "staging buffer must be 256-byte aligned");
  SimDev S;
  Layout L;
  rc = make_sim(ph, g, precision, ws, ws_bytes, st, S, L);
  if (rc != PCT_OK) return rc;
  if (cudaMemcpyAsync(row_ptr_host, row_ptr_dev, sizeof(int64_t) * (size_t)(L.rows + 1), cudaMemcpyDeviceToHost,
                      st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return cuda_check("pct_simulate_fill_host: row pointers");
  if (L.rows == 0) return PCT_OK;
  const long long* rph = (const long long*)row_ptr_host;
  if (rph[L.rows] > 0 && (!col_host || !val_host))
    return fail(PCT_EINVAL, "pct_simulate_fill_host: NULL col_host or val_host for %lld nonzeros", rph[L.rows]);
  HostStream hs;
  if ((rc = hs.init(st, staging, staging_bytes)) != PCT_OK) return rc;
  rc = hs.rows(S, L, ws, precision, L.rows, (const long long*)row_ptr_dev, rph, x, col_host, val_host, b_host);
  const pct_status fin = hs.finish("pct_simulate_fill_host");
  if (rc == PCT_EINVAL) return rc;
  if (fin != PCT_OK) return fin;
  unsigned long long bad;
  if ((rc = read_mismatch(ws, st, &bad)) != PCT_OK) return rc;
  return bad ? mismatch_error("pct_simulate_fill_host", bad) : PCT_OK;
}

namespace {

// the geometry of angles [a0, a1) of g: the acquisition's own rows
pct_geometry angle_block(const pct_geometry* g, int a0, int a1) {
  pct_geometry b = *g;
  b.angles_rad = g->angles_rad ? g->angles_rad + a0 : nullptr;
  b.n_angles = a1 - a0;
  b.first_row = g->first_row + (int64_t)a0 * g->paths_per_angle;
  return b;
}

// one block's layout (the largest block) and the offset of its row pointers
size_t host_block_layout(const pct_phantom* ph, const pct_geometry* g, int precision, int apb, size_t* rp_off) {
  const int n = std::min(apb, g->n_angles);
  const pct_geometry b = angle_block(g, 0, n);
  const Layout L = layout_of(ph, &b, precision);
  *rp_off = L.total;
  return L.total + align256(sizeof(long long) * (size_t)(L.rows + 1));
}

}  // namespace

extern "C" pct_status pct_simulate_host_workspace_size(const pct_phantom* ph, const pct_geometry* g, int32_t precision,
                                                       int32_t angles_per_block, size_t* bytes) {
  if (!bytes) return fail(PCT_EINVAL, "bytes is NULL");
  pct_status rc = check_geometry(ph, g, precision);
  if (rc != PCT_OK) return rc;
  if (angles_per_block < 1) return fail(PCT_EINVAL, "angles_per_block = %d must be >= 1", angles_per_block);
  size_t off;
  *bytes = host_block_layout(ph, g, precision, angles_per_block, &off);
  return PCT_OK;
}

extern "C" pct_status pct_simulate_host(const pct_phantom* ph, const pct_geometry* g, int32_t precision,
                                        int32_t angles_per_block, void* ws, size_t ws_bytes, const float* x,
                                        void* staging, size_t staging_bytes, int64_t* row_ptr_host, int32_t* col_host,
                                        float* val_host, float* b_host, int64_t nnz_capacity, int64_t* nnz_out,
                                        void* stream) {
  cudaStream_t st = (cudaStream_t)stream;
  // argument checks first (host only)
  pct_status rc = check_geometry(ph, g, precision);
  if (rc != PCT_OK) return rc;
  if (angles_per_block < 1) return fail(PCT_EINVAL, "angles_per_block = %d must be >= 1", angles_per_block);
  if (!row_ptr_host || !nnz_out) return fail(PCT_EINVAL, "pct_simulate_host: NULL row_ptr_host or nnz_out");
  if (nnz_capacity < 0) return fail(PCT_EINVAL, "nnz_capacity must be >= 0");
  const long long rows = (long long)g->n_angles * g->paths_per_angle;
  if (rows > 0 && (!x || !b_host || !staging)) return fail(PCT_EINVAL, "pct_simulate_host: NULL argument");
  if ((uintptr_t)staging % 256 != 0) return fail(PCT_EINVAL, "staging buffer must be 256-byte aligned");
  if (nnz_capacity > 0 && (!col_host || !val_host))
    return fail(PCT_EINVAL, "pct_simulate_host: NULL col_host or val_host with nnz_capacity %lld",
                (long long)nnz_capacity);
  *nnz_out = 0;
  row_ptr_host[0] = 0;
  if (rows == 0) return PCT_OK;
  size_t rp_off;
  const size_t need = host_block_layout(ph, g, precision, angles_per_block, &rp_off);
  if (!ws || ws_bytes < need)
    return fail(PCT_ENOMEM, "workspace of %zu bytes is smaller than the %zu needed", ws_bytes, need);
  long long* rp_dev = (long long*)((char*)ws + rp_off);
  if (cudaMemsetAsync(ws, 0, sizeof(unsigned long long), st) != cudaSuccess)
    return cuda_check("pct_simulate_host: row check");
  HostStream hs;
  if ((rc = hs.init(st, staging, staging_bytes)) != PCT_OK) return rc;
  long long nz = 0;
  bool filling = true;
  for (int a0 = 0; a0 < g->n_angles && rc == PCT_OK; a0 += angles_per_block) {
    const int a1 = std::min(a0 + angles_per_block, g->n_angles);
    const pct_geometry gb = angle_block(g, a0, a1);
    SimDev S;
    Layout L;
    if ((rc = make_sim(ph, &gb, precision, ws, rp_off, st, S, L)) != PCT_OK) break;
    const long long r0 = (long long)a0 * g->paths_per_angle;
    if (L.rows == 0) continue;
    // count and scan of the block (after the previous block's fills on st)
    if (precision == PCT_PREC_F64)
      launch_count_f64(S, 0, L.rows, rp_dev + 1, st);
    else
      launch_count_mixed(S, (const char*)ws + L.basis32, L.rows, (char*)ws + L.rec, rp_dev + 1, (char*)ws + L.args,
                         st, precision == PCT_PREC_MIXED_LEAN);
    if ((rc = cuda_check("pct_simulate_host: count launch")) != PCT_OK) break;
    launch_scan_rowptr(rp_dev, L.rows, (long long*)((char*)ws + L.partial), st);
    // the block's row pointers, local to the block, where its global ones go
    long long* rph = (long long*)row_ptr_host + r0;
    if (cudaMemcpyAsync(rph, rp_dev, sizeof(long long) * (size_t)(L.rows + 1), cudaMemcpyDeviceToHost, st) !=
            cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess) {
      rc = cuda_check("pct_simulate_host: row pointers");
      if (rc == PCT_OK) rc = fail(PCT_ECUDA, "pct_simulate_host: row pointers");
      break;
    }
    const long long nb = rph[L.rows];
    filling = filling && nz + nb <= nnz_capacity;
    if (filling) {
      rc = hs.rows(S, L, ws, precision, L.rows, rp_dev, rph, x, col_host + nz, val_host + nz, b_host + r0);
      if (rc != PCT_OK) break;
    }
    // global row pointers (the fills above have read the local ones)
    for (long long i = 0; i <= L.rows; ++i) rph[i] += nz;
    nz += nb;
  }
  const pct_status fin = hs.finish("pct_simulate_host");
  if (rc == PCT_OK) rc = fin;
  if (rc != PCT_OK) return rc == PCT_ECUDA && fin != PCT_OK ? fin : rc;
  *nnz_out = nz;
  if (!filling)
    return fail(PCT_ENOMEM, "pct_simulate_host: %lld nonzeros exceed nnz_capacity %lld (row pointers complete)", nz,
                (long long)nnz_capacity);
  unsigned long long bad;
  if ((rc = read_mismatch(ws, st, &bad)) != PCT_OK) return rc;
  return bad ? mismatch_error("pct_simulate_host", bad) : PCT_OK;
}

extern "C" pct_status pct_simulate_check(const void* ws, int64_t* mismatched_rows, void* stream) {
  if (!ws || !mismatched_rows) return fail(PCT_EINVAL, "pct_simulate_check: NULL argument");
  unsigned long long bad;
  const pct_status rc = read_mismatch(ws, (cudaStream_t)stream, &bad);
  *mismatched_rows = (int64_t)bad;
  return rc;
}

extern "C" pct_status pct_simulate(const pct_phantom* ph, const pct_geometry* g, int32_t precision,
                                   pct_alloc_fn alloc_fn, pct_free_fn free_fn, void* ctx, pct_csr* out,
                                   void* stream) {
  if (!alloc_fn || !free_fn || !out) return fail(PCT_EINVAL, "pct_simulate: NULL allocator or output");
  cudaStream_t st = (cudaStream_t)stream;
  pct_status rc = check_geometry(ph, g, precision);
  if (rc != PCT_OK) return rc;
  memset(out, 0, sizeof(*out));
  Layout L = layout_of(ph, g, precision);
  void* ws = nullptr;
  pct_csr c;
  memset(&c, 0, sizeof(c));
  c.n_rows = L.rows;
  c.n_cols = ph->nvox;
  auto cleanup = [&]() {
    if (ws) free_fn(ws, ctx);
    if (c.row_ptr) free_fn(c.row_ptr, ctx);
    if (c.col) free_fn(c.col, ctx);
    if (c.val) free_fn(c.val, ctx);
    if (c.b) free_fn(c.b, ctx);
    if (c.x_true) free_fn(c.x_true, ctx);
  };
  ws = alloc_fn(L.total, ctx);
  c.x_true = (float*)alloc_fn(sizeof(float) * (size_t)ph->nvox, ctx);
  c.row_ptr = (int64_t*)alloc_fn(sizeof(int64_t) * (size_t)(L.rows + 1), ctx);
  c.b = (float*)alloc_fn(sizeof(float) * (size_t)(L.rows > 0 ? L.rows : 1), ctx);
  if (!ws || !c.x_true || !c.row_ptr || !c.b) {
    cleanup();
    return fail(PCT_ENOMEM, "allocator returned NULL");
  }
  if ((rc = pct_phantom_rasterize(ph, c.x_true, stream)) != PCT_OK ||
      (rc = pct_simulate_count(ph, g, precision, ws, L.total, c.row_ptr, stream)) != PCT_OK) {
    cleanup();
    return rc;
  }
  long long nnz = 0;
  if (cudaMemcpyAsync(&nnz, c.row_ptr + L.rows, sizeof(long long), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess) {
    cleanup();
    return cuda_check("reading nnz");
  }
  c.nnz = nnz;
  c.col = (int32_t*)alloc_fn(sizeof(int32_t) * (size_t)(nnz > 0 ? nnz : 1), ctx);
  c.val = (float*)alloc_fn(sizeof(float) * (size_t)(nnz > 0 ? nnz : 1), ctx);
  if (!c.col || !c.val) {
    cleanup();
    return fail(PCT_ENOMEM, "allocator returned NULL for %lld nonzeros", nnz);
  }
  if ((rc = pct_simulate_fill(ph, g, precision, ws, L.total, c.row_ptr, c.x_true, c.col, c.val, c.b, stream)) !=
      PCT_OK) {
    cleanup();
    return rc;
  }
  unsigned long long bad;
  if ((rc = read_mismatch(ws, st, &bad)) != PCT_OK || (bad && (rc = mismatch_error("pct_simulate", bad)) != PCT_OK)) {
    cleanup();
    return rc;
  }
  free_fn(ws, ctx);
  *out = c;
  return PCT_OK;
}

// ---------------------------------------------------------------------------
// projectors
// ---------------------------------------------------------------------------
extern "C" pct_status pct_projector_workspace_size(const pct_phantom* ph, const pct_geometry* g, int32_t precision,
                                                   int64_t max_rows, size_t* bytes) {
  if (!bytes || max_rows < 0) return fail(PCT_EINVAL, "pct_projector_workspace_size: bad arguments");
  pct_status rc = check_geometry(ph, g, precision);
  if (rc != PCT_OK) return rc;
  *bytes = layout_of(ph, g, precision, max_rows).total;
  return PCT_OK;
}

namespace {

pct_status project(bool adjoint, const pct_phantom* ph, const pct_geometry* g, const pct_csr* A, int32_t precision,
                   int64_t row0, int64_t n_rows, const float* in, float* out, void* ws, size_t ws_bytes,
                   cudaStream_t st) {
  const char* what = adjoint ? "pct_adjoint" : "pct_forward";
  if (!in || !out) return fail(PCT_EINVAL, "%s: NULL input or output", what);
  if (row0 < 0 || n_rows < 0) return fail(PCT_EINVAL, "%s: negative row range", what);
  if (A) {
    if (!A->row_ptr || !A->col || !A->val) return fail(PCT_EINVAL, "%s: incomplete CSR", what);
    if (row0 + n_rows > A->n_rows) return fail(PCT_EINVAL, "%s: row range beyond the CSR", what);
    if (adjoint)
      launch_csr_adjoint((const long long*)A->row_ptr, A->col, A->val, row0, n_rows, in, out, st);
    else
      launch_csr_forward((const long long*)A->row_ptr, A->col, A->val, row0, n_rows, in, out, st);
    return cuda_check(what);
  }
  SimDev S;
  Layout L;
  pct_status rc = make_sim(ph, g, precision, ws, ws_bytes, st, S, L, n_rows);
  if (rc != PCT_OK) return rc;
  if (row0 + n_rows > L.rows) return fail(PCT_EINVAL, "%s: row range beyond the geometry", what);
  if (precision == PCT_PREC_F64) {
    if (adjoint)
      launch_mf_adjoint_f64(S, row0, n_rows, in, out, st);
    else
      launch_mf_forward_f64(S, row0, n_rows, in, out, st);
  } else {
    launch_proj_mixed(adjoint, S, (const char*)ws + L.basis32, row0, n_rows, (char*)ws + L.rec, in, out,
                      (char*)ws + L.args, st, precision == PCT_PREC_MIXED_LEAN);
  }
  return cuda_check(what);
}

}  // namespace

extern "C" pct_status pct_forward(const pct_phantom* ph, const pct_geometry* g, const pct_csr* A, int32_t precision,
                                  int64_t row0, int64_t n_rows, const float* x, float* y, void* ws, size_t ws_bytes,
                                  void* stream) {
  return project(false, ph, g, A, precision, row0, n_rows, x, y, ws, ws_bytes, (cudaStream_t)stream);
}

extern "C" pct_status pct_adjoint(const pct_phantom* ph, const pct_geometry* g, const pct_csr* A, int32_t precision,
                                  int64_t row0, int64_t n_rows, const float* r, float* gout, void* ws,
                                  size_t ws_bytes, void* stream) {
  return project(true, ph, g, A, precision, row0, n_rows, r, gout, ws, ws_bytes, (cudaStream_t)stream);
}

// ---------------------------------------------------------------------------
// batches
// ---------------------------------------------------------------------------
struct pct_batch {
  int n = 0;
  std::vector<pct_batch_item> items;      // as given
  std::vector<Layout> layouts;
  std::vector<size_t> base;               // workspace offset of each item's region
  std::vector<SimDev> sims;
  std::vector<BatchInst> by_item;         // order-independent instance fields, by item
  std::vector<BatchInst> inst;            // processing order
  std::vector<int> order;                 // processing position -> item index
  std::vector<int*> out_col;              // outputs by item (set by pct_batch_fill)
  std::vector<float*> out_val, out_b;
  BatchInst* d_inst = nullptr;
  unsigned long long* d_next = nullptr;   // two counters (2D, 3D launches)
  long long first3[3] = {0, 0, 0}, total[3] = {0, 0, 0};  // per phase: first 3D work item, work items
  pct_batch_tuning tune;                  // the launch shape in use
  bool lean = false;        // PCT_BATCH_LEAN: instances may take the lean form
  std::vector<char> lean_k; // by item: the lean form (no segment records, the fill rebuilds the table)
  long long f2[2][2][2] = {};  // fill phase: [dim 3][lean] first and last work item
  int bps2[2][2] = {{1, 1}, {1, 1}};  // fill phase: resident blocks per SM [dim 3][lean]
  bool autotune = false;
  bool fill_tuned = false;  // the fill's shape was timed (or taken from the cache)
  unsigned long long sig = 0;
  int bps[3][2] = {{1, 1}, {1, 1}, {1, 1}};  // resident blocks per SM [phase][dim 3]
  bool small[2] = {true, true};               // [dim 3]: every instance fits the smaller layout
  int sms = 1;
  cudaGraphExec_t e_count = nullptr, e_fill = nullptr;
  cudaGraph_t g_count = nullptr, g_fill = nullptr;
};

namespace {

struct TuneEntry {
  pct_batch_tuning t;
  bool fill_tuned;
};
std::mutex g_tune_mu;
std::map<unsigned long long, TuneEntry> g_tune_cache;  // batch signature -> launch shape

pct_batch_tuning default_tuning() {
  pct_batch_tuning t;
  t.order = 0;
  for (int p = 0; p < 3; ++p) {
    t.rows_per_item[p] = 128;
    t.grid_mult[p] = 1;
  }
  t.fill_prefetch = 1;
  return t;
}

unsigned long long batch_signature(const pct_batch& b) {
  unsigned long long h = 1469598103934665603ULL;
  auto mix = [&](unsigned long long v) {
    h ^= v;
    h *= 1099511628211ULL;
  };
  mix(b.lean ? 1ULL : 0ULL);
  for (int k = 0; k < b.n; ++k) {
    const pct_batch_item& it = b.items[k];
    mix(b.lean_k[k] ? 1ULL : 0ULL);
    mix((unsigned long long)it.phantom->dev.g.dim);
    for (int a = 0; a < 3; ++a) mix((unsigned long long)it.phantom->dev.g.n[a]);
    mix((unsigned long long)b.layouts[k].rows);
    mix((unsigned long long)it.geo.model.model);
  }
  return h;
}

// Processing order (2D instances first, then 3D; within each, the full form
// before the lean form, then item order or largest first) and each phase's
// work items of rows_per_item[phase] rows; uploads the instance table (with
// the outputs set so far).
pct_status batch_arrange(pct_batch& b, cudaStream_t st) {
  const int n = b.n;
  std::vector<int> ord(n);
  for (int k = 0; k < n; ++k) ord[k] = k;
  std::stable_sort(ord.begin(), ord.end(), [&](int x, int y) {
    const int dx = b.items[x].phantom->dev.g.dim, dy = b.items[y].phantom->dev.g.dim;
    if (dx != dy) return dx < dy;
    if (b.lean_k[x] != b.lean_k[y]) return b.lean_k[x] < b.lean_k[y];
    if (b.tune.order == 1) return b.layouts[x].rows > b.layouts[y].rows;
    return false;
  });
  b.order = ord;
  b.inst.resize(n);
  for (int pos = 0; pos < n; ++pos) {
    const int k = ord[pos];
    b.inst[pos] = b.by_item[k];
    b.inst[pos].col = b.out_col[k];
    b.inst[pos].val = b.out_val[k];
    b.inst[pos].b = b.out_b[k];
  }
  for (int p = 0; p < 3; ++p) {
    const long long R = b.tune.rows_per_item[p];
    long long item = 0;
    b.first3[p] = -1;
    for (int pos = 0; pos < n; ++pos) {
      if (b.first3[p] < 0 && b.inst[pos].S.ph.g.dim == 3) b.first3[p] = item;
      b.inst[pos].item0[p] = item;
      item += (b.inst[pos].n + R - 1) / R;
    }
    b.total[p] = item;
    if (b.first3[p] < 0) b.first3[p] = item;
  }
  // the fill phase's four launches: [dim 3][lean], each a contiguous item range
  {
    const long long R = b.tune.rows_per_item[2];
    for (int d = 0; d < 2; ++d)
      for (int l = 0; l < 2; ++l) b.f2[d][l][0] = b.f2[d][l][1] = 0;
    bool seen[2][2] = {{false, false}, {false, false}};
    for (int pos = 0; pos < n; ++pos) {
      const int d = b.inst[pos].S.ph.g.dim == 3 ? 1 : 0, l = b.lean_k[ord[pos]] ? 1 : 0;
      const long long i0 = b.inst[pos].item0[2], i1 = i0 + (b.inst[pos].n + R - 1) / R;
      if (!seen[d][l]) {
        b.f2[d][l][0] = i0;
        seen[d][l] = true;
      }
      b.f2[d][l][1] = i1;
    }
  }
  if (cudaMemcpyAsync(b.d_inst, b.inst.data(), sizeof(BatchInst) * n, cudaMemcpyHostToDevice, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return cuda_check("batch table upload");
  return PCT_OK;
}

void batch_launch_phase(pct_batch& b, int f, cudaStream_t st) {
  const pct_batch_tuning& t = b.tune;
  if (f == 2) {
    // full-form instances, then lean ones, per dimensionality (the
    // launches run in stream order, so two counters serve all four)
    for (int d = 0; d < 2; ++d)
      for (int l = 0; l < 2; ++l)
        launch_batch(2, d == 0 ? 2 : 3, b.small[d], l != 0, b.d_inst, b.n, b.f2[d][l][0], b.f2[d][l][1],
                     b.d_next + l, b.sms * b.bps2[d][l] * t.grid_mult[2], t.rows_per_item[2], t.fill_prefetch, st);
    return;
  }
  launch_batch(f, 2, b.small[0], b.lean, b.d_inst, b.n, 0, b.first3[f], b.d_next,
               b.sms * b.bps[f][0] * t.grid_mult[f], t.rows_per_item[f], t.fill_prefetch, st);
  launch_batch(f, 3, b.small[1], b.lean, b.d_inst, b.n, b.first3[f], b.total[f], b.d_next + 1,
               b.sms * b.bps[f][1] * t.grid_mult[f], t.rows_per_item[f], t.fill_prefetch, st);
}

void batch_phase(pct_batch& b, bool fill, cudaStream_t st) {
  if (!fill) {
    for (int k = 0; k < b.n; ++k)
      launch_raster(b.items[k].phantom->dev, b.items[k].x_true_dev, b.items[k].phantom->nvox, st);
  }
  // count: the FP64 path set-up, then the cooperative count; fill: the fill
  for (int f = fill ? 2 : 0; f <= (fill ? 2 : 1); ++f) batch_launch_phase(b, f, st);
  if (!fill) {
    for (int k = 0; k < b.n; ++k)
      launch_scan_rowptr((long long*)b.items[k].row_ptr_dev, b.layouts[k].rows,
                         (long long*)((char*)b.sims[k].cs - b.layouts[k].cs + b.layouts[k].partial), st);
  }
}

pct_status batch_capture(pct_batch& b, bool fill) {
  cudaStream_t cap;
  if (cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking) != cudaSuccess) return cuda_check("capture stream");
  cudaGraph_t g = nullptr;
  cudaGraphExec_t e = nullptr;
  bool ok = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
  if (ok) {
    batch_phase(b, fill, cap);
    ok = cudaStreamEndCapture(cap, &g) == cudaSuccess;
  }
  if (ok) ok = cudaGraphInstantiate(&e, g, 0) == cudaSuccess;
  cudaStreamDestroy(cap);
  if (!ok) {
    if (g) cudaGraphDestroy(g);
    return cuda_check("graph capture");
  }
  if (fill) {
    if (b.e_fill) cudaGraphExecDestroy(b.e_fill);
    if (b.g_fill) cudaGraphDestroy(b.g_fill);
    b.g_fill = g;
    b.e_fill = e;
  } else {
    if (b.e_count) cudaGraphExecDestroy(b.e_count);
    if (b.g_count) cudaGraphDestroy(b.g_count);
    b.g_count = g;
    b.e_count = e;
  }
  return PCT_OK;
}

// device ms of the given phases (one warm-up run, then one timed run)
pct_status time_phases(pct_batch& b, int p0, int p1, cudaStream_t st, float* ms) {
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return cuda_check("autotune events");
  for (int f = p0; f <= p1; ++f) batch_launch_phase(b, f, st);
  cudaEventRecord(e0, st);
  for (int f = p0; f <= p1; ++f) batch_launch_phase(b, f, st);
  cudaEventRecord(e1, st);
  pct_status rc = PCT_OK;
  if (cudaEventSynchronize(e1) != cudaSuccess)
    rc = cuda_check("autotune");
  else
    cudaEventElapsedTime(ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return rc;
}

// the best of rows per work item {64, 128, 256} x grid multiplier {1, 2}
// (x prefetch {0, 1} for the fill) for one phase, the others as they stand
pct_status tune_phase(pct_batch& b, int f, cudaStream_t st) {
  const int rows[3] = {64, 128, 256};
  pct_batch_tuning best = b.tune;
  float best_ms = 1e30f;
  for (int pf = (f == 2 ? 0 : 1); pf <= 1; ++pf)
    for (int ri = 0; ri < 3; ++ri)
      for (int gm = 1; gm <= 2; ++gm) {
        b.tune.rows_per_item[f] = rows[ri];
        b.tune.grid_mult[f] = gm;
        if (f == 2) b.tune.fill_prefetch = pf;
        pct_status rc = batch_arrange(b, st);
        float ms = 0.f;
        if (rc == PCT_OK) rc = time_phases(b, f, f, st, &ms);
        if (rc != PCT_OK) return rc;
        if (ms < best_ms) {
          best_ms = ms;
          best = b.tune;
        }
      }
  b.tune = best;
  return batch_arrange(b, st);
}

}  // namespace

extern "C" pct_status pct_batch_workspace_size(const pct_batch_item* items, int32_t n, int32_t flags,
                                                size_t* bytes) {
  if (!items || n < 1 || !bytes) return fail(PCT_EINVAL, "pct_batch_workspace_size: bad arguments");
  const int form = (flags & PCT_BATCH_LEAN) ? PCT_PREC_MIXED_LEAN : PCT_PREC_MIXED;
  size_t off = 0;
  for (int k = 0; k < n; ++k) {
    pct_status rc = check_geometry(items[k].phantom, &items[k].geo, form);
    if (rc != PCT_OK) return rc;
    off = align256(off + layout_of(items[k].phantom, &items[k].geo, form).total);
  }
  off = align256(off + sizeof(BatchInst) * (size_t)n);
  off = align256(off + 2 * sizeof(unsigned long long));
  *bytes = off;
  return PCT_OK;
}

extern "C" pct_status pct_batch_destroy(pct_batch* b) {
  if (!b) return PCT_OK;
  if (b->e_count) cudaGraphExecDestroy(b->e_count);
  if (b->e_fill) cudaGraphExecDestroy(b->e_fill);
  if (b->g_count) cudaGraphDestroy(b->g_count);
  if (b->g_fill) cudaGraphDestroy(b->g_fill);
  delete b;
  return PCT_OK;
}

extern "C" pct_status pct_batch_create(const pct_batch_item* items, int32_t n, void* ws, size_t ws_bytes,
                                       int32_t flags, void* stream, pct_batch** out) {
  if (!out) return fail(PCT_EINVAL, "pct_batch_create: out is NULL");
  *out = nullptr;
  size_t need = 0;
  pct_status rc = pct_batch_workspace_size(items, n, flags, &need);
  const int form = (flags & PCT_BATCH_LEAN) ? PCT_PREC_MIXED_LEAN : PCT_PREC_MIXED;
  if (rc != PCT_OK) return rc;
  if (!ws || ws_bytes < need) return fail(PCT_ENOMEM, "batch workspace of %zu bytes is smaller than %zu", ws_bytes, need);
  cudaStream_t st = (cudaStream_t)stream;
  pct_batch* b = new (std::nothrow) pct_batch;
  if (!b) return fail(PCT_ENOMEM, "out of host memory");
  b->n = n;
  b->lean = form == PCT_PREC_MIXED_LEAN;
  b->lean_k.assign(n, b->lean ? 1 : 0);
  if (b->lean) {
    // the workspace beyond the all-lean size holds segment records: the
    // largest instances take the full form (a fill twice as fast) while
    // their records fit
    size_t spare = ws_bytes - need;
    std::vector<int> by_rows(n);
    for (int k = 0; k < n; ++k) by_rows[k] = k;
    std::stable_sort(by_rows.begin(), by_rows.end(), [&](int x, int y) {
      return (long long)items[x].geo.n_angles * items[x].geo.paths_per_angle >
             (long long)items[y].geo.n_angles * items[y].geo.paths_per_angle;
    });
    for (int k : by_rows) {
      const size_t full = align256(layout_of(items[k].phantom, &items[k].geo, PCT_PREC_MIXED).total);
      const size_t lean = align256(layout_of(items[k].phantom, &items[k].geo, PCT_PREC_MIXED_LEAN).total);
      if (full > lean && full - lean <= spare) {
        b->lean_k[k] = 0;
        spare -= full - lean;
      }
    }
  }
  b->autotune = (flags & PCT_BATCH_AUTOTUNE) != 0;
  b->tune = default_tuning();
  b->items.assign(items, items + n);
  b->layouts.resize(n);
  b->base.resize(n);
  b->sims.resize(n);
  b->out_col.assign(n, nullptr);
  b->out_val.assign(n, nullptr);
  b->out_b.assign(n, nullptr);
  char* base = (char*)ws;
  size_t off = 0;
  for (int k = 0; k < n; ++k) {
    const pct_batch_item& it = items[k];
    const int form_k = b->lean_k[k] ? PCT_PREC_MIXED_LEAN : PCT_PREC_MIXED;
    Layout L = layout_of(it.phantom, &it.geo, form_k);
    if (L.rows > 0 && (!it.row_ptr_dev || !it.x_true_dev)) {
      pct_batch_destroy(b);
      return fail(PCT_EINVAL, "batch item %d: NULL row_ptr_dev or x_true_dev", k);
    }
    b->base[k] = off;
    Layout L2;
    rc = make_sim(it.phantom, &it.geo, form_k, base + off, L.total, st, b->sims[k], L2);
    if (rc != PCT_OK) {
      pct_batch_destroy(b);
      return rc;
    }
    b->layouts[k] = L2;
    off = align256(off + L.total);
  }
  b->d_inst = (BatchInst*)(base + off);
  off = align256(off + sizeof(BatchInst) * (size_t)n);
  b->d_next = (unsigned long long*)(base + off);
  int dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&b->sms, cudaDevAttrMultiProcessorCount, dev);
  // instance table contents (order-independent fields)
  b->by_item.resize(n);
  for (int k = 0; k < n; ++k) {
    BatchInst& I = b->by_item[k];
    memset(&I, 0, sizeof(I));
    I.S = b->sims[k];
    I.M = mix_args(b->sims[k], b->layouts[k].rows, (const char*)b->sims[k].cs - b->layouts[k].cs + b->layouts[k].basis32,
                   (char*)b->sims[k].cs - b->layouts[k].cs + b->layouts[k].rec, b->lean_k[k] != 0);
    I.n = b->layouts[k].rows;
    I.row_ptr_w = (long long*)items[k].row_ptr_dev;
    I.row_ptr = (const long long*)items[k].row_ptr_dev;
    I.x = items[k].x_true_dev;
    if (!small_cap(I.M.seg_stride, I.S.ph.g)) b->small[I.S.ph.g.dim == 3 ? 1 : 0] = false;
  }
  for (int f = 0; f < 3; ++f)
    for (int d = 0; d < 2; ++d) b->bps[f][d] = batch_blocks_per_sm(f, d == 0 ? 2 : 3, b->small[d], b->lean);
  for (int d = 0; d < 2; ++d)
    for (int l = 0; l < 2; ++l) b->bps2[d][l] = batch_blocks_per_sm(2, d == 0 ? 2 : 3, b->small[d], l != 0);
  b->sig = batch_signature(*b);
  bool cached = false;
  {
    std::lock_guard<std::mutex> lock(g_tune_mu);
    auto itc = g_tune_cache.find(b->sig);
    if (itc != g_tune_cache.end()) {
      b->tune = itc->second.t;
      b->fill_tuned = itc->second.fill_tuned;
      cached = true;
    }
  }
  if (b->autotune && !cached) {
    // item order on the whole count (path + count phases), then each
    // phase's rows per work item and grid size; the fill's at the first
    // pct_batch_fill (it needs the outputs)
    float best = 1e30f;
    int bo = 0;
    for (int om = 0; om < 2 && rc == PCT_OK; ++om) {
      b->tune.order = om;
      float ms = 0.f;
      if ((rc = batch_arrange(*b, st)) == PCT_OK && (rc = time_phases(*b, 0, 1, st, &ms)) == PCT_OK && ms < best) {
        best = ms;
        bo = om;
      }
    }
    b->tune.order = bo;
    if (rc == PCT_OK) rc = tune_phase(*b, 0, st);
    if (rc == PCT_OK) rc = tune_phase(*b, 1, st);
    if (rc != PCT_OK) {
      pct_batch_destroy(b);
      return rc;
    }
    std::lock_guard<std::mutex> lock(g_tune_mu);
    g_tune_cache[b->sig] = TuneEntry{b->tune, false};
  }
  if ((rc = batch_arrange(*b, st)) != PCT_OK || (rc = batch_capture(*b, false)) != PCT_OK ||
      (rc = batch_capture(*b, true)) != PCT_OK) {
    pct_batch_destroy(b);
    return rc;
  }
  *out = b;
  return PCT_OK;
}

extern "C" pct_status pct_batch_count(pct_batch* b, void* stream) {
  if (!b || !b->e_count) return fail(PCT_EINVAL, "pct_batch_count: no batch");
  if (cudaGraphLaunch(b->e_count, (cudaStream_t)stream) != cudaSuccess) return cuda_check("batch count graph");
  return PCT_OK;
}

extern "C" pct_status pct_batch_nnz(pct_batch* b, int64_t* nnz, void* stream) {
  if (!b || !nnz) return fail(PCT_EINVAL, "pct_batch_nnz: NULL argument");
  cudaStream_t st = (cudaStream_t)stream;
  for (int k = 0; k < b->n; ++k) {
    nnz[k] = 0;
    if (b->layouts[k].rows > 0 &&
        cudaMemcpyAsync(&nnz[k], b->items[k].row_ptr_dev + b->layouts[k].rows, sizeof(int64_t),
                        cudaMemcpyDeviceToHost, st) != cudaSuccess)
      return cuda_check("batch nnz");
  }
  if (cudaStreamSynchronize(st) != cudaSuccess) return cuda_check("batch nnz");
  return PCT_OK;
}

extern "C" pct_status pct_batch_fill(pct_batch* b, int32_t* const* col, float* const* val, float* const* bout,
                                     void* stream) {
  if (!b || !b->e_fill || !col || !val || !bout) return fail(PCT_EINVAL, "pct_batch_fill: NULL argument");
  cudaStream_t st = (cudaStream_t)stream;
  for (int k = 0; k < b->n; ++k) {
    if (b->layouts[k].rows > 0 && !bout[k]) return fail(PCT_EINVAL, "batch item %d: NULL b", k);
    b->out_col[k] = (int*)col[k];
    b->out_val[k] = val[k];
    b->out_b[k] = bout[k];
  }
  for (int pos = 0; pos < b->n; ++pos) {
    const int k = b->order[pos];
    b->inst[pos].col = b->out_col[k];
    b->inst[pos].val = b->out_val[k];
    b->inst[pos].b = b->out_b[k];
  }
  if (b->autotune && !b->fill_tuned) {
    // the fill's shape, timed once on these outputs (a fill rewrites the
    // same values), then the fill graph recaptured; the choice is cached
    pct_status rc = tune_phase(*b, 2, st);
    if (rc == PCT_OK) rc = batch_capture(*b, true);
    if (rc != PCT_OK) return rc;
    b->fill_tuned = true;
    std::lock_guard<std::mutex> lock(g_tune_mu);
    g_tune_cache[b->sig] = TuneEntry{b->tune, true};
  }
  // the graph reads the output pointers from the instance table in global
  // memory, so updating the table is enough (the copy is staged before return)
  if (cudaMemcpyAsync(b->d_inst, b->inst.data(), sizeof(BatchInst) * b->n, cudaMemcpyHostToDevice, st) != cudaSuccess)
    return cuda_check("batch table upload");
  if (cudaGraphLaunch(b->e_fill, st) != cudaSuccess) return cuda_check("batch fill graph");
  return PCT_OK;
}

extern "C" pct_status pct_batch_params(const pct_batch* b, pct_batch_tuning* out) {
  if (!b || !out) return fail(PCT_EINVAL, "pct_batch_params: NULL argument");
  *out = b->tune;
  return PCT_OK;
}

// ---------------------------------------------------------------------------
// reconstruction (Sec. II-D)
// ---------------------------------------------------------------------------
extern "C" pct_status pct_sap_workspace_size(int64_t n_cols, int32_t n_strings, size_t* bytes) {
  if (!bytes || n_cols < 0 || n_strings < 1 || n_strings > (1 << 24))
    return fail(PCT_EINVAL, "pct_sap_workspace_size: bad arguments");
  *bytes = sap_workspace_bytes(n_cols, n_strings);
  return PCT_OK;
}

extern "C" pct_status pct_sap(const pct_csr* A, const float* b, int32_t M, const double* weights, double lambda,
                              int32_t iterations, float* x, void* ws, size_t ws_bytes, void* stream) {
  if (!A || !x) return fail(PCT_EINVAL, "pct_sap: NULL A or x");
  if (A->n_rows < 0 || A->n_cols < 1 || A->n_cols >= (1LL << 31)) return fail(PCT_EINVAL, "pct_sap: bad A sizes");
  if (A->n_rows > 0 && (!A->row_ptr || !A->col || !A->val || !b)) return fail(PCT_EINVAL, "pct_sap: incomplete CSR or b");
  if (M < 1 || M > (1 << 24)) return fail(PCT_EINVAL, "pct_sap: n_strings = %d outside 1..2^24", M);
  if (iterations < 0) return fail(PCT_EINVAL, "pct_sap: negative iteration count");
  if (!std::isfinite(lambda)) return fail(PCT_EINVAL, "pct_sap: lambda must be finite");
  std::vector<double> w((size_t)M, 1.0 / (double)M);
  if (weights) {
    double s = 0.0;
    for (int t = 0; t < M; ++t) {
      if (!std::isfinite(weights[t])) return fail(PCT_EINVAL, "pct_sap: weight %d is not finite", t);
      w[t] = weights[t];
      s += weights[t];
    }
    if (std::fabs(s - 1.0) > 1e-9) return fail(PCT_EINVAL, "pct_sap: weights sum to %.17g, not 1", s);
  }
  const size_t need = sap_workspace_bytes(A->n_cols, M);
  if (!ws || ws_bytes < need) return fail(PCT_ENOMEM, "pct_sap: workspace of %zu bytes is smaller than %zu", ws_bytes, need);
  cudaStream_t st = (cudaStream_t)stream;
  // pageable source: the copy returns once the weights are staged
  if (cudaMemcpyAsync(ws, w.data(), sizeof(double) * (size_t)M, cudaMemcpyHostToDevice, st) != cudaSuccess)
    return cuda_check("pct_sap: weights");
  launch_sap((const long long*)A->row_ptr, A->col, A->val, b, A->n_rows, A->n_cols, M, (const double*)ws,
             (float)lambda, iterations, x, ws, st);
  return cuda_check("pct_sap launch");
}

extern "C" const char* pct_last_error(void) { return g_err.c_str(); }

pct_status pct::set_error(pct_status st, const char* msg) {
  g_err = msg;
  return st;
}

extern "C" const char* pct_version(void) { return "libpct 0.1 (sm_103a)"; }
