// pct_kernels.cuh -- launchers of the libpct kernels (host-callable).
#pragma once
#include "pct_device.cuh"

namespace pct {

// records msg as the calling thread's pct_last_error() and returns st
pct_status set_error(pct_status st, const char* msg);

// rows scanned per block by the row-pointer scan
constexpr int kScanTile = 4096;

void launch_raster(const PhantomDev& ph, float* x, long long nvox, cudaStream_t st);

// all-FP64 form (pct_f64.cu)
void launch_count_f64(const SimDev& S, long long row0, long long n, long long* counts, cudaStream_t st);
// rows [row0, row0 + n): row_ptr and b indexed from row0 (row_ptr[0] is
// row row0's), col / val by CSR position
void launch_fill_f64(const SimDev& S, long long row0, long long n, const long long* row_ptr,
                     const float* x, int* col, float* val, float* b, cudaStream_t st);
void launch_mf_forward_f64(const SimDev& S, long long row0, long long n, const float* x, float* y,
                           cudaStream_t st);
void launch_mf_adjoint_f64(const SimDev& S, long long row0, long long n, const float* r, float* g,
                           cudaStream_t st);

// double-float certified form (pct_mixed.cu).  rec: per-row records
// (mixed_record_size bytes); tab: Hermite basis table (basis_df_bytes(K + 1)
// bytes, filled on the host by fill_basis_df from s, h10, h11 at j = 0..K).
// lean: the count keeps no segment records (one flag byte per row instead)
// and the fill rebuilds each row's segment table
size_t mixed_record_size(long long rows, int dim, int model, int K, bool lean = false);
// compact segment records per row (the model's largest segment count, capped)
int seg_stride_of(int model, int K);
size_t mixed_args_bytes();
size_t basis_df_bytes(int n);
void fill_basis_df(const double* s, const double* h10, const double* h11, int n, void* host_out);
// args: mixed_args_bytes() of workspace for a global copy of the arguments
void launch_count_mixed(const SimDev& S, const void* tab, long long n, void* rec, long long* counts, void* args,
                        cudaStream_t st, bool lean = false);
// fill of rows [row_begin, row_end) (row_end < 0: n) of the n-row
// simulation: entries at CSR position k go to col / val[k - nz0], row r's
// WEPL to b[r - row_begin] (b[r] for the whole simulation).  upload = false
// reuses the argument copy of an earlier launch with the same S.
void launch_fill_mixed(const SimDev& S, const void* tab, long long n, const void* rec, const long long* row_ptr,
                       const float* x, int* col, float* val, float* b, void* args, cudaStream_t st,
                       long long row_begin = 0, long long row_end = -1, long long nz0 = 0, bool upload = true,
                       bool lean = false);

// matrix-free projector, rows [row_base, row_base + n): y = A x (in = x,
// out = y[n]) or g += A^T r (in = r[n], out = g); rec holds n rows of records
void launch_proj_mixed(bool adjoint, const SimDev& S, const void* tab, long long row_base, long long n, void* rec,
                       const float* in, float* out, void* args, cudaStream_t st, bool lean = false);

// row pointers (pct_scan.cu): row_ptr[0] = 0, row_ptr[1..n] = inclusive scan
// of the counts already stored in row_ptr[1..n]; partial holds
// ceil(n / kScanTile) + 1 int64 of scratch.
long long scan_partials_needed(long long n);
void launch_scan_rowptr(long long* row_ptr, long long n, long long* partial, cudaStream_t st);

// CSR projectors (pct_csr.cu)
void launch_csr_forward(const long long* row_ptr, const int* col, const float* val, long long row0,
                        long long n, const float* x, float* y, cudaStream_t st);
void launch_csr_adjoint(const long long* row_ptr, const int* col, const float* val, long long row0,
                        long long n, const float* r, float* g, cudaStream_t st);

// string-averaging projections (pct_sap.cu): workspace = M doubles of
// weights (256-byte aligned) then M x n_cols floats of string iterates
size_t sap_workspace_bytes(long long n_cols, int M);
void launch_sap(const long long* row_ptr, const int* col, const float* val, const float* b, long long n_rows,
                long long n_cols, int M, const double* w_dev, float lambda, int iterations, float* x, void* ws,
                cudaStream_t st);

}  // namespace pct
