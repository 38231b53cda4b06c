// pct_static.cu -- allocation-free row-pointer scan: the scan of
// pct_simulate_count with its scratch (one partial sum per tile of rows) in a
// static device array instead of a caller-provided workspace, for callers
// that cannot allocate device memory.
#include <cstdio>

#include "pct_kernels.cuh"

namespace {

// One int64 partial per tile of kScanTile rows, plus one: enough for
// PCT_STATIC_SCAN_MAX_ROWS rows (512 KB).  Every GPU that loads the library
// holds this array until the process exits.
constexpr long long kStaticTiles = PCT_STATIC_SCAN_MAX_ROWS / pct::kScanTile + 1;
static __device__ __align__(256) long long g_scan_scratch[kStaticTiles];

}  // namespace

extern "C" pct_status pct_scan_counts_static(int64_t* row_ptr_dev, int64_t n_rows, void* stream) {
  char msg[256];
  if (!row_ptr_dev) return pct::set_error(PCT_EINVAL, "pct_scan_counts_static: row_ptr_dev is NULL");
  if (n_rows < 0) return pct::set_error(PCT_EINVAL, "pct_scan_counts_static: negative n_rows");
  if (n_rows > PCT_STATIC_SCAN_MAX_ROWS) {
    snprintf(msg, sizeof(msg),
             "pct_scan_counts_static: %lld rows exceed the static scratch limit of %lld rows "
             "(use pct_simulate_count with a workspace)",
             (long long)n_rows, (long long)PCT_STATIC_SCAN_MAX_ROWS);
    return pct::set_error(PCT_EINVAL, msg);
  }
  // The array's name is a host-side stand-in; its device address comes from
  // the runtime, for the calling thread's current device and context.  It is
  // looked up on every call (no allocation, a table lookup once the module is
  // loaded), so a cudaDeviceReset or another context on the same device never
  // leaves a stale address behind.  The first call on a device loads the
  // module that holds the array.
  long long* scratch = nullptr;
  cudaError_t e = cudaGetSymbolAddress((void**)&scratch, g_scan_scratch);
  if (e != cudaSuccess || !scratch) {
    snprintf(msg, sizeof(msg), "pct_scan_counts_static: cudaGetSymbolAddress: %s", cudaGetErrorString(e));
    return pct::set_error(PCT_ECUDA, msg);
  }
  // every partial the scan reads is written by the same launch sequence first,
  // so the array needs no clearing between calls
  pct::launch_scan_rowptr((long long*)row_ptr_dev, (long long)n_rows, scratch, (cudaStream_t)stream);
  e = cudaGetLastError();
  if (e != cudaSuccess) {
    snprintf(msg, sizeof(msg), "pct_scan_counts_static: launch: %s", cudaGetErrorString(e));
    return pct::set_error(PCT_ECUDA, msg);
  }
  return PCT_OK;
}
