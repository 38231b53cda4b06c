// pct_io.cu -- the simulated system on disk (Sec. II-C: the simulator writes
// A to a file that reads back as CSR, with b and the true RSP vector x).
// Host code only: POSIX open / pwrite, no device work.
//
// File layout (little-endian):
//   bytes 0..127   header: magic "PCTCSR1\0", int64 n_rows, n_cols, nnz,
//                  then the byte offsets of the five sections below
//   row_ptr        int64 [n_rows + 1]   (global: row_ptr[0] = 0)
//   col            int32 [nnz]
//   val            float [nnz]
//   b              float [n_rows]
//   x_true         float [n_cols]
// Each section starts on a 4096-byte boundary.  A block of rows (an angle
// block of one GPU) is written at its global row and nonzero offsets, so the
// blocks of several writers land in one file that equals a single writer's.
#include <fcntl.h>
#include <unistd.h>

#include <cerrno>
#include <cstdio>
#include <cstring>
#include <vector>

#include "pct_kernels.cuh"

namespace {

constexpr char kMagic[8] = {'P', 'C', 'T', 'C', 'S', 'R', '1', '\0'};

struct Header {
  char magic[8];
  long long n_rows, n_cols, nnz;
  long long off_row_ptr, off_col, off_val, off_b, off_x;
  char pad[128 - 8 - 8 * 8];
};
static_assert(sizeof(Header) == 128, "header is 128 bytes");

long long page(long long v) { return (v + 4095) & ~4095LL; }

Header layout(long long n_rows, long long n_cols, long long nnz) {
  Header h;
  memset(&h, 0, sizeof(h));
  memcpy(h.magic, kMagic, 8);
  h.n_rows = n_rows;
  h.n_cols = n_cols;
  h.nnz = nnz;
  h.off_row_ptr = 4096;
  h.off_col = page(h.off_row_ptr + 8 * (n_rows + 1));
  h.off_val = page(h.off_col + 4 * nnz);
  h.off_b = page(h.off_val + 4 * nnz);
  h.off_x = page(h.off_b + 4 * n_rows);
  return h;
}

// all of [p, p + n) at offset off, or false
bool write_all(int fd, const void* p, long long n, long long off) {
  const char* c = (const char*)p;
  while (n > 0) {
    const long long chunk = n < (1LL << 30) ? n : (1LL << 30);
    const ssize_t w = pwrite(fd, c, (size_t)chunk, (off_t)off);
    if (w < 0) {
      if (errno == EINTR) continue;
      return false;
    }
    c += w;
    off += w;
    n -= w;
  }
  return true;
}

bool read_all(int fd, void* p, long long n, long long off) {
  char* c = (char*)p;
  while (n > 0) {
    const ssize_t r = pread(fd, c, (size_t)n, (off_t)off);
    if (r < 0 && errno == EINTR) continue;
    if (r <= 0) return false;
    c += r;
    off += r;
    n -= r;
  }
  return true;
}

pct_status io_fail(const char* what, const char* path) {
  char msg[512];
  snprintf(msg, sizeof(msg), "%s %s: %s", what, path, strerror(errno));
  return pct::set_error(PCT_EINVAL, msg);
}

}  // namespace

extern "C" pct_status pct_csr_file_create(const char* path, int64_t n_rows, int64_t n_cols, int64_t nnz,
                                          const float* x_true) {
  if (!path || n_rows < 0 || n_cols < 0 || nnz < 0 || (n_cols > 0 && !x_true))
    return pct::set_error(PCT_EINVAL, "pct_csr_file_create: bad arguments");
  const Header h = layout(n_rows, n_cols, nnz);
  const int fd = open(path, O_CREAT | O_WRONLY | O_TRUNC, 0644);
  if (fd < 0) return io_fail("cannot create", path);
  const long long zero = 0;
  const bool ok = write_all(fd, &h, sizeof(h), 0) && write_all(fd, &zero, 8, h.off_row_ptr) &&
                  write_all(fd, x_true, 4 * n_cols, h.off_x) && ftruncate(fd, (off_t)(h.off_x + 4 * n_cols)) == 0;
  const int e = errno;
  close(fd);
  errno = e;
  return ok ? PCT_OK : io_fail("cannot write", path);
}

extern "C" pct_status pct_csr_file_write_rows(const char* path, int64_t row0, int64_t n_rows, int64_t nz0,
                                              const int64_t* row_ptr, const int32_t* col, const float* val,
                                              const float* b) {
  if (!path || row0 < 0 || n_rows < 0 || nz0 < 0 || (n_rows > 0 && (!row_ptr || !b)))
    return pct::set_error(PCT_EINVAL, "pct_csr_file_write_rows: bad arguments");
  const int fd = open(path, O_WRONLY);
  if (fd < 0) return io_fail("cannot open", path);
  Header h;
  const int fdr = open(path, O_RDONLY);
  bool ok = fdr >= 0 && read_all(fdr, &h, sizeof(h), 0);
  if (fdr >= 0) close(fdr);
  if (!ok || memcmp(h.magic, kMagic, 8) != 0) {
    close(fd);
    return pct::set_error(PCT_EINVAL, "pct_csr_file_write_rows: not a file made by pct_csr_file_create");
  }
  const long long nnz = n_rows > 0 ? row_ptr[n_rows] - row_ptr[0] : 0;
  if (row0 + n_rows > h.n_rows || nz0 + nnz > h.nnz || (nnz > 0 && (!col || !val))) {
    close(fd);
    return pct::set_error(PCT_EINVAL, "pct_csr_file_write_rows: block beyond the file's sizes");
  }
  // global row pointers of rows row0 + 1 .. row0 + n_rows
  std::vector<long long> rp((size_t)n_rows);
  for (long long i = 0; i < n_rows; ++i) rp[i] = nz0 + (row_ptr[i + 1] - row_ptr[0]);
  ok = write_all(fd, rp.data(), 8 * n_rows, h.off_row_ptr + 8 * (row0 + 1)) &&
       write_all(fd, col, 4 * nnz, h.off_col + 4 * nz0) && write_all(fd, val, 4 * nnz, h.off_val + 4 * nz0) &&
       write_all(fd, b, 4 * n_rows, h.off_b + 4 * row0);
  const int e = errno;
  close(fd);
  errno = e;
  return ok ? PCT_OK : io_fail("cannot write", path);
}
