// kks_noalloc.cu -- a transpose entry point that allocates no memory.
//
// Some callers cannot allocate GPU memory at the moment they need a transpose:
// code that runs inside a custom allocator or an out-of-memory handler (where
// a nested cudaMalloc would recurse or fail), code on a path that must not
// synchronise the device (cudaFree does), or hosts whose GPU memory budget is
// fixed up front.  For them, spgemm_transpose_noalloc runs the same transpose
// kernels as spgemm_transpose, but its scratch (column counters, scatter
// cursors, staging of the scattered entries, the scan's partial sums and the
// status word) lives in one fixed file-scope device buffer, kScratchBytes
// large, that every GPU loading this library holds until the process exits.
//
// Rules of the buffer:
//  * Its device address is looked up once per device, on that device's first
//    call (cudaGetSymbolAddress); host code cannot use the symbol itself.
//  * Every call synchronises its stream (twice) and reads results into host
//    variables, so a call cannot be made while its stream is being captured
//    into a CUDA graph.
//  * All calls share it and it keeps the last call's contents; each call
//    clears what must start at zero.  Calls that overlap on the GPU (other
//    streams, other host threads) race on it: serialise them.
//  * A problem whose scratch would exceed kScratchBytes is rejected with
//    SPGEMM_ERR_OOM before any kernel runs (or, for columns longer than 16 384
//    entries whose sort buffers do not fit, after the counting pass).
#include <cstring>
#include <mutex>

#include "kkspgemm.h"
#include "kks_internal.h"

using namespace kks;

namespace {

constexpr size_t kScratchBytes = 32ull << 20;   // 32 MiB
constexpr size_t kStatusBytes = 256;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

std::mutex g_addr_mu;
unsigned char* g_addr[kMaxDevices] = {};

// Device address of the buffer on the current device (looked up once per device).
cudaError_t scratch_address(int dev, unsigned char** out) {
  std::lock_guard<std::mutex> lock(g_addr_mu);
  if (!g_addr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_addr[dev] = static_cast<unsigned char*>(p);
  }
  *out = g_addr[dev];
  return cudaSuccess;
}

spgemm_status_t to_status(cudaError_t e) {
  return e == cudaSuccess ? SPGEMM_OK : SPGEMM_ERR_CUDA;
}

}  // namespace

extern "C" spgemm_status_t spgemm_transpose_noalloc(const spgemm_csr_t* A, int64_t* At_rowptr, int32_t* At_colidx,
                                                    void* At_values, int64_t* perm, spgemm_stream_t stream) {
  if (!A || !At_rowptr) return SPGEMM_ERR_INVALID_ARG;
  if (A->nrows < 0 || A->ncols < 0 || A->nnz < 0 || !A->rowptr) return SPGEMM_ERR_INVALID_ARG;
  if (A->nnz > 0 && (!A->colidx || !At_colidx)) return SPGEMM_ERR_INVALID_ARG;
  if (At_values && A->nnz > 0 && !A->values) return SPGEMM_ERR_INVALID_ARG;
  if (A->dtype != SPGEMM_R32 && A->dtype != SPGEMM_R64) return SPGEMM_ERR_INVALID_ARG;
  if (A->nrows > 2147483647ll || A->ncols > 2147483647ll) return SPGEMM_ERR_INDEX_OVERFLOW;
  if (!A->rowptr_is_64 && A->nnz > 2147483647ll) return SPGEMM_ERR_INDEX_OVERFLOW;
  const size_t tmp_bytes = transpose_tmp_bytes(A->nrows, A->ncols, A->nnz);
  if (kStatusBytes + tmp_bytes > kScratchBytes) return SPGEMM_ERR_OOM;

  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess || dev < 0 || dev >= kMaxDevices) return SPGEMM_ERR_CUDA;
  unsigned char* base = nullptr;
  e = scratch_address(dev, &base);
  if (e != cudaSuccess) return SPGEMM_ERR_CUDA;
  int num_sms = 0, max_smem = 0;
  if (cudaDeviceGetAttribute(&num_sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess)
    return SPGEMM_ERR_CUDA;

  cudaStream_t s = (cudaStream_t)stream;
  LaunchCtx L;
  L.stream = s;
  L.num_sms = num_sms;
  L.max_smem_optin = max_smem;
  MatD M;
  M.rp = A->rowptr;
  M.cj = A->colidx;
  M.vx = At_values ? A->values : nullptr;
  M.nrows = A->nrows;
  M.ncols = A->ncols;
  M.nnz = A->nnz;
  M.rp64 = A->rowptr_is_64 ? 1 : 0;
  M.pad = 0;

  DevStatus* d_status = reinterpret_cast<DevStatus*>(base);
  void* tmp = base + kStatusBytes;
  unsigned long long longest = 0;   // host stack: the longest row of A^T
  DevStatus h_status;
  memset(&h_status, 0, sizeof(h_status));

  e = cudaMemsetAsync(d_status, 0, sizeof(DevStatus), s);
  if (e == cudaSuccess)
    e = launch_transpose_count(L, M, reinterpret_cast<long long*>(At_rowptr), tmp, &longest, d_status);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&h_status, d_status, sizeof(DevStatus), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return to_status(e);
  // out-of-range columns or row pointers that do not cover the entries: stop
  // before the scatter and sort read anything through them
  if (h_status.code == kDevBadIndex) return SPGEMM_ERR_BAD_INDEX;
  if (h_status.code != kDevOk) return SPGEMM_ERR_DEVICE_LIMIT;

  unsigned long long* gbuf = nullptr;
  long long gbuf_len = 0;
  int gchunks = 0;
  if ((long long)longest > 16384) {
    // sort buffers of rows longer than 16 384 entries come from the rest of the buffer
    gbuf_len = 1;
    while (gbuf_len < (long long)longest) gbuf_len <<= 1;
    const size_t off = (kStatusBytes + tmp_bytes + 255) & ~size_t(255);
    const size_t avail = kScratchBytes - off;
    long long nch = (long long)(avail / ((size_t)gbuf_len * 8));
    if (nch > num_sms) nch = num_sms;
    if (nch < 1) return SPGEMM_ERR_OOM;
    gbuf = reinterpret_cast<unsigned long long*>(base + off);
    gchunks = (int)nch;
  }
  e = launch_transpose_fill(L, M, (int)A->dtype, reinterpret_cast<const long long*>(At_rowptr), At_colidx, At_values,
                            reinterpret_cast<long long*>(perm), tmp, (long long)longest, gbuf, gbuf_len, gchunks,
                            d_status);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&h_status, d_status, sizeof(DevStatus), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return to_status(e);
  if (h_status.code == kDevBadIndex) return SPGEMM_ERR_BAD_INDEX;
  if (h_status.code != kDevOk) return SPGEMM_ERR_DEVICE_LIMIT;
  return SPGEMM_OK;
}
