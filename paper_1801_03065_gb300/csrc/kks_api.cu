// kks_api.cu -- the C ABI: handle, workspace, planning of the two phases.
//
// spgemm_symbolic runs the symbolic phase of Algorithm 2 on the GPU:
//   (1) compression pass 1: compressed row lengths of B, their scan
//   (2) row statistics rf_i (and rfc_i on the compressed B), per problem f_m,
//       maxrf and the compressed counterparts                      -> sync 1
//   (3) the 15 % rule: compress B iff f_m(compressed) / f_m < 0.85, pass 2
//   (4) row bins for the symbolic kernels                           -> sync 2
//   (5) symbolic kernels, scan of the row sizes, C row pointers
//   (6) row bins and accumulator pools for the numeric phase        -> sync 3
// spgemm_numeric (the numeric phase) then only launches the kernels of the
// planned bins: no synchronisation and no allocation.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "kkspgemm.h"
#include "kks_internal.h"

namespace kks {
size_t symbolic_team_bytes(int cls, int logT, int compressed);
size_t numeric_cta_bytes(int logT, int dtype, long long kwords);
long long numeric_rdense_vcap(long long kwords, int dtype, size_t max_smem, int small);
size_t numeric_spill_l1_bytes(int logT, int dtype);
size_t numeric_l2_chunk_bytes(long long slots, int dtype);
size_t masked_team_bytes(int cls, int logT, int dtype);
}  // namespace kks

using namespace kks;

std::atomic<long long> kks::g_launches{0};

namespace {

enum BufId {
  kBufInst, kBufArow0, kBufBrow0, kBufCnt, kBufBcp, kBufCsi, kBufCs, kBufRf, kBufRfc, kBufRowsize, kBufOffs,
  kBufScanTmp, kBufInstStats, kBufInstOut, kBufHist, kBufCursor, kBufSymRows, kBufNumRows, kBufSymPool,
  kBufNumPool2, kBufNumPool3, kBufStatus, kBufMaskRows, kBufMaskHist, kBufMaskPool, kBufTrTmp,
  kBufTrPool, kBufReuseRows, kBufReusePool, kBufBinCnt, kBufBinOfs, kBufMcCnt, kBufMcYcp, kBufMcCsi, kBufMcCs,
  kBufMcMax, kBufRapRf, kBufRapRtp, kBufRapRti, kBufRapRpe, kBufRapW, kBufRapCnt, kBufRapSymRows,
  kBufRapNumRows, kBufRapMeta, kBufRapTmp, kBufMcRows, kBufFetch, kBufLongB, kBufLongA, kBufRowSets, kBufRowSetCnt,
  kBufBlen, kNumBufs
};

// Row bins of a masked product, cached for numeric reuse on one pattern.
struct MaskPlan {
  bool valid = false;
  const void* sp = nullptr;
  const void* sj = nullptr;
  const void* xrp = nullptr;
  const void* xcj = nullptr;
  const void* yrp = nullptr;
  const void* ycj = nullptr;
  long long nrows = 0, snnz = 0;
  int dtype = 1;
  std::vector<std::pair<int, int>> cls_logT;
  std::vector<long long> off, cnt;
  int gchunks = 0;
  long long gslots = 0;
  bool sorted = false;   // every row of S strictly increasing: warp rows use column-set places
};

struct PatternId {
  const void* arp;
  const void* acj;
  const void* brp;
  const void* bcj;
  long long m, n, k, nnza, nnzb;
  int arp64, brp64;
  bool operator==(const PatternId& o) const {
    return arp == o.arp && acj == o.acj && brp == o.brp && bcj == o.bcj && m == o.m && n == o.n && k == o.k &&
           nnza == o.nnza && nnzb == o.nnzb && arp64 == o.arp64 && brp64 == o.brp64;
  }
};

// Plan of a Galerkin triple product (spgemm_rap_symbolic): the pattern it was
// made for and its numeric row classes.
struct RapPlan {
  bool ready = false;
  const void *arp = nullptr, *acj = nullptr, *prp = nullptr, *pcj = nullptr;
  long long n = 0, K = 0, nnza = 0, nnzp = 0, nnzc = 0;
  int arp64 = 0, prp64 = 0, dtype = 1, punit = 0;
  long long n_w = 0, n_c = 0;
  int logT_w = 1, logT_c = 1;
};

struct BinRun {
  int cls, logT, compressed;
  long long off, count;
  int hash;   // LpHash mode used for this bin (the tuner may change it)
  int part = 0;   // CTA hash classes: partitioning scheme (0 flat, 1 Team-Sequential + LL, 2 Thread-Parallel)
  int window = 0;   // W32 positions rows: bitmap window over the row's column sets
  int stage = 0;    // dense rows: B entries staged into shared memory by asynchronous copies
};

constexpr int kRing = 8;

}  // namespace

struct kks_handle {
  spgemm_options_t opt;
  int num_sms = 0;
  int max_smem = 0;
  void* buf[kNumBufs] = {};
  size_t cap[kNumBufs] = {};
  size_t total = 0;
  unsigned char* pinned = nullptr;   // readbacks and uploads
  unsigned char* pinned_dev = nullptr;   // its device alias (mapped memory)
  size_t pinned_bytes = 0;
  unsigned char* ring[kRing] = {};   // numeric table uploads
  size_t ring_bytes = 0;
  cudaEvent_t ring_ev[kRing] = {};
  int ring_next = 0;
  // plan
  bool ready = false;
  int ninst = 0;
  int dtype = 1;
  long long totalA = 0, totalB = 0;
  std::vector<InstD> inst;       // host copy of the device table
  std::vector<PatternId> pat;
  std::vector<BinRun> num_bins;
  long long num_kw_max = 0, num_kmax = 0;
  int num_spill_chunks = 0;
  long long num_spill_chunk_bytes = 0, num_spill_kw = 0, num_dense_kw = 0;
  int num_l1_logT = 0;
  spgemm_stats_t stats;
  MaskPlan reuse;
  MaskPlan masked;   // last plan of spgemm_masked (reused while the patterns are unchanged)
  bool tuned = false;
  bool positions_ok = false;   // every product of the plan runs on the compressed B
  bool row_sets = false;       // the symbolic phase records the column sets of its window rows
  bool b_sorted = false;       // every B row of the plan has increasing columns
  // tuner results by bin (class, log2 table, rows, dtype): a new plan of the
  // same problem reuses them instead of tuning again
  struct TuneEntry {
    int cls, logT, dtype, positions;
    long long count;
    BinRun pick;
  };
  std::vector<TuneEntry> tune_cache;
  RapPlan rap;
};

namespace {

spgemm_status_t cuda_status(cudaError_t e) {
  if (e == cudaSuccess) return SPGEMM_OK;
  if (e == cudaErrorMemoryAllocation) return SPGEMM_ERR_OOM;
  return SPGEMM_ERR_CUDA;
}

// CUDA failures are rare and otherwise opaque behind SPGEMM_ERR_CUDA: name the
// failing call on stderr.
#define KKS_CU(expr)                                                                              \
  do {                                                                                            \
    cudaError_t _e = (expr);                                                                      \
    if (_e != cudaSuccess) {                                                                      \
      fprintf(stderr, "kkspgemm: %s failed: %s (%s:%d)\n", #expr, cudaGetErrorString(_e), __FILE__, \
              __LINE__);                                                                          \
      return cuda_status(_e);                                                                     \
    }                                                                                             \
  } while (0)
#define KKS_ST(expr)                                        \
  do {                                                      \
    spgemm_status_t _s = (expr);                            \
    if (_s != SPGEMM_OK) return _s;                         \
  } while (0)

// Grows buffer id to at least bytes.  Only the planning calls allocate.
spgemm_status_t ensure(kks_handle* h, int id, size_t bytes) {
  if (bytes == 0) bytes = 16;
  if (h->cap[id] >= bytes) return SPGEMM_OK;
  size_t want = bytes + bytes / 4;
  size_t new_total = h->total - h->cap[id] + want;
  if (h->opt.workspace_limit_bytes > 0 && new_total > (size_t)h->opt.workspace_limit_bytes) {
    want = bytes;
    new_total = h->total - h->cap[id] + want;
    if (new_total > (size_t)h->opt.workspace_limit_bytes) return SPGEMM_ERR_OOM;
  }
  if (h->buf[id]) {
    cudaFree(h->buf[id]);
    h->total -= h->cap[id];
    h->buf[id] = nullptr;
    h->cap[id] = 0;
  }
  void* p = nullptr;
  cudaError_t e = cudaMalloc(&p, want);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return SPGEMM_ERR_OOM;
  }
  h->buf[id] = p;
  h->cap[id] = want;
  h->total += want;
  return SPGEMM_OK;
}

template <typename T>
T* B(kks_handle* h, int id) {
  return reinterpret_cast<T*>(h->buf[id]);
}

spgemm_status_t ensure_pinned(kks_handle* h, size_t bytes) {
  if (h->pinned_bytes >= bytes) return SPGEMM_OK;
  if (h->pinned) cudaFreeHost(h->pinned);
  h->pinned = nullptr;
  h->pinned_bytes = 0;
  size_t want = std::max<size_t>(bytes, 1 << 16);
  void* p = nullptr;
  if (cudaHostAlloc(&p, want, cudaHostAllocMapped) != cudaSuccess) {
    cudaGetLastError();
    return SPGEMM_ERR_OOM;
  }
  void* pd = nullptr;
  if (cudaHostGetDevicePointer(&pd, p, 0) != cudaSuccess) {
    cudaGetLastError();
    cudaFreeHost(p);
    return SPGEMM_ERR_CUDA;
  }
  h->pinned = (unsigned char*)p;
  h->pinned_dev = (unsigned char*)pd;
  h->pinned_bytes = want;
  return SPGEMM_OK;
}

LaunchCtx ctx(kks_handle* h, cudaStream_t s) {
  LaunchCtx L;
  L.stream = s;
  L.num_sms = h->num_sms;
  L.max_smem_optin = h->max_smem;
  return L;
}

ProbD prob(kks_handle* h) {
  ProbD P;
  P.inst = B<InstD>(h, kBufInst);
  P.arow0s = B<long long>(h, kBufArow0);
  P.brow0s = B<long long>(h, kBufBrow0);
  P.Bcp = B<long long>(h, kBufBcp);
  P.csi = B<int>(h, kBufCsi);
  P.cs = B<unsigned>(h, kBufCs);
  P.status = B<DevStatus>(h, kBufStatus);
  P.rsets = h->row_sets ? B<int2>(h, kBufRowSets) : nullptr;
  P.rcnt = h->row_sets ? B<int>(h, kBufRowSetCnt) : nullptr;
  P.ninst = h->ninst;
  P.hash_mode = h->opt.hash_function;
  return P;
}

spgemm_status_t check_csr(const spgemm_csr_t* M, bool need_values) {
  if (!M) return SPGEMM_ERR_INVALID_ARG;
  if (M->nrows < 0 || M->ncols < 0 || M->nnz < 0) return SPGEMM_ERR_INVALID_ARG;
  if (M->ncols > 2147483647ll || M->nrows > 2147483647ll) return SPGEMM_ERR_INDEX_OVERFLOW;
  if (!M->rowptr_is_64 && M->nnz > 2147483647ll) return SPGEMM_ERR_INDEX_OVERFLOW;
  if (!M->rowptr) return SPGEMM_ERR_INVALID_ARG;
  if (M->nnz > 0 && !M->colidx) return SPGEMM_ERR_INVALID_ARG;
  if (M->dtype != SPGEMM_R32 && M->dtype != SPGEMM_R64) return SPGEMM_ERR_INVALID_ARG;
  if (need_values && M->nnz > 0 && !M->values) return SPGEMM_ERR_INVALID_ARG;
  return SPGEMM_OK;
}

MatD matd(const spgemm_csr_t* M) {
  MatD d;
  d.rp = M->rowptr;
  d.cj = M->colidx;
  d.vx = M->values;
  d.nrows = M->nrows;
  d.ncols = M->ncols;
  d.nnz = M->nnz;
  d.rp64 = M->rowptr_is_64 ? 1 : 0;
  d.pad = 0;
  return d;
}

PatternId patid(const spgemm_csr_t* A, const spgemm_csr_t* Bm) {
  PatternId p;
  p.arp = A->rowptr;
  p.acj = A->colidx;
  p.brp = Bm->rowptr;
  p.bcj = Bm->colidx;
  p.m = A->nrows;
  p.n = A->ncols;
  p.k = Bm->ncols;
  p.nnza = A->nnz;
  p.nnzb = Bm->nnz;
  p.arp64 = A->rowptr_is_64;
  p.brp64 = Bm->rowptr_is_64;
  return p;
}

int device_code_to_status(int code) {
  switch (code) {
    case kDevOk: return SPGEMM_OK;
    case kDevBadIndex: return SPGEMM_ERR_BAD_INDEX;
    default: return SPGEMM_ERR_DEVICE_LIMIT;
  }
}

// Reads the device status word (already copied to host memory at *hs) and clears it.
spgemm_status_t consume_status(kks_handle* h, const DevStatus* hs, cudaStream_t s) {
  if (hs->code == kDevOk) return SPGEMM_OK;
  if (h->opt.verbose)
    fprintf(stderr, "kkspgemm: device status %d at site %d (info %lld)\n", hs->code, hs->where, hs->info);
  int code = hs->code;
  cudaMemsetAsync(h->buf[kBufStatus], 0, sizeof(DevStatus), s);
  cudaStreamSynchronize(s);
  return (spgemm_status_t)device_code_to_status(code);
}

long long kwords_of(long long k) { return (k + 31) >> 5; }

// Largest table (log2 slots) of a 1024-thread team that fits the shared memory
// (1 KB is left for the kernels' static scratch).
int cta_max_logT_sym(kks_handle* h, int comp) {
  int best = 4;
  for (int l = 4; l <= 20; ++l)
    if (symbolic_team_bytes(kClsC1024, l, comp) + 1024 <= (size_t)h->max_smem) best = l;
  return best;
}
int cta_max_logT_num(kks_handle* h, int dtype, long long kmax) {
  int best = 4;
  for (int l = 4; l <= 20; ++l)
    if (numeric_cta_bytes(l, dtype, kwords_of(kmax)) + 1024 <= (size_t)h->max_smem) best = l;
  return best;
}

BinCfg base_cfg(kks_handle* h) {
  BinCfg c;
  memset(&c, 0, sizeof(c));
  c.min_logT = 4;
  c.w8_max_logT = 5;
  c.w8_max_work = 64;
  c.w32_max_logT = 10;
  c.w32_max_work = 1ll << 15;
  c.c256_max_logT = 12;
  c.c256_max_work = 1ll << 17;
  c.dense_ok = h->opt.dense != 0;
  c.spill_ok = 1;
  c.force_cls = 0;
  c.force_logT = 0;
  c.slots_log2 = h->opt.slots_per_key_log2 > 0 ? h->opt.slots_per_key_log2 : 1;
  c.t1_max_work = 0;
  return c;
}

void clamp_cfg(kks_handle* h, BinCfg& c) {
  if (h->opt.l1_max_log2_slots > 0) {
    int l = std::max(4, (int)h->opt.l1_max_log2_slots);
    c.cta_max_logT = std::min(c.cta_max_logT, l);
    c.c256_max_logT = std::min(c.c256_max_logT, l);
    c.w32_max_logT = std::min(c.w32_max_logT, l);
    c.w8_max_logT = std::min(c.w8_max_logT, l);
  }
  if (h->opt.dense == 1) c.dense_ratio = 1ll << 40;
}

BinCfg sym_cfg(kks_handle* h, int comp) {
  BinCfg c = base_cfg(h);
  c.cta_max_logT = cta_max_logT_sym(h, comp);
  // 512-thread dense team: bitmap + chunk scratch in shared memory
  c.dense_max_kwords = ((long long)h->max_smem - 21 * 1024) / 4;
  // the bitmap (kw words) is preferred once the hash table (about 2u slots)
  // would reach half its size (plain rows: u * 128 >= k; 64 and 32 measured
  // slower on rows of random columns)
  c.dense_ratio = comp ? 4 : 128;
  // dense rows whose bitmap is at most 2^11 words (8 KB) take warp teams (on
  // the uniform-column rows of the 512-product batched workload: 13.5 ms for
  // the rows with bitmaps up to 2^11 words, which took 30.5 ms of the
  // 512-thread CTA kernel's 56.6 ms; with 2^12 and 2^13 words only 6 to 8
  // warps fit an SM and the warp rows ran 53 ms against 26.1 ms)
  c.dense_warp_log2w = 11;
  // one thread per row when the row has at most kT1SymKeys products
  c.t1_max_keys = kT1SymKeys;
  c.t1_max_work = kT1SymKeys;
  // on the compressed B the key bound min(rfc, k/32) counts compressed
  // products, of which many share a column set (that is why B was
  // compressed): a table of the next power of two >= the bound holds every key
  // and runs at low load, with half the sweep and twice the teams per SM
  if (comp && h->opt.slots_per_key_log2 == 0) c.slots_log2 = -1;
  clamp_cfg(h, c);
  return c;
}

// The paper's GPU meta-algorithm restated (Section 3.3): one team class for
// the whole problem, warp teams (kkmem, Thread-Sequential) when rows average
// fewer than 256 multiplications, CTA teams (kklp, Thread-Flat-Parallel)
// otherwise; the L1 table is sized from the average row size `est` (known in
// the numeric phase; estimated as flops / 8 in the symbolic phase); rows that
// do not fit L1 spill to an L2 table in global memory.
void plain_rule(BinCfg& c, double avg_flops, double est) {
  c.force_cls = avg_flops < 256.0 ? kClsW32 : kClsC256;
  const int cap = c.force_cls == kClsW32 ? c.w32_max_logT : c.c256_max_logT;
  int l = ilog2_ceil((long long)std::max(1.0, std::ceil(2.0 * est)));
  c.force_logT = std::max(c.min_logT, std::min(l, cap));
  c.dense_ok = 0;
  c.t1_max_work = 0;
}

BinCfg num_cfg(kks_handle* h, int dtype, long long kmax) {
  BinCfg c = base_cfg(h);
  c.cta_max_logT = cta_max_logT_num(h, dtype, kmax);
  // the dense accumulator works through shared-memory windows of the column
  // range, so any k fits; rows too large for a shared table always qualify,
  // and FP32 rows also once their size reaches k / 8 (FP64 rows of that size
  // stay in hash tables, which take fewer passes over their products)
  c.dense_max_kwords = 1ll << 40;
  c.dense_ratio = dtype == 1 ? 0 : 8;
  // dense rows whose values fit shared memory beside the k-bit bitmap keep
  // their values by rank (two passes over the products) instead of sweeping
  // the k columns in windows
  if (h->opt.dense != 1) {
    c.rdense_max = numeric_rdense_vcap(kwords_of(kmax), dtype, (size_t)h->max_smem, 0);
    c.rdense_small = numeric_rdense_vcap(kwords_of(kmax), dtype, (size_t)h->max_smem, 1);
  }
  // one thread per row: at most kT1MaxKeys columns of C and 64 products
  c.t1_max_keys = kT1MaxKeys;
  c.t1_max_work = 64;
  clamp_cfg(h, c);
  return c;
}

void set_default_options(spgemm_options_t* o) {
  memset(o, 0, sizeof(*o));
  o->compression = -1;
  o->compress_threshold = 0.85;
  o->l1_max_occupancy = 0.5;
  o->l1_max_log2_slots = 0;
  o->dense = -1;
  o->method = 0;
  o->workspace_limit_bytes = 0;
  o->pool_limit_bytes = 0;
  o->device = 0;
  o->hash_function = 1;
  o->verbose = 0;
  o->numeric_positions = 1;
  o->cta_partition = 0;
  o->window_positions = 1;
  o->sym_merge = 1;
}

// Long-row queue in buffer id (rows first, then three counters).
LongQueue long_queue(kks_handle* h, int id, long long rows) {
  LongQueue q;
  q.list = B<int>(h, id);
  const size_t off = (sizeof(int) * (size_t)(rows + 1) + 15) & ~size_t(15);
  q.ctr = reinterpret_cast<unsigned long long*>(reinterpret_cast<unsigned char*>(h->buf[id]) + off);
  return q;
}

// The 15 % rule of Section 3.2 for one product (mode: the option compression).
int compress_decision(int mode, double threshold, long long fm, long long fmc) {
  if (mode == 1) return 1;
  return (mode < 0 && fm > 0 && (double)fmc < threshold * (double)fm) ? 1 : 0;
}

// Upload the instance table through a pinned ring slot (numeric path).
spgemm_status_t upload_inst(kks_handle* h, cudaStream_t s) {
  size_t bytes = sizeof(InstD) * (size_t)h->ninst;
  if (h->ring_bytes < bytes) {
    for (int r = 0; r < kRing; ++r) {
      if (h->ring[r]) {
        cudaEventSynchronize(h->ring_ev[r]);
        cudaFreeHost(h->ring[r]);
        h->ring[r] = nullptr;
      }
    }
    size_t want = std::max<size_t>(bytes, 4096);
    for (int r = 0; r < kRing; ++r) {
      void* p = nullptr;
      if (cudaHostAlloc(&p, want, cudaHostAllocDefault) != cudaSuccess) {
        cudaGetLastError();
        return SPGEMM_ERR_OOM;
      }
      h->ring[r] = (unsigned char*)p;
    }
    h->ring_bytes = want;
  }
  const int r = h->ring_next;
  h->ring_next = (r + 1) % kRing;
  KKS_CU(cudaEventSynchronize(h->ring_ev[r]));
  memcpy(h->ring[r], h->inst.data(), bytes);
  KKS_CU(cudaMemcpyAsync(h->buf[kBufInst], h->ring[r], bytes, cudaMemcpyHostToDevice, s));
  KKS_CU(cudaEventRecord(h->ring_ev[r], s));
  return SPGEMM_OK;
}

// Read-back of `bytes` from device memory into the handle's pinned buffer
// (dst points into it) by a kernel writing the mapped alias.
cudaError_t to_host(kks_handle* h, void* dst, const void* src, size_t bytes, cudaStream_t s) {
  LaunchCtx L = ctx(h, s);
  return launch_copy_to_host(L, h->pinned_dev + ((unsigned char*)dst - h->pinned), src, bytes);
}

// Numeric rows whose warp-class bin takes output positions from the column sets.
long long rows_positions(const kks_handle* h) {
  long long n = 0;
  for (const BinRun& r : h->num_bins)
    if (r.compressed && (r.cls == kClsW8 || r.cls == kClsW32)) n += r.count;
  return n;
}

// ---------------------------------------------------------------------------
// symbolic (one plan of `count` products)
// ---------------------------------------------------------------------------
spgemm_status_t do_symbolic(kks_handle* h, int count, const spgemm_csr_t* A, const spgemm_csr_t* Bm,
                            int64_t* const* Crp, int64_t* nnzC, cudaStream_t s) {
  if (!h || count < 0 || (count > 0 && (!A || !Bm || !Crp || !nnzC))) return SPGEMM_ERR_INVALID_ARG;
  h->ready = false;
  long long totalA = 0, totalB = 0;
  int dtype = count > 0 ? (int)A[0].dtype : 1;
  for (int b = 0; b < count; ++b) {
    KKS_ST(check_csr(&A[b], false));
    KKS_ST(check_csr(&Bm[b], false));
    if (A[b].ncols != Bm[b].nrows) return SPGEMM_ERR_INVALID_ARG;
    if ((int)A[b].dtype != dtype || (int)Bm[b].dtype != dtype) return SPGEMM_ERR_INVALID_ARG;
    if (!Crp[b]) return SPGEMM_ERR_INVALID_ARG;
    totalA += A[b].nrows;
    totalB += Bm[b].nrows;
  }
  if (totalA >= 2147483647ll || totalB >= 2147483647ll) return SPGEMM_ERR_INDEX_OVERFLOW;
  KKS_CU(cudaSetDevice(h->opt.device));

  h->ninst = count;
  h->dtype = dtype;
  h->totalA = totalA;
  h->totalB = totalB;
  h->inst.assign(count, InstD{});
  h->pat.resize(count);
  std::vector<long long> arow0(count + 1, 0), brow0(count + 1, 0);
  for (int b = 0; b < count; ++b) {
    InstD& I = h->inst[b];
    memset(&I, 0, sizeof(I));
    I.A = matd(&A[b]);
    I.B = matd(&Bm[b]);
    I.arow0 = arow0[b];
    I.brow0 = brow0[b];
    I.Crp = reinterpret_cast<long long*>(Crp[b]);
    I.k = Bm[b].ncols;
    I.compressed = 0;
    arow0[b + 1] = arow0[b] + A[b].nrows;
    brow0[b + 1] = brow0[b] + Bm[b].nrows;
    h->pat[b] = patid(&A[b], &Bm[b]);
  }
  const int ni = std::max(count, 1);
  KKS_ST(ensure(h, kBufInst, sizeof(InstD) * ni));
  KKS_ST(ensure(h, kBufArow0, sizeof(long long) * (ni + 1)));
  KKS_ST(ensure(h, kBufBrow0, sizeof(long long) * (ni + 1)));
  KKS_ST(ensure(h, kBufCnt, sizeof(long long) * (totalB + 1)));
  KKS_ST(ensure(h, kBufBcp, sizeof(long long) * (totalB + 1)));
  if (h->opt.compression != 0) KKS_ST(ensure(h, kBufBlen, sizeof(longlong2) * (totalB + 1)));
  KKS_ST(ensure(h, kBufRf, sizeof(long long) * (totalA + 1)));
  KKS_ST(ensure(h, kBufRfc, sizeof(long long) * (totalA + 1)));
  KKS_ST(ensure(h, kBufRowsize, sizeof(long long) * (totalA + 1)));
  KKS_ST(ensure(h, kBufOffs, sizeof(long long) * (totalA + 1)));
  // stable binning: per-block bin counts of up to two passes and their scans
  const long long nbc = (long long)kNumBins * bin_blocks(totalA);
  KKS_ST(ensure(h, kBufBinCnt, sizeof(long long) * 2 * (nbc + 1)));
  KKS_ST(ensure(h, kBufBinOfs, sizeof(long long) * 2 * (nbc + 1)));
  KKS_ST(ensure(h, kBufScanTmp, scan_tmp_bytes(std::max(std::max(totalA, totalB), nbc) + 1)));
  KKS_ST(ensure(h, kBufInstStats, sizeof(unsigned long long) * (4 * ni + 1)));
  KKS_ST(ensure(h, kBufInstOut, sizeof(unsigned long long) * 2 * ni));
  KKS_ST(ensure(h, kBufHist, sizeof(unsigned long long) * 2 * kNumBins));
  KKS_ST(ensure(h, kBufCursor, sizeof(unsigned long long) * 2 * kNumBins));
  KKS_ST(ensure(h, kBufSymRows, sizeof(int) * (totalA + 1)));
  KKS_ST(ensure(h, kBufNumRows, sizeof(int) * (totalA + 1)));
  KKS_ST(ensure(h, kBufStatus, sizeof(DevStatus)));
  KKS_ST(ensure(h, kBufFetch, 16));
  KKS_ST(ensure(h, kBufLongB, sizeof(int) * (totalB + 1) + 64));
  KKS_ST(ensure(h, kBufLongA, sizeof(int) * (totalA + 1) + 64));
  KKS_ST(ensure(h, kBufCsi, 16));
  KKS_ST(ensure(h, kBufCs, 16));

  const size_t up_bytes = sizeof(InstD) * ni + 2 * sizeof(long long) * (ni + 1);
  const size_t rd_bytes = sizeof(unsigned long long) * (4 * ni + 2 * ni + 2 * kNumBins + 8) + sizeof(DevStatus);
  KKS_ST(ensure_pinned(h, up_bytes + rd_bytes + sizeof(unsigned long long) * 2 * kNumBins));
  unsigned char* up = h->pinned;
  unsigned char* rd = h->pinned + up_bytes;
  memcpy(up, h->inst.data(), sizeof(InstD) * count);
  memcpy(up + sizeof(InstD) * ni, arow0.data(), sizeof(long long) * (count + 1));
  memcpy(up + sizeof(InstD) * ni + sizeof(long long) * (ni + 1), brow0.data(), sizeof(long long) * (count + 1));
  KKS_CU(cudaMemcpyAsync(h->buf[kBufInst], up, sizeof(InstD) * ni, cudaMemcpyHostToDevice, s));
  KKS_CU(cudaMemcpyAsync(h->buf[kBufArow0], up + sizeof(InstD) * ni, sizeof(long long) * (count + 1),
                         cudaMemcpyHostToDevice, s));
  KKS_CU(cudaMemcpyAsync(h->buf[kBufBrow0], up + sizeof(InstD) * ni + sizeof(long long) * (ni + 1),
                         sizeof(long long) * (count + 1), cudaMemcpyHostToDevice, s));
  KKS_CU(cudaMemsetAsync(h->buf[kBufInstStats], 0, sizeof(unsigned long long) * (4 * ni + 1), s));
  KKS_CU(cudaMemsetAsync(h->buf[kBufInstOut], 0, sizeof(unsigned long long) * 2 * ni, s));
  KKS_CU(cudaMemsetAsync(h->buf[kBufHist], 0, sizeof(unsigned long long) * 2 * kNumBins, s));
  KKS_CU(cudaMemsetAsync(h->buf[kBufStatus], 0, sizeof(DevStatus), s));

  LaunchCtx L = ctx(h, s);
  ProbD P = prob(h);
  const bool comp_on = h->opt.compression != 0;

  // (1) compression pass 1 and (2) row statistics
  if (comp_on) {
    KKS_CU(launch_compress_count(L, P, totalB, B<long long>(h, kBufCnt),
                                 B<unsigned long long>(h, kBufInstStats) + 4 * ni, long_queue(h, kBufLongB, totalB),
                                 B<longlong2>(h, kBufBlen)));
    KKS_CU(launch_scan(L, B<long long>(h, kBufCnt), B<long long>(h, kBufBcp), totalB, h->buf[kBufScanTmp]));
  }
  KKS_CU(launch_row_stats(L, P, totalA, comp_on ? 1 : 0, B<long long>(h, kBufRf),
                          comp_on ? B<long long>(h, kBufRfc) : nullptr, B<unsigned long long>(h, kBufInstStats),
                          long_queue(h, kBufLongA, totalA), comp_on ? B<longlong2>(h, kBufBlen) : nullptr));
  unsigned long long* h_stats = (unsigned long long*)rd;
  long long* h_nbc = (long long*)(rd + sizeof(unsigned long long) * 4 * ni);
  DevStatus* h_status = (DevStatus*)(rd + sizeof(unsigned long long) * (4 * ni + 2 * ni + 2 * kNumBins + 8));
  unsigned long long* h_unsorted = (unsigned long long*)(rd + sizeof(unsigned long long) * (4 * ni + 2 * ni + 2 * kNumBins));
  unsigned long long* d_hist = B<unsigned long long>(h, kBufHist);
  unsigned long long* h_hist = (unsigned long long*)(rd + sizeof(unsigned long long) * (4 * ni + 2 * ni));
  *h_nbc = 0;
  *h_unsorted = 1;
  BinCfg cfg_c = sym_cfg(h, 1), cfg_u = sym_cfg(h, 0);
  std::vector<unsigned long long> hist(2 * kNumBins, 0);
  // With compression on and no per-problem rule, the 15 % rule is taken on the
  // device and the compressed B is sized by nnz(B): the statistics are read at
  // the same synchronisation as the symbolic bins (one host round trip fewer).
  long long nnzB_all = 0;
  for (int b = 0; b < count; ++b) nnzB_all += Bm[b].nnz;
  bool merged = comp_on && h->opt.method != 1;
  if (merged && (ensure(h, kBufCsi, sizeof(int) * (nnzB_all + 1)) != SPGEMM_OK ||
                 ensure(h, kBufCs, sizeof(unsigned) * (nnzB_all + 1)) != SPGEMM_OK)) {
    merged = false;   // no room for the bound: size it by the counted runs after a synchronisation
    KKS_ST(ensure(h, kBufCsi, 16));
    KKS_ST(ensure(h, kBufCs, 16));
  }
  if (merged) {
    P = prob(h);
    KKS_CU(launch_decide_compression(L, B<InstD>(h, kBufInst), B<unsigned long long>(h, kBufInstStats), count,
                                     h->opt.compression, h->opt.compress_threshold));
    KKS_CU(launch_compress_fill(L, P, totalB, B<int>(h, kBufCsi), B<unsigned>(h, kBufCs), long_queue(h, kBufLongB, totalB)));
    for (int pass = 0; pass < 2; ++pass) {
      BinCfg c = pass ? cfg_c : cfg_u;
      KKS_CU(launch_bin_count(L, P, totalA, pass ? 2 : 3, B<long long>(h, kBufRf), B<long long>(h, kBufRfc), nullptr,
                              c, d_hist + pass * kNumBins, B<long long>(h, kBufBinCnt) + pass * (nbc + 1)));
      KKS_CU(launch_scan(L, B<long long>(h, kBufBinCnt) + pass * (nbc + 1),
                         B<long long>(h, kBufBinOfs) + pass * (nbc + 1), nbc, h->buf[kBufScanTmp]));
    }
    KKS_CU(to_host(h, h_hist, d_hist, sizeof(unsigned long long) * 2 * kNumBins, s));
  }
  KKS_CU(to_host(h, h_stats, h->buf[kBufInstStats], sizeof(unsigned long long) * 4 * ni, s));
  if (comp_on) {
    KKS_CU(to_host(h, h_nbc, B<long long>(h, kBufBcp) + totalB, sizeof(long long), s));
    KKS_CU(to_host(h, h_unsorted, B<unsigned long long>(h, kBufInstStats) + 4 * ni, sizeof(unsigned long long), s));
  }
  KKS_CU(to_host(h, h_status, h->buf[kBufStatus], sizeof(DevStatus), s));
  KKS_CU(cudaStreamSynchronize(s));
  KKS_ST(consume_status(h, h_status, s));
  h->b_sorted = comp_on && *h_unsorted == 0;
  if (merged)
    for (int t = 0; t < 2 * kNumBins; ++t) hist[t] = h_hist[t];

  // (3) the 15 % rule, per product (the same test as the device's)
  long long fm_all = 0, fmc_all = 0, maxrf_all = 0, maxrfc_all = 0;
  int any_comp = 0, ncomp = 0;
  for (int b = 0; b < count; ++b) {
    long long fm = (long long)h_stats[4 * b], fmc = (long long)h_stats[4 * b + 2];
    fm_all += fm;
    fmc_all += fmc;
    maxrf_all = std::max(maxrf_all, (long long)h_stats[4 * b + 1]);
    maxrfc_all = std::max(maxrfc_all, (long long)h_stats[4 * b + 3]);
    int c = compress_decision(h->opt.compression, h->opt.compress_threshold, fm, fmc);
    h->inst[b].compressed = c;
    any_comp |= c;
    ncomp += c;
  }
  if (!merged) {
    if (any_comp) {
      const long long nbcomp = *h_nbc;
      KKS_ST(ensure(h, kBufCsi, sizeof(int) * (nbcomp + 1)));
      KKS_ST(ensure(h, kBufCs, sizeof(unsigned) * (nbcomp + 1)));
      P = prob(h);
      memcpy(up, h->inst.data(), sizeof(InstD) * count);
      KKS_CU(cudaMemcpyAsync(h->buf[kBufInst], up, sizeof(InstD) * count, cudaMemcpyHostToDevice, s));
      KKS_CU(launch_compress_fill(L, P, totalB, B<int>(h, kBufCsi), B<unsigned>(h, kBufCs), long_queue(h, kBufLongB, totalB)));
    }
    // (4) symbolic bins: the compressed and plain rows use separate bin ranges
    if (h->opt.method == 1 && totalA > 0) {
      const double avg = (double)fm_all / (double)totalA;
      plain_rule(cfg_u, avg, (double)fm_all / 8.0 / (double)totalA);
      plain_rule(cfg_c, avg, (double)fmc_all / 8.0 / (double)totalA);
    }
    // one launch per compression flag keeps the device bin function simple
    // (rows of the other kind land in the class-none bin of that launch and are ignored)
    for (int pass = 0; pass < 2; ++pass) {
      if (pass == 1 && !any_comp) break;
      if (pass == 0 && ncomp == count && count > 0) continue;
      KKS_CU(cudaMemsetAsync(d_hist, 0, sizeof(unsigned long long) * kNumBins, s));
      BinCfg c = pass ? cfg_c : cfg_u;
      KKS_CU(launch_bin_count(L, P, totalA, pass ? 2 : 3, B<long long>(h, kBufRf), B<long long>(h, kBufRfc), nullptr,
                              c, d_hist, B<long long>(h, kBufBinCnt) + pass * (nbc + 1)));
      KKS_CU(launch_scan(L, B<long long>(h, kBufBinCnt) + pass * (nbc + 1),
                         B<long long>(h, kBufBinOfs) + pass * (nbc + 1), nbc, h->buf[kBufScanTmp]));
      KKS_CU(to_host(h, h_hist, d_hist, sizeof(unsigned long long) * kNumBins, s));
      KKS_CU(cudaStreamSynchronize(s));
      for (int t = 0; t < kNumBins; ++t) hist[pass * kNumBins + t] = h_hist[t];
    }
  }
  // offsets over both passes (class-none rows are not listed)
  std::vector<long long> off(2 * kNumBins + 1, 0);
  for (int t = 0; t < 2 * kNumBins; ++t) {
    long long c = (bin_cls(t % kNumBins) == kClsNone) ? 0 : (long long)hist[t];
    off[t + 1] = off[t] + c;
  }
  unsigned long long* h_cur = (unsigned long long*)(rd + rd_bytes);
  for (int t = 0; t < 2 * kNumBins; ++t) h_cur[t] = (unsigned long long)off[t];
  KKS_CU(cudaMemcpyAsync(h->buf[kBufCursor], h_cur, sizeof(unsigned long long) * 2 * kNumBins,
                         cudaMemcpyHostToDevice, s));
  for (int pass = 0; pass < 2; ++pass) {
    if (pass == 1 && !any_comp) break;
    if (pass == 0 && ncomp == count && count > 0) continue;
    BinCfg c = pass ? cfg_c : cfg_u;
    KKS_CU(launch_bin_scatter(L, P, totalA, pass ? 2 : 3, B<long long>(h, kBufRf), B<long long>(h, kBufRfc),
                              B<long long>(h, kBufRowsize), c, B<unsigned long long>(h, kBufCursor) + pass * kNumBins,
                              B<long long>(h, kBufBinOfs) + pass * (nbc + 1), B<int>(h, kBufSymRows)));
  }

  // Column sets of the window rows for the numeric phase (compressed rows with
  // sorted B rows, positions on): kRowSetCap slots per row, for plans of at
  // most 2 M rows (512 B per row); rows without a record keep -1.
  h->row_sets = false;
  if (any_comp && h->b_sorted && h->opt.numeric_positions && (h->opt.window_positions & 1) &&
      totalA <= (2ll << 20)) {
    if (ensure(h, kBufRowSets, sizeof(int2) * (size_t)kRowSetCap * (size_t)(totalA + 1)) == SPGEMM_OK &&
        ensure(h, kBufRowSetCnt, sizeof(int) * (size_t)(totalA + 1)) == SPGEMM_OK) {
      h->row_sets = true;
      KKS_CU(cudaMemsetAsync(h->buf[kBufRowSetCnt], 0xff, sizeof(int) * (size_t)(totalA + 1), s));
    }
  }
  P = prob(h);

  // (5) symbolic kernels, bin by bin
  int nbins_sym = 0;
  for (int t = 0; t < 2 * kNumBins; ++t) {
    const long long cnt = off[t + 1] - off[t];
    if (cnt == 0) continue;
    const int bin = t % kNumBins;
    const int comp = t / kNumBins;
    ++nbins_sym;
    SymLaunch S;
    memset(&S, 0, sizeof(S));
    S.cls = bin_cls(bin);
    S.logT = bin_logT(bin);
    S.rows = B<int>(h, kBufSymRows) + off[t];
    S.nrows = cnt;
    S.compressed = comp;
    S.max_occ = h->opt.l1_max_occupancy;
    S.fetch = B<unsigned long long>(h, kBufFetch);
    S.window = (comp && h->b_sorted && (h->opt.window_positions & 1)) ? 1 : 0;
    S.merge = (S.window && h->opt.sym_merge) ? 1 : 0;
    long long kmax = 0;
    for (int b = 0; b < count; ++b) kmax = std::max<long long>(kmax, h->inst[b].k);
    // dense rows only come from products whose bitmap fits (checked per row)
    S.kwords_max = std::min(kwords_of(kmax), (comp ? cfg_c : cfg_u).dense_max_kwords);
    if (S.cls == kClsSpill) {
      const BinCfg& c = comp ? cfg_c : cfg_u;
      S.l1_logT = c.cta_max_logT;
      S.l2_chunk_slots = 1ll << S.logT;
      const long long chunk = S.l2_chunk_slots * (comp ? 8 : 4);
      long long pool_limit = h->opt.pool_limit_bytes > 0 ? h->opt.pool_limit_bytes : (8ll << 30);
      long long nch = std::min<long long>(std::min<long long>(2ll * h->num_sms, cnt), pool_limit / chunk);
      if (nch < 1) return SPGEMM_ERR_OOM;
      KKS_ST(ensure(h, kBufSymPool, (size_t)(nch * chunk)));
      S.l2_pool = h->buf[kBufSymPool];
      S.nchunks = (int)nch;
    }
    KKS_CU(launch_symbolic(L, P, S, B<long long>(h, kBufRowsize)));
  }

  // C row pointers
  KKS_CU(launch_scan(L, B<long long>(h, kBufRowsize), B<long long>(h, kBufOffs), totalA, h->buf[kBufScanTmp]));
  KKS_CU(launch_write_rowptr(L, P, totalA, B<long long>(h, kBufOffs), B<long long>(h, kBufRowsize),
                             B<unsigned long long>(h, kBufInstOut)));

  // (6) numeric bins
  long long kmax = 0;
  for (int b = 0; b < count; ++b) kmax = std::max<long long>(kmax, h->inst[b].k);
  BinCfg ncfg = num_cfg(h, dtype, kmax);
  if (h->opt.method == 1 && totalA > 0) {
    // the plain rule sizes L1 from the average row of C: read nnz(C) first
    unsigned long long* h_o = (unsigned long long*)(rd + sizeof(unsigned long long) * 4 * ni);
    KKS_CU(to_host(h, h_o, h->buf[kBufInstOut], sizeof(unsigned long long) * 2 * ni, s));
    KKS_CU(cudaStreamSynchronize(s));
    long long nz = 0;
    for (int b = 0; b < count; ++b) nz += (long long)h_o[2 * b];
    plain_rule(ncfg, (double)fm_all / (double)totalA, (double)nz / (double)totalA);
  }
  KKS_CU(cudaMemsetAsync(d_hist, 0, sizeof(unsigned long long) * kNumBins, s));
  KKS_CU(launch_bin_count(L, P, totalA, 1, B<long long>(h, kBufRf), nullptr, B<long long>(h, kBufRowsize), ncfg,
                          d_hist, B<long long>(h, kBufBinCnt)));
  KKS_CU(launch_scan(L, B<long long>(h, kBufBinCnt), B<long long>(h, kBufBinOfs), nbc, h->buf[kBufScanTmp]));
  unsigned long long* h_out = (unsigned long long*)(rd + sizeof(unsigned long long) * 4 * ni);
  KKS_CU(to_host(h, h_hist, d_hist, sizeof(unsigned long long) * kNumBins, s));
  KKS_CU(to_host(h, h_out, h->buf[kBufInstOut], sizeof(unsigned long long) * 2 * ni, s));
  KKS_CU(to_host(h, h_status, h->buf[kBufStatus], sizeof(DevStatus), s));
  KKS_CU(cudaStreamSynchronize(s));
  KKS_ST(consume_status(h, h_status, s));

  std::vector<long long> noff(kNumBins + 1, 0);
  for (int t = 0; t < kNumBins; ++t) {
    long long c = (bin_cls(t) == kClsNone) ? 0 : (long long)h_hist[t];
    noff[t + 1] = noff[t] + c;
  }
  for (int t = 0; t < kNumBins; ++t) h_cur[t] = (unsigned long long)noff[t];
  KKS_CU(cudaMemcpyAsync(h->buf[kBufCursor], h_cur, sizeof(unsigned long long) * kNumBins, cudaMemcpyHostToDevice,
                         s));
  KKS_CU(launch_bin_scatter(L, P, totalA, 1, B<long long>(h, kBufRf), nullptr, B<long long>(h, kBufRowsize), ncfg,
                            B<unsigned long long>(h, kBufCursor), B<long long>(h, kBufBinOfs), B<int>(h, kBufNumRows)));

  h->num_bins.clear();
  const bool positions_ok = h->opt.numeric_positions != 0 && count > 0 && ncomp == count;
  h->positions_ok = positions_ok;
  long long spill_rows = 0;
  int spill_logT = 0;
  long long cls_rows[kNumClasses] = {0};
  for (int t = 0; t < kNumBins; ++t) {
    const int cls = bin_cls(t);
    cls_rows[cls] += (long long)h_hist[t];
    const long long cnt = noff[t + 1] - noff[t];
    if (cnt == 0) continue;
    // warp-class rows of a plan whose products all run on the compressed B
    // take their output positions from the column sets
    const int pos = (positions_ok && (cls == kClsW8 || cls == kClsW32)) ? 1 : 0;
    h->num_bins.push_back(BinRun{cls, bin_logT(t), pos, noff[t], cnt, h->opt.hash_function,
                                 (cls == kClsC256 || cls == kClsC1024) ? h->opt.cta_partition : 0,
                                 (pos && cls == kClsW32 && h->b_sorted && (h->opt.window_positions & 2)) ? 1 : 0,
                                 cls == kClsDense ? h->opt.stage_b : 0});
    if (cls == kClsSpill) {
      spill_rows += cnt;
      spill_logT = std::max(spill_logT, bin_logT(t));
    }
  }
  // heaviest classes first so the long rows start early
  std::stable_sort(h->num_bins.begin(), h->num_bins.end(), [](const BinRun& a, const BinRun& b) {
    auto key = [](const BinRun& r) {
      return r.cls == kClsSpill ? 7 : r.cls == kClsDense ? 6 : r.cls == kClsT1 ? 0 : r.cls;
    };
    return key(a) * 64 + a.logT > key(b) * 64 + b.logT;
  });
  const int vt = dtype == 1 ? 8 : 4;
  long long pool_limit = h->opt.pool_limit_bytes > 0 ? h->opt.pool_limit_bytes : (8ll << 30);
  h->num_kmax = kmax;
  h->num_kw_max = kwords_of(kmax);
  h->num_dense_kw = std::min(kwords_of(kmax), ncfg.dense_max_kwords);
  h->num_spill_chunks = 0;
  if (spill_rows > 0) {
    const long long slots = 1ll << spill_logT;
    const long long chunk = (long long)numeric_l2_chunk_bytes(slots, dtype);
    const long long chunk2 = 2 * h->num_kw_max * 4;
    long long nch = std::min<long long>(std::min<long long>(2ll * h->num_sms, spill_rows), pool_limit / (chunk + chunk2));
    if (nch < 1) return SPGEMM_ERR_OOM;
    KKS_ST(ensure(h, kBufNumPool2, (size_t)(nch * chunk)));
    KKS_ST(ensure(h, kBufNumPool3, (size_t)(nch * chunk2)));
    KKS_CU(cudaMemsetAsync(h->buf[kBufNumPool3], 0, (size_t)(nch * chunk2), s));
    h->num_spill_chunks = (int)nch;
    h->num_spill_chunk_bytes = chunk;
    h->num_l1_logT = ncfg.cta_max_logT;
  }

  // results
  long long nnz_all = 0, maxrs_all = 0;
  for (int b = 0; b < count; ++b) {
    nnzC[b] = (int64_t)h_out[2 * b];
    nnz_all += (long long)h_out[2 * b];
    maxrs_all = std::max(maxrs_all, (long long)h_out[2 * b + 1]);
  }
  spgemm_stats_t& st = h->stats;
  memset(&st, 0, sizeof(st));
  if (count > 0) {
    st.m = A[0].nrows;
    st.n = A[0].ncols;
    st.k = Bm[0].ncols;
    st.nnzA = A[0].nnz;
    st.nnzB = Bm[0].nnz;
  }
  st.f_m = fm_all;
  st.maxrf = maxrf_all;
  st.f_m_compressed = comp_on ? fmc_all : fm_all;
  st.maxrf_compressed = comp_on ? maxrfc_all : maxrf_all;
  st.CF = fm_all > 0 ? (double)st.f_m_compressed / (double)fm_all : 1.0;
  st.CMRF = maxrf_all > 0 ? (double)st.maxrf_compressed / (double)maxrf_all : 1.0;
  st.compressed = any_comp;
  st.nbins_symbolic = nbins_sym;
  st.nbins_numeric = (int)h->num_bins.size();
  st.nnzC = nnz_all;
  st.maxrs = maxrs_all;
  st.ars = totalA > 0 ? (double)nnz_all / (double)totalA : 0.0;
  st.workspace_bytes = (int64_t)h->total;
  for (int c = 0; c < kNumClasses; ++c) st.bin_rows_numeric[c] = cls_rows[c];
  st.rows_positions = rows_positions(h);
  h->tuned = false;
  h->ready = true;
  return SPGEMM_OK;
}

// Launch the numeric kernel of one bin with its (possibly tuned) configuration.
cudaError_t launch_bin(kks_handle* h, const BinRun& r, cudaStream_t s) {
  LaunchCtx L = ctx(h, s);
  ProbD P = prob(h);
  P.hash_mode = r.hash;
  NumLaunch S;
  memset(&S, 0, sizeof(S));
  S.cls = r.cls;
  S.logT = r.logT;
  S.rows = B<int>(h, kBufNumRows) + r.off;
  S.nrows = r.count;
  S.dtype = h->dtype;
  S.kwords_max = h->num_kw_max;
  S.kmax = h->num_kmax;
  S.max_occ = h->opt.l1_max_occupancy;
  S.positions = (r.compressed && (r.cls == kClsW8 || r.cls == kClsW32)) ? 1 : 0;
  S.b_sorted = h->b_sorted ? 1 : 0;
  S.fetch = B<unsigned long long>(h, kBufFetch);
  S.part = (r.cls == kClsC256 || r.cls == kClsC1024) ? r.part : 0;
  S.window = (S.positions && r.cls == kClsW32) ? r.window : 0;
  S.stage = r.cls == kClsDense ? r.stage : 0;
  if (r.cls == kClsDense) {
    S.kwords_max = h->num_dense_kw;
  } else if (r.cls == kClsSpill) {
    S.pool = h->buf[kBufNumPool2];
    S.chunk_bytes = h->num_spill_chunk_bytes;
    S.pool2 = h->buf[kBufNumPool3];
    S.nchunks = h->num_spill_chunks;
    S.l1_logT = h->num_l1_logT;
  }
  cudaError_t e = launch_numeric(L, P, S);
  if (e != cudaSuccess)
    fprintf(stderr, "kkspgemm: numeric bin (class %d, log2 table %d, %lld rows, %d chunks, %lld bitmap words) failed\n",
            r.cls, r.logT, r.count, S.nchunks, S.kwords_max);
  return e;
}

// The autotuner: for every hash-table bin, time the kernel configurations that
// are valid for its rows (table one size larger, the next team class up or
// down, the other hash function) on the bin itself and keep the fastest.  Each
// launch computes the bin's rows of C completely, so tuning runs inside the
// first numeric call and leaves a correct C behind.
spgemm_status_t tune_numeric(kks_handle* h, cudaStream_t s) {
  const int cta_max = cta_max_logT_num(h, h->dtype, h->num_kmax);
  // timing events only when some bin is not in the cache (a re-plan of a
  // tuned problem costs no device work here)
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  auto events = [&]() -> cudaError_t {
    if (e0) return cudaSuccess;
    cudaError_t e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    return e;
  };
  int changed = 0;
  for (BinRun& r : h->num_bins) {
    if (r.cls != kClsW8 && r.cls != kClsW32 && r.cls != kClsC256 && r.cls != kClsC1024 &&
        !(r.cls == kClsDense && r.logT == 0 && h->b_sorted))
      continue;
    bool cached = false;
    for (const auto& te : h->tune_cache) {
      if (te.cls == r.cls && te.logT == r.logT && te.count == r.count && te.dtype == h->dtype &&
          te.positions == r.compressed) {
        BinRun p = te.pick;
        p.off = r.off;
        p.count = r.count;
        if (p.cls != r.cls || p.logT != r.logT || p.hash != r.hash || p.compressed != r.compressed ||
            p.part != r.part || p.window != r.window || p.stage != r.stage)
          ++changed;
        r = p;
        cached = true;
        break;
      }
    }
    if (cached) continue;
    const int cls0 = r.cls, logT0 = r.logT, pos0 = r.compressed;
    std::vector<BinRun> cand;
    cand.push_back(r);
    BinRun x = r;
    if (r.cls == kClsDense) {
      x.stage = 1 - r.stage;   // staged B entries against per-product loads
      cand.push_back(x);
    } else {
      x.hash = 1 - r.hash;
      cand.push_back(x);
    }
    if (h->positions_ok && (r.cls == kClsW8 || r.cls == kClsW32)) {
      x = r;
      x.compressed = 1 - r.compressed;   // column-set positions against the hash-and-sort kernel
      x.window = 0;
      cand.push_back(x);
    }
    if (r.compressed && r.cls == kClsW32 && h->b_sorted) {
      x = r;
      x.window = 1 - r.window;   // bitmap window against hash tables of column sets
      cand.push_back(x);
    }
    if (r.cls == kClsC256 || r.cls == kClsC1024) {
      // the other partitioning schemes of Section 3.1.1
      for (int part = 0; part <= 2; ++part) {
        if (part == r.part) continue;
        x = r;
        x.part = part;
        cand.push_back(x);
      }
    }
    auto max_logT = [&](int cls) {
      return cls == kClsW8 ? 5 : cls == kClsW32 ? 10 : cls == kClsC256 ? std::min(12, cta_max) : cta_max;
    };
    if (r.cls != kClsDense && r.logT + 1 <= max_logT(r.cls)) {
      x = r;
      x.logT = r.logT + 1;
      cand.push_back(x);
    }
    const int up = r.cls == kClsW8 ? kClsW32 : r.cls == kClsW32 ? kClsC256 : r.cls == kClsC256 ? kClsC1024 : 0;
    if (up && r.logT <= max_logT(up)) {
      x = r;
      x.cls = up;
      if (up != kClsW32) x.compressed = 0;
      x.window = (x.compressed && up == kClsW32 && h->b_sorted && (h->opt.window_positions & 2)) ? 1 : 0;
      cand.push_back(x);
    }
    if ((r.cls == kClsC256 || r.cls == kClsC1024) && h->opt.dense != 0) {
      x = r;   // the accumulator: dense windows of the row's columns instead of the hash table
      x.cls = kClsDense;
      x.logT = 0;
      x.compressed = 0;
      x.part = 0;
      cand.push_back(x);
      // or the rank-dense rows, when every row of the bin (at most 2^(logT-1)
      // columns) fits their values
      for (int small = 1; small >= 0; --small) {
        if (numeric_rdense_vcap(h->num_kw_max, h->dtype, (size_t)h->max_smem, small) >= (1ll << (r.logT - 1))) {
          x.logT = small ? 2 : 1;
          cand.push_back(x);
          break;
        }
      }
    }
    const int down = r.cls == kClsW32 ? kClsW8 : r.cls == kClsC256 ? kClsW32 : r.cls == kClsC1024 ? kClsC256 : 0;
    if (down && r.logT <= max_logT(down)) {
      x = r;
      x.cls = down;
      x.compressed = (h->positions_ok && (down == kClsW8 || down == kClsW32)) ? 1 : 0;
      x.window = (x.compressed && down == kClsW32 && h->b_sorted && (h->opt.window_positions & 2)) ? 1 : 0;
      cand.push_back(x);
    }
    float best = 1e30f;
    BinRun pick = r;
    KKS_CU(events());
    for (const BinRun& cd : cand) {
      float t_min = 1e30f;
      for (int rep = 0; rep < 3; ++rep) {
        KKS_CU(cudaEventRecord(e0, s));
        KKS_CU(launch_bin(h, cd, s));
        KKS_CU(cudaEventRecord(e1, s));
        KKS_CU(cudaEventSynchronize(e1));
        float ms = 0.f;
        KKS_CU(cudaEventElapsedTime(&ms, e0, e1));
        t_min = std::min(t_min, ms);
      }
      if (t_min < best) {
        best = t_min;
        pick = cd;
      }
    }
    if (pick.cls != r.cls || pick.logT != r.logT || pick.hash != r.hash || pick.compressed != r.compressed ||
        pick.part != r.part || pick.window != r.window || pick.stage != r.stage)
      ++changed;
    r = pick;
    h->tune_cache.push_back({cls0, logT0, h->dtype, pos0, r.count, pick});
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  h->tuned = true;
  h->stats.tuned_bins = changed;
  h->stats.rows_positions = rows_positions(h);
  return SPGEMM_OK;
}

spgemm_status_t do_numeric(kks_handle* h, int count, const spgemm_csr_t* A, const spgemm_csr_t* Bm,
                           int64_t* const* Crp, int32_t* const* Cj, void* const* Cx, cudaStream_t s) {
  if (!h) return SPGEMM_ERR_INVALID_ARG;
  if (!h->ready) return SPGEMM_ERR_NOT_READY;
  if (count != h->ninst || (count > 0 && (!A || !Bm || !Crp || !Cj || !Cx))) return SPGEMM_ERR_INVALID_ARG;
  bool changed = false;
  for (int b = 0; b < count; ++b) {
    KKS_ST(check_csr(&A[b], true));
    KKS_ST(check_csr(&Bm[b], true));
    if (!(patid(&A[b], &Bm[b]) == h->pat[b])) return SPGEMM_ERR_PATTERN_MISMATCH;
    if ((int)A[b].dtype != h->dtype || (int)Bm[b].dtype != h->dtype) return SPGEMM_ERR_INVALID_ARG;
    if (!Crp[b] || (!Cj[b] || !Cx[b])) {
      if (A[b].nrows > 0 && (!Crp[b])) return SPGEMM_ERR_INVALID_ARG;
    }
    InstD& I = h->inst[b];
    long long* crp = reinterpret_cast<long long*>(Crp[b]);
    if (I.A.vx != A[b].values || I.B.vx != Bm[b].values || I.Cj != Cj[b] || I.Cx != Cx[b] || I.Crp != crp) {
      changed = true;
      I.A.vx = A[b].values;
      I.B.vx = Bm[b].values;
      I.Cj = Cj[b];
      I.Cx = Cx[b];
      I.Crp = crp;
    }
  }
  KKS_CU(cudaSetDevice(h->opt.device));
  if (changed) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    KKS_CU(cudaStreamIsCapturing(s, &cs));
    if (cs != cudaStreamCaptureStatusNone) return SPGEMM_ERR_NOT_READY;
    KKS_ST(upload_inst(h, s));
  }
  if (h->opt.tune && !h->tuned) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    KKS_CU(cudaStreamIsCapturing(s, &cs));
    if (cs != cudaStreamCaptureStatusNone) return SPGEMM_ERR_NOT_READY;
    KKS_ST(tune_numeric(h, s));
  }
  for (const BinRun& r : h->num_bins) KKS_CU(launch_bin(h, r, s));
  return SPGEMM_OK;
}

// ---------------------------------------------------------------------------
// masked products (numeric reuse on C's pattern, gradients)
// ---------------------------------------------------------------------------
int cta_max_logT_msk(kks_handle* h, int dtype) {
  int best = 4;
  for (int l = 4; l <= 20; ++l)
    if (masked_team_bytes(kClsC1024, l, dtype) + 1024 <= (size_t)h->max_smem) best = l;
  return best;
}

spgemm_status_t check_masked(const spgemm_csr_t* X, const spgemm_csr_t* Y, const int64_t* Sp, const int32_t* Sj,
                             int64_t snnz, const void* out) {
  KKS_ST(check_csr(X, true));
  KKS_ST(check_csr(Y, true));
  if (X->ncols != Y->nrows || X->dtype != Y->dtype) return SPGEMM_ERR_INVALID_ARG;
  if (!Sp || snnz < 0 || (snnz > 0 && (!Sj || !out))) return SPGEMM_ERR_INVALID_ARG;
  return SPGEMM_OK;
}

MaskedD maskd(kks_handle* h, const spgemm_csr_t* X, const spgemm_csr_t* Y, const int64_t* Sp, const int32_t* Sj,
              void* out) {
  MaskedD M;
  M.X = matd(X);
  M.Y = matd(Y);
  M.Sp = reinterpret_cast<const long long*>(Sp);
  M.Sj = Sj;
  M.out = out;
  M.status = B<DevStatus>(h, kBufStatus);
  M.xperm = nullptr;
  M.yperm = nullptr;
  M.hash_mode = h->opt.hash_function;
  M.pad = 0;
  return M;
}

// Bins the rows of S (one synchronisation) into plan; rows into rows_buf.
spgemm_status_t plan_masked(kks_handle* h, const MaskedD& M, long long nrows, int dtype, int rows_buf, int pool_buf,
                            MaskPlan* plan, cudaStream_t s) {
  KKS_ST(ensure(h, kBufStatus, sizeof(DevStatus)));
  KKS_ST(ensure(h, kBufMaskHist, sizeof(unsigned long long) * (2 * kNumBins + 2)));
  KKS_ST(ensure(h, rows_buf, sizeof(int) * (nrows + 1)));
  KKS_ST(ensure_pinned(h, sizeof(unsigned long long) * (2 * kNumBins + 2) + sizeof(DevStatus)));
  const long long nbc = (long long)kNumBins * bin_blocks(nrows);
  KKS_ST(ensure(h, kBufBinCnt, sizeof(long long) * (nbc + 1)));
  KKS_ST(ensure(h, kBufBinOfs, sizeof(long long) * (nbc + 1)));
  KKS_ST(ensure(h, kBufScanTmp, scan_tmp_bytes(nbc + 1)));
  MaskedD Mx = M;
  Mx.status = B<DevStatus>(h, kBufStatus);
  BinCfg c = base_cfg(h);
  c.cta_max_logT = cta_max_logT_msk(h, dtype);
  c.dense_ok = 0;
  c.t1_max_work = 64;   // rows with <= 8 pattern entries and <= 64 products: one thread each
  clamp_cfg(h, c);
  unsigned long long* d_hist = B<unsigned long long>(h, kBufMaskHist);
  unsigned long long* h_hist = (unsigned long long*)h->pinned;
  LaunchCtx L = ctx(h, s);
  unsigned long long* d_unsorted = d_hist + 2 * kNumBins;
  unsigned long long* h_unsorted = h_hist + 2 * kNumBins;
  KKS_CU(cudaMemsetAsync(d_hist, 0, sizeof(unsigned long long) * kNumBins, s));
  KKS_CU(cudaMemsetAsync(d_unsorted, 0, sizeof(unsigned long long), s));
  KKS_CU(launch_masked_bin_count(L, Mx, nrows, c, d_hist, B<long long>(h, kBufBinCnt)));
  if (nrows > 0) KKS_CU(launch_scan(L, B<long long>(h, kBufBinCnt), B<long long>(h, kBufBinOfs), nbc, h->buf[kBufScanTmp]));
  if (h->opt.numeric_positions) KKS_CU(launch_pattern_unsorted(L, Mx, nrows, d_unsorted));
  KKS_CU(to_host(h, h_hist, d_hist, sizeof(unsigned long long) * kNumBins, s));
  KKS_CU(to_host(h, h_unsorted, d_unsorted, sizeof(unsigned long long), s));
  DevStatus* hs = (DevStatus*)(h->pinned + sizeof(unsigned long long) * (2 * kNumBins + 2));
  KKS_CU(to_host(h, hs, h->buf[kBufStatus], sizeof(DevStatus), s));
  KKS_CU(cudaStreamSynchronize(s));
  KKS_ST(consume_status(h, hs, s));
  plan->sorted = h->opt.numeric_positions != 0 && *h_unsorted == 0;
  plan->cls_logT.clear();
  plan->off.clear();
  plan->cnt.clear();
  long long o = 0;
  int glog = 0;
  long long grows = 0;
  std::vector<unsigned long long> cur(kNumBins, 0);
  for (int t = 0; t < kNumBins; ++t) {
    cur[t] = (unsigned long long)o;
    const long long n = (long long)h_hist[t];
    if (n == 0 || bin_cls(t) == kClsNone) continue;
    plan->cls_logT.push_back({bin_cls(t), bin_logT(t)});
    plan->off.push_back(o);
    plan->cnt.push_back(n);
    if (bin_cls(t) == kClsSpill) {
      glog = std::max(glog, bin_logT(t));
      grows += n;
    }
    o += n;
  }
  memcpy(h_hist + kNumBins, cur.data(), sizeof(unsigned long long) * kNumBins);
  KKS_CU(cudaMemcpyAsync(d_hist + kNumBins, h_hist + kNumBins, sizeof(unsigned long long) * kNumBins,
                         cudaMemcpyHostToDevice, s));
  KKS_CU(launch_masked_bin_scatter(L, Mx, nrows, c, d_hist + kNumBins, B<long long>(h, kBufBinOfs), B<int>(h, rows_buf)));
  plan->gchunks = 0;
  plan->gslots = 0;
  if (grows > 0) {
    const long long slots = 1ll << glog;
    const long long chunk = (long long)masked_global_chunk_bytes(slots, dtype);
    long long pool_limit = h->opt.pool_limit_bytes > 0 ? h->opt.pool_limit_bytes : (8ll << 30);
    long long nch = std::min<long long>(std::min<long long>(2ll * h->num_sms, grows), pool_limit / chunk);
    if (nch < 1) return SPGEMM_ERR_OOM;
    KKS_ST(ensure(h, pool_buf, (size_t)(nch * chunk)));
    plan->gchunks = (int)nch;
    plan->gslots = slots;
  }
  KKS_CU(cudaStreamSynchronize(s));
  plan->valid = true;
  return SPGEMM_OK;
}

spgemm_status_t run_masked_plan(kks_handle* h, const MaskedD& M, int dtype, int rows_buf, int pool_buf,
                                const MaskPlan& plan, cudaStream_t s) {
  LaunchCtx L = ctx(h, s);
  for (size_t b = 0; b < plan.cnt.size(); ++b) {
    MaskedLaunch S;
    memset(&S, 0, sizeof(S));
    S.cls = plan.cls_logT[b].first;
    S.logT = plan.cls_logT[b].second;
    S.rows = B<int>(h, rows_buf) + plan.off[b];
    S.nrows = plan.cnt[b];
    S.dtype = dtype;
    S.positions = (plan.sorted && (S.cls == kClsW8 || S.cls == kClsW32)) ? 1 : 0;
    S.window = (S.positions && S.cls == kClsW32 && (h->opt.window_positions & 4)) ? 1 : 0;
    if (S.cls == kClsSpill) {
      S.pool = h->buf[pool_buf];
      S.chunk_slots = plan.gslots;
      S.nchunks = plan.gchunks;
    }
    KKS_CU(launch_masked(L, M, S));
  }
  return SPGEMM_OK;
}

}  // namespace

// ===========================================================================
// C ABI
// ===========================================================================
extern "C" {

spgemm_status_t spgemm_options_default(spgemm_options_t* opt) {
  if (!opt) return SPGEMM_ERR_INVALID_ARG;
  set_default_options(opt);
  return SPGEMM_OK;
}

spgemm_status_t spgemm_handle_create(spgemm_handle_t* out, const spgemm_options_t* opt) {
  if (!out) return SPGEMM_ERR_INVALID_ARG;
  *out = nullptr;
  kks_handle* h = new (std::nothrow) kks_handle();
  if (!h) return SPGEMM_ERR_OOM;
  if (opt) h->opt = *opt; else set_default_options(&h->opt);
  if (!(h->opt.l1_max_occupancy > 0.0 && h->opt.l1_max_occupancy <= 1.0) || h->opt.compress_threshold < 0.0 ||
      h->opt.compression < -1 || h->opt.compression > 1 || h->opt.hash_function < 0 || h->opt.hash_function > 1 ||
      h->opt.slots_per_key_log2 < 0 || h->opt.slots_per_key_log2 > 4 || h->opt.numeric_positions < 0 ||
      h->opt.cta_partition < 0 || h->opt.cta_partition > 2 ||
      h->opt.numeric_positions > 1 || h->opt.window_positions < 0 || h->opt.window_positions > 7 ||
      h->opt.stage_b < 0 || h->opt.stage_b > 1 || h->opt.sym_merge < 0 || h->opt.sym_merge > 1) {
    delete h;
    return SPGEMM_ERR_INVALID_ARG;
  }
  int ndev = 0;
  cudaError_t e = cudaGetDeviceCount(&ndev);
  if (e != cudaSuccess || h->opt.device < 0 || h->opt.device >= ndev) {
    cudaGetLastError();
    delete h;
    return e != cudaSuccess ? SPGEMM_ERR_CUDA : SPGEMM_ERR_INVALID_ARG;
  }
  if (cudaSetDevice(h->opt.device) != cudaSuccess ||
      cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, h->opt.device) != cudaSuccess ||
      cudaDeviceGetAttribute(&h->max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, h->opt.device) != cudaSuccess) {
    cudaGetLastError();
    delete h;
    return SPGEMM_ERR_CUDA;
  }
  for (int r = 0; r < kRing; ++r) {
    if (cudaEventCreateWithFlags(&h->ring_ev[r], cudaEventDisableTiming) != cudaSuccess) {
      cudaGetLastError();
      delete h;
      return SPGEMM_ERR_CUDA;
    }
  }
  *out = h;
  return SPGEMM_OK;
}

spgemm_status_t spgemm_handle_destroy(spgemm_handle_t h) {
  if (!h) return SPGEMM_ERR_INVALID_ARG;
  cudaSetDevice(h->opt.device);
  cudaDeviceSynchronize();
  for (int i = 0; i < kNumBufs; ++i)
    if (h->buf[i]) cudaFree(h->buf[i]);
  if (h->pinned) cudaFreeHost(h->pinned);
  for (int r = 0; r < kRing; ++r) {
    if (h->ring[r]) cudaFreeHost(h->ring[r]);
    if (h->ring_ev[r]) cudaEventDestroy(h->ring_ev[r]);
  }
  delete h;
  return SPGEMM_OK;
}

spgemm_status_t spgemm_symbolic(spgemm_handle_t h, const spgemm_csr_t* A, const spgemm_csr_t* Bm, int64_t* C_rowptr,
                                int64_t* nnzC, spgemm_stream_t stream) {
  if (!h || !A || !Bm || !C_rowptr || !nnzC) return SPGEMM_ERR_INVALID_ARG;
  int64_t* crp[1] = {C_rowptr};
  return do_symbolic(h, 1, A, Bm, crp, nnzC, (cudaStream_t)stream);
}

spgemm_status_t spgemm_numeric(spgemm_handle_t h, const spgemm_csr_t* A, const spgemm_csr_t* Bm,
                               const int64_t* C_rowptr, int32_t* C_colidx, void* C_values, spgemm_stream_t stream) {
  if (!h || !A || !Bm || !C_rowptr) return SPGEMM_ERR_INVALID_ARG;
  if (h->ready && h->ninst == 1 && h->stats.nnzC > 0 && (!C_colidx || !C_values)) return SPGEMM_ERR_INVALID_ARG;
  int64_t* crp[1] = {const_cast<int64_t*>(C_rowptr)};
  int32_t* cj[1] = {C_colidx};
  void* cx[1] = {C_values};
  if (!C_colidx || !C_values) {
    // nnz(C) == 0: nothing to write
    if (!h->ready) return SPGEMM_ERR_NOT_READY;
    return SPGEMM_OK;
  }
  return do_numeric(h, 1, A, Bm, crp, cj, cx, (cudaStream_t)stream);
}

spgemm_status_t spgemm_handle_sync(spgemm_handle_t h, spgemm_stream_t stream) {
  if (!h) return SPGEMM_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  KKS_CU(cudaSetDevice(h->opt.device));
  if (!h->buf[kBufStatus]) {
    KKS_CU(cudaStreamSynchronize(s));
    return SPGEMM_OK;
  }
  KKS_ST(ensure_pinned(h, sizeof(DevStatus)));
  DevStatus* hs = (DevStatus*)h->pinned;
  KKS_CU(to_host(h, hs, h->buf[kBufStatus], sizeof(DevStatus), s));
  KKS_CU(cudaStreamSynchronize(s));
  return consume_status(h, hs, s);
}

spgemm_status_t spgemm_get_stats(spgemm_handle_t h, spgemm_stats_t* out) {
  if (!h || !out) return SPGEMM_ERR_INVALID_ARG;
  if (!h->ready && !h->rap.ready) return SPGEMM_ERR_NOT_READY;
  *out = h->stats;
  return SPGEMM_OK;
}

spgemm_status_t spgemm_batch_symbolic(spgemm_handle_t h, int32_t count, const spgemm_csr_t* A, const spgemm_csr_t* Bm,
                                      int64_t* const* C_rowptr, int64_t* nnzC, spgemm_stream_t stream) {
  if (!h) return SPGEMM_ERR_INVALID_ARG;
  return do_symbolic(h, count, A, Bm, C_rowptr, nnzC, (cudaStream_t)stream);
}

spgemm_status_t spgemm_batch_numeric(spgemm_handle_t h, int32_t count, const spgemm_csr_t* A, const spgemm_csr_t* Bm,
                                     int64_t* const* C_rowptr, int32_t* const* C_colidx, void* const* C_values,
                                     spgemm_stream_t stream) {
  if (!h) return SPGEMM_ERR_INVALID_ARG;
  return do_numeric(h, count, A, Bm, C_rowptr, C_colidx, C_values, (cudaStream_t)stream);
}

spgemm_status_t spgemm_masked(spgemm_handle_t h, const spgemm_csr_t* X, const spgemm_csr_t* Y,
                              const int64_t* S_rowptr, const int32_t* S_colidx, int64_t S_nnz, void* out,
                              const int64_t* X_perm, const int64_t* Y_perm, spgemm_stream_t stream) {
  if (!h) return SPGEMM_ERR_INVALID_ARG;
  KKS_ST(check_masked(X, Y, S_rowptr, S_colidx, S_nnz, out));
  cudaStream_t s = (cudaStream_t)stream;
  KKS_CU(cudaSetDevice(h->opt.device));
  if (X->nrows == 0 || S_nnz == 0) return SPGEMM_OK;
  KKS_ST(ensure(h, kBufStatus, sizeof(DevStatus)));
  MaskedD M = maskd(h, X, Y, S_rowptr, S_colidx, out);
  M.xperm = reinterpret_cast<const long long*>(X_perm);
  M.yperm = reinterpret_cast<const long long*>(Y_perm);
  // the row bins depend only on the three patterns: plan once, then reuse
  MaskPlan& P = h->masked;
  const bool same = P.valid && P.sp == S_rowptr && P.sj == S_colidx && P.xrp == X->rowptr && P.xcj == X->colidx &&
                    P.yrp == Y->rowptr && P.ycj == Y->colidx && P.nrows == X->nrows && P.snnz == S_nnz &&
                    P.dtype == (int)X->dtype;
  if (!same) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    KKS_CU(cudaStreamIsCapturing(s, &cs));
    if (cs != cudaStreamCaptureStatusNone) return SPGEMM_ERR_NOT_READY;
    P.valid = false;
    KKS_ST(plan_masked(h, M, X->nrows, (int)X->dtype, kBufMaskRows, kBufMaskPool, &P, s));
    P.sp = S_rowptr;
    P.sj = S_colidx;
    P.xrp = X->rowptr;
    P.xcj = X->colidx;
    P.yrp = Y->rowptr;
    P.ycj = Y->colidx;
    P.nrows = X->nrows;
    P.snnz = S_nnz;
    P.dtype = (int)X->dtype;
  }
  return run_masked_plan(h, M, (int)X->dtype, kBufMaskRows, kBufMaskPool, P, s);
}

spgemm_status_t spgemm_numeric_reuse(spgemm_handle_t h, const spgemm_csr_t* A, const spgemm_csr_t* Bm,
                                     const int64_t* C_rowptr, const int32_t* C_colidx, void* C_values,
                                     spgemm_stream_t stream) {
  if (!h || !A || !Bm) return SPGEMM_ERR_INVALID_ARG;
  if (!h->ready) return SPGEMM_ERR_NOT_READY;
  if (h->ninst != 1) return SPGEMM_ERR_INVALID_ARG;
  if (!(patid(A, Bm) == h->pat[0])) return SPGEMM_ERR_PATTERN_MISMATCH;
  const long long snnz = h->stats.nnzC;
  KKS_ST(check_masked(A, Bm, C_rowptr, C_colidx, snnz, C_values));
  if ((int)A->dtype != h->dtype) return SPGEMM_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  KKS_CU(cudaSetDevice(h->opt.device));
  if (A->nrows == 0 || snnz == 0) return SPGEMM_OK;
  MaskedD M = maskd(h, A, Bm, C_rowptr, C_colidx, C_values);
  MaskPlan& P = h->reuse;
  const bool same = P.valid && P.sp == C_rowptr && P.sj == C_colidx && P.xrp == A->rowptr && P.xcj == A->colidx &&
                    P.yrp == Bm->rowptr && P.ycj == Bm->colidx && P.nrows == A->nrows && P.snnz == snnz &&
                    P.dtype == (int)A->dtype;
  if (!same) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    KKS_CU(cudaStreamIsCapturing(s, &cs));
    if (cs != cudaStreamCaptureStatusNone) return SPGEMM_ERR_NOT_READY;
    P.valid = false;
    KKS_ST(plan_masked(h, M, A->nrows, (int)A->dtype, kBufReuseRows, kBufReusePool, &P, s));
    P.sp = C_rowptr;
    P.sj = C_colidx;
    P.xrp = A->rowptr;
    P.xcj = A->colidx;
    P.yrp = Bm->rowptr;
    P.ycj = Bm->colidx;
    P.nrows = A->nrows;
    P.snnz = snnz;
    P.dtype = (int)A->dtype;
  }
  return run_masked_plan(h, M, (int)A->dtype, kBufReuseRows, kBufReusePool, P, s);
}

spgemm_status_t spgemm_masked_count(spgemm_handle_t h, const spgemm_csr_t* X, const spgemm_csr_t* Y,
                                    const int64_t* S_rowptr, const int32_t* S_colidx, int64_t S_nnz,
                                    int64_t* row_counts, spgemm_stream_t stream) {
  if (!h || !X || !Y || !S_rowptr || !row_counts) return SPGEMM_ERR_INVALID_ARG;
  KKS_ST(check_csr(X, false));
  KKS_ST(check_csr(Y, false));
  if (X->ncols != Y->nrows || S_nnz < 0 || (S_nnz > 0 && !S_colidx)) return SPGEMM_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  KKS_CU(cudaSetDevice(h->opt.device));
  if (X->nrows == 0) return SPGEMM_OK;
  MaskedD M = maskd(h, X, Y, S_rowptr, S_colidx, nullptr);
  const long long ny = Y->nrows;
  KKS_ST(ensure(h, kBufStatus, sizeof(DevStatus)));
  KKS_ST(ensure(h, kBufMcCnt, sizeof(long long) * (ny + 1)));
  KKS_ST(ensure(h, kBufMcYcp, sizeof(long long) * (ny + 1)));
  KKS_ST(ensure(h, kBufMcMax, 128));
  KKS_ST(ensure(h, kBufMcRows, sizeof(int) * 3 * (X->nrows + 1)));
  KKS_ST(ensure(h, kBufScanTmp, scan_tmp_bytes(ny + 1)));
  KKS_ST(ensure_pinned(h, 64 + sizeof(DevStatus)));
  M.status = B<DevStatus>(h, kBufStatus);
  LaunchCtx L = ctx(h, s);
  KKS_CU(cudaMemsetAsync(h->buf[kBufStatus], 0, sizeof(DevStatus), s));
  // (1) Y's compressed row lengths and their scan; the longest row of S
  KKS_CU(launch_mc_compress(L, M, 0, nullptr, B<long long>(h, kBufMcCnt), nullptr, nullptr));
  KKS_CU(launch_scan(L, B<long long>(h, kBufMcCnt), B<long long>(h, kBufMcYcp), ny, h->buf[kBufScanTmp]));
  KKS_CU(launch_row_len_max(L, reinterpret_cast<const long long*>(S_rowptr), X->nrows,
                            B<unsigned long long>(h, kBufMcMax)));
  long long* h_nc = (long long*)h->pinned;
  unsigned long long* h_max = (unsigned long long*)(h->pinned + 16);
  DevStatus* hs = (DevStatus*)(h->pinned + 64);
  KKS_CU(to_host(h, h_nc, B<long long>(h, kBufMcYcp) + ny, sizeof(long long), s));
  KKS_CU(to_host(h, h_max, h->buf[kBufMcMax], sizeof(unsigned long long), s));
  KKS_CU(to_host(h, hs, h->buf[kBufStatus], sizeof(DevStatus), s));
  KKS_CU(cudaStreamSynchronize(s));
  KKS_ST(consume_status(h, hs, s));
  const long long nc = *h_nc;
  // (2) the compressed Y, (3) the counts
  KKS_ST(ensure(h, kBufMcCsi, sizeof(int) * (nc + 1)));
  KKS_ST(ensure(h, kBufMcCs, sizeof(unsigned) * (nc + 1)));
  KKS_CU(launch_mc_compress(L, M, 1, B<long long>(h, kBufMcYcp), nullptr, B<int>(h, kBufMcCsi),
                            B<unsigned>(h, kBufMcCs)));
  cudaError_t e = launch_masked_count(L, M, B<long long>(h, kBufMcYcp), B<int>(h, kBufMcCsi),
                                      B<unsigned>(h, kBufMcCs), reinterpret_cast<long long*>(row_counts),
                                      (long long)*h_max, B<int>(h, kBufMcRows),
                                      B<unsigned long long>(h, kBufMcMax) + 2);
  if (e == cudaErrorInvalidConfiguration) return SPGEMM_ERR_DEVICE_LIMIT;
  KKS_CU(e);
  KKS_CU(to_host(h, hs, h->buf[kBufStatus], sizeof(DevStatus), s));
  KKS_CU(cudaStreamSynchronize(s));
  return consume_status(h, hs, s);
}

namespace {

RapD rapd(kks_handle* h, const spgemm_csr_t* A, const spgemm_csr_t* P) {
  RapD R;
  R.A = matd(A);
  R.P = matd(P);
  R.Rtp = B<long long>(h, kBufRapRtp);
  R.Rti = B<int>(h, kBufRapRti);
  R.Rpe = B<long long>(h, kBufRapRpe);
  R.status = B<DevStatus>(h, kBufStatus);
  R.punit = 0;
  R.pad = 0;
  return R;
}

bool rap_same_pattern(const RapPlan& p, const spgemm_csr_t* A, const spgemm_csr_t* P) {
  return p.arp == A->rowptr && p.acj == (const void*)A->colidx && p.prp == P->rowptr &&
         p.pcj == (const void*)P->colidx && p.n == A->nrows && p.K == P->ncols && p.nnza == A->nnz &&
         p.nnzp == P->nnz && p.arp64 == A->rowptr_is_64 && p.prp64 == P->rowptr_is_64;
}

}  // namespace

spgemm_status_t spgemm_rap_symbolic(spgemm_handle_t h, const spgemm_csr_t* A, const spgemm_csr_t* P,
                                    int64_t* C_rowptr, int64_t* nnzC, spgemm_stream_t stream) {
  if (!h || !A || !P || !C_rowptr || !nnzC) return SPGEMM_ERR_INVALID_ARG;
  KKS_ST(check_csr(A, false));
  KKS_ST(check_csr(P, false));
  if (A->nrows != A->ncols || A->ncols != P->nrows) return SPGEMM_ERR_INVALID_ARG;
  if (A->dtype != P->dtype) return SPGEMM_ERR_INVALID_ARG;
  if (P->nrows > 2147483647ll || P->ncols > 2147483647ll) return SPGEMM_ERR_INDEX_OVERFLOW;
  cudaStream_t s = (cudaStream_t)stream;
  KKS_CU(cudaSetDevice(h->opt.device));
  RapPlan& pl = h->rap;
  pl.ready = false;
  const long long n = A->nrows, K = P->ncols, nnzp = P->nnz;
  const int dtype = (int)A->dtype;
  KKS_ST(ensure(h, kBufStatus, sizeof(DevStatus)));
  KKS_ST(ensure(h, kBufRapRf, sizeof(long long) * (n + 1)));
  KKS_ST(ensure(h, kBufRapRtp, sizeof(long long) * (K + 1)));
  KKS_ST(ensure(h, kBufRapRti, sizeof(int) * (nnzp + 1)));
  KKS_ST(ensure(h, kBufRapRpe, sizeof(long long) * (nnzp + 1)));
  KKS_ST(ensure(h, kBufRapW, sizeof(long long) * (K + 1)));
  KKS_ST(ensure(h, kBufRapCnt, sizeof(long long) * (K + 1)));
  KKS_ST(ensure(h, kBufRapSymRows, sizeof(int) * 2 * (K + 1)));
  KKS_ST(ensure(h, kBufRapNumRows, sizeof(int) * 2 * (K + 1)));
  KKS_ST(ensure(h, kBufRapMeta, sizeof(unsigned long long) * 16));
  KKS_ST(ensure(h, kBufRapTmp, std::max(transpose_pattern_tmp_bytes(K), scan_tmp_bytes(K + 1))));
  KKS_ST(ensure_pinned(h, 256 + sizeof(DevStatus)));
  KKS_CU(cudaMemsetAsync(h->buf[kBufStatus], 0, sizeof(DevStatus), s));
  KKS_CU(cudaMemsetAsync(h->buf[kBufRapMeta], 0, sizeof(unsigned long long) * 16, s));
  RapD R = rapd(h, A, P);
  LaunchCtx L = ctx(h, s);
  unsigned long long* meta = B<unsigned long long>(h, kBufRapMeta);
  int* sym_w = B<int>(h, kBufRapSymRows);
  int* sym_c = sym_w + (K + 1);
  int* num_w = B<int>(h, kBufRapNumRows);
  int* num_c = num_w + (K + 1);
  // tables: up to 8 KB per warp team (8 teams per CTA); a CTA team takes what
  // its shared memory holds beside its scratch
  const size_t warp_table = 8192;
  const size_t cta_table = (size_t)h->max_smem - rap_sym_team_bytes_host(1, 0) - 1024;
  unsigned long long* h_meta = (unsigned long long*)h->pinned;
  DevStatus* hs = (DevStatus*)(h->pinned + 256);
  // (1) products per row of A*P, the pattern of P^T, row bounds and classes
  KKS_CU(launch_rap_prepare(L, R, B<long long>(h, kBufRapRf), B<long long>(h, kBufRapW),
                            B<long long>(h, kBufRapCnt), sym_w, sym_c, meta, warp_table, cta_table,
                            h->buf[kBufRapTmp]));
  KKS_CU(to_host(h, h_meta, meta, sizeof(unsigned long long) * 16, s));
  KKS_CU(to_host(h, hs, h->buf[kBufStatus], sizeof(DevStatus), s));
  KKS_CU(cudaStreamSynchronize(s));
  KKS_ST(consume_status(h, hs, s));
  const long long fm = (long long)h_meta[4];
  R.punit = h_meta[10] == 0 ? 1 : 0;
  // (2) row sizes of C and their scan into C's row pointers
  KKS_CU(launch_rap_symbolic(L, R, B<long long>(h, kBufRapW), B<long long>(h, kBufRapCnt), sym_w,
                             (long long)h_meta[0], (size_t)h_meta[2], sym_c, (long long)h_meta[1],
                             (size_t)h_meta[3], h->opt.hash_function));
  KKS_CU(launch_scan(L, B<long long>(h, kBufRapCnt), reinterpret_cast<long long*>(C_rowptr), K,
                     h->buf[kBufRapTmp]));
  // (3) numeric classes by row size
  int warp_logT = 1, cta_logT = 1;
  for (int l = 1; l <= 24; ++l) {
    if (rap_num_team_bytes_host(0, dtype, l) * 8 <= kTeamSmemBudget) warp_logT = l;
    if (rap_num_team_bytes_host(1, dtype, l) + 1024 <= (size_t)h->max_smem) cta_logT = l;
  }
  KKS_CU(launch_rap_num_bin(L, reinterpret_cast<const long long*>(C_rowptr), K, num_w, num_c, meta, warp_logT,
                            cta_logT, B<DevStatus>(h, kBufStatus)));
  long long* h_nnz = (long long*)(h->pinned + 128);
  *h_nnz = 0;
  KKS_CU(to_host(h, h_meta, meta, sizeof(unsigned long long) * 16, s));
  KKS_CU(to_host(h, h_nnz, reinterpret_cast<const long long*>(C_rowptr) + K, sizeof(long long), s));
  KKS_CU(to_host(h, hs, h->buf[kBufStatus], sizeof(DevStatus), s));
  KKS_CU(cudaStreamSynchronize(s));
  KKS_ST(consume_status(h, hs, s));
  pl.arp = A->rowptr;
  pl.acj = A->colidx;
  pl.prp = P->rowptr;
  pl.pcj = P->colidx;
  pl.n = n;
  pl.K = K;
  pl.nnza = A->nnz;
  pl.nnzp = nnzp;
  pl.nnzc = *h_nnz;
  pl.arp64 = A->rowptr_is_64;
  pl.prp64 = P->rowptr_is_64;
  pl.dtype = dtype;
  pl.punit = R.punit;
  pl.n_w = (long long)h_meta[5];
  pl.n_c = (long long)h_meta[6];
  pl.logT_w = std::max(1, (int)h_meta[7]);
  pl.logT_c = std::max(1, (int)h_meta[8]);
  spgemm_stats_t& st = h->stats;
  memset(&st, 0, sizeof(st));
  st.m = K;
  st.n = n;
  st.k = K;
  st.nnzA = A->nnz;
  st.nnzB = nnzp;
  st.f_m = fm;
  st.f_m_compressed = fm;
  st.CF = 1.0;
  st.CMRF = 1.0;
  st.nnzC = *h_nnz;
  st.maxrs = (long long)h_meta[9];
  st.ars = K > 0 ? (double)*h_nnz / (double)K : 0.0;
  st.workspace_bytes = (int64_t)h->total;
  st.bin_rows_numeric[kClsW32] = pl.n_w;
  st.bin_rows_numeric[kClsC256] = pl.n_c;
  *nnzC = *h_nnz;
  pl.ready = true;
  return SPGEMM_OK;
}

spgemm_status_t spgemm_rap_numeric(spgemm_handle_t h, const spgemm_csr_t* A, const spgemm_csr_t* P,
                                   const int64_t* C_rowptr, int32_t* C_colidx, void* C_values,
                                   spgemm_stream_t stream) {
  if (!h || !A || !P || !C_rowptr) return SPGEMM_ERR_INVALID_ARG;
  KKS_ST(check_csr(A, true));
  KKS_ST(check_csr(P, true));
  const RapPlan& pl = h->rap;
  if (!pl.ready || !rap_same_pattern(pl, A, P)) return SPGEMM_ERR_NOT_READY;
  if ((int)A->dtype != pl.dtype || (int)P->dtype != pl.dtype) return SPGEMM_ERR_INVALID_ARG;
  if (pl.nnzc > 0 && (!C_colidx || !C_values)) return SPGEMM_ERR_INVALID_ARG;
  KKS_CU(cudaSetDevice(h->opt.device));
  cudaStream_t s = (cudaStream_t)stream;
  RapD R = rapd(h, A, P);
  R.punit = pl.punit;
  LaunchCtx L = ctx(h, s);
  int* num_w = B<int>(h, kBufRapNumRows);
  KKS_CU(launch_rap_numeric(L, R, pl.dtype, reinterpret_cast<const long long*>(C_rowptr), C_colidx, C_values, num_w,
                            pl.n_w, pl.logT_w, num_w + (pl.K + 1), pl.n_c, pl.logT_c, h->opt.hash_function));
  return SPGEMM_OK;
}

spgemm_status_t spgemm_transpose(spgemm_handle_t h, const spgemm_csr_t* A, int64_t* At_rowptr, int32_t* At_colidx,
                                 void* At_values, int64_t* perm, spgemm_stream_t stream) {
  if (!h) return SPGEMM_ERR_INVALID_ARG;
  KKS_ST(check_csr(A, At_values != nullptr));
  if (!At_rowptr || (A->nnz > 0 && !At_colidx)) return SPGEMM_ERR_INVALID_ARG;
  if (A->nrows > 2147483647ll) return SPGEMM_ERR_INDEX_OVERFLOW;
  cudaStream_t s = (cudaStream_t)stream;
  KKS_CU(cudaSetDevice(h->opt.device));
  KKS_ST(ensure(h, kBufStatus, sizeof(DevStatus)));
  KKS_ST(ensure(h, kBufTrTmp, transpose_tmp_bytes(A->nrows, A->ncols, A->nnz)));
  KKS_ST(ensure_pinned(h, 64 + sizeof(DevStatus)));
  MatD M = matd(A);
  if (!At_values) M.vx = nullptr;
  LaunchCtx L = ctx(h, s);
  unsigned long long* hmax = (unsigned long long*)h->pinned;
  *hmax = 0;
  KKS_CU(cudaMemsetAsync(h->buf[kBufStatus], 0, sizeof(DevStatus), s));
  DevStatus* hs = (DevStatus*)(h->pinned + 64);
  KKS_CU(launch_transpose_count(L, M, reinterpret_cast<long long*>(At_rowptr), h->buf[kBufTrTmp], hmax,
                                B<DevStatus>(h, kBufStatus)));
  KKS_CU(to_host(h, hs, h->buf[kBufStatus], sizeof(DevStatus), s));
  KKS_CU(cudaStreamSynchronize(s));
  KKS_ST(consume_status(h, hs, s));
  const long long max_len = (long long)*hmax;
  unsigned long long* gbuf = nullptr;
  long long gbuf_len = 0;
  int gchunks = 0;
  if (max_len > 16384) {
    gbuf_len = 1;
    while (gbuf_len < max_len) gbuf_len <<= 1;
    long long pool_limit = h->opt.pool_limit_bytes > 0 ? h->opt.pool_limit_bytes : (8ll << 30);
    long long nch = std::min<long long>(h->num_sms, pool_limit / (gbuf_len * 8));
    if (nch < 1) return SPGEMM_ERR_OOM;
    KKS_ST(ensure(h, kBufTrPool, (size_t)(nch * gbuf_len * 8)));
    gbuf = B<unsigned long long>(h, kBufTrPool);
    gchunks = (int)nch;
  }
  KKS_CU(launch_transpose_fill(L, M, (int)A->dtype, reinterpret_cast<const long long*>(At_rowptr), At_colidx,
                               At_values, reinterpret_cast<long long*>(perm), h->buf[kBufTrTmp], max_len, gbuf,
                               gbuf_len, gchunks, B<DevStatus>(h, kBufStatus)));
  return SPGEMM_OK;
}

spgemm_status_t spgemm_gather(spgemm_handle_t h, spgemm_dtype_t dtype, const void* src, const int64_t* perm, void* dst,
                              int64_t n, spgemm_stream_t stream) {
  if (!h || n < 0 || (n > 0 && (!src || !perm || !dst))) return SPGEMM_ERR_INVALID_ARG;
  if (dtype != SPGEMM_R32 && dtype != SPGEMM_R64) return SPGEMM_ERR_INVALID_ARG;
  KKS_CU(cudaSetDevice(h->opt.device));
  LaunchCtx L = ctx(h, (cudaStream_t)stream);
  KKS_CU(launch_gather_values(L, (int)dtype, src, reinterpret_cast<const long long*>(perm), dst, n));
  return SPGEMM_OK;
}

const char* spgemm_status_string(spgemm_status_t s) {
  switch (s) {
    case SPGEMM_OK: return "SPGEMM_OK";
    case SPGEMM_ERR_INVALID_ARG: return "SPGEMM_ERR_INVALID_ARG";
    case SPGEMM_ERR_NOT_READY: return "SPGEMM_ERR_NOT_READY";
    case SPGEMM_ERR_OOM: return "SPGEMM_ERR_OOM";
    case SPGEMM_ERR_INDEX_OVERFLOW: return "SPGEMM_ERR_INDEX_OVERFLOW";
    case SPGEMM_ERR_DEVICE_LIMIT: return "SPGEMM_ERR_DEVICE_LIMIT";
    case SPGEMM_ERR_CUDA: return "SPGEMM_ERR_CUDA";
    case SPGEMM_ERR_PATTERN_MISMATCH: return "SPGEMM_ERR_PATTERN_MISMATCH";
    case SPGEMM_ERR_BAD_INDEX: return "SPGEMM_ERR_BAD_INDEX";
  }
  return "SPGEMM_ERR_UNKNOWN";
}

int32_t spgemm_version(void) { return 100; }

int64_t spgemm_launch_count(void) { return (int64_t)g_launches.load(std::memory_order_relaxed); }

spgemm_status_t spgemm_row_flops(spgemm_handle_t h, const spgemm_csr_t* A, const spgemm_csr_t* Bm, int64_t* prefix,
                                 spgemm_stream_t stream) {
  if (!h || !A || !Bm || !prefix) return SPGEMM_ERR_INVALID_ARG;
  KKS_ST(check_csr(A, false));
  KKS_ST(check_csr(Bm, false));
  if (A->ncols != Bm->nrows) return SPGEMM_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  KKS_CU(cudaSetDevice(h->opt.device));
  const long long m = A->nrows;
  KKS_ST(ensure(h, kBufStatus, sizeof(DevStatus)));
  KKS_ST(ensure(h, kBufRf, sizeof(long long) * (m + 1)));
  KKS_ST(ensure(h, kBufScanTmp, scan_tmp_bytes(m + 1)));
  KKS_ST(ensure_pinned(h, sizeof(DevStatus)));
  LaunchCtx L = ctx(h, s);
  KKS_CU(cudaMemsetAsync(h->buf[kBufStatus], 0, sizeof(DevStatus), s));
  KKS_CU(launch_row_flops(L, matd(A), matd(Bm), B<long long>(h, kBufRf), B<DevStatus>(h, kBufStatus)));
  KKS_CU(launch_scan(L, B<long long>(h, kBufRf), reinterpret_cast<long long*>(prefix), m, h->buf[kBufScanTmp]));
  DevStatus* hs = (DevStatus*)h->pinned;
  KKS_CU(to_host(h, hs, h->buf[kBufStatus], sizeof(DevStatus), s));
  KKS_CU(cudaStreamSynchronize(s));
  return consume_status(h, hs, s);
}

spgemm_status_t spgemm_partition_rows(const int64_t* prefix, int64_t m, int32_t parts, int64_t* bounds) {
  if (!prefix || !bounds || m < 0 || parts < 1) return SPGEMM_ERR_INVALID_ARG;
  for (int64_t i = 0; i < m; ++i)
    if (prefix[i + 1] < prefix[i]) return SPGEMM_ERR_INVALID_ARG;
  const long double total = (long double)prefix[m];
  bounds[0] = 0;
  bounds[parts] = m;
  if (total <= 0) {   // no products: equal row counts
    for (int32_t p = 1; p < parts; ++p) bounds[p] = (int64_t)((long double)m * p / parts);
    return SPGEMM_OK;
  }
  for (int32_t p = 1; p < parts; ++p) {
    // the first row whose prefix reaches p / parts of the work (rows stay whole)
    const long double target = total * (long double)p / (long double)parts;
    int64_t lo = bounds[p - 1], hi = m;
    while (lo < hi) {
      const int64_t mid = lo + (hi - lo) / 2;
      if ((long double)prefix[mid] < target) lo = mid + 1;
      else hi = mid;
    }
    // of the two rows around the target, the boundary nearer to it
    if (lo > bounds[p - 1] && target - (long double)prefix[lo - 1] < (long double)prefix[lo] - target) --lo;
    bounds[p] = lo;
  }
  bounds[parts] = m;
  return SPGEMM_OK;
}

}  // extern "C"


