// kks_internal.h -- host/device declarations shared by the library's translation units.
#pragma once

#include <atomic>
#include <cstdint>
#include <cuda_runtime.h>

#include "kks_device.cuh"

namespace kks {

// Kernels launched by the library in this process (reported by spgemm_launch_count).
extern std::atomic<long long> g_launches;
#define KKS_LAUNCHED() ::kks::g_launches.fetch_add(1, std::memory_order_relaxed)

// ---------------------------------------------------------------------------
// Row binning.  A row of C is assigned to a team class and an accumulator
// size from two numbers: u, an upper bound on its distinct keys (exact in the
// numeric phase), and work, its product count.  This replaces the paper's
// per-problem choice between kkmem / kklp and its L1 sizing (Section 3.3) by a
// per-row choice, so one matrix uses several kernels at once.
// ---------------------------------------------------------------------------
enum TeamClass : int {
  kClsNone = 0,    // empty row: nothing to compute
  kClsW8 = 1,      // 8-lane sub-warp team, shared LP table
  kClsW32 = 2,     // warp team, shared LP table
  kClsC256 = 3,    // 256-thread CTA team (numeric: 512 from 4096 slots), shared LP table
  kClsC1024 = 4,   // 1024-thread CTA team, shared LP table
  kClsDense = 5,   // CTA team, dense accumulator (bitmap in shared memory)
  kClsSpill = 6,   // CTA team, shared L1 LP table + global L2 LP table
  kClsT1 = 7,      // one thread per row, keys and accumulators in registers
  kNumClasses = 8,
};
constexpr int kT1MaxKeys = 8;   // rows of class T1 have at most this many keys (numeric, masked)
constexpr int kT1SymKeys = 32;  // symbolic T1 rows: at most this many products, hence keys
constexpr int kBinsPerClass = 32;
constexpr int kNumBins = kNumClasses * kBinsPerClass;

__host__ __device__ inline int bin_id(int cls, int logT) { return cls * kBinsPerClass + logT; }
__host__ __device__ inline int bin_cls(int bin) { return bin / kBinsPerClass; }
__host__ __device__ inline int bin_logT(int bin) { return bin % kBinsPerClass; }

struct BinCfg {
  int min_logT;            // smallest table
  int w8_max_logT;         // sub-warp teams up to this table size ...
  long long w8_max_work;   // ... and this many products
  int w32_max_logT;
  long long w32_max_work;
  int c256_max_logT;
  long long c256_max_work;
  int cta_max_logT;        // largest shared-memory table (L1)
  int dense_ok;            // dense accumulator allowed at all
  long long dense_max_kwords;  // bitmap words that fit shared memory
  long long dense_ratio;   // prefer dense when u * dense_ratio >= kk
  int spill_ok;            // L1 + L2 hash allowed
  int force_cls;           // >0: every non-empty row goes to this class
  int force_logT;          // with force_cls: table size used for every row
  int slots_log2;          // table slots per key bound, log2 (0 = 1: at most 50 % load; -1: next power of two)
  long long t1_max_work;   // > 0: rows with u <= t1_max_keys and work <= this go to class T1
  int t1_max_keys;         // 0: kT1MaxKeys
  int dense_warp_log2w;    // > 0: dense rows of at most 2^this bitmap words and w32_max_work products
                           // take warp teams, binned by the bitmap size (bin logT = its log2, at
                           // least 5); 0: one CTA class
  long long rdense_max;    // numeric: dense rows of at most this many columns take the rank-dense
  long long rdense_small;  // kernel (bin logT 1), of at most rdense_small its 512-thread form (logT 2)
};

// kk: the key range the dense test compares against (k, or k/32 compressed);
// kwords: bitmap words of the dense accumulator (ceil(k / 32)).
__host__ __device__ inline int choose_bin(long long u, long long work, long long kk, long long kwords,
                                          const BinCfg& c) {
  if (u <= 0 || work <= 0) return bin_id(kClsNone, 0);
  int logT = ilog2_ceil(u) + (c.slots_log2 > 0 ? c.slots_log2 : (c.slots_log2 < 0 ? 0 : 1));
  if (logT < c.min_logT) logT = c.min_logT;
  if (logT > 30) logT = 30;   // bin ids hold logT < kBinsPerClass; such rows fail pool sizing
  if (c.force_cls > 0) {
    // one team class and table size for the whole problem (the paper's
    // per-problem choice); rows too large for that L1 go to L1 + L2
    if (logT <= c.force_logT) return bin_id(c.force_cls, c.force_logT);
    return bin_id(kClsSpill, logT);
  }
  if (c.t1_max_work > 0 && u <= (c.t1_max_keys > 0 ? c.t1_max_keys : kT1MaxKeys) && work <= c.t1_max_work)
    return bin_id(kClsT1, 0);
  bool dense_fit = c.dense_ok && kwords <= c.dense_max_kwords;
  const int dense_bin = (c.dense_warp_log2w > 0 && kwords <= (1ll << c.dense_warp_log2w) && work <= c.w32_max_work)
                            ? bin_id(kClsDense, ilog2_ceil(kwords) > 5 ? ilog2_ceil(kwords) : 5)
                        : (u <= c.rdense_small) ? bin_id(kClsDense, 2)
                        : (u <= c.rdense_max)   ? bin_id(kClsDense, 1)
                                                : bin_id(kClsDense, 0);
  if (dense_fit && (logT > c.cta_max_logT || u * c.dense_ratio >= kk)) return dense_bin;
  if (logT <= c.w8_max_logT && work <= c.w8_max_work) return bin_id(kClsW8, logT);
  if (logT <= c.w32_max_logT && work <= c.w32_max_work) return bin_id(kClsW32, logT);
  if (logT <= c.c256_max_logT && work <= c.c256_max_work) return bin_id(kClsC256, logT);
  if (logT <= c.cta_max_logT) return bin_id(kClsC1024, logT);
  if (c.spill_ok || !dense_fit) return bin_id(kClsSpill, logT);
  return dense_bin;
}

// ---------------------------------------------------------------------------
// launchers (all asynchronous on the given stream)
// ---------------------------------------------------------------------------
struct LaunchCtx {
  cudaStream_t stream;
  int num_sms;
  int max_smem_optin;   // bytes of dynamic shared memory a CTA may use
};

// Shared memory per CTA of the team kernels: up to 8 warp teams of a 256-slot
// FP64 table, so that four such CTAs (32 warps) share one SM's 228 KB.
constexpr size_t kTeamSmemBudget = 56 * 1024;

// CTAs of `kernel` (threads, dynamic shared memory smem) that fit on one SM,
// remembered per configuration (a host-side query, no device work).
int resident_per_sm(const void* kernel, int threads, size_t smem);

// Grid of a persistent team kernel: enough CTAs for the rows, at most the
// CTAs that are resident at once, so the rows in flight are one contiguous
// window of the (row-ordered) bin list and its B rows stay in L2.
template <class K>
inline unsigned resident_grid(K kernel, int threads, size_t smem, int num_sms, long long need) {
  const long long cap = (long long)num_sms * resident_per_sm(reinterpret_cast<const void*>(kernel), threads, smem);
  long long g = need < cap ? need : cap;
  if (g < 1) g = 1;
  return (unsigned)g;
}

// device -> mapped pinned host memory through a kernel (4-byte aligned; bytes
// rounded up to whole words)
cudaError_t launch_copy_to_host(const LaunchCtx&, void* dst_mapped, const void* src, size_t bytes);

// prep: statistics, compression, scans, binning
// A queue of the rows longer than 1024 entries (row indices of A or B, and
// three counters) that the per-block passes hand to a second launch where
// whole warps take them one at a time.
struct LongQueue {
  int* list;                 // >= totalA (totalB) entries
  unsigned long long* ctr;   // 3 counters
};
// per-row compressed lengths; *unsorted += rows of B whose columns do not increase;
// blen (may be null): per B row (length, compressed length) for the row statistics
cudaError_t launch_compress_count(const LaunchCtx&, const ProbD&, long long totalB, long long* cnt,
                                  unsigned long long* unsorted, const LongQueue& q, longlong2* blen);
// (the queue of the preceding count pass)
cudaError_t launch_compress_fill(const LaunchCtx&, const ProbD&, long long totalB, int* csi, unsigned* cs,
                                 const LongQueue& q);
// the 15 % rule on the device: inst[b].compressed from the row statistics
// (inst_stats[4b] = f_m, [4b + 2] = f_m on the compressed B); mode is the
// option compression (-1 auto, 1 always)
cudaError_t launch_decide_compression(const LaunchCtx&, InstD* inst, const unsigned long long* inst_stats, int count,
                                      int mode, double threshold);
// rf[i] = multiplications of row i of A*B (one plain product, no instance table)
cudaError_t launch_row_flops(const LaunchCtx&, const MatD& A, const MatD& B, long long* rf, DevStatus* st);
// blen (may be null): the (length, compressed length) pairs of the count pass,
// one load per entry of A instead of two pairs of row pointers
cudaError_t launch_row_stats(const LaunchCtx&, const ProbD&, long long totalA, int use_bc,
                             long long* rf, long long* rfc, unsigned long long* inst_stats, const LongQueue& q,
                             const longlong2* blen);
// exclusive scan of in[0, n) into out[0, n], out[n] = total; tmp >= scan_tmp_bytes(n)
size_t scan_tmp_bytes(long long n);
cudaError_t launch_scan(const LaunchCtx&, const long long* in, long long* out, long long n, void* tmp);
// phase 1 = numeric (u = row size); phase 2 / 3 = symbolic rows of compressed /
// uncompressed products (u from rfc / rf); rows of the other kind are skipped.
// Stable binning: the count adds the bin histogram into hist and writes the
// per-block counts bcnt[bin * bin_blocks + block] (kNumBins * bin_blocks
// entries); the scatter takes their exclusive scan bofs and the first slot of
// every bin (cursor) and lists each bin's rows in increasing row order.
constexpr int kBinRows = 1024;
constexpr int kBinThreads = 256;
inline long long bin_blocks(long long totalA) { return totalA > 0 ? (totalA + kBinRows - 1) / kBinRows : 1; }

// Device halves of the stable binning, for a block of kBinThreads threads over
// the rows [r0, r1).  key(g): the bin of row g, or -1 for a row not listed.
// Count: the block's histogram h (kNumBins, zeroed by the caller).
template <class Key>
__device__ __forceinline__ void bin_block_count(long long r0, long long r1, Key key, unsigned long long* h) {
  for (long long base = r0; base < r1; base += kBinThreads) {
    const long long g = base + threadIdx.x;
    const int bin = (g < r1) ? key(g) : -1;
    const unsigned grp = __match_any_sync(0xffffffffu, bin);
    if (bin >= 0 && (__ffs(grp) - 1) == (int)(threadIdx.x & 31)) atomicAdd(&h[bin], (unsigned long long)__popc(grp));
  }
}

// List: run[bin] holds the block's first slot in each bin's list; rows are
// written in increasing order.  wcnt: kBinThreads / 32 x kNumBins zeroed ints.
template <class Key>
__device__ __forceinline__ void bin_block_list(long long r0, long long r1, Key key, long long* run,
                                               int (*wcnt)[kNumBins], int* rows) {
  constexpr int kWarps = kBinThreads / 32;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  unsigned lt;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(lt));
  for (long long base = r0; base < r1; base += kBinThreads) {
    const long long g = base + threadIdx.x;
    const int bin = (g < r1) ? key(g) : -1;
    const unsigned grp = __match_any_sync(0xffffffffu, bin);
    if (bin >= 0 && lane == __ffs(grp) - 1) wcnt[warp][bin] = __popc(grp);
    __syncthreads();
    if (bin >= 0) {
      long long pos = run[bin];
      for (int w = 0; w < warp; ++w) pos += wcnt[w][bin];
      rows[pos + __popc(grp & lt)] = (int)g;
    }
    __syncthreads();
    for (int t = threadIdx.x; t < kNumBins; t += kBinThreads) {
      long long add = 0;
      for (int w = 0; w < kWarps; ++w) {
        add += wcnt[w][t];
        wcnt[w][t] = 0;
      }
      run[t] += add;
    }
    __syncthreads();
  }
}
cudaError_t launch_bin_count(const LaunchCtx&, const ProbD&, long long totalA, int phase,
                             const long long* rf, const long long* rfc, const long long* rowsize,
                             BinCfg cfg, unsigned long long* hist, long long* bcnt);
cudaError_t launch_bin_scatter(const LaunchCtx&, const ProbD&, long long totalA, int phase,
                               const long long* rf, const long long* rfc, const long long* rowsize,
                               BinCfg cfg, const unsigned long long* cursor, const long long* bofs, int* rows);
// C row pointers per instance from the global scan; per-instance nnz and max row size
cudaError_t launch_write_rowptr(const LaunchCtx&, const ProbD&, long long totalA, const long long* offs,
                                const long long* rowsize, unsigned long long* inst_out);

// symbolic: row sizes of C for the rows of one bin
struct SymLaunch {
  int cls, logT;
  const int* rows;
  long long nrows;
  int compressed;        // keys are column-set indices with OR-ed masks
  long long kwords_max;  // dense: bitmap words (max over instances)
  int l1_logT;           // spill: L1 table size
  double max_occ;        // L1 maximum occupancy for new keys
  void* l2_pool;         // spill: global pool
  long long l2_chunk_slots;
  int nchunks;
  unsigned long long* fetch;   // CTA classes: row counter (zeroed by the launcher)
  int window;            // compressed W32 rows with every B row sorted: bitmap-window kernel
  int merge;             // window kernel: rows of one chunk merge their sorted compressed B rows
};
cudaError_t launch_symbolic(const LaunchCtx&, const ProbD&, const SymLaunch&, long long* rowsize);

// numeric: columns and values of C for the rows of one bin
struct NumLaunch {
  int cls, logT;
  const int* rows;
  long long nrows;
  int dtype;             // 0 = float, 1 = double
  long long kwords_max;  // dense / spill: bitmap words
  long long kmax;        // dense: values per chunk
  int l1_logT;
  double max_occ;
  void* pool;            // dense values or spill L2 tables
  long long chunk_bytes;
  void* pool2;           // spill: bitmap + prefix words
  long long chunk2_words;
  int nchunks;
  int positions;         // warp classes: compressed-position kernel (every product's B compressed)
  int b_sorted;          // dense class: every B row has increasing columns
  unsigned long long* fetch;   // CTA classes: row counter (zeroed by the launcher)
  int part;              // CTA hash classes: 0 flat (Thread-Flat-Parallel), 1 Team-Sequential + LL,
                         // 2 Thread-Parallel (Section 3.1.1)
  int window;            // warp positions rows with b_sorted: bitmap-window kernel (rows whose set
                         // window is too wide fall back to the hash path inside it)
  int stage;             // dense class: B entries of one-chunk rows staged by cp.async
  int pad;
};
cudaError_t launch_numeric(const LaunchCtx&, const ProbD&, const NumLaunch&);

// masked values-only product: out(i, l) = sum_j X(i,j) Y(j,l) for (i,l) in S.
struct MaskedD {
  MatD X, Y;             // X: rows x n, Y: n x k
  const long long* Sp;   // pattern row pointers (int64)
  const int* Sj;         // pattern columns (any order within a row)
  void* out;             // values on the pattern
  DevStatus* status;
  const long long* xperm;  // optional: the value of X's entry p is X.vx[xperm[p]]
  const long long* yperm;  // optional: the value of Y's entry q is Y.vx[yperm[q]]
  int hash_mode;
  int pad;
};
struct MaskedLaunch {
  int cls, logT;
  const int* rows;
  long long nrows;
  int dtype;
  void* pool;            // big rows: global tables
  long long chunk_slots;
  int nchunks;
  int positions;         // warp classes: S's rows are sorted, places from its column sets
  int window;            // with positions, W32 rows: bitmap window of S(i,:)'s column sets
};
cudaError_t launch_pattern_unsorted(const LaunchCtx&, const MaskedD&, long long nrows, unsigned long long* count);
// stable binning of the pattern's rows (bcnt / bofs as launch_bin_count / launch_bin_scatter)
cudaError_t launch_masked_bin_count(const LaunchCtx&, const MaskedD&, long long nrows, BinCfg cfg,
                                    unsigned long long* hist, long long* bcnt);
cudaError_t launch_masked_bin_scatter(const LaunchCtx&, const MaskedD&, long long nrows, BinCfg cfg,
                                      const unsigned long long* cursor, const long long* bofs, int* rows);
cudaError_t launch_masked(const LaunchCtx&, const MaskedD&, const MaskedLaunch&);
// masked count: Y's compression (pass 0: run counts into cnt; pass 1: fill csi / cs
// from the scanned counts), then the per-row counts (warp rows of S up to 1024
// entries, CTA rows above when has_big_rows; those need ceil(k/32) words of
// shared memory)
constexpr int kMcBigRow = 1024;
cudaError_t launch_mc_compress(const LaunchCtx&, const MaskedD&, int pass, const long long* ycp, long long* cnt,
                               int* csi, unsigned* cs);
// max_row: the longest row of S (rows above kMcBigRow entries take a CTA each);
// lists: 3 * X.nrows ints of scratch, ctr: 6 counters of scratch
cudaError_t launch_masked_count(const LaunchCtx&, const MaskedD&, const long long* Ycp, const int* csi,
                                const unsigned* cs, long long* counts, long long max_row, int* lists,
                                unsigned long long* ctr);
// *out = the longest row of a pattern with int64 row pointers (device)
cudaError_t launch_row_len_max(const LaunchCtx&, const long long* Sp, long long nrows, unsigned long long* out);

size_t masked_global_chunk_bytes(long long slots, int dtype);

// transpose: At (n x m) with int64 row pointers and a value permutation.
// count: column counts, their scan into Atp, and the longest row into *h_max
// (host pinned); fill: scatter and per-row sort (rows longer than 16384 sort in
// gbuf chunks of gbuf_len keys).
size_t transpose_tmp_bytes(long long m, long long n, long long nnz);
cudaError_t launch_transpose_count(const LaunchCtx&, const MatD& A, long long* Atp, void* tmp,
                                   unsigned long long* h_max, DevStatus* st);
cudaError_t launch_transpose_fill(const LaunchCtx&, const MatD& A, int dtype, const long long* Atp, int* Atj,
                                  void* Atx, long long* perm, void* tmp, long long max_len,
                                  unsigned long long* gbuf, long long gbuf_len, int gbuf_chunks, DevStatus* st);
cudaError_t launch_gather_values(const LaunchCtx&, int dtype, const void* src, const long long* perm,
                                 void* dst, long long n);
// pattern of A^T only: column counts, their scan into Atp (m + 1 = ncols + 1
// entries), and per entry of A^T its row of A (trow) and its entry of A
// (tperm), rows of A^T in no particular order.  tmp >= transpose_pattern_tmp_bytes.
size_t transpose_pattern_tmp_bytes(long long ncols);
cudaError_t launch_transpose_pattern(const LaunchCtx&, const MatD& A, long long* Atp, int* trow, long long* tperm,
                                     void* tmp, DevStatus* st);

// ---------------------------------------------------------------------------
// Galerkin triple product C = P^T * A * P (A n x n, P n x K, C K x K)
// ---------------------------------------------------------------------------
constexpr int kRapCtaThreads = 256;

struct RapD {
  MatD A;
  MatD P;
  const long long* Rtp;   // K + 1: row pointers of P^T
  const int* Rti;         // per entry of P^T: its column (the row i of P)
  const long long* Rpe;   // per entry of P^T: the entry of P holding its value
  DevStatus* status;
  int punit;              // every row i of P holds one entry, at position i
  int pad;
};

__host__ __device__ int rap_sym_logT(long long w, long long K);
__host__ __device__ bool rap_sym_bitmap(long long w, long long K);
__host__ __device__ size_t rap_sym_table_bytes(long long w, long long K);
__host__ __device__ int rap_num_logT(long long s);
size_t rap_sym_team_bytes_host(int cta, size_t table);
size_t rap_num_team_bytes_host(int cta, int dtype, int logT);
// products per row of A*P (rf), the pattern of P^T (into R's Rtp / Rti / Rpe),
// per row of C its product count (w) and symbolic class; rows without
// products get cnt 0.  meta (16 zeroed words): [0] / [1] warp / CTA rows,
// [2] / [3] their largest table bytes, [4] total products, [10] nonzero
// unless every row i of P holds exactly one entry at position i.
cudaError_t launch_rap_prepare(const LaunchCtx&, const RapD& R, long long* rf, long long* w, long long* cnt,
                               int* rows_w, int* rows_c, unsigned long long* meta, size_t warp_table,
                               size_t cta_table, void* tmp);
cudaError_t launch_rap_symbolic(const LaunchCtx&, const RapD& R, const long long* w, long long* cnt,
                                const int* rows_w, long long n_w, size_t table_w, const int* rows_c, long long n_c,
                                size_t table_c, int hash_mode);
// numeric classes from C's row pointers: meta [5] / [6] warp / CTA rows, [7] /
// [8] their largest log2 table, [9] the longest row
cudaError_t launch_rap_num_bin(const LaunchCtx&, const long long* Crp, long long K, int* rows_w, int* rows_c,
                               unsigned long long* meta, int warp_logT, int cta_logT, DevStatus* st);
cudaError_t launch_rap_numeric(const LaunchCtx&, const RapD& R, int dtype, const long long* Crp, int* Cj, void* Cx,
                               const int* rows_w, long long n_w, int logT_w, const int* rows_c, long long n_c,
                               int logT_c, int hash_mode);

}  // namespace kks
