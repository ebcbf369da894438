// kks_prep.cu -- row statistics, column-set compression, scans and row binning.
//
// Row statistics follow the paper's definitions: the product count of row i
// is rf_i = sum over j in A(i,:) of |B(j,:)| and f_m = sum rf_i (Section 2,
// after Algorithm 1); maxrf = max rf_i sizes the L2 accumulators (Section
// 3.1.2, memory pool).  Compression (Section 3.2) packs the columns of a B row
// into column-set indices CSI = col >> 5 with a 32-bit set CS; a first pass
// counts the compressed row lengths so the compressed product count can decide
// whether compressing pays (more than a 15 % reduction), a second pass fills.
#include <mutex>
#include <vector>

#include "kks_internal.h"

namespace kks {

namespace {

constexpr int kBlock = 256;

__device__ __forceinline__ int lanemask_lt() {
  unsigned r;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(r));
  return (int)r;
}

inline int grid_for(long long items, int per_block, int num_sms, int cap_per_sm = 32) {
  long long g = (items + per_block - 1) / per_block;
  long long cap = (long long)num_sms * cap_per_sm;
  if (g > cap) g = cap;
  if (g < 1) g = 1;
  return (int)g;
}

// -------------------------------------------------------------- compression
// Both passes take kBlock consecutive rows of B per block: a thread handles
// its own row when it has at most kShortRow entries (every row of the block in
// flight at once), and 8-lane teams share the longer rows afterwards.
constexpr int kShortRowB = 32;

// Compressed row lengths: runs of equal CSI in row order.  Also counts the B
// rows whose columns are not strictly increasing (the dense numeric windows
// look up column ranges by binary search only when none is).
// Rows longer than this go to a queue served by whole warps in a second
// launch, so a few very long rows (graph hubs) do not hold their block while
// the rest of the grid has finished.
constexpr int kLongRow = 1024;

// The next entry of a long-row queue for the calling warp (warp-uniform).
__device__ __forceinline__ long long long_next(unsigned long long* fetch) {
  unsigned long long x = 0;
  if ((threadIdx.x & 31) == 0) x = atomicAdd(fetch, 1ull);
  return (long long)__shfl_sync(0xffffffffu, x, 0);
}

// Compressed length of B row gb by a team of TW lanes.
template <int TW>
__device__ __forceinline__ void compress_count_team(const Team<TW>& tm, const ProbD& P, long long gb, long long* cnt,
                                                    unsigned long long* unsorted, longlong2* blen) {
  const int b = inst_of(P.brow0s, P.ninst, gb);
  const InstD& I = P.inst[b];
  const long long j = gb - I.brow0;
  const long long s = rp_at(I.B, j), e = rp_at(I.B, j + 1);
  const int* cj = I.B.cj;
  long long c = 0;
  bool bad = false;
  for (long long p = s + tm.lane; p < e; p += TW) {
    int col = cj[p];
    if ((unsigned long long)(unsigned)col >= (unsigned long long)I.k) dev_fail(P.status, kDevBadIndex, 41, gb);
    const int prev = p > s ? cj[p - 1] : -1;
    if (p == s || (col >> 5) != (prev >> 5)) ++c;
    bad |= p > s && col <= prev;
  }
  c = warp_team_sum<TW>(tm, c);
  if (tm.lane == 0) {
    cnt[gb] = c;
    if (blen) blen[gb] = make_longlong2(e - s, c);
  }
  if (__any_sync(tm.mask, bad) && tm.lane == 0) atomicAdd(unsorted, 1ull);
}

template <int TW>
__global__ void __launch_bounds__(kBlock) k_compress_count(ProbD P, long long totalB, long long* cnt,
                                                           unsigned long long* unsorted, int* list,
                                                           unsigned long long* nlist, longlong2* blen) {
  Team<TW> tm;
  __shared__ int nlong;
  __shared__ int longrows[kBlock];
  const long long g0 = (long long)blockIdx.x * kBlock;
  if (g0 >= totalB) return;
  const long long g1 = g0 + kBlock < totalB ? g0 + kBlock : totalB;
  if (threadIdx.x == 0) nlong = 0;
  __syncthreads();
  {
    const long long gb = g0 + threadIdx.x;
    if (gb < g1) {
      const int b = inst_of(P.brow0s, P.ninst, gb);
      const InstD& I = P.inst[b];
      const long long j = gb - I.brow0;
      const long long s = rp_at(I.B, j), e = rp_at(I.B, j + 1);
      if (s < 0 || s > e || e > I.B.nnz) {   // malformed row pointers: report, read nothing
        dev_fail(P.status, kDevBadIndex, 40, gb);
        cnt[gb] = 0;
        if (blen) blen[gb] = make_longlong2(0, 0);
      } else if (e - s <= kShortRowB) {
        const int* cj = I.B.cj;
        long long c = 0;
        int prev = -1;
        bool bad = false;
#pragma unroll 4
        for (long long p = s; p < e; ++p) {
          const int col = cj[p];
          if ((unsigned long long)(unsigned)col >= (unsigned long long)I.k) dev_fail(P.status, kDevBadIndex, 41, gb);
          if (p == s || (col >> 5) != (prev >> 5)) ++c;
          bad |= p > s && col <= prev;
          prev = col;
        }
        cnt[gb] = c;
        if (blen) blen[gb] = make_longlong2(e - s, c);
        if (bad) atomicAdd(unsorted, 1ull);
      } else if (e - s > kLongRow) {
        list[atomicAdd(nlist, 1ull)] = (int)gb;
      } else {
        longrows[atomicAdd(&nlong, 1)] = (int)(gb - g0);
      }
    }
  }
  __syncthreads();
  for (int x = tm.id; x < nlong; x += tm.per_cta)
    compress_count_team<TW>(tm, P, g0 + longrows[x], cnt, unsorted, blen);
}

// Rows of B longer than kLongRow entries, from the queue the block pass built,
// one warp each (a warp takes the next row from a counter).
__global__ void __launch_bounds__(kBlock) k_compress_count_long(ProbD P, const int* list, const unsigned long long* n,
                                                                unsigned long long* fetch, long long* cnt,
                                                                unsigned long long* unsorted, longlong2* blen) {
  Team<32> tm;
  for (long long x = long_next(fetch); x < (long long)*n; x = long_next(fetch))
    compress_count_team<32>(tm, P, list[x], cnt, unsorted, blen);
}

// Runs of equal CSI in row order become one compressed entry; rows with sorted
// columns therefore get exactly one entry per distinct CSI.  Short rows are
// written by their thread run by run.  In the team loop of long rows the
// chunk where a run starts stores its bits and later chunks of the same run
// OR in theirs (cs needs no clearing).
// Compressed row gb of B by a team of TW lanes (lanes in order over the row).
template <int TW>
__device__ __forceinline__ void compress_fill_team(const Team<TW>& tm, const ProbD& P, long long gb, int* csi,
                                                   unsigned* cs) {
  const int base_lane = (threadIdx.x & 31) & ~(TW - 1);
  const int b = inst_of(P.brow0s, P.ninst, gb);
  const InstD& I = P.inst[b];
  const long long j = gb - I.brow0;
  const long long s = rp_at(I.B, j), e = rp_at(I.B, j + 1);
  const int* cj = I.B.cj;
  long long run = P.Bcp[gb] - 1;   // index of the last run opened so far
  for (long long c0 = s; c0 < e; c0 += TW) {
    const long long p = c0 + tm.lane;
    const bool valid = p < e;
    const int col = valid ? cj[p] : 0;
    const bool head = valid && (p == s || (col >> 5) != (cj[p - 1] >> 5));
    const unsigned hb = (__ballot_sync(tm.mask, head) >> base_lane) & ((TW == 32) ? 0xffffffffu : ((1u << TW) - 1u));
    const unsigned le = (tm.lane == 31) ? 0xffffffffu : ((2u << tm.lane) - 1u);
    const long long ridx = run + __popc(hb & le);
    if (head) csi[ridx] = col >> 5;
    // segmented OR over the lanes of each run inside this chunk
    unsigned v = valid ? (1u << (col & 31)) : 0u;
    int f = (head || tm.lane == 0) ? 1 : 0;
#pragma unroll
    for (int d = 1; d < TW; d <<= 1) {
      unsigned vu = __shfl_up_sync(tm.mask, v, d, TW);
      int fu = __shfl_up_sync(tm.mask, f, d, TW);
      if (tm.lane >= d && !f) {
        v |= vu;
        f = fu;
      }
    }
    const bool next_head = (tm.lane + 1 < TW) && ((hb >> (tm.lane + 1)) & 1u);
    const bool tail = valid && (tm.lane == TW - 1 || p + 1 >= e || next_head);
    if (tail) {
      if (hb & le) cs[ridx] = v;     // the run starts in this chunk
      else atomicOr(cs + ridx, v);   // continuation of the previous chunk's last run
    }
    run += __popc(hb);
    tm.sync();
  }
}

template <int TW>
__global__ void __launch_bounds__(kBlock) k_compress_fill(ProbD P, long long totalB, int* csi, unsigned* cs) {
  Team<TW> tm;
  __shared__ int nlong;
  __shared__ int longrows[kBlock];
  const long long g0 = (long long)blockIdx.x * kBlock;
  if (g0 >= totalB) return;
  const long long g1 = g0 + kBlock < totalB ? g0 + kBlock : totalB;
  if (threadIdx.x == 0) nlong = 0;
  __syncthreads();
  const int base_lane = (threadIdx.x & 31) & ~(TW - 1);
  {
    const long long gb = g0 + threadIdx.x;
    int b = 0;
    long long s = 0, e = 0;
    if (gb < g1) {
      b = inst_of(P.brow0s, P.ninst, gb);
      const InstD& I = P.inst[b];
      if (I.compressed) {
        s = rp_at(I.B, gb - I.brow0);
        e = rp_at(I.B, gb - I.brow0 + 1);
        // malformed row pointers (reported by the count pass, which gave the
        // row no compressed entries): read nothing
        if (s < 0 || s > e || e > I.B.nnz) s = e = 0;
      }
    }
    if (gb < g1) {
      const InstD& I = P.inst[b];
      if (I.compressed) {
        if (e - s <= kShortRowB) {
          const int* cj = I.B.cj;
          long long run = P.Bcp[gb] - 1;
          int set = -1;
          unsigned bits = 0u;
#pragma unroll 4
          for (long long p = s; p < e; ++p) {
            const int col = cj[p];
            if (p == s || (col >> 5) != set) {
              if (p > s) cs[run] = bits;
              ++run;
              set = col >> 5;
              csi[run] = set;
              bits = 0u;
            }
            bits |= 1u << (col & 31);
          }
          if (e > s) cs[run] = bits;
        } else if (e - s <= kLongRow) {
          longrows[atomicAdd(&nlong, 1)] = (int)(gb - g0);
        }   // longer rows: k_compress_fill_long, from the queue of the count pass
      }
    }
  }
  __syncthreads();
  for (int x = tm.id; x < nlong; x += tm.per_cta) compress_fill_team<TW>(tm, P, g0 + longrows[x], csi, cs);
}

__global__ void __launch_bounds__(kBlock) k_compress_fill_long(ProbD P, const int* list, const unsigned long long* n,
                                                               unsigned long long* fetch, int* csi, unsigned* cs) {
  Team<32> tm;
  for (long long x = long_next(fetch); x < (long long)*n; x = long_next(fetch)) {
    const long long gb = list[x];
    if (P.inst[inst_of(P.brow0s, P.ninst, gb)].compressed) compress_fill_team<32>(tm, P, gb, csi, cs);
  }
}

// -------------------------------------------------------------- row statistics
// inst_stats per instance: [f_m, maxrf, f_m compressed, maxrf compressed]
// Row statistics: rf_i = sum over j in A(i,:) of |B(j,:)| (and rfc_i on the
// compressed B), per instance f_m, maxrf and the compressed counterparts.  A
// block takes kBlock consecutive rows: each thread counts its own row when it
// has at most kShortRow entries (every row of the block in flight at once),
// and 8-lane teams share the longer rows afterwards.  This is also the first
// kernel that follows A's indices into B, so it validates them.
constexpr int kShortRow = 32;

// Adds to *f / *fc the lengths of the B (compressed B) rows of the entries
// p0, p0 + step, ... < e of A row g; the loads of four entries at a time are
// issued together.
__device__ __forceinline__ void row_stats_entries(const ProbD& P, const InstD& I, long long g, long long p0,
                                                  long long e, long long step, int use_bc, long long* f,
                                                  long long* fc, const longlong2* blen) {
  constexpr int kU = 4;
  for (; p0 < e; p0 += (long long)kU * step) {
    int jj[kU];
#pragma unroll
    for (int u = 0; u < kU; ++u) {
      const long long p = p0 + (long long)u * step;
      jj[u] = p < e ? I.A.cj[p] : -1;
      if (p < e && (unsigned long long)(unsigned)jj[u] >= (unsigned long long)I.A.ncols) {
        dev_fail(P.status, kDevBadIndex, 43, g);
        jj[u] = -1;
      }
    }
    if (blen) {
      // the count pass validated B's row pointers and stored both lengths
      longlong2 ln[kU];
#pragma unroll
      for (int u = 0; u < kU; ++u) ln[u] = jj[u] >= 0 ? blen[I.brow0 + jj[u]] : make_longlong2(0, 0);
#pragma unroll
      for (int u = 0; u < kU; ++u) {
        *f += ln[u].x;
        *fc += ln[u].y;
      }
      continue;
    }
    long long bs[kU], be[kU], cs[kU], ce[kU];
#pragma unroll
    for (int u = 0; u < kU; ++u) {
      bs[u] = be[u] = cs[u] = ce[u] = 0;
      if (jj[u] >= 0) {
        bs[u] = rp_at(I.B, jj[u]);
        be[u] = rp_at(I.B, jj[u] + 1);
        if (use_bc) {
          cs[u] = P.Bcp[I.brow0 + jj[u]];
          ce[u] = P.Bcp[I.brow0 + jj[u] + 1];
        }
      }
    }
#pragma unroll
    for (int u = 0; u < kU; ++u) {
      if (bs[u] < 0 || bs[u] > be[u] || be[u] > I.B.nnz) {
        dev_fail(P.status, kDevBadIndex, 44, g);
        continue;
      }
      *f += be[u] - bs[u];
      *fc += ce[u] - cs[u];
    }
  }
}

// Row statistics of the A rows longer than kLongRow entries (queued by
// k_row_stats), one warp each; instance totals by atomics.
__global__ void __launch_bounds__(kBlock) k_row_stats_long(ProbD P, int use_bc, const int* list,
                                                           const unsigned long long* n, unsigned long long* fetch,
                                                           long long* rf, long long* rfc,
                                                           unsigned long long* inst_stats, const longlong2* blen) {
  Team<32> tm;
  for (long long x = long_next(fetch); x < (long long)*n; x = long_next(fetch)) {
    const long long g = list[x];
    const int b = inst_of(P.arow0s, P.ninst, g);
    const InstD& I = P.inst[b];
    const long long i = g - I.arow0;
    const long long s = rp_at(I.A, i), e = rp_at(I.A, i + 1);
    long long f = 0, fc = 0;
    row_stats_entries(P, I, g, s + tm.lane, e, 32, use_bc, &f, &fc, blen);
    f = warp_team_sum<32>(tm, f);
    fc = warp_team_sum<32>(tm, fc);
    if (tm.lane == 0) {
      rf[g] = f;
      if (rfc) rfc[g] = fc;
      unsigned long long* st = inst_stats + 4ll * b;
      atomicAdd(st + 0, (unsigned long long)f);
      atomicMax(st + 1, (unsigned long long)f);
      atomicAdd(st + 2, (unsigned long long)fc);
      atomicMax(st + 3, (unsigned long long)fc);
    }
  }
}

template <int TW>
__global__ void __launch_bounds__(kBlock) k_row_stats(ProbD P, long long totalA, int use_bc, long long* rf,
                                                      long long* rfc, unsigned long long* inst_stats, int* list,
                                                      unsigned long long* nlist, const longlong2* blen) {
  Team<TW> tm;
  __shared__ unsigned long long acc[4];
  __shared__ int b_first, b_last, nlong;
  __shared__ int longrows[kBlock];
  const long long g0 = (long long)blockIdx.x * kBlock;
  if (g0 >= totalA) return;
  const long long g1 = g0 + kBlock < totalA ? g0 + kBlock : totalA;
  if (threadIdx.x == 0) {
    acc[0] = acc[1] = acc[2] = acc[3] = 0ull;
    nlong = 0;
    b_first = inst_of(P.arow0s, P.ninst, g0);
    b_last = inst_of(P.arow0s, P.ninst, g1 - 1);
  }
  __syncthreads();
  const bool single = (b_first == b_last);
  unsigned long long t_sum = 0, t_max = 0, t_csum = 0, t_cmax = 0;
  auto record = [&](long long g, int b, long long f, long long fc) {
    rf[g] = f;
    if (rfc) rfc[g] = fc;
    if (single) {
      t_sum += (unsigned long long)f;
      t_max = t_max > (unsigned long long)f ? t_max : (unsigned long long)f;
      t_csum += (unsigned long long)fc;
      t_cmax = t_cmax > (unsigned long long)fc ? t_cmax : (unsigned long long)fc;
    } else {
      unsigned long long* st = inst_stats + 4ll * b;
      atomicAdd(st + 0, (unsigned long long)f);
      atomicMax(st + 1, (unsigned long long)f);
      atomicAdd(st + 2, (unsigned long long)fc);
      atomicMax(st + 3, (unsigned long long)fc);
    }
  };
  auto entries = [&](const InstD& I, long long g, long long p0, long long e, long long step, long long* f,
                     long long* fc) { row_stats_entries(P, I, g, p0, e, step, use_bc, f, fc, blen); };
  // (1) short rows, one thread each
  {
    const long long g = g0 + threadIdx.x;
    if (g < g1) {
      const int b = single ? b_first : inst_of(P.arow0s, P.ninst, g);
      const InstD& I = P.inst[b];
      const long long i = g - I.arow0;
      const long long s = rp_at(I.A, i), e = rp_at(I.A, i + 1);
      if (!(s >= 0 && s <= e && e <= I.A.nnz)) {
        dev_fail(P.status, kDevBadIndex, 42, g);
      } else if (e - s <= kShortRow) {
        long long f = 0, fc = 0;
        entries(I, g, s, e, 1, &f, &fc);
        record(g, b, f, fc);
      } else if (e - s > kLongRow) {
        list[atomicAdd(nlist, 1ull)] = (int)g;
      } else {
        longrows[atomicAdd(&nlong, 1)] = (int)(g - g0);
      }
    }
  }
  __syncthreads();
  // (2) long rows, one 8-lane team each
  for (int x = tm.id; x < nlong; x += tm.per_cta) {
    const long long g = g0 + longrows[x];
    const int b = single ? b_first : inst_of(P.arow0s, P.ninst, g);
    const InstD& I = P.inst[b];
    const long long i = g - I.arow0;
    const long long s = rp_at(I.A, i), e = rp_at(I.A, i + 1);
    long long f = 0, fc = 0;
    entries(I, g, s + tm.lane, e, TW, &f, &fc);
    f = warp_team_sum<TW>(tm, f);
    fc = warp_team_sum<TW>(tm, fc);
    if (tm.lane == 0) record(g, b, f, fc);
  }
  // per-block totals: a warp reduction, then one shared update per warp
  if (single) {
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) {
      t_sum += __shfl_xor_sync(0xffffffffu, t_sum, d);
      t_csum += __shfl_xor_sync(0xffffffffu, t_csum, d);
      t_max = max(t_max, __shfl_xor_sync(0xffffffffu, t_max, d));
      t_cmax = max(t_cmax, __shfl_xor_sync(0xffffffffu, t_cmax, d));
    }
    if ((threadIdx.x & 31) == 0) {
      atomicAdd(&acc[0], t_sum);
      atomicMax(&acc[1], t_max);
      atomicAdd(&acc[2], t_csum);
      atomicMax(&acc[3], t_cmax);
    }
  }
  __syncthreads();
  if (single && threadIdx.x == 0) {
    unsigned long long* st = inst_stats + 4ll * b_first;
    atomicAdd(st + 0, acc[0]);
    atomicMax(st + 1, acc[1]);
    atomicAdd(st + 2, acc[2]);
    atomicMax(st + 3, acc[3]);
  }
}

// -------------------------------------------------------------- scan
constexpr int kScanThreads = 256;
constexpr int kScanItems = 8;
constexpr int kScanTile = kScanThreads * kScanItems;

__device__ __forceinline__ long long block_excl_scan(long long v, long long* total) {
  __shared__ long long ws[33];
  const int l = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  long long x = v;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    long long y = __shfl_up_sync(0xffffffffu, x, d);
    if (l >= d) x += y;
  }
  if (l == 31) ws[w] = x;
  __syncthreads();
  if (w == 0) {
    long long s = (l < nw) ? ws[l] : 0;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      long long y = __shfl_up_sync(0xffffffffu, s, d);
      if (l >= d) s += y;
    }
    if (l < nw) ws[l] = s;
    if (l == 31) ws[32] = s;
  }
  __syncthreads();
  long long r = ((w > 0) ? ws[w - 1] : 0) + x - v;
  *total = ws[32];
  __syncthreads();
  return r;
}

__global__ void __launch_bounds__(kScanThreads) k_scan_reduce(const long long* in, long long n, long long* bsum) {
  const long long base = (long long)blockIdx.x * kScanTile;
  long long s = 0;
#pragma unroll
  for (int t = 0; t < kScanItems; ++t) {
    long long idx = base + (long long)t * kScanThreads + threadIdx.x;
    if (idx < n) s += in[idx];
  }
  long long tot;
  block_excl_scan(s, &tot);
  if (threadIdx.x == 0) bsum[blockIdx.x] = tot;
}

__global__ void __launch_bounds__(1024) k_scan_top(long long* bsum, long long nb) {
  long long carry = 0;
  for (long long base = 0; base < nb; base += blockDim.x) {
    long long idx = base + threadIdx.x;
    long long v = (idx < nb) ? bsum[idx] : 0;
    long long tot;
    long long ex = block_excl_scan(v, &tot);
    if (idx < nb) bsum[idx] = carry + ex;
    carry += tot;
  }
}

__global__ void __launch_bounds__(kScanThreads) k_scan_apply(const long long* in, long long* out, long long n,
                                                             const long long* bsum) {
  const long long base = (long long)blockIdx.x * kScanTile;
  long long v[kScanItems];
  long long s = 0;
  // each thread owns kScanItems consecutive items
#pragma unroll
  for (int t = 0; t < kScanItems; ++t) {
    long long idx = base + (long long)threadIdx.x * kScanItems + t;
    v[t] = (idx < n) ? in[idx] : 0;
    s += v[t];
  }
  long long tot;
  long long run = block_excl_scan(s, &tot) + bsum[blockIdx.x];
#pragma unroll
  for (int t = 0; t < kScanItems; ++t) {
    long long idx = base + (long long)threadIdx.x * kScanItems + t;
    if (idx < n) out[idx] = run;
    run += v[t];
    if (idx == n - 1) out[n] = run;
  }
}

__global__ void k_set_zero_ll(long long* p) { *p = 0; }

// -------------------------------------------------------------- binning
struct RowBin {
  __device__ __forceinline__ static int get(const ProbD& P, long long g, int phase, const long long* rf,
                                            const long long* rfc, const long long* rowsize, const BinCfg& cfg) {
    const int b = inst_of(P.arow0s, P.ninst, g);
    const InstD& I = P.inst[b];
    const long long k = I.k;
    const long long kw = (k + 31) >> 5;
    if (phase == 2 || phase == 3) {
      // symbolic: phase 2 lists the rows of compressed products, phase 3 the others
      if ((phase == 2) != (I.compressed != 0)) return -1;
      if (I.compressed) {
        long long w = rfc[g];
        long long u = w < kw ? w : kw;
        return choose_bin(u, w, kw, kw, cfg);
      }
      long long w = rf[g];
      long long u = w < k ? w : k;
      return choose_bin(u, w, k, kw, cfg);
    }
    return choose_bin(rowsize[g], rf[g], k, kw, cfg);
  }
};

// Binning is stable: block b takes the contiguous rows [b * kBinRows,
// (b + 1) * kBinRows), counts them per bin into bcnt[bin * nblk + b], and the
// scatter places them in row order after the rows of earlier blocks, so each
// bin's list keeps the order of A's rows and concurrently running teams touch
// neighbouring rows of B.
__global__ void __launch_bounds__(kBinThreads) k_bin_count(ProbD P, long long totalA, int phase, const long long* rf,
                                                           const long long* rfc, const long long* rowsize,
                                                           BinCfg cfg, unsigned long long* hist, long long* bcnt,
                                                           long long nblk) {
  __shared__ unsigned long long h[kNumBins];
  for (int t = threadIdx.x; t < kNumBins; t += blockDim.x) h[t] = 0ull;
  __syncthreads();
  const long long r0 = (long long)blockIdx.x * kBinRows;
  const long long r1 = r0 + kBinRows < totalA ? r0 + kBinRows : totalA;
  bin_block_count(r0, r1, [&](long long g) { return RowBin::get(P, g, phase, rf, rfc, rowsize, cfg); }, h);
  __syncthreads();
  for (int t = threadIdx.x; t < kNumBins; t += blockDim.x) {
    bcnt[(long long)t * nblk + blockIdx.x] = (long long)h[t];
    if (h[t]) atomicAdd(&hist[t], h[t]);
  }
}

// cursor[bin]: first slot of the bin's list; bofs: exclusive scan of bcnt.
// Rows of the class-none bin are not listed (symbolic: their size is 0).
__global__ void __launch_bounds__(kBinThreads) k_bin_scatter(ProbD P, long long totalA, int phase,
                                                             const long long* rf, const long long* rfc,
                                                             long long* rowsize, BinCfg cfg,
                                                             const unsigned long long* cursor, const long long* bofs,
                                                             long long nblk, int* rows) {
  __shared__ long long run[kNumBins];
  __shared__ int wcnt[kBinThreads / 32][kNumBins];
  for (int t = threadIdx.x; t < kNumBins; t += blockDim.x) {
    run[t] = (long long)cursor[t] + bofs[(long long)t * nblk + blockIdx.x] - bofs[(long long)t * nblk];
    for (int w = 0; w < kBinThreads / 32; ++w) wcnt[w][t] = 0;
  }
  __syncthreads();
  const long long r0 = (long long)blockIdx.x * kBinRows;
  const long long r1 = r0 + kBinRows < totalA ? r0 + kBinRows : totalA;
  auto key = [&](long long g) {
    const int bin = RowBin::get(P, g, phase, rf, rfc, rowsize, cfg);
    if (bin >= 0 && bin_cls(bin) == kClsNone && phase != 1) rowsize[g] = 0;
    return (bin >= 0 && bin_cls(bin) != kClsNone) ? bin : -1;
  };
  bin_block_list(r0, r1, key, run, wcnt, rows);
}

// -------------------------------------------------------------- C row pointers
// inst_out per instance: [nnz(C), maxrs]
__global__ void __launch_bounds__(kBlock) k_write_rowptr(ProbD P, long long totalA, const long long* offs,
                                                         const long long* rowsize, unsigned long long* inst_out) {
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long base = (long long)blockIdx.x * blockDim.x; base < totalA; base += stride) {
    const long long g = base + threadIdx.x;
    int b = -1;
    unsigned rs = 0;
    if (g < totalA) {
      b = inst_of(P.arow0s, P.ninst, g);
      const InstD& I = P.inst[b];
      const long long i = g - I.arow0;
      const long long o0 = offs[I.arow0];
      I.Crp[i] = offs[g] - o0;
      if (i == I.A.nrows - 1) {
        I.Crp[i + 1] = offs[g + 1] - o0;
        inst_out[2ll * b] = (unsigned long long)(offs[g + 1] - o0);
      }
      rs = (unsigned)rowsize[g];
    }
    const int b0 = __shfl_sync(0xffffffffu, b, 0);
    if (__all_sync(0xffffffffu, b == b0)) {
      const unsigned mx = __reduce_max_sync(0xffffffffu, rs);
      if (b0 >= 0 && (threadIdx.x & 31) == 0) atomicMax(&inst_out[2ll * b0 + 1], (unsigned long long)mx);
    } else if (b >= 0) {
      atomicMax(&inst_out[2ll * b + 1], (unsigned long long)rs);
    }
  }
}

__global__ void k_empty_instances(ProbD P, unsigned long long* inst_out) {
  for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < P.ninst; b += gridDim.x * blockDim.x) {
    const InstD& I = P.inst[b];
    if (I.A.nrows == 0) {
      I.Crp[0] = 0;
      inst_out[2ll * b] = 0ull;
    }
  }
}

}  // namespace

// A few words from device memory into mapped pinned host memory.  The
// planning calls read their statistics back this way rather than with a copy
// engine, so the read-backs never queue behind large copies that the caller
// runs on other streams.
__global__ void k_copy_to_host(const unsigned* __restrict__ src, unsigned* dst, long long words) {
  for (long long x = (long long)blockIdx.x * blockDim.x + threadIdx.x; x < words; x += (long long)gridDim.x * blockDim.x)
    dst[x] = src[x];
}

// ============================================================== launchers
cudaError_t launch_copy_to_host(const LaunchCtx& L, void* dst_mapped, const void* src, size_t bytes) {
  if (bytes == 0) return cudaSuccess;
  const long long words = (long long)((bytes + 3) / 4);
  KKS_LAUNCHED();
  k_copy_to_host<<<(unsigned)std::min<long long>((words + 255) / 256, 64), 256, 0, L.stream>>>(
      reinterpret_cast<const unsigned*>(src), reinterpret_cast<unsigned*>(dst_mapped), words);
  return cudaGetLastError();
}

int resident_per_sm(const void* kernel, int threads, size_t smem) {
  struct Entry {
    const void* k;
    int dev, threads;
    size_t smem;
    int per_sm;
  };
  static std::mutex mu;
  static std::vector<Entry> cache;
  int dev = 0;
  cudaGetDevice(&dev);
  std::lock_guard<std::mutex> lock(mu);
  for (const Entry& e : cache)
    if (e.k == kernel && e.dev == dev && e.threads == threads && e.smem == smem) return e.per_sm;
  int n = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kernel, threads, smem) != cudaSuccess || n < 1) {
    cudaGetLastError();
    n = 1;
  }
  cache.push_back({kernel, dev, threads, smem, n});
  return n;
}

// Long-row queue layout: queue[0] = entries, [1] = fetch counter of the
// count pass, [2] = fetch counter of the fill pass (zeroed here).
cudaError_t launch_compress_count(const LaunchCtx& L, const ProbD& P, long long totalB, long long* cnt,
                                  unsigned long long* unsorted, const LongQueue& q, longlong2* blen) {
  if (totalB <= 0) return cudaSuccess;
  cudaError_t e = cudaMemsetAsync(q.ctr, 0, 3 * sizeof(unsigned long long), L.stream);
  if (e != cudaSuccess) return e;
  const long long grid = (totalB + kBlock - 1) / kBlock;
  KKS_LAUNCHED();
  k_compress_count<8><<<(unsigned)grid, kBlock, 0, L.stream>>>(P, totalB, cnt, unsorted, q.list, q.ctr, blen);
  KKS_LAUNCHED();
  k_compress_count_long<<<grid_for(totalB, kBlock, L.num_sms, 4), kBlock, 0, L.stream>>>(P, q.list, q.ctr, q.ctr + 1,
                                                                                        cnt, unsorted, blen);
  return cudaGetLastError();
}

cudaError_t launch_compress_fill(const LaunchCtx& L, const ProbD& P, long long totalB, int* csi, unsigned* cs,
                                 const LongQueue& q) {
  if (totalB <= 0) return cudaSuccess;
  const long long grid = (totalB + kBlock - 1) / kBlock;
  KKS_LAUNCHED();
  k_compress_fill<8><<<(unsigned)grid, kBlock, 0, L.stream>>>(P, totalB, csi, cs);
  KKS_LAUNCHED();
  k_compress_fill_long<<<grid_for(totalB, kBlock, L.num_sms, 4), kBlock, 0, L.stream>>>(P, q.list, q.ctr, q.ctr + 2,
                                                                                       csi, cs);
  return cudaGetLastError();
}

namespace {
// rf[i] = sum over A(i,:) of |B(j,:)| (Algorithm 1's multiplications of row i).
__global__ void k_row_flops(MatD A, MatD B, long long* rf, DevStatus* st) {
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < A.nrows; i += stride) {
    const long long a0 = rp_at(A, i), a1 = rp_at(A, i + 1);
    long long w = 0;
    if (a0 < 0 || a0 > a1 || a1 > A.nnz) {
      dev_fail(st, kDevBadIndex, 45, i);
    } else {
#pragma unroll 4
      for (long long p = a0; p < a1; ++p) {
        const int j = A.cj[p];
        if ((unsigned long long)(unsigned)j < (unsigned long long)B.nrows) w += rp_at(B, j + 1) - rp_at(B, j);
        else dev_fail(st, kDevBadIndex, 46, i);
      }
    }
    rf[i] = w;
  }
}
}  // namespace

cudaError_t launch_row_flops(const LaunchCtx& L, const MatD& A, const MatD& B, long long* rf, DevStatus* st) {
  if (A.nrows <= 0) return cudaSuccess;
  KKS_LAUNCHED();
  k_row_flops<<<grid_for(A.nrows, 256, L.num_sms, 16), 256, 0, L.stream>>>(A, B, rf, st);
  return cudaGetLastError();
}

__global__ void k_decide_compression(InstD* inst, const unsigned long long* st, int count, int mode, double thr) {
  for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < count; b += gridDim.x * blockDim.x) {
    const long long fm = (long long)st[4 * b], fmc = (long long)st[4 * b + 2];
    int c = 0;
    if (mode == 1) c = 1;
    else if (mode < 0 && fm > 0 && (double)fmc < thr * (double)fm) c = 1;
    inst[b].compressed = c;
  }
}

cudaError_t launch_decide_compression(const LaunchCtx& L, InstD* inst, const unsigned long long* inst_stats, int count,
                                      int mode, double threshold) {
  if (count <= 0) return cudaSuccess;
  KKS_LAUNCHED();
  k_decide_compression<<<(count + 255) / 256, 256, 0, L.stream>>>(inst, inst_stats, count, mode, threshold);
  return cudaGetLastError();
}

cudaError_t launch_row_stats(const LaunchCtx& L, const ProbD& P, long long totalA, int use_bc, long long* rf,
                             long long* rfc, unsigned long long* inst_stats, const LongQueue& q,
                             const longlong2* blen) {
  if (totalA <= 0) return cudaSuccess;
  cudaError_t e = cudaMemsetAsync(q.ctr, 0, 2 * sizeof(unsigned long long), L.stream);
  if (e != cudaSuccess) return e;
  const long long grid = (totalA + kBlock - 1) / kBlock;
  KKS_LAUNCHED();
  k_row_stats<8><<<(unsigned)grid, kBlock, 0, L.stream>>>(P, totalA, use_bc, rf, rfc, inst_stats, q.list, q.ctr,
                                                          blen);
  KKS_LAUNCHED();
  k_row_stats_long<<<grid_for(totalA, kBlock, L.num_sms, 4), kBlock, 0, L.stream>>>(P, use_bc, q.list, q.ctr,
                                                                                   q.ctr + 1, rf, rfc, inst_stats,
                                                                                   blen);
  return cudaGetLastError();
}

size_t scan_tmp_bytes(long long n) {
  long long nb = (n + kScanTile - 1) / kScanTile;
  if (nb < 1) nb = 1;
  return (size_t)nb * sizeof(long long);
}

cudaError_t launch_scan(const LaunchCtx& L, const long long* in, long long* out, long long n, void* tmp) {
  if (n <= 0) {
    KKS_LAUNCHED();
    k_set_zero_ll<<<1, 1, 0, L.stream>>>(out);
    return cudaGetLastError();
  }
  long long nb = (n + kScanTile - 1) / kScanTile;
  long long* bsum = (long long*)tmp;
  KKS_LAUNCHED();
  k_scan_reduce<<<(unsigned)nb, kScanThreads, 0, L.stream>>>(in, n, bsum);
  KKS_LAUNCHED();
  k_scan_top<<<1, 1024, 0, L.stream>>>(bsum, nb);
  KKS_LAUNCHED();
  k_scan_apply<<<(unsigned)nb, kScanThreads, 0, L.stream>>>(in, out, n, bsum);
  return cudaGetLastError();
}

cudaError_t launch_bin_count(const LaunchCtx& L, const ProbD& P, long long totalA, int phase, const long long* rf,
                             const long long* rfc, const long long* rowsize, BinCfg cfg, unsigned long long* hist,
                             long long* bcnt) {
  if (totalA <= 0) return cudaSuccess;
  const long long nblk = bin_blocks(totalA);
  KKS_LAUNCHED();
  k_bin_count<<<(unsigned)nblk, kBinThreads, 0, L.stream>>>(P, totalA, phase, rf, rfc, rowsize, cfg, hist, bcnt, nblk);
  return cudaGetLastError();
}

cudaError_t launch_bin_scatter(const LaunchCtx& L, const ProbD& P, long long totalA, int phase, const long long* rf,
                               const long long* rfc, const long long* rowsize, BinCfg cfg,
                               const unsigned long long* cursor, const long long* bofs, int* rows) {
  if (totalA <= 0) return cudaSuccess;
  const long long nblk = bin_blocks(totalA);
  KKS_LAUNCHED();
  k_bin_scatter<<<(unsigned)nblk, kBinThreads, 0, L.stream>>>(P, totalA, phase, rf, rfc, const_cast<long long*>(rowsize),
                                                         cfg, cursor, bofs, nblk, rows);
  return cudaGetLastError();
}

cudaError_t launch_write_rowptr(const LaunchCtx& L, const ProbD& P, long long totalA, const long long* offs,
                                const long long* rowsize, unsigned long long* inst_out) {
  KKS_LAUNCHED();
  k_empty_instances<<<(P.ninst + 255) / 256, 256, 0, L.stream>>>(P, inst_out);
  if (totalA > 0) {
    int grid = grid_for(totalA, kBlock, L.num_sms, 8);
    KKS_LAUNCHED();
    k_write_rowptr<<<grid, kBlock, 0, L.stream>>>(P, totalA, offs, rowsize, inst_out);
  }
  return cudaGetLastError();
}

}  // namespace kks
