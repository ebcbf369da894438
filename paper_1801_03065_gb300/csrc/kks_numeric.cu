// kks_numeric.cu -- numeric phase: columns and values of every row of C.
//
// Algorithm 3 with Phase = numeric: each product A(i,j) * B(j,l) is inserted
// (accumulated) into the team's accumulator under key l; at the end of the
// row the accumulator is written to C(i,:) at C_row_pointers(i).  The output
// is canonical: every row is written sorted by column.
//   k_num_hash<TW, VT>  : shared LP table (key, value) holding the whole row;
//                         emission = compaction + bitonic sort of
//                         (column << 32 | slot) in shared memory
//   k_num_dense<TW, VT> : dense accumulator (Section 3.1.2): values in a
//                         global k-wide pool chunk, column marker as a bitmap
//                         in shared memory; emission walks the bitmap, so the
//                         row comes out sorted and the chunk is reset to zero
//   k_num_spill<TW, VT> : two-level LP accumulator (Algorithm 3, Section 3.1.2):
//                         L1 in shared memory with the maximum-occupancy
//                         cut-off, L2 in a global pool chunk; L2 entries whose
//                         key also reached L1 are folded into L1, then each
//                         entry is written at its rank from a column bitmap
#include "kks_internal.h"

namespace kks {

namespace {

__host__ __device__ constexpr size_t al16(size_t x) { return (x + 15) & ~size_t(15); }

// CTA teams (one row per CTA).  kw_cap > 0: every row of the plan has a
// column range of at most kw_cap 32-bit words and is written by rank instead
// of sorted: a k-bit bitmap of the row's columns, the count of set bits before
// every word (16 bits: a row holds at most T / 2 < 65 536 columns), and for
// each entry the rank = that count + set bits below it in its word.  This
// replaces a block-wide bitonic sort with O(k / 32 + s) work, and the table
// needs no sort buffer.
constexpr long long kRankMaxWords = 16384;   // rank bitmaps cover k <= 524 288 columns

template <int TW, typename VT>
__host__ __device__ size_t num_cta_bytes(int T, long long kw_cap) {
  const int half = T / 2 > 0 ? T / 2 : 1;
  size_t b = al16((size_t)T * sizeof(VT)) + al16((size_t)T * 4) + al16(sizeof(ChunkScratch<TW, VT>)) +
             al16((size_t)kStagedPasses * TW * 4) + 16;
  if (kw_cap > 0) return b + al16((size_t)((kw_cap + 3) & ~3ll) * 4) + al16((size_t)(kw_cap + 1) * 2);
  return b + al16((size_t)half * 8);
}

// Direct rows (rank bitmap in use, the row's products fit half the table):
// no hash table.  Product x of the row is stored at slot x of the table's
// first half and its column marked in the bitmap; a bit that was already set
// flags the product as a repeat of its column.  After the prefix of the words
// each product knows its column's rank in C(i,:): first occurrences are
// stored at that rank in the second half, repeats added there after a
// barrier, and the second half is written out in order.  This drops the
// table reset, the probes and the two sweeps of the table per row, which
// dominate rows of random columns (few repeats, table half empty).
constexpr int kRepeatFlag = int(0x80000000u);

template <int TW, typename VT>
__global__ void __launch_bounds__(TW) k_num_hash(ProbD P, const int* __restrict__ rows, long long nrows, int logT,
                                                 long long kw_cap, unsigned long long* fetch) {
  static_assert(TW > 32, "CTA teams only");
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ long long scan_scratch[33];
  __shared__ long long fetch_s;
  Team<TW> tm;
  const int T = 1 << logT;
  const LpHash tmask(logT, P.hash_mode);
  const int half = T / 2 > 0 ? T / 2 : 1;
  VT* vals = reinterpret_cast<VT*>(smem);
  int* keys = reinterpret_cast<int*>(smem + al16((size_t)T * sizeof(VT)));
  ChunkScratch<TW, VT>* csc =
      reinterpret_cast<ChunkScratch<TW, VT>*>(smem + al16((size_t)T * sizeof(VT)) + al16((size_t)T * 4));
  int* seg = reinterpret_cast<int*>(reinterpret_cast<unsigned char*>(csc) + al16(sizeof(ChunkScratch<TW, VT>)));
  unsigned char* tail =
      reinterpret_cast<unsigned char*>(seg) + al16((size_t)kStagedPasses * TW * 4) + 16;
  unsigned long long* sortb = reinterpret_cast<unsigned long long*>(tail);   // kw_cap == 0
  unsigned* bm = reinterpret_cast<unsigned*>(tail);                          // kw_cap > 0
  unsigned short* gp = reinterpret_cast<unsigned short*>(bm + ((kw_cap + 3) & ~3ll));

  for (long long r = cta_next_row(fetch, &fetch_s); r < nrows; r = cta_next_row(fetch, &fetch_s)) {
    const long long g = rows[r];
    const int b = inst_of(P.arow0s, P.ninst, g);
    const InstD& I = P.inst[b];
    const long long i = g - I.arow0;
    const long long c0 = I.Crp[i];
    const long long s = I.Crp[i + 1] - c0;
    const long long a0 = rp_at(I.A, i), a1 = rp_at(I.A, i + 1);
    const VT* __restrict__ Ax = reinterpret_cast<const VT*>(I.A.vx);
    const VT* __restrict__ Bx = reinterpret_cast<const VT*>(I.B.vx);
    const int* __restrict__ Bj = I.B.cj;
    const long long kw = (I.k + 31) >> 5;
    const bool ranked = kw_cap > 0 && kw <= kw_cap;
    auto range = [&](int j, long long* bs, long long* be) {
      *bs = rp_at(I.B, j);
      *be = rp_at(I.B, j + 1);
    };
    auto aval = [&](long long p) { return Ax[p]; };
    auto pf = [&](long long q) {
      prefetch_l1(Bj + q);
      prefetch_l1(Bx + q);
    };
    // set bits before every word of the rank bitmap: each thread sums a
    // contiguous run of words, the runs are scanned across the team, then
    // each word gets its prefix; returns the row's column count
    auto word_prefix = [&]() {
      const long long sg = (kw + TW - 1) / TW;
      const long long w0 = tm.lane * sg, w1 = w0 + sg < kw ? w0 + sg : kw;
      int cseg = 0;
      for (long long w = w0; w < w1; ++w) cseg += __popc(bm[w]);
      long long run;
      long long pre = team_excl_scan<TW>(tm, cseg, &run, scan_scratch);
      for (long long w = w0; w < w1; ++w) {
        gp[w] = (unsigned short)pre;
        pre += __popc(bm[w]);
      }
      return run;
    };
    if (ranked) {
      for (long long w = tm.lane; w < kw; w += TW) bm[w] = 0u;
      // the product count: the chunk's scan when A(i,:) is one chunk (kept
      // for its products), else a sum over the row
      const bool one = a1 - a0 <= TW;
      long long f = 0, ex1 = 0, bs1 = 0, be1 = 0;
      if (one) {
        const long long p = a0 + tm.lane;
        VT av = VT(0);
        if (p < a1) {
          range(I.A.cj[p], &bs1, &be1);
          av = Ax[p];
        }
        ex1 = chunk_scan<TW, VT>(tm, csc, scan_scratch, bs1, be1, av, &f);
      } else {
        for (long long p = a0 + tm.lane; p < a1; p += TW) {
          const int j = I.A.cj[p];
          f += rp_at(I.B, j + 1) - rp_at(I.B, j);
        }
        f = team_sum<TW>(tm, f, scan_scratch);
      }
      if (f <= half) {
        int* okeys = keys + half;
        VT* ovals = vals + half;
        long long base = 0;
        int repeats = 0;
        auto dbody = [&](long long q, int t) {
          const int col = Bj[q];
          const long long x = base + csc->pre[t] + (q - csc->bs[t]);
          if ((unsigned long long)(unsigned)col < (unsigned long long)I.k) {
            const unsigned bit = 1u << (col & 31);
            const unsigned old = atomicOr(bm + (col >> 5), bit);
            const bool rep = (old & bit) != 0u;
            repeats |= rep ? 1 : 0;
            keys[x] = rep ? (col | kRepeatFlag) : col;
            vals[x] = csc->av[t] * Bx[q];
          } else {
            keys[x] = kEmpty;
            dev_fail(P.status, kDevBadIndex, 15, g);
          }
        };
        if (one) {
          chunk_products<TW, VT>(tm, csc, scan_scratch, ex1, f, bs1, be1, dbody, pf, seg);
        } else {
          for (long long c = a0; c < a1; c += TW) {
            const long long p = c + tm.lane;
            long long bs = 0, be = 0;
            VT av = VT(0);
            if (p < a1) {
              range(I.A.cj[p], &bs, &be);
              av = Ax[p];
            }
            base += for_each_product_chunk<TW, VT>(tm, csc, scan_scratch, bs, be, av, dbody, pf, seg);
          }
        }
        const long long run = word_prefix();
        if (tm.lane == 0 && run != s) dev_fail(P.status, kDevRowSizeMismatch, 16, g);
        tm.sync();
        auto rank_of = [&](int col) {
          const int w = col >> 5;
          return (long long)gp[w] + __popc(bm[w] & ((1u << (col & 31)) - 1u));
        };
        for (long long x = tm.lane; x < f; x += TW) {
          const int kk = keys[x];
          if (kk < 0) continue;
          const long long rk = rank_of(kk);
          if (rk < s) {
            okeys[rk] = kk;
            ovals[rk] = vals[x];
          }
        }
        if (__syncthreads_or(repeats)) {
          for (long long x = tm.lane; x < f; x += TW) {
            const int kk = keys[x];
            if (kk >= 0 || kk == kEmpty) continue;
            const long long rk = rank_of(kk & ~kRepeatFlag);
            if (rk < s) atomicAdd(ovals + rk, vals[x]);
          }
          tm.sync();
        }
        VT* __restrict__ Cx = reinterpret_cast<VT*>(I.Cx);
        int* __restrict__ Cj = I.Cj;
        const long long nw = run < s ? run : s;
        for (long long x = tm.lane; x < nw; x += TW) {
          Cj[c0 + x] = okeys[x];
          Cx[c0 + x] = ovals[x];
        }
        continue;
      }
    }
    for (int x = tm.lane; x < T; x += TW) {
      keys[x] = kEmpty;
      vals[x] = VT(0);
    }
    tm.sync();
    auto body = [&](long long q, int t) {
      const int key = Bj[q];
      const VT v = csc->av[t] * Bx[q];
      const int slot = lp_insert(keys, tmask, nullptr, -1, key);
      if (slot >= 0) atomicAdd(vals + slot, v);
      else dev_fail(P.status, kDevTableFull, 10, g);
    };
    for_each_product<TW, VT>(tm, csc, scan_scratch, I.A.cj, a0, a1, range, aval, body, pf, seg);
    if (ranked) {
      VT* __restrict__ Cx = reinterpret_cast<VT*>(I.Cx);
      int* __restrict__ Cj = I.Cj;
      // (the bitmap was cleared before the row's products)
      for (int x = tm.lane; x < T; x += TW) {
        const int kk = keys[x];
        if (kk == kEmpty) continue;
        if ((unsigned long long)(unsigned)kk < (unsigned long long)I.k) atomicOr(bm + (kk >> 5), 1u << (kk & 31));
        else dev_fail(P.status, kDevBadIndex, 17, g);
      }
      tm.sync();
      const long long run = word_prefix();
      if (tm.lane == 0 && run != s) dev_fail(P.status, kDevRowSizeMismatch, 9, g);
      tm.sync();
      for (int x = tm.lane; x < T; x += TW) {
        const int kk = keys[x];
        if (kk == kEmpty || (unsigned long long)(unsigned)kk >= (unsigned long long)I.k) continue;
        const int w = kk >> 5;
        const long long rk = (long long)gp[w] + __popc(bm[w] & ((1u << (kk & 31)) - 1u));
        if (rk < s) {
          Cj[c0 + rk] = kk;
          Cx[c0 + rk] = vals[x];
        }
      }
      tm.sync();
      continue;
    }
    // compaction of the occupied slots into (column << 32 | slot)
    long long cnt = 0;
    for (int xb = 0; xb < T; xb += TW) {
      const int x = xb + tm.lane;
      const bool o = x < T && keys[x] != kEmpty;
      long long tot;
      const long long ex = team_excl_scan<TW>(tm, o ? 1 : 0, &tot, scan_scratch);
      if (o && cnt + ex < half)
        sortb[cnt + ex] = ((unsigned long long)(unsigned)keys[x] << 32) | (unsigned)x;
      cnt += tot;
    }
    if (tm.lane == 0 && cnt != s) dev_fail(P.status, kDevRowSizeMismatch, 11, g);
    const int n = (int)(cnt < half ? cnt : half);
    int N = 1;
    while (N < n) N <<= 1;
    for (int x = n + tm.lane; x < N; x += TW) sortb[x] = ~0ull;
    tm.sync();
    team_bitonic<TW>(tm, sortb, N);
    const long long nw = n < s ? n : s;
    VT* __restrict__ Cx = reinterpret_cast<VT*>(I.Cx);
    int* __restrict__ Cj = I.Cj;
    for (long long x = tm.lane; x < nw; x += TW) {
      const unsigned long long e = sortb[x];
      Cj[c0 + x] = (int)(e >> 32);
      Cx[c0 + x] = vals[(unsigned)(e & 0xffffffffull)];
    }
    tm.sync();
  }
}

// ---------------------------------------------------------------------------
// The other partitioning schemes of Section 3.1.1 for CTA rows, offered to the
// autotuner beside the flat kernel above (Thread-Flat-Parallel):
//  kPartTeamSeq, Team-Sequential with the linked-list accumulator (LL) of
//    Section 3.1.2: the whole CTA takes the entries of A(i,:) one at a time
//    and spreads B(j,:) over its threads, so the keys of a pass are distinct.
//    A key is looked up by walking its bucket's list and its value updated
//    without atomics; a new key takes the next node (an atomic counter) and
//    is pushed at the head of its list with a compare-and-swap.  Nodes fill
//    0, 1, ... in order, so the row's keys are compact for the sort.
//  kPartThreadPar, Thread-Parallel: each warp takes its own entries of A(i,:)
//    and its lanes share B(j,:); the warps insert into the LP table together,
//    values with atomic adds.
// The LP table has 2^logT slots; LL has 2^logT / 2 nodes and as many buckets
// (a row of the bin has at most 2^logT / 2 columns).
// ---------------------------------------------------------------------------
constexpr int kPartTeamSeq = 1;
constexpr int kPartThreadPar = 2;

template <int TW, typename VT>
__host__ __device__ size_t part_cta_bytes(int T) {
  const size_t half = T / 2 > 0 ? (size_t)(T / 2) : 1;
  const size_t lp = al16((size_t)T * sizeof(VT)) + al16((size_t)T * 4);
  const size_t ll = al16(half * 4) * 3 + al16(half * sizeof(VT));
  return (lp > ll ? lp : ll) + al16(half * 8) + 16;
}

template <int TW, typename VT, int MODE>
__global__ void __launch_bounds__(TW) k_num_part(ProbD P, const int* __restrict__ rows, long long nrows, int logT,
                                                 unsigned long long* fetch) {
  static_assert(TW > 32, "CTA teams only");
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ long long scan_scratch[33];
  __shared__ long long fetch_s;
  Team<TW> tm;
  const int T = 1 << logT;
  const int half = T / 2 > 0 ? T / 2 : 1;
  const size_t lp = al16((size_t)T * sizeof(VT)) + al16((size_t)T * 4);
  const size_t llb = al16((size_t)half * 4) * 3 + al16((size_t)half * sizeof(VT));
  unsigned long long* sortb = reinterpret_cast<unsigned long long*>(smem + (lp > llb ? lp : llb));
  int* counter = reinterpret_cast<int*>(reinterpret_cast<unsigned char*>(sortb) + al16((size_t)half * 8));
  // LP layout
  VT* lvals = reinterpret_cast<VT*>(smem);
  int* lkeys = reinterpret_cast<int*>(smem + al16((size_t)T * sizeof(VT)));
  // LL layout
  int* begins = reinterpret_cast<int*>(smem);
  int* ids = reinterpret_cast<int*>(smem + al16((size_t)half * 4));
  int* nexts = reinterpret_cast<int*>(smem + 2 * al16((size_t)half * 4));
  VT* nvals = reinterpret_cast<VT*>(smem + 3 * al16((size_t)half * 4));
  const int lane32 = threadIdx.x & 31, warp = threadIdx.x >> 5;
  constexpr int kWarps = TW / 32;

  for (long long r = cta_next_row(fetch, &fetch_s); r < nrows; r = cta_next_row(fetch, &fetch_s)) {
    const long long g = rows[r];
    const int b = inst_of(P.arow0s, P.ninst, g);
    const InstD& I = P.inst[b];
    const long long i = g - I.arow0;
    const long long c0 = I.Crp[i];
    const long long s = I.Crp[i + 1] - c0;
    const long long a0 = rp_at(I.A, i), a1 = rp_at(I.A, i + 1);
    const VT* __restrict__ Ax = reinterpret_cast<const VT*>(I.A.vx);
    const VT* __restrict__ Bx = reinterpret_cast<const VT*>(I.B.vx);
    const int* __restrict__ Bj = I.B.cj;
    const int* __restrict__ Aj = I.A.cj;
    long long cnt = 0;
    if (MODE == kPartTeamSeq) {
      for (int x = tm.lane; x < half; x += TW) begins[x] = -1;
      if (tm.lane == 0) *counter = 0;
      const LpHash hb(ilog2_ceil(half), P.hash_mode);
      tm.sync();
      for (long long p = a0; p < a1; ++p) {
        const int j = Aj[p];
        const VT a = Ax[p];
        const long long bs = rp_at(I.B, j), be = rp_at(I.B, j + 1);
        for (long long q = bs + tm.lane; q < be; q += TW) {
          const int key = Bj[q];
          const VT v = a * Bx[q];
          const unsigned h = hb(key);
          int e = *((volatile int*)(begins + h));
          bool found = false;
          for (int steps = 0; e >= 0 && steps < half; ++steps) {
            if (*((volatile int*)(ids + e)) == key) {
              nvals[e] += v;   // the keys of a pass are distinct: no other thread holds this node
              found = true;
              break;
            }
            e = *((volatile int*)(nexts + e));
          }
          if (found) continue;
          const int slot = atomicAdd(counter, 1);
          if (slot >= half) {
            dev_fail(P.status, kDevTableFull, 14, g);
            continue;
          }
          ids[slot] = key;
          nvals[slot] = v;
          // push at the head of the list; a failed compare-and-swap means another
          // thread pushed first, so the retries are bounded by the CTA's threads
          int head = *((volatile int*)(begins + h));
          bool pushed = false;
          for (int tries = 0; tries <= 2 * TW && !pushed; ++tries) {
            nexts[slot] = head;
            __threadfence_block();
            const int old = atomicCAS(begins + h, head, slot);
            pushed = old == head;
            head = old;
          }
          if (!pushed) dev_fail(P.status, kDevTableFull, 17, g);
        }
        tm.sync();   // the next pass may find these keys
      }
      cnt = *counter < half ? *counter : half;
      for (int x = tm.lane; x < cnt; x += TW) sortb[x] = ((unsigned long long)(unsigned)ids[x] << 32) | (unsigned)x;
    } else {
      for (int x = tm.lane; x < T; x += TW) {
        lkeys[x] = kEmpty;
        lvals[x] = VT(0);
      }
      const LpHash hs(logT, P.hash_mode);
      tm.sync();
      for (long long p = a0 + warp; p < a1; p += kWarps) {
        const int j = Aj[p];
        const VT a = Ax[p];
        const long long bs = rp_at(I.B, j), be = rp_at(I.B, j + 1);
        for (long long q = bs + lane32; q < be; q += 32) {
          const int slot = lp_insert(lkeys, hs, nullptr, -1, Bj[q]);
          if (slot >= 0) atomicAdd(lvals + slot, a * Bx[q]);
          else dev_fail(P.status, kDevTableFull, 15, g);
        }
      }
      tm.sync();
      for (int xb = 0; xb < T; xb += TW) {
        const int x = xb + tm.lane;
        const bool o = x < T && lkeys[x] != kEmpty;
        long long tot;
        const long long ex = team_excl_scan<TW>(tm, o ? 1 : 0, &tot, scan_scratch);
        if (o && cnt + ex < half) sortb[cnt + ex] = ((unsigned long long)(unsigned)lkeys[x] << 32) | (unsigned)x;
        cnt += tot;
      }
    }
    if (tm.lane == 0 && cnt != s) dev_fail(P.status, kDevRowSizeMismatch, 16, g);
    const int n = (int)(cnt < half ? cnt : half);
    int N = 1;
    while (N < n) N <<= 1;
    for (int x = n + tm.lane; x < N; x += TW) sortb[x] = ~0ull;
    tm.sync();
    team_bitonic<TW>(tm, sortb, N);
    const long long nw = n < s ? n : s;
    VT* __restrict__ Cx = reinterpret_cast<VT*>(I.Cx);
    int* __restrict__ Cj = I.Cj;
    const VT* vsrc = MODE == kPartTeamSeq ? nvals : lvals;
    for (long long x = tm.lane; x < nw; x += TW) {
      const unsigned long long e = sortb[x];
      Cj[c0 + x] = (int)(e >> 32);
      Cx[c0 + x] = vsrc[(unsigned)(e & 0xffffffffull)];
    }
  }
}

// ---------------------------------------------------------------------------
// Warp / sub-warp teams (TW <= 32).  Products go into the LP table with plain
// read-modify-writes of the values: no two lanes ever update one slot in the
// same step, so no floating-point atomics are needed.
//  * sequential mode (the chunk's B rows average >= TW/2 entries): one B row
//    per pass, so the keys of a pass are distinct (the paper's Thread-Sequential
//    guarantee of unique inserts, Section 3.1.1);
//  * flat mode (short B rows): products of several B rows share a pass; equal
//    keys are grouped with __match_any_sync, their values summed through a
//    per-team exchange buffer, and only the group's first lane updates.
// ---------------------------------------------------------------------------
// Warp rows of more than 2 * TW keys are emitted by a bucket sort (below)
// unless a bucket would hold more than this many keys.
constexpr int kBucketMax = 24;

// Bucket sort of a warp row's n entries (column << 32 | position) of sortb
// into outb: each entry goes to its bucket (an equal share of [kmn, kmx], a
// power of two >= n of them, at most `half`) by a count in bcnt, a scan and a
// scatter, and each lane sorts its buckets by insertion.  The entries of outb
// carry their position in sortb.  Returns false (outb undefined) when the
// fullest bucket would hold more than kBucketMax entries (keys bunched
// unevenly), for a bitonic sort instead.
__device__ __forceinline__ bool warp_bucket_sort(const unsigned long long* sortb, unsigned long long* outb,
                                                 int* bcnt, int n, unsigned kmn, unsigned kmx) {
  constexpr int TW = 32;
  const int lane = threadIdx.x & 31;
  int nb = 32;
  while (nb < n) nb <<= 1;
  int sh = 0;
  while (((kmx - kmn) >> sh) >= (unsigned)nb) ++sh;
  for (int b = lane; b < nb; b += TW) bcnt[b] = 0;
  __syncwarp();
  for (int x = lane; x < n; x += TW) {
    const unsigned key = (unsigned)(sortb[x] >> 32);
    atomicAdd(&bcnt[(key - kmn) >> sh], 1);
  }
  __syncwarp();
  // exclusive scan of the counts: each lane a contiguous run of nb / 32 buckets
  const int per = nb / TW;
  int run = 0, mxb = 0;
  for (int q = 0; q < per; ++q) {
    const int c = bcnt[lane * per + q];
    run += c;
    mxb = max(mxb, c);
  }
  int incl = run;
#pragma unroll
  for (int d = 1; d < TW; d <<= 1) {
    const int y = __shfl_up_sync(0xffffffffu, incl, d);
    if (lane >= d) incl += y;
  }
  mxb = __reduce_max_sync(0xffffffffu, (unsigned)mxb);
  if (mxb > kBucketMax) return false;
  int start = incl - run;
  for (int q = 0; q < per; ++q) {
    const int c = bcnt[lane * per + q];
    bcnt[lane * per + q] = start;
    start += c;
  }
  __syncwarp();
  for (int x = lane; x < n; x += TW) {
    const unsigned long long e = sortb[x];
    const int b = (int)(((unsigned)(e >> 32) - kmn) >> sh);
    const int at = atomicAdd(&bcnt[b], 1);
    outb[at] = (e & 0xffffffff00000000ull) | (unsigned)x;
  }
  __syncwarp();
  // bcnt[b] is now the end of bucket b; the start is the end of b - 1
  for (int b = lane; b < nb; b += TW) {
    const int e1 = bcnt[b], e0 = b > 0 ? bcnt[b - 1] : 0;
    for (int x = e0 + 1; x < e1; ++x) {
      const unsigned long long v = outb[x];
      int y = x - 1;
      while (y >= e0 && outb[y] > v) {
        outb[y + 1] = outb[y];
        --y;
      }
      outb[y + 1] = v;
    }
  }
  __syncwarp();
  return true;
}

template <int TW, typename VT>
__host__ __device__ size_t warp_team_bytes(int T) {
  const int half = T / 2 > 0 ? T / 2 : 1;
  return al16((size_t)T * sizeof(VT)) + al16((size_t)T * 4) + al16((size_t)half * 8) +
         al16(sizeof(ChunkScratch<TW, VT>)) + al16((size_t)TW * sizeof(VT));
}

template <int TW, typename VT>
__global__ void __launch_bounds__(256, 3) k_num_warp(ProbD P, const int* __restrict__ rows, long long nrows, int logT) {
  extern __shared__ __align__(16) unsigned char smem[];
  Team<TW> tm;
  const int T = 1 << logT;
  const LpHash tmask(logT, P.hash_mode);
  const int half = T / 2 > 0 ? T / 2 : 1;
  unsigned char* base = smem + (size_t)tm.id * warp_team_bytes<TW, VT>(T);
  VT* vals = reinterpret_cast<VT*>(base);
  int* keys = reinterpret_cast<int*>(base + al16((size_t)T * sizeof(VT)));
  unsigned long long* sortb =
      reinterpret_cast<unsigned long long*>(base + al16((size_t)T * sizeof(VT)) + al16((size_t)T * 4));
  ChunkScratch<TW, VT>* csc = reinterpret_cast<ChunkScratch<TW, VT>*>(
      base + al16((size_t)T * sizeof(VT)) + al16((size_t)T * 4) + al16((size_t)half * 8));
  VT* xchg = reinterpret_cast<VT*>(reinterpret_cast<unsigned char*>(csc) + al16(sizeof(ChunkScratch<TW, VT>)));
  const unsigned lane_lt = (1u << tm.lane) - 1u;
  const int lane_base = (threadIdx.x & 31) & ~(TW - 1);

  const long long team = (long long)blockIdx.x * tm.per_cta + tm.id;
  const long long nteams = (long long)gridDim.x * tm.per_cta;
  for (long long r = team; r < nrows; r += nteams) {
    const long long g = rows[r];
    const int b = inst_of(P.arow0s, P.ninst, g);
    const InstD& I = P.inst[b];
    const long long i = g - I.arow0;
    const long long c0 = I.Crp[i];
    const long long s = I.Crp[i + 1] - c0;
    const long long a0 = rp_at(I.A, i), a1 = rp_at(I.A, i + 1);
    const VT* __restrict__ Ax = reinterpret_cast<const VT*>(I.A.vx);
    const VT* __restrict__ Bx = reinterpret_cast<const VT*>(I.B.vx);
    const int* __restrict__ Bj = I.B.cj;
    const int* __restrict__ Aj = I.A.cj;
    VT* __restrict__ Cx = reinterpret_cast<VT*>(I.Cx);
    int* __restrict__ Cj = I.Cj;
    if constexpr (TW == 32) {
      // Direct rows (products fit half the table): no hash table.  Product x
      // of the row is stored at position x, value in the key region and
      // (column << 32 | x) in the sort buffer; the entries are sorted by
      // column (then position), and the first entry of each column sums its
      // run and writes C(i,:) at its rank.  This drops the table reset, the
      // probes and the compaction sweep, which dominate rows of random
      // columns (few repeats, table half empty).
      long long f = 0;
      for (long long p = a0 + tm.lane; p < a1; p += TW) {
        const int j = Aj[p];
        f += rp_at(I.B, j + 1) - rp_at(I.B, j);
      }
#pragma unroll
      for (int d = 16; d > 0; d >>= 1) f += __shfl_xor_sync(0xffffffffu, f, d);
      if (f > 0 && f <= half) {
        const int n = (int)f;
        VT* cv = reinterpret_cast<VT*>(keys);   // half values
        unsigned kmn = 0xffffffffu, kmx = 0u;
        int base = 0;
        for (long long c = a0; c < a1; c += TW) {
          const long long p = c + tm.lane;
          long long bs = 0;
          int len = 0;
          VT av = VT(0);
          if (p < a1) {
            const int j = Aj[p];
            bs = rp_at(I.B, j);
            len = (int)(rp_at(I.B, j + 1) - bs);
            av = Ax[p];
          }
          int ex = len;
#pragma unroll
          for (int d = 1; d < 32; d <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, ex, d);
            if (tm.lane >= d) ex += y;
          }
          const int tot = __shfl_sync(0xffffffffu, ex, 31);
          csc->pre[tm.lane] = ex - len;
          csc->bs[tm.lane] = bs;
          csc->av[tm.lane] = av;
          if (tm.lane == 0) csc->pre[TW] = tot;
          __syncwarp();
          // the B entries of kDirectU passes are located and loaded together
          // (their latencies overlap), then stored
          constexpr int kDirectU = 4;
          int t = 0;
          for (int xb = 0; xb < tot; xb += kDirectU * TW) {
            long long q[kDirectU];
            int tt[kDirectU], col[kDirectU];
            VT bv[kDirectU];
#pragma unroll
            for (int u = 0; u < kDirectU; ++u) {
              const int x = xb + u * TW + tm.lane;
              q[u] = -1;
              if (x < tot) {
                while (csc->pre[t + 1] <= x) ++t;
                q[u] = csc->bs[t] + (x - csc->pre[t]);
              }
              tt[u] = t;
            }
#pragma unroll
            for (int u = 0; u < kDirectU; ++u) {
              col[u] = q[u] >= 0 ? Bj[q[u]] : 0;
              bv[u] = q[u] >= 0 ? Bx[q[u]] : VT(0);
            }
#pragma unroll
            for (int u = 0; u < kDirectU; ++u) {
              if (q[u] < 0) continue;
              const int x = base + xb + u * TW + tm.lane;
              if ((unsigned long long)(unsigned)col[u] >= (unsigned long long)I.k) dev_fail(P.status, kDevBadIndex, 20, g);
              sortb[x] = ((unsigned long long)(unsigned)col[u] << 32) | (unsigned)x;
              cv[x] = csc->av[tt[u]] * bv[u];
              kmn = min(kmn, (unsigned)col[u]);
              kmx = max(kmx, (unsigned)col[u]);
            }
          }
          base += tot;
          __syncwarp();
        }
        kmn = __reduce_min_sync(0xffffffffu, kmn);
        kmx = __reduce_max_sync(0xffffffffu, kmx);
        const unsigned long long* srt = sortb;
        unsigned long long* outb = reinterpret_cast<unsigned long long*>(vals);   // half entries
        int* bcnt = sizeof(VT) == 8 ? reinterpret_cast<int*>(outb + half) : reinterpret_cast<int*>(cv + half);
        if (n > 2 * TW && warp_bucket_sort(sortb, outb, bcnt, n, kmn, kmx)) {
          srt = outb;
        } else {
          int N = 1;
          while (N < n) N <<= 1;
          for (int x = n + tm.lane; x < N; x += TW) sortb[x] = ~0ull;
          __syncwarp();
          team_bitonic<TW>(tm, sortb, N);
        }
        // runs of equal columns: the first entry of each sums the run
        int run = 0;
        for (int xb = 0; xb < n; xb += TW) {
          const int x = xb + tm.lane;
          unsigned col = 0u;
          bool head = false;
          if (x < n) {
            col = (unsigned)(srt[x] >> 32);
            head = x == 0 || (unsigned)(srt[x - 1] >> 32) != col;
          }
          const unsigned bal = __ballot_sync(0xffffffffu, head);
          if (head) {
            const long long rk = run + __popc(bal & lane_lt);
            VT v = cv[(unsigned)(srt[x] & 0xffffffffull)];
            for (int y = x + 1; y < n && (unsigned)(srt[y] >> 32) == col; ++y) v += cv[(unsigned)(srt[y] & 0xffffffffull)];
            if (rk < s) {
              Cj[c0 + rk] = (int)col;
              Cx[c0 + rk] = v;
            }
          }
          run += __popc(bal);
        }
        if (tm.lane == 0 && run != s) dev_fail(P.status, kDevRowSizeMismatch, 21, g);
        __syncwarp();
        continue;
      }
    }
    for (int x = tm.lane; x < T; x += TW) {
      keys[x] = kEmpty;
      vals[x] = VT(0);
    }
    __syncwarp(tm.mask);
    for (long long c = a0; c < a1; c += TW) {
      const long long p = c + tm.lane;
      long long bs = 0;
      int len = 0;
      VT av = VT(0);
      if (p < a1) {
        const int j = Aj[p];
        bs = rp_at(I.B, j);
        len = (int)(rp_at(I.B, j + 1) - bs);
        av = Ax[p];
      }
      const int nc = (a1 - c) < TW ? (int)(a1 - c) : TW;
      int tot = len;
#pragma unroll
      for (int d = TW / 2; d > 0; d >>= 1) tot += __shfl_xor_sync(tm.mask, tot, d, TW);
      if (2 * tot >= nc * TW) {
        // sequential: one B row per pass, distinct keys inside a pass; the
        // first TW entries of kU passes are loaded together to overlap their
        // latencies, then inserted pass by pass
        constexpr int kU = 4;
        for (int t0 = 0; t0 < nc; t0 += kU) {
          int key[kU], lent[kU];
          long long bst[kU];
          VT at[kU], bv[kU];
#pragma unroll
          for (int u = 0; u < kU; ++u) {
            const int t = (t0 + u < nc) ? t0 + u : nc - 1;
            bst[u] = __shfl_sync(tm.mask, bs, t, TW);
            const int l = __shfl_sync(tm.mask, len, t, TW);
            at[u] = __shfl_sync(tm.mask, av, t, TW);
            lent[u] = (t0 + u < nc) ? l : 0;
            key[u] = -1;
            bv[u] = VT(0);
            if (tm.lane < lent[u]) {
              key[u] = Bj[bst[u] + tm.lane];
              bv[u] = Bx[bst[u] + tm.lane];
            }
          }
#pragma unroll
          for (int u = 0; u < kU; ++u) {
            // one fused multiply-add per product: the FP64 pipe is the scarce unit
            const int slot = lp_insert_team(tm.mask, keys, tmask, key[u] >= 0, key[u]);
            if (slot >= 0) vals[slot] = fma_acc(at[u], bv[u], vals[slot]);
            else if (slot == -2) dev_fail(P.status, kDevTableFull, 17, g);
            if (lent[u] > TW) {   // the rest of a long B row: still one row, distinct keys
              for (int x = tm.lane + TW; x < lent[u]; x += TW) {
                const int kk = Bj[bst[u] + x];
                const VT bb = Bx[bst[u] + x];
                const int slot = lp_insert(keys, tmask, nullptr, -1, kk);
                if (slot >= 0) vals[slot] = fma_acc(at[u], bb, vals[slot]);
                else dev_fail(P.status, kDevTableFull, 17, g);
              }
            }
            __syncwarp(tm.mask);
          }
        }
      } else {
        // flat: the chunk's products spread over the lanes
        int ex = len;
#pragma unroll
        for (int d = 1; d < TW; d <<= 1) {
          const int y = __shfl_up_sync(tm.mask, ex, d, TW);
          if (tm.lane >= d) ex += y;
        }
        ex -= len;
        csc->pre[tm.lane] = ex;
        csc->bs[tm.lane] = bs;
        csc->av[tm.lane] = av;
        if (tm.lane == 0) csc->pre[TW] = tot;
        __syncwarp(tm.mask);
        int t = 0;
        for (int xb = 0; xb < tot; xb += TW) {
          const int x = xb + tm.lane;
          int key = -1 - tm.lane;   // inactive lanes: a distinct negative key
          VT v = VT(0);
          if (x < tot) {
            while (csc->pre[t + 1] <= x) ++t;
            const long long q = csc->bs[t] + (x - csc->pre[t]);
            key = Bj[q];
            v = csc->av[t] * Bx[q];
          }
          const unsigned grp = (__match_any_sync(tm.mask, key) >> lane_base) & ((TW == 32) ? 0xffffffffu : ((1u << TW) - 1u));
          const bool leader = (grp & lane_lt) == 0;
          if (__any_sync(tm.mask, __popc(grp) > 1)) {
            xchg[tm.lane] = v;
            __syncwarp(tm.mask);
            if (leader) {
              unsigned rest = grp & ~(1u << tm.lane);
              while (rest) {
                const int o = __ffs(rest) - 1;
                rest &= rest - 1u;
                v += xchg[o];
              }
            }
            __syncwarp(tm.mask);
          }
          if (x < tot && leader) {
            const int slot = lp_insert(keys, tmask, nullptr, -1, key);
            if (slot >= 0) vals[slot] += v;
            else dev_fail(P.status, kDevTableFull, 18, g);
          }
          __syncwarp(tm.mask);
        }
      }
    }
    // compaction of the occupied slots into (column << 32 | slot)
    int cnt = 0;
    unsigned kmn = 0xffffffffu, kmx = 0u;
    for (int xb = 0; xb < T; xb += TW) {
      const int x = xb + tm.lane;
      const int key = x < T ? keys[x] : kEmpty;
      const bool o = key != kEmpty;
      const unsigned bal = (__ballot_sync(tm.mask, o) >> lane_base) & ((TW == 32) ? 0xffffffffu : ((1u << TW) - 1u));
      const int pos = cnt + __popc(bal & lane_lt);
      if (o && pos < half) sortb[pos] = ((unsigned long long)(unsigned)key << 32) | (unsigned)x;
      if (o) {
        kmn = min(kmn, (unsigned)key);
        kmx = max(kmx, (unsigned)key);
      }
      cnt += __popc(bal);
    }
    if (tm.lane == 0 && cnt != s) dev_fail(P.status, kDevRowSizeMismatch, 19, g);
    const int n = cnt < half ? cnt : half;
    const long long nw = n < s ? n : s;
    if (TW == 32 && n > 2 * TW) {
      // Bucket sort by column (rows of many keys) into the value region, once
      // the values have moved to a compact array in the key region; keys
      // bunched unevenly take the bitonic sort instead.
      kmn = __reduce_min_sync(tm.mask, kmn);
      kmx = __reduce_max_sync(tm.mask, kmx);
      __syncwarp(tm.mask);
      VT* cv = reinterpret_cast<VT*>(keys);                                       // half values
      unsigned long long* outb = reinterpret_cast<unsigned long long*>(vals);     // half entries
      int* bcnt = sizeof(VT) == 8 ? reinterpret_cast<int*>(outb + half) : reinterpret_cast<int*>(cv + half);
      // values by compact position, into the key region (every key was read above)
      for (int x = tm.lane; x < n; x += TW) cv[x] = vals[(unsigned)(sortb[x] & 0xffffffffull)];
      __syncwarp(tm.mask);   // the value region is free from here on
      if (warp_bucket_sort(sortb, outb, bcnt, n, kmn, kmx)) {
        for (long long x = tm.lane; x < nw; x += TW) {
          const unsigned long long e = outb[x];
          Cj[c0 + x] = (int)(e >> 32);
          Cx[c0 + x] = cv[(unsigned)(e & 0xffffffffull)];
        }
        __syncwarp(tm.mask);
        continue;
      }
      // uneven keys: bitonic sort of (column, compact position)
      for (int x = tm.lane; x < n; x += TW) sortb[x] = (sortb[x] & 0xffffffff00000000ull) | (unsigned)x;
      int N = 1;
      while (N < n) N <<= 1;
      for (int x = n + tm.lane; x < N; x += TW) sortb[x] = ~0ull;
      __syncwarp(tm.mask);
      team_bitonic<TW>(tm, sortb, N);
      for (long long x = tm.lane; x < nw; x += TW) {
        const unsigned long long e = sortb[x];
        Cj[c0 + x] = (int)(e >> 32);
        Cx[c0 + x] = cv[(unsigned)(e & 0xffffffffull)];
      }
      __syncwarp(tm.mask);
      continue;
    }
    int N = 1;
    while (N < n) N <<= 1;
    for (int x = n + tm.lane; x < N; x += TW) sortb[x] = ~0ull;
    __syncwarp(tm.mask);
    team_bitonic<TW>(tm, sortb, N);
    for (long long x = tm.lane; x < nw; x += TW) {
      const unsigned long long e = sortb[x];
      Cj[c0 + x] = (int)(e >> 32);
      Cx[c0 + x] = vals[(unsigned)(e & 0xffffffffull)];
    }
    __syncwarp(tm.mask);
  }
}

// ---------------------------------------------------------------------------
// Compressed-position numeric (warp teams, products whose B was compressed).
// The compressed B of the symbolic phase (Section 3.2) fixes each row's
// sorted column list, so every product's output position can be computed
// instead of sorting the accumulator afterwards:
//   1. OR the column sets of the compressed B rows over A(i,:) into a table
//      keyed by column-set index (the symbolic insert, CF times fewer keys)
//   2. sort the column-set indices, give each the count of set bits before it
//      (its base) and write C(i,:)'s columns from the sets
//   3. each product goes to base(col >> 5) + popcount of the lower bits of
//      its set: one fused multiply-add into a row-local array (positions are
//      distinct within a pass, as in k_num_warp)
//   4. the row's values are written in order
// A table slot holds (column-set index, set bits, base) in 16 bytes, so the
// lookup of step 3 is one shared-memory load per probe.
// ---------------------------------------------------------------------------
template <int TW, typename VT>
__host__ __device__ size_t cpn_team_bytes(int T) {
  const int half = T / 2 > 0 ? T / 2 : 1;
  return al16((size_t)T * 16) + al16((size_t)half * 8) + al16(sizeof(ChunkScratch<TW, VT>)) +
         al16((size_t)TW * sizeof(VT));
}

// One row g of C by the team, in the team's shared memory at base_p
// (cpn_team_bytes<TW, VT>(2^logT) bytes).
template <int TW, typename VT>
__device__ __forceinline__ void cpn_row(const Team<TW>& tm, const ProbD& P, unsigned char* base_p, int logT,
                                        const LpHash& hs, long long g) {
  const int T = 1 << logT;
  const int half = T / 2 > 0 ? T / 2 : 1;
  int4* tab = reinterpret_cast<int4*>(base_p);
  // step 2 sorts (set << 32 | slot) and stages C's columns here; steps 3-4 accumulate here
  unsigned long long* sortb = reinterpret_cast<unsigned long long*>(base_p + al16((size_t)T * 16));
  int* colst = reinterpret_cast<int*>(sortb);
  VT* outv = reinterpret_cast<VT*>(sortb);
  ChunkScratch<TW, VT>* csc =
      reinterpret_cast<ChunkScratch<TW, VT>*>(base_p + al16((size_t)T * 16) + al16((size_t)half * 8));
  VT* xchg = reinterpret_cast<VT*>(reinterpret_cast<unsigned char*>(csc) + al16(sizeof(ChunkScratch<TW, VT>)));
  const unsigned lane_lt = (1u << tm.lane) - 1u;
  const int lane_base = (threadIdx.x & 31) & ~(TW - 1);
  const unsigned tbits = (TW == 32) ? 0xffffffffu : ((1u << TW) - 1u);

  {
    const int b = inst_of(P.arow0s, P.ninst, g);
    const InstD& I = P.inst[b];
    const long long i = g - I.arow0;
    const long long c0 = I.Crp[i];
    const int s = (int)(I.Crp[i + 1] - c0);
    for (int x = tm.lane; x < T; x += TW) tab[x] = make_int4(kEmpty, 0, 0, 0);
    __syncwarp(tm.mask);
    const long long a0 = rp_at(I.A, i), a1 = rp_at(I.A, i + 1);
    const VT* __restrict__ Ax = reinterpret_cast<const VT*>(I.A.vx);
    const VT* __restrict__ Bx = reinterpret_cast<const VT*>(I.B.vx);
    const int* __restrict__ Bj = I.B.cj;
    const int* __restrict__ Aj = I.A.cj;
    const long long brow0 = I.brow0;
    // the operands of one chunk of A(i,:): B row range, compressed B row range, a_ij
    long long bs = 0, cbs = 0;
    int len = 0, clen = 0;
    VT av = VT(0);
    auto load_chunk = [&](long long c) {
      const long long p = c + tm.lane;
      bs = 0;
      cbs = 0;
      len = 0;
      clen = 0;
      av = VT(0);
      if (p < a1) {
        const int j = Aj[p];
        av = Ax[p];
        bs = rp_at(I.B, j);
        len = (int)(rp_at(I.B, j + 1) - bs);
        cbs = P.Bcp[brow0 + j];
        clen = (int)(P.Bcp[brow0 + j + 1] - cbs);
      }
    };
    const bool one_chunk = a1 - a0 <= TW;
    int cnt = 0;
    const int sw = s < half ? s : half;
    const int stored = (TW == 32 && P.rcnt != nullptr) ? P.rcnt[g] : -1;
    int run = 0;
    if (stored >= 0) {
      // 1'-2'. the row's column sets as the symbolic phase recorded them, in
      // increasing set order (no union, no sort): lane t takes sets 2t and
      // 2t + 1, their bases are a scan of the set-bit counts
      const int2* src = P.rsets + g * kRowSetCap;
      const int x0 = 2 * tm.lane;
      int4 e = make_int4(kEmpty, 0, kEmpty, 0);
      if (x0 + 1 < stored) {
        e = *reinterpret_cast<const int4*>(src + x0);
      } else if (x0 < stored) {
        const int2 e0 = src[x0];
        e.x = e0.x;
        e.y = e0.y;
      }
      const int n0 = __popc((unsigned)e.y), n1 = __popc((unsigned)e.w);
      int incl = n0 + n1;
#pragma unroll
      for (int d = 1; d < TW; d <<= 1) {
        const int y = __shfl_up_sync(tm.mask, incl, d, TW);
        if (tm.lane >= d) incl += y;
      }
      run = __shfl_sync(tm.mask, incl, TW - 1, TW);
      const int b0 = incl - n0 - n1;
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int key = h ? e.z : e.x;
        if (key == kEmpty) continue;
        const unsigned mk = (unsigned)(h ? e.w : e.y);
        const int o0 = h ? b0 + n0 : b0;
        int fresh = 0;
        const int slot = slot_insert<4>(reinterpret_cast<int*>(tab), hs, key, &fresh);
        if (slot >= 0) {
          tab[slot].y = (int)mk;
          tab[slot].z = o0;
        } else {
          dev_fail(P.status, kDevTableFull, 29, g);
        }
        // C(i,:)'s columns staged in shared memory
        unsigned m = mk;
        int o = o0;
        while (m) {
          const int bit = __ffs(m) - 1;
          m &= m - 1u;
          if (o < sw) colst[o] = key * 32 + bit;
          ++o;
        }
      }
      if (one_chunk) load_chunk(a0);
    } else {
      // 1. union of the compressed B rows
      int* upre = reinterpret_cast<int*>(csc);
      long long* uqs =
          reinterpret_cast<long long*>(reinterpret_cast<unsigned char*>(csc) + al16((size_t)(TW + 1) * 4));
      for (long long c = a0; c < a1; c += TW) {
        load_chunk(c);
        union_chunk<TW, 4, true>(tm.mask, tm.lane, upre, uqs, cbs, clen, P.csi, P.cs, reinterpret_cast<int*>(tab),
                                 hs, P.status, 25, g);
      }
      // 2. sorted column sets, their bases, and C(i,:)'s columns
      for (int xb = 0; xb < T; xb += TW) {
        const int x = xb + tm.lane;
        const bool o = x < T && tab[x].x != kEmpty;
        const unsigned bal = (__ballot_sync(tm.mask, o) >> lane_base) & tbits;
        const int pos = cnt + __popc(bal & lane_lt);
        if (o && pos < half) sortb[pos] = ((unsigned long long)(unsigned)tab[x].x << 32) | (unsigned)x;
        cnt += __popc(bal);
      }
    }
    const int n = cnt < half ? cnt : half;
    __syncwarp(tm.mask);
    if (stored >= 0) {
      // (bases and columns above)
    } else if (n <= 2 * TW) {
      // up to two sets per lane: sorted in registers, slots found again by key
      unsigned v0 = tm.lane < n ? (unsigned)(sortb[tm.lane] >> 32) : 0xffffffffu;
      unsigned v1 = tm.lane + TW < n ? (unsigned)(sortb[tm.lane + TW] >> 32) : 0xffffffffu;
      if (n <= TW) v0 = team_sort1<TW>(tm.mask, tm.lane, v0);
      else team_sort2<TW>(tm.mask, tm.lane, v0, v1);
      int sl[2] = {-1, -1}, bs2[2] = {0, 0};
      unsigned mk[2] = {0u, 0u};
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const unsigned v = h ? v1 : v0;
        if (v != 0xffffffffu) {
          sl[h] = set_slot(tab, hs, (int)v);
          if (sl[h] >= 0) mk[h] = (unsigned)tab[sl[h]].y;
        }
        const int c = __popc(mk[h]);
        int incl = c;
#pragma unroll
        for (int d = 1; d < TW; d <<= 1) {
          const int y = __shfl_up_sync(tm.mask, incl, d, TW);
          if (tm.lane >= d) incl += y;
        }
        bs2[h] = run + incl - c;
        if (sl[h] >= 0) tab[sl[h]].z = bs2[h];
        run += __shfl_sync(tm.mask, incl, TW - 1, TW);
      }
      __syncwarp(tm.mask);
      // columns staged in shared memory (over the compaction list, now read)
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        unsigned m = mk[h];
        int o = bs2[h];
        const int key = (int)(h ? v1 : v0);
        while (m) {
          const int bit = __ffs(m) - 1;
          m &= m - 1u;
          if (o < sw) colst[o] = key * 32 + bit;
          ++o;
        }
      }
    } else {
      int N = 1;
      while (N < n) N <<= 1;
      for (int x = n + tm.lane; x < N; x += TW) sortb[x] = ~0ull;
      __syncwarp(tm.mask);
      team_bitonic<TW>(tm, sortb, N);
      for (int xb = 0; xb < n; xb += TW) {
        const int x = xb + tm.lane;
        int c = 0, slot = 0;
        if (x < n) {
          slot = (int)(sortb[x] & 0xffffffffull);
          c = __popc((unsigned)tab[slot].y);
        }
        int incl = c;
#pragma unroll
        for (int d = 1; d < TW; d <<= 1) {
          const int y = __shfl_up_sync(tm.mask, incl, d, TW);
          if (tm.lane >= d) incl += y;
        }
        if (x < n) tab[slot].z = run + incl - c;
        run += __shfl_sync(tm.mask, incl, TW - 1, TW);
      }
      __syncwarp(tm.mask);
      // columns staged in shared memory from the table
      for (int x = tm.lane; x < T; x += TW) {
        const int4 e = tab[x];
        if (e.x != kEmpty) {
          unsigned m = (unsigned)e.y;
          int o = e.z;
          while (m) {
            const int bit = __ffs(m) - 1;
            m &= m - 1u;
            if (o < sw) colst[o] = e.x * 32 + bit;
            ++o;
          }
        }
      }
    }
    if (tm.lane == 0 && run != s) dev_fail(P.status, kDevRowSizeMismatch, 26, g);
    __syncwarp(tm.mask);
    int* __restrict__ Cj = I.Cj;
    for (int x = tm.lane; x < sw; x += TW) Cj[c0 + x] = colst[x];
    __syncwarp(tm.mask);
    for (int x = tm.lane; x < half; x += TW) outv[x] = VT(0);
    __syncwarp(tm.mask);
    // 3. products to their positions
    auto pos_of = [&](int col) -> int {
      const int4 e = set_find(tab, hs, col >> 5);
      if (e.x == kEmpty) return -1;
      return e.z + __popc((unsigned)e.y & ((1u << (col & 31)) - 1u));
    };
    for (long long c = a0; c < a1; c += TW) {
      if (!one_chunk) load_chunk(c);
      const int nc = (a1 - c) < TW ? (int)(a1 - c) : TW;
      int tot = len;
#pragma unroll
      for (int d = TW / 2; d > 0; d >>= 1) tot += __shfl_xor_sync(tm.mask, tot, d, TW);
      if (2 * tot >= nc * TW) {
        // sequential: one B row per pass, distinct positions inside a pass;
        // the loads of two passes are issued together (four measured slower:
        // register spills of the 256 x 4 launch bound)
        // the chunk's (B row start, length, a_ij) go to shared memory once;
        // each pass reads its entry's with broadcast loads
        constexpr int kU = 2;
        csc->bs[tm.lane] = bs;
        csc->pre[tm.lane] = len;
        csc->av[tm.lane] = av;
        __syncwarp(tm.mask);
        for (int t0 = 0; t0 < nc; t0 += kU) {
          int q[kU], lent[kU];
          long long bst[kU];
          VT at[kU], bv[kU];
#pragma unroll
          for (int u = 0; u < kU; ++u) {
            const int t = (t0 + u < nc) ? t0 + u : nc - 1;
            bst[u] = csc->bs[t];
            const int l = (int)csc->pre[t];
            at[u] = csc->av[t];
            lent[u] = (t0 + u < nc) ? l : 0;
            q[u] = -1;
            bv[u] = VT(0);
            if (tm.lane < lent[u]) {
              q[u] = Bj[bst[u] + tm.lane];
              bv[u] = Bx[bst[u] + tm.lane];
            }
          }
#pragma unroll
          for (int u = 0; u < kU; ++u) {
            if (q[u] >= 0) {
              const int o = pos_of(q[u]);
              if (o >= 0 && o < half) outv[o] = fma_acc(at[u], bv[u], outv[o]);
              else dev_fail(P.status, kDevTableFull, 27, g);
            }
            for (int x = tm.lane + TW; x < lent[u]; x += TW) {
              const int o = pos_of(Bj[bst[u] + x]);
              if (o >= 0 && o < half) outv[o] = fma_acc(at[u], Bx[bst[u] + x], outv[o]);
              else dev_fail(P.status, kDevTableFull, 27, g);
            }
            __syncwarp(tm.mask);
          }
        }
      } else {
        // flat: the chunk's products over the lanes, equal positions pre-summed
        int ex = len;
#pragma unroll
        for (int d = 1; d < TW; d <<= 1) {
          const int y = __shfl_up_sync(tm.mask, ex, d, TW);
          if (tm.lane >= d) ex += y;
        }
        ex -= len;
        csc->pre[tm.lane] = ex;
        csc->bs[tm.lane] = bs;
        csc->av[tm.lane] = av;
        if (tm.lane == 0) csc->pre[TW] = tot;
        __syncwarp(tm.mask);
        int t = 0;
        for (int xb = 0; xb < tot; xb += TW) {
          const int x = xb + tm.lane;
          int o = -1 - tm.lane;
          VT v = VT(0);
          if (x < tot) {
            while (csc->pre[t + 1] <= x) ++t;
            const long long qq = csc->bs[t] + (x - csc->pre[t]);
            o = pos_of(Bj[qq]);
            v = csc->av[t] * Bx[qq];
            if (o < 0 || o >= half) {
              dev_fail(P.status, kDevTableFull, 28, g);
              o = -1 - tm.lane;
            }
          }
          const unsigned grp = (__match_any_sync(tm.mask, o) >> lane_base) & tbits;
          const bool leader = (grp & lane_lt) == 0;
          if (__any_sync(tm.mask, __popc(grp) > 1)) {
            xchg[tm.lane] = v;
            __syncwarp(tm.mask);
            if (leader) {
              unsigned rest = grp & ~(1u << tm.lane);
              while (rest) {
                const int oo = __ffs(rest) - 1;
                rest &= rest - 1u;
                v += xchg[oo];
              }
            }
            __syncwarp(tm.mask);
          }
          if (o >= 0 && leader) outv[o] += v;
          __syncwarp(tm.mask);
        }
        __syncwarp(tm.mask);
      }
    }
    // 4. values in order
    VT* __restrict__ Cx = reinterpret_cast<VT*>(I.Cx);
    for (int x = tm.lane; x < sw; x += TW) Cx[c0 + x] = outv[x];
    __syncwarp(tm.mask);
  }
}

template <int TW, typename VT>
__global__ void __launch_bounds__(256, 4) k_num_cpn(ProbD P, const int* __restrict__ rows, long long nrows, int logT) {
  extern __shared__ __align__(16) unsigned char smem[];
  Team<TW> tm;
  const LpHash hs(logT, P.hash_mode);
  unsigned char* base_p = smem + (size_t)tm.id * cpn_team_bytes<TW, VT>(1 << logT);
  const long long team = (long long)blockIdx.x * tm.per_cta + tm.id;
  const long long nteams = (long long)gridDim.x * tm.per_cta;
  for (long long r = team; r < nrows; r += nteams) cpn_row<TW, VT>(tm, P, base_p, logT, hs, rows[r]);
}

// ---------------------------------------------------------------------------
// Bitmap-window positions (warp teams, compressed products, B rows sorted).
// The column sets of C(i,:) lie between the first set of the first and the
// last set of the last column among the compressed B rows over A(i,:) (each
// compressed row is sorted, so its first and last entries bound it).  When
// that window is at most kWbLimit sets wide, the row's union of column sets is
// a bitmap over the window addressed directly by set index: the dense
// accumulator of Section 3.1.2 restricted to the row's own column range, in
// the 32-column sets of Section 3.2.
//   1. OR every compressed product's set bits into bits[set - smin]
//   2. per set word, the count of set bits before it in the window (its base):
//      lanes take contiguous runs of words, a warp scan joins them
//   3. each product goes to base + the set bits below its column: one fused
//      multiply-add into the row's value array; its column is staged at the
//      same place (every column of C(i,:) receives at least one product)
//   4. the row's columns and values are written in order; the window's words
//      are cleared for the next row
// No hashing, no probing, no sort of the sets.  Rows with a wider window take
// the hash path of k_num_cpn (cpn_row) in the same shared memory.
// ---------------------------------------------------------------------------
constexpr int kWbLimit = 1344;   // widest window in column sets (43 008 columns)
constexpr int kWbWords = 1408;   // bitmap words per team: the scan's per-lane runs round a window up to this
constexpr int kWbTeams = 4;      // warp teams per CTA

template <typename VT>
__host__ __device__ size_t wb_team_bytes(int T) {
  const int half = T / 2 > 0 ? T / 2 : 1;
  const size_t wb = al16((size_t)kWbWords * 4) + al16((size_t)kWbWords * 2) + al16((size_t)half * 4) +
                    al16((size_t)half * sizeof(VT)) + al16(sizeof(ChunkScratch<32, VT>)) + al16(32 * sizeof(VT));
  const size_t hp = cpn_team_bytes<32, VT>(T);
  return wb > hp ? wb : hp;
}

// Words per lane of the base scan over a window of span words: a multiple of
// 4 (16-byte loads) that is not a multiple of 8, so the eight lanes of each
// 16-byte load phase hit distinct banks.  32 * the result <= kWbWords for
// span <= kWbLimit.
__device__ __forceinline__ int wb_words_per_lane(unsigned span) {
  int pw = ((int)((span + 31u) >> 5) + 3) & ~3;
  if ((pw & 7) == 0) pw += 4;
  return pw;
}

template <typename VT>
__global__ void __launch_bounds__(32 * kWbTeams, 5) k_num_wb(ProbD P, const int* __restrict__ rows, long long nrows,
                                                             int logT) {
  extern __shared__ __align__(16) unsigned char smem[];
  Team<32> tm;
  const int T = 1 << logT;
  const int half = T / 2 > 0 ? T / 2 : 1;
  const LpHash hs(logT, P.hash_mode);
  unsigned char* base_p = smem + (size_t)tm.id * wb_team_bytes<VT>(T);
  unsigned* bits = reinterpret_cast<unsigned*>(base_p);
  unsigned short* wbase = reinterpret_cast<unsigned short*>(base_p + al16((size_t)kWbWords * 4));
  int* colst = reinterpret_cast<int*>(base_p + al16((size_t)kWbWords * 4) + al16((size_t)kWbWords * 2));
  VT* outv = reinterpret_cast<VT*>(reinterpret_cast<unsigned char*>(colst) + al16((size_t)half * 4));
  ChunkScratch<32, VT>* csc = reinterpret_cast<ChunkScratch<32, VT>*>(reinterpret_cast<unsigned char*>(outv) +
                                                                      al16((size_t)half * sizeof(VT)));
  VT* xchg = reinterpret_cast<VT*>(reinterpret_cast<unsigned char*>(csc) + al16(sizeof(ChunkScratch<32, VT>)));
  int* upre = reinterpret_cast<int*>(csc);
  long long* uqs = reinterpret_cast<long long*>(reinterpret_cast<unsigned char*>(csc) + al16((size_t)33 * 4));
  const int lane = tm.lane;
  const unsigned lane_lt = (1u << lane) - 1u;
  const unsigned full = 0xffffffffu;
  bool clean = false;   // every word of bits[] is zero

  const long long team = (long long)blockIdx.x * tm.per_cta + tm.id;
  const long long nteams = (long long)gridDim.x * tm.per_cta;
  // The next row's head (id, instance, row range of A, first chunk of A's
  // columns and values) is loaded while the current row runs.
  long long g_n = -1, a0_n = 0, a1_n = 0;
  int b_n = 0, j_n = 0;
  VT av_n = VT(0);
  auto fetch_head = [&](long long rr) {
    g_n = -1;
    if (rr < nrows) {
      g_n = rows[rr];
      b_n = inst_of(P.arow0s, P.ninst, g_n);
      const InstD& In = P.inst[b_n];
      a0_n = rp_at(In.A, g_n - In.arow0);
      a1_n = rp_at(In.A, g_n - In.arow0 + 1);
    }
  };
  auto fetch_first = [&]() {
    if (g_n >= 0 && a0_n + lane < a1_n) {
      const InstD& In = P.inst[b_n];
      j_n = In.A.cj[a0_n + lane];
      av_n = reinterpret_cast<const VT*>(In.A.vx)[a0_n + lane];
    }
  };
  fetch_head(team);
  fetch_first();
  for (long long r = team; r < nrows; r += nteams) {
    const long long g = g_n;
    const int b = b_n;
    const InstD& I = P.inst[b];
    const long long i = g - I.arow0;
    const long long a0 = a0_n, a1 = a1_n;
    const int j0 = j_n;
    const VT av0 = av_n;
    fetch_head(r + nteams);
    const VT* __restrict__ Ax = reinterpret_cast<const VT*>(I.A.vx);
    const VT* __restrict__ Bx = reinterpret_cast<const VT*>(I.B.vx);
    const int* __restrict__ Bj = I.B.cj;
    const int* __restrict__ Aj = I.A.cj;
    const long long brow0 = I.brow0;
    long long bs = 0, cbs = 0;
    int len = 0, clen = 0;
    VT av = VT(0);
    auto load_chunk = [&](long long c) {
      const long long p = c + lane;
      bs = 0;
      cbs = 0;
      len = 0;
      clen = 0;
      av = VT(0);
      if (p < a1) {
        const int j = c == a0 ? j0 : Aj[p];
        av = c == a0 ? av0 : Ax[p];
        bs = rp_at(I.B, j);
        len = (int)(rp_at(I.B, j + 1) - bs);
        cbs = P.Bcp[brow0 + j];
        clen = (int)(P.Bcp[brow0 + j + 1] - cbs);
      }
    };
    // 0. the window
    unsigned smin = 0xffffffffu, smax = 0u;
    for (long long c = a0; c < a1; c += 32) {
      load_chunk(c);
      if (clen > 0) {
        smin = min(smin, (unsigned)P.csi[cbs]);
        smax = max(smax, (unsigned)P.csi[cbs + clen - 1]);
      }
    }
    smin = __reduce_min_sync(full, smin);
    smax = __reduce_max_sync(full, smax);
    if (smin > smax || smax - smin >= (unsigned)kWbLimit) {
      cpn_row<32, VT>(tm, P, base_p, logT, hs, g);
      clean = false;
      fetch_first();
      __syncwarp();
      continue;
    }
    const unsigned span = smax - smin + 1u;
    const int pw = wb_words_per_lane(span);
    if (!clean) {
      uint4* c4 = reinterpret_cast<uint4*>(bits);
      for (int x = lane; x < kWbWords / 4; x += 32) c4[x] = make_uint4(0u, 0u, 0u, 0u);
      clean = true;
      __syncwarp();
    }
    const long long c0 = I.Crp[i];
    const int s = (int)(I.Crp[i + 1] - c0);
    const bool one_chunk = a1 - a0 <= 32;
    // 1. union of the compressed B rows
    for (long long c = a0; c < a1; c += 32) {
      if (!one_chunk) load_chunk(c);
      wb_union_chunk<32, false>(full, lane, upre, uqs, cbs, clen, P.csi, P.cs, bits, smin, span, P.status, 36, g);
    }
    fetch_first();
    if (!one_chunk) load_chunk(a0);
    // 2. bases of the set words
    const uint4* b4 = reinterpret_cast<const uint4*>(bits + lane * pw);
    int cnt = 0;
    unsigned nz = 0u;   // this lane's 16-byte groups that hold set bits (pw / 4 <= 11)
    for (int k = 0; k < pw / 4; ++k) {
      const uint4 v = b4[k];
      cnt += __popc(v.x) + __popc(v.y) + __popc(v.z) + __popc(v.w);
      if ((v.x | v.y | v.z | v.w) != 0u) nz |= 1u << k;
    }
    int incl = cnt;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const int y = __shfl_up_sync(full, incl, d);
      if (lane >= d) incl += y;
    }
    const int total = __shfl_sync(full, incl, 31);
    int run = incl - cnt;
    unsigned short* wb = wbase + lane * pw;
    for (unsigned m = nz; m != 0u; m &= m - 1u) {
      const int k = __ffs(m) - 1;
      const uint4 v = b4[k];
      if (v.x) wb[4 * k] = (unsigned short)run;
      run += __popc(v.x);
      if (v.y) wb[4 * k + 1] = (unsigned short)run;
      run += __popc(v.y);
      if (v.z) wb[4 * k + 2] = (unsigned short)run;
      run += __popc(v.z);
      if (v.w) wb[4 * k + 3] = (unsigned short)run;
      run += __popc(v.w);
    }
    if (lane == 0 && total != s) dev_fail(P.status, kDevRowSizeMismatch, 37, g);
    const int sw = s < half ? s : half;
    for (int x = lane; x < sw; x += 32) outv[x] = VT(0);
    __syncwarp();
    // 3. products to their places
    auto pos_of = [&](int col) -> int {
      const unsigned w = (unsigned)(col >> 5) - smin;
      if (w >= span) return -1;
      const unsigned m = bits[w];
      const unsigned bit = 1u << (col & 31);
      if (!(m & bit)) return -1;
      const int o = (int)wbase[w] + __popc(m & (bit - 1u));
      return o < sw ? o : -1;
    };
    for (long long c = a0; c < a1; c += 32) {
      if (!one_chunk && c != a0) load_chunk(c);
      const int nc = (a1 - c) < 32 ? (int)(a1 - c) : 32;
      const int tot = __reduce_add_sync(full, (unsigned)len);
      if (2 * tot >= nc * 32) {
        // sequential: one B row per pass, distinct places inside a pass
        constexpr int kU = 4;
        for (int t0 = 0; t0 < nc; t0 += kU) {
          int q[kU], lent[kU];
          long long bst[kU];
          VT at[kU], bv[kU];
#pragma unroll
          for (int u = 0; u < kU; ++u) {
            const int t = (t0 + u < nc) ? t0 + u : nc - 1;
            bst[u] = __shfl_sync(full, bs, t);
            const int l = __shfl_sync(full, len, t);
            at[u] = __shfl_sync(full, av, t);
            lent[u] = (t0 + u < nc) ? l : 0;
            q[u] = -1;
            bv[u] = VT(0);
            if (lane < lent[u]) {
              q[u] = Bj[bst[u] + lane];
              bv[u] = Bx[bst[u] + lane];
            }
          }
#pragma unroll
          for (int u = 0; u < kU; ++u) {
            if (q[u] >= 0) {
              const int o = pos_of(q[u]);
              if (o >= 0) {
                outv[o] = fma_acc(at[u], bv[u], outv[o]);
                colst[o] = q[u];
              } else {
                dev_fail(P.status, kDevTableFull, 38, g);
              }
            }
            for (int x = lane + 32; x < lent[u]; x += 32) {
              const int col = Bj[bst[u] + x];
              const int o = pos_of(col);
              if (o >= 0) {
                outv[o] = fma_acc(at[u], Bx[bst[u] + x], outv[o]);
                colst[o] = col;
              } else {
                dev_fail(P.status, kDevTableFull, 38, g);
              }
            }
            __syncwarp();
          }
        }
      } else {
        // flat: the chunk's products over the lanes, equal places pre-summed
        int ex = len;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
          const int y = __shfl_up_sync(full, ex, d);
          if (lane >= d) ex += y;
        }
        ex -= len;
        csc->pre[lane] = ex;
        csc->bs[lane] = bs;
        csc->av[lane] = av;
        if (lane == 0) csc->pre[32] = tot;
        __syncwarp();
        int t = 0;
        for (int xb = 0; xb < tot; xb += 32) {
          const int x = xb + lane;
          int o = -1 - lane;
          VT v = VT(0);
          if (x < tot) {
            while (csc->pre[t + 1] <= x) ++t;
            const long long qq = csc->bs[t] + (x - csc->pre[t]);
            const int col = Bj[qq];
            const int oo = pos_of(col);
            if (oo >= 0) {
              o = oo;
              v = csc->av[t] * Bx[qq];
              colst[oo] = col;
            } else {
              dev_fail(P.status, kDevTableFull, 39, g);
            }
          }
          const unsigned grp = __match_any_sync(full, o);
          const bool leader = (grp & lane_lt) == 0;
          if (__any_sync(full, __popc(grp) > 1)) {
            xchg[lane] = v;
            __syncwarp();
            if (leader) {
              unsigned rest = grp & ~(1u << lane);
              while (rest) {
                const int oo = __ffs(rest) - 1;
                rest &= rest - 1u;
                v += xchg[oo];
              }
            }
            __syncwarp();
          }
          if (o >= 0 && leader) outv[o] += v;
          __syncwarp();
        }
        __syncwarp();
      }
    }
    __syncwarp();
    // 4. the row in order; the window cleared
    int* __restrict__ Cj = I.Cj;
    VT* __restrict__ Cx = reinterpret_cast<VT*>(I.Cx);
    for (int x = lane; x < sw; x += 32) {
      Cj[c0 + x] = colst[x];
      Cx[c0 + x] = outv[x];
    }
    // the window's words: each lane clears its own groups that hold bits
    uint4* c4 = reinterpret_cast<uint4*>(bits + lane * pw);
    for (unsigned m = nz; m != 0u; m &= m - 1u) c4[__ffs(m) - 1] = make_uint4(0u, 0u, 0u, 0u);
    __syncwarp();
  }
}

// One thread per row for rows of C with at most kT1MaxKeys columns and few
// products (Thread-Sequential with a team of one, Section 3.1.1): the keys
// stay in registers, a product is matched with integer compares and goes to
// one accumulator in the thread's column of shared memory (one FP64
// instruction per product), and the row is written in column order from the
// ranks of its keys.
template <typename VT>
__global__ void __launch_bounds__(256, 3) k_num_thread(ProbD P, const int* __restrict__ rows, long long nrows) {
  __shared__ VT accs[kT1MaxKeys][256];
  const int tid = threadIdx.x;
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long r = (long long)blockIdx.x * blockDim.x + tid; r < nrows; r += stride) {
    const long long g = rows[r];
    const int b = inst_of(P.arow0s, P.ninst, g);
    const InstD& I = P.inst[b];
    const long long i = g - I.arow0;
    const long long c0 = I.Crp[i];
    const int s = (int)(I.Crp[i + 1] - c0);
    const long long a0 = rp_at(I.A, i), a1 = rp_at(I.A, i + 1);
    const VT* __restrict__ Ax = reinterpret_cast<const VT*>(I.A.vx);
    const VT* __restrict__ Bx = reinterpret_cast<const VT*>(I.B.vx);
    const int* __restrict__ Bj = I.B.cj;
    int key[kT1MaxKeys];
#pragma unroll
    for (int t = 0; t < kT1MaxKeys; ++t) {
      key[t] = -1;
      accs[t][tid] = VT(0);
    }
    int n = 0;
    bool over = false;
    auto add = [&](int c, VT a, VT y) {
      int hit = -1;
#pragma unroll
      for (int t = 0; t < kT1MaxKeys; ++t) hit = (key[t] == c) ? t : hit;
      if (hit < 0) {
        if (n < kT1MaxKeys) {
#pragma unroll
          for (int t = 0; t < kT1MaxKeys; ++t) key[t] = (t == n) ? c : key[t];
          hit = n++;
        } else {
          over = true;
        }
      }
      if (hit >= 0) accs[hit][tid] = fma_acc(a, y, accs[hit][tid]);
    };
    constexpr int kX = 4, kQ = 4;
    for (long long c = a0; c < a1; c += kX) {
      long long qs[kX], qe[kX];
      VT a[kX];
#pragma unroll
      for (int u = 0; u < kX; ++u) {
        const bool ok = c + u < a1;
        const int j = ok ? I.A.cj[c + u] : -1;
        a[u] = ok ? Ax[c + u] : VT(0);
        qs[u] = j >= 0 ? rp_at(I.B, j) : 0;
        qe[u] = j >= 0 ? rp_at(I.B, j + 1) : 0;
      }
#pragma unroll
      for (int u = 0; u < kX; ++u) {
        for (long long q = qs[u]; q < qe[u]; q += kQ) {
          int cc[kQ];
          VT y[kQ];
#pragma unroll
          for (int v = 0; v < kQ; ++v) {
            const bool ok = q + v < qe[u];
            cc[v] = ok ? Bj[q + v] : -1;
            y[v] = ok ? Bx[q + v] : VT(0);
          }
#pragma unroll
          for (int v = 0; v < kQ; ++v)
            if (cc[v] >= 0) add(cc[v], a[u], y[v]);
        }
      }
    }
    if (over || n != s) dev_fail(P.status, over ? kDevTableFull : kDevRowSizeMismatch, 29, g);
    int* __restrict__ Cj = I.Cj;
    VT* __restrict__ Cx = reinterpret_cast<VT*>(I.Cx);
#pragma unroll
    for (int t = 0; t < kT1MaxKeys; ++t) {
      if (t < n) {
        int rk = 0;
#pragma unroll
        for (int t2 = 0; t2 < kT1MaxKeys; ++t2) rk += (t2 < n && key[t2] < key[t]) ? 1 : 0;
        if (rk < s) {
          Cj[c0 + rk] = key[t];
          Cx[c0 + rk] = accs[t][tid];
        }
      }
    }
  }
}

// Dense accumulator (Section 3.1.2) for rows whose column count is a large
// fraction of k or too large for a shared table, kept in shared memory: the
// column range is cut into windows of W = 2^win_log2 columns and the row is
// accumulated window by window (products outside the window are skipped), so
// every add is a shared-memory atomic and a window's columns come out in
// order from its bitmap.  Values of emitted columns are cleared as they are
// read, so each window starts from zero without a sweep.  When every B row
// has increasing columns (sorted_b), the part of a B row inside the window is
// found by binary search, so each product is visited in one window only.
__device__ __forceinline__ long long lower_col(const int* __restrict__ cj, long long lo, long long hi, long long c) {
  while (lo < hi) {
    const long long mid = (lo + hi) >> 1;
    if ((long long)cj[mid] < c) lo = mid + 1;
    else hi = mid;
  }
  return lo;
}

// Staged products (option stage_b): blocks of kStageE * TW products, two
// blocks in flight.
constexpr int kStageE = 2;

template <int TW, typename VT, bool STAGE>
__host__ __device__ size_t dense_win_bytes(int win_log2) {
  const size_t W = (size_t)1 << win_log2;
  const size_t base = al16(W * sizeof(VT)) + al16((W / 32) * 4) + al16(sizeof(ChunkScratch<TW, VT>));
  if (STAGE) {
    const size_t S = (size_t)kStageE * TW;
    return base + 2 * al16(S * 4) + 2 * al16(S * 4) + 2 * al16(S * sizeof(VT));
  }
  return base + al16((size_t)kStagedPasses * TW * 4);
}

__device__ __forceinline__ void cp_async_4(void* dst, const void* src) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  const size_t g = __cvta_generic_to_global(src);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(d), "l"(g) : "memory");
}
__device__ __forceinline__ void cp_async_8(void* dst, const void* src) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  const size_t g = __cvta_generic_to_global(src);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(d), "l"(g) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

// The products of one chunk of A entries (thread t: B range [bs, be), value
// av) with their B entries staged in shared memory: blocks of S = kStageE *
// TW products, each product's A entry found through a segment map (a forward
// max-fill of where each range starts), its column and value copied by
// cp.async into the block's buffer while the previous block is added.  The
// copies of block b + 1 are issued before block b is consumed, so a block's
// loads are in flight during the previous block's atomics instead of one
// dependent global load per product.  body(col, bval, t).  Returns the
// chunk's product count.
template <int TW, typename VT, class Body>
__device__ __forceinline__ long long staged_products(const Team<TW>& tm, ChunkScratch<TW, VT>* cs,
                                                     long long* scan_scratch, long long bs, long long be, VT av,
                                                     const int* __restrict__ Bj, const VT* __restrict__ Bx,
                                                     int* seg2, int* sj2, VT* sx2, Body body) {
  constexpr int E = kStageE;
  constexpr long long S = (long long)kStageE * TW;
  long long total;
  const long long ex = team_excl_scan<TW>(tm, be - bs, &total, scan_scratch);
  cs->pre[tm.lane] = ex;
  cs->bs[tm.lane] = bs;
  cs->av[tm.lane] = av;
  if (tm.lane == 0) cs->pre[TW] = total;
  tm.sync();
  const long long nblk = (total + S - 1) / S;
  int carry = -1;
  // segment map of block b into seg2 + (b & 1) * S
  auto build = [&](long long b) {
    int* sg = seg2 + (b & 1) * S;
    const long long x0 = b * S;
#pragma unroll
    for (int e = 0; e < E; ++e) sg[tm.lane * E + e] = -1;
    tm.sync();
    if (be > bs && ex >= x0 && ex < x0 + S) sg[ex - x0] = tm.lane;
    tm.sync();
    int v[E];
    int m = -1;
#pragma unroll
    for (int e = 0; e < E; ++e) {
      v[e] = sg[tm.lane * E + e];
      m = max(m, v[e]);
    }
    int run = max(carry, team_excl_max<TW>(tm, m, scan_scratch));
#pragma unroll
    for (int e = 0; e < E; ++e) {
      run = max(run, v[e]);
      sg[tm.lane * E + e] = run;
    }
    tm.sync();
    carry = sg[S - 1];
  };
  // asynchronous copies of block b's B entries
  auto issue = [&](long long b) {
    const int* sg = seg2 + (b & 1) * S;
    int* dj = sj2 + (b & 1) * S;
    VT* dx = sx2 + (b & 1) * S;
#pragma unroll
    for (int u = 0; u < E; ++u) {
      const long long k = (long long)u * TW + tm.lane;
      const long long xu = b * S + k;
      if (xu < total) {
        const int t = sg[k];
        const long long q = cs->bs[t] + (xu - cs->pre[t]);
        cp_async_4(dj + k, Bj + q);
        if (sizeof(VT) == 8) cp_async_8(dx + k, Bx + q);
        else cp_async_4(dx + k, Bx + q);
      }
    }
    cp_async_commit();
  };
  if (nblk > 0) {
    build(0);
    issue(0);
  }
  for (long long b = 0; b < nblk; ++b) {
    if (b + 1 < nblk) {
      build(b + 1);
      issue(b + 1);
      cp_async_wait<1>();
    } else {
      cp_async_wait<0>();
    }
    tm.sync();   // every thread's copies of block b have landed
    const int* sg = seg2 + (b & 1) * S;
    const int* dj = sj2 + (b & 1) * S;
    const VT* dx = sx2 + (b & 1) * S;
#pragma unroll
    for (int u = 0; u < E; ++u) {
      const long long k = (long long)u * TW + tm.lane;
      if (b * S + k < total) body(dj[k], dx[k], sg[k]);
    }
    tm.sync();   // block b's buffers are free for block b + 2
  }
  return total;
}

template <int TW, typename VT>
__host__ __device__ size_t dense_win_bytes(int win_log2) {
  return dense_win_bytes<TW, VT, false>(win_log2);
}

template <int TW, typename VT, bool STAGE>
__global__ void __launch_bounds__(TW) k_num_dense(ProbD P, const int* __restrict__ rows, long long nrows,
                                                  int win_log2, int sorted_b, unsigned long long* fetch) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ long long scan_scratch[33];
  __shared__ long long fetch_s;
  Team<TW> tm;
  const long long W = 1ll << win_log2;
  const long long ww = W / 32;
  VT* acc = reinterpret_cast<VT*>(smem);
  unsigned* bm = reinterpret_cast<unsigned*>(smem + al16((size_t)W * sizeof(VT)));
  ChunkScratch<TW, VT>* csc =
      reinterpret_cast<ChunkScratch<TW, VT>*>(smem + al16((size_t)W * sizeof(VT)) + al16((size_t)ww * 4));
  // products find their A entry through a segment map (a window holds many
  // short or empty B ranges, where a search per product takes many steps)
  int* seg = reinterpret_cast<int*>(reinterpret_cast<unsigned char*>(csc) + al16(sizeof(ChunkScratch<TW, VT>)));
  // staged variant: two segment maps, two blocks of columns and of values
  constexpr size_t kS = (size_t)kStageE * TW;
  int* sj2 = seg + 2 * kS;
  VT* sx2 = reinterpret_cast<VT*>(sj2 + 2 * kS);
  for (long long x = tm.lane; x < W; x += TW) acc[x] = VT(0);
  for (long long x = tm.lane; x < ww; x += TW) bm[x] = 0u;
  for (long long r = cta_next_row(fetch, &fetch_s); r < nrows; r = cta_next_row(fetch, &fetch_s)) {
    const long long g = rows[r];
    const int b = inst_of(P.arow0s, P.ninst, g);
    const InstD& I = P.inst[b];
    const long long i = g - I.arow0;
    const long long c0 = I.Crp[i];
    const long long s = I.Crp[i + 1] - c0;
    const long long k = I.k;
    const long long a0 = rp_at(I.A, i), a1 = rp_at(I.A, i + 1);
    const VT* __restrict__ Ax = reinterpret_cast<const VT*>(I.A.vx);
    const VT* __restrict__ Bx = reinterpret_cast<const VT*>(I.B.vx);
    const int* __restrict__ Bj = I.B.cj;
    VT* __restrict__ Cx = reinterpret_cast<VT*>(I.Cx);
    int* __restrict__ Cj = I.Cj;
    auto aval = [&](long long p) { return Ax[p]; };
    auto pf = [&](long long q) {
      prefetch_l1(Bj + q);
      prefetch_l1(Bx + q);
    };
    long long run = 0;
    // rows of one chunk on sorted B rows keep each A entry's cursor across
    // windows: one binary search per window, and empty windows are skipped
    const bool one_chunk = sorted_b && a1 - a0 <= TW;
    long long cur = 0, end = 0;
    VT av1 = VT(0);
    if (one_chunk && a0 + tm.lane < a1) {
      const int j = I.A.cj[a0 + tm.lane];
      cur = rp_at(I.B, j);
      end = rp_at(I.B, j + 1);
      av1 = Ax[a0 + tm.lane];
    }
    for (long long w0 = 0; w0 < k; w0 += W) {
      auto range = [&](int j, long long* bs, long long* be) {
        *bs = rp_at(I.B, j);
        *be = rp_at(I.B, j + 1);
        if (sorted_b && *be > *bs) {
          *bs = lower_col(Bj, *bs, *be, w0);
          *be = lower_col(Bj, *bs, *be, w0 + W);
        }
      };
      auto body = [&](long long q, int t) {
        const int col = Bj[q];
        if ((unsigned long long)(unsigned)col >= (unsigned long long)k) {
          if (w0 == 0) dev_fail(P.status, kDevBadIndex, 12, g);
          return;
        }
        const long long x = (long long)col - w0;
        if ((unsigned long long)x < (unsigned long long)W) {
          atomicAdd(acc + x, csc->av[t] * Bx[q]);
          atomicOr(bm + (x >> 5), 1u << (x & 31));
        }
      };
      if (one_chunk) {
        long long ub = cur;
        if (cur < end && (long long)Bj[cur] < w0 + W) ub = lower_col(Bj, cur, end, w0 + W);
        long long tot;
        if (STAGE) {
          auto sbody = [&](int col, VT bv, int t) {
            const long long x = (long long)col - w0;
            if ((unsigned long long)x < (unsigned long long)W) {
              atomicAdd(acc + x, csc->av[t] * bv);
              atomicOr(bm + (x >> 5), 1u << (x & 31));
            } else if ((unsigned long long)(unsigned)col >= (unsigned long long)k) {
              dev_fail(P.status, kDevBadIndex, 14, g);
            }
          };
          tot = staged_products<TW, VT>(tm, csc, scan_scratch, cur, ub, av1, Bj, Bx, seg, sj2, sx2, sbody);
        } else {
          tot = for_each_product_chunk<TW, VT>(tm, csc, scan_scratch, cur, ub, av1, body, pf, seg);
        }
        cur = ub;
        __syncthreads();
        if (tot == 0) continue;
      } else {
        for_each_product<TW, VT>(tm, csc, scan_scratch, I.A.cj, a0, a1, range, aval, body, pf, seg);
        __syncthreads();
      }
      // the window's columns in order: a prefix of the words' set-bit counts
      // over the CTA, then each warp emits its 32 words one word at a time,
      // lane l taking bit l, so the reads of the accumulator are consecutive
      // and the writes of C(i,:) coalesced
      const long long nw = ((k - w0 + 31) >> 5) < ww ? ((k - w0 + 31) >> 5) : ww;
      const unsigned lt = (1u << (threadIdx.x & 31)) - 1u;
      for (long long wb = 0; wb < nw; wb += TW) {
        const long long wi = wb + tm.lane;
        const unsigned word = (wi < nw) ? bm[wi] : 0u;
        long long tot;
        const long long pos = run + team_excl_scan<TW>(tm, __popc(word), &tot, scan_scratch);
        const long long wfirst = wi - (threadIdx.x & 31);   // first word of this warp
#pragma unroll 4
        for (int q = 0; q < 32; ++q) {
          const unsigned wd = __shfl_sync(0xffffffffu, word, q);
          if (wd == 0u) continue;
          const long long base = __shfl_sync(0xffffffffu, pos, q);
          if ((wd >> (threadIdx.x & 31)) & 1u) {
            const long long at = base + __popc(wd & lt);
            const long long x = (wfirst + q) * 32 + (threadIdx.x & 31);
            const VT v = acc[x];
            acc[x] = VT(0);
            if (at < s) {
              Cj[c0 + at] = (int)(w0 + x);
              Cx[c0 + at] = v;
            }
          }
        }
        if (wi < nw) bm[wi] = 0u;
        run += tot;
      }
      __syncthreads();
    }
    if (tm.lane == 0 && run != s) dev_fail(P.status, kDevRowSizeMismatch, 13, g);
  }
}

template <int TW, typename VT>
__host__ __device__ size_t spill_l1_bytes(int T) {
  return al16((size_t)T * sizeof(VT)) + al16((size_t)T * 4) + al16(sizeof(ChunkScratch<TW, VT>)) + 16;
}

template <int TW, typename VT>
__global__ void __launch_bounds__(TW) k_num_spill(ProbD P, const int* __restrict__ rows, long long nrows,
                                                  int l1_logT, int cap, unsigned char* pool, long long l2_slots,
                                                  long long chunk_bytes, unsigned* pool2, long long kw_max,
                                                  unsigned long long* fetch) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ long long fetch_s;
  __shared__ long long scan_scratch[33];
  Team<TW> tm;
  const int T = 1 << l1_logT;
  const LpHash tmask(l1_logT, P.hash_mode);
  VT* vals1 = reinterpret_cast<VT*>(smem);
  int* keys1 = reinterpret_cast<int*>(smem + al16((size_t)T * sizeof(VT)));
  ChunkScratch<TW, VT>* csc =
      reinterpret_cast<ChunkScratch<TW, VT>*>(smem + al16((size_t)T * sizeof(VT)) + al16((size_t)T * 4));
  int* occ = reinterpret_cast<int*>(reinterpret_cast<unsigned char*>(csc) + al16(sizeof(ChunkScratch<TW, VT>)));
  int* keys2 = reinterpret_cast<int*>(pool + (long long)blockIdx.x * chunk_bytes);
  VT* vals2 = reinterpret_cast<VT*>(reinterpret_cast<unsigned char*>(keys2) + al16((size_t)l2_slots * 4));
  const LpHash t2mask(ilog2_ceil(l2_slots), P.hash_mode);
  unsigned* bm = pool2 + (long long)blockIdx.x * 2 * kw_max;
  unsigned* pre = bm + kw_max;

  for (long long r = cta_next_row(fetch, &fetch_s); r < nrows; r = cta_next_row(fetch, &fetch_s)) {
    const long long g = rows[r];
    const int b = inst_of(P.arow0s, P.ninst, g);
    const InstD& I = P.inst[b];
    const long long i = g - I.arow0;
    const long long c0 = I.Crp[i];
    const long long s = I.Crp[i + 1] - c0;
    const long long k = I.k;
    const long long kw = (k + 31) >> 5;
    for (int x = tm.lane; x < T; x += TW) {
      keys1[x] = kEmpty;
      vals1[x] = VT(0);
    }
    for (long long x = tm.lane; x < l2_slots; x += TW) {
      keys2[x] = kEmpty;
      vals2[x] = VT(0);
    }
    if (tm.lane == 0) *occ = 0;
    __threadfence_block();
    __syncthreads();
    const long long a0 = rp_at(I.A, i), a1 = rp_at(I.A, i + 1);
    const VT* __restrict__ Ax = reinterpret_cast<const VT*>(I.A.vx);
    const VT* __restrict__ Bx = reinterpret_cast<const VT*>(I.B.vx);
    const int* __restrict__ Bj = I.B.cj;
    auto range = [&](int j, long long* bs, long long* be) {
      *bs = rp_at(I.B, j);
      *be = rp_at(I.B, j + 1);
    };
    auto aval = [&](long long p) { return Ax[p]; };
    auto body = [&](long long q, int t) {
      const int key = Bj[q];
      if ((unsigned long long)(unsigned)key >= (unsigned long long)k) {
        dev_fail(P.status, kDevBadIndex, 14, g);
        return;
      }
      const VT v = csc->av[t] * Bx[q];
      const int s1 = lp_insert(keys1, tmask, occ, cap, key);
      if (s1 >= 0) {
        atomicAdd(vals1 + s1, v);
      } else {
        const int s2 = lp_insert(keys2, t2mask, nullptr, -1, key);
        if (s2 >= 0) atomicAdd(vals2 + s2, v);
        else dev_fail(P.status, kDevTableFull, 15, g);
      }
    };
    auto pf = [&](long long q) {
      prefetch_l1(Bj + q);
      prefetch_l1(Bx + q);
    };
    for_each_product<TW, VT>(tm, csc, scan_scratch, I.A.cj, a0, a1, range, aval, body, pf);
    __threadfence_block();
    __syncthreads();
    // fold L2 entries whose key also reached L1 into L1
    for (long long x = tm.lane; x < l2_slots; x += TW) {
      const int kk = keys2[x];
      if (kk < 0) continue;
      const int s1 = lp_find(keys1, tmask, kk);
      if (s1 >= 0) {
        vals1[s1] += vals2[x];
        keys2[x] = -2;
      }
    }
    __threadfence_block();
    __syncthreads();
    for (int x = tm.lane; x < T; x += TW) {
      const int kk = keys1[x];
      if (kk >= 0) atomicOr(bm + (kk >> 5), 1u << (kk & 31));
    }
    for (long long x = tm.lane; x < l2_slots; x += TW) {
      const int kk = keys2[x];
      if (kk >= 0) atomicOr(bm + (kk >> 5), 1u << (kk & 31));
    }
    __threadfence_block();
    __syncthreads();
    long long run = 0;
    for (long long wb = 0; wb < kw; wb += TW) {
      const long long w = wb + tm.lane;
      const unsigned word = (w < kw) ? bm[w] : 0u;
      long long tot;
      const long long ex = team_excl_scan<TW>(tm, __popc(word), &tot, scan_scratch);
      if (w < kw) pre[w] = (unsigned)(run + ex);
      run += tot;
    }
    if (tm.lane == 0 && run != s) dev_fail(P.status, kDevRowSizeMismatch, 16, g);
    __threadfence_block();
    __syncthreads();
    VT* __restrict__ Cx = reinterpret_cast<VT*>(I.Cx);
    int* __restrict__ Cj = I.Cj;
    auto rank_of = [&](int kk) -> long long {
      const int w = kk >> 5;
      return (long long)pre[w] + __popc(bm[w] & ((1u << (kk & 31)) - 1u));
    };
    for (int x = tm.lane; x < T; x += TW) {
      const int kk = keys1[x];
      if (kk < 0) continue;
      const long long p = rank_of(kk);
      if (p < s) {
        Cj[c0 + p] = kk;
        Cx[c0 + p] = vals1[x];
      }
    }
    for (long long x = tm.lane; x < l2_slots; x += TW) {
      const int kk = keys2[x];
      if (kk < 0) continue;
      const long long p = rank_of(kk);
      if (p < s) {
        Cj[c0 + p] = kk;
        Cx[c0 + p] = vals2[x];
      }
    }
    __threadfence_block();
    __syncthreads();
    for (long long w = tm.lane; w < kw; w += TW) bm[w] = 0u;
    __threadfence_block();
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// Rank-dense rows (CTA teams): the dense accumulator of Section 3.1.2 with
// its values kept by rank instead of by column.  Rows of this class have more
// columns than the largest shared hash table holds, but few enough that the
// row's values fit shared memory next to a k-bit column bitmap:
//   1. every product marks its column in the bitmap (first pass over the
//      products, columns only)
//   2. the count of set bits before every word (its rank base)
//   3. every product adds a_ij * b_jl to the value at its column's rank
//      (second pass; shared atomic adds)
//   4. values written in order; columns from the bitmap, each word's set bits
//      at its base
// Per row this costs O(k / 32) for the bitmap and O(f) for the products,
// where the windowed dense rows sweep their k values in windows.
// ---------------------------------------------------------------------------
template <int TW, typename VT>
__host__ __device__ size_t rdense_fixed_bytes(long long kw_cap) {
  return al16((size_t)((kw_cap + 3) & ~3ll) * 4) + al16((size_t)(kw_cap + 1) * 2) +
         al16(sizeof(ChunkScratch<TW, VT>)) + al16((size_t)kStagedPasses * TW * 4) + 16;
}

template <int TW, typename VT>
__global__ void __launch_bounds__(TW) k_num_rdense(ProbD P, const int* __restrict__ rows, long long nrows,
                                                   long long kw_cap, long long vcap, unsigned long long* fetch) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ long long scan_scratch[33];
  __shared__ long long fetch_s;
  Team<TW> tm;
  unsigned* bm = reinterpret_cast<unsigned*>(smem);
  unsigned short* gp = reinterpret_cast<unsigned short*>(smem + al16((size_t)((kw_cap + 3) & ~3ll) * 4));
  ChunkScratch<TW, VT>* csc = reinterpret_cast<ChunkScratch<TW, VT>*>(
      reinterpret_cast<unsigned char*>(gp) + al16((size_t)(kw_cap + 1) * 2));
  int* seg = reinterpret_cast<int*>(reinterpret_cast<unsigned char*>(csc) + al16(sizeof(ChunkScratch<TW, VT>)));
  VT* vals = reinterpret_cast<VT*>(smem + rdense_fixed_bytes<TW, VT>(kw_cap));
  for (long long r = cta_next_row(fetch, &fetch_s); r < nrows; r = cta_next_row(fetch, &fetch_s)) {
    const long long g = rows[r];
    const int b = inst_of(P.arow0s, P.ninst, g);
    const InstD& I = P.inst[b];
    const long long i = g - I.arow0;
    const long long c0 = I.Crp[i];
    const long long s = I.Crp[i + 1] - c0;
    const long long k = I.k;
    const long long kw = (k + 31) >> 5;
    if (s > vcap || kw > kw_cap) {   // binning keeps every row of the class within both
      if (tm.lane == 0) dev_fail(P.status, kDevTableFull, 19, g);
      continue;
    }
    const long long a0 = rp_at(I.A, i), a1 = rp_at(I.A, i + 1);
    const VT* __restrict__ Ax = reinterpret_cast<const VT*>(I.A.vx);
    const VT* __restrict__ Bx = reinterpret_cast<const VT*>(I.B.vx);
    const int* __restrict__ Bj = I.B.cj;
    auto range = [&](int j, long long* bs, long long* be) {
      *bs = rp_at(I.B, j);
      *be = rp_at(I.B, j + 1);
    };
    for (long long w = tm.lane; w < kw; w += TW) bm[w] = 0u;
    tm.sync();
    // 1. columns
    auto no_val = [&](long long) { return VT(0); };
    auto mark = [&](long long q, int) {
      const int col = Bj[q];
      if ((unsigned long long)(unsigned)col < (unsigned long long)k) atomicOr(bm + (col >> 5), 1u << (col & 31));
      else dev_fail(P.status, kDevBadIndex, 20, g);
    };
    auto pf_col = [&](long long q) { prefetch_l1(Bj + q); };
    for_each_product<TW, VT>(tm, csc, scan_scratch, I.A.cj, a0, a1, range, no_val, mark, pf_col, seg);
    // 2. rank bases: each thread sums a contiguous run of words, the runs are
    // scanned across the team, then each word of the run gets its base
    {
      const long long sg = (kw + TW - 1) / TW;
      const long long w0 = tm.lane * sg, w1 = w0 + sg < kw ? w0 + sg : kw;
      int cseg = 0;
      for (long long w = w0; w < w1; ++w) cseg += __popc(bm[w]);
      long long run;
      long long pre = team_excl_scan<TW>(tm, cseg, &run, scan_scratch);
      for (long long w = w0; w < w1; ++w) {
        gp[w] = (unsigned short)pre;
        pre += __popc(bm[w]);
      }
      if (tm.lane == 0 && run != s) dev_fail(P.status, kDevRowSizeMismatch, 21, g);
    }
    for (long long x = tm.lane; x < s; x += TW) vals[x] = VT(0);
    tm.sync();
    // 3. values at their ranks
    auto aval = [&](long long p) { return Ax[p]; };
    auto add = [&](long long q, int t) {
      const int col = Bj[q];
      if ((unsigned long long)(unsigned)col >= (unsigned long long)k) return;
      const int w = col >> 5;
      const long long rk = (long long)gp[w] + __popc(bm[w] & ((1u << (col & 31)) - 1u));
      if (rk < s) atomicAdd(vals + rk, csc->av[t] * Bx[q]);
    };
    auto pf = [&](long long q) {
      prefetch_l1(Bj + q);
      prefetch_l1(Bx + q);
    };
    for_each_product<TW, VT>(tm, csc, scan_scratch, I.A.cj, a0, a1, range, aval, add, pf, seg);
    // 4. the row in order
    VT* __restrict__ Cx = reinterpret_cast<VT*>(I.Cx);
    int* __restrict__ Cj = I.Cj;
    for (long long x = tm.lane; x < s; x += TW) Cx[c0 + x] = vals[x];
    for (long long w = tm.lane; w < kw; w += TW) {
      unsigned m = bm[w];
      long long o = gp[w];
      while (m) {
        const int bit = __ffs(m) - 1;
        m &= m - 1u;
        if (o < s) Cj[c0 + o] = (int)(32 * w + bit);
        ++o;
      }
    }
  }
}

template <class K>
cudaError_t set_smem(K kernel, size_t bytes) {
  // the kernels also hold up to 1 KB of static shared memory: opt in above 47 KB of dynamic
  if (bytes + 1024 > 48 * 1024) return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  return cudaSuccess;
}

template <int TW, typename VT>
cudaError_t run_hash(const LaunchCtx& L, const ProbD& P, const NumLaunch& S) {
  const int T = 1 << S.logT;
  // the rank bitmap when every row's column range fits it, else the sort buffer
  long long kw_cap = 0;
  if (S.kwords_max > 0 && S.kwords_max <= kRankMaxWords &&
      num_cta_bytes<TW, VT>(T, S.kwords_max) + 1024 <= (size_t)L.max_smem_optin)
    kw_cap = S.kwords_max;
  const size_t smem = num_cta_bytes<TW, VT>(T, kw_cap);
  if (smem > (size_t)L.max_smem_optin) return cudaErrorInvalidConfiguration;
  auto kern = k_num_hash<TW, VT>;
  cudaError_t e = set_smem(kern, smem);
  if (e != cudaSuccess) return e;
  const unsigned grid = resident_grid(kern, TW, smem, L.num_sms, S.nrows);
  e = cudaMemsetAsync(S.fetch, 0, sizeof(unsigned long long), L.stream);
  if (e != cudaSuccess) return e;
  KKS_LAUNCHED();
  kern<<<grid, TW, smem, L.stream>>>(P, S.rows, S.nrows, S.logT, kw_cap, S.fetch);
  return cudaGetLastError();
}

template <int TW, typename VT>
cudaError_t run_warp(const LaunchCtx& L, const ProbD& P, const NumLaunch& S) {
  const int T = 1 << S.logT;
  const size_t tb = warp_team_bytes<TW, VT>(T);
  int teams = (int)(kTeamSmemBudget / tb);
  const int tmax = 256 / TW;
  if (teams > tmax) teams = tmax;
  if (teams < 1) teams = 1;
  const size_t smem = tb * teams;
  if (smem > (size_t)L.max_smem_optin) return cudaErrorInvalidConfiguration;
  auto kern = k_num_warp<TW, VT>;
  cudaError_t e = set_smem(kern, smem);
  if (e != cudaSuccess) return e;
  const unsigned grid = resident_grid(kern, TW * teams, smem, L.num_sms, (S.nrows + teams - 1) / teams);
  KKS_LAUNCHED();
  kern<<<grid, TW * teams, smem, L.stream>>>(P, S.rows, S.nrows, S.logT);
  return cudaGetLastError();
}

template <int TW, typename VT>
cudaError_t run_cpn(const LaunchCtx& L, const ProbD& P, const NumLaunch& S) {
  const int T = 1 << S.logT;
  const size_t tb = cpn_team_bytes<TW, VT>(T);
  int teams = (int)(kTeamSmemBudget / tb);
  const int tmax = 256 / TW;
  if (teams > tmax) teams = tmax;
  if (teams < 1) teams = 1;
  const size_t smem = tb * teams;
  if (smem > (size_t)L.max_smem_optin) return cudaErrorInvalidConfiguration;
  auto kern = k_num_cpn<TW, VT>;
  cudaError_t e = set_smem(kern, smem);
  if (e != cudaSuccess) return e;
  const unsigned grid = resident_grid(kern, TW * teams, smem, L.num_sms, (S.nrows + teams - 1) / teams);
  KKS_LAUNCHED();
  kern<<<grid, TW * teams, smem, L.stream>>>(P, S.rows, S.nrows, S.logT);
  return cudaGetLastError();
}

template <typename VT>
cudaError_t run_wb(const LaunchCtx& L, const ProbD& P, const NumLaunch& S) {
  const size_t smem = wb_team_bytes<VT>(1 << S.logT) * kWbTeams;
  if (smem > (size_t)L.max_smem_optin) return cudaErrorInvalidConfiguration;
  auto kern = k_num_wb<VT>;
  cudaError_t e = set_smem(kern, smem);
  if (e != cudaSuccess) return e;
  const unsigned grid = resident_grid(kern, 32 * kWbTeams, smem, L.num_sms, (S.nrows + kWbTeams - 1) / kWbTeams);
  KKS_LAUNCHED();
  kern<<<grid, 32 * kWbTeams, smem, L.stream>>>(P, S.rows, S.nrows, S.logT);
  return cudaGetLastError();
}

template <typename VT, bool STAGE>
cudaError_t run_dense(const LaunchCtx& L, const ProbD& P, const NumLaunch& S) {
  constexpr int TW = 1024;
  // the widest window that fits one CTA's shared memory (a 1024-thread CTA
  // of this kernel holds a whole SM's registers, so one CTA runs per SM)
  int wl = 17;
  while (wl > 10 && dense_win_bytes<TW, VT, STAGE>(wl) + 1024 > (size_t)L.max_smem_optin) --wl;
  const size_t smem = dense_win_bytes<TW, VT, STAGE>(wl);
  if (smem > (size_t)L.max_smem_optin) return cudaErrorInvalidConfiguration;
  auto kern = k_num_dense<TW, VT, STAGE>;
  cudaError_t e = set_smem(kern, smem);
  if (e != cudaSuccess) return e;
  const unsigned grid = resident_grid(kern, TW, smem, L.num_sms, S.nrows);
  e = cudaMemsetAsync(S.fetch, 0, sizeof(unsigned long long), L.stream);
  if (e != cudaSuccess) return e;
  KKS_LAUNCHED();
  kern<<<grid, TW, smem, L.stream>>>(P, S.rows, S.nrows, wl, S.b_sorted, S.fetch);
  return cudaGetLastError();
}

// Rank-dense rows: bin logT 1 takes 1024-thread CTAs (one per SM, values of
// rows up to the class limit), logT 2 takes 512-thread CTAs with half the
// shared memory each (two per SM, smaller rows).
template <typename VT>
cudaError_t run_rdense(const LaunchCtx& L, const ProbD& P, const NumLaunch& S) {
  const long long kw_cap = S.kwords_max;
  auto go = [&](auto kern, int tw, size_t fixed, size_t budget) -> cudaError_t {
    if (fixed + 1024 >= budget) return cudaErrorInvalidConfiguration;
    long long vcap = (long long)((budget - 1024 - fixed) / sizeof(VT));
    if (vcap > 65535) vcap = 65535;   // 16-bit rank bases
    const size_t smem = fixed + al16((size_t)vcap * sizeof(VT));
    if (smem > (size_t)L.max_smem_optin) return cudaErrorInvalidConfiguration;
    cudaError_t e = set_smem(kern, smem);
    if (e != cudaSuccess) return e;
    const unsigned grid = resident_grid(kern, tw, smem, L.num_sms, S.nrows);
    e = cudaMemsetAsync(S.fetch, 0, sizeof(unsigned long long), L.stream);
    if (e != cudaSuccess) return e;
    KKS_LAUNCHED();
    kern<<<grid, tw, smem, L.stream>>>(P, S.rows, S.nrows, kw_cap, vcap, S.fetch);
    return cudaGetLastError();
  };
  if (S.logT == 2)
    return go(k_num_rdense<512, VT>, 512, rdense_fixed_bytes<512, VT>(kw_cap), (size_t)L.max_smem_optin / 2);
  return go(k_num_rdense<1024, VT>, 1024, rdense_fixed_bytes<1024, VT>(kw_cap), (size_t)L.max_smem_optin);
}

template <typename VT>
cudaError_t run_spill(const LaunchCtx& L, const ProbD& P, const NumLaunch& S) {
  constexpr int TW = 1024;
  const int T = 1 << S.l1_logT;
  const size_t smem = spill_l1_bytes<TW, VT>(T);
  if (smem > (size_t)L.max_smem_optin) return cudaErrorInvalidConfiguration;
  auto kern = k_num_spill<TW, VT>;
  cudaError_t e = set_smem(kern, smem);
  if (e != cudaSuccess) return e;
  int cap = (int)(S.max_occ * T);
  if (cap < 1) cap = 1;
  if (cap > T - 1) cap = T - 1;
  long long grid = S.nchunks;
  if (grid > S.nrows) grid = S.nrows;
  const long long l2_slots = 1ll << S.logT;
  e = cudaMemsetAsync(S.fetch, 0, sizeof(unsigned long long), L.stream);
  if (e != cudaSuccess) return e;
  KKS_LAUNCHED();
  kern<<<(unsigned)grid, TW, smem, L.stream>>>(P, S.rows, S.nrows, S.l1_logT, cap, (unsigned char*)S.pool, l2_slots,
                                               S.chunk_bytes, (unsigned*)S.pool2, S.kwords_max, S.fetch);
  return cudaGetLastError();
}

template <typename VT>
cudaError_t run_thread(const LaunchCtx& L, const ProbD& P, const NumLaunch& S) {
  auto kern = k_num_thread<VT>;
  KKS_LAUNCHED();
  kern<<<resident_grid(kern, 256, 0, L.num_sms, (S.nrows + 255) / 256), 256, 0, L.stream>>>(P, S.rows, S.nrows);
  return cudaGetLastError();
}

template <int TW, typename VT, int MODE>
cudaError_t run_part(const LaunchCtx& L, const ProbD& P, const NumLaunch& S) {
  const size_t smem = part_cta_bytes<TW, VT>(1 << S.logT);
  if (smem + 1024 > (size_t)L.max_smem_optin) return cudaErrorInvalidConfiguration;
  auto kern = k_num_part<TW, VT, MODE>;
  cudaError_t e = set_smem(kern, smem);
  if (e != cudaSuccess) return e;
  const unsigned grid = resident_grid(kern, TW, smem, L.num_sms, S.nrows);
  e = cudaMemsetAsync(S.fetch, 0, sizeof(unsigned long long), L.stream);
  if (e != cudaSuccess) return e;
  KKS_LAUNCHED();
  kern<<<grid, TW, smem, L.stream>>>(P, S.rows, S.nrows, S.logT, S.fetch);
  return cudaGetLastError();
}

template <typename VT>
cudaError_t dispatch(const LaunchCtx& L, const ProbD& P, const NumLaunch& S) {
  switch (S.cls) {
    case kClsT1: return run_thread<VT>(L, P, S);
    case kClsW8: return S.positions ? run_cpn<8, VT>(L, P, S) : run_warp<8, VT>(L, P, S);
    case kClsW32:
      if (!S.positions) return run_warp<32, VT>(L, P, S);
      return S.b_sorted && S.window ? run_wb<VT>(L, P, S) : run_cpn<32, VT>(L, P, S);
    case kClsC256:
      if (S.part == kPartTeamSeq) return run_part<256, VT, kPartTeamSeq>(L, P, S);
      if (S.part == kPartThreadPar) return run_part<256, VT, kPartThreadPar>(L, P, S);
      // tables of 4096 slots or more: 512 threads per row (the shared memory
      // allows two CTAs per SM either way)
      if (S.logT >= 12) return run_hash<512, VT>(L, P, S);
      return run_hash<256, VT>(L, P, S);
    case kClsC1024:
      if (S.part == kPartTeamSeq) return run_part<1024, VT, kPartTeamSeq>(L, P, S);
      if (S.part == kPartThreadPar) return run_part<1024, VT, kPartThreadPar>(L, P, S);
      return run_hash<1024, VT>(L, P, S);
    case kClsDense:
      if (S.logT == 1 || S.logT == 2) return run_rdense<VT>(L, P, S);
      return (S.stage && S.b_sorted) ? run_dense<VT, true>(L, P, S) : run_dense<VT, false>(L, P, S);
    case kClsSpill: return run_spill<VT>(L, P, S);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace

size_t numeric_cta_bytes(int logT, int dtype, long long kwords) {
  // the launcher takes the rank layout when it fits, else the sort buffer
  const int T = 1 << logT;
  const long long kw = (kwords > 0 && kwords <= kRankMaxWords) ? kwords : 0;
  if (dtype == 1) {
    const size_t a = num_cta_bytes<1024, double>(T, kw), b = num_cta_bytes<1024, double>(T, 0);
    return a < b ? a : b;
  }
  const size_t a = num_cta_bytes<1024, float>(T, kw), b = num_cta_bytes<1024, float>(T, 0);
  return a < b ? a : b;
}

// Largest row (columns) of the rank-dense class: 1024-thread CTAs on the
// whole shared memory (small = 0) or 512-thread CTAs on half of it (small = 1);
// 0 when the bitmap of kwords words leaves no room.
long long numeric_rdense_vcap(long long kwords, int dtype, size_t max_smem, int small) {
  if (kwords <= 0 || kwords > kRankMaxWords) return 0;
  const size_t budget = small ? max_smem / 2 : max_smem;
  const size_t fixed = dtype == 1 ? (small ? rdense_fixed_bytes<512, double>(kwords) : rdense_fixed_bytes<1024, double>(kwords))
                                  : (small ? rdense_fixed_bytes<512, float>(kwords) : rdense_fixed_bytes<1024, float>(kwords));
  if (fixed + 1024 >= budget) return 0;
  long long v = (long long)((budget - 1024 - fixed) / (dtype == 1 ? 8 : 4));
  return v > 65535 ? 65535 : v;
}

size_t numeric_spill_l1_bytes(int logT, int dtype) {
  return dtype == 1 ? spill_l1_bytes<1024, double>(1 << logT) : spill_l1_bytes<1024, float>(1 << logT);
}

size_t numeric_l2_chunk_bytes(long long slots, int dtype) {
  return al16((size_t)slots * 4) + al16((size_t)slots * (dtype == 1 ? 8 : 4));
}

cudaError_t launch_numeric(const LaunchCtx& L, const ProbD& P, const NumLaunch& S) {
  if (S.nrows <= 0) return cudaSuccess;
  return S.dtype == 1 ? dispatch<double>(L, P, S) : dispatch<float>(L, P, S);
}

}  // namespace kks
