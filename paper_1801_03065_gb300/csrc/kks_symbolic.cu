// kks_symbolic.cu -- symbolic phase: the size of every row of C.
//
// Algorithm 3 with Phase = symbolic: a team takes a row i of A, runs over the
// products of A(i,:) with the rows of B and inserts the column keys into its
// level-1 accumulator; C_row_pointers(i) is the number of distinct columns.
// On the compressed B (Section 3.2) the keys are column-set indices and the
// accumulator ORs the 32-bit column sets, so the row size is the number of
// set bits of the union.  Variants:
//   k_sym_thread<COMP>          : one thread per row of at most 32 products
//   k_sym_warp<TW, COMP>        : warp teams (8 or 32 lanes), shared LP table
//                                 sized to hold the row, batched loads
//   k_sym_hash<TW, COMP, false> : CTA teams, shared LP table sized to hold the row
//   k_sym_hash<TW, COMP, true>  : shared L1 table with the maximum-occupancy
//                                 cut-off plus a global L2 table (Algorithm 3's
//                                 two-level accumulator); a key may sit in both levels,
//                                 so the count merges them (union)
//   k_sym_dense<COMP>           : a k-bit bitmap in shared memory (the dense
//                                 accumulator of Section 3.1.2 in bit form)
//   k_sym_dwarp<COMP, U>        : the same bitmap per warp team, for bitmaps of
//                                 at most 2^11 words (rows binned by bitmap size)
#include "kks_internal.h"

namespace kks {

namespace {

__host__ __device__ constexpr size_t al16(size_t x) { return (x + 15) & ~size_t(15); }

template <int TW, bool COMP>
__host__ __device__ size_t sym_team_bytes(int T) {
  return al16((size_t)T * 4) * (COMP ? 2 : 1) + al16(sizeof(ChunkScratch<TW, int>)) + 16;
}

template <int TW, bool COMP, bool SPILL>
__global__ void k_sym_hash(ProbD P, const int* __restrict__ rows, long long nrows, int logT, int cap,
                           int* l2_pool, long long l2_slots, long long* __restrict__ rowsize,
                           unsigned long long* fetch) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ long long scan_scratch[33];
  __shared__ long long fetch_s;
  Team<TW> tm;
  const int T = 1 << logT;
  const LpHash tmask(logT, P.hash_mode);
  unsigned char* base = smem + (size_t)tm.id * sym_team_bytes<TW, COMP>(T);
  int* keys = reinterpret_cast<int*>(base);
  unsigned* masks = reinterpret_cast<unsigned*>(base + al16((size_t)T * 4));
  ChunkScratch<TW, int>* csc =
      reinterpret_cast<ChunkScratch<TW, int>*>(base + al16((size_t)T * 4) * (COMP ? 2 : 1));
  int* occ = reinterpret_cast<int*>(reinterpret_cast<unsigned char*>(csc) + al16(sizeof(ChunkScratch<TW, int>)));

  const long long team = (long long)blockIdx.x * tm.per_cta + tm.id;
  const long long nteams = (long long)gridDim.x * tm.per_cta;
  int* k2 = nullptr;
  unsigned* m2 = nullptr;
  const LpHash t2mask(ilog2_ceil(l2_slots), P.hash_mode);
  if (SPILL) {
    k2 = l2_pool + team * l2_slots * (COMP ? 2 : 1);
    m2 = reinterpret_cast<unsigned*>(k2 + l2_slots);
  }

  // CTA teams take their rows from the counter, warp teams by a fixed stride
  constexpr bool kFetch = Team<TW>::kCta;
  for (long long r = kFetch ? cta_next_row(fetch, &fetch_s) : team; r < nrows;
       r = kFetch ? cta_next_row(fetch, &fetch_s) : r + nteams) {
    const long long g = rows[r];
    const int b = inst_of(P.arow0s, P.ninst, g);
    const InstD& I = P.inst[b];
    const long long i = g - I.arow0;
    for (int x = tm.lane; x < T; x += TW) {
      keys[x] = kEmpty;
      if (COMP) masks[x] = 0u;
    }
    if (SPILL) {
      for (long long x = tm.lane; x < l2_slots; x += TW) {
        k2[x] = kEmpty;
        if (COMP) m2[x] = 0u;
      }
    }
    if (tm.lane == 0) *occ = 0;
    if (SPILL) __threadfence_block();
    tm.sync();
    const long long a0 = rp_at(I.A, i), a1 = rp_at(I.A, i + 1);
    const long long brow0 = I.brow0;
    auto range = [&](int j, long long* bs, long long* be) {
      if (COMP) {
        *bs = P.Bcp[brow0 + j];
        *be = P.Bcp[brow0 + j + 1];
      } else {
        *bs = rp_at(I.B, j);
        *be = rp_at(I.B, j + 1);
      }
    };
    auto aval = [&](long long) { return 0; };
    const int* __restrict__ Bj = I.B.cj;
    auto body = [&](long long q, int) {
      const int key = COMP ? P.csi[q] : Bj[q];
      const unsigned m = COMP ? P.cs[q] : 0u;
      int s = lp_insert(keys, tmask, occ, SPILL ? cap : -1, key);
      if (s >= 0) {
        if (COMP) atomicOr(masks + s, m);
      } else if (SPILL) {   // refused by the occupancy cut-off (-1) or L1 full (-2)
        int s2 = lp_insert(k2, t2mask, nullptr, -1, key);
        if (s2 >= 0) {
          if (COMP) atomicOr(m2 + s2, m);
        } else {
          dev_fail(P.status, kDevTableFull, 2, g);
        }
      } else {
        dev_fail(P.status, kDevTableFull, 1, g);
      }
    };
    auto pf = [&](long long q) {
      if (COMP) {
        prefetch_l1(P.csi + q);
        prefetch_l1(P.cs + q);
      } else {
        prefetch_l1(Bj + q);
      }
    };
    for_each_product<TW, int>(tm, csc, scan_scratch, I.A.cj, a0, a1, range, aval, body, pf);
    if (SPILL) {
      __threadfence_block();
      tm.sync();
    }
    long long c = 0;
    for (int x = tm.lane; x < T; x += TW) {
      if (keys[x] != kEmpty) c += COMP ? __popc(masks[x]) : 1;
    }
    if (SPILL) {
      for (long long x = tm.lane; x < l2_slots; x += TW) {
        const int kk = k2[x];
        if (kk == kEmpty) continue;
        const int s1 = lp_find(keys, tmask, kk);
        if (COMP) c += __popc(m2[x] & (s1 >= 0 ? ~masks[s1] : 0xffffffffu));
        else c += (s1 < 0) ? 1 : 0;
      }
    }
    c = team_sum<TW>(tm, c, scan_scratch);
    if (tm.lane == 0) rowsize[g] = c;
    tm.sync();
  }
}

// Warp teams (W8, W32 rows): slots of one key (or key + column-set word), the
// union of union_chunk with the loads of several passes in flight; the row
// size is the number of claimed slots, or of the column bits set first by an
// insert (counted as they are ORed in, so no sweep of the table is needed).
template <int TW, bool COMP>
__host__ __device__ size_t symw_team_bytes(int T) {
  return al16((size_t)T * 4 * (COMP ? 2 : 1)) + al16((size_t)(TW + 1) * 4) + al16((size_t)TW * 8);
}

// One row g by a warp team whose table of 2^logT slots sits at words.
template <int TW, bool COMP>
__device__ __forceinline__ void sym_warp_row(const Team<TW>& tm, const ProbD& P, int* words, int* pre, long long* qsv,
                                             int logT, const LpHash& hs, long long g, long long* __restrict__ rowsize) {
  constexpr int S = COMP ? 2 : 1;
  const int T = 1 << logT;
  const int b = inst_of(P.arow0s, P.ninst, g);
  const InstD& I = P.inst[b];
  const long long i = g - I.arow0;
  for (int x = tm.lane; x < T; x += TW) {
    if (COMP) reinterpret_cast<int2*>(words)[x] = make_int2(kEmpty, 0);
    else words[x] = kEmpty;
  }
  __syncwarp(tm.mask);
  const long long a0 = rp_at(I.A, i), a1 = rp_at(I.A, i + 1);
  const long long brow0 = I.brow0;
  const int* __restrict__ Aj = I.A.cj;
  int fresh = 0;
  for (long long c = a0; c < a1; c += TW) {
    const long long p = c + tm.lane;
    long long qs = 0;
    int ql = 0;
    if (p < a1) {
      const int j = Aj[p];
      if (COMP) {
        qs = P.Bcp[brow0 + j];
        ql = (int)(P.Bcp[brow0 + j + 1] - qs);
      } else {
        qs = rp_at(I.B, j);
        ql = (int)(rp_at(I.B, j + 1) - qs);
      }
    }
    fresh += union_chunk<TW, S, COMP>(tm.mask, tm.lane, pre, qsv, qs, ql, COMP ? P.csi : I.B.cj, P.cs, words,
                                      hs, P.status, 1, g);
  }
  // claimed slots, or (compressed) newly set column bits, summed over the team
  long long cnt = fresh;
#pragma unroll
  for (int d = TW / 2; d > 0; d >>= 1) cnt += __shfl_xor_sync(tm.mask, cnt, d, TW);
  if (tm.lane == 0) rowsize[g] = cnt;
  __syncwarp(tm.mask);
}

template <int TW, bool COMP>
__global__ void __launch_bounds__(256, 4) k_sym_warp(ProbD P, const int* __restrict__ rows, long long nrows,
                                                     int logT, long long* __restrict__ rowsize) {
  extern __shared__ __align__(16) unsigned char smem[];
  Team<TW> tm;
  constexpr int S = COMP ? 2 : 1;
  const int T = 1 << logT;
  const LpHash hs(logT, P.hash_mode);
  unsigned char* base = smem + (size_t)tm.id * symw_team_bytes<TW, COMP>(T);
  int* words = reinterpret_cast<int*>(base);
  int* pre = reinterpret_cast<int*>(base + al16((size_t)T * 4 * S));
  long long* qsv = reinterpret_cast<long long*>(base + al16((size_t)T * 4 * S) + al16((size_t)(TW + 1) * 4));
  const long long team = (long long)blockIdx.x * tm.per_cta + tm.id;
  const long long nteams = (long long)gridDim.x * tm.per_cta;
  for (long long r = team; r < nrows; r += nteams)
    sym_warp_row<TW, COMP>(tm, P, words, pre, qsv, logT, hs, rows[r], rowsize);
}

// Compressed warp rows on a bitmap window (B rows sorted): the column sets of
// row i lie between the first set of the first and the last set of the last
// column among the compressed B rows over A(i,:); when that window is at most
// kSymWbWords sets wide the union is a bitmap over it, addressed directly by
// set index (no hashing, no probing), and the row size is the number of
// column bits the inserts set first.  Every word an insert turns nonzero is
// flagged in a summary bitmap (one bit per word); after the row, lane L walks
// the flags of words [64 L, 64 L + 64), so the row's column sets come out in
// increasing set order (recorded for the numeric phase) and exactly the words
// that were set are cleared.  Wider rows take the hash path (sym_warp_row) in
// the same shared memory.
//
// Rows of one chunk of A (at most 32 entries) whose compressed B rows hold at
// most kMergeLen sets each can instead merge those rows (option sym_merge):
// every compressed B row is sorted by set index, so the union of Section 3.2
// is produced one set at a time, smallest first: the warp takes the minimum
// of the lanes' current set indices, ORs the bits of the lanes that hold it,
// and those lanes move to their next entry.  The number of steps is the
// number of column sets of C(i,:); no atomics, no window limit, and the sets
// come out in increasing order for the numeric phase.  Each lane's row is
// staged in shared memory first (the bitmap's words, which are cleared again
// before a later row ORs into them).
constexpr int kSymWbWords = 1344;
constexpr int kSymWbSumm = 64;   // summary words: 32 lanes x 2 cover 2048 >= kSymWbWords window words
constexpr int kMergeLen = 19;    // staged entries per lane (odd stride: no bank conflicts in the stores)
static_assert(64 * kMergeLen + 2 * kRowSetCap <= kSymWbWords, "merge staging must fit the window bitmap");

__host__ __device__ size_t symwb_team_bytes(int T) {
  const size_t a = al16((size_t)kSymWbWords * 4), h = al16((size_t)T * 8);
  return (a > h ? a : h) + al16((size_t)33 * 4) + al16((size_t)32 * 8) + al16((size_t)kSymWbSumm * 4);
}

__global__ void __launch_bounds__(256, 4) k_sym_wb(ProbD P, const int* __restrict__ rows, long long nrows, int logT,
                                                   long long* __restrict__ rowsize, int merge) {
  extern __shared__ __align__(16) unsigned char smem[];
  Team<32> tm;
  const int T = 1 << logT;
  const LpHash hs(logT, P.hash_mode);
  const size_t tb = symwb_team_bytes(T);
  unsigned char* base = smem + (size_t)tm.id * tb;
  const size_t tab = tb - al16((size_t)33 * 4) - al16((size_t)32 * 8) - al16((size_t)kSymWbSumm * 4);
  unsigned* bits = reinterpret_cast<unsigned*>(base);
  int* pre = reinterpret_cast<int*>(base + tab);
  long long* qsv = reinterpret_cast<long long*>(base + tab + al16((size_t)33 * 4));
  // one flag per window word that became nonzero (the row's column sets)
  unsigned* summ = reinterpret_cast<unsigned*>(base + tab + al16((size_t)33 * 4) + al16((size_t)32 * 8));
  const bool record = P.rcnt != nullptr;
  const int lane = tm.lane;
  const unsigned full = 0xffffffffu;
  bool clean = false;
  summ[2 * tm.lane] = 0u;
  summ[2 * tm.lane + 1] = 0u;
  const long long team = (long long)blockIdx.x * tm.per_cta + tm.id;
  const long long nteams = (long long)gridDim.x * tm.per_cta;
  // The next row's head (its id, instance, row range and first chunk of A
  // column indices) is loaded while the current row runs, so a row starts
  // with its loads of the compressed B row ranges.
  long long g_n = -1, a0_n = 0, a1_n = 0;
  int b_n = 0, j_n = -1;
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
  auto fetch_j = [&]() {
    j_n = -1;
    if (g_n >= 0 && a0_n + lane < a1_n) j_n = P.inst[b_n].A.cj[a0_n + lane];
  };
  fetch_head(team);
  fetch_j();
  for (long long r = team; r < nrows; r += nteams) {
    const long long g = g_n;
    const int b = b_n;
    const InstD& I = P.inst[b];
    const long long a0 = a0_n, a1 = a1_n;
    const int j0 = j_n;
    fetch_head(r + nteams);
    const long long brow0 = I.brow0;
    const int* __restrict__ Aj = I.A.cj;
    long long qs = 0;
    int ql = 0;
    auto load_chunk = [&](long long c) {
      const long long p = c + lane;
      qs = 0;
      ql = 0;
      if (p < a1) {
        const int j = c == a0 ? j0 : Aj[p];
        qs = P.Bcp[brow0 + j];
        ql = (int)(P.Bcp[brow0 + j + 1] - qs);
      }
    };
    if (merge && a1 - a0 <= 32) {
      load_chunk(a0);
      const int mq = (int)__reduce_max_sync(full, (unsigned)ql);
      if (mq <= kMergeLen) {
        unsigned* scsi = bits;                  // [32][kMergeLen]: the lanes' set indices
        unsigned* scs = bits + 32 * kMergeLen;  // [32][kMergeLen]: their bits
        int2* sout = reinterpret_cast<int2*>(bits + 64 * kMergeLen);   // the row's sets, kRowSetCap
        for (int u0 = 0; u0 < mq; u0 += 4) {
          unsigned w[4], m[4];
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            if (u0 + u < ql) {
              w[u] = (unsigned)P.csi[qs + u0 + u];
              m[u] = P.cs[qs + u0 + u];
            }
          }
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            if (u0 + u < ql) {
              scsi[lane * kMergeLen + u0 + u] = w[u];
              scs[lane * kMergeLen + u0 + u] = m[u];
            }
          }
        }
        fetch_j();
        __syncwarp();
        constexpr unsigned kNone = 0xffffffffu;   // above every set index (k < 2^31)
        unsigned hk = ql > 0 ? scsi[lane * kMergeLen] : kNone;
        unsigned hb = ql > 0 ? scs[lane * kMergeLen] : 0u;
        int at = 0, nw = 0;
        unsigned cnt = 0;
        for (;;) {
          const unsigned mn = __reduce_min_sync(full, hk);
          if (mn == kNone) break;
          const bool mine = hk == mn;
          const unsigned bb = __reduce_or_sync(full, mine ? hb : 0u);
          cnt += (unsigned)__popc(bb);
          if (lane == 0 && nw < kRowSetCap) sout[nw] = make_int2((int)mn, (int)bb);
          ++nw;
          if (mine) {
            ++at;
            hk = at < ql ? scsi[lane * kMergeLen + at] : kNone;
            hb = at < ql ? scs[lane * kMergeLen + at] : 0u;
          }
        }
        __syncwarp();
        if (lane == 0) rowsize[g] = (long long)cnt;
        if (record) {
          if (nw <= kRowSetCap) {
            int2* dst = P.rsets + g * kRowSetCap;
            for (int x = lane; x < nw; x += 32) dst[x] = sout[x];
          }
          if (lane == 0) P.rcnt[g] = nw <= kRowSetCap ? nw : -1;
        }
        clean = false;
        __syncwarp();
        continue;
      }
    }
    unsigned smin = 0xffffffffu, smax = 0u;
    for (long long c = a0; c < a1; c += 32) {
      load_chunk(c);
      if (ql > 0) {
        smin = min(smin, (unsigned)P.csi[qs]);
        smax = max(smax, (unsigned)P.csi[qs + ql - 1]);
      }
    }
    smin = __reduce_min_sync(full, smin);
    smax = __reduce_max_sync(full, smax);
    if (smin > smax || smax - smin >= (unsigned)(kSymWbWords - 3)) {
      sym_warp_row<32, true>(tm, P, reinterpret_cast<int*>(bits), pre, qsv, logT, hs, g, rowsize);
      clean = false;
      fetch_j();
      continue;
    }
    const unsigned span = smax - smin + 1u;
    if (!clean) {
      uint4* c4 = reinterpret_cast<uint4*>(bits);
      for (int x = lane; x < kSymWbWords / 4; x += 32) c4[x] = make_uint4(0u, 0u, 0u, 0u);
      clean = true;
      __syncwarp();
    }
    int nb = 0;
    const bool one_chunk = a1 - a0 <= 32;
    const int mq = one_chunk ? (int)__reduce_max_sync(full, (unsigned)ql) : 0;
    const int tq = one_chunk ? (int)__reduce_add_sync(full, (unsigned)ql) : 0;
    if (one_chunk && mq * (int)(a1 - a0) <= 2 * tq) {
      // one chunk of compressed B rows of similar lengths: each lane ORs the
      // entries of its own B row (no search for a product's A entry); a lane
      // starts at offset lane mod ql of its row, so lanes whose B rows carry
      // nearly the same sets (neighbouring rows of a stencil) do not hit one
      // word in the same step.  Four entries' loads are issued together.
      const int rot = ql > 0 ? (int)((unsigned)lane % (unsigned)ql) : 0;
      for (int u0 = 0; u0 < mq; u0 += 4) {
        unsigned w[4], m[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int k = u0 + u;
          w[u] = 0xffffffffu;
          m[u] = 0u;
          if (k < ql) {
            int o = rot + k;
            if (o >= ql) o -= ql;
            w[u] = (unsigned)P.csi[qs + o] - smin;
            m[u] = P.cs[qs + o];
          }
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          if (w[u] < span) {
            const unsigned old = atomicOr(bits + w[u], m[u]);
            nb += __popc(m[u] & ~old);
            if (old == 0u && m[u] != 0u) atomicOr(summ + (w[u] >> 5), 1u << (w[u] & 31u));
          } else if (m[u] != 0u) {
            dev_fail(P.status, kDevBadIndex, 4, g);
          }
        }
      }
      __syncwarp();
    } else {
      for (long long c = a0; c < a1; c += 32) {
        if (!one_chunk) load_chunk(c);
        nb += wb_union_chunk<32, true>(full, lane, pre, qsv, qs, ql, P.csi, P.cs, bits, smin, span, P.status, 4, g,
                                       summ);
      }
    }
    fetch_j();
    const unsigned cnt = __reduce_add_sync(full, (unsigned)nb);
    if (lane == 0) rowsize[g] = (long long)cnt;
    // the words that became nonzero, in increasing order: recorded as the
    // row's column sets (set index, bits) for the numeric phase, then cleared
    const unsigned f0 = summ[2 * lane], f1 = summ[2 * lane + 1];
    const int nf = __popc(f0) + __popc(f1);
    int incl = nf;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const int y = __shfl_up_sync(full, incl, d);
      if (lane >= d) incl += y;
    }
    const int nw = __shfl_sync(full, incl, 31);
    int2* dst = (record && nw <= kRowSetCap) ? P.rsets + g * kRowSetCap : nullptr;
    int at = incl - nf;
#pragma unroll
    for (int hh = 0; hh < 2; ++hh) {
      unsigned f = hh ? f1 : f0;
      while (f) {
        const int wd = 64 * lane + 32 * hh + __ffs(f) - 1;
        f &= f - 1u;
        if (dst != nullptr) dst[at] = make_int2((int)smin + wd, (int)bits[wd]);
        bits[wd] = 0u;
        ++at;
      }
    }
    summ[2 * lane] = 0u;
    summ[2 * lane + 1] = 0u;
    if (record && lane == 0) P.rcnt[g] = nw <= kRowSetCap ? nw : -1;
    __syncwarp();
  }
}

// One thread per row for rows with at most kT1SymKeys products
// (Thread-Sequential with a team of one, Section 3.1.1): the row's distinct
// keys (and, compressed, their column sets) go to a short list in the
// thread's own column of shared memory, searched linearly.  Whole bins of
// short rows are in flight at once, which hides their chains of dependent
// loads; the loads of 4 entries of A(i,:) and of 4 keys at a time are issued
// together.
constexpr int kSymThreads = 128;

template <bool COMP>
__global__ void __launch_bounds__(kSymThreads) k_sym_thread(ProbD P, const int* __restrict__ rows, long long nrows,
                                                            long long* __restrict__ rowsize) {
  __shared__ int lk[kT1SymKeys][kSymThreads];
  __shared__ unsigned lm[COMP ? kT1SymKeys : 1][kSymThreads];
  const int tid = threadIdx.x;
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long r = (long long)blockIdx.x * blockDim.x + tid; r < nrows; r += stride) {
    const long long g = rows[r];
    const int b = inst_of(P.arow0s, P.ninst, g);
    const InstD& I = P.inst[b];
    const long long i = g - I.arow0;
    const long long a0 = rp_at(I.A, i), a1 = rp_at(I.A, i + 1);
    const long long brow0 = I.brow0;
    const int* __restrict__ ksrc = COMP ? P.csi : I.B.cj;
    int n = 0;
    bool over = false;
    auto add = [&](int key, unsigned m) {
      int t = 0;
      while (t < n && lk[t][tid] != key) ++t;
      if (t < n) {
        if (COMP) lm[t][tid] |= m;
      } else if (n < kT1SymKeys) {
        lk[n][tid] = key;
        if (COMP) lm[n][tid] = m;
        ++n;
      } else {
        over = true;
      }
    };
    constexpr int kX = 4, kQ = 4;
    for (long long c = a0; c < a1; c += kX) {
      long long qs[kX], qe[kX];
#pragma unroll
      for (int u = 0; u < kX; ++u) {
        const int j = c + u < a1 ? I.A.cj[c + u] : -1;
        qs[u] = 0;
        qe[u] = 0;
        if (j >= 0) {
          if (COMP) {
            qs[u] = P.Bcp[brow0 + j];
            qe[u] = P.Bcp[brow0 + j + 1];
          } else {
            qs[u] = rp_at(I.B, j);
            qe[u] = rp_at(I.B, j + 1);
          }
        }
      }
#pragma unroll
      for (int u = 0; u < kX; ++u) {
        for (long long q = qs[u]; q < qe[u]; q += kQ) {
          int kk[kQ];
          unsigned mm[kQ];
#pragma unroll
          for (int v = 0; v < kQ; ++v) {
            const bool ok = q + v < qe[u];
            kk[v] = ok ? ksrc[q + v] : -1;
            mm[v] = (COMP && ok) ? P.cs[q + v] : 0u;
          }
#pragma unroll
          for (int v = 0; v < kQ; ++v)
            if (kk[v] >= 0) add(kk[v], mm[v]);
        }
      }
    }
    if (over) dev_fail(P.status, kDevTableFull, 3, g);
    long long cnt = n;
    if (COMP) {
      cnt = 0;
      for (int t = 0; t < n; ++t) cnt += __popc(lm[t][tid]);
    }
    rowsize[g] = cnt;
  }
}

template <int TW, bool COMP>
__global__ void __launch_bounds__(TW) k_sym_dense(ProbD P, const int* __restrict__ rows, long long nrows,
                                                  long long kw_max, long long* __restrict__ rowsize,
                                                  unsigned long long* fetch) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ long long scan_scratch[33];
  __shared__ long long fetch_s;
  Team<TW> tm;
  unsigned* bm = reinterpret_cast<unsigned*>(smem);
  ChunkScratch<TW, int>* csc = reinterpret_cast<ChunkScratch<TW, int>*>(smem + al16((size_t)kw_max * 4));
  // products find their A entry through a segment map
  int* seg = reinterpret_cast<int*>(reinterpret_cast<unsigned char*>(csc) + al16(sizeof(ChunkScratch<TW, int>)));
  for (long long w = tm.lane; w < kw_max; w += TW) bm[w] = 0u;
  for (long long r = cta_next_row(fetch, &fetch_s); r < nrows; r = cta_next_row(fetch, &fetch_s)) {
    const long long g = rows[r];
    const int b = inst_of(P.arow0s, P.ninst, g);
    const InstD& I = P.inst[b];
    const long long i = g - I.arow0;
    const long long k = I.k;
    const long long kw = (k + 31) >> 5;
    const long long a0 = rp_at(I.A, i), a1 = rp_at(I.A, i + 1);
    const long long brow0 = I.brow0;
    auto range = [&](int j, long long* bs, long long* be) {
      if (COMP) {
        *bs = P.Bcp[brow0 + j];
        *be = P.Bcp[brow0 + j + 1];
      } else {
        *bs = rp_at(I.B, j);
        *be = rp_at(I.B, j + 1);
      }
    };
    auto aval = [&](long long) { return 0; };
    const int* __restrict__ Bj = I.B.cj;
    auto body = [&](long long q, int) {
      if (COMP) {
        const int w = P.csi[q];
        if ((unsigned)w < (unsigned)kw) atomicOr(bm + w, P.cs[q]);
        else dev_fail(P.status, kDevBadIndex, 3, g);
      } else {
        const int col = Bj[q];
        if ((unsigned)col < (unsigned long long)k) atomicOr(bm + (col >> 5), 1u << (col & 31));
        else dev_fail(P.status, kDevBadIndex, 4, g);
      }
    };
    auto pf = [&](long long q) {
      if (COMP) {
        prefetch_l1(P.csi + q);
        prefetch_l1(P.cs + q);
      } else {
        prefetch_l1(Bj + q);
      }
    };
    for_each_product<TW, int>(tm, csc, scan_scratch, I.A.cj, a0, a1, range, aval, body, pf, seg);
    long long c = 0;
    for (long long w = tm.lane; w < kw; w += TW) {
      c += __popc(bm[w]);
      bm[w] = 0u;
    }
    c = team_sum<TW>(tm, c, scan_scratch);
    if (tm.lane == 0) rowsize[g] = c;
    __syncthreads();
  }
}

// Dense rows by warp teams: each warp ORs the products of its row into its
// own bitmap of kw_cap words (the dense accumulator of Section 3.1.2 in bit
// form, one per warp instead of one per CTA, so many rows are in flight on
// an SM and no block-wide barrier separates them).  The row size is the number
// of column bits the inserts set first, so no sweep of the bitmap counts the
// row; every word an insert turns nonzero is flagged in a summary bitmap and
// the flagged words alone are cleared after the row.  Rows of one bin have
// bitmaps of at most kw_cap words (the bin is the bitmap size class).
// Products: when the chunk's B rows (compressed rows on the compressed B) have
// similar lengths each lane ORs its own row's entries, U loads in flight,
// from a rotated start (neighbouring rows of a stencil carry nearly equal
// columns); otherwise the chunk's products are spread flat over the lanes.
__host__ __device__ inline size_t symdw_team_bytes(long long kw_cap) {
  return al16((size_t)kw_cap * 4) + al16((size_t)((kw_cap + 31) / 32) * 4) + al16((size_t)33 * 4) +
         al16((size_t)32 * 8);
}

template <bool COMP, int U>
__global__ void __launch_bounds__(256) k_sym_dwarp(ProbD P, const int* __restrict__ rows, long long nrows,
                                                   long long kw_cap, long long* __restrict__ rowsize) {
  extern __shared__ __align__(16) unsigned char smem[];
  Team<32> tm;
  const long long nsum = (kw_cap + 31) / 32;
  unsigned char* base = smem + (size_t)tm.id * symdw_team_bytes(kw_cap);
  unsigned* bits = reinterpret_cast<unsigned*>(base);
  unsigned* summ = reinterpret_cast<unsigned*>(base + al16((size_t)kw_cap * 4));
  int* pre = reinterpret_cast<int*>(base + al16((size_t)kw_cap * 4) + al16((size_t)nsum * 4));
  long long* qsv = reinterpret_cast<long long*>(reinterpret_cast<unsigned char*>(pre) + al16((size_t)33 * 4));
  const int lane = tm.lane;
  const unsigned full = 0xffffffffu;
  for (long long w = lane; w < kw_cap; w += 32) bits[w] = 0u;
  for (long long w = lane; w < nsum; w += 32) summ[w] = 0u;
  __syncwarp();
  const long long team = (long long)blockIdx.x * tm.per_cta + tm.id;
  const long long nteams = (long long)gridDim.x * tm.per_cta;
  for (long long r = team; r < nrows; r += nteams) {
    const long long g = rows[r];
    const int b = inst_of(P.arow0s, P.ninst, g);
    const InstD& I = P.inst[b];
    const long long i = g - I.arow0;
    const long long kw = (I.k + 31) >> 5;
    const long long a0 = rp_at(I.A, i), a1 = rp_at(I.A, i + 1);
    if (kw > kw_cap) {   // binning keeps every row of the bin within kw_cap
      if (lane == 0) dev_fail(P.status, kDevTableFull, 5, g);
      continue;
    }
    const unsigned span = (unsigned)kw;
    const int* __restrict__ Bj = I.B.cj;
    // word and bits of entry q of the (compressed) B
    auto entry = [&](long long q, unsigned* w, unsigned* m) {
      if (COMP) {
        *w = (unsigned)P.csi[q];
        *m = P.cs[q];
      } else {
        const int col = Bj[q];
        *w = (unsigned)col >> 5;
        *m = 1u << (col & 31);
      }
    };
    auto insert = [&](unsigned w, unsigned m) -> int {
      if (w < span) {
        const unsigned old = atomicOr(bits + w, m);
        if (old == 0u && m != 0u) atomicOr(summ + (w >> 5), 1u << (w & 31u));
        return __popc(m & ~old);
      }
      if (m != 0u) dev_fail(P.status, kDevBadIndex, COMP ? 3 : 4, g);
      return 0;
    };
    int nb = 0;
    for (long long c = a0; c < a1; c += 32) {
      const long long p = c + lane;
      long long qs = 0;
      int ql = 0;
      if (p < a1) {
        const int j = I.A.cj[p];
        if (COMP) {
          qs = P.Bcp[I.brow0 + j];
          ql = (int)(P.Bcp[I.brow0 + j + 1] - qs);
        } else {
          qs = rp_at(I.B, j);
          ql = (int)(rp_at(I.B, j + 1) - qs);
        }
      }
      const int nc = (a1 - c) < 32 ? (int)(a1 - c) : 32;
      const int mq = (int)__reduce_max_sync(full, (unsigned)ql);
      const int tq = (int)__reduce_add_sync(full, (unsigned)ql);
      if ((long long)mq * nc <= 2ll * tq) {
        const int rot = ql > 0 ? (int)((unsigned)lane % (unsigned)ql) : 0;
        for (int u0 = 0; u0 < mq; u0 += U) {
          unsigned w[U], m[U];
#pragma unroll
          for (int u = 0; u < U; ++u) {
            const int kq = u0 + u;
            w[u] = 0xffffffffu;
            m[u] = 0u;
            if (kq < ql) {
              int o = rot + kq;
              if (o >= ql) o -= ql;
              entry(qs + o, &w[u], &m[u]);
            }
          }
#pragma unroll
          for (int u = 0; u < U; ++u) nb += insert(w[u], m[u]);
        }
      } else {
        int ex = ql;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
          const int y = __shfl_up_sync(full, ex, d);
          if (lane >= d) ex += y;
        }
        pre[lane] = ex - ql;
        qsv[lane] = qs;
        if (lane == 31) pre[32] = ex;
        __syncwarp();
        int t = 0;
        for (int xb = 0; xb < tq; xb += U * 32) {
          unsigned w[U], m[U];
#pragma unroll
          for (int u = 0; u < U; ++u) {
            const int x = xb + u * 32 + lane;
            w[u] = 0xffffffffu;
            m[u] = 0u;
            if (x < tq) {
              while (pre[t + 1] <= x) ++t;
              entry(qsv[t] + (x - pre[t]), &w[u], &m[u]);
            }
          }
#pragma unroll
          for (int u = 0; u < U; ++u) nb += insert(w[u], m[u]);
        }
      }
      __syncwarp();
    }
    const unsigned cnt = __reduce_add_sync(full, (unsigned)nb);
    if (lane == 0) rowsize[g] = (long long)cnt;
    // clear the words that became nonzero
    for (long long x = lane; x < (kw + 31) / 32; x += 32) {
      unsigned f = summ[x];
      if (f) {
        summ[x] = 0u;
        while (f) {
          bits[32 * x + __ffs(f) - 1] = 0u;
          f &= f - 1u;
        }
      }
    }
    __syncwarp();
  }
}

template <class K>
cudaError_t set_smem(K kernel, size_t bytes) {
  // the kernels also hold up to 1 KB of static shared memory: opt in above 47 KB of dynamic
  if (bytes + 1024 > 48 * 1024) return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  return cudaSuccess;
}

template <int TW, bool COMP>
cudaError_t run_hash(const LaunchCtx& L, const ProbD& P, const SymLaunch& S, long long* rowsize) {
  const int T = 1 << S.logT;
  const size_t tb = sym_team_bytes<TW, COMP>(T);
  int teams = 1;
  if (TW <= 32) {
    teams = (int)(kTeamSmemBudget / tb);
    int tmax = 256 / TW;
    if (teams > tmax) teams = tmax;
    if (teams < 1) teams = 1;
  }
  const size_t smem = tb * teams;
  if (smem > (size_t)L.max_smem_optin) return cudaErrorInvalidConfiguration;
  auto kern = k_sym_hash<TW, COMP, false>;
  cudaError_t e = set_smem(kern, smem);
  if (e != cudaSuccess) return e;
  e = cudaMemsetAsync(S.fetch, 0, sizeof(unsigned long long), L.stream);
  if (e != cudaSuccess) return e;
  KKS_LAUNCHED();
  kern<<<resident_grid(kern, TW * teams, smem, L.num_sms, (S.nrows + teams - 1) / teams), TW * teams, smem,
         L.stream>>>(P, S.rows, S.nrows, S.logT, -1, nullptr, 0, rowsize, S.fetch);
  return cudaGetLastError();
}

template <int TW, bool COMP>
cudaError_t run_warp(const LaunchCtx& L, const ProbD& P, const SymLaunch& S, long long* rowsize) {
  const int T = 1 << S.logT;
  const size_t tb = symw_team_bytes<TW, COMP>(T);
  int teams = (int)(kTeamSmemBudget / tb);
  const int tmax = 256 / TW;
  if (teams > tmax) teams = tmax;
  if (teams < 1) teams = 1;
  const size_t smem = tb * teams;
  if (smem > (size_t)L.max_smem_optin) return cudaErrorInvalidConfiguration;
  auto kern = k_sym_warp<TW, COMP>;
  cudaError_t e = set_smem(kern, smem);
  if (e != cudaSuccess) return e;
  KKS_LAUNCHED();
  kern<<<resident_grid(kern, TW * teams, smem, L.num_sms, (S.nrows + teams - 1) / teams), TW * teams, smem,
         L.stream>>>(P, S.rows, S.nrows, S.logT, rowsize);
  return cudaGetLastError();
}

cudaError_t run_wb(const LaunchCtx& L, const ProbD& P, const SymLaunch& S, long long* rowsize) {
  const size_t tb = symwb_team_bytes(1 << S.logT);
  const int teams = 8;
  const size_t smem = tb * teams;
  if (smem > (size_t)L.max_smem_optin) return cudaErrorInvalidConfiguration;
  auto kern = k_sym_wb;
  cudaError_t e = set_smem(kern, smem);
  if (e != cudaSuccess) return e;
  KKS_LAUNCHED();
  kern<<<resident_grid(kern, 32 * teams, smem, L.num_sms, (S.nrows + teams - 1) / teams), 32 * teams, smem,
         L.stream>>>(P, S.rows, S.nrows, S.logT, rowsize, S.merge);
  return cudaGetLastError();
}

template <bool COMP>
cudaError_t run_thread(const LaunchCtx& L, const ProbD& P, const SymLaunch& S, long long* rowsize) {
  auto kern = k_sym_thread<COMP>;
  KKS_LAUNCHED();
  kern<<<resident_grid(kern, kSymThreads, 0, L.num_sms, (S.nrows + kSymThreads - 1) / kSymThreads), kSymThreads, 0,
         L.stream>>>(P, S.rows, S.nrows, rowsize);
  return cudaGetLastError();
}

template <bool COMP>
cudaError_t run_spill(const LaunchCtx& L, const ProbD& P, const SymLaunch& S, long long* rowsize) {
  constexpr int TW = 1024;
  const int T = 1 << S.l1_logT;
  const size_t smem = sym_team_bytes<TW, COMP>(T);
  if (smem > (size_t)L.max_smem_optin) return cudaErrorInvalidConfiguration;
  auto kern = k_sym_hash<TW, COMP, true>;
  cudaError_t e = set_smem(kern, smem);
  if (e != cudaSuccess) return e;
  int cap = (int)(S.max_occ * T);
  if (cap < 1) cap = 1;
  if (cap > T - 1) cap = T - 1;
  int grid = S.nchunks;
  if (grid > S.nrows) grid = (int)S.nrows;
  e = cudaMemsetAsync(S.fetch, 0, sizeof(unsigned long long), L.stream);
  if (e != cudaSuccess) return e;
  KKS_LAUNCHED();
  kern<<<grid, TW, smem, L.stream>>>(P, S.rows, S.nrows, S.l1_logT, cap, (int*)S.l2_pool, S.l2_chunk_slots,
                                     rowsize, S.fetch);
  return cudaGetLastError();
}

template <bool COMP>
cudaError_t run_dwarp(const LaunchCtx& L, const ProbD& P, const SymLaunch& S, long long* rowsize) {
  long long kw_cap = 1ll << S.logT;
  if (kw_cap > S.kwords_max && S.kwords_max > 0) kw_cap = S.kwords_max;
  const size_t tb = symdw_team_bytes(kw_cap);
  // up to 8 warp teams per CTA, within about 200 KB of shared memory
  int teams = (int)((size_t)(200 * 1024) / tb);
  if (teams > 8) teams = 8;
  if (teams < 1) teams = 1;
  const size_t smem = tb * teams;
  if (smem > (size_t)L.max_smem_optin) return cudaErrorInvalidConfiguration;
  auto kern = k_sym_dwarp<COMP, 4>;
  cudaError_t e = set_smem(kern, smem);
  if (e != cudaSuccess) return e;
  KKS_LAUNCHED();
  kern<<<resident_grid(kern, 32 * teams, smem, L.num_sms, (S.nrows + teams - 1) / teams), 32 * teams, smem,
         L.stream>>>(P, S.rows, S.nrows, kw_cap, rowsize);
  return cudaGetLastError();
}

template <bool COMP>
cudaError_t run_dense(const LaunchCtx& L, const ProbD& P, const SymLaunch& S, long long* rowsize) {
  if (S.logT > 0) return run_dwarp<COMP>(L, P, S, rowsize);
  constexpr int TW = 512;
  const size_t smem = al16((size_t)S.kwords_max * 4) + al16(sizeof(ChunkScratch<TW, int>)) +
                      al16((size_t)kStagedPasses * TW * 4);
  if (smem > (size_t)L.max_smem_optin) return cudaErrorInvalidConfiguration;
  auto kern = k_sym_dense<TW, COMP>;
  cudaError_t e = set_smem(kern, smem);
  if (e != cudaSuccess) return e;
  int per_sm = (int)((size_t)L.max_smem_optin / (smem + 1024));
  if (per_sm < 1) per_sm = 1;
  if (per_sm > 4) per_sm = 4;
  long long grid = (long long)L.num_sms * per_sm;
  if (grid > S.nrows) grid = S.nrows;
  e = cudaMemsetAsync(S.fetch, 0, sizeof(unsigned long long), L.stream);
  if (e != cudaSuccess) return e;
  KKS_LAUNCHED();
  kern<<<(unsigned)grid, TW, smem, L.stream>>>(P, S.rows, S.nrows, S.kwords_max, rowsize, S.fetch);
  return cudaGetLastError();
}

template <bool COMP>
cudaError_t dispatch(const LaunchCtx& L, const ProbD& P, const SymLaunch& S, long long* rowsize) {
  switch (S.cls) {
    case kClsT1: return run_thread<COMP>(L, P, S, rowsize);
    case kClsW8: return run_warp<8, COMP>(L, P, S, rowsize);
    case kClsW32: return (COMP && S.window) ? run_wb(L, P, S, rowsize) : run_warp<32, COMP>(L, P, S, rowsize);
    case kClsC256: return run_hash<256, COMP>(L, P, S, rowsize);
    case kClsC1024: return run_hash<1024, COMP>(L, P, S, rowsize);
    case kClsDense: return run_dense<COMP>(L, P, S, rowsize);
    case kClsSpill: return run_spill<COMP>(L, P, S, rowsize);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace

size_t symbolic_team_bytes(int cls, int logT, int compressed) {
  const int T = 1 << logT;
  switch (cls) {
    case kClsW8: return compressed ? sym_team_bytes<8, true>(T) : sym_team_bytes<8, false>(T);
    case kClsW32: return compressed ? sym_team_bytes<32, true>(T) : sym_team_bytes<32, false>(T);
    case kClsC256: return compressed ? sym_team_bytes<256, true>(T) : sym_team_bytes<256, false>(T);
    default: return compressed ? sym_team_bytes<1024, true>(T) : sym_team_bytes<1024, false>(T);
  }
}

cudaError_t launch_symbolic(const LaunchCtx& L, const ProbD& P, const SymLaunch& S, long long* rowsize) {
  if (S.nrows <= 0) return cudaSuccess;
  return S.compressed ? dispatch<true>(L, P, S, rowsize) : dispatch<false>(L, P, S, rowsize);
}

}  // namespace kks
