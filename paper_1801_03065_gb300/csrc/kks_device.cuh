// kks_device.cuh -- device-side building blocks shared by the SpGEMM kernels.
//
// Teams (the paper's Kokkos "team", Section 2.3 / 3.1.1) are groups of TW
// threads that compute one row of C at a time:
//   * TW <= 32  : a sub-warp or a warp; several teams per CTA, synchronised
//                 with __syncwarp(mask)
//   * TW  > 32  : the whole CTA is one team (TW == blockDim.x), synchronised
//                 with __syncthreads()
// Inside a team the products of a row are flattened and spread over the
// threads (Thread-Flat-Parallel partitioning, Section 3.1.1), so inserts into
// an accumulator are not unique and use atomics.
//
// Accumulators are linear-probing hash tables (LP, Section 3.1.2) addressed
// through generic pointers, so the same code serves the level-1 table in
// shared memory and the level-2 table in a global-memory pool chunk.  Table
// sizes are powers of two; the slot of a key is the paper's key & (size - 1)
// (Section 3.1.2) with option hash_function = 0, and by default (1) the top
// log2(size) bits of key * 2654435761 (multiplicative hashing, see LpHash).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace kks {

constexpr int kEmpty = -1;

// Device status word: kernels never trap; they record the first problem here
// and the host turns it into a status code at the next synchronisation point.
enum DevCode : int {
  kDevOk = 0,
  kDevTableFull = 1,        // an accumulator had no free slot (internal sizing bug)
  kDevRowSizeMismatch = 2,  // numeric produced a row size != symbolic's
  kDevBadIndex = 3,         // a column index outside [0, k)
  kDevSortOverflow = 4,     // a row larger than its sort buffer
  kDevRowTooLarge = 5,      // a row whose table fits no team's shared memory
};

struct DevStatus {
  int code;
  int where;
  long long info;
};

__device__ __forceinline__ void dev_fail(DevStatus* st, int code, int where, long long info) {
  if (atomicCAS(&st->code, 0, code) == 0) {
    st->where = where;
    st->info = info;
  }
}

// CSR operand with int32 or int64 row pointers.
struct MatD {
  const void* rp;
  const int* cj;
  const void* vx;
  long long nrows, ncols, nnz;
  int rp64;
  int pad;
};

__device__ __forceinline__ long long rp_at(const MatD& M, long long i) {
  return M.rp64 ? reinterpret_cast<const long long*>(M.rp)[i]
                : (long long)reinterpret_cast<const int*>(M.rp)[i];
}

// One multiplication C = A * B of a plan (a plain call is a plan of one).
struct InstD {
  MatD A, B;
  long long arow0;     // first global row of this instance's A rows
  long long brow0;     // first global row of this instance's B rows
  long long* Crp;      // caller's C row pointers (m + 1)
  int* Cj;             // caller's C column indices
  void* Cx;            // caller's C values
  long long k;         // columns of B (= of C)
  int compressed;      // symbolic runs on the compressed B
  int pad;
};

// Per-launch view of a plan.
// Column sets of the rows of C, left by the symbolic phase for the numeric
// phase: row g's sets (index, bits; in increasing index order) at rsets[g *
// kRowSetCap ...], their number at rcnt[g], or -1 where the symbolic kernel
// of that row did not record them (then the numeric phase forms the union).
constexpr int kRowSetCap = 64;

struct ProbD {
  const InstD* inst;
  const long long* arow0s;   // ninst + 1 prefix of A-row counts
  const long long* brow0s;   // ninst + 1 prefix of B-row counts
  const long long* Bcp;      // compressed B row pointers over global B rows (+1)
  const int* csi;            // column-set index (col >> 5)
  const unsigned* cs;        // column set bits
  DevStatus* status;
  int2* rsets;               // nullptr: no column sets recorded
  int* rcnt;
  int ninst;
  int hash_mode;             // LpHash mode of every table of the plan
};

// Largest b with row0s[b] <= g; such an instance is never empty.
__device__ __forceinline__ int inst_of(const long long* row0s, int ninst, long long g) {
  int lo = 0, hi = ninst - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (row0s[mid] <= g) lo = mid; else hi = mid - 1;
  }
  return lo;
}

__host__ __device__ __forceinline__ int ilog2_ceil(long long x) {
  int l = 0;
  while ((1ll << l) < x) ++l;
  return l;
}

// --------------------------------------------------------------------------
// team primitives
// --------------------------------------------------------------------------
template <int TW>
struct Team {
  static constexpr bool kCta = TW > 32;
  unsigned mask;   // sub-warp teams: the team's lanes
  int lane;        // 0 .. TW-1
  int id;          // team index inside the CTA
  int per_cta;     // teams per CTA

  __device__ __forceinline__ Team() {
    if constexpr (kCta) {
      mask = 0xffffffffu;
      lane = threadIdx.x;
      id = 0;
      per_cta = 1;
    } else {
      int l = threadIdx.x & 31;
      lane = l & (TW - 1);
      if constexpr (TW == 32) mask = 0xffffffffu;
      else mask = ((1u << TW) - 1u) << (l & ~(TW - 1));
      id = threadIdx.x / TW;
      per_cta = blockDim.x / TW;
    }
  }
  __device__ __forceinline__ void sync() const {
    if constexpr (kCta) __syncthreads(); else __syncwarp(mask);
  }
};

// Exclusive prefix sum over the team; *total receives the team sum.
// scratch: 33 long longs of shared memory, used by CTA teams only.
template <int TW>
__device__ __forceinline__ long long team_excl_scan(const Team<TW>& tm, long long v, long long* total,
                                                    long long* scratch) {
  if constexpr (!Team<TW>::kCta) {
    long long x = v;
#pragma unroll
    for (int d = 1; d < TW; d <<= 1) {
      long long y = __shfl_up_sync(tm.mask, x, d, TW);
      if (tm.lane >= d) x += y;
    }
    *total = __shfl_sync(tm.mask, x, TW - 1, TW);
    return x - v;
  } else {
    const int l = threadIdx.x & 31, w = threadIdx.x >> 5, nw = TW / 32;
    long long x = v;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      long long y = __shfl_up_sync(0xffffffffu, x, d);
      if (l >= d) x += y;
    }
    if (l == 31) scratch[w] = x;
    __syncthreads();
    if (w == 0) {
      long long s = (l < nw) ? scratch[l] : 0;
#pragma unroll
      for (int d = 1; d < 32; d <<= 1) {
        long long y = __shfl_up_sync(0xffffffffu, s, d);
        if (l >= d) s += y;
      }
      if (l < nw) scratch[l] = s;          // inclusive warp prefix
      if (l == 31) scratch[32] = s;        // team total
    }
    __syncthreads();
    long long base = (w > 0) ? scratch[w - 1] : 0;
    *total = scratch[32];
    long long r = base + x - v;
    __syncthreads();                       // scratch reusable after return
    return r;
  }
}

template <int TW>
__device__ __forceinline__ long long team_sum(const Team<TW>& tm, long long v, long long* scratch) {
  long long tot;
  team_excl_scan<TW>(tm, v, &tot, scratch);
  return tot;
}

// Sum over a warp or sub-warp team (register shuffles only).
template <int TW>
__device__ __forceinline__ long long warp_team_sum(const Team<TW>& tm, long long v) {
#pragma unroll
  for (int d = TW / 2; d > 0; d >>= 1) v += __shfl_xor_sync(tm.mask, v, d, TW);
  return v;
}

// acc + a * b with one rounding (fused multiply-add)
__device__ __forceinline__ double fma_acc(double a, double b, double acc) { return fma(a, b, acc); }
__device__ __forceinline__ float fma_acc(float a, float b, float acc) { return fmaf(a, b, acc); }

// --------------------------------------------------------------------------
// linear-probing hash table (LP accumulator, Section 3.1.2)
// --------------------------------------------------------------------------
// Slot of a key in a table of 2^logT slots.  Mode 0 is the paper's BitwiseAnd
// of the key with size - 1 (Section 3.1.2).  Mode 1 takes the top logT bits of
// key * 2654435761 (Fibonacci hashing): stencil rows hold runs of consecutive
// columns spaced by the grid strides, which BitwiseAnd packs into long linear
// probing clusters.
struct LpHash {
  unsigned mask;
  int shift;
  int mode;
  __device__ __forceinline__ LpHash(int logT, int mode_)
      : mask((1u << logT) - 1u), shift(32 - logT), mode(logT > 0 ? mode_ : 0) {}
  __device__ __forceinline__ unsigned operator()(int key) const {
    return mode ? (((unsigned)key * 2654435761u) >> shift) : ((unsigned)key & mask);
  }
};

// Find or claim the slot of key.  cap < 0: no occupancy limit.  Otherwise a new
// key is only placed while *occ < cap (the maximum-occupancy rule of the LP
// accumulator); a refused key returns -1 and goes to the next level.
// Returns -2 when the table has no free slot at all.
__device__ __forceinline__ int lp_insert(int* keys, const LpHash& hs, int* occ, int cap, int key) {
  const unsigned tmask = hs.mask;
  unsigned h = hs(key);
  for (unsigned probe = 0; probe <= tmask; ++probe) {
    int cur = *((volatile int*)(keys + h));
    if (cur == key) return (int)h;
    if (cur == kEmpty) {
      if (cap >= 0 && *((volatile int*)occ) >= cap) return -1;
      int old = atomicCAS(keys + h, kEmpty, key);
      if (old == kEmpty) {
        if (cap >= 0) atomicAdd(occ, 1);
        return (int)h;
      }
      if (old == key) return (int)h;
    }
    h = (h + 1) & tmask;
  }
  return -2;
}

// Team-wide insert of one key per active lane (keys of one call pairwise
// distinct or equal keys resolved by the CAS).  The probe loop runs while any
// lane of the team is unresolved, so its trip count is uniform and the body is
// a short predicated step: lanes with short probe chains do not diverge from
// the team.  Returns the slot, -1 for inactive lanes, -2 if the table is full.
__device__ __forceinline__ int lp_insert_team(unsigned team_mask, int* keys, const LpHash& hs, bool active,
                                              int key) {
  unsigned h = active ? hs(key) : 0u;
  bool pending = active;
  int slot = -1;
  unsigned probes = 0;
  while (__any_sync(team_mask, pending)) {
    if (pending) {
      const int cur = *((volatile int*)(keys + h));
      bool claim = cur == key;
      if (cur == kEmpty) {
        const int old = atomicCAS(keys + h, kEmpty, key);
        claim = (old == kEmpty || old == key);
      }
      if (claim) {
        slot = (int)h;
        pending = false;
      } else if (++probes > hs.mask) {
        slot = -2;
        pending = false;
      } else {
        h = (h + 1) & hs.mask;
      }
    }
  }
  return slot;
}

// Probe-only lookup; -1 when absent.  Valid once no insert is in flight.
__device__ __forceinline__ int lp_find(const int* keys, const LpHash& hs, int key) {
  const unsigned tmask = hs.mask;
  unsigned h = hs(key);
  for (unsigned probe = 0; probe <= tmask; ++probe) {
    int cur = *((const volatile int*)(keys + h));
    if (cur == key) return (int)h;
    if (cur == kEmpty) return -1;
    h = (h + 1) & tmask;
  }
  return -1;
}

// --------------------------------------------------------------------------
// Union of keys over one chunk of A(i,:) for warp teams (Algorithm 3's insert
// loop).  Lane t holds the range [qs, qs + ql) of keys of the B row of its
// entry of the chunk.  Every key goes into an LP table whose slots are STRIDE
// words with the key first; with BITS the key's 32-bit column set (Section
// 3.2) is ORed into the slot's second word.  Products are spread flat over the
// lanes, and the loads of kUnionPasses passes are issued before their inserts
// so that their latencies overlap.  pre holds TW + 1 ints, qsv TW offsets.
// Returns the number of slots this lane claimed, or with BITS the number of
// column bits this lane was first to set (their team sum is the row size).
// --------------------------------------------------------------------------
constexpr int kUnionPasses = 4;

template <int STRIDE>
__device__ __forceinline__ int slot_insert(int* words, const LpHash& hs, int key, int* fresh) {
  unsigned h = hs(key);
  for (unsigned probe = 0; probe <= hs.mask; ++probe) {
    const int cur = *((volatile int*)(words + STRIDE * h));
    if (cur == key) return (int)h;
    if (cur == kEmpty) {
      const int old = atomicCAS(words + STRIDE * h, kEmpty, key);
      if (old == kEmpty) {
        ++*fresh;
        return (int)h;
      }
      if (old == key) return (int)h;
    }
    h = (h + 1) & hs.mask;
  }
  return -2;
}

template <int TW, int STRIDE, bool BITS>
__device__ __forceinline__ int union_chunk(unsigned team_mask, int lane, int* pre, long long* qsv, long long qs,
                                           int ql, const int* __restrict__ ksrc, const unsigned* __restrict__ bsrc,
                                           int* words, const LpHash& hs, DevStatus* status, int code, long long g) {
  int ex = ql;
#pragma unroll
  for (int d = 1; d < TW; d <<= 1) {
    const int y = __shfl_up_sync(team_mask, ex, d, TW);
    if (lane >= d) ex += y;
  }
  const int tot = __shfl_sync(team_mask, ex, TW - 1, TW);
  pre[lane] = ex - ql;
  qsv[lane] = qs;
  if (lane == 0) pre[TW] = tot;
  __syncwarp(team_mask);
  int fresh = 0, nbits = 0;
  int t = 0;
  for (int xb = 0; xb < tot; xb += kUnionPasses * TW) {
    int key[kUnionPasses];
    unsigned m[kUnionPasses];
#pragma unroll
    for (int u = 0; u < kUnionPasses; ++u) {
      const int x = xb + u * TW + lane;
      key[u] = -1;
      m[u] = 0u;
      if (x < tot) {
        while (pre[t + 1] <= x) ++t;
        const long long q = qsv[t] + (x - pre[t]);
        key[u] = ksrc[q];
        if (BITS) m[u] = bsrc[q];
      }
    }
#pragma unroll
    for (int u = 0; u < kUnionPasses; ++u) {
      if (key[u] >= 0) {
        const int slot = slot_insert<STRIDE>(words, hs, key[u], &fresh);
        if (slot >= 0) {
          if (BITS) {
            const unsigned old = atomicOr(reinterpret_cast<unsigned*>(words + STRIDE * slot + 1), m[u]);
            nbits += __popc(m[u] & ~old);
          }
        } else {
          dev_fail(status, kDevTableFull, code, g);
        }
      }
    }
  }
  __syncwarp(team_mask);
  return BITS ? nbits : fresh;
}

// Union of compressed products into a bitmap window (direct addressing, no
// hashing): lane t holds the compressed range [qs, qs + ql) of the B row of its
// entry of the chunk; the set bits of every product go into bits[csi - smin]
// (a window of span words starting at set smin).  Products are spread flat
// over the lanes as in union_chunk.  With COUNT the return value is the number
// of column bits this lane was first to set (their team sum is the row size).
// With summ (COUNT only), every word that an insert turns from zero to nonzero
// is flagged in the summary bitmap: bit (w & 31) of summ[w >> 5].
template <int TW, bool COUNT>
__device__ __forceinline__ int wb_union_chunk(unsigned team_mask, int lane, int* pre, long long* qsv, long long qs,
                                              int ql, const int* __restrict__ csi, const unsigned* __restrict__ cs,
                                              unsigned* bits, unsigned smin, unsigned span, DevStatus* status,
                                              int code, long long g, unsigned* summ = nullptr) {
  int ex = ql;
#pragma unroll
  for (int d = 1; d < TW; d <<= 1) {
    const int y = __shfl_up_sync(team_mask, ex, d, TW);
    if (lane >= d) ex += y;
  }
  const int tot = __shfl_sync(team_mask, ex, TW - 1, TW);
  pre[lane] = ex - ql;
  qsv[lane] = qs;
  if (lane == 0) pre[TW] = tot;
  __syncwarp(team_mask);
  int nbits = 0;
  int t = 0;
  for (int xb = 0; xb < tot; xb += kUnionPasses * TW) {
    unsigned w[kUnionPasses];
    unsigned m[kUnionPasses];
#pragma unroll
    for (int u = 0; u < kUnionPasses; ++u) {
      const int x = xb + u * TW + lane;
      w[u] = 0xffffffffu;
      m[u] = 0u;
      if (x < tot) {
        while (pre[t + 1] <= x) ++t;
        const long long q = qsv[t] + (x - pre[t]);
        w[u] = (unsigned)csi[q] - smin;
        m[u] = cs[q];
      }
    }
#pragma unroll
    for (int u = 0; u < kUnionPasses; ++u) {
      if (w[u] < span) {
        if (COUNT) {
          const unsigned old = atomicOr(bits + w[u], m[u]);
          nbits += __popc(m[u] & ~old);
          if (summ != nullptr && old == 0u) atomicOr(summ + (w[u] >> 5), 1u << (w[u] & 31u));
        } else {
          atomicOr(bits + w[u], m[u]);
        }
      } else if (m[u] != 0u) {
        dev_fail(status, kDevBadIndex, code, g);
      }
    }
  }
  __syncwarp(team_mask);
  return nbits;
}

// Tables of 16-byte slots (column-set index, set bits, base, unused): the
// place of column c in a sorted row is base(c >> 5) + the number of set bits
// below bit c & 31.  Lookups once the table is complete.
__device__ __forceinline__ int4 set_find(const int4* tab, const LpHash& hs, int key) {
  unsigned h = hs(key);
  for (unsigned probe = 0; probe <= hs.mask; ++probe) {
    const int4 e = tab[h];
    if (e.x == key || e.x == kEmpty) return e;
    h = (h + 1) & hs.mask;
  }
  return make_int4(kEmpty, 0, 0, 0);
}

__device__ __forceinline__ int set_slot(const int4* tab, const LpHash& hs, int key) {
  unsigned h = hs(key);
  for (unsigned probe = 0; probe <= hs.mask; ++probe) {
    const int k = tab[h].x;
    if (k == key) return (int)h;
    if (k == kEmpty) return -1;
    h = (h + 1) & hs.mask;
  }
  return -1;
}

// Probe-only lookup over a plain key array once the table is complete (-1:
// absent); the sorted-pattern masked kernel keeps its (set bits, base) pairs
// beside the keys.
__device__ __forceinline__ int key_slot(const int* keys, const LpHash& hs, int key) {
  unsigned h = hs(key);
  for (unsigned probe = 0; probe <= hs.mask; ++probe) {
    const int k = keys[h];
    if (k == key) return (int)h;
    if (k == kEmpty) return -1;
    h = (h + 1) & hs.mask;
  }
  return -1;
}

// Ascending bitonic sort of one 32-bit key per lane of a team of TW lanes
// (register exchanges only).
template <int TW>
__device__ __forceinline__ unsigned team_sort1(unsigned team_mask, int lane, unsigned v) {
#pragma unroll
  for (int k = 2; k <= TW; k <<= 1) {
#pragma unroll
    for (int j = k >> 1; j > 0; j >>= 1) {
      const unsigned o = __shfl_xor_sync(team_mask, v, j, TW);
      const bool up = (lane & k) == 0;
      const bool lower = (lane & j) == 0;
      v = (lower == up) ? min(v, o) : max(v, o);
    }
  }
  return v;
}

// Ascending bitonic sort of 2 * TW keys, two per lane: v0 is element lane,
// v1 element lane + TW.
template <int TW>
__device__ __forceinline__ void team_sort2(unsigned team_mask, int lane, unsigned& v0, unsigned& v1) {
#pragma unroll
  for (int k = 2; k <= 2 * TW; k <<= 1) {
#pragma unroll
    for (int j = k >> 1; j > 0; j >>= 1) {
      if (j == TW) {
        const unsigned lo = min(v0, v1), hi = max(v0, v1);
        v0 = lo;
        v1 = hi;
      } else {
        const unsigned o0 = __shfl_xor_sync(team_mask, v0, j, TW);
        const unsigned o1 = __shfl_xor_sync(team_mask, v1, j, TW);
        const bool lower = (lane & j) == 0;
        const bool up0 = (lane & k) == 0;
        const bool up1 = ((lane + TW) & k) == 0;
        v0 = (lower == up0) ? min(v0, o0) : max(v0, o0);
        v1 = (lower == up1) ? min(v1, o1) : max(v1, o1);
      }
    }
  }
}

template <int TW, typename T>
__device__ __forceinline__ void team_fill_n(const Team<TW>& tm, T* p, long long n, T v) {
  for (long long x = tm.lane; x < n; x += TW) p[x] = v;
}

// Bitonic sort of buf[0, N) ascending, N a power of two (pads must hold ~0).
template <int TW>
__device__ __forceinline__ void team_bitonic(const Team<TW>& tm, unsigned long long* buf, int N) {
  for (int k = 2; k <= N; k <<= 1) {
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int idx = tm.lane; idx < (N >> 1); idx += TW) {
        int lo = ((idx & ~(j - 1)) << 1) | (idx & (j - 1));
        int hi = lo + j;
        bool asc = (lo & k) == 0;
        unsigned long long a = buf[lo], b = buf[hi];
        if ((a > b) == asc) {
          buf[lo] = b;
          buf[hi] = a;
        }
      }
      tm.sync();
    }
  }
}

// --------------------------------------------------------------------------
// flat traversal of a row's products (Thread-Flat-Parallel, Section 3.1.1)
// --------------------------------------------------------------------------
// Per-team shared scratch for one chunk of TW entries of A(i,:).
template <int TW, typename VT>
struct ChunkScratch {
  long long pre[TW + 1];   // exclusive prefix of B-row lengths
  long long bs[TW];        // B-row start of each entry
  VT av[TW];               // A values of the chunk (numeric only)
  long long nne;           // non-empty B ranges of the chunk (set by chunk_scan)
};

// Calls body(q, t) for every product of row i: q indexes B's entry, t the
// chunk slot holding the A entry.  range(j, &bs, &be) gives the B range of
// A column j; aval(p) the value of A entry p (or 0 when unused).  The entries
// of kStagedPasses passes are located first and handed to prefetch(q), which
// may pull their B data into L1, so the body's loads of a whole group are in
// flight together instead of one dependent miss per pass.
constexpr int kStagedPasses = 4;

__device__ __forceinline__ void prefetch_l1(const void* p) {
  asm volatile("prefetch.global.L1 [%0];" ::"l"(p));
}

// Rows of a bin for CTA teams, taken one at a time from a counter zeroed
// before the launch, so that a few heavy rows (skewed graphs) do not leave the
// CTAs that drew them by a fixed stride running long after the others.  Every
// call is a barrier of the CTA; the first call gives its first row.
__device__ __forceinline__ long long cta_next_row(unsigned long long* fetch, long long* slot) {
  __syncthreads();
  if (threadIdx.x == 0) *slot = (long long)atomicAdd(fetch, 1ull);
  __syncthreads();
  return *slot;
}

// Exclusive max-scan over a CTA team (int values, -1 before the first thread).
template <int TW>
__device__ __forceinline__ int team_excl_max(const Team<TW>& tm, int v, long long* scratch) {
  static_assert(Team<TW>::kCta, "CTA teams only");
  const int l = threadIdx.x & 31, w = threadIdx.x >> 5, nw = TW / 32;
  int x = v;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const int y = __shfl_up_sync(0xffffffffu, x, d);
    if (l >= d) x = max(x, y);
  }
  int within = __shfl_up_sync(0xffffffffu, x, 1);
  if (l == 0) within = -1;
  if (l == 31) scratch[w] = x;
  __syncthreads();
  if (w == 0) {
    int s = (l < nw) ? (int)scratch[l] : -1;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, s, d);
      if (l >= d) s = max(s, y);
    }
    if (l < nw) scratch[l] = s;
  }
  __syncthreads();
  const int before = w > 0 ? (int)scratch[w - 1] : -1;
  __syncthreads();
  return max(before, within);
}

// With seg (CTA teams, kStagedPasses * TW ints of shared memory) the A entry
// of each product is not searched for: per block of kStagedPasses * TW
// products, every non-empty B range marks where it starts and a forward fill
// (max-scan) gives every product its range, one shared load per product.
// This pays off when the chunk holds many short or empty B ranges (dense
// windows, short B rows), where the search below needs many steps; a chunk
// whose non-empty ranges average kSegMaxAvg products or more takes the search
// (a few linear steps per pass), which needs no barrier per block.
constexpr long long kSegMaxAvg = 128;
// One chunk of A(i,:): lane t holds the B range [bs, be) and the value av of
// its A entry.  Returns the chunk's product count (the same in every lane).
// The chunk's scan (the lane's first product ex, the chunk's product count
// total) and its entries in cs; chunk_products then calls the body.
template <int TW, typename VT>
__device__ __forceinline__ long long chunk_scan(const Team<TW>& tm, ChunkScratch<TW, VT>* cs, long long* scan_scratch,
                                                long long bs, long long be, VT av, long long* total) {
  // one scan carries the lengths (high bits) and the non-empty count (low 11 bits)
  long long tp;
  long long ex = team_excl_scan<TW>(tm, (be - bs) * 2048 + (be > bs ? 1 : 0), &tp, scan_scratch) >> 11;
  *total = tp >> 11;
  cs->pre[tm.lane] = ex;
  cs->bs[tm.lane] = bs;
  cs->av[tm.lane] = av;
  if (tm.lane == 0) {
    cs->pre[TW] = *total;
    cs->nne = tp & 2047;
  }
  tm.sync();
  return ex;
}

template <int TW, typename VT, class Body, class Prefetch>
__device__ __forceinline__ long long chunk_products(const Team<TW>& tm, ChunkScratch<TW, VT>* cs,
                                                    long long* scan_scratch, long long ex, long long total,
                                                    long long bs, long long be, Body body, Prefetch prefetch,
                                                    int* seg) {
  if constexpr (Team<TW>::kCta) {
    if (seg != nullptr && total < kSegMaxAvg * cs->nne) {
      constexpr int E = kStagedPasses;
      constexpr long long S = (long long)kStagedPasses * TW;
      int carry = -1;
      for (long long x0 = 0; x0 < total; x0 += S) {
#pragma unroll
        for (int e = 0; e < E; ++e) seg[tm.lane * E + e] = -1;
        tm.sync();
        if (be > bs && ex >= x0 && ex < x0 + S) seg[ex - x0] = tm.lane;
        tm.sync();
        int v[E];
        int m = -1;
#pragma unroll
        for (int e = 0; e < E; ++e) {
          v[e] = seg[tm.lane * E + e];
          m = max(m, v[e]);
        }
        int run = max(carry, team_excl_max<TW>(tm, m, scan_scratch));
#pragma unroll
        for (int e = 0; e < E; ++e) {
          run = max(run, v[e]);
          seg[tm.lane * E + e] = run;
        }
        tm.sync();
        carry = seg[S - 1];
        long long q[kStagedPasses];
        int tt[kStagedPasses];
#pragma unroll
        for (int u = 0; u < kStagedPasses; ++u) {
          const long long xu = x0 + (long long)u * TW + tm.lane;
          q[u] = -1;
          tt[u] = 0;
          if (xu < total) {
            const int t = seg[xu - x0];
            q[u] = cs->bs[t] + (xu - cs->pre[t]);
            tt[u] = t;
            prefetch(q[u]);
          }
        }
#pragma unroll
        for (int u = 0; u < kStagedPasses; ++u)
          if (q[u] >= 0) body(q[u], tt[u]);
        tm.sync();
      }
      return total;
    }
  }
  if (total > 0) {
    long long x = tm.lane;
    if (x < total) {
      // first product: binary search for the last t with pre[t] <= x
      int lo = 0, hi = TW - 1;
      while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (cs->pre[mid] <= x) lo = mid; else hi = mid - 1;
      }
      int t = lo;
      for (; x < total; x += (long long)kStagedPasses * TW) {
        long long q[kStagedPasses];
        int tt[kStagedPasses];
#pragma unroll
        for (int u = 0; u < kStagedPasses; ++u) {
          const long long xu = x + (long long)u * TW;
          q[u] = -1;
          tt[u] = t;
          if (xu < total) {
            // the A entry of product xu: a few linear steps (long B ranges),
            // then a binary search (many short or empty ranges per pass)
            for (int st = 0; st < 8 && cs->pre[t + 1] <= xu; ++st) ++t;
            if (cs->pre[t + 1] <= xu) {
              int lo2 = t + 1, hi2 = TW - 1;
              while (lo2 < hi2) {
                const int mid = (lo2 + hi2 + 1) >> 1;
                if (cs->pre[mid] <= xu) lo2 = mid; else hi2 = mid - 1;
              }
              t = lo2;
            }
            q[u] = cs->bs[t] + (xu - cs->pre[t]);
            tt[u] = t;
            prefetch(q[u]);
          }
        }
#pragma unroll
        for (int u = 0; u < kStagedPasses; ++u)
          if (q[u] >= 0) body(q[u], tt[u]);
      }
    }
  }
  tm.sync();
  return total;
}

template <int TW, typename VT, class Body, class Prefetch>
__device__ __forceinline__ long long for_each_product_chunk(const Team<TW>& tm, ChunkScratch<TW, VT>* cs,
                                                            long long* scan_scratch, long long bs, long long be,
                                                            VT av, Body body, Prefetch prefetch, int* seg) {
  long long total;
  const long long ex = chunk_scan<TW, VT>(tm, cs, scan_scratch, bs, be, av, &total);
  return chunk_products<TW, VT>(tm, cs, scan_scratch, ex, total, bs, be, body, prefetch, seg);
}

template <int TW, typename VT, class Range, class AVal, class Body, class Prefetch>
__device__ __forceinline__ void for_each_product(const Team<TW>& tm, ChunkScratch<TW, VT>* cs,
                                                 long long* scan_scratch, const int* Aj,
                                                 long long a_beg, long long a_end, Range range,
                                                 AVal aval, Body body, Prefetch prefetch, int* seg) {
  for (long long c = a_beg; c < a_end; c += TW) {
    long long p = c + tm.lane;
    long long bs = 0, be = 0;
    VT av = VT(0);
    if (p < a_end) {
      int j = Aj[p];
      range(j, &bs, &be);
      av = aval(p);
    }
    for_each_product_chunk<TW, VT>(tm, cs, scan_scratch, bs, be, av, body, prefetch, seg);
  }
}

template <int TW, typename VT, class Range, class AVal, class Body>
__device__ __forceinline__ void for_each_product(const Team<TW>& tm, ChunkScratch<TW, VT>* cs,
                                                 long long* scan_scratch, const int* Aj,
                                                 long long a_beg, long long a_end, Range range,
                                                 AVal aval, Body body) {
  for_each_product<TW, VT>(tm, cs, scan_scratch, Aj, a_beg, a_end, range, aval, body, [](long long) {}, nullptr);
}

template <int TW, typename VT, class Range, class AVal, class Body, class Prefetch>
__device__ __forceinline__ void for_each_product(const Team<TW>& tm, ChunkScratch<TW, VT>* cs,
                                                 long long* scan_scratch, const int* Aj,
                                                 long long a_beg, long long a_end, Range range,
                                                 AVal aval, Body body, Prefetch prefetch) {
  for_each_product<TW, VT>(tm, cs, scan_scratch, Aj, a_beg, a_end, range, aval, body, prefetch, nullptr);
}

}  // namespace kks
