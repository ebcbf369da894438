// kks_rap.cu -- the Galerkin triple product C = P^T * A * P in one plan.
//
// Multigrid setup multiplies the restriction R = P^T, the fine operator A and
// the prolongation P (the R x A x P products of Section 4).  Instead of two
// SpGEMM plans and a materialised A*P, each row I of C is one team's work:
//
//   C(I,:) = sum_{i in R(I,:)} r_Ii * sum_{j in A(i,:)} a_ij * P(j,:)
//
// i.e. a row-wise product (Algorithm 1) whose "A row" is the concatenation of
// the rows A(i,:) over the entries of R(I,:), scaled by r_Ii.  R is never
// materialised with values: the symbolic phase builds the pattern of P^T
// (row index i and the entry of P holding r_Ii), and the numeric phase reads
// r_Ii from P through that entry, so new values of A and P need no transpose
// or gather.  As in Algorithm 2, a symbolic phase fixes the row sizes of C
// (the union of the P rows reached from row I, on a shared bitmap of
// ceil(K/32) words or an LP table, whichever is smaller) and a numeric phase
// accumulates into an LP table sized from the known row size (Section 3.1.2)
// and writes each row sorted by column.

#include <algorithm>

#include "kks_internal.h"

namespace kks {

namespace {

__host__ __device__ constexpr size_t al16(size_t x) { return (x + 15) & ~size_t(15); }

inline unsigned rap_grid(long long items, int per, int num_sms, int per_sm) {
  long long g = (items + per - 1) / per;
  const long long cap = (long long)num_sms * per_sm;
  if (g > cap) g = cap;
  if (g < 1) g = 1;
  return (unsigned)g;
}

}  // namespace

// log2 slots of the symbolic LP table of a row with w products (key bound
// min(w, K), at most 50 % load) and whether a bitmap of K bits is smaller.
__host__ __device__ int rap_sym_logT(long long w, long long K) {
  const long long b = w < K ? w : K;
  return ilog2_ceil(b > 1 ? 2 * b : 2);
}
__host__ __device__ bool rap_sym_bitmap(long long w, long long K) {
  return ((K + 31) >> 5) <= (1ll << rap_sym_logT(w, K));
}
__host__ __device__ size_t rap_sym_table_bytes(long long w, long long K) {
  return rap_sym_bitmap(w, K) ? (size_t)((K + 31) >> 5) * 4 : ((size_t)4 << rap_sym_logT(w, K));
}
// log2 slots of the numeric table of a row of C with s entries
__host__ __device__ int rap_num_logT(long long s) { return ilog2_ceil(s > 1 ? 2 * s : 2); }

// Rows of R with at least this many entries take one lane per entry (a fine
// row i), which combines its products by column in registers first.
constexpr int kLaneRowsMin = 8;
// columns one lane combines before it sends further products straight to the table
constexpr int kLaneKeys = 8;

template <int TW>
__host__ __device__ constexpr int rap_touch_cap() { return TW > 32 ? 1024 : 256; }

// symbolic team: chunk scratch | table (bitmap words or LP keys) | list of
// touched bitmap words | its length
template <int TW>
__host__ __device__ size_t rap_sym_team_bytes(size_t table) {
  return al16(sizeof(ChunkScratch<TW, double>)) + al16(table) + al16((size_t)rap_touch_cap<TW>() * 4) + 16;
}
// numeric team: chunk scratch | keys | values | sort buffer | exchange | the
// lanes' combined values (warp teams)
template <int TW, typename VT>
__host__ __device__ size_t rap_num_team_bytes(int logT) {
  const size_t T = (size_t)1 << logT;
  return al16(sizeof(ChunkScratch<TW, VT>)) + al16(T * 4) + al16(T * sizeof(VT)) + al16(T / 2 * 8) +
         al16((size_t)TW * sizeof(VT)) + (TW > 32 ? 0 : al16((size_t)kLaneKeys * TW * sizeof(VT)));
}

size_t rap_sym_team_bytes_host(int cta, size_t table) {
  return cta ? rap_sym_team_bytes<kRapCtaThreads>(table) : rap_sym_team_bytes<32>(table);
}
size_t rap_num_team_bytes_host(int cta, int dtype, int logT) {
  if (dtype == 1) return cta ? rap_num_team_bytes<kRapCtaThreads, double>(logT) : rap_num_team_bytes<32, double>(logT);
  return cta ? rap_num_team_bytes<kRapCtaThreads, float>(logT) : rap_num_team_bytes<32, float>(logT);
}

namespace {

// Products of row i of A*P: sum over A(i,:) of the lengths of the P rows.
// Also flags (*not_unit = 1) unless every row i of P holds exactly one entry
// at position i (plain aggregation), which lets the product loops take P's
// entry of row j at j without reading its row pointers.
__global__ void k_rap_fine_rf(RapD R, long long* rf, unsigned long long* not_unit) {
  const long long stride = (long long)gridDim.x * blockDim.x;
  bool unit = true;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < R.P.nrows; i += stride)
    unit &= rp_at(R.P, i) == i && rp_at(R.P, i + 1) == i + 1;
  if (__any_sync(0xffffffffu, !unit) && (threadIdx.x & 31) == 0) atomicOr(not_unit, 1ull);
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < R.A.nrows; i += stride) {
    const long long a0 = rp_at(R.A, i), a1 = rp_at(R.A, i + 1);
    long long w = 0;
    if (a0 < 0 || a0 > a1 || a1 > R.A.nnz) {
      dev_fail(R.status, kDevBadIndex, 60, i);
    } else {
#pragma unroll 4
      for (long long p = a0; p < a1; ++p) {
        const int j = R.A.cj[p];
        if ((unsigned long long)(unsigned)j >= (unsigned long long)R.P.nrows) {
          dev_fail(R.status, kDevBadIndex, 61, i);
          continue;
        }
        w += rp_at(R.P, j + 1) - rp_at(R.P, j);
      }
    }
    rf[i] = w;
  }
}

// Appends row I to list c (warp-aggregated: one atomic per warp and list).
__device__ __forceinline__ void rap_append(int cls, int c, long long I, unsigned long long* count, int* list) {
  const unsigned m = __ballot_sync(0xffffffffu, cls == c);
  if (m == 0u) return;
  const int lane = threadIdx.x & 31;
  const int leader = __ffs(m) - 1;
  unsigned long long base = 0;
  if (lane == leader) base = atomicAdd(count, (unsigned long long)__popc(m));
  base = __shfl_sync(0xffffffffu, base, leader);
  if (cls == c) list[base + __popc(m & ((1u << lane) - 1u))] = (int)I;
}

// Warp maximum / sum folded into one global atomic per warp.
__device__ __forceinline__ void warp_atomic_max(unsigned long long* dst, unsigned long long v) {
#pragma unroll
  for (int d = 16; d > 0; d >>= 1) {
    const unsigned long long o = __shfl_xor_sync(0xffffffffu, v, d);
    v = o > v ? o : v;
  }
  if ((threadIdx.x & 31) == 0 && v > 0) atomicMax(dst, v);
}
__device__ __forceinline__ void warp_atomic_add(unsigned long long* dst, unsigned long long v) {
#pragma unroll
  for (int d = 16; d > 0; d >>= 1) v += __shfl_xor_sync(0xffffffffu, v, d);
  if ((threadIdx.x & 31) == 0 && v > 0) atomicAdd(dst, v);
}

// Calls f(l, a_ij, p_jl) for every product of the row A(i,:) (entries
// [as, ae)) with P: the loads of kLaneBatch A entries, of their P row
// pointers and of the first entry of each P row are issued together, so one
// lane walking its row waits for a few dependent misses per batch instead of
// per entry.  kVals = false skips the values (a, p are then 0).
constexpr int kLaneBatch = 4;

template <bool kVals, typename VT, class F>
__device__ __forceinline__ void rap_lane_products(const RapD& R, const VT* __restrict__ Ax, const VT* __restrict__ Px,
                                                  long long as, long long ae, long long I, F f) {
  for (long long p = as; p < ae; p += kLaneBatch) {
    int j[kLaneBatch], plen[kLaneBatch], l0[kLaneBatch];
    long long q0[kLaneBatch];
    VT a[kLaneBatch], pv0[kLaneBatch];
#pragma unroll
    for (int u = 0; u < kLaneBatch; ++u) {
      j[u] = 0;
      a[u] = VT(0);
      plen[u] = 0;
      q0[u] = 0;
      if (p + u < ae) {
        j[u] = R.A.cj[p + u];
        if (kVals) a[u] = Ax[p + u];
        if ((unsigned long long)(unsigned)j[u] < (unsigned long long)R.P.nrows) plen[u] = 1;
        else dev_fail(R.status, kDevBadIndex, 63, I);
      }
    }
#pragma unroll
    for (int u = 0; u < kLaneBatch; ++u) {
      if (plen[u]) {
        if (R.punit) {
          q0[u] = j[u];
        } else {
          q0[u] = rp_at(R.P, j[u]);
          plen[u] = (int)(rp_at(R.P, j[u] + 1) - q0[u]);
        }
      }
    }
#pragma unroll
    for (int u = 0; u < kLaneBatch; ++u) {
      l0[u] = 0;
      pv0[u] = VT(0);
      if (plen[u] > 0) {
        l0[u] = R.P.cj[q0[u]];
        if (kVals) pv0[u] = Px[q0[u]];
      }
    }
#pragma unroll
    for (int u = 0; u < kLaneBatch; ++u) {
      if (plen[u] > 0) {
        f(l0[u], a[u], pv0[u]);
        for (int t = 1; t < plen[u]; ++t) f(R.P.cj[q0[u] + t], a[u], kVals ? Px[q0[u] + t] : VT(0));
      }
    }
  }
}

// Per row I of C: its product count w(I) = sum over R(I,:) of the A*P row
// products, and its symbolic team class (warp or CTA, by table bytes).
// meta: [0] warp rows, [1] CTA rows, [2] largest warp table, [3] largest CTA
// table, [4] sum of w.  Empty rows get their count 0 here.
__global__ void k_rap_bound(RapD R, const long long* rf, long long* w_out, long long* cnt, int* rows_w, int* rows_c,
                            unsigned long long* meta, unsigned long long warp_table, unsigned long long cta_table) {
  const long long K = R.P.ncols;
  const long long stride = (long long)gridDim.x * blockDim.x;
  // uniform trip count: the appends are warp collectives
  for (long long b0 = (long long)blockIdx.x * blockDim.x; b0 < K; b0 += stride) {
    const long long I = b0 + threadIdx.x;
    int cls = 0;
    unsigned long long bw = 0, bc = 0, ws = 0;
    if (I < K) {
      long long w = 0;
      const long long x0 = R.Rtp[I], x1 = R.Rtp[I + 1];
      for (long long x = x0; x < x1; ++x) {
        const int i = R.Rti[x];
        if ((unsigned long long)(unsigned)i < (unsigned long long)R.A.nrows) w += rf[i];
        else dev_fail(R.status, kDevBadIndex, 59, I);
      }
      w_out[I] = w;
      if (w > 0) {
        const unsigned long long bytes = rap_sym_table_bytes(w, K);
        if (bytes <= warp_table) {
          cls = 1;
          bw = bytes;
        } else if (bytes <= cta_table) {
          cls = 2;
          bc = bytes;
        } else {
          dev_fail(R.status, kDevRowTooLarge, 62, I);
        }
        ws = (unsigned long long)w;
      }
      if (cls == 0) cnt[I] = 0;
    }
    warp_atomic_max(&meta[2], bw);
    warp_atomic_max(&meta[3], bc);
    warp_atomic_add(&meta[4], ws);
    rap_append(cls, 1, I, &meta[0], rows_w);
    rap_append(cls, 2, I, &meta[1], rows_c);
  }
}

// Symbolic: the size of each listed row of C.  The team's table region holds
// zeros between rows: a bitmap row records the words it touches and clears
// only those, a hash row clears its slots after counting.
template <int TW>
__global__ void __launch_bounds__(256) k_rap_sym(RapD R, const int* __restrict__ rows, long long nrows,
                                                 const long long* __restrict__ w_in, long long* cnt,
                                                 size_t team_bytes, long long table_words, int hash_mode) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ long long scan_scratch[33];
  Team<TW> tm;
  constexpr int kCap = rap_touch_cap<TW>();
  unsigned char* base = smem + (size_t)tm.id * team_bytes;
  auto* cs = reinterpret_cast<ChunkScratch<TW, double>*>(base);
  int* tab = reinterpret_cast<int*>(base + al16(sizeof(ChunkScratch<TW, double>)));
  int* touched = reinterpret_cast<int*>(reinterpret_cast<unsigned char*>(tab) + al16((size_t)table_words * 4));
  int* ntouch = touched + kCap;
  unsigned* bm = reinterpret_cast<unsigned*>(tab);
  const long long K = R.P.ncols;
  for (long long x = tm.lane; x < table_words; x += TW) tab[x] = 0;
  tm.sync();
  const long long team = (long long)blockIdx.x * tm.per_cta + tm.id;
  const long long nteams = (long long)gridDim.x * tm.per_cta;
  for (long long r = team; r < nrows; r += nteams) {
    const long long I = rows[r];
    const long long w = w_in[I];
    const bool bmp = rap_sym_bitmap(w, K);
    const int logT = rap_sym_logT(w, K);
    const long long nw = bmp ? ((K + 31) >> 5) : (1ll << logT);
    if (!bmp)
      for (long long x = tm.lane; x < nw; x += TW) tab[x] = kEmpty;
    if (tm.lane == 0) *ntouch = 0;
    tm.sync();
    const LpHash hs(bmp ? 1 : logT, hash_mode);
    auto insert = [&](int l) {
      if ((unsigned long long)(unsigned)l >= (unsigned long long)K) {
        dev_fail(R.status, kDevBadIndex, 64, I);
        return;
      }
      if (bmp) {
        const unsigned old = atomicOr(bm + (l >> 5), 1u << (l & 31));
        if (old == 0u) {
          const int t = atomicAdd(ntouch, 1);
          if (t < kCap) touched[t] = l >> 5;
        }
      } else if (lp_insert(tab, hs, nullptr, -1, l) < 0) {
        dev_fail(R.status, kDevTableFull, 65, I);
      }
    };
    const long long x0 = R.Rtp[I], x1 = R.Rtp[I + 1];
    for (long long c = x0; c < x1; c += TW) {
      // a chunk of R(I,:): its rows A(i,:), products spread flat over the team
      const long long x = c + tm.lane;
      long long as = 0, len = 0;
      if (x < x1) {
        const int i = R.Rti[x];
        as = rp_at(R.A, i);
        len = rp_at(R.A, i + 1) - as;
      }
      long long tot;
      const long long ex = team_excl_scan<TW>(tm, len, &tot, scan_scratch);
      cs->pre[tm.lane] = ex;
      cs->bs[tm.lane] = as;
      if (tm.lane == 0) cs->pre[TW] = tot;
      tm.sync();
      int t = 0;
      for (long long yb = 0; yb < tot; yb += (long long)kLaneBatch * TW) {
        // kLaneBatch products per lane: their A entries, P row pointers and
        // first P entries are loaded together
        int j[kLaneBatch], plen[kLaneBatch], l0[kLaneBatch];
        long long q0[kLaneBatch];
#pragma unroll
        for (int u = 0; u < kLaneBatch; ++u) {
          const long long y = yb + (long long)u * TW + tm.lane;
          plen[u] = 0;
          j[u] = 0;
          if (y < tot) {
            while (cs->pre[t + 1] <= y) ++t;
            j[u] = R.A.cj[cs->bs[t] + (y - cs->pre[t])];
            if ((unsigned long long)(unsigned)j[u] < (unsigned long long)R.P.nrows) plen[u] = 1;
            else dev_fail(R.status, kDevBadIndex, 63, I);
          }
        }
#pragma unroll
        for (int u = 0; u < kLaneBatch; ++u) {
          q0[u] = j[u];
          if (plen[u] && !R.punit) {
            q0[u] = rp_at(R.P, j[u]);
            plen[u] = (int)(rp_at(R.P, j[u] + 1) - q0[u]);
          }
        }
#pragma unroll
        for (int u = 0; u < kLaneBatch; ++u) l0[u] = plen[u] > 0 ? R.P.cj[q0[u]] : 0;
#pragma unroll
        for (int u = 0; u < kLaneBatch; ++u) {
          if (plen[u] > 0) {
            insert(l0[u]);
            for (int e = 1; e < plen[u]; ++e) insert(R.P.cj[q0[u] + e]);
          }
        }
      }
      tm.sync();
    }
    tm.sync();
    long long c = 0;
    const int nt = *ntouch;
    const bool listed = bmp && nt <= kCap;
    if (listed) {
      for (int t = tm.lane; t < nt; t += TW) c += __popc(bm[touched[t]]);
    } else {
      for (long long x = tm.lane; x < nw; x += TW) c += bmp ? __popc(bm[x]) : (tab[x] != kEmpty ? 1 : 0);
    }
    const long long total = team_sum<TW>(tm, c, scan_scratch);
    if (tm.lane == 0) cnt[I] = total;
    tm.sync();
    if (listed) {
      for (int t = tm.lane; t < nt; t += TW) bm[touched[t]] = 0u;
    } else {
      for (long long x = tm.lane; x < nw; x += TW) tab[x] = 0;
    }
    tm.sync();
  }
}

// Numeric team classes from the row sizes of C.  meta: [5] warp rows, [6] CTA
// rows, [7] largest warp log2 table, [8] largest CTA log2 table, [9] largest row.
__global__ void k_rap_num_bin(const long long* Crp, long long K, int* rows_w, int* rows_c, unsigned long long* meta,
                              int warp_logT, int cta_logT, DevStatus* st) {
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long b0 = (long long)blockIdx.x * blockDim.x; b0 < K; b0 += stride) {
    const long long I = b0 + threadIdx.x;
    int cls = 0;
    unsigned long long lw = 0, lc = 0, sm = 0;
    if (I < K) {
      const long long s = Crp[I + 1] - Crp[I];
      if (s > 0) {
        const int l = rap_num_logT(s);
        if (l <= warp_logT) {
          cls = 1;
          lw = (unsigned long long)l;
        } else if (l <= cta_logT) {
          cls = 2;
          lc = (unsigned long long)l;
        } else {
          dev_fail(st, kDevRowTooLarge, 66, I);
        }
        sm = (unsigned long long)s;
      }
    }
    warp_atomic_max(&meta[7], lw);
    warp_atomic_max(&meta[8], lc);
    warp_atomic_max(&meta[9], sm);
    rap_append(cls, 1, I, &meta[5], rows_w);
    rap_append(cls, 2, I, &meta[6], rows_c);
  }
}

// Adds v to the value of column l of the row (one call per lane of a warp,
// all lanes together; has = false lanes only take part).  Lanes whose columns
// meet in one slot are summed by the group's lowest lane first, which then
// adds alone (warp teams) or atomically (CTA teams, whose warps share the
// table).
template <bool kAtomic, typename VT>
__device__ __forceinline__ void rap_add_grouped(int* keys, VT* vals, VT* xchg, const LpHash& hs, bool has, int l,
                                                VT v, DevStatus* st, long long I) {
  const int lane32 = threadIdx.x & 31;
  const unsigned lt = (1u << lane32) - 1u;
  const int slot = lp_insert_team(0xffffffffu, keys, hs, has, l);
  if (has && slot < 0) dev_fail(st, kDevTableFull, 68, I);
  const int g = (has && slot >= 0) ? slot : -1 - lane32;
  const unsigned grp = __match_any_sync(0xffffffffu, g);
  const bool leader = (grp & lt) == 0;
  if (__any_sync(0xffffffffu, __popc(grp) > 1)) {
    xchg[lane32] = v;
    __syncwarp();
    if (leader) {
      unsigned rest = grp & ~(1u << lane32);
      while (rest) {
        const int o = __ffs(rest) - 1;
        rest &= rest - 1u;
        v += xchg[o];
      }
    }
    __syncwarp();
  }
  if (g >= 0 && leader) {
    if constexpr (kAtomic) atomicAdd(vals + g, v);
    else vals[g] += v;
  }
  __syncwarp();
}

// Numeric: values of each listed row of C, written sorted by column.
//  - rows of R with at least kLaneRowsMin entries (warp teams): a lane per
//    fine row i combines a_ij * p_jl by column in its own column of shared
//    memory (up to kLaneKeys columns, keys in registers; Thread-Sequential,
//    Section 3.1.1), then the lanes add r_Ii times their sums to the row's
//    table together;
//  - other rows (and CTA teams): the products are spread flat over the team
//    (Thread-Flat-Parallel), one A entry per lane and pass.
template <int TW, typename VT>
__global__ void __launch_bounds__(256) k_rap_num(RapD R, const int* __restrict__ rows, long long nrows,
                                                 const long long* __restrict__ Crp, int* __restrict__ Cj,
                                                 VT* __restrict__ Cx, size_t team_bytes, int hash_mode) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ long long scan_scratch[33];
  Team<TW> tm;
  constexpr bool kCta = Team<TW>::kCta;
  unsigned char* base = smem + (size_t)tm.id * team_bytes;
  auto* cs = reinterpret_cast<ChunkScratch<TW, VT>*>(base);
  int* keys = reinterpret_cast<int*>(base + al16(sizeof(ChunkScratch<TW, VT>)));
  const VT* __restrict__ Ax = reinterpret_cast<const VT*>(R.A.vx);
  const VT* __restrict__ Px = reinterpret_cast<const VT*>(R.P.vx);
  const int lane32 = threadIdx.x & 31;
  const unsigned lt = (1u << lane32) - 1u;
  const long long team = (long long)blockIdx.x * tm.per_cta + tm.id;
  const long long nteams = (long long)gridDim.x * tm.per_cta;
  for (long long r = team; r < nrows; r += nteams) {
    const long long I = rows[r];
    const long long c0 = Crp[I];
    const long long s = Crp[I + 1] - c0;
    const int logT = rap_num_logT(s);
    const int T = 1 << logT;
    const int half = T / 2;
    VT* vals = reinterpret_cast<VT*>(reinterpret_cast<unsigned char*>(keys) + al16((size_t)T * 4));
    unsigned long long* sortb =
        reinterpret_cast<unsigned long long*>(reinterpret_cast<unsigned char*>(vals) + al16((size_t)T * sizeof(VT)));
    VT* xchg = reinterpret_cast<VT*>(reinterpret_cast<unsigned char*>(sortb) + al16((size_t)half * 8));
    VT* lanev = reinterpret_cast<VT*>(reinterpret_cast<unsigned char*>(xchg) + al16((size_t)TW * sizeof(VT)));
    for (int x = tm.lane; x < T; x += TW) {
      keys[x] = kEmpty;
      vals[x] = VT(0);
    }
    tm.sync();
    const LpHash hs(logT, hash_mode);
    const long long x0 = R.Rtp[I], x1 = R.Rtp[I + 1];
    if (!kCta && x1 - x0 >= kLaneRowsMin) {
      for (long long c = x0; c < x1; c += TW) {
        const long long x = c + tm.lane;
        int ck[kLaneKeys];
#pragma unroll
        for (int k = 0; k < kLaneKeys; ++k) {
          ck[k] = -1;
          lanev[k * TW + tm.lane] = VT(0);
        }
        VT rv = VT(0);
        if (x < x1) {
          const int i = R.Rti[x];
          rv = Px[R.Rpe[x]];
          const long long as = rp_at(R.A, i), ae = rp_at(R.A, i + 1);
          rap_lane_products<true, VT>(R, Ax, Px, as, ae, I, [&](int l, VT a, VT pv) {
              int hit = -1;
#pragma unroll
              for (int k = 0; k < kLaneKeys; ++k) hit = ck[k] == l ? k : hit;
              if (hit < 0) {
#pragma unroll
                for (int k = kLaneKeys - 1; k >= 0; --k) hit = ck[k] < 0 ? k : hit;
                if (hit >= 0) {
#pragma unroll
                  for (int k = 0; k < kLaneKeys; ++k)
                    if (k == hit) ck[k] = l;
                }
              }
              if (hit >= 0) {
                VT* acc = lanev + hit * TW + tm.lane;
                *acc = fma_acc(a, pv, *acc);
              } else {
                // more columns than the lane keeps: straight to the table
                const int slot = lp_insert(keys, hs, nullptr, -1, l);
                if (slot < 0) dev_fail(R.status, kDevTableFull, 70, I);
                else atomicAdd(vals + slot, rv * (a * pv));
              }
          });
        }
        __syncwarp();
        // the lanes' sums, scaled by r_Ii, into the row's table
        int nk = 0;
#pragma unroll
        for (int k = 0; k < kLaneKeys; ++k) nk += ck[k] >= 0 ? 1 : 0;
        const int rounds = (int)__reduce_max_sync(0xffffffffu, (unsigned)nk);
#pragma unroll
        for (int k = 0; k < kLaneKeys; ++k) {
          if (k < rounds) {
            const bool has = ck[k] >= 0;
            const VT v = has ? rv * lanev[k * TW + tm.lane] : VT(0);
            rap_add_grouped<false, VT>(keys, vals, xchg, hs, has, has ? ck[k] : 0, v, R.status, I);
          }
        }
      }
    } else {
      for (long long c = x0; c < x1; c += TW) {
        // a chunk of R(I,:): the rows A(i,:) and the values r_Ii
        const long long x = c + tm.lane;
        long long as = 0, len = 0;
        VT rv = VT(0);
        if (x < x1) {
          const int i = R.Rti[x];
          rv = Px[R.Rpe[x]];
          as = rp_at(R.A, i);
          len = rp_at(R.A, i + 1) - as;
        }
        long long tot;
        const long long ex = team_excl_scan<TW>(tm, len, &tot, scan_scratch);
        cs->pre[tm.lane] = ex;
        cs->bs[tm.lane] = as;
        cs->av[tm.lane] = rv;
        if (tm.lane == 0) cs->pre[TW] = tot;
        tm.sync();
        int t = 0;
        for (long long yb = 0; yb < tot; yb += TW) {
          const long long y = yb + tm.lane;
          long long p0 = 0;
          int plen = 0;
          VT ra = VT(0);
          if (y < tot) {
            // the chunk entry of product y (non-decreasing in y for each lane)
            while (cs->pre[t + 1] <= y) ++t;
            const long long q = cs->bs[t] + (y - cs->pre[t]);
            const int j = R.A.cj[q];
            if ((unsigned long long)(unsigned)j < (unsigned long long)R.P.nrows) {
              ra = cs->av[t] * Ax[q];
              p0 = rp_at(R.P, j);
              plen = (int)(rp_at(R.P, j + 1) - p0);
            } else {
              dev_fail(R.status, kDevBadIndex, 67, I);
            }
          }
          const int steps = (int)__reduce_max_sync(0xffffffffu, (unsigned)plen);
          for (int u = 0; u < steps; ++u) {
            const bool has = u < plen;
            int l = 0;
            VT v = VT(0);
            if (has) {
              l = R.P.cj[p0 + u];
              v = ra * Px[p0 + u];
            }
            rap_add_grouped<kCta, VT>(keys, vals, xchg + (tm.lane & ~31), hs, has, l, v, R.status, I);
          }
        }
        tm.sync();
      }
    }
    tm.sync();
    // C(I,:) in column order
    if (!kCta && half <= TW) {
      // at most 32 columns: keys sorted in registers, values found by key
      const unsigned o = (tm.lane < T && keys[tm.lane] != kEmpty) ? 1u : 0u;
      const unsigned o2 = (tm.lane + TW < T && keys[tm.lane + TW] != kEmpty) ? 1u : 0u;
      const unsigned b1 = __ballot_sync(0xffffffffu, o), b2 = __ballot_sync(0xffffffffu, o2);
      const int cnt = __popc(b1) + __popc(b2);
      if (tm.lane == 0 && cnt != s) dev_fail(R.status, kDevRowSizeMismatch, 69, I);
      const int p1 = __popc(b1 & lt), p2 = __popc(b1) + __popc(b2 & lt);
      if (o && p1 < half) sortb[p1] = (unsigned)keys[tm.lane];
      if (o2 && p2 < half) sortb[p2] = (unsigned)keys[tm.lane + TW];
      __syncwarp();
      const int n = cnt < half ? cnt : half;
      unsigned v = tm.lane < n ? (unsigned)sortb[tm.lane] : 0xffffffffu;
      v = team_sort1<32>(0xffffffffu, tm.lane, v);
      const long long nw = n < s ? n : s;
      if (tm.lane < nw) {
        const int slot = key_slot(keys, hs, (int)v);
        Cj[c0 + tm.lane] = (int)v;
        Cx[c0 + tm.lane] = slot >= 0 ? vals[slot] : VT(0);
      }
      __syncwarp();
    } else {
      long long cnt = 0;
      for (int xb = 0; xb < T; xb += TW) {
        const int x = xb + tm.lane;
        const int o = (x < T && keys[x] != kEmpty) ? 1 : 0;
        long long t2;
        const long long pos = cnt + team_excl_scan<TW>(tm, o, &t2, scan_scratch);
        if (o && pos < half) sortb[pos] = ((unsigned long long)(unsigned)keys[x] << 32) | (unsigned)x;
        cnt += t2;
      }
      if (tm.lane == 0 && cnt != s) dev_fail(R.status, kDevRowSizeMismatch, 69, I);
      const int n = cnt < half ? (int)cnt : half;
      int N = 1;
      while (N < n) N <<= 1;
      for (int x = n + tm.lane; x < N; x += TW) sortb[x] = ~0ull;
      tm.sync();
      team_bitonic<TW>(tm, sortb, N);
      const long long nw = n < s ? n : s;
      for (long long x = tm.lane; x < nw; x += TW) {
        const unsigned long long e = sortb[x];
        Cj[c0 + x] = (int)(e >> 32);
        Cx[c0 + x] = vals[(unsigned)(e & 0xffffffffull)];
      }
    }
    tm.sync();
  }
}

template <class K>
cudaError_t rap_set_smem(K kernel, size_t bytes) {
  return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

}  // namespace

cudaError_t launch_rap_prepare(const LaunchCtx& L, const RapD& R, long long* rf, long long* w, long long* cnt,
                               int* rows_w, int* rows_c, unsigned long long* meta, size_t warp_table,
                               size_t cta_table, void* tmp) {
  // (1) products of the rows of A*P
  if (R.A.nrows > 0 || R.P.nrows > 0) {
    KKS_LAUNCHED();
    k_rap_fine_rf<<<rap_grid(std::max(R.A.nrows, R.P.nrows), 256, L.num_sms, 16), 256, 0, L.stream>>>(R, rf, meta + 10);
  }
  // (2) the pattern of P^T: rows of R with the entry of P behind each value
  cudaError_t e = launch_transpose_pattern(L, R.P, const_cast<long long*>(R.Rtp), const_cast<int*>(R.Rti),
                                           const_cast<long long*>(R.Rpe), tmp, R.status);
  if (e != cudaSuccess) return e;
  // (3) row bounds and symbolic classes of C
  const long long K = R.P.ncols;
  if (K > 0) {
    KKS_LAUNCHED();
    k_rap_bound<<<rap_grid(K, 256, L.num_sms, 8), 256, 0, L.stream>>>(R, rf, w, cnt, rows_w, rows_c, meta,
                                                                     (unsigned long long)warp_table,
                                                                     (unsigned long long)cta_table);
  }
  return cudaGetLastError();
}

cudaError_t launch_rap_symbolic(const LaunchCtx& L, const RapD& R, const long long* w, long long* cnt,
                                const int* rows_w, long long n_w, size_t table_w, const int* rows_c, long long n_c,
                                size_t table_c, int hash_mode) {
  if (n_w > 0) {
    const size_t tb = rap_sym_team_bytes<32>(table_w);
    const size_t smem = tb * 8;
    auto kern = k_rap_sym<32>;
    cudaError_t e = rap_set_smem(kern, smem);
    if (e != cudaSuccess) return e;
    const unsigned grid = resident_grid(kern, 256, smem, L.num_sms, (n_w + 7) / 8);
    KKS_LAUNCHED();
    kern<<<grid, 256, smem, L.stream>>>(R, rows_w, n_w, w, cnt, tb, (long long)(al16(table_w) / 4), hash_mode);
  }
  if (n_c > 0) {
    const size_t tb = rap_sym_team_bytes<kRapCtaThreads>(table_c);
    auto kern = k_rap_sym<kRapCtaThreads>;
    cudaError_t e = rap_set_smem(kern, tb);
    if (e != cudaSuccess) return e;
    const unsigned grid = resident_grid(kern, kRapCtaThreads, tb, L.num_sms, n_c);
    KKS_LAUNCHED();
    kern<<<grid, kRapCtaThreads, tb, L.stream>>>(R, rows_c, n_c, w, cnt, tb, (long long)(al16(table_c) / 4),
                                                   hash_mode);
  }
  return cudaGetLastError();
}

cudaError_t launch_rap_num_bin(const LaunchCtx& L, const long long* Crp, long long K, int* rows_w, int* rows_c,
                               unsigned long long* meta, int warp_logT, int cta_logT, DevStatus* st) {
  if (K <= 0) return cudaSuccess;
  KKS_LAUNCHED();
  k_rap_num_bin<<<rap_grid(K, 256, L.num_sms, 8), 256, 0, L.stream>>>(Crp, K, rows_w, rows_c, meta, warp_logT,
                                                                      cta_logT, st);
  return cudaGetLastError();
}

template <typename VT>
static cudaError_t launch_rap_numeric_t(const LaunchCtx& L, const RapD& R, const long long* Crp, int* Cj, void* Cx,
                                        const int* rows_w, long long n_w, int logT_w, const int* rows_c,
                                        long long n_c, int logT_c, int hash_mode) {
  if (n_w > 0) {
    const size_t tb = rap_num_team_bytes<32, VT>(logT_w);
    const size_t smem = tb * 8;
    auto kern = k_rap_num<32, VT>;
    cudaError_t e = rap_set_smem(kern, smem);
    if (e != cudaSuccess) return e;
    const unsigned grid = resident_grid(kern, 256, smem, L.num_sms, (n_w + 7) / 8);
    KKS_LAUNCHED();
    kern<<<grid, 256, smem, L.stream>>>(R, rows_w, n_w, Crp, Cj, reinterpret_cast<VT*>(Cx), tb, hash_mode);
  }
  if (n_c > 0) {
    const size_t tb = rap_num_team_bytes<kRapCtaThreads, VT>(logT_c);
    auto kern = k_rap_num<kRapCtaThreads, VT>;
    cudaError_t e = rap_set_smem(kern, tb);
    if (e != cudaSuccess) return e;
    const unsigned grid = resident_grid(kern, kRapCtaThreads, tb, L.num_sms, n_c);
    KKS_LAUNCHED();
    kern<<<grid, kRapCtaThreads, tb, L.stream>>>(R, rows_c, n_c, Crp, Cj, reinterpret_cast<VT*>(Cx), tb, hash_mode);
  }
  return cudaGetLastError();
}

cudaError_t launch_rap_numeric(const LaunchCtx& L, const RapD& R, int dtype, const long long* Crp, int* Cj, void* Cx,
                               const int* rows_w, long long n_w, int logT_w, const int* rows_c, long long n_c,
                               int logT_c, int hash_mode) {
  if (dtype == 1)
    return launch_rap_numeric_t<double>(L, R, Crp, Cj, Cx, rows_w, n_w, logT_w, rows_c, n_c, logT_c, hash_mode);
  return launch_rap_numeric_t<float>(L, R, Crp, Cj, Cx, rows_w, n_w, logT_w, rows_c, n_c, logT_c, hash_mode);
}

}  // namespace kks
