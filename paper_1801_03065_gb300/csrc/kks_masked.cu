// kks_masked.cu -- products restricted to a known pattern, and CSR transpose.
//
// Masked product: out(i,l) = sum_j X(i,j) * Y(j,l) for (i,l) in S.  The team's
// LP accumulator is keyed by S(i,:) before any product is formed (probe-only
// inserts), so products outside the pattern are dropped and each value lands
// at the position of its column in S(i,:): the result needs no sort.  Uses:
//   * numeric reuse on C's known pattern (X = A, Y = B, S = C)
//   * gradients of L(C), C = A * B, on fixed patterns:
//     dA = G * B^T on A's pattern (X = G, Y = B^T), dB = A^T * G on B's
//     pattern (X = A^T, Y = G).
// Rows of S larger than the shared table use the same code with the table in
// a global pool chunk.  When every row of S is sorted, warp-team rows key the
// table by S's column sets instead and compute each column's place in S(i,:)
// from the set bits (k_masked_pos).
//
// Transpose: column counts, their scan, an atomic scatter of (row, position)
// and a per-row bitonic sort by row, which also yields the permutation that
// maps A's values to A^T's (a later value-only update is a gather).
#include "kks_internal.h"

namespace kks {

namespace {

__host__ __device__ constexpr size_t al16(size_t x) { return (x + 15) & ~size_t(15); }

template <int TW, typename VT>
__host__ __device__ size_t msk_team_bytes(int T) {
  const int half = T / 2 > 0 ? T / 2 : 1;
  return al16((size_t)T * 4) * 2 + al16((size_t)half * sizeof(VT)) + al16(sizeof(ChunkScratch<TW, VT>));
}

template <int TW, typename VT, bool GTAB>
__global__ void k_masked(MaskedD M, const int* __restrict__ rows, long long nrows, int logT,
                         unsigned char* pool, long long chunk_bytes) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ long long scan_scratch[33];
  Team<TW> tm;
  const int T = 1 << logT;
  const LpHash tmask(logT, M.hash_mode);
  const int half = T / 2 > 0 ? T / 2 : 1;
  unsigned char* base;
  ChunkScratch<TW, VT>* csc;
  if (GTAB) {
    base = pool + (long long)blockIdx.x * chunk_bytes;
    csc = reinterpret_cast<ChunkScratch<TW, VT>*>(smem);
  } else {
    base = smem + (size_t)tm.id * msk_team_bytes<TW, VT>(T);
    csc = reinterpret_cast<ChunkScratch<TW, VT>*>(base + al16((size_t)T * 4) * 2 + al16((size_t)half * sizeof(VT)));
  }
  int* keys = reinterpret_cast<int*>(base);
  int* pos = reinterpret_cast<int*>(base + al16((size_t)T * 4));
  VT* acc = reinterpret_cast<VT*>(base + al16((size_t)T * 4) * 2);
  const VT* __restrict__ Xx = reinterpret_cast<const VT*>(M.X.vx);
  const VT* __restrict__ Yx = reinterpret_cast<const VT*>(M.Y.vx);
  // values may be read through a permutation (a transpose's values without a gather)
  auto XV = [&](long long p) -> VT { return Xx[M.xperm ? M.xperm[p] : p]; };
  auto YV = [&](long long q) -> VT { return Yx[M.yperm ? M.yperm[q] : q]; };
  const int* __restrict__ Yj = M.Y.cj;
  VT* __restrict__ out = reinterpret_cast<VT*>(M.out);

  const long long team = (long long)blockIdx.x * tm.per_cta + tm.id;
  const long long nteams = (long long)gridDim.x * tm.per_cta;
  for (long long r = team; r < nrows; r += nteams) {
    const long long i = rows[r];
    const long long s0 = M.Sp[i];
    const long long s = M.Sp[i + 1] - s0;
    for (int x = tm.lane; x < T; x += TW) keys[x] = kEmpty;
    if (GTAB) __threadfence_block();
    tm.sync();
    for (long long p = tm.lane; p < s; p += TW) {
      const int slot = lp_insert(keys, tmask, nullptr, -1, M.Sj[s0 + p]);
      if (slot >= 0 && p < half) {
        pos[slot] = (int)p;
        acc[p] = VT(0);
      } else {
        dev_fail(M.status, kDevTableFull, 20, i);
      }
    }
    if (GTAB) __threadfence_block();
    tm.sync();
    const long long a0 = rp_at(M.X, i), a1 = rp_at(M.X, i + 1);
    auto range = [&](int j, long long* bs, long long* be) {
      *bs = rp_at(M.Y, j);
      *be = rp_at(M.Y, j + 1);
    };
    auto aval = [&](long long p) { return XV(p); };
    auto body = [&](long long q, int t) {
      const int slot = lp_find(keys, tmask, Yj[q]);
      if (slot >= 0) atomicAdd(acc + pos[slot], csc->av[t] * YV(q));
    };
    auto pf = [&](long long q) {
      prefetch_l1(Yj + q);
      prefetch_l1(Yx + (M.yperm ? M.yperm[q] : q));
    };
    for_each_product<TW, VT>(tm, csc, scan_scratch, M.X.cj, a0, a1, range, aval, body, pf);
    if (GTAB) {
      __threadfence_block();
      tm.sync();
    }
    const long long sw = s < half ? s : half;
    for (long long p = tm.lane; p < sw; p += TW) out[s0 + p] = acc[p];
    if (GTAB) __threadfence_block();
    tm.sync();
  }
}

// Warp / sub-warp teams (TW <= 32): the same probe-only accumulation without
// floating-point atomics.  One Y row per pass when Y rows are long (distinct
// keys, so distinct positions), otherwise the chunk's products are spread over
// the lanes and equal keys are summed through match_any before one lane
// updates the position.
template <int TW, typename VT>
__host__ __device__ size_t mskw_team_bytes(int T) {
  const int half = T / 2 > 0 ? T / 2 : 1;
  return al16((size_t)T * 4) * 2 + al16((size_t)half * sizeof(VT)) + al16(sizeof(ChunkScratch<TW, VT>)) +
         al16((size_t)TW * sizeof(VT));
}

template <int TW, typename VT>
__global__ void __launch_bounds__(256) k_masked_warp(MaskedD M, const int* __restrict__ rows, long long nrows,
                                                     int logT) {
  extern __shared__ __align__(16) unsigned char smem[];
  Team<TW> tm;
  const int T = 1 << logT;
  const LpHash tmask(logT, M.hash_mode);
  const int half = T / 2 > 0 ? T / 2 : 1;
  unsigned char* base = smem + (size_t)tm.id * mskw_team_bytes<TW, VT>(T);
  int* keys = reinterpret_cast<int*>(base);
  int* pos = reinterpret_cast<int*>(base + al16((size_t)T * 4));
  VT* acc = reinterpret_cast<VT*>(base + al16((size_t)T * 4) * 2);
  ChunkScratch<TW, VT>* csc =
      reinterpret_cast<ChunkScratch<TW, VT>*>(base + al16((size_t)T * 4) * 2 + al16((size_t)half * sizeof(VT)));
  VT* xchg = reinterpret_cast<VT*>(reinterpret_cast<unsigned char*>(csc) + al16(sizeof(ChunkScratch<TW, VT>)));
  const VT* __restrict__ Xx = reinterpret_cast<const VT*>(M.X.vx);
  const VT* __restrict__ Yx = reinterpret_cast<const VT*>(M.Y.vx);
  // values may be read through a permutation (a transpose's values without a gather)
  auto XV = [&](long long p) -> VT { return Xx[M.xperm ? M.xperm[p] : p]; };
  auto YV = [&](long long q) -> VT { return Yx[M.yperm ? M.yperm[q] : q]; };
  const int* __restrict__ Yj = M.Y.cj;
  const int* __restrict__ Xj = M.X.cj;
  VT* __restrict__ out = reinterpret_cast<VT*>(M.out);
  const unsigned lane_lt = (1u << tm.lane) - 1u;
  const int lane_base = (threadIdx.x & 31) & ~(TW - 1);
  const unsigned tbits = (TW == 32) ? 0xffffffffu : ((1u << TW) - 1u);

  const long long team = (long long)blockIdx.x * tm.per_cta + tm.id;
  const long long nteams = (long long)gridDim.x * tm.per_cta;
  for (long long r = team; r < nrows; r += nteams) {
    const long long i = rows[r];
    const long long s0 = M.Sp[i];
    const long long s = M.Sp[i + 1] - s0;
    const long long a0 = rp_at(M.X, i), a1 = rp_at(M.X, i + 1);
    // the first chunk of X(i,:) is fetched before the pattern is keyed, so the
    // two chains of dependent loads overlap
    long long bs = 0;
    int len = 0;
    VT av = VT(0);
    if (a0 + tm.lane < a1) {
      const int j = Xj[a0 + tm.lane];
      bs = rp_at(M.Y, j);
      len = (int)(rp_at(M.Y, j + 1) - bs);
      av = XV(a0 + tm.lane);
    }
    const int pk = (tm.lane < s) ? M.Sj[s0 + tm.lane] : 0;
    for (int x = tm.lane; x < T; x += TW) keys[x] = kEmpty;
    __syncwarp(tm.mask);
    for (long long p = tm.lane; p < s; p += TW) {
      const int slot = lp_insert(keys, tmask, nullptr, -1, p < TW ? pk : M.Sj[s0 + p]);
      if (slot >= 0 && p < half) {
        pos[slot] = (int)p;
        acc[p] = VT(0);
      } else {
        dev_fail(M.status, kDevTableFull, 22, i);
      }
    }
    __syncwarp(tm.mask);
    for (long long c = a0; c < a1; c += TW) {
      if (c != a0) {
        const long long p = c + tm.lane;
        bs = 0;
        len = 0;
        av = VT(0);
        if (p < a1) {
          const int j = Xj[p];
          bs = rp_at(M.Y, j);
          len = (int)(rp_at(M.Y, j + 1) - bs);
          av = XV(p);
        }
      }
      const int nc = (a1 - c) < TW ? (int)(a1 - c) : TW;
      int tot = len;
#pragma unroll
      for (int d = TW / 2; d > 0; d >>= 1) tot += __shfl_xor_sync(tm.mask, tot, d, TW);
      if (2 * tot >= nc * TW) {
        // one Y row per pass; the first TW entries of kU passes load together
        constexpr int kU = 4;
        for (int t0 = 0; t0 < nc; t0 += kU) {
          int key[kU], lent[kU];
          long long bst[kU];
          VT at[kU], yv[kU];
#pragma unroll
          for (int u = 0; u < kU; ++u) {
            const int t = (t0 + u < nc) ? t0 + u : nc - 1;
            bst[u] = __shfl_sync(tm.mask, bs, t, TW);
            const int l = __shfl_sync(tm.mask, len, t, TW);
            at[u] = __shfl_sync(tm.mask, av, t, TW);
            lent[u] = (t0 + u < nc) ? l : 0;
            key[u] = -1;
            yv[u] = VT(0);
            if (tm.lane < lent[u]) {
              key[u] = Yj[bst[u] + tm.lane];
              yv[u] = YV(bst[u] + tm.lane);
            }
          }
#pragma unroll
          for (int u = 0; u < kU; ++u) {
            if (key[u] >= 0) {
              const int slot = lp_find(keys, tmask, key[u]);
              if (slot >= 0) {
                const int q = pos[slot];
                acc[q] = fma_acc(at[u], yv[u], acc[q]);
              }
            }
            for (int x = tm.lane + TW; x < lent[u]; x += TW) {
              const int slot = lp_find(keys, tmask, Yj[bst[u] + x]);
              if (slot >= 0) {
                const int q = pos[slot];
                acc[q] = fma_acc(at[u], YV(bst[u] + x), acc[q]);
              }
            }
            __syncwarp(tm.mask);
          }
        }
      } else {
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
          int q = -1 - tm.lane;   // inactive or masked-out lanes: a distinct negative id
          VT v = VT(0);
          if (x < tot) {
            while (csc->pre[t + 1] <= x) ++t;
            const long long yq = csc->bs[t] + (x - csc->pre[t]);
            const int slot = lp_find(keys, tmask, Yj[yq]);
            if (slot >= 0) {
              q = pos[slot];
              v = csc->av[t] * YV(yq);
            }
          }
          const unsigned grp = (__match_any_sync(tm.mask, q) >> lane_base) & tbits;
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
          if (q >= 0 && leader) acc[q] += v;
          __syncwarp(tm.mask);
        }
      }
    }
    const long long sw = s < half ? s : half;
    for (long long p = tm.lane; p < sw; p += TW) out[s0 + p] = acc[p];
    __syncwarp(tm.mask);
  }
}

// Warp / sub-warp teams on a pattern whose rows are sorted (strictly
// increasing columns, as every C of this library): the table is keyed by the
// column sets of S(i,:) (Section 3.2's 32-column sets), each slot holding the
// set bits and the position of the set's first column in S(i,:), so the place
// of a product's column is base + popcount of the bits below it and a column
// outside the pattern is a missing key or a clear bit.  Products are added as
// in k_masked_warp.
template <int TW, typename VT>
__host__ __device__ size_t mskp_team_bytes(int T) {
  const int half = T / 2 > 0 ? T / 2 : 1;
  return al16((size_t)T * 4) + al16((size_t)T * 8) + al16((size_t)half * sizeof(VT)) +
         al16(sizeof(ChunkScratch<TW, VT>)) + al16((size_t)TW * sizeof(VT));
}

// One row i of S by the team, in its shared memory at base
// (mskp_team_bytes<TW, VT>(2^logT) bytes).
template <int TW, typename VT>
__device__ __forceinline__ void masked_pos_row(const Team<TW>& tm, const MaskedD& M, unsigned char* base, int logT,
                                               const LpHash& hs, long long i) {
  const int T = 1 << logT;
  const int half = T / 2 > 0 ? T / 2 : 1;
  int* keys = reinterpret_cast<int*>(base);
  int2* mb = reinterpret_cast<int2*>(base + al16((size_t)T * 4));   // (set bits, position of the set's first column)
  const size_t tabb = al16((size_t)T * 4) + al16((size_t)T * 8);
  VT* acc = reinterpret_cast<VT*>(base + tabb);
  ChunkScratch<TW, VT>* csc = reinterpret_cast<ChunkScratch<TW, VT>*>(base + tabb + al16((size_t)half * sizeof(VT)));
  VT* xchg = reinterpret_cast<VT*>(reinterpret_cast<unsigned char*>(csc) + al16(sizeof(ChunkScratch<TW, VT>)));
  const VT* __restrict__ Xx = reinterpret_cast<const VT*>(M.X.vx);
  const VT* __restrict__ Yx = reinterpret_cast<const VT*>(M.Y.vx);
  auto XV = [&](long long p) -> VT { return Xx[M.xperm ? M.xperm[p] : p]; };
  auto YV = [&](long long q) -> VT { return Yx[M.yperm ? M.yperm[q] : q]; };
  const int* __restrict__ Yj = M.Y.cj;
  const int* __restrict__ Xj = M.X.cj;
  VT* __restrict__ out = reinterpret_cast<VT*>(M.out);
  const unsigned lane_lt = (1u << tm.lane) - 1u;
  const int lane_base = (threadIdx.x & 31) & ~(TW - 1);
  const unsigned tbits = (TW == 32) ? 0xffffffffu : ((1u << TW) - 1u);

  {
    const long long s0 = M.Sp[i];
    const int s = (int)(M.Sp[i + 1] - s0);
    const long long a0 = rp_at(M.X, i), a1 = rp_at(M.X, i + 1);
    // the first chunk of X(i,:) is fetched before the pattern is keyed
    long long bs = 0;
    int len = 0;
    VT av = VT(0);
    if (a0 + tm.lane < a1) {
      const int j = Xj[a0 + tm.lane];
      bs = rp_at(M.Y, j);
      len = (int)(rp_at(M.Y, j + 1) - bs);
      av = XV(a0 + tm.lane);
    }
    for (int x = tm.lane; x < T; x += TW) {
      keys[x] = kEmpty;
      mb[x] = make_int2(0, 0);
    }
    const int sw = s < half ? s : half;
    for (int x = tm.lane; x < sw; x += TW) acc[x] = VT(0);
    __syncwarp(tm.mask);
    // the pattern's column sets: the lane holding a set's first column claims
    // its slot and records the position; the last lane of each run of one set
    // inside a pass ORs in the run's bits (a segmented OR over the lanes)
    for (int pb = 0; pb < s; pb += TW) {
      const int p = pb + tm.lane;
      const int col = p < s ? M.Sj[s0 + p] : -1;
      int prev = __shfl_up_sync(tm.mask, col, 1, TW);
      if (tm.lane == 0) prev = pb > 0 ? M.Sj[s0 + pb - 1] : -1;
      const int set = col >= 0 ? (col >> 5) : -1 - tm.lane;
      if (col >= 0 && p > 0 && prev >= col) dev_fail(M.status, kDevBadIndex, 29, i);   // not sorted
      unsigned bits = col >= 0 ? (1u << (col & 31)) : 0u;
#pragma unroll
      for (int d = 1; d < TW; d <<= 1) {
        const unsigned y = __shfl_up_sync(tm.mask, bits, d, TW);
        const int ys = __shfl_up_sync(tm.mask, set, d, TW);
        if (tm.lane >= d && ys == set) bits |= y;
      }
      const int next_set = __shfl_down_sync(tm.mask, set, 1, TW);
      const bool last = col >= 0 && (tm.lane == TW - 1 || p + 1 >= s || next_set != set);
      const bool head = col >= 0 && (p == 0 || (prev >> 5) != set);
      if (head) {
        int fresh = 0;
        const int slot = slot_insert<1>(keys, hs, set, &fresh);
        if (slot >= 0) mb[slot].y = p;
        else dev_fail(M.status, kDevTableFull, 30, i);
      }
      __syncwarp(tm.mask);
      if (last) {
        const int slot = key_slot(keys, hs, set);
        if (slot >= 0) mb[slot].x |= (int)bits;
      }
      __syncwarp(tm.mask);
    }
    auto pos_of = [&](int c) -> int {
      const int slot = key_slot(keys, hs, c >> 5);
      if (slot < 0) return -1;
      const int2 e = mb[slot];
      const unsigned m = (unsigned)e.x;
      if (!((m >> (c & 31)) & 1u)) return -1;
      return e.y + __popc(m & ((1u << (c & 31)) - 1u));
    };
    for (long long c = a0; c < a1; c += TW) {
      if (c != a0) {
        const long long p = c + tm.lane;
        bs = 0;
        len = 0;
        av = VT(0);
        if (p < a1) {
          const int j = Xj[p];
          bs = rp_at(M.Y, j);
          len = (int)(rp_at(M.Y, j + 1) - bs);
          av = XV(p);
        }
      }
      const int nc = (a1 - c) < TW ? (int)(a1 - c) : TW;
      int tot = len;
#pragma unroll
      for (int d = TW / 2; d > 0; d >>= 1) tot += __shfl_xor_sync(tm.mask, tot, d, TW);
      if (2 * tot >= nc * TW) {
        constexpr int kU = 4;
        for (int t0 = 0; t0 < nc; t0 += kU) {
          int key[kU], lent[kU];
          long long bst[kU];
          VT at[kU], yv[kU];
#pragma unroll
          for (int u = 0; u < kU; ++u) {
            const int t = (t0 + u < nc) ? t0 + u : nc - 1;
            bst[u] = __shfl_sync(tm.mask, bs, t, TW);
            const int l = __shfl_sync(tm.mask, len, t, TW);
            at[u] = __shfl_sync(tm.mask, av, t, TW);
            lent[u] = (t0 + u < nc) ? l : 0;
            key[u] = -1;
            yv[u] = VT(0);
            if (tm.lane < lent[u]) {
              key[u] = Yj[bst[u] + tm.lane];
              yv[u] = YV(bst[u] + tm.lane);
            }
          }
#pragma unroll
          for (int u = 0; u < kU; ++u) {
            if (key[u] >= 0) {
              const int o = pos_of(key[u]);
              if (o >= 0 && o < half) acc[o] = fma_acc(at[u], yv[u], acc[o]);
            }
            for (int x = tm.lane + TW; x < lent[u]; x += TW) {
              const int o = pos_of(Yj[bst[u] + x]);
              if (o >= 0 && o < half) acc[o] = fma_acc(at[u], YV(bst[u] + x), acc[o]);
            }
            __syncwarp(tm.mask);
          }
        }
      } else {
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
          int q = -1 - tm.lane;   // inactive or masked-out lanes: a distinct negative id
          VT v = VT(0);
          if (x < tot) {
            while (csc->pre[t + 1] <= x) ++t;
            const long long yq = csc->bs[t] + (x - csc->pre[t]);
            const int o = pos_of(Yj[yq]);
            if (o >= 0 && o < half) {
              q = o;
              v = csc->av[t] * YV(yq);
            }
          }
          const unsigned grp = (__match_any_sync(tm.mask, q) >> lane_base) & tbits;
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
          if (q >= 0 && leader) acc[q] += v;
          __syncwarp(tm.mask);
        }
        __syncwarp(tm.mask);
      }
    }
    for (int p = tm.lane; p < sw; p += TW) out[s0 + p] = acc[p];
    __syncwarp(tm.mask);
  }
}

template <int TW, typename VT>
__global__ void __launch_bounds__(256, 4) k_masked_pos(MaskedD M, const int* __restrict__ rows, long long nrows,
                                                       int logT) {
  extern __shared__ __align__(16) unsigned char smem[];
  Team<TW> tm;
  const LpHash hs(logT, M.hash_mode);
  unsigned char* base = smem + (size_t)tm.id * mskp_team_bytes<TW, VT>(1 << logT);
  const long long team = (long long)blockIdx.x * tm.per_cta + tm.id;
  const long long nteams = (long long)gridDim.x * tm.per_cta;
  for (long long r = team; r < nrows; r += nteams) masked_pos_row<TW, VT>(tm, M, base, logT, hs, rows[r]);
}

// Warp teams on a sorted pattern whose row S(i,:) spans at most kMwLimit
// column sets (first to last column): the sets of S(i,:) are kept in a bitmap
// window addressed directly by set index, each word with the position of its
// first column in S(i,:), so the place of a product's column is that position
// + the set bits below it, and a column outside the pattern meets a clear bit
// (the words of the row are cleared after it).  No hashing and no probing;
// wider rows take the hashed path (masked_pos_row) in the same shared memory.
constexpr int kMwLimit = 1344;
constexpr int kMwTeams = 4;

template <typename VT>
__host__ __device__ size_t mskw_team_bytes(int T) {
  const int half = T / 2 > 0 ? T / 2 : 1;
  const size_t wb = al16((size_t)kMwLimit * 4) + al16((size_t)kMwLimit * 2) + al16((size_t)half * sizeof(VT)) +
                    al16(sizeof(ChunkScratch<32, VT>)) + al16(32 * sizeof(VT));
  const size_t hp = mskp_team_bytes<32, VT>(T);
  return wb > hp ? wb : hp;
}

template <typename VT>
__global__ void __launch_bounds__(32 * kMwTeams, 5) k_masked_win(MaskedD M, const int* __restrict__ rows,
                                                                 long long nrows, int logT) {
  extern __shared__ __align__(16) unsigned char smem[];
  Team<32> tm;
  const int T = 1 << logT;
  const int half = T / 2 > 0 ? T / 2 : 1;
  const LpHash hs(logT, M.hash_mode);
  unsigned char* base = smem + (size_t)tm.id * mskw_team_bytes<VT>(T);
  unsigned* wbits = reinterpret_cast<unsigned*>(base);
  unsigned short* wpos = reinterpret_cast<unsigned short*>(base + al16((size_t)kMwLimit * 4));
  VT* acc = reinterpret_cast<VT*>(base + al16((size_t)kMwLimit * 4) + al16((size_t)kMwLimit * 2));
  ChunkScratch<32, VT>* csc =
      reinterpret_cast<ChunkScratch<32, VT>*>(reinterpret_cast<unsigned char*>(acc) + al16((size_t)half * sizeof(VT)));
  VT* xchg = reinterpret_cast<VT*>(reinterpret_cast<unsigned char*>(csc) + al16(sizeof(ChunkScratch<32, VT>)));
  const VT* __restrict__ Xx = reinterpret_cast<const VT*>(M.X.vx);
  const VT* __restrict__ Yx = reinterpret_cast<const VT*>(M.Y.vx);
  auto XV = [&](long long p) -> VT { return Xx[M.xperm ? M.xperm[p] : p]; };
  auto YV = [&](long long q) -> VT { return Yx[M.yperm ? M.yperm[q] : q]; };
  const int* __restrict__ Yj = M.Y.cj;
  const int* __restrict__ Xj = M.X.cj;
  VT* __restrict__ out = reinterpret_cast<VT*>(M.out);
  const int lane = tm.lane;
  const unsigned lane_lt = (1u << lane) - 1u;
  const unsigned full = 0xffffffffu;
  bool clean = false;
  const long long team = (long long)blockIdx.x * tm.per_cta + tm.id;
  const long long nteams = (long long)gridDim.x * tm.per_cta;
  for (long long r = team; r < nrows; r += nteams) {
    const long long i = rows[r];
    const long long s0 = M.Sp[i];
    const int s = (int)(M.Sp[i + 1] - s0);
    if (s <= 0) continue;
    const unsigned smin = (unsigned)M.Sj[s0] >> 5, smax = (unsigned)M.Sj[s0 + s - 1] >> 5;
    if (smin > smax || smax - smin >= (unsigned)kMwLimit || s > half) {
      masked_pos_row<32, VT>(tm, M, base, logT, hs, i);
      clean = false;
      __syncwarp();
      continue;
    }
    const unsigned span = smax - smin + 1u;
    const long long a0 = rp_at(M.X, i), a1 = rp_at(M.X, i + 1);
    // the first chunk of X(i,:) is fetched before the pattern is placed
    long long bs = 0;
    int len = 0;
    VT av = VT(0);
    if (a0 + lane < a1) {
      const int j = Xj[a0 + lane];
      bs = rp_at(M.Y, j);
      len = (int)(rp_at(M.Y, j + 1) - bs);
      av = XV(a0 + lane);
    }
    if (!clean) {
      uint4* c4 = reinterpret_cast<uint4*>(wbits);
      for (int x = lane; x < kMwLimit / 4; x += 32) c4[x] = make_uint4(0u, 0u, 0u, 0u);
      clean = true;
      __syncwarp();
    }
    for (int x = lane; x < s; x += 32) acc[x] = VT(0);
    // the pattern's sets: the first column of each set records its position,
    // then every column sets its bit
    for (int pb = 0; pb < s; pb += 32) {
      const int p = pb + lane;
      const int col = p < s ? M.Sj[s0 + p] : -1;
      int prev = __shfl_up_sync(full, col, 1);
      if (lane == 0) prev = pb > 0 ? M.Sj[s0 + pb - 1] : -1;
      const unsigned w = (unsigned)(col >> 5) - smin;
      if (col >= 0 && p > 0 && prev >= col) dev_fail(M.status, kDevBadIndex, 40, i);   // not sorted
      const bool ok = col >= 0 && w < span;
      if (ok && (p == 0 || (prev >> 5) != (col >> 5))) wpos[w] = (unsigned short)p;
      __syncwarp();
      if (ok) atomicOr(wbits + w, 1u << (col & 31));
      __syncwarp();
    }
    auto pos_of = [&](int c) -> int {
      const unsigned w = (unsigned)(c >> 5) - smin;
      if (w >= span) return -1;
      const unsigned m = wbits[w];
      const unsigned bit = 1u << (c & 31);
      if (!(m & bit)) return -1;
      return (int)wpos[w] + __popc(m & (bit - 1u));
    };
    for (long long c = a0; c < a1; c += 32) {
      if (c != a0) {
        const long long p = c + lane;
        bs = 0;
        len = 0;
        av = VT(0);
        if (p < a1) {
          const int j = Xj[p];
          bs = rp_at(M.Y, j);
          len = (int)(rp_at(M.Y, j + 1) - bs);
          av = XV(p);
        }
      }
      const int nc = (a1 - c) < 32 ? (int)(a1 - c) : 32;
      const int tot = (int)__reduce_add_sync(full, (unsigned)len);
      if (2 * tot >= nc * 32) {
        constexpr int kU = 4;
        for (int t0 = 0; t0 < nc; t0 += kU) {
          int key[kU], lent[kU];
          long long bst[kU];
          VT at[kU], yv[kU];
#pragma unroll
          for (int u = 0; u < kU; ++u) {
            const int t = (t0 + u < nc) ? t0 + u : nc - 1;
            bst[u] = __shfl_sync(full, bs, t);
            const int l = __shfl_sync(full, len, t);
            at[u] = __shfl_sync(full, av, t);
            lent[u] = (t0 + u < nc) ? l : 0;
            key[u] = -1;
            yv[u] = VT(0);
            if (lane < lent[u]) {
              key[u] = Yj[bst[u] + lane];
              yv[u] = YV(bst[u] + lane);
            }
          }
#pragma unroll
          for (int u = 0; u < kU; ++u) {
            if (key[u] >= 0) {
              const int o = pos_of(key[u]);
              if (o >= 0) acc[o] = fma_acc(at[u], yv[u], acc[o]);
            }
            for (int x = lane + 32; x < lent[u]; x += 32) {
              const int o = pos_of(Yj[bst[u] + x]);
              if (o >= 0) acc[o] = fma_acc(at[u], YV(bst[u] + x), acc[o]);
            }
            __syncwarp();
          }
        }
      } else {
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
          int q = -1 - lane;
          VT v = VT(0);
          if (x < tot) {
            while (csc->pre[t + 1] <= x) ++t;
            const long long yq = csc->bs[t] + (x - csc->pre[t]);
            const int o = pos_of(Yj[yq]);
            if (o >= 0) {
              q = o;
              v = csc->av[t] * YV(yq);
            }
          }
          const unsigned grp = __match_any_sync(full, q);
          const bool leader = (grp & lane_lt) == 0;
          if (__any_sync(full, __popc(grp) > 1)) {
            xchg[lane] = v;
            __syncwarp();
            if (leader) {
              unsigned rest = grp & ~(1u << lane);
              while (rest) {
                const int o = __ffs(rest) - 1;
                rest &= rest - 1u;
                v += xchg[o];
              }
            }
            __syncwarp();
          }
          if (q >= 0 && leader) acc[q] += v;
          __syncwarp();
        }
        __syncwarp();
      }
    }
    for (int x = lane; x < s; x += 32) out[s0 + x] = acc[x];
    // clear the row's words
    for (int pb = 0; pb < s; pb += 32) {
      const int p = pb + lane;
      if (p < s) {
        const unsigned w = (unsigned)(M.Sj[s0 + p] >> 5) - smin;
        if (w < span) wbits[w] = 0u;
      }
    }
    __syncwarp();
  }
}

// Rows of S whose columns are not strictly increasing (one warp per row).
__global__ void k_pattern_unsorted(MaskedD M, long long nrows, unsigned long long* count) {
  const int lane = threadIdx.x & 31;
  const long long warp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
  for (long long i = warp; i < nrows; i += nwarps) {
    const long long s0 = M.Sp[i], s1 = M.Sp[i + 1];
    bool bad = false;
    for (long long p = s0 + 1 + lane; p < s1; p += 32) bad |= M.Sj[p] <= M.Sj[p - 1];
    if (__any_sync(0xffffffffu, bad) && lane == 0) atomicAdd(count, 1ull);
  }
}

// One thread per row for rows with at most kT1MaxKeys pattern entries and a
// few products (Thread-Sequential with a team of one, Section 3.1.1): the
// pattern's keys and their accumulators stay in registers, a product is
// matched by comparing with every key, and all rows of the bin are in flight
// at once, which hides the chains of dependent loads of short rows.
// STAGED = false: one product at a time (rows whose Y rows hold one or two
// entries); STAGED = true: loads staged in groups (longer Y rows).
// The matching key is found with integer compares and the product goes to one
// accumulator in shared memory: a predicated FMA per key would issue
// kT1MaxKeys FP64 instructions per product on the scarce FP64 pipe.
template <typename VT, bool STAGED>
__global__ void __launch_bounds__(256, 4) k_masked_thread(MaskedD M, const int* __restrict__ rows, long long nrows) {
  __shared__ VT accs[kT1MaxKeys][256];
  const VT* __restrict__ Xx = reinterpret_cast<const VT*>(M.X.vx);
  const VT* __restrict__ Yx = reinterpret_cast<const VT*>(M.Y.vx);
  // values may be read through a permutation (a transpose's values without a gather)
  auto XV = [&](long long p) -> VT { return Xx[M.xperm ? M.xperm[p] : p]; };
  auto YV = [&](long long q) -> VT { return Yx[M.yperm ? M.yperm[q] : q]; };
  const int* __restrict__ Yj = M.Y.cj;
  const int* __restrict__ Xj = M.X.cj;
  VT* __restrict__ out = reinterpret_cast<VT*>(M.out);
  const int tid = threadIdx.x;
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x; r < nrows; r += stride) {
    const long long i = rows[r];
    const long long s0 = M.Sp[i];
    const int s = (int)(M.Sp[i + 1] - s0);
    const long long a0 = rp_at(M.X, i), a1 = rp_at(M.X, i + 1);
    int key[kT1MaxKeys];
#pragma unroll
    for (int t = 0; t < kT1MaxKeys; ++t) {
      key[t] = (t < s) ? M.Sj[s0 + t] : -1;
      accs[t][tid] = VT(0);
    }
    auto add = [&](int c, VT a, VT y) {
      int hit = -1;
#pragma unroll
      for (int t = 0; t < kT1MaxKeys; ++t) hit = (key[t] == c) ? t : hit;
      if (hit >= 0) accs[hit][tid] = fma_acc(a, y, accs[hit][tid]);
    };
    if (!STAGED) {
      for (long long p = a0; p < a1; ++p) {
        const int j = Xj[p];
        const VT a = XV(p);
        const long long b0 = rp_at(M.Y, j), b1 = rp_at(M.Y, j + 1);
        for (long long q = b0; q < b1; ++q) add(Yj[q], a, YV(q));
      }
    }
    // staged loads: 4 entries of X(i,:), then their Y ranges, then the Y
    // entries 4 at a time, so each thread keeps several loads in flight
    constexpr int kX = 4, kQ = 4;
    for (long long c0 = STAGED ? a0 : a1; c0 < a1; c0 += kX) {
      int j[kX];
      VT a[kX];
      long long b0[kX], b1[kX];
#pragma unroll
      for (int u = 0; u < kX; ++u) {
        const bool ok = c0 + u < a1;
        j[u] = ok ? Xj[c0 + u] : -1;
        a[u] = ok ? XV(c0 + u) : VT(0);
      }
#pragma unroll
      for (int u = 0; u < kX; ++u) {
        b0[u] = j[u] >= 0 ? rp_at(M.Y, j[u]) : 0;
        b1[u] = j[u] >= 0 ? rp_at(M.Y, j[u] + 1) : 0;
      }
#pragma unroll
      for (int u = 0; u < kX; ++u) {
        for (long long q = b0[u]; q < b1[u]; q += kQ) {
          int c[kQ];
          VT y[kQ];
#pragma unroll
          for (int v = 0; v < kQ; ++v) {
            const bool ok = q + v < b1[u];
            c[v] = ok ? Yj[q + v] : -1;
            y[v] = ok ? YV(q + v) : VT(0);
          }
#pragma unroll
          for (int v = 0; v < kQ; ++v) add(c[v], a[u], y[v]);
        }
      }
    }
#pragma unroll
    for (int t = 0; t < kT1MaxKeys; ++t)
      if (t < s) out[s0 + t] = accs[t][tid];
  }
}

// work_i = sum over j in X(i,:) of |Y(j,:)|, then the bin from (|S(i,:)|,
// work_i); -1 for rows without work and for invalid rows (reported when
// `report`, which turns the call's status into SPGEMM_ERR_BAD_INDEX).
__device__ __forceinline__ int masked_row_bin(const MaskedD& M, long long i, const BinCfg& cfg, bool report) {
  long long w = 0;
  const long long a0 = rp_at(M.X, i), a1 = rp_at(M.X, i + 1);
  bool ok = a0 >= 0 && a0 <= a1 && a1 <= M.X.nnz;
  for (long long p = a0; ok && p < a1; ++p) {
    const int j = M.X.cj[p];
    if ((unsigned long long)(unsigned)j >= (unsigned long long)M.X.ncols) {
      ok = false;
      break;
    }
    const long long bs = rp_at(M.Y, j), be = rp_at(M.Y, j + 1);
    if (bs < 0 || bs > be || be > M.Y.nnz) {
      ok = false;
      break;
    }
    w += be - bs;
  }
  if (!ok) {
    if (report) dev_fail(M.status, kDevBadIndex, 21, i);
    return -1;
  }
  const long long s = M.Sp[i + 1] - M.Sp[i];
  int bin = choose_bin(s, w > 0 ? w : (s > 0 ? 1 : 0), M.Y.ncols, (M.Y.ncols + 31) >> 5, cfg);
  if (bin_cls(bin) == kClsNone) return -1;
  // thread-per-row rows: staged loads once Y rows average more than 2 entries
  if (bin_cls(bin) == kClsT1 && w > 2 * (a1 - a0)) bin = bin_id(kClsT1, 1);
  return bin;
}

// Stable binning of the pattern's rows (as the product's row binning).
__global__ void __launch_bounds__(kBinThreads) k_masked_bin_count(MaskedD M, long long nrows, BinCfg cfg,
                                                                  unsigned long long* hist, long long* bcnt,
                                                                  long long nblk) {
  __shared__ unsigned long long h[kNumBins];
  for (int t = threadIdx.x; t < kNumBins; t += blockDim.x) h[t] = 0ull;
  __syncthreads();
  const long long r0 = (long long)blockIdx.x * kBinRows;
  const long long r1 = r0 + kBinRows < nrows ? r0 + kBinRows : nrows;
  bin_block_count(r0, r1, [&](long long i) { return masked_row_bin(M, i, cfg, true); }, h);
  __syncthreads();
  for (int t = threadIdx.x; t < kNumBins; t += blockDim.x) {
    bcnt[(long long)t * nblk + blockIdx.x] = (long long)h[t];
    if (h[t]) atomicAdd(&hist[t], h[t]);
  }
}

__global__ void __launch_bounds__(kBinThreads) k_masked_bin_list(MaskedD M, long long nrows, BinCfg cfg,
                                                                 const unsigned long long* cursor,
                                                                 const long long* bofs, long long nblk, int* rows) {
  __shared__ long long run[kNumBins];
  __shared__ int wcnt[kBinThreads / 32][kNumBins];
  for (int t = threadIdx.x; t < kNumBins; t += blockDim.x) {
    run[t] = (long long)cursor[t] + bofs[(long long)t * nblk + blockIdx.x] - bofs[(long long)t * nblk];
    for (int w = 0; w < kBinThreads / 32; ++w) wcnt[w][t] = 0;
  }
  __syncthreads();
  const long long r0 = (long long)blockIdx.x * kBinRows;
  const long long r1 = r0 + kBinRows < nrows ? r0 + kBinRows : nrows;
  bin_block_list(r0, r1, [&](long long i) { return masked_row_bin(M, i, cfg, false); }, run, wcnt, rows);
}

// ---------------------------------------------------------------- masked count
// Structural counts on the compressed Y (symbolic-only use of the two-phase
// method for graph analytics, Section 2; compression, Section 3.2):
// count_i = sum over l in S(i,:) of |{ j : (i,j) in X, (j,l) in Y }|.  Y's
// rows become runs of (column-set index, bits); S(i,:) becomes a table of
// (set index, bits); each compressed product adds popcount(Y bits & S bits).

// Runs of equal column-set index per row of Y (cnt[j] = compressed length).
__global__ void __launch_bounds__(256) k_mc_compress_count(MatD Y, long long* cnt, DevStatus* st) {
  Team<8> tm;
  const long long nteams = (long long)gridDim.x * tm.per_cta;
  for (long long j = (long long)blockIdx.x * tm.per_cta + tm.id; j < Y.nrows; j += nteams) {
    const long long s = rp_at(Y, j), e = rp_at(Y, j + 1);
    long long c = 0;
    if (s < 0 || s > e || e > Y.nnz) {
      if (tm.lane == 0) {
        dev_fail(st, kDevBadIndex, 50, j);
        cnt[j] = 0;
      }
      continue;
    }
    for (long long p = s + tm.lane; p < e; p += 8) {
      const int col = Y.cj[p];
      if ((unsigned long long)(unsigned)col >= (unsigned long long)Y.ncols) dev_fail(st, kDevBadIndex, 51, j);
      if (p == s || (col >> 5) != (Y.cj[p - 1] >> 5)) ++c;
    }
    c = warp_team_sum<8>(tm, c);
    if (tm.lane == 0) cnt[j] = c;
  }
}

// The runs themselves: csi and the OR of their bits (a run is stored by the
// chunk where it starts and ORed by later chunks, so cs needs no clearing).
__global__ void __launch_bounds__(256) k_mc_compress_fill(MatD Y, const long long* __restrict__ Ycp, int* csi,
                                                          unsigned* cs) {
  Team<8> tm;
  const long long nteams = (long long)gridDim.x * tm.per_cta;
  const int base_lane = (threadIdx.x & 31) & ~7;
  for (long long j = (long long)blockIdx.x * tm.per_cta + tm.id; j < Y.nrows; j += nteams) {
    const long long s = rp_at(Y, j), e = rp_at(Y, j + 1);
    if (s < 0 || s > e || e > Y.nnz) continue;
    long long run = Ycp[j] - 1;
    for (long long c0 = s; c0 < e; c0 += 8) {
      const long long p = c0 + tm.lane;
      const bool valid = p < e;
      const int col = valid ? Y.cj[p] : 0;
      const bool head = valid && (p == s || (col >> 5) != (Y.cj[p - 1] >> 5));
      const unsigned hb = (__ballot_sync(tm.mask, head) >> base_lane) & 0xffu;
      const unsigned le = (2u << tm.lane) - 1u;
      const long long ridx = run + __popc(hb & le);
      if (head) csi[ridx] = col >> 5;
      unsigned v = valid ? (1u << (col & 31)) : 0u;
      int f = (head || tm.lane == 0) ? 1 : 0;
#pragma unroll
      for (int d = 1; d < 8; d <<= 1) {
        const unsigned vu = __shfl_up_sync(tm.mask, v, d, 8);
        const int fu = __shfl_up_sync(tm.mask, f, d, 8);
        if (tm.lane >= d && !f) {
          v |= vu;
          f = fu;
        }
      }
      const bool next_head = (tm.lane + 1 < 8) && ((hb >> (tm.lane + 1)) & 1u);
      const bool tail = valid && (tm.lane == 7 || p + 1 >= e || next_head);
      if (tail) {
        if (hb & le) cs[ridx] = v;
        else atomicOr(cs + ridx, v);
      }
      run += __popc(hb);
      __syncwarp(tm.mask);
    }
  }
}

constexpr int kMcWarpMaxRow = kMcBigRow;   // S rows up to this size: warp teams with a hash table
constexpr int kMcWarpSlots = 2048;    // table slots of the largest warp tables (keys + bits: 16 KB)
constexpr int kMcSmallSlots = 256;    // most rows: tables of up to 256 slots (2 KB per warp)

// Longest row of S (int64 row pointers).
__global__ void k_row_len_max(const long long* __restrict__ Sp, long long n, unsigned long long* out) {
  unsigned long long m = 0;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const long long l = Sp[i + 1] - Sp[i];
    m = l > (long long)m ? (unsigned long long)l : m;
  }
  m = __reduce_max_sync(0xffffffffu, (unsigned)(m > 0xffffffffull ? 0xffffffffull : m));
  if ((threadIdx.x & 31) == 0) atomicMax(out, m);
}

// Row classes of the masked count: 0 = table of at most kMcSmallSlots slots,
// 1 = larger warp tables, 2 = rows of at least cta_from entries (a CTA each,
// S(i,:) as a bitmap: cta_from is kMcSmallSlots / 2 + 1 when that bitmap fits
// shared memory, so no row needs the 16 KB warp tables, else kMcWarpMaxRow + 1).
// Rows of each class are listed (any order) and fetched by the teams from a
// shared counter: the heavy rows of skewed graphs have indices with many
// trailing zero bits, which a fixed row-to-team stride would send to a few
// teams.  Empty rows get their count here.  cnt: [0..2] list lengths.
__device__ __forceinline__ int mc_class(long long ns, long long cta_from) {
  if (ns >= cta_from) return 2;
  return 2 * ns > kMcSmallSlots ? 1 : 0;
}

__global__ void k_mc_classify(MaskedD M, int* lists, unsigned long long* cnt, long long* counts, long long cta_from) {
  const long long n = M.X.nrows;
  const long long stride = (long long)gridDim.x * blockDim.x;
  const int lane = threadIdx.x & 31;
  for (long long b0 = (long long)blockIdx.x * blockDim.x; b0 < n; b0 += stride) {
    const long long i = b0 + threadIdx.x;
    int c = -1;
    if (i < n) {
      const long long ns = M.Sp[i + 1] - M.Sp[i];
      if (ns <= 0) counts[i] = 0;
      else c = mc_class(ns, cta_from);
    }
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const unsigned m = __ballot_sync(0xffffffffu, c == k);
      if (m == 0u) continue;
      const int leader = __ffs(m) - 1;
      unsigned long long base = 0;
      if (lane == leader) base = atomicAdd(cnt + k, (unsigned long long)__popc(m));
      base = __shfl_sync(0xffffffffu, base, leader);
      if (c == k) lists[(long long)k * n + (long long)base + __popc(m & ((1u << lane) - 1u))] = (int)i;
    }
  }
}

// Warp per listed row of S whose table (2 slots per entry, a power of two)
// holds at most SLOTS slots; rows are taken CHUNK at a time from *next.
template <int SLOTS, int WARPS, int CHUNK>
__global__ void __launch_bounds__(WARPS * 32) k_masked_count_warp(MaskedD M, const long long* __restrict__ Ycp,
                                                                  const int* __restrict__ csi,
                                                                  const unsigned* __restrict__ cs,
                                                                  long long* __restrict__ counts,
                                                                  const int* __restrict__ list,
                                                                  const unsigned long long* nlist,
                                                                  unsigned long long* next) {
  extern __shared__ __align__(16) unsigned char smem[];
  Team<32> tm;
  int* keys = reinterpret_cast<int*>(smem) + (size_t)tm.id * 2 * SLOTS;
  unsigned* bits = reinterpret_cast<unsigned*>(keys + SLOTS);
  __shared__ int pre_s[WARPS][33];
  __shared__ long long qs_s[WARPS][32];
  int* pre = pre_s[tm.id];
  long long* qsv = qs_s[tm.id];
  const unsigned long long nrows = *nlist;
  for (;;) {
    unsigned long long base = 0;
    if (tm.lane == 0) base = atomicAdd(next, (unsigned long long)CHUNK);
    base = __shfl_sync(0xffffffffu, base, 0);
    if (base >= nrows) break;
    const unsigned long long end = base + CHUNK < nrows ? base + CHUNK : nrows;
    for (unsigned long long r = base; r < end; ++r) {
      const long long i = list[r];
      const long long s0 = M.Sp[i], s1 = M.Sp[i + 1];
      const long long ns = s1 - s0;
      int logT = 1;
      while ((1ll << logT) < 2 * ns) ++logT;
      const int T = 1 << logT;
      if (T > SLOTS) {   // not this class: a malformed list
        if (tm.lane == 0) dev_fail(M.status, kDevTableFull, 57, i);
        continue;
      }
      const LpHash hs(logT, M.hash_mode);
      for (int x = tm.lane; x < T; x += 32) {
        keys[x] = kEmpty;
        bits[x] = 0u;
      }
      __syncwarp();
      int fresh = 0;
      for (long long p = s0 + tm.lane; p < s1; p += 32) {
        const int l = M.Sj[p];
        if ((unsigned long long)(unsigned)l >= (unsigned long long)M.Y.ncols) {
          dev_fail(M.status, kDevBadIndex, 52, i);
          continue;
        }
        const int slot = slot_insert<1>(keys, hs, l >> 5, &fresh);
        if (slot >= 0) atomicOr(bits + slot, 1u << (l & 31));
        else dev_fail(M.status, kDevTableFull, 53, i);
      }
      __syncwarp();
      long long cnt = 0;
      const long long a0 = rp_at(M.X, i), a1 = rp_at(M.X, i + 1);
      for (long long c = a0; c < a1; c += 32) {
        const long long p = c + tm.lane;
        long long q0 = 0;
        int ql = 0;
        if (p < a1) {
          const int j = M.X.cj[p];
          if ((unsigned long long)(unsigned)j < (unsigned long long)M.Y.nrows) {
            q0 = Ycp[j];
            ql = (int)(Ycp[j + 1] - q0);
          } else {
            dev_fail(M.status, kDevBadIndex, 54, i);
          }
        }
        int ex = ql;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
          const int y = __shfl_up_sync(0xffffffffu, ex, d);
          if (tm.lane >= d) ex += y;
        }
        const int tot = __shfl_sync(0xffffffffu, ex, 31);
        pre[tm.lane] = ex - ql;
        qsv[tm.lane] = q0;
        if (tm.lane == 0) pre[32] = tot;
        __syncwarp();
        int t = 0;
        for (int xb = 0; xb < tot; xb += 4 * 32) {
          int key[4];
          unsigned m[4];
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            const int x = xb + u * 32 + tm.lane;
            key[u] = -1;
            m[u] = 0u;
            if (x < tot) {
              while (pre[t + 1] <= x) ++t;
              const long long q = qsv[t] + (x - pre[t]);
              key[u] = csi[q];
              m[u] = cs[q];
            }
          }
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            if (key[u] >= 0) {
              const int slot = key_slot(keys, hs, key[u]);
              if (slot >= 0) cnt += __popc(m[u] & bits[slot]);
            }
          }
        }
        __syncwarp();
      }
#pragma unroll
      for (int d = 16; d > 0; d >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, d);
      if (tm.lane == 0) counts[i] = cnt;
      __syncwarp();
    }
  }
}

// CTA per listed row of S (class 2 above): S(i,:) as a bitmap of
// ceil(k / 32) words in shared memory, set and cleared by its own entries.
__global__ void __launch_bounds__(256) k_masked_count_cta(MaskedD M, const long long* __restrict__ Ycp,
                                                          const int* __restrict__ csi,
                                                          const unsigned* __restrict__ cs,
                                                          long long* __restrict__ counts, long long kw,
                                                          const int* __restrict__ list,
                                                          const unsigned long long* nlist,
                                                          unsigned long long* next) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ long long scan_scratch[33];
  __shared__ ChunkScratch<256, int> csc;
  __shared__ long long row_s;
  Team<256> tm;
  unsigned* bm = reinterpret_cast<unsigned*>(smem);
  for (long long w = tm.lane; w < kw; w += 256) bm[w] = 0u;
  const unsigned long long nrows = *nlist;
  for (;;) {
    if (tm.lane == 0) {
      const unsigned long long r = atomicAdd(next, 1ull);
      row_s = r < nrows ? (long long)list[r] : -1;
    }
    __syncthreads();
    const long long i = row_s;
    __syncthreads();
    if (i < 0) break;
    const long long s0 = M.Sp[i], s1 = M.Sp[i + 1];
    for (long long p = s0 + tm.lane; p < s1; p += 256) {
      const int l = M.Sj[p];
      if ((unsigned long long)(unsigned)l < (unsigned long long)M.Y.ncols) atomicOr(bm + (l >> 5), 1u << (l & 31));
      else dev_fail(M.status, kDevBadIndex, 55, i);
    }
    __syncthreads();
    long long cnt = 0;
    const long long a0 = rp_at(M.X, i), a1 = rp_at(M.X, i + 1);
    auto range = [&](int j, long long* bs, long long* be) {
      if ((unsigned long long)(unsigned)j < (unsigned long long)M.Y.nrows) {
        *bs = Ycp[j];
        *be = Ycp[j + 1];
      } else {
        dev_fail(M.status, kDevBadIndex, 56, i);
        *bs = *be = 0;
      }
    };
    auto aval = [&](long long) { return 0; };
    auto body = [&](long long q, int) { cnt += __popc(cs[q] & bm[csi[q]]); };
    auto pf = [&](long long q) {
      prefetch_l1(csi + q);
      prefetch_l1(cs + q);
    };
    for_each_product<256, int>(tm, &csc, scan_scratch, M.X.cj, a0, a1, range, aval, body, pf);
    long long tot = team_sum<256>(tm, cnt, scan_scratch);
    if (tm.lane == 0) counts[i] = tot;
    for (long long p = s0 + tm.lane; p < s1; p += 256) {
      const int l = M.Sj[p];
      if ((unsigned long long)(unsigned)l < (unsigned long long)M.Y.ncols) bm[l >> 5] = 0u;
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------- transpose
__global__ void k_tr_count(MatD A, unsigned long long* cnt, DevStatus* st) {
  const long long stride = (long long)gridDim.x * blockDim.x;
  // the rows must cover the entries exactly: every counted entry is scattered
  // once, so no slot of the transpose is left unwritten
  if (blockIdx.x == 0 && threadIdx.x == 0 && (rp_at(A, 0) != 0 || rp_at(A, A.nrows) != A.nnz))
    dev_fail(st, kDevBadIndex, 34, rp_at(A, A.nrows));
  for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < A.nnz; p += stride) {
    const int c = A.cj[p];
    if ((unsigned long long)(unsigned)c < (unsigned long long)A.ncols) atomicAdd(&cnt[c], 1ull);
    else dev_fail(st, kDevBadIndex, 32, p);
  }
}

__global__ void k_tr_scatter(MatD A, const long long* Atp, unsigned long long* cursor, int* trow, long long* tperm,
                             DevStatus* st) {
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < A.nrows; i += stride) {
    const long long a0 = rp_at(A, i), a1 = rp_at(A, i + 1);
    if (a0 < 0 || a0 > a1 || a1 > A.nnz) {
      dev_fail(st, kDevBadIndex, 31, i);
      continue;
    }
    for (long long p = a0; p < a1; ++p) {
      const int c = A.cj[p];
      if ((unsigned long long)(unsigned)c >= (unsigned long long)A.ncols) {
        dev_fail(st, kDevBadIndex, 30, i);
        continue;
      }
      const long long q = Atp[c] + (long long)atomicAdd(&cursor[c], 1ull);
      if (q >= Atp[c + 1]) {   // overlapping row ranges: more entries than counted
        dev_fail(st, kDevBadIndex, 33, i);
        continue;
      }
      trow[q] = (int)i;
      tperm[q] = p;
    }
  }
}

// sort row c of A^T by row index; buffers of N = nextpow2(len) keys
// Entries whose row or source entry is out of range (a slot the scatter never
// wrote, because of malformed row pointers) are recorded in st and skipped.
template <int TW, bool GBUF>
__global__ void k_tr_sort(long long n, const long long* Atp, const int* trow, const long long* tperm, int* Atj,
                          long long* perm, const void* Ax, void* Atx, int vbytes, long long min_len, long long max_len,
                          unsigned long long* gbuf, long long gbuf_len, long long a_nrows, long long a_nnz,
                          DevStatus* st) {
  extern __shared__ __align__(16) unsigned char smem[];
  Team<TW> tm;
  unsigned long long* buf;
  if (GBUF) buf = gbuf + (long long)blockIdx.x * gbuf_len;
  else buf = reinterpret_cast<unsigned long long*>(smem) + (size_t)tm.id * (size_t)max_len;
  const long long team = (long long)blockIdx.x * tm.per_cta + tm.id;
  const long long nteams = (long long)gridDim.x * tm.per_cta;
  for (long long c = team; c < n; c += nteams) {
    const long long t0 = Atp[c], len = Atp[c + 1] - t0;
    if (len < min_len || len > max_len || len == 0) continue;
    int N = 1;
    while (N < len) N <<= 1;
    for (long long x = tm.lane; x < N; x += TW)
      buf[x] = (x < len) ? (((unsigned long long)(unsigned)trow[t0 + x] << 32) | (unsigned long long)x) : ~0ull;
    if (GBUF) __threadfence_block();
    tm.sync();
    team_bitonic<TW>(tm, buf, N);
    for (long long x = tm.lane; x < len; x += TW) {
      const unsigned long long e = buf[x];
      const long long src = t0 + (long long)(e & 0xffffffffull);
      const long long p = tperm[src];
      const int row = (int)(e >> 32);
      if (p < 0 || p >= a_nnz || row < 0 || (long long)row >= a_nrows) {
        dev_fail(st, kDevBadIndex, 35, c);
        continue;
      }
      Atj[t0 + x] = row;
      if (perm) perm[t0 + x] = p;
      if (Atx) {
        if (vbytes == 8) reinterpret_cast<double*>(Atx)[t0 + x] = reinterpret_cast<const double*>(Ax)[p];
        else reinterpret_cast<float*>(Atx)[t0 + x] = reinterpret_cast<const float*>(Ax)[p];
      }
    }
    if (GBUF) __threadfence_block();
    tm.sync();
  }
}

__global__ void k_reduce_max_ll(const unsigned long long* cnt, long long n, unsigned long long* out) {
  unsigned long long m = 0;
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) m = cnt[i] > m ? cnt[i] : m;
  m = __reduce_max_sync(0xffffffffu, (unsigned)(m > 0xffffffffull ? 0xffffffffull : m));
  if ((threadIdx.x & 31) == 0) atomicMax(out, m);
}

template <typename VT>
__global__ void k_gather(const VT* src, const long long* perm, VT* dst, long long n) {
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < n; q += stride) dst[q] = src[perm[q]];
}

template <class K>
cudaError_t set_smem(K kernel, size_t bytes) {
  // the kernels also hold up to 1 KB of static shared memory: opt in above 47 KB of dynamic
  if (bytes + 1024 > 48 * 1024) return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  return cudaSuccess;
}

inline unsigned grid_cap(long long items, int per, int num_sms, int per_sm) {
  long long g = (items + per - 1) / per;
  long long cap = (long long)num_sms * per_sm;
  if (g > cap) g = cap;
  if (g < 1) g = 1;
  return (unsigned)g;
}

template <int TW, typename VT>
cudaError_t run_masked_hash(const LaunchCtx& L, const MaskedD& M, const MaskedLaunch& S) {
  const int T = 1 << S.logT;
  const size_t tb = msk_team_bytes<TW, VT>(T);
  int teams = 1;
  if (TW <= 32) {
    teams = (int)(kTeamSmemBudget / tb);
    int tmax = 256 / TW;
    if (teams > tmax) teams = tmax;
    if (teams < 1) teams = 1;
  }
  const size_t smem = tb * teams;
  if (smem > (size_t)L.max_smem_optin) return cudaErrorInvalidConfiguration;
  auto kern = k_masked<TW, VT, false>;
  cudaError_t e = set_smem(kern, smem);
  if (e != cudaSuccess) return e;
  KKS_LAUNCHED();
  kern<<<resident_grid(kern, TW * teams, smem, L.num_sms, (S.nrows + teams - 1) / teams), TW * teams, smem,
         L.stream>>>(M, S.rows, S.nrows, S.logT, nullptr, 0);
  return cudaGetLastError();
}

template <int TW, typename VT>
cudaError_t run_masked_warp(const LaunchCtx& L, const MaskedD& M, const MaskedLaunch& S) {
  const int T = 1 << S.logT;
  const size_t tb = mskw_team_bytes<TW, VT>(T);
  int teams = (int)(kTeamSmemBudget / tb);
  const int tmax = 256 / TW;
  if (teams > tmax) teams = tmax;
  if (teams < 1) teams = 1;
  const size_t smem = tb * teams;
  if (smem > (size_t)L.max_smem_optin) return cudaErrorInvalidConfiguration;
  auto kern = k_masked_warp<TW, VT>;
  cudaError_t e = set_smem(kern, smem);
  if (e != cudaSuccess) return e;
  KKS_LAUNCHED();
  kern<<<resident_grid(kern, TW * teams, smem, L.num_sms, (S.nrows + teams - 1) / teams), TW * teams, smem,
         L.stream>>>(M, S.rows, S.nrows, S.logT);
  return cudaGetLastError();
}

template <typename VT>
cudaError_t run_masked_win(const LaunchCtx& L, const MaskedD& M, const MaskedLaunch& S) {
  const size_t smem = mskw_team_bytes<VT>(1 << S.logT) * kMwTeams;
  if (smem > (size_t)L.max_smem_optin) return cudaErrorInvalidConfiguration;
  auto kern = k_masked_win<VT>;
  cudaError_t e = set_smem(kern, smem);
  if (e != cudaSuccess) return e;
  KKS_LAUNCHED();
  kern<<<resident_grid(kern, 32 * kMwTeams, smem, L.num_sms, (S.nrows + kMwTeams - 1) / kMwTeams), 32 * kMwTeams,
         smem, L.stream>>>(M, S.rows, S.nrows, S.logT);
  return cudaGetLastError();
}

template <int TW, typename VT>
cudaError_t run_masked_pos(const LaunchCtx& L, const MaskedD& M, const MaskedLaunch& S) {
  const int T = 1 << S.logT;
  const size_t tb = mskp_team_bytes<TW, VT>(T);
  int teams = (int)(kTeamSmemBudget / tb);
  const int tmax = 256 / TW;
  if (teams > tmax) teams = tmax;
  if (teams < 1) teams = 1;
  const size_t smem = tb * teams;
  if (smem > (size_t)L.max_smem_optin) return cudaErrorInvalidConfiguration;
  auto kern = k_masked_pos<TW, VT>;
  cudaError_t e = set_smem(kern, smem);
  if (e != cudaSuccess) return e;
  KKS_LAUNCHED();
  kern<<<resident_grid(kern, TW * teams, smem, L.num_sms, (S.nrows + teams - 1) / teams), TW * teams, smem,
         L.stream>>>(M, S.rows, S.nrows, S.logT);
  return cudaGetLastError();
}

template <typename VT>
cudaError_t run_masked_global(const LaunchCtx& L, const MaskedD& M, const MaskedLaunch& S) {
  constexpr int TW = 1024;
  const size_t smem = al16(sizeof(ChunkScratch<TW, VT>));
  auto kern = k_masked<TW, VT, true>;
  cudaError_t e = set_smem(kern, smem);
  if (e != cudaSuccess) return e;
  long long grid = S.nchunks;
  if (grid > S.nrows) grid = S.nrows;
  const long long chunk = (long long)msk_team_bytes<TW, VT>((int)S.chunk_slots);
  KKS_LAUNCHED();
  kern<<<(unsigned)grid, TW, smem, L.stream>>>(M, S.rows, S.nrows, ilog2_ceil(S.chunk_slots),
                                               (unsigned char*)S.pool, chunk);
  return cudaGetLastError();
}

template <typename VT>
cudaError_t masked_dispatch(const LaunchCtx& L, const MaskedD& M, const MaskedLaunch& S) {
  switch (S.cls) {
    case kClsT1: {
      KKS_LAUNCHED();
      if (S.logT == 0)
        k_masked_thread<VT, false><<<grid_cap(S.nrows, 256, L.num_sms, 32), 256, 0, L.stream>>>(M, S.rows, S.nrows);
      else
        k_masked_thread<VT, true><<<grid_cap(S.nrows, 256, L.num_sms, 32), 256, 0, L.stream>>>(M, S.rows, S.nrows);
      return cudaGetLastError();
    }
    case kClsW8: return S.positions ? run_masked_pos<8, VT>(L, M, S) : run_masked_warp<8, VT>(L, M, S);
    case kClsW32:
      if (!S.positions) return run_masked_warp<32, VT>(L, M, S);
      return S.window ? run_masked_win<VT>(L, M, S) : run_masked_pos<32, VT>(L, M, S);
    case kClsC256: return run_masked_hash<256, VT>(L, M, S);
    case kClsC1024: return run_masked_hash<1024, VT>(L, M, S);
    case kClsSpill: return run_masked_global<VT>(L, M, S);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace

size_t masked_team_bytes(int cls, int logT, int dtype) {
  const int T = 1 << logT;
  if (dtype == 1) {
    switch (cls) {
      case kClsW8: return msk_team_bytes<8, double>(T);
      case kClsW32: return msk_team_bytes<32, double>(T);
      case kClsC256: return msk_team_bytes<256, double>(T);
      default: return msk_team_bytes<1024, double>(T);
    }
  }
  switch (cls) {
    case kClsW8: return msk_team_bytes<8, float>(T);
    case kClsW32: return msk_team_bytes<32, float>(T);
    case kClsC256: return msk_team_bytes<256, float>(T);
    default: return msk_team_bytes<1024, float>(T);
  }
}

cudaError_t launch_masked_bin_count(const LaunchCtx& L, const MaskedD& M, long long nrows, BinCfg cfg,
                                    unsigned long long* hist, long long* bcnt) {
  if (nrows <= 0) return cudaSuccess;
  const long long nblk = bin_blocks(nrows);
  KKS_LAUNCHED();
  k_masked_bin_count<<<(unsigned)nblk, kBinThreads, 0, L.stream>>>(M, nrows, cfg, hist, bcnt, nblk);
  return cudaGetLastError();
}

cudaError_t launch_masked_bin_scatter(const LaunchCtx& L, const MaskedD& M, long long nrows, BinCfg cfg,
                                      const unsigned long long* cursor, const long long* bofs, int* rows) {
  if (nrows <= 0) return cudaSuccess;
  const long long nblk = bin_blocks(nrows);
  KKS_LAUNCHED();
  k_masked_bin_list<<<(unsigned)nblk, kBinThreads, 0, L.stream>>>(M, nrows, cfg, cursor, bofs, nblk, rows);
  return cudaGetLastError();
}

cudaError_t launch_mc_compress(const LaunchCtx& L, const MaskedD& M, int pass, const long long* cnt_or_ycp,
                               long long* cnt, int* csi, unsigned* cs) {
  if (M.Y.nrows <= 0) return cudaSuccess;
  const unsigned grid = grid_cap(M.Y.nrows, 32, L.num_sms, 16);
  KKS_LAUNCHED();
  if (pass == 0) k_mc_compress_count<<<grid, 256, 0, L.stream>>>(M.Y, cnt, M.status);
  else k_mc_compress_fill<<<grid, 256, 0, L.stream>>>(M.Y, cnt_or_ycp, csi, cs);
  return cudaGetLastError();
}

cudaError_t launch_row_len_max(const LaunchCtx& L, const long long* Sp, long long nrows, unsigned long long* out) {
  cudaError_t e = cudaMemsetAsync(out, 0, sizeof(unsigned long long), L.stream);
  if (e != cudaSuccess || nrows <= 0) return e;
  KKS_LAUNCHED();
  k_row_len_max<<<grid_cap(nrows, 256, L.num_sms, 4), 256, 0, L.stream>>>(Sp, nrows, out);
  return cudaGetLastError();
}

cudaError_t launch_masked_count(const LaunchCtx& L, const MaskedD& M, const long long* Ycp, const int* csi,
                                const unsigned* cs, long long* counts, long long max_row, int* lists,
                                unsigned long long* ctr) {
  const long long n = M.X.nrows;
  if (n <= 0) return cudaSuccess;
  const long long kw = (M.Y.ncols + 31) >> 5;
  const size_t bm_smem = (size_t)kw * 4;
  const bool bm_fits = bm_smem + 16 * 1024 <= (size_t)L.max_smem_optin;
  if (max_row > kMcWarpMaxRow && !bm_fits) return cudaErrorInvalidConfiguration;
  const long long cta_from = bm_fits ? kMcSmallSlots / 2 + 1 : kMcWarpMaxRow + 1;
  // ctr: [0..2] class list lengths, [3..5] the classes' fetch counters
  cudaError_t e = cudaMemsetAsync(ctr, 0, 6 * sizeof(unsigned long long), L.stream);
  if (e != cudaSuccess) return e;
  KKS_LAUNCHED();
  k_mc_classify<<<grid_cap(n, 256, L.num_sms, 8), 256, 0, L.stream>>>(M, lists, ctr, counts, cta_from);
  {
    auto kern = k_masked_count_warp<kMcSmallSlots, 8, 8>;
    const size_t smem = (size_t)8 * 2 * kMcSmallSlots * 4;
    e = set_smem(kern, smem);
    if (e != cudaSuccess) return e;
    KKS_LAUNCHED();
    kern<<<resident_grid(kern, 256, smem, L.num_sms, (n + 7) / 8), 256, smem, L.stream>>>(
        M, Ycp, csi, cs, counts, lists, ctr + 0, ctr + 3);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  if (max_row > kMcSmallSlots / 2 && cta_from > kMcSmallSlots / 2 + 1) {   // mid rows left for warps
    auto kern = k_masked_count_warp<kMcWarpSlots, 4, 1>;
    const size_t smem = (size_t)4 * 2 * kMcWarpSlots * 4;
    e = set_smem(kern, smem);
    if (e != cudaSuccess) return e;
    KKS_LAUNCHED();
    kern<<<resident_grid(kern, 128, smem, L.num_sms, (n + 3) / 4), 128, smem, L.stream>>>(
        M, Ycp, csi, cs, counts, lists + n, ctr + 1, ctr + 4);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  if (max_row >= cta_from) {
    const size_t smem = bm_smem;
    auto kern = k_masked_count_cta;
    e = set_smem(kern, smem);
    if (e != cudaSuccess) return e;
    KKS_LAUNCHED();
    kern<<<resident_grid(kern, 256, smem, L.num_sms, n), 256, smem, L.stream>>>(M, Ycp, csi, cs, counts, kw,
                                                                              lists + 2 * n, ctr + 2, ctr + 5);
    return cudaGetLastError();
  }
  return cudaSuccess;
}

cudaError_t launch_masked(const LaunchCtx& L, const MaskedD& M, const MaskedLaunch& S) {
  if (S.nrows <= 0) return cudaSuccess;
  return S.dtype == 1 ? masked_dispatch<double>(L, M, S) : masked_dispatch<float>(L, M, S);
}

cudaError_t launch_pattern_unsorted(const LaunchCtx& L, const MaskedD& M, long long nrows,
                                    unsigned long long* count) {
  if (nrows <= 0) return cudaSuccess;
  KKS_LAUNCHED();
  k_pattern_unsorted<<<grid_cap(nrows, 8, L.num_sms, 8), 256, 0, L.stream>>>(M, nrows, count);
  return cudaGetLastError();
}

size_t masked_global_chunk_bytes(long long slots, int dtype) {
  return dtype == 1 ? msk_team_bytes<1024, double>((int)slots) : msk_team_bytes<1024, float>((int)slots);
}

// Transpose, in three launches plus one readback of the longest row.
// tmp layout: cnt/cursor (n + 1 ull) | trow (nnz int) | tperm (nnz ll) | max (ull) | scan tmp
size_t transpose_tmp_bytes(long long m, long long n, long long nnz) {
  (void)m;
  return al16((size_t)(n + 1) * 8) * 2 + al16((size_t)(nnz + 1) * 4) + al16((size_t)(nnz + 1) * 8) + 16 +
         scan_tmp_bytes(n + 1);
}

cudaError_t launch_transpose_count(const LaunchCtx& L, const MatD& A, long long* Atp, void* tmp,
                                   unsigned long long* h_max, DevStatus* st) {
  unsigned char* t = (unsigned char*)tmp;
  const long long n = A.ncols;
  unsigned long long* cnt = (unsigned long long*)t;
  unsigned long long* mx = (unsigned long long*)(t + al16((size_t)(n + 1) * 8) * 2 + al16((size_t)(A.nnz + 1) * 4) +
                                                 al16((size_t)(A.nnz + 1) * 8));
  void* stmp = (unsigned char*)mx + 16;
  cudaError_t e = cudaMemsetAsync(cnt, 0, sizeof(unsigned long long) * (n + 1), L.stream);
  if (e != cudaSuccess) return e;
  e = cudaMemsetAsync(mx, 0, 16, L.stream);
  if (e != cudaSuccess) return e;
  if (A.nnz > 0) {
    KKS_LAUNCHED();
    k_tr_count<<<grid_cap(A.nnz, 256, L.num_sms, 16), 256, 0, L.stream>>>(A, cnt, st);
  }
  e = launch_scan(L, (const long long*)cnt, Atp, n, stmp);
  if (e != cudaSuccess) return e;
  if (n > 0) {
    KKS_LAUNCHED();
    k_reduce_max_ll<<<grid_cap(n, 256, L.num_sms, 4), 256, 0, L.stream>>>(cnt, n, mx);
  }
  return cudaMemcpyAsync(h_max, mx, sizeof(unsigned long long), cudaMemcpyDeviceToHost, L.stream);
}

cudaError_t launch_transpose_fill(const LaunchCtx& L, const MatD& A, int dtype, const long long* Atp, int* Atj,
                                  void* Atx, long long* perm, void* tmp, long long max_len,
                                  unsigned long long* gbuf, long long gbuf_len, int gbuf_chunks, DevStatus* st) {
  unsigned char* t = (unsigned char*)tmp;
  const long long n = A.ncols;
  unsigned long long* cursor = (unsigned long long*)(t + al16((size_t)(n + 1) * 8));
  int* trow = (int*)(t + al16((size_t)(n + 1) * 8) * 2);
  long long* tperm = (long long*)(t + al16((size_t)(n + 1) * 8) * 2 + al16((size_t)(A.nnz + 1) * 4));
  cudaError_t e = cudaMemsetAsync(cursor, 0, sizeof(unsigned long long) * (n + 1), L.stream);
  if (e != cudaSuccess) return e;
  if (A.nnz == 0 || n == 0) return cudaSuccess;
  KKS_LAUNCHED();
  k_tr_scatter<<<grid_cap(A.nrows, 256, L.num_sms, 16), 256, 0, L.stream>>>(A, Atp, cursor, trow, tperm, st);
  const int vbytes = dtype == 1 ? 8 : 4;
  // rows up to 256 entries: warp teams with shared buffers
  {
    const long long cap = 256;
    const size_t smem = (size_t)cap * 8 * 8;  // 8 warps
    auto kern = k_tr_sort<32, false>;
    e = set_smem(kern, smem);
    if (e != cudaSuccess) return e;
    KKS_LAUNCHED();
    kern<<<grid_cap(n, 8, L.num_sms, 16), 256, smem, L.stream>>>(n, Atp, trow, tperm, Atj, perm, A.vx, Atx, vbytes, 1,
                                                                 cap, nullptr, 0, A.nrows, A.nnz, st);
  }
  if (max_len > 256) {
    const long long cap = 16384;
    const size_t smem = (size_t)cap * 8;
    auto kern = k_tr_sort<1024, false>;
    e = set_smem(kern, smem);
    if (e != cudaSuccess) return e;
    KKS_LAUNCHED();
    kern<<<grid_cap(n, 1, L.num_sms, 2), 1024, smem, L.stream>>>(n, Atp, trow, tperm, Atj, perm, A.vx, Atx, vbytes,
                                                                 257, cap, nullptr, 0, A.nrows, A.nnz, st);
  }
  if (max_len > 16384) {
    auto kern = k_tr_sort<1024, true>;
    KKS_LAUNCHED();
    kern<<<gbuf_chunks, 1024, 0, L.stream>>>(n, Atp, trow, tperm, Atj, perm, A.vx, Atx, vbytes, 16385, gbuf_len, gbuf,
                                            gbuf_len, A.nrows, A.nnz, st);
  }
  return cudaGetLastError();
}

size_t transpose_pattern_tmp_bytes(long long ncols) {
  return al16((size_t)(ncols + 1) * 8) * 2 + scan_tmp_bytes(ncols + 1);
}

cudaError_t launch_transpose_pattern(const LaunchCtx& L, const MatD& A, long long* Atp, int* trow, long long* tperm,
                                     void* tmp, DevStatus* st) {
  unsigned char* t = (unsigned char*)tmp;
  const long long n = A.ncols;
  unsigned long long* cnt = (unsigned long long*)t;
  unsigned long long* cursor = (unsigned long long*)(t + al16((size_t)(n + 1) * 8));
  void* stmp = t + al16((size_t)(n + 1) * 8) * 2;
  cudaError_t e = cudaMemsetAsync(cnt, 0, al16((size_t)(n + 1) * 8) * 2, L.stream);
  if (e != cudaSuccess) return e;
  if (A.nnz > 0) {
    KKS_LAUNCHED();
    k_tr_count<<<grid_cap(A.nnz, 256, L.num_sms, 16), 256, 0, L.stream>>>(A, cnt, st);
  }
  e = launch_scan(L, (const long long*)cnt, Atp, n, stmp);
  if (e != cudaSuccess) return e;
  if (A.nnz > 0 && A.nrows > 0) {
    KKS_LAUNCHED();
    k_tr_scatter<<<grid_cap(A.nrows, 256, L.num_sms, 16), 256, 0, L.stream>>>(A, Atp, cursor, trow, tperm, st);
  }
  return cudaGetLastError();
}

cudaError_t launch_gather_values(const LaunchCtx& L, int dtype, const void* src, const long long* perm, void* dst,
                                 long long n) {
  if (n <= 0) return cudaSuccess;
  if (dtype == 1)
    { KKS_LAUNCHED(); k_gather<double><<<grid_cap(n, 256, L.num_sms, 16), 256, 0, L.stream>>>((const double*)src, perm, (double*)dst, n); }
  else
    { KKS_LAUNCHED(); k_gather<float><<<grid_cap(n, 256, L.num_sms, 16), 256, 0, L.stream>>>((const float*)src, perm, (float*)dst, n); }
  return cudaGetLastError();
}

}  // namespace kks
