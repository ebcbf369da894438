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
// a global pool chunk.
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
    auto aval = [&](long long p) { return Xx[p]; };
    auto body = [&](long long q, int t) {
      const int slot = lp_find(keys, tmask, Yj[q]);
      if (slot >= 0) atomicAdd(acc + pos[slot], csc->av[t] * Yx[q]);
    };
    for_each_product<TW, VT>(tm, csc, scan_scratch, M.X.cj, a0, a1, range, aval, body);
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

// work_i = sum over j in X(i,:) of |Y(j,:)|, then bins from (|S(i,:)|, work_i)
__global__ void k_masked_bins(MaskedD M, long long nrows, int phase, BinCfg cfg, unsigned long long* hist,
                              unsigned long long* cursor, int* rows) {
  __shared__ unsigned long long h[kNumBins];
  if (phase == 0) {
    for (int t = threadIdx.x; t < kNumBins; t += blockDim.x) h[t] = 0ull;
    __syncthreads();
  }
  const long long stride = (long long)gridDim.x * blockDim.x;
  const int lane = threadIdx.x & 31;
  for (long long base = (long long)blockIdx.x * blockDim.x; base < nrows; base += stride) {
    const long long i = base + threadIdx.x;
    int bin = -1;
    if (i < nrows) {
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
      const long long s = M.Sp[i + 1] - M.Sp[i];
      if (!ok) {
        // the row is not computed; the status word turns into SPGEMM_ERR_BAD_INDEX
        if (phase == 0) dev_fail(M.status, kDevBadIndex, 21, i);
      } else {
        bin = choose_bin(s, w > 0 ? w : (s > 0 ? 1 : 0), M.Y.ncols, (M.Y.ncols + 31) >> 5, cfg);
        if (bin_cls(bin) == kClsNone) bin = -1;
      }
    }
    const unsigned grp = __match_any_sync(0xffffffffu, bin);
    const int leader = __ffs(grp) - 1;
    if (phase == 0) {
      if (bin >= 0 && lane == leader) atomicAdd(&h[bin], (unsigned long long)__popc(grp));
    } else {
      unsigned long long p = 0;
      if (bin >= 0 && lane == leader) p = atomicAdd(&cursor[bin], (unsigned long long)__popc(grp));
      p = __shfl_sync(0xffffffffu, p, leader);
      unsigned lt;
      asm("mov.u32 %0, %%lanemask_lt;" : "=r"(lt));
      if (bin >= 0) rows[p + __popc(grp & lt)] = (int)i;
    }
  }
  if (phase == 0) {
    __syncthreads();
    for (int t = threadIdx.x; t < kNumBins; t += blockDim.x)
      if (h[t]) atomicAdd(&hist[t], h[t]);
  }
}

// ---------------------------------------------------------------- transpose
__global__ void k_tr_count(MatD A, unsigned long long* cnt, DevStatus* st) {
  const long long stride = (long long)gridDim.x * blockDim.x;
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
template <int TW, bool GBUF>
__global__ void k_tr_sort(long long n, const long long* Atp, const int* trow, const long long* tperm, int* Atj,
                          long long* perm, const void* Ax, void* Atx, int vbytes, long long min_len, long long max_len,
                          unsigned long long* gbuf, long long gbuf_len) {
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
      Atj[t0 + x] = (int)(e >> 32);
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
  if (bytes > 48 * 1024) return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
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
    teams = (int)((48 * 1024) / tb);
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
  kern<<<grid_cap(S.nrows, teams, L.num_sms, 64), TW * teams, smem, L.stream>>>(M, S.rows, S.nrows, S.logT, nullptr, 0);
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
    case kClsW8: return run_masked_hash<8, VT>(L, M, S);
    case kClsW32: return run_masked_hash<32, VT>(L, M, S);
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
                                    unsigned long long* hist) {
  if (nrows <= 0) return cudaSuccess;
  KKS_LAUNCHED();
  k_masked_bins<<<grid_cap(nrows, 256, L.num_sms, 8), 256, 0, L.stream>>>(M, nrows, 0, cfg, hist, nullptr, nullptr);
  return cudaGetLastError();
}

cudaError_t launch_masked_bin_scatter(const LaunchCtx& L, const MaskedD& M, long long nrows, BinCfg cfg,
                                      unsigned long long* cursor, int* rows) {
  if (nrows <= 0) return cudaSuccess;
  KKS_LAUNCHED();
  k_masked_bins<<<grid_cap(nrows, 256, L.num_sms, 8), 256, 0, L.stream>>>(M, nrows, 1, cfg, nullptr, cursor, rows);
  return cudaGetLastError();
}

cudaError_t launch_masked(const LaunchCtx& L, const MaskedD& M, const MaskedLaunch& S) {
  if (S.nrows <= 0) return cudaSuccess;
  return S.dtype == 1 ? masked_dispatch<double>(L, M, S) : masked_dispatch<float>(L, M, S);
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
                                                                 cap, nullptr, 0);
  }
  if (max_len > 256) {
    const long long cap = 16384;
    const size_t smem = (size_t)cap * 8;
    auto kern = k_tr_sort<1024, false>;
    e = set_smem(kern, smem);
    if (e != cudaSuccess) return e;
    KKS_LAUNCHED();
    kern<<<grid_cap(n, 1, L.num_sms, 2), 1024, smem, L.stream>>>(n, Atp, trow, tperm, Atj, perm, A.vx, Atx, vbytes,
                                                                 257, cap, nullptr, 0);
  }
  if (max_len > 16384) {
    auto kern = k_tr_sort<1024, true>;
    KKS_LAUNCHED();
    kern<<<gbuf_chunks, 1024, 0, L.stream>>>(n, Atp, trow, tperm, Atj, perm, A.vx, Atx, vbytes, 16385, gbuf_len, gbuf,
                                            gbuf_len);
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
