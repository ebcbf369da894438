/*
 * kkspgemm.h -- C ABI of the GB300 two-phase sparse matrix-matrix multiply.
 *
 * Computes C = A * B for CSR matrices A (m x n) and B (n x k), the problem of
 * Deveci, Trott and Rajamanickam, "Multi-threaded Sparse Matrix-Matrix
 * Multiplication for Many-Core and GPU Architectures" (Section 2).  The calls
 * follow the paper's two-phase structure (Algorithm 2):
 *
 *   spgemm_symbolic   the symbolic phase: row statistics, compression of B,
 *                     and the size of every row of C -> C row pointers, nnz(C)
 *   (caller)          allocation of C's column indices and values
 *   spgemm_numeric    the numeric phase: C's columns and values
 *
 * Numeric reuse (Section 2, two-phase methods; Section 4 "Reuse"): after one
 * symbolic call, spgemm_numeric may be called any number of times with new
 * values on the same A and B patterns.
 *
 * Conventions shared by every call
 * --------------------------------
 *  - All array arguments are DEVICE pointers (memory of the GPU selected by
 *    the handle), except those documented as host pointers.
 *  - A and B: row pointers int32 or int64 (rowptr_is_64), column indices
 *    int32 in [0, ncols), any order inside a row, no duplicate (i, j).
 *    k = B.ncols must be <= 2^31 - 1.
 *  - C: row pointers int64[m + 1]; column indices int32; values of the same
 *    type as A and B.  Every row of C is sorted by column and holds every
 *    structural product, numerical zeros included.
 *  - Ownership: the caller owns A, B and all of C.  The handle owns every
 *    scratch buffer (statistics, compressed B, row bins, accumulator pools).
 *  - Streams: spgemm_stream_t is a cudaStream_t.  One handle serves one
 *    stream at a time and is not thread-safe.
 *  - Errors: every call returns a status and never throws or aborts.  Device
 *    kernels never trap; a problem they detect is recorded in the handle and
 *    returned by the next call that synchronises (spgemm_symbolic, or
 *    spgemm_handle_sync after numeric calls).
 */
#ifndef KKSPGEMM_H
#define KKSPGEMM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st *spgemm_stream_t; /* same type as cudaStream_t */
typedef struct kks_handle *spgemm_handle_t;

typedef enum {
  SPGEMM_OK = 0,
  SPGEMM_ERR_INVALID_ARG = 1,      /* null pointer, bad sizes, mismatched dims or dtypes */
  SPGEMM_ERR_NOT_READY = 2,        /* numeric before a symbolic call on this handle */
  SPGEMM_ERR_OOM = 3,              /* device memory (or the workspace limit) exhausted */
  SPGEMM_ERR_INDEX_OVERFLOW = 4,   /* a size exceeds the supported index range */
  SPGEMM_ERR_DEVICE_LIMIT = 5,     /* a kernel hit an internal limit (recorded on device) */
  SPGEMM_ERR_CUDA = 6,             /* a CUDA runtime call failed */
  SPGEMM_ERR_PATTERN_MISMATCH = 7, /* numeric called with operands other than symbolic's */
  SPGEMM_ERR_BAD_INDEX = 8         /* a column index outside its range (detected on device) */
} spgemm_status_t;

typedef enum { SPGEMM_R32 = 0, SPGEMM_R64 = 1 } spgemm_dtype_t;

/* A CSR operand (device pointers). */
typedef struct {
  int64_t nrows, ncols, nnz;
  int32_t rowptr_is_64;   /* 1: rowptr is int64[nrows + 1]; 0: int32[nrows + 1] */
  spgemm_dtype_t dtype;   /* type of values */
  const void *rowptr;
  const int32_t *colidx;
  const void *values;     /* may be NULL for the symbolic phase */
} spgemm_csr_t;

/*
 * Tunables.  The defaults restate the paper's parameters for GB300:
 * compression when it cuts the product count by more than 15 % (Section 3.2),
 * 50 % maximum occupancy of the LP level-1 accumulator (Section 3.1.2), level-1
 * tables in shared memory (up to 227 KB per CTA on GB300), level-2 tables and
 * dense accumulators in global-memory pools (Section 3.1.2, memory pool).
 */
typedef struct {
  int32_t compression;           /* -1 auto (the 15 % rule), 0 never, 1 always */
  double compress_threshold;     /* compress iff compressed f_m / f_m < this (0.85) */
  double l1_max_occupancy;       /* LP level-1 cut-off for new keys (0.5) */
  int32_t l1_max_log2_slots;     /* 0 = auto; caps shared tables at 2^this slots */
  int32_t dense;                 /* -1 auto, 0 never use dense accumulators, 1 prefer */
  int32_t method;                /* 0 binned (per-row team + accumulator),
                                    1 paper meta-algorithm (one team class per problem) */
  int64_t workspace_limit_bytes; /* 0 = no limit; above it calls fail with SPGEMM_ERR_OOM */
  int64_t pool_limit_bytes;      /* cap on accumulator pools (0 = 8 GiB) */
  int32_t device;                /* CUDA device ordinal used by the handle */
  int32_t hash_function;         /* 0 = key & (size - 1) (the paper's), 1 = multiplicative (default) */
  int32_t verbose;               /* 1: print device-detected errors to stderr */
  int32_t slots_per_key_log2;    /* hash-table slots per key bound, log2 (0 = default 1: 50 % load) */
  int32_t tune;                  /* 1: the first numeric call of a plan times candidate kernel
                                    configurations per row bin and keeps the fastest (synchronises) */
  int32_t numeric_positions;     /* 1 (default): when every product of a plan runs on the compressed B,
                                    warp-team rows of the numeric phase take each product's place in
                                    C(i,:) from the column sets (Section 3.2) instead of sorting the
                                    accumulator; masked products and numeric reuse whose pattern rows
                                    are all sorted key their warp-team tables by the pattern's column
                                    sets.  0: hash-and-sort numeric, column-keyed masked tables */
  int32_t cta_partition;         /* numeric rows of the CTA hash classes (Section 3.1.1): 0 (default)
                                    Thread-Flat-Parallel, 1 Team-Sequential with the linked-list
                                    accumulator (Section 3.1.2), 2 Thread-Parallel; with tune = 1 the
                                    tuner also times the other two per bin */
  int32_t window_positions;      /* bitmap windows of column sets: warp-team rows of compressed
                                    products whose B rows are all sorted keep their column sets in a
                                    bitmap over the row's window of sets (first to last set, at most
                                    1344 sets = 43 008 columns), addressed directly instead of hashed
                                    (Section 3.1.2's dense accumulator over the row's own range);
                                    wider rows use the hash tables.  bit 0 (default on): symbolic
                                    phase; bit 1: numeric phase with numeric_positions (the tuner
                                    also times it per bin); bit 2: masked products and numeric reuse
                                    on sorted patterns.  0: hash tables only.  Values 0 to 7 */
  int32_t stage_b;               /* dense-window numeric rows (one chunk of A, sorted B rows): 1 copies
                                    the B entries of the next block of products into shared memory with
                                    asynchronous copies (cp.async) while the current block is added,
                                    instead of loading them from global memory per product; 0 (default)
                                    loads them per product */
  int32_t sym_merge;             /* symbolic window rows (window_positions bit 0) with at most 32 entries
                                    of A whose compressed B rows hold at most 19 column sets each: 1
                                    (default) merges the sorted compressed B rows (Section 3.2's OR of
                                    column sets, one set index at a time, smallest first) instead of
                                    OR-ing them into the window bitmap with shared-memory atomics;
                                    0: bitmap only.  The row sizes and recorded sets are the same */
} spgemm_options_t;

/* Statistics of the last symbolic call (Section 4 results-table columns). */
typedef struct {
  int64_t m, n, k, nnzA, nnzB;
  int64_t f_m;            /* multiplications of A*B (uncompressed) */
  int64_t maxrf;          /* max multiplications of one row */
  int64_t f_m_compressed; /* multiplications on the compressed B */
  int64_t maxrf_compressed;
  double CF;              /* f_m_compressed / f_m */
  double CMRF;            /* maxrf_compressed / maxrf */
  int32_t compressed;     /* 1 if the symbolic phase ran on the compressed B */
  int32_t nbins_symbolic; /* non-empty row bins used by the symbolic phase */
  int32_t nbins_numeric;  /* non-empty row bins used by the numeric phase */
  int32_t tuned_bins;     /* numeric bins whose configuration the tuner changed */
  int64_t nnzC;
  int64_t maxrs;          /* largest row of C */
  double ars;             /* average row size of C */
  int64_t workspace_bytes;/* device scratch held by the handle */
  int64_t bin_rows_numeric[8]; /* rows per team class: none, w8, w32, c256, c1024, dense, spill, thread */
  int64_t rows_positions; /* numeric rows that take their output positions from the column sets */
} spgemm_stats_t;

/* Fills *opt with the defaults.  Returns SPGEMM_ERR_INVALID_ARG for NULL. */
spgemm_status_t spgemm_options_default(spgemm_options_t *opt);

/* Creates a handle (opt may be NULL for defaults).  *out receives it. */
spgemm_status_t spgemm_handle_create(spgemm_handle_t *out, const spgemm_options_t *opt);

/* Frees the handle and all scratch it owns (synchronises its device). */
spgemm_status_t spgemm_handle_destroy(spgemm_handle_t h);

/*
 * Symbolic phase (Algorithm 2).  Computes the row pointers of C into
 * C_rowptr (device, int64[m + 1], caller-allocated) and writes nnz(C) to
 * *nnzC (HOST pointer).  Values of A and B are not read.  Synchronises the
 * stream once to return nnz(C), and plans the numeric phase.
 */
spgemm_status_t spgemm_symbolic(spgemm_handle_t h, const spgemm_csr_t *A, const spgemm_csr_t *B,
                                int64_t *C_rowptr, int64_t *nnzC, spgemm_stream_t stream);

/*
 * Numeric phase (Algorithm 2).  A and B must be the operands of the
 * last symbolic call on h (same patterns, same device pointers for the
 * patterns; the value pointers may change).  Writes C_colidx (int32[nnzC])
 * and C_values (nnzC values of A's dtype), rows sorted by column.  Fully
 * asynchronous; allocates nothing.
 */
spgemm_status_t spgemm_numeric(spgemm_handle_t h, const spgemm_csr_t *A, const spgemm_csr_t *B,
                               const int64_t *C_rowptr, int32_t *C_colidx, void *C_values,
                               spgemm_stream_t stream);

/*
 * Numeric reuse on a known pattern of C: recomputes only C_values for new
 * values of A and B, with C_rowptr / C_colidx as written by spgemm_numeric
 * on the same handle.  The accumulator of each row is keyed by C's pattern
 * (probe only), so no sort is needed.  Asynchronous; allocates nothing.
 */
spgemm_status_t spgemm_numeric_reuse(spgemm_handle_t h, const spgemm_csr_t *A, const spgemm_csr_t *B,
                                     const int64_t *C_rowptr, const int32_t *C_colidx, void *C_values,
                                     spgemm_stream_t stream);

/* Waits for the stream, then reports (and clears) any device-detected error. */
spgemm_status_t spgemm_handle_sync(spgemm_handle_t h, spgemm_stream_t stream);

/* Statistics of the last symbolic call (host struct). */
spgemm_status_t spgemm_get_stats(spgemm_handle_t h, spgemm_stats_t *out);

/*
 * Masked product on a given pattern: out(i, l) = sum_j X(i, j) * Y(j, l) for
 * every (i, l) stored in S (S_rowptr int64[X.nrows + 1], S_colidx int32, any
 * order inside a row); products whose column is not in S(i,:) are dropped.
 * This gives the gradients of a loss L(C), C = A * B, on fixed patterns:
 * dA = (G * B^T) on A's pattern and dB = (A^T * G) on B's pattern, with G the
 * gradient on C's pattern.  out has nnz(S) values of X's dtype.  The first call
 * on a set of patterns synchronises the stream once (to plan the row bins);
 * later calls with the same X, Y and S pattern pointers reuse the plan and are
 * asynchronous (value pointers may change between calls).
 * X_perm / Y_perm (device int64, may be NULL): when given, the value of X's
 * entry p is X.values[X_perm[p]] (likewise for Y), so a transpose built by
 * spgemm_transpose can take the current values of its source without a gather.
 */
spgemm_status_t spgemm_masked(spgemm_handle_t h, const spgemm_csr_t *X, const spgemm_csr_t *Y,
                              const int64_t *S_rowptr, const int32_t *S_colidx, int64_t S_nnz,
                              void *out, const int64_t *X_perm, const int64_t *Y_perm,
                              spgemm_stream_t stream);

/*
 * Structural masked count on the compressed Y (the symbolic-only use of the
 * two-phase method for graph analytics, Section 2, with the compression of
 * Section 3.2):
 *     row_counts[i] = sum over l in S(i,:) of |{ j : (i,j) in X and (j,l) in Y }|,
 * the row sums of (X*Y) sampled on S over the counting semiring; values are
 * never read (X.values and Y.values may be NULL).  With X = Y = S = L, the
 * strictly lower triangle of an undirected graph, the sum of row_counts is the
 * number of triangles.  Y's rows are compressed into 32-column sets inside
 * the call, and every compressed product adds the popcount of its set bits
 * that S(i,:) also holds.  S: int64 row pointers [X.nrows + 1] and S_nnz
 * int32 columns, distinct within a row, any order.  row_counts: int64
 * [X.nrows], device.  Synchronises the stream twice.  Rows of S with more
 * than 128 entries are counted by a CTA each against a bitmap of
 * ceil(Y.ncols / 32) words in shared memory when that fits (Y.ncols up to
 * about 1.6 M); otherwise rows up to 1024 entries use warp hash tables and a
 * longer row makes the call return SPGEMM_ERR_DEVICE_LIMIT.  Out-of-range
 * indices give SPGEMM_ERR_BAD_INDEX.
 */
spgemm_status_t spgemm_masked_count(spgemm_handle_t h, const spgemm_csr_t *X, const spgemm_csr_t *Y,
                                    const int64_t *S_rowptr, const int32_t *S_colidx, int64_t S_nnz,
                                    int64_t *row_counts, spgemm_stream_t stream);

/*
 * Galerkin triple product C = P^T * A * P in one plan (the R x A x P products
 * of multigrid setup, Section 4, with R = P^T): A is n x n, P is n x K, C is
 * K x K with int64 row pointers C_rowptr[K + 1], int32 columns sorted within
 * each row and values in A's dtype.  A and P share one dtype.  C's pattern is
 * the structural product (every (I, J) with some i, j such that P(i, I),
 * A(i, j) and P(j, J) are stored; numerical zeros kept).
 *
 * Unlike two calls of spgemm_symbolic / spgemm_numeric, A*P is never formed:
 * row I of C is accumulated directly from the rows A(i,:) of the entries
 * P(i, I) of column I of P.  The symbolic call builds the pattern of P^T
 * (which entry of P holds each value of R) and keeps it in the handle; the
 * numeric call reads R's values from P through it, so new values of A and P
 * on the same patterns need no transpose or gather.  Each row of C is one
 * warp (or, for large rows, one 256-thread CTA) with its accumulator in
 * shared memory: a bitmap of ceil(K / 32) words or an LP table (Section
 * 3.1.2), whichever is smaller, in the symbolic call; an LP table sized from
 * the row's known size in the numeric call.
 *
 * spgemm_rap_symbolic writes C_rowptr (device, caller-owned, K + 1 entries)
 * and *nnzC (host); it synchronises the stream twice.  Values of A and P may
 * be NULL (their dtype fields still select the numeric plan).  Afterwards
 * spgemm_get_stats describes this product (f_m = the number of products
 * r * a * p).  Errors: SPGEMM_ERR_INVALID_ARG for mismatched shapes or dtypes,
 * SPGEMM_ERR_INDEX_OVERFLOW when n or K exceeds 2^31 - 1,
 * SPGEMM_ERR_BAD_INDEX for malformed row pointers or out-of-range columns,
 * SPGEMM_ERR_DEVICE_LIMIT when a row of C needs more shared memory than one
 * CTA has (symbolic: more than about 50 K keys with K above about 1.6 M;
 * numeric: rows of more than 4096 entries in FP64, 8192 in FP32): multiply in
 * two steps (spgemm_transpose, spgemm_symbolic / spgemm_numeric) instead.
 *
 * spgemm_rap_numeric fills C_colidx and C_values (device, caller-owned, nnzC
 * entries each) on the pattern of the last spgemm_rap_symbolic call of this
 * handle.  It returns SPGEMM_ERR_NOT_READY unless A and P have that call's
 * patterns (the same row-pointer and column pointers and sizes), allocates
 * nothing and does not synchronise (it can be captured in a CUDA graph);
 * device-detected problems are returned by spgemm_handle_sync.
 */
spgemm_status_t spgemm_rap_symbolic(spgemm_handle_t h, const spgemm_csr_t *A, const spgemm_csr_t *P,
                                    int64_t *C_rowptr, int64_t *nnzC, spgemm_stream_t stream);
spgemm_status_t spgemm_rap_numeric(spgemm_handle_t h, const spgemm_csr_t *A, const spgemm_csr_t *P,
                                   const int64_t *C_rowptr, int32_t *C_colidx, void *C_values,
                                   spgemm_stream_t stream);

/*
 * Transpose: At = A^T (A.ncols x A.nrows) with At_rowptr int64[A.ncols + 1],
 * At_colidx int32[nnz] (rows sorted), At_values (A's dtype, may be NULL when
 * A.values is NULL) and perm int64[nnz] (may be NULL): At_values[q] =
 * A.values[perm[q]], so later value-only updates are a gather
 * (spgemm_gather).  Asynchronous.
 */
spgemm_status_t spgemm_transpose(spgemm_handle_t h, const spgemm_csr_t *A, int64_t *At_rowptr,
                                 int32_t *At_colidx, void *At_values, int64_t *perm,
                                 spgemm_stream_t stream);

/*
 * Transpose without allocating anything (the paper has no counterpart; this
 * is a deployment convenience).  For callers that cannot allocate GPU memory
 * when they need the transpose: code running inside a custom allocator or an
 * out-of-memory handler, where a nested cudaMalloc would recurse or fail, code
 * that must not synchronise the device as cudaFree does, or processes with a
 * fixed GPU memory budget.  Same arguments and results as spgemm_transpose,
 * without a handle.  Its scratch is one fixed 32 MiB device buffer inside the
 * library, held by every GPU that loads it until the process exits:
 *  - the first call on a device looks up the buffer's address on that device
 *    (once; the device must be current);
 *  - every call synchronises its stream, so no call can be made while that
 *    stream is being captured into a CUDA graph;
 *  - all calls share the buffer and it keeps the last call's contents (each
 *    call clears what it needs); calls that overlap on the GPU race on it, so
 *    serialise them;
 *  - a problem needing more scratch (about 16 bytes per column of A plus 12
 *    bytes per nonzero) returns SPGEMM_ERR_OOM before any kernel runs.
 * Synchronises the stream twice (the longest column and the status of the
 * counting pass, then the final status).  Row pointers that do not start at 0
 * and end at nnz, or out-of-range columns, give SPGEMM_ERR_BAD_INDEX before
 * any entry is scattered.
 */
spgemm_status_t spgemm_transpose_noalloc(const spgemm_csr_t *A, int64_t *At_rowptr, int32_t *At_colidx,
                                         void *At_values, int64_t *perm, spgemm_stream_t stream);

/* dst[q] = src[perm[q]] for q < n (dtype selects 4- or 8-byte values). */
spgemm_status_t spgemm_gather(spgemm_handle_t h, spgemm_dtype_t dtype, const void *src, const int64_t *perm,
                              void *dst, int64_t n, spgemm_stream_t stream);

/*
 * Batched symbolic / numeric: count independent products C_b = A_b * B_b in
 * one plan, rows of all instances binned together (one launch per bin for all
 * instances).  A, B: host arrays of count operand descriptors; C_rowptr,
 * C_colidx, C_values: host arrays of count device pointers; nnzC: host array
 * of count outputs.  All instances share one dtype.  Numeric reuse rules are
 * those of the single calls.
 *
 * Plan lifecycle: there is no separate plan object.  spgemm_batch_symbolic
 * plans the batch (row statistics, compression, bins, pools) and keeps the
 * plan in the handle; spgemm_batch_numeric runs it any number of times (new
 * values, same patterns); the plan is released by the next symbolic call on
 * the handle (single or batched) or by spgemm_handle_destroy.  So a plan is
 * created with spgemm_handle_create + spgemm_batch_symbolic and destroyed
 * with spgemm_handle_destroy; use one handle per live plan.
 */
spgemm_status_t spgemm_batch_symbolic(spgemm_handle_t h, int32_t count, const spgemm_csr_t *A,
                                      const spgemm_csr_t *B, int64_t *const *C_rowptr, int64_t *nnzC,
                                      spgemm_stream_t stream);
spgemm_status_t spgemm_batch_numeric(spgemm_handle_t h, int32_t count, const spgemm_csr_t *A,
                                     const spgemm_csr_t *B, int64_t *const *C_rowptr,
                                     int32_t *const *C_colidx, void *const *C_values, spgemm_stream_t stream);

/*
 * Row flops for partitioning: prefix[0] = 0 and prefix[i + 1] = prefix[i] + the
 * multiplications of row i of A*B (the sum over A(i,:) of the lengths of the
 * rows of B: f_m row by row, Section 2).  prefix: device, int64[A.nrows + 1],
 * caller-owned.  Synchronises the stream once (for the status).  Out-of-range
 * columns of A or malformed row pointers give SPGEMM_ERR_BAD_INDEX.
 */
spgemm_status_t spgemm_row_flops(spgemm_handle_t h, const spgemm_csr_t *A, const spgemm_csr_t *B,
                                 int64_t *prefix, spgemm_stream_t stream);

/*
 * Row-range sharding of C = A*B over `parts` devices (the 1-D row partition
 * of Section 3.1.1 applied across GPUs): bounds[0] = 0 <= bounds[1] <= ... <=
 * bounds[parts] = m, each boundary the row nearest to an equal share of the
 * flops in `prefix` (host memory, int64[m + 1], non-decreasing, e.g. a copy of
 * spgemm_row_flops's output); rows are never split.  Shard p multiplies the
 * rows [bounds[p], bounds[p + 1]) of A by the whole B on its own device, with
 * no exchange but the shards' nnz (to place its block of C).  With no flops
 * at all the rows are split evenly.  Host only: needs no handle and no GPU.
 * SPGEMM_ERR_INVALID_ARG for a decreasing prefix, parts < 1 or m < 0.
 */
spgemm_status_t spgemm_partition_rows(const int64_t *prefix, int64_t m, int32_t parts, int64_t *bounds);

/* Human-readable name of a status code (static string). */
const char *spgemm_status_string(spgemm_status_t s);

/* Library version as an integer (major * 10000 + minor * 100 + patch). */
int32_t spgemm_version(void);

/* Number of CUDA kernels the library has launched in this process (a
 * diagnostic counter; host-side, no synchronisation). */
int64_t spgemm_launch_count(void);

#ifdef __cplusplus
}
#endif

#endif /* KKSPGEMM_H */
