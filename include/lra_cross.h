/*
 * lra_cross.h -- C ABI of the GB300 cross-approximation (C-A) CUR library.
 *
 * Method: Pan, Luan, Svadlenka, Zhao, "Superfast Low-Rank Approximation and
 * Least Squares Regression", arXiv:1611.01391.
 *   - Problem statement (Section 5.1, Algorithm 5.1 preamble; Section 6.5):
 *     an m x n matrix M reachable entry by entry, a target rank k and a cross
 *     size l >= k; the result is a CUR approximation C U R.
 *   - Primitive Algorithm (Section 6.5): C = M[:, J], R = M[I, :], the CUR
 *     generator M[I, J] and the nucleus U = (M[I, J]_k)^+ (rank-k truncated
 *     pseudo-inverse).
 *   - C-A iterations (Section 6.5; dual start of Remark rec-atnsr): alternate
 *     a vertical step (choose I inside M[:, J]) and a horizontal step (choose J
 *     inside M[I, :]) for a fixed number of sweeps, or until the error
 *     estimate drops below a tolerance.  Each step picks an l x l submatrix of
 *     locally maximal volume (volume footnote of Section 6.5; Section 12.2).
 *   - Appendix F: a posteriori error estimate on a random q x s submatrix of
 *     the error matrix.
 *   - Section 9: the same iteration, rank-adaptive, on many blocks of one
 *     generated matrix (the far-field generators of HSS / FMM matrices) in
 *     one batched launch (lra_cross_submit_batch).
 *
 * Conventions
 *   - Every call returns an lra_status (0 on success, negative on error);
 *     no call aborts or throws.  lra_cross_last_error() gives a message.
 *   - Indices are 0-based int32; matrices are row-major.
 *   - Source buffers (dense matrix, point coordinates) are DEVICE pointers,
 *     BORROWED: they must stay valid and unchanged until the job is DONE,
 *     FAILED or cancelled.  Host arrays in lra_params are copied at submit.
 *   - Outputs are caller-allocated (host or device, see lra_cur_out).
 *   - A context works on one device, on the caller's stream or on a pool of
 *     its own streams (lra_ctx_params.n_streams).  Each job runs in order on
 *     one stream; jobs on different streams overlap on the device.  Calls on
 *     one context are thread-safe: each holds the context's lock only for
 *     its bookkeeping, and calls that wait for a job (wait, fetch, cancel)
 *     wait with the lock released, so other threads keep submitting and
 *     polling meanwhile.
 *   - All computation happens in the library's CUDA kernels; there is no
 *     CPU fallback.  Without a usable device, create fails with LRA_ECUDA.
 */
#ifndef LRA_CROSS_H
#define LRA_CROSS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  LRA_OK = 0,
  LRA_PENDING = 1,        /* job still queued or running                      */
  LRA_EINVAL = -1,        /* bad argument (sizes, pointers, k > l, ...)       */
  LRA_ENOMEM = -2,        /* device allocation failed                         */
  LRA_EBUSY = -3,         /* admission refused: slots or memory budget full   */
  LRA_ESINGULAR = -4,     /* a strip has no nonsingular l x l submatrix       */
  LRA_ENONFINITE = -5,    /* an entry of M (or of B) is NaN or infinite       */
  LRA_ETIMEOUT = -6,      /* a bounded device wait gave up                    */
  LRA_ECUDA = -7,         /* CUDA runtime error                               */
  LRA_ENOTFOUND = -8,     /* unknown job handle                               */
  LRA_ECANCELED = -9,     /* job was cancelled                                */
  LRA_ETOOLARGE = -10     /* strip exceeds the on-chip working-set limit      */
} lra_status;

typedef enum {
  LRA_DENSE_F32 = 0,      /* a: float, m x n, row stride lda (elements)       */
  LRA_DENSE_F64 = 1,      /* a: double, m x n, row stride lda; gathered as FP32 */
  LRA_GEN_CAUCHY = 2,     /* a_ij = 1/(x_i - y_j); x: m floats, y: n floats   */
  LRA_GEN_GAUSS = 3,      /* a_ij = exp(-|x_i - y_j|^2 / h^2), dim-D points   */
  LRA_GEN_INVDIST = 4,    /* a_ij = 1/|x_i - y_j|, dim-D points               */
  LRA_PRE_AH = 5          /* M_bar = F M H for a stored FP32 M (a, lda) and the
                             abridged Hadamard multipliers of the pre_* fields
                             (Section 8.1 family (i)); plain solves only       */
} lra_kind;

/* Decision log entry kinds (lra_cur_out.trace). */
enum { LRA_TRACE_GEPP = 0, LRA_TRACE_SWAP = 1, LRA_TRACE_STOP = 2, LRA_TRACE_CAP = 3 };

/* lra_params.flags */
enum {
  LRA_FLAG_PROFILE = 1,        /* time every launch with CUDA events (lra_info.t_*_ms)     */
  LRA_FLAG_FULL_RESIDUAL = 2   /* also compute ||M - CUR||_F / ||M||_F over all m n entries
                                  (LRA_DENSE_F32 sources with lda % 4 == 0 and a 16-byte
                                  aligned base; tcgen05 tensor cores); lra_info.full_rel_err */
};

/* Job states (lra_info.state). */
enum { LRA_STATE_RUNNING = 0, LRA_STATE_DONE = 1, LRA_STATE_FAILED = 2 };

typedef struct lra_ctx lra_ctx;
typedef uint64_t lra_job;

typedef struct {
  int32_t device;             /* CUDA device ordinal                                */
  int32_t max_slots;          /* max jobs held at once (<= 0: 64)                   */
  uint64_t mem_budget_bytes;  /* device-memory admission budget (0: unlimited)      */
  void* stream;               /* cudaStream_t to run every job on, or NULL: own streams */
  int32_t n_streams;          /* own streams (1..32; <= 0: 1).  A job runs on the
                                 least loaded one, so jobs submitted while others
                                 run overlap on the device (continuous admission).
                                 With one stream the cross inverse of a warm-started
                                 step runs inside that step's maxvol launch (every
                                 CTA inverts the cross itself) when it fits on chip;
                                 with more than one it runs as its own one-CTA
                                 launch, leaving the other SMs to the other jobs. */
  int32_t max_grid;           /* CTAs per maxvol launch at most (<= 0: one per SM).
                                 A smaller grid leaves SMs to the other jobs in
                                 flight; a strip whose chunks would not fit in
                                 shared memory still gets the CTAs it needs. */
} lra_ctx_params;

typedef struct {
  int32_t kind;               /* lra_kind                                           */
  int32_t dim;                /* point dimension for LRA_GEN_GAUSS / _INVDIST (1..3) */
  int64_t m, n;               /* matrix size                                        */
  const void* a;              /* dense: device pointer                              */
  int64_t lda;                /* dense: row stride in elements (>= n)               */
  const float* x;             /* generators: device, m points (point-major, dim)    */
  const float* y;             /* generators: device, n points                       */
  float h;                    /* LRA_GEN_GAUSS width                                */
  /* LRA_PRE_AH (Section 8.1, family (i), with Section 6.6's nonsingular
   * multipliers): F = D_r P_r H_{m,d} and H = H_{n,d} P_c D_c, with H_{n,d}
   * the d-abridged Hadamard matrix (the recursion H_2s = [[H_s, H_s],
   * [H_s, -H_s]] run d times from I_{n/2^d}; 2^d must divide m and n), P
   * permutations and D diagonal +-1 scalings given by the caller (device
   * arrays): row i of F is sign_rows[i] times row perm_rows[i] of H_{m,d},
   * column j of H is sign_cols[j] times column perm_cols[j] of H_{n,d}.
   * Entry (i, j) of M_bar is sign_rows[i] sign_cols[j] times entry
   * (perm_rows[i], perm_cols[j]) of H_{m,d} M H_{n,d}: a sum of 4^d entries
   * of M in FP64, in the order of the recursive steps (M's row blocks
   * first, lowest bit first), rounded to FP32.  With pre_materialized != 0,
   * a holds H_{m,d} M H_{n,d} itself (lra_preprocess_materialize) and an
   * entry is one signed read. */
  int32_t pre_d;              /* recursion depth d, 0..10                           */
  const int32_t* pre_perm_rows;   /* device, m: a permutation of 0..m-1             */
  const float* pre_sign_rows;     /* device, m: +-1                                 */
  const int32_t* pre_perm_cols;   /* device, n: a permutation of 0..n-1             */
  const float* pre_sign_cols;     /* device, n: +-1                                 */
  int32_t pre_materialized;       /* a is H_{m,d} M H_{n,d}, not M                   */
} lra_source;

typedef struct {
  int32_t k;                  /* truncation rank, 1 <= k <= l                       */
  int32_t l;                  /* cross size |I| = |J| = l, l <= 96, l <= min(m, n)  */
  int32_t sweeps;             /* C-A sweeps (vertical + horizontal step), >= 1      */
  int32_t max_swaps;          /* maxvol swap cap per half-step (<= 0: 64 l)         */
  double delta;               /* maxvol stops when max |B| <= 1 + delta (> 0)       */
  double rank_tol;            /* nucleus keeps sigma_j > rank_tol * sigma_1         */
  double tol;                 /* > 0: stop after a sweep once the estimate <= tol   */
  const int32_t* init_J;      /* host, l distinct column indices (initial J), or NULL:
                                 J is drawn from `seed` (lra_draw_columns)          */
  int64_t resid_q, resid_s;   /* Appendix F sample size (0: no estimate)            */
  const int32_t* resid_rows;  /* host, resid_q distinct row indices                 */
  const int32_t* resid_cols;  /* host, resid_s distinct column indices              */
  int32_t trace_cap;          /* decisions to record (0: none)                      */
  int32_t flags;              /* LRA_FLAG_* bits                                    */
  const int32_t* init_I;      /* host, l distinct row indices, or NULL.  Given: the
                                 first vertical step is a warm start from this I
                                 (maxvol from B = S X^{-1}) instead of Gaussian
                                 elimination, so a run checkpointed after s sweeps
                                 as (I, J) and resubmitted with init_I = I,
                                 init_J = J and the remaining sweeps returns the
                                 same I, J, U bit for bit as the uninterrupted run */
  uint64_t seed;              /* initial-J seed, used only when init_J is NULL      */
} lra_params;

typedef struct {
  int32_t state;              /* LRA_STATE_*                                        */
  int32_t status;             /* lra_status of the job (LRA_OK when DONE)           */
  int32_t sweeps_done;
  int32_t k_eff;              /* kept singular triplets of the nucleus              */
  int32_t swaps_total;        /* maxvol swaps over all half-steps                   */
  int32_t converged;          /* 1 if no half-step hit the swap cap                 */
  int32_t trace_len;          /* decisions recorded (<= trace_cap)                  */
  int32_t reserved;
  double est_rel_err;         /* Appendix F: sqrt(sum E^2 / sum M^2) on the sample  */
  double est_mu;              /* observed mean of the sampled error entries         */
  double est_var;             /* observed variance (1/K normalisation)              */
  double sigma_max;           /* sigma_1 of the final cross                         */
  double gpu_ms;              /* device time from first to last kernel of the job   */
  int32_t kernel_launches;    /* kernels the job launched                           */
  int32_t maxvol_launches;
  double maxvol_flops;        /* algorithmic flops of all maxvol half-steps         */
  double t_gather_ms;         /* with LRA_FLAG_PROFILE: device time per kernel class */
  double t_maxvol_ms;
  double t_cross_ms;
  double t_resid_ms;
  double t_inverse_ms;        /* fresh cross inverses run as their own launches
                                 (inverses inside a maxvol launch count there)      */
  double full_rel_err;        /* LRA_FLAG_FULL_RESIDUAL: ||M - CUR||_F / ||M||_F (else -1) */
  double t_fullres_ms;        /* with LRA_FLAG_PROFILE: full-residual kernels       */
} lra_info;

typedef struct {
  int32_t on_device;          /* 1: the pointers below are device pointers          */
  int32_t* I;                 /* l row indices                                      */
  int32_t* J;                 /* l column indices                                   */
  double* U;                  /* l x l nucleus, row-major (C U R)                   */
  double* sigma;              /* l singular values of M[I, J], descending (nullable) */
  float* C;                   /* m x l, row-major (nullable)                        */
  float* R;                   /* l x n, row-major (nullable)                        */
  int32_t* trace;             /* 4 ints per decision: half_step, kind, i, j (nullable) */
  double* trace_val;          /* 1 double per decision: winning |value| (nullable)  */
} lra_cur_out;

/* ---- Batched form: many blocks of one source in one launch --------------
 * Section 9 (superfast multipole method): the generators of the neutered
 * block columns / far-field blocks are low-rank approximations of many
 * submatrices of one matrix, computed here by C-A iterations (Section 6.5)
 * with the rank chosen per block.  Block b is the submatrix
 * M[row0 : row0 + m, col0 : col0 + n] of the source (1 <= m, n <= 2048).
 *
 * Per block (reading of the paper for blocks of unknown rank; the paper's
 * HSS test of Section 12.8 searches the rank instead):
 *   - the cross starts at l = l_init with the first columns of cand_J;
 *   - a sweep is a vertical and a horizontal step (Section 6.5).  Each strip
 *     starts from B = S X^{-1} for the previous index set (computed as
 *     Gaussian elimination with partial pivoting whose pivots are restricted
 *     to that set, step t placing its pivot row in position t; the very
 *     first strip and the rows a grown cross lacks pivot freely) and then
 *     runs maxvol swaps, in double-float arithmetic;
 *   - after every sweep, k = #{sigma_j(M[I, J]) > tol sigma_1}.  If k = l,
 *     k < k_max, l < min(l_max, m, n) and unused columns of cand_J remain,
 *     the cross grows to min(2 l, l_max, m, n) with the next unused columns
 *     and the sweeps restart at that size;
 *   - otherwise U = (X_k)^+ with k_eff = min(k_max, k) and the Appendix F
 *     estimate on the sample rows x sample columns are written, and the block
 *     stops once k >= k_max, the estimate is <= tol, or `sweeps` sweeps were
 *     made at this size. */
typedef struct {
  int64_t row0, m;            /* rows of M in the block                             */
  int64_t col0, n;            /* columns of M in the block                          */
} lra_block;

typedef struct {
  int32_t l_init;             /* first cross size (1..l_max)                        */
  int32_t l_max;              /* largest cross size (<= 96)                         */
  int32_t k_max;              /* largest kept rank (<= l_max)                       */
  int32_t sweeps;             /* sweeps per cross size (>= 1)                       */
  int32_t max_swaps;          /* maxvol swap cap per strip (<= 0: 64 l)             */
  int32_t sample;             /* q: q x q sampled entries per block (0..64)         */
  double tol;                 /* rank tolerance (relative)                          */
  double delta;               /* maxvol stops when max |B| <= 1 + delta             */
  const int32_t* cand_J;      /* host, n_blocks x l_max distinct local columns      */
  const int32_t* sample_rows; /* host, n_blocks x q local rows (nullable if q = 0)  */
  const int32_t* sample_cols; /* host, n_blocks x q local columns                   */
  int32_t flags;              /* reserved, 0                                        */
  int32_t trace_cap;          /* decisions logged per block (0: none), <= 2^20      */
  /* Launch shape (0 = default; lra_cross_tune_batch picks them per workload).
   * None of them changes a block's result, only the time. */
  int32_t cluster_mask;       /* passes to run: bit c = clusters of 2^c CTAs (c = 0..3);
                                 the 8-CTA pass always runs last; 0: 1, 4, 8 CTAs   */
  int32_t cutover_side;       /* blocks whose larger side exceeds this skip the first
                                 pass and start in the next (0: none)               */
  int32_t order;              /* queue order: 0 as given, 1 largest (m + n) first   */
} lra_batch_params;

typedef struct {
  int32_t on_device;          /* 1: the pointers below are device pointers          */
  int32_t* status;            /* n_blocks lra_status values                         */
  int32_t* l;                 /* n_blocks final cross sizes                         */
  int32_t* k_eff;             /* n_blocks kept ranks                                */
  int32_t* swaps;             /* n_blocks maxvol swaps                              */
  int32_t* I;                 /* n_blocks x l_max local rows (-1 past l)            */
  int32_t* J;                 /* n_blocks x l_max local columns (-1 past l)         */
  double* U;                  /* n_blocks x l_max x l_max, the l x l nucleus row-major
                                 in the leading part of each block's slot (nullable);
                                 FP64: with cond(X_k) up to 1/tol an FP32 nucleus
                                 would dominate the error of C U R              */
  float* sigma;               /* n_blocks x l_max singular values of the cross (nullable) */
  double* est_err;            /* n_blocks Appendix F estimates (nullable)           */
  int32_t* trace_len;         /* n_blocks decisions logged (nullable; trace_cap > 0) */
  int32_t* trace;             /* n_blocks x trace_cap x 4: half_step, kind, i, j
                                 (local strip row and position), as lra_cur_out.trace;
                                 half-steps count from 0 per block (nullable)     */
  double* trace_val;          /* n_blocks x trace_cap: |value| of each decision (nullable) */
} lra_batch_out;

/* Section 9 (far-field generators of the multipole method), with C-A
 * iterations of Section 6.5 per block.  Validate and enqueue one persistent
 * launch over all blocks (LRA_EBUSY when admission fails; LRA_EINVAL for a
 * block outside the source, a side above 2048, repeated candidates).  The
 * host arrays of params are copied before the call returns.  Poll / wait /
 * cancel work on the returned job; per-block failures are reported in
 * lra_batch_out.status. */
lra_status lra_cross_submit_batch(lra_ctx* ctx, const lra_source* src, const lra_block* blocks,
                                  int32_t n_blocks, const lra_batch_params* params, lra_job* out);

/* ---- Cynical algorithms (Section 6.5), as in Tests 3 and 4 of Section 12.2
 * Tests 3: a Cynical algorithm with p = q: the r x r CUR generator of M is
 *   taken from the q x q submatrix M[K, L] (q = 4 r in the paper), as the
 *   generator of locally maximal volume that C-A iterations inside M[K, L]
 *   find (inner_sweeps sweeps from its first r columns, the first vertical
 *   step starting from Gaussian elimination).
 * Tests 4: outer_loops C-A loops on M with q x q generators from the
 *   columns L (giving K', L'), then Tests 3 on M[K', L'].
 * Output: I = K[I'], J = L[J'] and U = (M[I, J]_r)^+ (the inverse of a
 * nonsingular generator, as in Tests 1). */
typedef struct {
  int32_t r;                  /* generator size, 1 <= r <= q                         */
  int32_t q;                  /* |K| = |L| = q, q <= 96 and q <= min(m, n)           */
  int32_t outer_loops;        /* 0: Tests 3 (K and L given); >= 1: Tests 4            */
  int32_t inner_sweeps;       /* C-A sweeps inside M[K, L], >= 1                      */
  double delta;               /* maxvol stops when max |B| <= 1 + delta (> 0)         */
  double rank_tol;            /* nucleus keeps sigma_j > rank_tol sigma_1             */
  const int32_t* K;           /* host, q distinct rows (Tests 3; unused for Tests 4)  */
  const int32_t* L;           /* host, q distinct columns                             */
} lra_cynical_params;

typedef struct {
  int32_t* I;                 /* host, r rows of M                                   */
  int32_t* J;                 /* host, r columns of M                                */
  double* U;                  /* host, r x r nucleus, row-major                      */
  int32_t* K;                 /* host, q rows of the submatrix used (nullable)       */
  int32_t* L;                 /* host, q columns of the submatrix used (nullable)    */
} lra_cynical_out;

/* Run Tests 3 or 4 on ctx (blocking): the outer solve and the inner solve
 * are ordinary jobs of the context (its slots and budget apply), the
 * submatrix M[K, L] is gathered on the device with the entry kernel of
 * lra_gather_entries.  LRA_EINVAL for bad sizes or index sets; a job's own
 * failure status otherwise. */
lra_status lra_cross_cynical(lra_ctx* ctx, const lra_source* src, const lra_cynical_params* params,
                             const lra_cynical_out* out);

/* ---- Refinement of a C-A CUR by leverage scores (Section 7.2; Remark
 * resnrg: C-A iterations give a crude LRA M' = C U R, sampling refines it)
 * From the index sets (I, J) of a C-A solve: C = M[:, J], R = M[I, :], the
 * nucleus U = (X_r)^+ of X = M[I, J] at rank r = min(r, #{sigma_j >
 * rank_tol sigma_1}); the leverage scores (beta = 1, eq. levsc1) of the
 * columns and of the rows of M' (its top-r right and left singular
 * subspaces, Algorithm D.1 of Appendix D); Algorithm 7.1 with Exactly(l)
 * sampling and re-scaling (Algorithm C.1 of Appendix C, its uniforms given):
 * l columns `cols` with scales d, l rows `rows` with scales dbar, and the
 * nucleus U' = D (Mk_r)^+ Dbar of Mk = Dbar M[rows, cols] D, truncated at
 * rank r.  The refined approximation is M[:, cols] U' M[rows, :]. */
typedef struct {
  int32_t r;                  /* rank of the approximation (1..l)                     */
  int32_t l_new;              /* rows and columns sampled, 1..96 (a square generator) */
  double rank_tol;            /* singular values kept: sigma_j > rank_tol sigma_1     */
  const double* u_cols;       /* host, l_new uniforms in [0, 1): the column draws     */
  const double* u_rows;       /* host, l_new uniforms in [0, 1): the row draws        */
  int64_t resid_q, resid_s;   /* Appendix F sample of the refined CUR (0: none)       */
  const int32_t* resid_rows;  /* host, resid_q distinct rows                          */
  const int32_t* resid_cols;  /* host, resid_s distinct columns                       */
} lra_refine_params;

typedef struct {
  int32_t* cols;              /* host, l_new sampled columns (repeats possible)       */
  double* d;                  /* host, l_new column scales 1 / sqrt(l_new p_col)      */
  int32_t* rows;              /* host, l_new sampled rows                             */
  double* dbar;               /* host, l_new row scales                               */
  double* U;                  /* host, l_new x l_new nucleus U', row-major            */
  double* p_cols;             /* host, n column scores (nullable)                     */
  double* p_rows;             /* host, m row scores (nullable)                        */
  double* est_rel_err;        /* host, 1: Appendix F estimate of the refined CUR (nullable) */
  int32_t* k_eff;             /* host, 1: the rank used (nullable)                    */
} lra_refine_out;

/* Blocking; runs on ctx's first stream with memory from ctx's pool (not
 * counted against the admission budget).  I, J: host, l distinct rows and
 * columns (l <= 96), e.g. from lra_cross_fetch_cur.  LRA_EINVAL for bad
 * sizes or index sets; LRA_ESINGULAR when the cross has rank 0 or a score
 * basis turns out rank-deficient. */
lra_status lra_cross_refine(lra_ctx* ctx, const lra_source* src, const int32_t* I, const int32_t* J, int32_t l,
                            const lra_refine_params* params, const lra_refine_out* out);

/* Launch-shape tuner of the batched form (the paper has no counterpart:
 * the shape does not change any result).  Looks up, in the JSON file at
 * cache_path (NULL: no cache), the shape stored for this GPU (device name)
 * and the workload's bucket: source kind, l_max, k_max, and the powers of
 * two at or above the block count, the median and the largest block side.
 * Without an entry it runs the batch once per candidate shape (cluster
 * chains {1,4,8}, {1,2,8}, {1,2,4,8}, {1,8}, {2,4,8}; cut-over sides none,
 * 1024, 512; queue order as given or largest first), each twice, checks
 * that every candidate returns the same per-block l, k_eff, I, J and
 * estimate bit for bit (LRA_ECUDA with a message otherwise), keeps the
 * fastest (ties within 2% go to the default shape) and writes it to the
 * cache.  *tuned receives a copy of *params with cluster_mask, cutover_side
 * and order set; ms_default / ms_tuned (nullable) receive the device time of
 * one launch with the default and the chosen shape (-1 when the shape came
 * from the cache).  Blocking; uses ctx's slots and budget like any batch. */
lra_status lra_cross_tune_batch(lra_ctx* ctx, const lra_source* src, const lra_block* blocks, int32_t n_blocks,
                                const lra_batch_params* params, const char* cache_path, lra_batch_params* tuned,
                                double* ms_default, double* ms_tuned);

/* Host only (no device needed): the cache lookup of lra_cross_tune_batch for
 * a device named gpu_name.  LRA_OK with *tuned filled when the cache holds
 * this bucket, LRA_ENOTFOUND otherwise. */
lra_status lra_batch_tuning_lookup(const char* cache_path, const char* gpu_name, const lra_source* src,
                                   const lra_block* blocks, int32_t n_blocks, const lra_batch_params* params,
                                   lra_batch_params* tuned);

/* Section 9 / Section 6.5 (Primitive Algorithm outputs per block).  Wait for
 * the batch job, copy the per-block results into the caller's buffers (host
 * or device per out->on_device), then release the job; the handle is invalid
 * afterwards.  Returns the job's status (LRA_OK, or the failure that ended
 * the launch). */
lra_status lra_cross_fetch_batch(lra_ctx* ctx, lra_job job, const lra_batch_out* out);

/* Problem statement of Section 6.5 (an m x n matrix reachable entry by
 * entry, Section 1.1): a context owns the device state of the C-A solves on
 * params->device.  *out receives the handle.  LRA_ECUDA without a usable
 * device (or one without cooperative launch), LRA_ENOMEM when pinned host
 * memory cannot be had. */
lra_status lra_cross_create(lra_ctx** out, const lra_ctx_params* params);

/* Wait for every job, free all device memory and the context.  No other
 * call on ctx may run concurrently or follow. */
lra_status lra_cross_destroy(lra_ctx* ctx);

/* Section 6.5: Primitive Algorithm inputs (target rank k, cross size l,
 * Section 6.5 with r <= k <= l) and the C-A iterations (fixed number of
 * sweeps, or stop once the Appendix F estimate is <= tol: step 6 of the C-A
 * iterations).  Validate (LRA_EINVAL), admit (slots and memory budget;
 * LRA_EBUSY when full, LRA_ETOOLARGE when a strip cannot be held on chip)
 * and enqueue a full C-A solve on one of the context's streams.  The host
 * arrays of params are copied before the call returns; the source stays
 * borrowed until the job ends.  The context's own streams are non-blocking:
 * they do not wait for work queued on other streams, so the source's device
 * arrays must be complete when the call is made (synchronise their producer
 * first, or create the context on the producer's stream).  Non-blocking:
 * returns once the work is queued.  *out receives the job handle. */
lra_status lra_cross_submit(lra_ctx* ctx, const lra_source* src,
                            const lra_params* params, lra_job* out);

/* Step 4/6 of the C-A iterations of Section 6.5 (has the solve finished?).
 * Non-blocking: LRA_PENDING while the job runs, else LRA_OK with *out filled
 * (the job's own outcome is out->status).  LRA_ENOTFOUND for an unknown or
 * released handle. */
lra_status lra_cross_poll(lra_ctx* ctx, lra_job job, lra_info* out);

/* Blocking variant of lra_cross_poll (waits without holding the context's
 * lock).  The job must not be fetched or cancelled meanwhile by another
 * thread. */
lra_status lra_cross_wait(lra_ctx* ctx, lra_job job, lra_info* out);

/* Primitive Algorithm, stage 4 (Section 6.5): the outputs C = M[:, J],
 * U = (M[I, J]_k)^+ and R = M[I, :] of a solve.  Waits for the job (without
 * holding the context's lock: submit and poll from other threads go on),
 * copies I, J, U (and C, R, sigma, trace where non-NULL) into the caller's
 * buffers (host or device per out->on_device), then releases the job's slot
 * and device memory; the handle is invalid from the moment the call starts.
 * Returns the job's own status (the outputs are written only for LRA_OK). */
lra_status lra_cross_fetch_cur(lra_ctx* ctx, lra_job job, const lra_cur_out* out);

/* Step 6 of the C-A iterations of Section 6.5 (the caller ends the
 * iteration early).  Release a job: a job still running is first marked
 * LRA_ECANCELED (a copy on a control stream), so its kernels not yet started
 * return at once (a batch job takes no further block); then the call waits,
 * without holding the context's lock, for the job's stream work to end and
 * frees it.  The handle is invalid from the moment the call starts; the job
 * must not be waited on concurrently from another thread.  LRA_ENOTFOUND for
 * an unknown handle. */
lra_status lra_cross_cancel(lra_ctx* ctx, lra_job job);

/* Bytes of device memory a job with these arguments holds while admitted
 * (the measure that memory-budget admission charges).  LRA_EINVAL as for
 * submit. */
lra_status lra_cross_footprint(const lra_source* src, const lra_params* params,
                               uint64_t* bytes);

/* One maxvol half-step that allocates no device memory.  The paper has no
 * counterpart: this entry point exists for callers that cannot call
 * cudaMalloc/cudaFree while they run, for instance because those calls may
 * synchronise the whole device, or because another allocator (a framework's
 * caching allocator, a serving process that reserved its memory up front)
 * owns the device memory.
 *
 * It runs the same kernel as the maxvol step of lra_cross_submit on an N x l
 * FP32 strip S held by the caller in device memory, element (i, t) at
 * strip[i*row_stride + t*col_stride]:
 *   xinv == NULL: Gauss-Jordan start with partial pivoting, then maxvol swaps;
 *                 pos[0..l) receives the selected rows (device int32, output).
 *   xinv != NULL: warm start from pos[0..l) (device int32, in/out) with xinv
 *                 the row-major FP64 inverse of S[pos, :] (device, l x l).
 * status_out (device int32[3]) receives {lra_status, swaps, converged}.
 * Everything is enqueued on `stream` (cudaStream_t, NULL = legacy default);
 * the call returns without waiting for the GPU.
 *
 * Scratch: a static device array of about 325 KB (candidate words, candidate
 * rows of up to 96 entries for 160 CTAs, the caller's inverse split into
 * FP32 pairs, the grid barrier and the status word), present on every GPU
 * that loads this library until exit.
 * Limits: l <= 96, and the strip must fit the shared memory of <= 160 CTAs;
 * otherwise LRA_ETOOLARGE is returned and nothing is launched.  Bad pointers
 * or sizes return LRA_EINVAL, and so do strides that are not both >= 1 or
 * that make two of the N x l elements share an address (valid:
 * row_stride >= l * col_stride, or col_stride >= N * row_stride).
 * Errors: each launch is checked through its own return code; LRA_ECUDA
 * means the launch that failed and everything after it were not enqueued.
 * The runtime's last-error state is neither read nor cleared.
 * The first call on a device (with that device current) looks up the
 * device address of the array; make that first call before any stream
 * capture.  Every call shares the one array and clears what must start at
 * zero: calls whose kernels overlap on the GPU race, so issue them on one
 * stream (or otherwise serialise them). */
lra_status lra_maxvol_noalloc(const float* strip, int64_t N, int32_t l,
                              int64_t row_stride, int64_t col_stride, int32_t* pos,
                              const double* xinv, double delta, int32_t max_swaps,
                              int32_t* status_out, void* stream);

/* Section 8.1 (the fast product with H_{n,d}: d recursive steps, at most
 * 2dn additions per vector): G = H_{m,d} M H_{n,d} for the stored FP32 M
 * of an LRA_PRE_AH source (a, lda; pre_materialized = 0) with d = pre_d
 * <= 5, in one pass over M: every entry of M read once, every entry of G
 * written once (FP64 transforms in the order of the recursive steps,
 * rounded once to FP32: the same values as the entry-by-entry evaluation).
 * G: device FP32, m x n, row stride ldg >= n, not overlapping M.  A source
 * with a = G, lda = ldg and pre_materialized = 1 then gives the same
 * entries of M_bar with one read each.  Enqueued on `stream`; LRA_EINVAL
 * for another kind, d > 5 or ldg < n. */
lra_status lra_preprocess_materialize(const lra_source* pre, float* G, int64_t ldg, void* stream);

/* Section 6.6 (recovery of an LRA with nonsingular multipliers): from an
 * LRA Cbar U Rbar of the pre-processed M_bar = F M H of an LRA_PRE_AH
 * source (e.g. C, U, R of a solve on it), the factors of the induced LRA
 * A U B of M: A = F^T Cbar / 2^d (m x l) and B = Rbar H^T / 2^d (l x n),
 * since F F^T = 2^d I and H^T H = 2^d I; its error is the error on M_bar
 * divided by 2^d.  Cbar (m x l), Rbar (l x n), A, B: device FP32,
 * row-major; each entry an FP64 sum of 2^d terms in the order of the
 * recursive steps, scaled by 2^-d and rounded to FP32.
 * Enqueued on `stream` (takes m + n ints of stream-ordered scratch);
 * LRA_EINVAL for a source of another kind or l outside 1..96. */
lra_status lra_preprocessed_recover(const lra_source* pre, const float* Cbar, const float* Rbar, int32_t l, float* A,
                                    float* B, void* stream);

/* Section 12.2 (the C-A tests start from random columns): the initial
 * column set drawn from a seed, as submit draws it when init_J is NULL.
 * Host only (no device needed).  out: host int32[l], l distinct values of
 * [0, n) in the order drawn.  Generator: SplitMix64 (state = seed; each draw
 * adds 0x9E3779B97F4A7C15 to the state, then z ^= z >> 30, z *=
 * 0xBF58476D1CE4E5B9, z ^= z >> 27, z *= 0x94D049BB133111EB, z ^= z >> 31);
 * sample: Floyd's algorithm, for c = n - l ... n - 1 take t = draw mod
 * (c + 1), then t if new, else c.  LRA_EINVAL unless 1 <= l <= n <= 2^30. */
lra_status lra_draw_columns(uint64_t seed, int64_t n, int32_t l, int32_t* out);

/* Section 1.1 (the matrix is reachable entry by entry): out[a * s + b] =
 * M(rows[a], cols[b]) for a < q, b < s, as the FP32 values every kernel of
 * the library sees (stored FP64 entries rounded to FP32; generator entries
 * evaluated with the same FP32 operations).  rows, cols: device int32
 * arrays; out: device float[q * s], row-major.  An index outside M gives a
 * NaN entry and no memory access.  Enqueued on `stream` (cudaStream_t, NULL
 * = legacy default); returns without waiting.  LRA_EINVAL for a bad source
 * or size, LRA_ECUDA when the launch fails (checked through its own return
 * code). */
lra_status lra_gather_entries(const lra_source* src, const int32_t* rows, int64_t q,
                              const int32_t* cols, int64_t s, float* out, void* stream);

/* ---- Algorithm 5.1a: LRA via range finder with a sub-identity multiplier */

typedef struct {
  int32_t r;                  /* target rank, 1 <= r <= l                              */
  double rank_tol;            /* numerical rank of Y = M H: R_jj > rank_tol R_00 for the
                                 pivoted factor (>= 1e-7: the Gram route resolves R_jj
                                 to about sqrt(2^-53) R_00)                            */
  int64_t resid_q, resid_s;   /* optional Appendix F sample (0 = none)                  */
  const int32_t* resid_rows;  /* host, resid_q distinct rows                            */
  const int32_t* resid_cols;  /* host, resid_s distinct columns                         */
  /* Multiplier (Section 8.1's ASPH family, Section 3's recipe (i) for
   * mult_d = 0): column t of H is mult_sign[t] times column J[t] of the
   * d-abridged Hadamard matrix H_{n,d} (2^d must divide n); mult_d = 0 is
   * the sub-identity multiplier e_J (Y = M[:, J], mult_sign ignored). */
  int32_t mult_d;             /* 0 .. 10                                                */
  const float* mult_sign;     /* host, l signs +-1, or NULL (all +1)                    */
} lra_rf_params;

typedef struct {
  float* U;                   /* device, m x r row-major: orthonormal columns           */
  float* V;                   /* device, r x n row-major: U^T M                         */
  int32_t* piv;               /* host, l: column order of the pivoted QR of Y (indices
                                 into J)                                                */
  int32_t* nrank;             /* host: numerical rank of Y                              */
  double* est_rel_err;        /* host or NULL: Appendix F estimate of ||M - U V|| / ||M|| */
  int32_t* gemm_mode;         /* host or NULL: 1 = V on the tensor cores (FP32 emulated
                                 through BF16 products), 0 = FP32 SIMT                  */
} lra_rf_out;

/* Algorithm 5.1 (LRA via range finder), variant (a), with the sub-identity
 * multiplier H = (e_J[0], ..., e_J[l-1]) (Section 3's superfast recipe (i):
 * Y = M H = M[:, J] involves no flops) or an ASPH multiplier (mult_d > 0:
 * each entry of Y a signed sum of 2^d entries of M's row, in the order of
 * the recursive Hadamard steps, in FP32): Y is formed, its rank-revealing
 * QR is computed as pivoted Cholesky of the FP64 Gram matrix Y^T Y (the
 * pivots of QR with column pivoting in exact arithmetic) followed by a
 * CholeskyQR2 pass for the orthonormal factor, U = the r leftmost columns,
 * and V = U^+ M = U^T M by a GEMM over the stored matrix (cuBLAS, FP32
 * accuracy through BF16 tensor-core products where available).  The LRA of
 * M is U V.  src: LRA_DENSE_F32 (the GEMM reads M); J: host, l distinct
 * columns, r <= l <= 96.  Blocking.  LRA_EINVAL for bad sizes, source kind
 * or index sets; LRA_ESINGULAR (the algorithm's FAILURE) when the numerical
 * rank of Y is below r, with *nrank and piv set. */
lra_status lra_range_finder(lra_ctx* ctx, const lra_source* src, const int32_t* J, int32_t l,
                            const lra_rf_params* params, const lra_rf_out* out);

/* ---- Algorithm 3.1 with a sub-identity multiplier: superfast dual LSR */

typedef struct {
  int32_t passes;             /* CholeskyQR passes, 1..4 (3 by default)                  */
  int32_t shifted;            /* nonzero: the first passes - 2 passes (at least one)
                                 factor Y^T Y + s I, s = 11 (k (n+1) + (n+1) (n+2))
                                 2^-53 ||Y||_F^2 (shifted CholeskyQR; each shifted pass
                                 divides the condition number by about s^(-1/2) ||Y||,
                                 so 4 passes reach condition numbers near 1e14)         */
  /* Multiplier: row t of F is mult_sign[t] times row rows[t] of H_{m,d}
   * (the ASPH family of Section 8.1; 2^d must divide m); mult_d = 0 is the
   * sub-identity multiplier that keeps the rows (mult_sign ignored). */
  int32_t mult_d;             /* 0 .. 10                                                */
  const float* mult_sign;     /* host, k signs +-1, or NULL (all +1)                    */
} lra_lsr_params;

typedef struct {
  double* x;                  /* host, n: the least squares solution of the k rows      */
  double* rho;                /* host or NULL: the sampled problem's residual norm      */
} lra_lsr_out;

/* Problem 3.1 through Algorithm 3.1 with the multiplier F = sqrt(m/k)
 * (I_k | O) P (Section 3, "Superfast dual LSR": a permutation followed by a
 * sub-identity matrix, no flops), or with k rows of an ASPH multiplier
 * (mult_d > 0: each row of F W a signed sum of 2^d rows of W in the order of
 * the recursive Hadamard steps, in FP64): W = (A | b) is an m x (n+1) stored
 * matrix (LRA_DENSE_F64 or LRA_DENSE_F32; the last column is b); the k rows
 * `rows` (host, distinct, n+1 <= k <= m, n+1 <= 1024) are gathered in FP64
 * and x = argmin ||A[rows] x - b[rows]|| is computed by CholeskyQR
 * (Fukaya et al.) on the k x (n+1) matrix: (F W) = Q R_p ... R_1, x =
 * R_nn^{-1} R[:n, n].  The scale sqrt(m/k) does not change x.  Blocking.
 * LRA_EINVAL for bad sizes or rows; LRA_ESINGULAR when a Cholesky pivot is
 * not positive, or, in an unshifted pass, at most 1e-3 s_rel times its
 * column's squared norm (s = s_rel ||Y||_F^2 the shift above): the sampled
 * rows are numerically rank deficient, or too ill conditioned for the
 * passes given. */
lra_status lra_dual_lsr(lra_ctx* ctx, const lra_source* W, const int32_t* rows, int32_t k,
                        const lra_lsr_params* params, const lra_lsr_out* out);

/* Static message for a status code. */
const char* lra_status_str(int32_t status);

/* Message of the last failed call on ctx (thread-unsafe snapshot). */
const char* lra_cross_last_error(lra_ctx* ctx);

#ifdef __cplusplus
}
#endif

#endif /* LRA_CROSS_H */
