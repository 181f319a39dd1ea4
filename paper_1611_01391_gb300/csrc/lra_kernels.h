// Host-side launchers of the library's kernels (one per translation unit).
#pragma once

#include <cuda_runtime.h>

#include "lra_internal.cuh"

struct lra_ctx;

namespace lra {

// Context accessors for the other translation units of the runtime.
int ctx_device(::lra_ctx* ctx);
void set_ctx_error(::lra_ctx* ctx, const char* msg);

struct SourceDev;
struct JobStatus;
struct GridBarrier;

cudaError_t launch_gather_cols(const SourceDev& s, const int* J, int l, float* C,
                               const JobStatus* js, int skip_on_stop, int sms,
                               cudaStream_t st);
// Opaque copy of a CUtensorMap (128 bytes, 64-byte aligned), so that
// translation units without the driver header can hold one.
struct alignas(64) TmaMap {
  unsigned char bytes[128];
};
// Tensor map of a stored FP32 matrix for launch_gather_cols_tma (false when
// the base is not 16-byte aligned, lda is not a multiple of 4, or encoding
// fails).
bool make_cols_map(TmaMap* map, const float* a, long long m, long long n, long long lda);
cudaError_t launch_gather_cols_tma(const TmaMap& map, const int* J, int l, long long m, float* C, JobStatus* js,
                                   int skip_on_stop, int sms, cudaStream_t st);
cudaError_t launch_gather_entries(const SourceDev& s, const int* rows, long long q, const int* cols,
                                  long long sN, float* out, cudaStream_t st);
cudaError_t launch_gather_rows(const SourceDev& s, const int* I, int l, float* R,
                               const JobStatus* js, int sms, cudaStream_t st, int skip_on_stop = 1);

// One maxvol half-step on an N x l FP32 strip whose element (i, t) sits at
// strip[i*si + t*st].  gepp = 1: Gauss-Jordan elimination with partial
// pivoting selects the initial rows; gepp = 0: warm start from pos[] with xin
// = inverse of the strip's cross S[pos, :] (row-major, each entry split into
// an FP32 pair x + y, see split_double), or with self_inverse set, the
// launch inverts the cross itself.  On exit pos[] holds the selected rows.
struct MaxvolArgs {
  const float* strip;
  long long N;
  int l;
  long long si, st;
  int gepp;
  int* pos;
  const float2* xin;
  unsigned long long* win_ring;  // kWinRing candidate words (zero for a new job)
  float2* cand_rows;   // one published row of W per CTA and buffer (pairs)
  GridBarrier* bar;
  JobStatus* js;
  int* trace_i;
  double* trace_v;
  int half_step;
  double delta;
  int max_swaps;
  int rows_per_cta;
  int stage_xinv;   // copy X^{-1} into shared memory for the warm start
  int self_inverse; // warm start: every CTA inverts S[pos, :] itself (xin unused);
                    // needs a plan with stage_xinv
  int count_sweep;  // the last half-step of a sweep: count it in js->sweeps_done
  // gen != 0: the strip is not in memory; its entries are evaluated from a
  // generator source (Cauchy, Gaussian or inverse-distance kernel): gen = 1,
  // S[i][t] = M(i, gen_idx[t]) (vertical strip); gen = 2, S[i][t] =
  // M(gen_idx[t], i) (horizontal strip, i.e. R^T)
  int gen;
  const int* gen_idx;
  SourceDev src;
  // fixed_point_exit: once two warm-started half-steps in a row make no
  // swap, the iteration is at a fixed point and every later half-step of
  // the budget (total_half_steps) would repeat the same decisions; the
  // launch then logs their STOP decisions, counts their sweeps and sets
  // js->stop, and the later launches return at once
  int fixed_point_exit;
  int total_half_steps;
};

struct MaxvolPlan {
  int grid;
  int threads;
  int rows_per_cta;
  int stage_xinv;
  size_t smem;
};

// Grid and shared-memory plan for a strip; returns false if it cannot be
// held on chip.
bool plan_maxvol(long long N, int l, int sms, size_t smem_limit, MaxvolPlan* plan);
cudaError_t launch_maxvol(MaxvolArgs a, const MaxvolPlan& plan, cudaStream_t st);

// Inverse of the cross S[pos, :] of a strip (double-float Gauss-Jordan with
// partial pivoting), row-major into xinv as FP32 pairs: on one CTA, or with
// cluster set and l = 96 on a cluster of 8 CTAs (the same result bit for
// bit, for a job that has the GPU to itself).
cudaError_t launch_cross_inverse(const float* strip, long long si, long long st, const int* pos,
                                 int l, float2* xinv, JobStatus* js, cudaStream_t stream, bool cluster = false);

// Nucleus of the final cross X = C[I, :] (one CTA, double-float QRCP +
// one-sided Jacobi SVD).  NucExtra (all nullable): row / column scales of X
// (with them U is diag(cs) (X_k)^+ diag(rs)), and outputs for the kept left
// (Pk) and right (Vk) singular vectors as l x l row-major columns.
struct NucExtra {
  const double* rs = nullptr;
  const double* cs = nullptr;
  double* Pk = nullptr;
  double* Vk = nullptr;
};
// cluster: with l = 48 or 96 on a cluster of 8 or 16 CTAs (the same result
// bit for bit, for a job that has the GPU to itself).
cudaError_t launch_nucleus(const float* C, const int* I, int l, int k, double rank_tol,
                           double* U, double* sigma, JobStatus* js, cudaStream_t st,
                           const NucExtra& xa = NucExtra(), bool cluster = false);

// Appendix F sampled residual of C U R on rows x cols.
cudaError_t launch_sampled_residual(const SourceDev& s, const int* rows, int q,
                                    const int* cols, int sN, int l, const float* C,
                                    const double* U, const float* R, float* CUq,
                                    double* partials, int max_partials, JobStatus* js,
                                    cudaStream_t st);
int sampled_residual_partials(int q, int sN);

// Full residual ||A - C U R||_F / ||A||_F of a stored FP32 matrix on the
// tensor cores (tcgen05); ws holds fullres_workspace_bytes(m, n, l, grid_cap).
size_t fullres_workspace_bytes(long long m, long long n, int l, int grid_cap);
cudaError_t launch_full_residual(const float* A, long long lda, long long m, long long n, int l,
                                 const float* C, const double* U, const float* R, void* ws,
                                 int grid_cap, JobStatus* js, cudaStream_t st);

// Batched C-A: one persistent launch of 4-CTA clusters over a work queue.
struct BatchArgs;
// Opt a kernel in to `bytes` of dynamic shared memory on the current device
// (the attribute is per device; done once per kernel, device and size).
cudaError_t smem_optin(const void* func, int bytes);

size_t batch_smem_bytes();
cudaError_t launch_batch(const BatchArgs& a, int cluster_mask, int sms, cudaStream_t st);

// Leverage scores of a C-A approximation and Exactly(l) sampling (k_lev.cu).
int lev_partials(long long N);
cudaError_t launch_lev_factors(const double* U, const double* Pk, const double* Vk, int l, int k, double* G1,
                               double* G2t, const JobStatus* js, cudaStream_t st);
cudaError_t launch_lev_project(const float* S, long long N, int l, long long si, long long st_, const double* G,
                               int k, double* Y, double* partials, int nparts, const JobStatus* js,
                               cudaStream_t st);
cudaError_t launch_lev_chol(const double* partials, int nparts, int k, double* Linv, JobStatus* js,
                            cudaStream_t st);
cudaError_t launch_lev_scores_sample(const double* Y, long long N, int k, const double* Linv, double* w,
                                     const double* u, int ls, int* idx, double* d, double* scores,
                                     const JobStatus* js, cudaStream_t st);

// Section 6.6: A = F^T Cbar / 2^d and B = Rbar H^T / 2^d for the abridged
// Hadamard multipliers of a pre-processed source; inv: m + n ints of scratch.
// Section 8.1: G = H_{m,d} M H_{n,d} in one pass (d <= 5).
cudaError_t launch_pre_materialize(const float* M, long long lda, float* G, long long ldg, long long m, long long n,
                                   int d, cudaStream_t st);
cudaError_t launch_pre_recover(const SourceDev& s, const float* Cbar, const float* Rbar, int l, float* A, float* B,
                               int* inv, cudaStream_t st);

// Range finder and dual LSR (k_rf.cu): tall-skinny FP64 factorisations.
int ts_gram_chunks(long long N, int k);
cudaError_t launch_ts_gram_f32(const float* Y, long long N, int k, long long si, long long st, double* partials,
                               int nchunks, const JobStatus* js, cudaStream_t s);
cudaError_t launch_ts_gram_f64(const double* Y, long long N, int k, double* partials, int nchunks,
                               const JobStatus* js, cudaStream_t s);
cudaError_t launch_pchol(const double* partials, int nparts, int k, int r, double rank_tol, double* Gm, int* piv,
                         JobStatus* js, cudaStream_t s);
cudaError_t launch_rf_finish(const double* Q1, long long N, int r, const double* Linv, float* U, const JobStatus* js,
                             int sms, cudaStream_t s);
cudaError_t launch_gather_rows_f64(const SourceDev& src, const int* rows, int k, double* FW, int sms, cudaStream_t s);
cudaError_t launch_asph_cols(const float* M, long long lda, long long m, long long n, int d, const int* J,
                             const float* sign, int l, float* Y, int sms, cudaStream_t s);
cudaError_t launch_asph_rows_f64(const SourceDev& src, int d, const int* rows, const float* sign, int k, double* FW,
                                 int sms, cudaStream_t s);
cudaError_t launch_chol_coop(const double* partials, int nparts, int k, double shift_rel, double floor_rel,
                             double* G, double* Gd, double* R, double* Rt, unsigned int* bar, JobStatus* js, int sms,
                             cudaStream_t s);
cudaError_t launch_trsm_rows(const double* W, long long N, int k, const double* Rt, double* Q, const JobStatus* js,
                             int sms, cudaStream_t s);
cudaError_t launch_lsr_solve(const double* Rs, int p, int k, double* v, double* x, double* rho, const JobStatus* js,
                             cudaStream_t s);

// Small control kernels.
cudaError_t launch_tol_check(JobStatus* js, double tol, cudaStream_t st);

}  // namespace lra
