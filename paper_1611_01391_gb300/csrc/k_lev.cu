// Leverage scores of a C-A approximation and Exactly(l) sampling: the
// refinement of Section 7.2 (Remark resnrg: C-A iterations give a crude
// CUR, sampling by leverage scores refines it; Algorithm 7.1, Appendix C
// Algorithm C.1).
//
// The C-A approximation is M' = C U R with U = (X_k)^+ = V_k S_k^{-1} P_k^T
// for the cross X = M[I, J] = P S V^T.  Written as M' = H S_k Z with
//     H = C U P_k = C V_k S_k^{-1}        (m x k),
//     Z = V_k^T U R = S_k^{-1} P_k^T R    (k x n),
// its top-k left singular subspace is range(H) and the right one range(Z^T).
// In exact arithmetic C = B_C X with B_C = C X^{-1} the interpolation matrix
// of the vertical strip (the identity on the rows I, other entries bounded
// near 1 by maxvol), so H = B_C P_k has singular values >= 1 and of the
// order of its size: it is well conditioned even when C and X are not (the
// Cauchy strips have kappa ~ 1e8).  The same holds for Z.  So the scores
// come from FP64 Gram matrices of H and Z^T (condition squared but small),
// their Cholesky factors L, and the squared row norms of H L^{-T}:
//     p_i = ||L^{-1} h_i||^2 / sum_i ||L^{-1} h_i||^2,
// the squared row norms of an orthonormal basis of the subspace, i.e. the
// SVD-based leverage scores with beta = 1 (eq. levsc1).  The rounding
// errors of the FP64 products C (U P_k) relative to H stay at about
// 2^-53 kappa(X); the singular vectors from the double-float SVD of the
// nucleus bring about 2^-48 kappa(X_k).
#include <cfloat>

#include "lra_internal.cuh"
#include "lra_kernels.h"

namespace lra {
namespace {

constexpr int kLevThreads = 256;
constexpr int kGramThreads = 512;
constexpr int kSmallThreads = 1024;

// G1[p][t] = sum_q U[p][q] Pk[q][t],  G2t[q][t] = sum_p U[p][q] Vk[p][t],
// t < k (U, Pk, Vk l x l row-major; G1, G2t l x k row-major).
__global__ void __launch_bounds__(kSmallThreads) lev_factors_kernel(const double* __restrict__ U,
                                                                    const double* __restrict__ Pk,
                                                                    const double* __restrict__ Vk, int l,
                                                                    int k, double* __restrict__ G1,
                                                                    double* __restrict__ G2t,
                                                                    const JobStatus* js) {
  if (js->status != LRA_OK) return;
  for (int e = threadIdx.x; e < l * k; e += blockDim.x) {
    const int a = e / k, t = e - a * k;
    double g1 = 0.0, g2 = 0.0;
    for (int c = 0; c < l; ++c) {
      g1 = fma(U[(size_t)a * l + c], Pk[(size_t)c * l + t], g1);
      g2 = fma(U[(size_t)c * l + a], Vk[(size_t)c * l + t], g2);
    }
    G1[e] = g1;
    G2t[e] = g2;
  }
}

// Y[i][t] = sum_c S(i, c) G[c][t] for the N x l FP32 strip S (element (i, c)
// at S[i*si + c*st]) and the l x k FP64 matrix G; Y is N x k row-major.
// A CTA takes kProjRows rows at a time: their entries are converted to FP64
// once, into shared memory beside G (not once per output: on this part the
// conversion runs on the FP64 pipe like the multiply-add), then thread
// (row, t) sums over c in order; consecutive threads take consecutive t.
constexpr int kProjRows = 32;

__global__ void __launch_bounds__(kLevThreads) lev_project_kernel(const float* __restrict__ S, long long N,
                                                                  int l, long long si, long long st,
                                                                  const double* __restrict__ G, int k,
                                                                  double* __restrict__ Y,
                                                                  const JobStatus* js) {
  if (js->status != LRA_OK) return;
  extern __shared__ double lp_sm[];
  double* Gs = lp_sm;                    // l x k
  double* Ss = lp_sm + (size_t)l * k;    // kProjRows x l
  for (int e = threadIdx.x; e < l * k; e += blockDim.x) Gs[e] = G[e];
  for (long long r0 = (long long)blockIdx.x * kProjRows; r0 < N; r0 += (long long)gridDim.x * kProjRows) {
    const int nr = (int)min((long long)kProjRows, N - r0);
    __syncthreads();   // the previous rows' reads done (G in place on the first pass)
    for (int e = threadIdx.x; e < nr * l; e += blockDim.x) {
      const int r = e / l, c = e - r * l;
      Ss[e] = (double)__ldg(S + (r0 + r) * si + (long long)c * st);
    }
    __syncthreads();
    for (int e = threadIdx.x; e < nr * k; e += blockDim.x) {
      const int r = e / k, t = e - r * k;
      const double* srow = Ss + (size_t)r * l;
      double acc = 0.0;
      for (int c = 0; c < l; ++c) acc = fma(srow[c], Gs[c * k + t], acc);
      Y[(r0 + r) * k + t] = acc;
    }
  }
}

// Per-CTA partial Gram matrices Y^T Y (k x k, upper triangle with the
// diagonal) over a contiguous range of rows; partials[b][a*k + c].
__global__ void __launch_bounds__(kGramThreads) lev_gram_kernel(const double* __restrict__ Y, long long N,
                                                                int k, double* __restrict__ partials,
                                                                const JobStatus* js) {
  if (js->status != LRA_OK) return;
  const long long per = (N + gridDim.x - 1) / gridDim.x;
  const long long r0 = blockIdx.x * per, r1 = min(N, r0 + per);
  double* out = partials + (size_t)blockIdx.x * k * k;
  for (int e = threadIdx.x; e < k * k; e += blockDim.x) {
    const int a = e / k, c = e - a * k;
    double acc = 0.0;
    if (c >= a)
      for (long long i = r0; i < r1; ++i) acc = fma(Y[i * k + a], Y[i * k + c], acc);
    out[e] = acc;
  }
}

// One CTA: G = sum of the partials (fixed order), Cholesky G = L L^T
// (column by column), Linv = L^{-1} (lower triangular), k x k row-major.
// A non-positive pivot (a rank-deficient basis) sets LRA_ESINGULAR.
__global__ void __launch_bounds__(kSmallThreads) lev_chol_kernel(const double* __restrict__ partials,
                                                                 int nparts, int k,
                                                                 double* __restrict__ Linv, JobStatus* js) {
  if (js->status != LRA_OK) return;
  extern __shared__ double chol_sm[];   // G and L, k x k each
  double* G = chol_sm;
  double* Lm = chol_sm + k * k;
  __shared__ int bad;
  const int tid = threadIdx.x;
  if (tid == 0) bad = 0;
  for (int e = tid; e < k * k; e += blockDim.x) {
    const int a = e / k, c = e - a * k;
    double s = 0.0;
    if (c >= a)
      for (int b = 0; b < nparts; ++b) s += partials[(size_t)b * k * k + e];
    G[e] = s;
    Lm[e] = 0.0;
  }
  __syncthreads();
  for (int e = tid; e < k * k; e += blockDim.x) {   // symmetric completion
    const int a = e / k, c = e - a * k;
    if (c < a) G[e] = G[c * k + a];
  }
  __syncthreads();
  for (int j = 0; j < k; ++j) {
    if (tid == 0) {
      double d = G[j * k + j];
      for (int c = 0; c < j; ++c) d -= Lm[j * k + c] * Lm[j * k + c];
      if (!(d > 0.0)) {
        bad = 1;
        d = 1.0;
      }
      Lm[j * k + j] = sqrt(d);
    }
    __syncthreads();
    for (int i = j + 1 + tid; i < k; i += blockDim.x) {
      double v = G[i * k + j];
      for (int c = 0; c < j; ++c) v -= Lm[i * k + c] * Lm[j * k + c];
      Lm[i * k + j] = v / Lm[j * k + j];
    }
    __syncthreads();
  }
  if (bad) {
    if (tid == 0) set_status(js, LRA_ESINGULAR);
    return;
  }
  // Linv column by column: L x = e_c, forward substitution
  for (int c = tid; c < k; c += blockDim.x) {
    for (int i = 0; i < k; ++i) {
      double v = (i == c) ? 1.0 : 0.0;
      for (int q = c; q < i; ++q) v -= Lm[i * k + q] * Linv[(size_t)q * k + c];
      Linv[(size_t)i * k + c] = i < c ? 0.0 : v / Lm[i * k + i];
    }
  }
}

// w_i = ||Linv y_i||^2 for every row of Y (N x k).
__global__ void __launch_bounds__(kLevThreads) lev_scores_kernel(const double* __restrict__ Y, long long N, int k,
                                                                 const double* __restrict__ Linv,
                                                                 double* __restrict__ w,
                                                                 const JobStatus* js) {
  if (js->status != LRA_OK) return;
  extern __shared__ double Ls[];   // k x k
  for (int e = threadIdx.x; e < k * k; e += blockDim.x) Ls[e] = Linv[e];
  __syncthreads();
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N;
       i += (long long)gridDim.x * blockDim.x) {
    const double* y = Y + i * k;
    double s = 0.0;
    for (int a = 0; a < k; ++a) {
      double v = 0.0;
      for (int c = 0; c <= a; ++c) v = fma(Ls[a * k + c], y[c], v);
      s = fma(v, v, s);
    }
    w[i] = s;
  }
}

// Algorithm C.1 (Exactly(l)) with its uniforms given, one CTA: the
// cumulative sums of w in a fixed order (each thread a contiguous chunk,
// chunk offsets by a sequential scan), then for draw t the smallest i with
// cumsum_i > u_t total, and d_t = 1 / sqrt(l w_i / total).
__global__ void __launch_bounds__(kSmallThreads) lev_sample_kernel(const double* __restrict__ w, long long N,
                                                                   const double* __restrict__ u, int ls,
                                                                   int* __restrict__ idx, double* __restrict__ d,
                                                                   double* __restrict__ scores,
                                                                   const JobStatus* js) {
  if (js->status != LRA_OK) return;
  __shared__ double off[kSmallThreads + 1];
  const int tid = threadIdx.x, nt = blockDim.x;
  const long long per = (N + nt - 1) / nt;
  const long long c0 = tid * per, c1 = min(N, c0 + per);
  double s = 0.0;
  for (long long i = c0; i < c1; ++i) s += w[i];
  off[tid + 1] = s;
  __syncthreads();
  if (tid == 0) {
    off[0] = 0.0;
    for (int q = 1; q <= nt; ++q) off[q] += off[q - 1];
  }
  __syncthreads();
  const double total = off[nt];   // the scan's own total, in the scan's order
  if (scores)
    for (long long i = blockIdx.x * (long long)nt + tid; i < N; i += (long long)nt) scores[i] = w[i] / total;
  for (int t = tid; t < ls; t += nt) {
    const double target = u[t] * total;
    // the chunk: the last q with off[q] <= target
    int lo = 0, hi = nt;
    while (hi - lo > 1) {
      const int mid = (lo + hi) / 2;
      if (off[mid] <= target) lo = mid; else hi = mid;
    }
    const long long a0 = lo * per, a1 = min(N, a0 + per);
    double run = off[lo];
    long long pick = N - 1;
    for (long long i = a0; i < a1; ++i) {
      run += w[i];
      if (run > target) {
        pick = i;
        break;
      }
    }
    while (pick > 0 && !(w[pick] > 0.0)) --pick;   // never a zero-probability index
    idx[t] = (int)pick;
    d[t] = 1.0 / sqrt((double)ls * (w[pick] / total));
  }
}

}  // namespace

int lev_partials(long long N) {
  long long g = (N + 1023) / 1024;
  if (g < 1) g = 1;
  if (g > 304) g = 304;
  return (int)g;
}

cudaError_t launch_lev_factors(const double* U, const double* Pk, const double* Vk, int l, int k, double* G1,
                               double* G2t, const JobStatus* js, cudaStream_t st) {
  lev_factors_kernel<<<1, kSmallThreads, 0, st>>>(U, Pk, Vk, l, k, G1, G2t, js);
  return cudaGetLastError();
}

cudaError_t launch_lev_project(const float* S, long long N, int l, long long si, long long stv, const double* G,
                               int k, double* Y, double* partials, int nparts, const JobStatus* js,
                               cudaStream_t st) {
  long long g = (N + kProjRows - 1) / kProjRows;
  if (g > 152 * 3) g = 152 * 3;
  if (g < 1) g = 1;
  const int sm = (int)(sizeof(double) * ((size_t)l * k + (size_t)kProjRows * l));
  cudaError_t e = smem_optin(reinterpret_cast<const void*>(lev_project_kernel), sm);
  if (e) return e;
  lev_project_kernel<<<(int)g, kLevThreads, sm, st>>>(S, N, l, si, stv, G, k, Y, js);
  if (nparts > 0) lev_gram_kernel<<<nparts, kGramThreads, 0, st>>>(Y, N, k, partials, js);
  return cudaGetLastError();
}

cudaError_t launch_lev_chol(const double* partials, int nparts, int k, double* Linv, JobStatus* js,
                            cudaStream_t st) {
  const int sm = (int)(sizeof(double) * 2 * k * k);
  cudaError_t e = smem_optin(reinterpret_cast<const void*>(lev_chol_kernel), sm);
  if (e) return e;
  lev_chol_kernel<<<1, kSmallThreads, sm, st>>>(partials, nparts, k, Linv, js);
  return cudaGetLastError();
}

cudaError_t launch_lev_scores_sample(const double* Y, long long N, int k, const double* Linv, double* w,
                                     const double* u, int ls, int* idx, double* d, double* scores,
                                     const JobStatus* js, cudaStream_t st) {
  const int sm = (int)(sizeof(double) * k * k);
  cudaError_t e = smem_optin(reinterpret_cast<const void*>(lev_scores_kernel), sm);
  if (e) return e;
  long long g = (N + kLevThreads - 1) / kLevThreads;
  if (g > 152 * 4) g = 152 * 4;
  lev_scores_kernel<<<(int)g, kLevThreads, sm, st>>>(Y, N, k, Linv, w, js);
  lev_sample_kernel<<<1, kSmallThreads, 0, st>>>(w, N, u, ls, idx, d, scores, js);
  return cudaGetLastError();
}

}  // namespace lra
