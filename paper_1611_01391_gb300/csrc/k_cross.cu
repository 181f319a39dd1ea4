// Nucleus of the CUR approximation (Primitive Algorithm, stages 2-3 of
// Section 6.5): the l x l CUR generator X = M[I, J], its SVD, the rank-k
// truncation and U = (X_k)^+.  Also the inverse of a strip's cross for the
// warm start of maxvol (Section 6.5, each half-step from the previous
// index set).
//
// The SVD (svd_dd.cuh) is QR with column pivoting followed by one-sided
// Jacobi on R^T, in double-float arithmetic; the left singular vectors of
// the kept triplets are X v_b / sigma_b.  X is first scaled by a power
// of two so that max |X| lies in [0.5, 1) (exact); sigma and U are scaled
// back.
#include <cfloat>

#include "lra_kernels.h"
#include "lra_internal.cuh"
#include "inverse_dd.cuh"
#include "svd_dd.cuh"

namespace lra {

constexpr int kNucThreads = 512;

// L > 0: a build for l == L exactly (the served cross sizes); L == 0: any l.
// Optional (NucExtra, all nullable): row and column scales of the cross,
// X[a][b] = rs[a] C[I[a]][b] cs[b] (then U is returned as
// diag(cs) (X_k)^+ diag(rs), the nucleus of the unscaled factors), and the
// kept singular vectors: Pk[q*l + r] = u_r[q] (left, over the rows of X),
// Vk[p*l + r] = v_r[p] (right, over the columns of X), r < k_eff, zero
// beyond.
template <int L>
__global__ void __launch_bounds__(kNucThreads, 1)
nucleus_kernel(const float* __restrict__ C, const int* __restrict__ I, int l_arg, int k,
               double rank_tol, double* __restrict__ U, double* __restrict__ sigma_out,
               JobStatus* js, NucExtra xa) {
  if (js->status != LRA_OK) return;
  const int l = L > 0 ? L : l_arg;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  dd* W = reinterpret_cast<dd*>(smem_raw);           // column b at W + b*l
  dd* Z = W + (size_t)l * l;                          // column b at Z + b*l
  double* sig = reinterpret_cast<double*>(Z + (size_t)l * l);  // l
  dd* inv2 = reinterpret_cast<dd*>(sig + kMaxL);      // l
  SvdScratch* sc = reinterpret_cast<SvdScratch*>(inv2 + kMaxL);
  int* order = reinterpret_cast<int*>(sc + 1);        // l: order[rank] = column
  int* keff_s = order + kMaxL;
  int* scale_e = keff_s + 1;

  const int tid = threadIdx.x, nthr = blockDim.x;
  if (tid == 0) *scale_e = 0;
  __syncthreads();
  // power-of-two scale so that max |X| is in [0.5, 1)
  const bool scaled = xa.rs != nullptr;
  float amax = 0.0f;
  for (int e = tid; e < l * l; e += nthr) {
    const int a = e / l, b = e - a * l;
    const float c = C[(size_t)__ldg(I + a) * l + b];
    amax = fmaxf(amax, scaled ? (float)fabs((double)c * xa.rs[a] * xa.cs[b]) : fabsf(c));
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) amax = fmaxf(amax, __shfl_xor_sync(0xffffffffu, amax, off));
  if ((tid & 31) == 0 && amax > 0.0f) {
    int ex;
    frexpf(amax, &ex);
    atomicMax(scale_e, ex + 1024);  // offset keeps the stored value positive
  }
  __syncthreads();
  const int ex = *scale_e ? *scale_e - 1024 : 0;
  for (int e = tid; e < l * l; e += nthr) {
    const int a = e / l, b = e - a * l;             // X[a][b] = C[I[a]][b]
    const float c = C[(size_t)__ldg(I + a) * l + b];
    // scaled crosses: the entry times its row and column scale, as a pair
    // (the FP32 entry is exact; the FP64 scale product rounds to 48 bits)
    W[(size_t)b * l + a] = scaled ? dd_mul(dd_make(c), dd_from_double(ldexp(xa.rs[a] * xa.cs[b], -ex)))
                                  : dd_make(ldexpf(c, -ex));
  }
  __syncthreads();
  svd_dd<kNucThreads, L>(W, Z, l, sc);
  jacobi_sigma<kNucThreads>(W, l, sig, order);
  if (tid == 0) {
    const double s1 = sig[order[0]];
    int ke = 0;
    if (s1 > 0.0)
      while (ke < k && ke < l && sig[order[ke]] > rank_tol * s1) ++ke;
    *keff_s = ke;
    js->k_eff = ke;
    js->sigma_max = ldexp(s1, ex);
  }
  for (int r = tid; r < l; r += nthr) {
    const double sb = sig[order[r]];
    inv2[r] = dd_from_double(sb > 0.0 ? 1.0 / (sb * sb) : 0.0);
    sigma_out[r] = ldexp(sb, ex);
  }
  __syncthreads();
  const int ke = *keff_s;
  left_vectors<kNucThreads, L>(W, Z, l, ke, order, inv2, sc->perm);
  if (xa.Vk) {
    // right singular vector r = P W_{b_r} / sigma_{b_r}; left = column r of Z
    for (int e = tid; e < l * l; e += nthr) {
      const int c = e / l, r = e - c * l;   // entry c of vector r
      double v = 0.0, u = 0.0;
      if (r < ke) {
        const int b = order[r];
        v = dd_to_double(W[(size_t)b * l + c]) / sig[b];
        u = dd_to_double(Z[(size_t)r * l + c]);
      }
      xa.Vk[(size_t)sc->perm[c] * l + r] = v;
      xa.Pk[(size_t)c * l + r] = u;
    }
  }
  if (scaled) {
    nucleus_from_svd<kNucThreads, L>(W, Z, sc->perm, l, ke, order, inv2, [&](int e, double v) {
      const int p = e / l, q = e - p * l;   // U[p][q]: p a column of X, q a row
      U[e] = xa.cs[p] * ldexp(v, -ex) * xa.rs[q];
    });
  } else {
    nucleus_from_svd<kNucThreads, L>(W, Z, sc->perm, l, ke, order, inv2,
                                  [&](int e, double v) { U[e] = ldexp(v, -ex); });
  }
}

// X^{-1} of the cross X[a][b] = S[pos[a]][b] of a strip, by one CTA of
// 1024 threads in double-float arithmetic (inverse_dd.cuh: Gauss-Jordan
// with partial pivoting and a one-step look-ahead), written row-major as
// FP32 pairs with the row interchanges undone.  One SM: the jobs of a serving context keep the
// other SMs.
constexpr int kInvThreads = 1024;

template <int L>   // L > 0: a build for l == L exactly
__global__ void __launch_bounds__(kInvThreads, 1)
cross_inverse_kernel(const float* __restrict__ strip, long long si, long long st,
                     const int* __restrict__ pos, int l_arg, float2* __restrict__ xinv, JobStatus* js) {
  if (js->status != LRA_OK || js->stop) return;
  const int l = L > 0 ? L : l_arg;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  dd* A0 = reinterpret_cast<dd*>(smem_raw);                  // l * l
  dd* A1 = A0 + (size_t)l * l;                                // l * l
  InvLaScratch w;
  w.stride = kMaxL;
  w.rowt = A1 + (size_t)l * l;           // 2 * kMaxL
  w.colt = w.rowt + 2 * kMaxL;           // 2 * kMaxL
  w.swaps = reinterpret_cast<int*>(w.colt + 2 * kMaxL);
  w.at = w.swaps + kMaxL;
  w.pinfo = w.at + kMaxL;
  int* pos_s = w.pinfo + 2;                                   // l
  for (int t = threadIdx.x; t < l; t += blockDim.x) pos_s[t] = pos[t];
  __syncthreads();
  const dd* A = invert_cross_la<kInvThreads, L>(strip, si, st, l, js, pos_s, A0, A1, w);
  if (!A) return;
  for (int e = threadIdx.x; e < l * l; e += blockDim.x) {
    const int r = e / l, q = e - r * l;
    const dd v = A[(size_t)r * l + w.at[q]];
    xinv[e] = make_float2(v.hi, v.lo);
  }
}

static size_t inverse_smem(int l) {
  return 2 * (size_t)l * l * sizeof(dd) + 4 * kMaxL * sizeof(dd) + (3 * kMaxL + 2) * sizeof(int);
}

template <int L>
static cudaError_t launch_inverse_l(const float* strip, long long si, long long st, const int* pos,
                                    int l, float2* xinv, JobStatus* js, cudaStream_t stream) {
  const size_t smem = inverse_smem(l);
  const cudaError_t e = smem_optin(reinterpret_cast<const void*>(cross_inverse_kernel<L>), (int)smem);
  if (e) return e;
  cross_inverse_kernel<L><<<1, kInvThreads, smem, stream>>>(strip, si, st, pos, l, xinv, js);
  return cudaGetLastError();
}

cudaError_t launch_cross_inverse(const float* strip, long long si, long long st, const int* pos,
                                 int l, float2* xinv, JobStatus* js, cudaStream_t stream) {
  switch (l) {
    case 12: return launch_inverse_l<12>(strip, si, st, pos, l, xinv, js, stream);
    case 24: return launch_inverse_l<24>(strip, si, st, pos, l, xinv, js, stream);
    case 48: return launch_inverse_l<48>(strip, si, st, pos, l, xinv, js, stream);
    case 96: return launch_inverse_l<96>(strip, si, st, pos, l, xinv, js, stream);
    default: return launch_inverse_l<0>(strip, si, st, pos, l, xinv, js, stream);
  }
}

template <int L>
static cudaError_t launch_nucleus_l(const float* C, const int* I, int l, int k, double rank_tol,
                                    double* U, double* sigma, JobStatus* js, cudaStream_t st,
                                    const NucExtra& xa) {
  const size_t smem = 2 * (size_t)l * l * sizeof(dd) + kMaxL * (sizeof(double) + sizeof(dd)) +
                      sizeof(SvdScratch) + (kMaxL + 2) * sizeof(int);
  const cudaError_t e = smem_optin(reinterpret_cast<const void*>(nucleus_kernel<L>), 227 * 1024);
  if (e != cudaSuccess) return e;
  nucleus_kernel<L><<<1, kNucThreads, smem, st>>>(C, I, l, k, rank_tol, U, sigma, js, xa);
  return cudaGetLastError();
}

cudaError_t launch_nucleus(const float* C, const int* I, int l, int k, double rank_tol,
                           double* U, double* sigma, JobStatus* js, cudaStream_t st, const NucExtra& xa) {
  switch (l) {
    case 12: return launch_nucleus_l<12>(C, I, l, k, rank_tol, U, sigma, js, st, xa);
    case 24: return launch_nucleus_l<24>(C, I, l, k, rank_tol, U, sigma, js, st, xa);
    case 48: return launch_nucleus_l<48>(C, I, l, k, rank_tol, U, sigma, js, st, xa);
    case 96: return launch_nucleus_l<96>(C, I, l, k, rank_tol, U, sigma, js, st, xa);
    default: return launch_nucleus_l<0>(C, I, l, k, rank_tol, U, sigma, js, st, xa);
  }
}

}  // namespace lra
