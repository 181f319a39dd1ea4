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
#include <cooperative_groups.h>

#include <cfloat>

#include "lra_kernels.h"
#include "lra_internal.cuh"
#include "inverse_dd.cuh"
#include "svd_dd.cuh"

namespace lra {

namespace cg = cooperative_groups;

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

// The nucleus on a cluster of NC CTAs, for a job that has the GPU to
// itself.  Every CTA loads and scales X and runs the QR with column
// pivoting (the same values in every CTA); the Jacobi sweeps run on the
// cluster (jacobi_dd_cluster), after which every CTA holds the whole W.
// Each CTA then forms the left vectors and the entries of U of the rows
// q = rank, rank + NC, ... of X.  Every value takes the operations of
// nucleus_kernel in the same order, so U, sigma and the vectors are bitwise
// the one-CTA kernel's.  NC = 16 (three column pairs per CTA at l = 96, one
// warp per SM sub-partition) where the GPU can hold such a cluster, else 8.
template <int L, int NC>
__global__ void __launch_bounds__(kNucThreads, 1)
nucleus_cluster_kernel(const float* __restrict__ C, const int* __restrict__ I, int k, double rank_tol,
                       double* __restrict__ U, double* __restrict__ sigma_out, JobStatus* js, NucExtra xa) {
  constexpr int l = L;
  static_assert(sizeof(SvdScratch) % 8 == 0 && (kMaxL + 6) % 2 == 0, "column buffers 8-byte aligned");
  cg::cluster_group cl = cg::this_cluster();
  const int rank = (int)cl.block_rank();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  dd* W = reinterpret_cast<dd*>(smem_raw);           // column b at W + b*l
  dd* Z = W + (size_t)l * l;                          // column b at Z + b*l
  double* sig = reinterpret_cast<double*>(Z + (size_t)l * l);  // l
  dd* inv2 = reinterpret_cast<dd*>(sig + kMaxL);      // l
  SvdScratch* sc = reinterpret_cast<SvdScratch*>(inv2 + kMaxL);
  int* order = reinterpret_cast<int*>(sc + 1);        // l: order[rank] = column
  int* keff_s = order + kMaxL;
  int* scale_e = keff_s + 1;
  int* go_s = scale_e + 1;
  int* flags = go_s + 2;                              // 2
  dd* cb = reinterpret_cast<dd*>(flags + 2);          // 2 * 2S * l (8-byte aligned: see the launch)

  const int tid = threadIdx.x, nthr = kNucThreads;
  // CTA 0 decides whether the job still runs (a cancellation can change the
  // status meanwhile); every CTA follows its answer
  if (tid == 0) {
    *scale_e = 0;
    if (rank == 0) go_s[0] = js->status == LRA_OK ? 1 : 0;
  }
  cl.sync();
  if (tid == 0) go_s[1] = *cl.map_shared_rank(&go_s[0], 0);
  __syncthreads();
  if (!go_s[1]) {
    cl.sync();
    return;
  }
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
    atomicMax(scale_e, ex + 1024);
  }
  __syncthreads();
  const int ex = *scale_e ? *scale_e - 1024 : 0;
  for (int e = tid; e < l * l; e += nthr) {
    const int a = e / l, b = e - a * l;
    const float c = C[(size_t)__ldg(I + a) * l + b];
    W[(size_t)b * l + a] = scaled ? dd_mul(dd_make(c), dd_from_double(ldexp(xa.rs[a] * xa.cs[b], -ex)))
                                  : dd_make(ldexpf(c, -ex));
  }
  __syncthreads();
  svd_dd_precondition<kNucThreads, L>(W, Z, l, sc);
  jacobi_dd_cluster<kNucThreads, L, NC>(cl, W, cb, flags);
  jacobi_sigma<kNucThreads>(W, l, sig, order);
  if (tid == 0) {
    const double s1 = sig[order[0]];
    int ke = 0;
    if (s1 > 0.0)
      while (ke < k && ke < l && sig[order[ke]] > rank_tol * s1) ++ke;
    *keff_s = ke;
    if (rank == 0) {
      js->k_eff = ke;
      js->sigma_max = ldexp(s1, ex);
    }
  }
  for (int r = tid; r < l; r += nthr) {
    const double sb = sig[order[r]];
    inv2[r] = dd_from_double(sb > 0.0 ? 1.0 / (sb * sb) : 0.0);
    if (rank == 0) sigma_out[r] = ldexp(sb, ex);
  }
  __syncthreads();
  const int ke = *keff_s;
  left_vectors<kNucThreads, L>(W, Z, l, ke, order, inv2, sc->perm, rank, NC);
  constexpr int nq = (l + NC - 1) / NC;
  if (xa.Vk) {
    // entry c of right vector r and entry c of left vector r, for the rows
    // c of X this CTA formed
    for (int e = tid; e < nq * l; e += nthr) {
      const int c = rank + (e / l) * NC, r = e - (e / l) * l;
      if (c >= l) continue;
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
      const int p = e / l, q = e - p * l;
      U[e] = xa.cs[p] * ldexp(v, -ex) * xa.rs[q];
    }, rank, NC);
  } else {
    nucleus_from_svd<kNucThreads, L>(W, Z, sc->perm, l, ke, order, inv2,
                                  [&](int e, double v) { U[e] = ldexp(v, -ex); }, rank, NC);
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

// The same elimination spread over a cluster of kInvCluster CTAs, for a job
// that has the GPU to itself.  CTA c owns the column block [c w, (c + 1) w),
// w = L / kInvCluster, of the matrix in its shared memory (two buffers: the
// matrix before and after the step).  Step t needs three things from the
// owner of column t: the pivot row p, the reciprocal rp of the pivot and
// column t with rows t and p interchanged.  With a one-step look-ahead as in
// invert_cross_la, the owner of column t + 1 forms that column of step t's
// result first, picks the next pivot and writes (p, rp, column) into a slot
// of every CTA of the cluster (distributed shared memory, two slots by
// parity); one cluster barrier per step publishes it.  Every CTA then scales
// its part of the pivot row and updates its own columns.  Every entry takes
// the operations of invert_cross_la in the same order, so the result is
// bitwise the one-CTA kernel's.
constexpr int kInvCluster = 8;
constexpr int kInvClThreads = 256;

struct InvStep {
  dd colt[kMaxL];   // column t of the matrix step t works on, rows t and p interchanged
  dd rp;            // 1 / pivot
  int p;            // pivot row (-1: no nonzero candidate)
};

// Warp 0 of the owner of column tn: v = that column of the matrix step tn
// works on (entry u of the lane: row lane + 32 u); choose the pivot among
// rows >= tn and publish step tn in the slot of its parity of every CTA.
template <int L, int kLn>
__device__ __forceinline__ void inv_publish_step(cg::cluster_group& cl, InvStep* slot, int tn, const dd (&v)[kLn]) {
  const int lane = threadIdx.x & 31;
  unsigned long long key = 0ull;
#pragma unroll
  for (int u = 0; u < kLn; ++u) {
    const int r = lane + 32 * u;
    if (r < L && r >= tn) {
      const unsigned long long k = pivot_word(v[u], r);
      key = k > key ? k : key;
    }
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    const unsigned long long o = __shfl_xor_sync(0xffffffffu, key, off);
    key = o > key ? o : key;
  }
  const int p = (key >> 32) != 0ull ? (int)(0xffffffffu - (unsigned int)key) : -1;
  dd vt = dd_make(0.0f), rp = dd_make(0.0f);
  if (p >= 0) {
    // the pivot and the entry of row tn, from the lanes that hold them
    dd vp = dd_make(0.0f);
#pragma unroll
    for (int u = 0; u < kLn; ++u) {
      const float ph = __shfl_sync(0xffffffffu, v[u].hi, p & 31), pl = __shfl_sync(0xffffffffu, v[u].lo, p & 31);
      const float th = __shfl_sync(0xffffffffu, v[u].hi, tn & 31), tl = __shfl_sync(0xffffffffu, v[u].lo, tn & 31);
      if (u == p / 32) vp = dd{ph, pl};
      if (u == tn / 32) vt = dd{th, tl};
    }
    rp = dd_div(dd_make(1.0f), vp);
  }
#pragma unroll
  for (int d = 0; d < kInvCluster; ++d) {
    InvStep* s = cl.map_shared_rank(&slot[tn & 1], d);
    if (p >= 0) {
#pragma unroll
      for (int u = 0; u < kLn; ++u) {
        const int r = lane + 32 * u;
        if (r < L) s->colt[r] = (r == p) ? vt : v[u];
      }
    }
    if (lane == 0) {
      s->rp = rp;
      s->p = p;
    }
  }
}

template <int L>
__global__ void __cluster_dims__(kInvCluster, 1, 1) __launch_bounds__(kInvClThreads, 1)
cross_inverse_cluster_kernel(const float* __restrict__ strip, long long si, long long st,
                             const int* __restrict__ pos, float2* __restrict__ xinv, JobStatus* js) {
  static_assert(L % kInvCluster == 0 && L <= kMaxL, "column blocks");
  constexpr int Wc = L / kInvCluster;      // columns per CTA
  constexpr int kLn = (L + 31) / 32;       // a column's entries per lane
  cg::cluster_group cl = cg::this_cluster();
  const int rank = (int)cl.block_rank();
  const int c0 = rank * Wc;
  __shared__ dd blk[2][L * Wc];            // rows r, local columns j: [r * Wc + j]
  __shared__ InvStep slot[2];
  __shared__ dd rowt[Wc];
  __shared__ int pos_s[L], swaps[L], at[L], iat[L];
  __shared__ int go_s, go_b;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  // CTA 0 decides whether the job still runs; every CTA reads its answer
  // (the status can change under a concurrent cancellation)
  if (rank == 0 && tid == 0) go_s = (js->status == LRA_OK && !js->stop) ? 1 : 0;
  for (int t = tid; t < L; t += kInvClThreads) pos_s[t] = pos[t];
  cl.sync();
  if (tid == 0) go_b = *cl.map_shared_rank(&go_s, 0);
  __syncthreads();
  if (!go_b) {
    cl.sync();   // CTA 0's answer read everywhere before any CTA leaves
    return;
  }
  // every CTA reads the whole cross (a uniform non-finite verdict) and keeps its columns
  int bad = 0;
  for (int e = tid; e < L * L; e += kInvClThreads) {
    const int r = e / L, c = e - r * L;
    const float x = strip[(long long)pos_s[r] * si + (long long)c * st];
    if (!(fabsf(x) <= FLT_MAX)) bad = 1;
    if (c >= c0 && c < c0 + Wc) blk[0][r * Wc + (c - c0)] = dd_make(x);
  }
  if (__syncthreads_or(bad)) {
    if (rank == 0 && tid == 0) set_status(js, LRA_ENONFINITE);
    cl.sync();
    return;
  }
  // warp 0 of the owner of column tn: v = that column of the matrix step tn
  // works on (rows lane + 32 u); choose the pivot among rows >= tn and
  // publish step tn in every CTA's slot of its parity
  if (rank == 0 && warp == 0) {
    dd v[kLn];
#pragma unroll
    for (int u = 0; u < kLn; ++u) {
      const int r = lane + 32 * u;
      v[u] = r < L ? blk[0][r * Wc] : dd_make(0.0f);
    }
    inv_publish_step<L, kLn>(cl, slot, 0, v);
  }
  cl.sync();
  int cb = 0;
  for (int t = 0; t < L; ++t) {
    const InvStep& S = slot[t & 1];
    const int p = S.p;
    if (p < 0) {   // the same value in every CTA; nothing remote is in flight
      if (rank == 0 && tid == 0) set_status(js, LRA_ESINGULAR);
      return;
    }
    const dd* cur = blk[cb];
    dd* nxt = blk[cb ^ 1];
    if (tid < Wc) rowt[tid] = (c0 + tid == t) ? S.rp : dd_mul(cur[p * Wc + tid], S.rp);
    if (tid == 0) swaps[t] = p;
    __syncthreads();
    // entry (r, c0 + j) of the matrix after step t
    auto entry = [&](int r, int j) -> dd {
      if (r == t) return rowt[j];
      const dd av = (c0 + j == t) ? dd_make(0.0f) : cur[(r == p ? t : r) * Wc + j];
      return dd_fnma(S.colt[r], rowt[j], av);
    };
    const int tn = t + 1;
    const bool own_next = tn < L && tn >= c0 && tn < c0 + Wc;
    if (warp == 0) {
      if (own_next) {
        dd v[kLn];
#pragma unroll
        for (int u = 0; u < kLn; ++u) {
          const int r = lane + 32 * u;
          v[u] = dd_make(0.0f);
          if (r < L) {
            v[u] = entry(r, tn - c0);
            nxt[r * Wc + (tn - c0)] = v[u];
          }
        }
        inv_publish_step<L, kLn>(cl, slot, tn, v);
      }
    } else {
      for (int e = tid - 32; e < L * Wc; e += kInvClThreads - 32) {
        const int r = e / Wc, j = e - r * Wc;
        if (!(own_next && j == tn - c0)) nxt[e] = entry(r, j);
      }
    }
    cl.sync();   // step t complete everywhere, step t + 1 published
    cb ^= 1;
  }
  // the interchanges undone as a column map: X^{-1}[:, q] = A[:, at[q]]
  if (tid == 0) {
    for (int q = 0; q < L; ++q) at[q] = q;
    for (int t = L - 1; t >= 0; --t) {
      const int p = swaps[t], x = at[t];
      at[t] = at[p];
      at[p] = x;
    }
    for (int q = 0; q < L; ++q) iat[at[q]] = q;
  }
  __syncthreads();
  const dd* res = blk[cb];
  for (int e = tid; e < L * Wc; e += kInvClThreads) {
    const int r = e / Wc, j = e - r * Wc;
    const dd v = res[e];
    xinv[(size_t)r * L + iat[c0 + j]] = make_float2(v.hi, v.lo);
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

template <int L>
static cudaError_t launch_inverse_cluster_l(const float* strip, long long si, long long st, const int* pos,
                                            float2* xinv, JobStatus* js, cudaStream_t stream) {
  cross_inverse_cluster_kernel<L><<<kInvCluster, kInvClThreads, 0, stream>>>(strip, si, st, pos, xinv, js);
  return cudaGetLastError();
}

cudaError_t launch_cross_inverse(const float* strip, long long si, long long st, const int* pos,
                                 int l, float2* xinv, JobStatus* js, cudaStream_t stream, bool cluster) {
  // (at l = 48 the inverse fits beside the strip inside the maxvol launch
  // except for strips of about 82 k to 92 k rows: the one-CTA kernel)
  if (cluster && l == 96) return launch_inverse_cluster_l<96>(strip, si, st, pos, xinv, js, stream);
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

template <int L, int NC>
static cudaError_t launch_nucleus_cluster_nc(const float* C, const int* I, int k, double rank_tol, double* U,
                                             double* sigma, JobStatus* js, cudaStream_t st, const NucExtra& xa,
                                             bool* unavailable) {
  constexpr int S = L / (2 * NC);
  size_t smem = 2 * (size_t)L * L * sizeof(dd) + kMaxL * (sizeof(double) + sizeof(dd)) + sizeof(SvdScratch) +
                (kMaxL + 6) * sizeof(int);
  smem = (smem + 7) & ~(size_t)7;   // the column buffers are read as 8-byte pairs
  smem += 2 * (size_t)(2 * S) * L * sizeof(dd);
  const void* f = reinterpret_cast<const void*>(nucleus_cluster_kernel<L, NC>);
  cudaError_t e = smem_optin(f, 227 * 1024);
  if (e != cudaSuccess) return e;
  if (NC > 8 && (e = cudaFuncSetAttribute(f, cudaFuncAttributeNonPortableClusterSizeAllowed, 1)) != cudaSuccess)
    return e;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(NC);
  cfg.blockDim = dim3(kNucThreads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = NC;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  int nclusters = 0;
  if ((e = cudaOccupancyMaxActiveClusters(&nclusters, f, &cfg)) != cudaSuccess || nclusters < 1) {
    cudaGetLastError();   // a size this GPU cannot hold: not an error of the job
    *unavailable = true;
    return cudaSuccess;
  }
  *unavailable = false;
  return cudaLaunchKernelEx(&cfg, nucleus_cluster_kernel<L, NC>, C, I, k, rank_tol, U, sigma, js, xa);
}

template <int L>
static cudaError_t launch_nucleus_cluster_l(const float* C, const int* I, int k, double rank_tol, double* U,
                                            double* sigma, JobStatus* js, cudaStream_t st, const NucExtra& xa) {
  bool unavailable = true;
  cudaError_t e = cudaSuccess;
  if constexpr (L % 32 == 0) {
    e = launch_nucleus_cluster_nc<L, 16>(C, I, k, rank_tol, U, sigma, js, st, xa, &unavailable);
    if (e != cudaSuccess || !unavailable) return e;
  }
  e = launch_nucleus_cluster_nc<L, 8>(C, I, k, rank_tol, U, sigma, js, st, xa, &unavailable);
  if (e != cudaSuccess || !unavailable) return e;
  return launch_nucleus_l<L>(C, I, L, k, rank_tol, U, sigma, js, st, xa);   // one CTA
}

cudaError_t launch_nucleus(const float* C, const int* I, int l, int k, double rank_tol,
                           double* U, double* sigma, JobStatus* js, cudaStream_t st, const NucExtra& xa,
                           bool cluster) {
  if (cluster && l == 96) return launch_nucleus_cluster_l<96>(C, I, k, rank_tol, U, sigma, js, st, xa);
  if (cluster && l == 48) return launch_nucleus_cluster_l<48>(C, I, k, rank_tol, U, sigma, js, st, xa);
  switch (l) {
    case 12: return launch_nucleus_l<12>(C, I, l, k, rank_tol, U, sigma, js, st, xa);
    case 24: return launch_nucleus_l<24>(C, I, l, k, rank_tol, U, sigma, js, st, xa);
    case 48: return launch_nucleus_l<48>(C, I, l, k, rank_tol, U, sigma, js, st, xa);
    case 96: return launch_nucleus_l<96>(C, I, l, k, rank_tol, U, sigma, js, st, xa);
    default: return launch_nucleus_l<0>(C, I, l, k, rank_tol, U, sigma, js, st, xa);
  }
}

}  // namespace lra
