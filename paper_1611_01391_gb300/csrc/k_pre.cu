// Pre-processing with abridged Hadamard multipliers (Section 8.1, family
// (i)) and recovery of the LRA of M from an LRA of M_bar = F M H (Section
// 6.6).  Every sum over the 2^d terms of H_{2^d} is taken in the order of
// the recursive steps H_{2s} = [[H_s, H_s], [H_s, -H_s]], lowest bit first
// (the fast transform's order).  The entries of M_bar are FP32 sums (every
// step rounded to FP32, the arithmetic of the stored matrix), so that the
// materialised M_bar and the entry-by-entry evaluation agree bit for bit;
// the recovered factors are FP64 sums rounded once to FP32.
#include <cuda_runtime.h>

#include <algorithm>

#include "lra_internal.cuh"
#include "lra_kernels.h"

namespace lra {
namespace {

// In-place H_{2^LD} x, butterflies with the lowest bit first: the pair
// (x[i], x[i + h]) (bit log2 h of i clear) becomes (x[i] + x[i + h],
// x[i] - x[i + h]) -- the merges of butterfly_push, all outputs at once.
template <int LD>
__device__ __forceinline__ void fwht(float (&x)[1 << LD]) {
#pragma unroll
  for (int h = 1; h < (1 << LD); h <<= 1) {
#pragma unroll
    for (int i = 0; i < (1 << LD); ++i) {
      if (i & h) continue;
      const float u = x[i], v = x[i + h];
      x[i] = __fadd_rn(u, v);
      x[i + h] = __fsub_rn(u, v);
    }
  }
}

template <int V> struct VecOf;
template <> struct VecOf<1> { using T = float; };
template <> struct VecOf<2> { using T = float2; };
template <> struct VecOf<4> { using T = float4; };

template <int V>
__device__ __forceinline__ void vload(const float* p, float* out) {
  const typename VecOf<V>::T v = __ldg(reinterpret_cast<const typename VecOf<V>::T*>(p));
  *reinterpret_cast<typename VecOf<V>::T*>(out) = v;
}

template <int V>
__device__ __forceinline__ void vstore(float* p, const float* in) {
  *reinterpret_cast<typename VecOf<V>::T*>(p) = *reinterpret_cast<const typename VecOf<V>::T*>(in);
}

constexpr int kMatThreads = 256;

// G = H_{m,d} M H_{n,d}.  With M viewed as M[p][o_r][q][o_c] (p, q < 2^d,
// o_r < sm, o_c < sn), G[p'][o_r][q'][o_c] is the 2-D transform over (p, q).
// One work item: one o_r and W = (256 / 2^d) V consecutive o_c, i.e. the
// 2^d x 2^d x W entries M[p sm + o_r][q sn + o_c]; each is read once and
// written once.  Phase 1, thread (q, c): V adjacent columns of the 2^d
// entries along p in registers, F applied (the transform over p), into
// shared memory; phase 2, thread (p', c): the 2^d values along q, H applied,
// stored.  Threads of a warp share q (phase 1) or p' (phase 2) and run along
// o_c, so every global access is a run of W consecutive floats.
template <int LD, int V>
__global__ void __launch_bounds__(kMatThreads)
    pre_materialize_kernel(const float* __restrict__ M, long long lda, float* __restrict__ G, long long ldg,
                           long long sm, long long sn, long long n_items) {
  constexpr int D = 1 << LD;
  constexpr int CT = kMatThreads / D;   // column threads per item
  constexpr int W = CT * V;             // columns per item
  extern __shared__ __align__(16) float T[];   // T[p][q][W]
  const int c = threadIdx.x % CT, g = threadIdx.x / CT;
  const long long chunks = (sn + W - 1) / W;
  for (long long it = blockIdx.x; it < n_items; it += gridDim.x) {
    const long long orow = it / chunks;
    const long long oc = (it - orow * chunks) * W + (long long)c * V;
    const bool ok = oc < sn;   // V divides sn: a vector is wholly in or out
    float x[V][D];
    if (ok) {
      const float* src = M + orow * lda + (long long)g * sn + oc;
#pragma unroll
      for (int p = 0; p < D; ++p) {
        float t[V];
        vload<V>(src + (long long)p * sm * lda, t);
#pragma unroll
        for (int v = 0; v < V; ++v) x[v][p] = t[v];
      }
    } else {
#pragma unroll
      for (int v = 0; v < V; ++v)
#pragma unroll
        for (int p = 0; p < D; ++p) x[v][p] = 0.0f;
    }
#pragma unroll
    for (int v = 0; v < V; ++v) fwht<LD>(x[v]);
#pragma unroll
    for (int p = 0; p < D; ++p) {
      float t[V];
#pragma unroll
      for (int v = 0; v < V; ++v) t[v] = x[v][p];
      vstore<V>(T + (p * D + g) * W + c * V, t);
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < D; ++q) {
      float t[V];
      *reinterpret_cast<typename VecOf<V>::T*>(t) =
          *reinterpret_cast<const typename VecOf<V>::T*>(T + (g * D + q) * W + c * V);
#pragma unroll
      for (int v = 0; v < V; ++v) x[v][q] = t[v];
    }
#pragma unroll
    for (int v = 0; v < V; ++v) fwht<LD>(x[v]);
    if (ok) {
      float* dst = G + ((long long)g * sm + orow) * ldg + oc;
#pragma unroll
      for (int q = 0; q < D; ++q) {
        float t[V];
#pragma unroll
        for (int v = 0; v < V; ++v) t[v] = x[v][q];
        vstore<V>(dst + (long long)q * sn, t);
      }
    }
    __syncthreads();
  }
}

template <int LD, int V>
cudaError_t launch_materialize_v(const float* M, long long lda, float* G, long long ldg, long long m, long long n,
                                 cudaStream_t st) {
  constexpr int D = 1 << LD;
  constexpr int W = (kMatThreads / D) * V;
  const long long sm = m >> LD, sn = n >> LD;
  const size_t smem = sizeof(float) * D * D * W;
  const void* fn = reinterpret_cast<const void*>(pre_materialize_kernel<LD, V>);
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e) return e;
  int dev = 0, sms = 0, per_sm = 0;
  if ((e = cudaGetDevice(&dev)) || (e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev))) return e;
  if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kMatThreads, smem))) return e;
  const long long items = sm * ((sn + W - 1) / W);
  const long long grid = std::min<long long>(items, (long long)sms * std::max(per_sm, 1));
  void* args[] = {(void*)&M, (void*)&lda, (void*)&G, (void*)&ldg, (void*)&sm, (void*)&sn, (void*)&items};
  return cudaLaunchKernel(fn, dim3((unsigned)grid), dim3(kMatThreads), args, smem, st);
}

// V = min(4, 64 / 2^d) adjacent columns per thread where the pointers, the
// strides and the column offset sn allow vectors of V floats; else V = 1.
template <int LD>
cudaError_t launch_materialize_d(const float* M, long long lda, float* G, long long ldg, long long m, long long n,
                                 cudaStream_t st) {
  constexpr int VM = (64 >> LD) < 4 ? (64 >> LD) : 4;
  const long long sn = n >> LD;
  const bool vec = ((uintptr_t)M % (4 * VM)) == 0 && ((uintptr_t)G % (4 * VM)) == 0 && lda % VM == 0 &&
                   ldg % VM == 0 && sn % VM == 0;
  return vec ? launch_materialize_v<LD, VM>(M, lda, G, ldg, m, n, st)
             : launch_materialize_v<LD, 1>(M, lda, G, ldg, m, n, st);
}

__global__ void invert_perm_kernel(const int* __restrict__ perm, long long n, int* __restrict__ inv) {
  for (long long x = blockIdx.x * (long long)blockDim.x + threadIdx.x; x < n; x += (long long)gridDim.x * blockDim.x) {
    const int p = __ldg(perm + x);
    if ((unsigned long long)p < (unsigned long long)n) inv[p] = (int)x;
  }
}

// A = F^T Cbar / 2^d = H_{m,d} Y / 2^d with Y[pr[i]] = sr[i] Cbar[i]:
// A[a][t] = 2^-d sum_p (+-1) Y[p sm + oa][t], signs by ba, (ba, oa) = divmod(a, sm).
__global__ void pre_recover_left_kernel(SourceDev s, const float* __restrict__ Cbar, int l,
                                        const int* __restrict__ inv_r, float* __restrict__ A) {
  const long long total = s.m * l;
  const int D = 1 << s.pre_d;
  double stk[kMaxPreD + 1];
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const long long a = e / l;
    const int t = (int)(e - a * l);
    const long long ba = a / s.pre_sm, oa = a - ba * s.pre_sm;
    double acc = 0.0;
    for (int pp = 0; pp < D; ++pp) {
      long long i = inv_r[pp * s.pre_sm + oa];
      if ((unsigned long long)i >= (unsigned long long)s.m) i = 0;
      acc = butterfly_push(stk, pp, (double)__ldg(s.pre_sr + i) * (double)Cbar[i * l + t], (unsigned)ba);
    }
    A[e] = __double2float_rn(ldexp(acc, -s.pre_d));
  }
}

// B = Rbar H^T / 2^d = Z H_{n,d} / 2^d with Z[:, pc[j]] = sc[j] Rbar[:, j]:
// B[t][b] = 2^-d sum_q (+-1) Z[t][q sn + ob], signs by bb, (bb, ob) = divmod(b, sn).
__global__ void pre_recover_right_kernel(SourceDev s, const float* __restrict__ Rbar, int l,
                                         const int* __restrict__ inv_c, float* __restrict__ B) {
  const long long total = s.n * l;
  const int D = 1 << s.pre_d;
  double stk[kMaxPreD + 1];
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const long long t = e / s.n, b = e - t * s.n;
    const long long bb = b / s.pre_sn, ob = b - bb * s.pre_sn;
    double acc = 0.0;
    for (int qq = 0; qq < D; ++qq) {
      long long j = inv_c[qq * s.pre_sn + ob];
      if ((unsigned long long)j >= (unsigned long long)s.n) j = 0;
      acc = butterfly_push(stk, qq, (double)__ldg(s.pre_sc + j) * (double)Rbar[t * s.n + j], (unsigned)bb);
    }
    B[e] = __double2float_rn(ldexp(acc, -s.pre_d));
  }
}

}  // namespace

cudaError_t launch_pre_materialize(const float* M, long long lda, float* G, long long ldg, long long m, long long n,
                                   int d, cudaStream_t st) {
  switch (d) {
    case 0: return launch_materialize_d<0>(M, lda, G, ldg, m, n, st);
    case 1: return launch_materialize_d<1>(M, lda, G, ldg, m, n, st);
    case 2: return launch_materialize_d<2>(M, lda, G, ldg, m, n, st);
    case 3: return launch_materialize_d<3>(M, lda, G, ldg, m, n, st);
    case 4: return launch_materialize_d<4>(M, lda, G, ldg, m, n, st);
    case 5: return launch_materialize_d<5>(M, lda, G, ldg, m, n, st);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_pre_recover(const SourceDev& s, const float* Cbar, const float* Rbar, int l, float* A, float* B,
                               int* inv, cudaStream_t st) {
  int* inv_r = inv;
  int* inv_c = inv + s.m;
  // an array that is not a permutation leaves some entries unset: start them at 0
  cudaError_t e = cudaMemsetAsync(inv, 0, sizeof(int) * (size_t)(s.m + s.n), st);
  if (e) return e;
  invert_perm_kernel<<<256, 256, 0, st>>>(s.pre_pr, s.m, inv_r);
  invert_perm_kernel<<<256, 256, 0, st>>>(s.pre_pc, s.n, inv_c);
  pre_recover_left_kernel<<<608, 256, 0, st>>>(s, Cbar, l, inv_r, A);
  pre_recover_right_kernel<<<608, 256, 0, st>>>(s, Rbar, l, inv_c, B);
  return cudaGetLastError();
}

}  // namespace lra
