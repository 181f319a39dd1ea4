// Internal device/host definitions shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/lra_cross.h"

namespace lra {

constexpr int kMaxL = 96;            // largest cross size handled on chip
constexpr int kMaxGrid = 160;        // candidate slots per exchange buffer (>= SM count)
constexpr unsigned long long kWaitNs = 2000000000ull;  // bounded device waits: 2 s

// ---------------------------------------------------------------------------
// Entry access to M (Section 1.1: the matrix is reachable entry by entry).
// ---------------------------------------------------------------------------
struct SourceDev {
  int kind;
  int dim;
  long long m, n;
  const void* a;
  long long lda;
  const float* x;
  const float* y;
  float h2;          // h*h rounded to FP32 (Gaussian kernel)
  // LRA_PRE_AH: base matrix in a / lda, multipliers
  int pre_d;
  int pre_mat;                // a holds H_{m,d} M H_{n,d} (lra_preprocess_materialize)
  long long pre_sm, pre_sn;   // m / 2^d, n / 2^d
  const int* pre_pr;
  const float* pre_sr;
  const int* pre_pc;
  const float* pre_sc;
};

// |x_i - y_j|^2 accumulated coordinate by coordinate with one rounding per
// operation (no FMA contraction), so the value is reproducible bit for bit.
__device__ __forceinline__ float dist2(const SourceDev& s, long long i, long long j) {
  const float* xi = s.x + i * s.dim;
  const float* yj = s.y + j * s.dim;
  float d = __fsub_rn(xi[0], yj[0]);
  float acc = __fmul_rn(d, d);
  for (int c = 1; c < s.dim; ++c) {
    d = __fsub_rn(xi[c], yj[c]);
    acc = __fadd_rn(acc, __fmul_rn(d, d));
  }
  return acc;
}

// Section 8.1 multiplies by H_{2^d} through d recursive steps
// H_{2s} = [[H_s, H_s], [H_s, -H_s]].  One entry b of that product, summed
// in the same order as the fast transform: the terms t = 0, 1, ... arrive
// in order and are merged like a binary counter, the merge at level k being
// left + right, or left - right when bit k of b is 1, each rounded in T.
// After term 2^d - 1 the returned value is the entry.  stk holds d + 1
// partial sums.
constexpr int kMaxPreD = 10;

__device__ __forceinline__ float bfly_add(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float bfly_sub(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ double bfly_add(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ double bfly_sub(double a, double b) { return __dsub_rn(a, b); }

template <typename T>
__device__ __forceinline__ T butterfly_push(T* stk, int t, T v, unsigned b) {
  int k = 0;
  while ((t >> k) & 1) {
    v = ((b >> k) & 1u) ? bfly_sub(stk[k], v) : bfly_add(stk[k], v);
    ++k;
  }
  stk[k] = v;
  return v;
}

template <int KIND>
__device__ __forceinline__ float entry(const SourceDev& s, long long i, long long j) {
  if constexpr (KIND == LRA_DENSE_F32) {
    return __ldg(static_cast<const float*>(s.a) + i * s.lda + j);
  } else if constexpr (KIND == LRA_DENSE_F64) {
    return __double2float_rn(__ldg(static_cast<const double*>(s.a) + i * s.lda + j));
  } else if constexpr (KIND == LRA_GEN_CAUCHY) {
    return __fdiv_rn(1.0f, __fsub_rn(__ldg(s.x + i), __ldg(s.y + j)));
  } else if constexpr (KIND == LRA_GEN_GAUSS) {
    return expf(-__fdiv_rn(dist2(s, i, j), s.h2));
  } else if constexpr (KIND == LRA_GEN_INVDIST) {
    return __fdiv_rn(1.0f, __fsqrt_rn(dist2(s, i, j)));
  } else {
    // M_bar[i][j] = sr[i] sc[j] (H_{m,d} M H_{n,d})[pr[i]][pc[j]]: with
    // (bi, oi) = divmod(pr[i], sm), (bj, oj) = divmod(pc[j], sn), the sum
    // over q (signs by bj) of the sums over p (signs by bi) of
    // M[p sm + oi][q sn + oj], each in the butterfly order, in FP32.
    long long xi = __ldg(s.pre_pr + i), yj = __ldg(s.pre_pc + j);
    // a caller's array that is not a permutation cannot move a read outside M
    if ((unsigned long long)xi >= (unsigned long long)s.m) xi = 0;
    if ((unsigned long long)yj >= (unsigned long long)s.n) yj = 0;
    const float sgn = __ldg(s.pre_sr + i) * __ldg(s.pre_sc + j);
    const float* a = static_cast<const float*>(s.a);
    if (s.pre_mat) return sgn * __ldg(a + xi * s.lda + yj);   // a holds H_{m,d} M H_{n,d}
    const long long bi = xi / s.pre_sm, oi = xi - bi * s.pre_sm;
    const long long bj = yj / s.pre_sn, oj = yj - bj * s.pre_sn;
    const int D = 1 << s.pre_d;
    float so[kMaxPreD + 1], si[kMaxPreD + 1];
    float acc = 0.0f;
    for (int qq = 0; qq < D; ++qq) {
      const float* col = a + oi * s.lda + qq * s.pre_sn + oj;
      float inner = 0.0f;
      for (int pp = 0; pp < D; ++pp)
        inner = butterfly_push(si, pp, __ldg(col + pp * s.pre_sm * s.lda), (unsigned)bi);
      acc = butterfly_push(so, qq, inner, (unsigned)bj);
    }
    return sgn * acc;
  }
}

// As LRA_DISPATCH_KIND, with the pre-processed source as well (the kernels
// of a plain solve that evaluate entries: gathers and the residual).
#define LRA_DISPATCH_KIND_ALL(kind, BODY)                               \
  switch (kind) {                                                      \
    case LRA_DENSE_F32: { constexpr int K = LRA_DENSE_F32; BODY; } break; \
    case LRA_DENSE_F64: { constexpr int K = LRA_DENSE_F64; BODY; } break; \
    case LRA_GEN_CAUCHY: { constexpr int K = LRA_GEN_CAUCHY; BODY; } break; \
    case LRA_GEN_GAUSS: { constexpr int K = LRA_GEN_GAUSS; BODY; } break; \
    case LRA_PRE_AH: { constexpr int K = LRA_PRE_AH; BODY; } break;     \
    default: { constexpr int K = LRA_GEN_INVDIST; BODY; } break;       \
  }

// Calls F<KIND> with the source kind as a compile-time constant.
#define LRA_DISPATCH_KIND(kind, BODY)                                   \
  switch (kind) {                                                      \
    case LRA_DENSE_F32: { constexpr int K = LRA_DENSE_F32; BODY; } break; \
    case LRA_DENSE_F64: { constexpr int K = LRA_DENSE_F64; BODY; } break; \
    case LRA_GEN_CAUCHY: { constexpr int K = LRA_GEN_CAUCHY; BODY; } break; \
    case LRA_GEN_GAUSS: { constexpr int K = LRA_GEN_GAUSS; BODY; } break; \
    default: { constexpr int K = LRA_GEN_INVDIST; BODY; } break;       \
  }

// ---------------------------------------------------------------------------
// Per-job device state.
// ---------------------------------------------------------------------------
struct JobStatus {
  int status;        // lra_status; kernels do nothing once it is not LRA_OK
  int stop;          // tolerance reached: remaining sweeps are skipped
  int sweeps_done;
  int k_eff;
  int swaps_total;
  int converged;
  int trace_len;
  int trace_cap;
  double est_rel, est_mu, est_var, est_sse, est_ssa;
  double sigma_max;
  double maxvol_flops;
  double full_sse, full_ssa, full_rel;
  // fixed-point exit of a fixed-budget solve: consecutive warm-started
  // half-steps without a swap, and the last STOP decision of each
  // orientation (vertical 0, horizontal 1): row, column, |value|
  int noswap_run;
  int stop_i[2], stop_j[2];
  double stop_v[2];
};

// Batched C-A (many blocks of one source, one launch).
constexpr int kMaxBatchSide = 2048;  // rows / columns of a block
constexpr int kDefaultClusterMask = 1 | 4 | 8;  // batch passes of 1, 4 and 8 CTAs

struct BatchArgs {
  SourceDev src;
  const long long* blocks;  // n_blocks x 4: row0, m, col0, n
  int n_blocks;
  const int* jcand;         // n_blocks x l_max candidate columns (local to the block)
  const int* srow;          // n_blocks x q sample rows (local)
  const int* scol;          // n_blocks x q sample columns (local)
  int q;
  int l_init, l_max, k_max, sweeps, max_swaps;
  double tol, delta;
  int* queue;               // four work counters (one per pass), zero at launch
  int pass_idx, pass_first; // set per launched pass
  int cutover;              // first pass: blocks with a larger side go to the next pass (0: none)
  const int* order;         // n_blocks queue order (nullptr: 0, 1, 2, ...)
  int trace_cap;            // decisions logged per block (0: none)
  int* trace;               // n_blocks x trace_cap x 4: half_step, kind, i, j
  double* trace_v;          // n_blocks x trace_cap: |value| of each decision
  int* trace_len;           // n_blocks
  int* out_status;
  int* out_l;
  int* out_keff;
  int* out_swaps;
  int* out_I;               // n_blocks x l_max
  int* out_J;
  double* out_U;            // n_blocks x l_max x l_max (l x l used, row-major)
  float* out_sigma;         // n_blocks x l_max
  double* out_err;          // n_blocks
  JobStatus* js;            // maxvol_flops accumulates the elimination / update FLOPs
};

// Grid barrier and decision counter of a job's maxvol launches (zero for a
// new job).  count: arrivals at the grid barrier, left at a multiple of 256
// by every launch.  seq: decisions taken so far; decision s of the job is
// exchanged in word s % kWinRing of the job's ring of candidate words.
struct GridBarrier {
  unsigned int count;
  unsigned int seq;
};
constexpr int kWinRing = 4;

// x as an FP32 pair: hi = x rounded to FP32, lo = the rest rounded to FP32
// (about 48 significant bits of x).
__device__ __forceinline__ float2 split_double(double x) {
  const float h = (float)x;
  return make_float2(h, (float)(x - (double)h));
}

__device__ __forceinline__ unsigned long long globaltimer_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ unsigned int ld_acquire_u32(const unsigned int* p) {
  unsigned int v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ void set_status(JobStatus* js, int code) {
  atomicCAS(&js->status, (int)LRA_OK, code);
}

}  // namespace lra
