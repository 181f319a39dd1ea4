// Maxvol half-step of the C-A iteration (Section 6.5; the l x l generator of
// each strip has locally maximal volume, Section 12.2 and the volume footnote
// of Section 6.5).
//
// Design (one cooperative launch per half-step, the strip's B resident in
// shared memory across the whole grid):
//   * The N x l strip S is split into contiguous row chunks, one chunk per
//     CTA, held as FP64 in shared memory (W).
//   * Every decision is the same primitive: pick (i*, j*), then apply the
//     rank-one update  W <- W - W[:, j*] (W[i*, :] - e_j*^T) / W[i*, j*].
//       - First half-step: Gauss-Jordan elimination with partial pivoting;
//         step t forces j* = t and takes i* = argmax over the not yet pivoted
//         rows of |W[:, t]| (the GEPP pivot).  After l steps W = S X^{-1}
//         with X = S[I, :].
//       - Later half-steps start from W = S X^{-1}, where X^{-1} is computed
//         afresh from the new cross by cross_inverse_kernel (an inverse
//         carried from strip to strip by rank-one updates loses a factor
//         cond(X) of accuracy on the ill-conditioned crosses of smooth
//         kernels).
//       - Maxvol swaps take (i*, j*) = argmax |B| and stop once it is
//         <= 1 + delta.
//   * Per decision: each CTA reduces its best (|value|, flat index) with warp
//     shuffles, publishes it together with that row of W, one grid barrier,
//     then every CTA reduces the <= 152 candidates itself and applies the
//     update to its chunk while scanning for the next decision (fused pass).
//   * Ties in |value| go to the smaller flat index i*l + j (smaller row, then
//     smaller column), the same rule as the FP64 oracle.
#include <cfloat>

#include "lra_kernels.h"
#include "lra_internal.cuh"

namespace lra {

constexpr int kMaxvolThreads = 512;
constexpr int kNone = 0x7fffffff;

// Candidates are compared on k = the IEEE-754 bit pattern of |value| as an
// unsigned 64-bit integer, which orders non-negative doubles exactly like
// their values.  Integer compares keep the argmax off the FP64 pipe (a
// double compare issues at the FP64 rate, 1/64 of FP32 on this part).
struct Best {
  unsigned long long k;
  int idx;
  int nf;
};

constexpr unsigned long long kAbsMask = 0x7fffffffffffffffull;
constexpr unsigned long long kInfBits = 0x7ff0000000000000ull;

__device__ __forceinline__ void consider(Best& b, double x, int idx) {
  const unsigned long long k = abs_bits(x);
  if (k >= kInfBits) {
    b.nf = 1;
  } else if (k > b.k || (k == b.k && idx < b.idx)) {
    b.k = k;
    b.idx = idx;
  }
}

__device__ __forceinline__ void merge(Best& b, unsigned long long k, int idx, int nf) {
  b.nf |= nf;
  if (k > b.k || (k == b.k && idx < b.idx)) {
    b.k = k;
    b.idx = idx;
  }
}

__device__ __forceinline__ Best warp_reduce(Best b) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    const unsigned long long k = __shfl_down_sync(0xffffffffu, b.k, off);
    const int i = __shfl_down_sync(0xffffffffu, b.idx, off);
    const int f = __shfl_down_sync(0xffffffffu, b.nf, off);
    merge(b, k, i, f);
  }
  return b;
}

// Block-wide reduction; the result is broadcast through *out.
__device__ __forceinline__ void block_reduce(Best b, Best* red, Best* out) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  b = warp_reduce(b);
  if (lane == 0) red[warp] = b;
  __syncthreads();
  if (warp == 0) {
    const int nw = blockDim.x >> 5;
    Best c = (lane < nw) ? red[lane] : Best{0ull, kNone, 0};
    c = warp_reduce(c);
    if (lane == 0) *out = c;
  }
  __syncthreads();
}

struct Ctl {
  Best cta_best;
  Best win;
  unsigned int gen;
  int timed_out;
};

// Warm start of the rows of this CTA: W[r, :] = S[g, :] X^{-1}.  A group of
// GS lanes owns a row; lane gl computes columns gl + GS c, c < NC, so every
// issued DFMA is useful work (NC = ceil(l / GS) exactly).
template <int GS, int NC, typename XPtr>
__device__ __forceinline__ void warm_rows(const MaxvolArgs& a, double* B, int nrows, long long row0,
                                          XPtr X) {
  const int l = a.l;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  constexpr int kGpw = 32 / GS;
  const int gl = lane % GS;
  const int ngroups = nwarps * kGpw;
  for (int base = warp * kGpw; base < nrows; base += ngroups) {
    const int r = base + lane / GS;
    const bool active = r < nrows;
    const long long g = row0 + r;
    double* brow = B + (size_t)r * l;
    if (active)
#pragma unroll
      for (int c = 0; c < NC; ++c) {
        const int t = gl + GS * c;
        if (t < l) brow[t] = (double)a.strip[g * a.si + (long long)t * a.st];
      }
    __syncwarp();
    double acc[NC];
#pragma unroll
    for (int c = 0; c < NC; ++c) acc[c] = 0.0;
    if (active) {
      for (int p = 0; p < l; ++p) {
        const double sp = brow[p];
#pragma unroll
        for (int c = 0; c < NC; ++c) {
          const int q = gl + GS * c;
          if (q < l) acc[c] = fma(sp, X[(size_t)p * l + q], acc[c]);
        }
      }
    }
    __syncwarp();
    if (active)
#pragma unroll
      for (int c = 0; c < NC; ++c) {
        const int q = gl + GS * c;
        if (q < l) brow[q] = acc[c];
      }
  }
}

struct GlobalX {  // read-only path for an X^{-1} that does not fit on chip
  const double* p;
  __device__ __forceinline__ double operator[](size_t i) const { return __ldg(p + i); }
};

template <int GS, int NC>
__global__ void __launch_bounds__(kMaxvolThreads, 1) maxvol_kernel(MaxvolArgs a) {
  if (a.js->status != LRA_OK || a.js->stop) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int l = a.l;
  const int tid = threadIdx.x, nthr = blockDim.x;
  const int G = gridDim.x, cta = blockIdx.x;
  const long long N = a.N;
  const long long row0 = (long long)cta * a.rows_per_cta;
  const int nrows = (int)max(0LL, min((long long)a.rows_per_cta, N - row0));
  const int rpc = a.rows_per_cta;

  double* B = reinterpret_cast<double*>(smem_raw);          // rpc * l
  double* colj = B + (size_t)rpc * l;                        // rpc
  double* rraw = colj + rpc;                                 // l
  double* rvec = rraw + kMaxL;                               // l
  double* xs = rvec + kMaxL;                                 // l*l when staged
  Best* red = reinterpret_cast<Best*>(xs + (a.stage_xinv ? (size_t)l * l : 0));  // 32
  Ctl* ctl = reinterpret_cast<Ctl*>(red + 32);
  int* pos_s = reinterpret_cast<int*>(ctl + 1);              // l
  unsigned char* used = reinterpret_cast<unsigned char*>(pos_s + kMaxL);  // rpc

  const int lane = tid & 31, warp = tid >> 5, nwarps = nthr >> 5;
  constexpr int kGpw = 32 / GS;
  const int gl = lane % GS;
  const int ngroups = nwarps * kGpw;

  for (int t = tid; t < l; t += nthr) pos_s[t] = a.gepp ? -1 : a.pos[t];
  for (int r = tid; r < nrows; r += nthr) used[r] = 0;
  if (tid == 0) {
    ctl->gen = ld_acquire_u32(&a.bar->gen);
    ctl->timed_out = 0;
  }
  __syncthreads();

  // ---- W = S (Gauss-Jordan start) or S X^{-1} (warm start)
  if (a.gepp) {
    for (int e = tid; e < nrows * l; e += nthr) {
      const int r = e / l, t = e - r * l;
      B[e] = (double)a.strip[(row0 + r) * a.si + (long long)t * a.st];
    }
  } else {
    if (a.stage_xinv) {
      for (int e = tid; e < l * l; e += nthr) xs[e] = a.xin[e];
      __syncthreads();
      warm_rows<GS, NC>(a, B, nrows, row0, static_cast<const double*>(xs));
    } else {
      warm_rows<GS, NC>(a, B, nrows, row0, GlobalX{a.xin});
    }
    __syncthreads();
    // rows currently selected are exactly the unit vectors of B = S X^{-1}
    for (int t = 0; t < l; ++t) {
      const long long g = pos_s[t];
      if (g >= row0 && g < row0 + nrows)
        for (int c = tid; c < l; c += nthr) B[(size_t)(g - row0) * l + c] = (c == t) ? 1.0 : 0.0;
    }
  }
  __syncthreads();

  // ---- initial scan
  Best mine{0ull, kNone, 0};
  bool gepp_phase = a.gepp != 0;
  for (int e = tid; e < nrows * l; e += nthr) {
    const int r = e / l, t = e - r * l;
    if (gepp_phase && t != 0) continue;
    consider(mine, B[e], (int)((row0 + r) * l + t));
  }

  int buf = 0, step = 0, swaps = 0, capped = 0;
  for (;;) {
    block_reduce(mine, red, &ctl->cta_best);
    Best win;
    if (G > 1) {
      const Best cb = ctl->cta_best;
      Cand* slot = a.cand + buf * kMaxGrid + cta;
      if (tid == 0) *slot = Cand{cb.k, cb.idx, cb.nf};
      if (cb.idx != kNone && tid < l) {
        const int r = (int)(cb.idx / l - row0);
        a.cand_rows[((size_t)buf * kMaxGrid + cta) * l + tid] = B[(size_t)r * l + tid];
      }
      if (!grid_sync(a.bar, &ctl->gen, &ctl->timed_out)) {
        if (tid == 0) set_status(a.js, LRA_ETIMEOUT);
        return;
      }
      Best c{0ull, kNone, 0};
      for (int k = tid; k < G; k += nthr) {
        const Cand* p = a.cand + buf * kMaxGrid + k;
        merge(c, __ldcg(&p->key), __ldcg(&p->idx), __ldcg(&p->flags));
      }
      block_reduce(c, red, &ctl->win);
      win = ctl->win;
    } else {
      win = ctl->cta_best;
    }

    // ---- decision (identical in every CTA)
    const double wv = __longlong_as_double((long long)win.k);
    int kind;
    if (win.nf) {
      if (cta == 0 && tid == 0) set_status(a.js, LRA_ENONFINITE);
      return;
    }
    if (gepp_phase) {
      if (!(wv > 0.0) || win.idx == kNone) {
        if (cta == 0 && tid == 0) set_status(a.js, LRA_ESINGULAR);
        return;
      }
      kind = LRA_TRACE_GEPP;
    } else if (wv <= 1.0 + a.delta) {
      kind = LRA_TRACE_STOP;
    } else if (swaps >= a.max_swaps) {
      kind = LRA_TRACE_CAP;
      capped = 1;
    } else {
      kind = LRA_TRACE_SWAP;
    }
    const long long istar = (win.idx == kNone) ? -1 : win.idx / l;
    const int jstar = (win.idx == kNone) ? 0 : (int)(win.idx - istar * l);
    if (cta == 0 && tid == 0) {
      const int n = a.js->trace_len;
      if (n < a.js->trace_cap) {
        a.trace_i[4 * n + 0] = a.half_step;
        a.trace_i[4 * n + 1] = kind;
        a.trace_i[4 * n + 2] = (int)istar;
        a.trace_i[4 * n + 3] = jstar;
        a.trace_v[n] = wv;
        a.js->trace_len = n + 1;
      }
    }
    if (kind == LRA_TRACE_STOP || kind == LRA_TRACE_CAP) break;

    // ---- pivot row and column of W
    const bool own_piv = istar >= row0 && istar < row0 + nrows;
    if (tid < l) {
      if (G > 1) {
        const int owner = (int)(istar / rpc);
        rraw[tid] = __ldcg(a.cand_rows + ((size_t)buf * kMaxGrid + owner) * l + tid);
      } else {
        rraw[tid] = B[(size_t)(istar - row0) * l + tid];
      }
    }
    for (int r = tid; r < nrows; r += nthr) colj[r] = B[(size_t)r * l + jstar];
    if (tid == 0) {
      if (gepp_phase && own_piv) used[istar - row0] = 1;
      pos_s[jstar] = (int)istar;
    }
    __syncthreads();
    if (tid < l) {
      const double piv = rraw[jstar];
      rvec[tid] = (rraw[tid] - (tid == jstar ? 1.0 : 0.0)) / piv;
    }
    __syncthreads();

    // ---- fused update + scan for the next decision
    const bool next_gepp = gepp_phase && (step + 1 < l);
    const int next_col = step + 1;
    mine = Best{0ull, kNone, 0};
    for (int base = warp * kGpw; base < nrows; base += ngroups) {
      const int r = base + lane / GS;
      if (r < nrows) {
        const long long g = row0 + r;
        double* brow = B + (size_t)r * l;
        if (g == istar) {
#pragma unroll
          for (int cc = 0; cc < NC; ++cc) {
            const int t = gl + GS * cc;
            if (t < l) {
              const double v = (t == jstar) ? 1.0 : 0.0;
              brow[t] = v;
              if (!next_gepp) consider(mine, v, (int)(g * l + t));
            }
          }
        } else {
          const double c = colj[r];
          const bool scan_row = !(next_gepp && used[r]);
#pragma unroll
          for (int cc = 0; cc < NC; ++cc) {
            const int t = gl + GS * cc;
            if (t < l) {
              const double v = fma(-c, rvec[t], brow[t]);
              brow[t] = v;
              if (scan_row && (!next_gepp || t == next_col)) consider(mine, v, (int)(g * l + t));
            }
          }
        }
      }
    }
    if (gepp_phase) {
      if (++step == l) gepp_phase = false;
    } else {
      ++swaps;
    }
    buf ^= 1;
    __syncthreads();
  }

  // ---- epilogue: positions and counters
  if (cta == 0 && tid < l) a.pos[tid] = pos_s[tid];
  if (cta == 0 && tid == 0) {
    a.js->swaps_total += swaps;
    if (capped) a.js->converged = 0;
    // algorithmic flops: warm-start product S X^{-1} plus one rank-one
    // update of the N x l matrix W per GEPP step or swap
    const double upd = (double)(step + swaps) * 2.0 * (double)N * l;
    const double init = a.gepp ? 0.0 : 2.0 * (double)N * l * l;
    a.js->maxvol_flops += upd + init;
  }
}

static size_t maxvol_smem(int rpc, int l, bool stage_xinv) {
  size_t b = (size_t)rpc * l * sizeof(double) + (size_t)rpc * sizeof(double) +
             2 * kMaxL * sizeof(double) + (stage_xinv ? (size_t)l * l * sizeof(double) : 0) +
             32 * sizeof(Best) + sizeof(Ctl) + kMaxL * sizeof(int) + (size_t)rpc;
  return (b + 15) & ~(size_t)15;
}

bool plan_maxvol(long long N, int l, int sms, size_t smem_limit, MaxvolPlan* plan) {
  // about 4096 entries of W per CTA before a second CTA pays for its barrier
  long long g = (N * l + 4095) / 4096;
  if (g < 1) g = 1;
  if (g > sms) g = sms;
  if (g > kMaxGrid) g = kMaxGrid;
  for (;;) {
    const long long rpc = (N + g - 1) / g;
    // stage X^{-1} in shared memory when it fits beside the chunk of W
    for (int stage = 1; stage >= 0; --stage) {
      const size_t sm = maxvol_smem((int)rpc, l, stage != 0);
      if (sm <= smem_limit) {
        plan->grid = (int)g;
        plan->rows_per_cta = (int)rpc;
        plan->threads = kMaxvolThreads;
        plan->smem = sm;
        plan->stage_xinv = stage;
        return true;
      }
    }
    if (g >= sms || g >= kMaxGrid) return false;
    ++g;
  }
}

template <int GS, int NC>
static cudaError_t launch_gs(MaxvolArgs& a, const MaxvolPlan& plan, cudaStream_t st) {
  const cudaError_t e = smem_optin(reinterpret_cast<const void*>(maxvol_kernel<GS, NC>), 227 * 1024);
  if (e != cudaSuccess) return e;
  void* args[] = {&a};
  return cudaLaunchCooperativeKernel(reinterpret_cast<void*>(maxvol_kernel<GS, NC>),
                                     dim3(plan.grid), dim3(plan.threads), args, plan.smem, st);
}

// Lanes per row group: 8 for l <= 24 (4 rows per warp), 16 for l <= 48,
// 32 above; each lane then owns NC = ceil(l / GS) <= 3 columns.
template <int GS>
static cudaError_t launch_nc(MaxvolArgs& a, const MaxvolPlan& plan, cudaStream_t st) {
  switch ((a.l + GS - 1) / GS) {
    case 1: return launch_gs<GS, 1>(a, plan, st);
    case 2: return launch_gs<GS, 2>(a, plan, st);
    default: return launch_gs<GS, 3>(a, plan, st);
  }
}

cudaError_t launch_maxvol(MaxvolArgs a, const MaxvolPlan& plan, cudaStream_t st) {
  a.rows_per_cta = plan.rows_per_cta;
  a.stage_xinv = plan.stage_xinv;
  if (a.l <= 24) return launch_nc<8>(a, plan, st);
  if (a.l <= 48) return launch_nc<16>(a, plan, st);
  return launch_nc<32>(a, plan, st);
}

}  // namespace lra
