// Maxvol half-step of the C-A iteration (Section 6.5; the l x l generator of
// each strip has locally maximal volume, Section 12.2 and the volume footnote
// of Section 6.5).
//
// Design (one cooperative launch per half-step, the strip's B resident in
// shared memory across the whole grid):
//   * The N x l strip S is split into contiguous row chunks, one chunk per
//     CTA, held in shared memory (W) as double-float pairs: about 48
//     significant bits from FP32 instructions, which this GPU issues at 64
//     times its FP64 rate.
//   * Every decision is the same primitive: pick (i*, j*), then apply the
//     rank-one update  W <- W - W[:, j*] (W[i*, :] - e_j*^T) / W[i*, j*].
//       - First half-step: Gauss-Jordan elimination with partial pivoting;
//         step t forces j* = t and takes i* = argmax over the not yet pivoted
//         rows of |W[:, t]| (the GEPP pivot).  After l steps W = S X^{-1}
//         with X = S[I, :].
//       - Later half-steps start from W = S X^{-1}, where X^{-1} is computed
//         afresh from the new cross (an inverse carried from strip to strip
//         by rank-one updates loses a factor cond(X) of accuracy on the
//         ill-conditioned crosses of smooth kernels): by every CTA of this
//         launch itself (kSelf builds, double-float Gauss-Jordan of
//         inverse_dd.cuh, when X^{-1} fits beside the chunk), or by the
//         separate cross inverse kernel, which hands it over as hi/lo FP32
//         pairs.  The product S X^{-1} is a compensated (Dot2) sum per entry.
//       - Maxvol swaps take (i*, j*) = argmax |B| and stop once it is
//         <= 1 + delta.
//   * Per decision: every warp reduces its best candidate word (|value| and
//     flat index in one 64-bit integer) with shuffles; one block barrier;
//     warp 0 takes the CTA's best, publishes that row of W, folds the word
//     into the decision's word in global memory with one atomic max, arrives
//     at the grid barrier, reads the maximum back (one load per CTA), fetches
//     the winner's row and forms the update vector
//     (W[i*, :] - e_j*^T) / W[i*, j*]; a second block barrier; every warp
//     then applies the update to its rows while scanning for the next
//     decision (fused pass).  Every CTA reads the same few words and one
//     row, so the exchange costs few requests on those hot L2 lines.
//   * Ties in |value| go to the smaller flat index i*l + j (smaller row, then
//     smaller column), the same rule as the FP64 oracle; candidates are
//     ranked by the FP32 high part of their pairs, so values within 2^-24 of
//     each other count as ties.
#include <cfloat>

#include "dd_arith.cuh"
#include "inverse_dd.cuh"
#include "lra_kernels.h"
#include "lra_internal.cuh"

namespace lra {

constexpr int kMaxvolThreads = 1024;

// Candidates are compared on one unsigned 64-bit word: the FP32 bit pattern
// of |hi| (non-negative FP32 patterns order like their values as unsigned
// integers) above 0xffffffff - the flat index i*l + j.  The largest word is
// the largest |value|, ties to the smaller flat index (smaller row, then
// smaller column), the rule of the FP64 oracle; values whose high parts are
// equal (within 2^-24 of each other) are treated as ties.  Infinite and NaN
// patterns sort above every finite one, so a non-finite entry always wins
// and is caught at the decision.  An integer max per scanned entry, no FP64
// instruction.
__device__ __forceinline__ unsigned long long cand_word(dd x, long long idx) {
  const unsigned int kh = __float_as_uint(x.hi) & 0x7fffffffu;
  return ((unsigned long long)kh << 32) | (0xffffffffu - (unsigned int)idx);
}

__device__ __forceinline__ unsigned long long umax64(unsigned long long a, unsigned long long b) {
  return a > b ? a : b;
}

__device__ __forceinline__ unsigned long long warp_max(unsigned long long v) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) v = umax64(v, __shfl_xor_sync(0xffffffffu, v, off));
  return v;
}

// The generator's entry from the coordinates of its two points (xp on the
// x side, yq on the y side): the operations of entry<KIND>, in order.
__device__ __forceinline__ float gen_eval(const SourceDev& s, const float* xp, const float* yq) {
  if (s.kind == LRA_GEN_CAUCHY) return __fdiv_rn(1.0f, __fsub_rn(xp[0], yq[0]));
  float d = __fsub_rn(xp[0], yq[0]);
  float acc = __fmul_rn(d, d);
  if (s.dim > 1) {
    d = __fsub_rn(xp[1], yq[1]);
    acc = __fadd_rn(acc, __fmul_rn(d, d));
  }
  if (s.dim > 2) {
    d = __fsub_rn(xp[2], yq[2]);
    acc = __fadd_rn(acc, __fmul_rn(d, d));
  }
  if (s.kind == LRA_GEN_GAUSS) return expf(-__fdiv_rn(acc, s.h2));
  return __fdiv_rn(1.0f, __fsqrt_rn(acc));
}

// Generated strips: the points of the strip's l columns (y[gen_idx[t]] for
// a vertical strip, x[gen_idx[t]] for a horizontal one), 3 floats each, in
// shared memory; entry (g, t) pairs them with the point of row g.
__device__ __forceinline__ float gen_strip_entry(const MaxvolArgs& a, const float* colpt, const float* rowpt,
                                                 int t) {
  const float* cp = colpt + 3 * t;
  return a.gen == 1 ? gen_eval(a.src, rowpt, cp) : gen_eval(a.src, cp, rowpt);
}

__device__ __forceinline__ void load_row_point(const MaxvolArgs& a, long long g, float* rowpt) {
  const float* p = (a.gen == 1 ? a.src.x : a.src.y) + g * a.src.dim;
  rowpt[0] = __ldg(p);
  rowpt[1] = a.src.dim > 1 ? __ldg(p + 1) : 0.0f;
  rowpt[2] = a.src.dim > 2 ? __ldg(p + 2) : 0.0f;
}

// What warp 0 decided, for the other warps.
struct Ctl {
  long long istar;
  unsigned int base;   // grid-barrier arrivals before this launch
  unsigned int seq0;   // the job's decision counter when this launch started
  int kind;            // LRA_TRACE_*, or kFailed: the launch ends
  int jstar;
};

constexpr int kFailed = -1, kUndecided = -2;
enum { kBarOk = 0, kBarTimeout = 1, kBarStatus = 2 };

// Grid-wide barrier of a cooperative launch on a counter that only grows:
// the n-th barrier of a launch waits until the counter reaches base + n G.
// Called by one thread, after a warp or block barrier that orders its CTA's
// writes before it; the arrival is a release add (it publishes them), the
// polls are acquire loads (they order the reads after it).  The wait ends early when the job's status leaves LRA_OK
// (a cancellation, a failure in another CTA) or after 2 s.
__device__ __forceinline__ int grid_arrive_wait(unsigned int* count, unsigned int target,
                                                const int* status) {
  asm volatile("red.release.gpu.global.add.u32 [%0], 1;" ::"l"(count) : "memory");
  const unsigned long long t0 = globaltimer_ns();
  for (unsigned int it = 1;; ++it) {
    if ((int)(ld_acquire_u32(count) - target) >= 0) return kBarOk;
    if ((it & 63u) == 0) {
      if (*reinterpret_cast<const volatile int*>(status) != LRA_OK) return kBarStatus;
      if (globaltimer_ns() - t0 > kWaitNs) return kBarTimeout;
    }
  }
}

// Warm start of the rows of this CTA: W[r, :] = S[g, :] X^{-1}, each entry a
// compensated dot product (Dot2) of the exact FP32 strip row with the pairs
// of X^{-1}; for rows of 8 lanes (l <= 24) as two interleaved sums (even
// and odd terms: two independent dependency chains) added at the end, which
// measured faster there and slower for wider rows.  A group of GS lanes owns a row; lane gl computes columns
// gl + GS c, c < NC, so every issued instruction is useful work
// (NC = ceil(l / GS) exactly).
template <int GS, int NC, typename XPtr>
__device__ __forceinline__ void warm_rows(const MaxvolArgs& a, const int l, dd* B, int nrows, long long row0,
                                          XPtr X, const float* colpt) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  constexpr int kGpw = 32 / GS;
  const int gl = lane % GS;
  const int ngroups = nwarps * kGpw;
  for (int base = warp * kGpw; base < nrows; base += ngroups) {
    const int r = base + lane / GS;
    const bool active = r < nrows;
    const long long g = row0 + r;
    dd* brow = B + (size_t)r * l;
    if (active) {
      if (a.gen) {
        float rowpt[3];
        load_row_point(a, g, rowpt);
#pragma unroll
        for (int c = 0; c < NC; ++c) {
          const int t = gl + GS * c;
          if (t < l) brow[t] = dd_make(gen_strip_entry(a, colpt, rowpt, t));
        }
      } else {
#pragma unroll
        for (int c = 0; c < NC; ++c) {
          const int t = gl + GS * c;
          if (t < l) brow[t] = dd_make(a.strip[g * a.si + (long long)t * a.st]);
        }
      }
    }
    __syncwarp();
    dacc acc[NC];
    int qc[NC];   // the lane's columns, as stored in X
#pragma unroll
    for (int c = 0; c < NC; ++c) {
      acc[c] = dacc{0.0f, 0.0f};
      qc[c] = X.col(min(gl + GS * c, l - 1));
    }
    if (active) {
      if constexpr (GS == 8) {
        dacc acc2[NC];
#pragma unroll
        for (int c = 0; c < NC; ++c) acc2[c] = dacc{0.0f, 0.0f};
        int p = 0;
        for (; p + 1 < l; p += 2) {
          const float sp = brow[p].hi, sq = brow[p + 1].hi;
#pragma unroll
          for (int c = 0; c < NC; ++c) {
            const int q = gl + GS * c;
            if (q < l) {
              acc_fma_f(acc[c], sp, X.at((size_t)p * l + qc[c]));
              acc_fma_f(acc2[c], sq, X.at((size_t)(p + 1) * l + qc[c]));
            }
          }
        }
        if (p < l) {
          const float sp = brow[p].hi;
#pragma unroll
          for (int c = 0; c < NC; ++c) {
            const int q = gl + GS * c;
            if (q < l) acc_fma_f(acc[c], sp, X.at((size_t)p * l + qc[c]));
          }
        }
#pragma unroll
        for (int c = 0; c < NC; ++c) acc[c] = acc_add(acc[c], acc2[c]);
      } else {
        for (int p = 0; p < l; ++p) {
          const float sp = brow[p].hi;
#pragma unroll
          for (int c = 0; c < NC; ++c) {
            const int q = gl + GS * c;
            if (q < l) acc_fma_f(acc[c], sp, X.at((size_t)p * l + qc[c]));
          }
        }
      }
    }
    __syncwarp();
    if (active)
#pragma unroll
      for (int c = 0; c < NC; ++c) {
        const int q = gl + GS * c;
        if (q < l) brow[q] = acc_value(acc[c]);
      }
  }
}

// X^{-1} accessors: col(q) is where column q of X^{-1} is stored, at(i)
// the entry at row-major position i.
struct SharedX {
  const dd* p;
  __device__ __forceinline__ int col(int q) const { return q; }
  __device__ __forceinline__ dd at(size_t i) const { return p[i]; }
};

struct SharedXMapped {  // the in-kernel inverse: column q of X^{-1} is column map[q]
  const dd* p;
  const int* map;
  __device__ __forceinline__ int col(int q) const { return map[q]; }
  __device__ __forceinline__ dd at(size_t i) const { return p[i]; }
};

struct GlobalX {  // read-only path for an X^{-1} that does not fit on chip
  const float2* p;
  __device__ __forceinline__ int col(int q) const { return q; }
  __device__ __forceinline__ dd at(size_t i) const {
    const float2 v = __ldg(p + i);
    return dd{v.x, v.y};
  }
};

// kSelf: the warm start inverts the cross itself (a separate instantiation,
// so that launches without it keep their own register allocation).
// L > 0: a build for l == L exactly (loops and bounds fold at compile time);
// L == 0: any l.
template <int GS, int NC, bool kSelf, int L>
__global__ void __launch_bounds__(kMaxvolThreads, 1) maxvol_kernel(MaxvolArgs a) {
  if (a.js->status != LRA_OK || a.js->stop) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int l = L > 0 ? L : a.l;
  const int tid = threadIdx.x, nthr = blockDim.x;
  const int G = gridDim.x, cta = blockIdx.x;
  const long long N = a.N;
  const long long row0 = (long long)cta * a.rows_per_cta;
  const int nrows = (int)max(0LL, min((long long)a.rows_per_cta, N - row0));
  const int rpc = a.rows_per_cta;

  dd* B = reinterpret_cast<dd*>(smem_raw);                   // rpc * l
  dd* rvec = B + (size_t)rpc * l;                             // l: the update's row factor
  dd* xs = rvec + kMaxL;                                      // l*l when staged
  // the CTA's best word of the current and the next decision (shared atomic max)
  unsigned long long* red = reinterpret_cast<unsigned long long*>(xs + (a.stage_xinv ? (size_t)l * l : 0));
  Ctl* ctl = reinterpret_cast<Ctl*>(red + 2);
  int* pos_s = reinterpret_cast<int*>(ctl + 1);              // l
  InvScratch inv;                                            // the in-kernel inverse
  inv.rowt = rvec;
  inv.colt = reinterpret_cast<dd*>(pos_s + kMaxL);
  inv.rowold = inv.colt + kMaxL;
  inv.pkey = reinterpret_cast<unsigned long long*>(inv.rowold + kMaxL);
  inv.swaps = reinterpret_cast<int*>(inv.pkey + 2);
  inv.at = inv.swaps + kMaxL;
  inv.p_s = inv.at + kMaxL;
  float* colpt = reinterpret_cast<float*>(inv.p_s + 2);     // 3 * kMaxL: generated strips' column points
  unsigned char* used = reinterpret_cast<unsigned char*>(colpt + 3 * kMaxL);  // rpc
  dd* cand_rows = reinterpret_cast<dd*>(a.cand_rows);

  const int lane = tid & 31, warp = tid >> 5;
  constexpr int kGpw = 32 / GS;
  const int gl = lane % GS;
  const int ngroups = (nthr >> 5) * kGpw;

  for (int t = tid; t < l; t += nthr) pos_s[t] = a.gepp ? -1 : a.pos[t];
  if (a.gen)
    for (int e = tid; e < l * a.src.dim; e += nthr) {
      const int t = e / a.src.dim, c = e - t * a.src.dim;
      const float* pts = a.gen == 1 ? a.src.y : a.src.x;
      colpt[3 * t + c] = __ldg(pts + (long long)__ldg(a.gen_idx + t) * a.src.dim + c);
    }
  for (int r = tid; r < nrows; r += nthr) used[r] = 0;
  if (tid < 2) red[tid] = 0ull;
  if (tid == 0) {
    // every launch leaves the counter at a multiple of 256 > G, and no CTA
    // can pass the first barrier before this one arrives
    ctl->base = ld_acquire_u32(&a.bar->count) & ~255u;
    ctl->seq0 = a.bar->seq;   // written by the previous launch of this job
  }
  __syncthreads();

  // ---- W = S (Gauss-Jordan start) or S X^{-1} (warm start)
  if (a.gepp) {
    for (int e = tid; e < nrows * l; e += nthr) {
      const int r = e / l, t = e - r * l;
      float rowpt[3];
      if (a.gen) load_row_point(a, row0 + r, rowpt);
      B[e] = dd_make(a.gen ? gen_strip_entry(a, colpt, rowpt, t) : a.strip[(row0 + r) * a.si + (long long)t * a.st]);
    }
  } else {
    if constexpr (kSelf) {
      // the two-phase elimination: inside this launch it measured faster
      // than the look-ahead form at l = 24
      const auto S = [&](long long g, int c) -> float {
        if (!a.gen) return a.strip[g * a.si + (long long)c * a.st];
        float rowpt[3];
        load_row_point(a, g, rowpt);
        return gen_strip_entry(a, colpt, rowpt, c);
      };
      if (!invert_cross<kMaxvolThreads, L>(S, l, a.js, pos_s, xs, inv)) return;
      warm_rows<GS, NC>(a, l, B, nrows, row0, SharedXMapped{xs, inv.at}, colpt);
    } else if (a.stage_xinv) {
      for (int e = tid; e < l * l; e += nthr) {
        const float2 v = a.xin[e];
        xs[e] = dd{v.x, v.y};
      }
      __syncthreads();
      warm_rows<GS, NC>(a, l, B, nrows, row0, SharedX{xs}, colpt);
    } else {
      warm_rows<GS, NC>(a, l, B, nrows, row0, GlobalX{a.xin}, colpt);
    }
    __syncthreads();
    // rows currently selected are exactly the unit vectors of B = S X^{-1}
    for (int t = 0; t < l; ++t) {
      const long long g = pos_s[t];
      if (g >= row0 && g < row0 + nrows)
        for (int c = tid; c < l; c += nthr) B[(size_t)(g - row0) * l + c] = dd_make(c == t ? 1.0f : 0.0f);
    }
  }
  __syncthreads();

  // ---- initial scan
  unsigned long long mine = 0ull;
  bool gepp_phase = a.gepp != 0;
  for (int e = tid; e < nrows * l; e += nthr) {
    const int r = e / l, t = e - r * l;
    if (gepp_phase && t != 0) continue;
    mine = umax64(mine, cand_word(B[e], (row0 + r) * l + t));
  }

  int buf = 0, step = 0, swaps = 0, capped = 0;
  unsigned int dec = 0, nbar = 0;   // decisions (all threads) and grid barriers (warp 0) of this launch
  for (;;) {
    mine = warp_max(mine);
    if (lane == 0) atomicMax(red + (dec & 1u), mine);
    __syncthreads();

    // ---- warp 0: the CTA's candidate, the grid exchange and the decision
    if (warp == 0) {
      unsigned long long win = red[dec & 1u];
      if (lane == 0) red[(dec + 1u) & 1u] = 0ull;   // the next decision's word
      int kind = kUndecided;
      const dd* prow = nullptr;   // the winner's row of W
      bool prow_global = false;
      const unsigned int s = ctl->seq0 + dec;   // the job's decision number
      if (G > 1) {
        // publish this CTA's row, fold its word into the decision's word,
        // meet the other CTAs, read the maximum
        const unsigned int own_idx = 0xffffffffu - (unsigned int)win;
        if (win != 0ull) {
          const int r = (int)((long long)own_idx / l - row0);
          dd* rec = cand_rows + ((size_t)buf * kMaxGrid + cta) * l;
          for (int t = lane; t < l; t += 32) rec[t] = B[(size_t)r * l + t];
        }
        unsigned long long* word = a.win_ring + (s % kWinRing);
        if (lane == 0 && win != 0ull) atomicMax(word, win);
        __syncwarp();
        ++nbar;
        int code = kBarOk;
        if (lane == 0) code = grid_arrive_wait(&a.bar->count, ctl->base + nbar * (unsigned)G, &a.js->status);
        code = __shfl_sync(0xffffffffu, code, 0);
        if (code != kBarOk) {
          if (code == kBarTimeout && lane == 0) set_status(a.js, LRA_ETIMEOUT);
          kind = kFailed;
        } else {
          if (lane == 0) {
            win = __ldcg(word);
            // every CTA has read the word of decision s - 1 before arriving
            // here, and the word of decision s + 2 is first written after
            // the next barrier, which this thread reaches after this store
            if (cta == 0) a.win_ring[(s + 2) % kWinRing] = 0ull;
          }
          win = __shfl_sync(0xffffffffu, win, 0);
          if (win != 0ull) {
            const long long widx = 0xffffffffu - (unsigned int)win;
            prow = cand_rows + ((size_t)buf * kMaxGrid + (widx / l) / rpc) * l;
            prow_global = true;
          }
        }
      } else if (win != 0ull) {
        prow = B + (size_t)((long long)(0xffffffffu - (unsigned int)win) / l - row0) * l;
      }
      auto load = [&](int t) -> dd {
        if (prow_global) {
          const float2 v = __ldcg(reinterpret_cast<const float2*>(prow + t));
          return dd{v.x, v.y};
        }
        return prow[t];
      };
      const bool none = win == 0ull;
      const long long widx = none ? -1 : (long long)(0xffffffffu - (unsigned int)win);
      const long long istar = none ? -1 : widx / l;
      const int jstar = none ? 0 : (int)(widx - istar * l);
      // the pivot and this lane's entries of the winner's row, issued together
      dd piv = dd_make(0.0f);
      dd rown[kMaxL / 32];
#pragma unroll
      for (int u = 0; u < kMaxL / 32; ++u) rown[u] = dd_make(0.0f);
      if (kind == kUndecided && !none) {
        piv = load(jstar);
#pragma unroll
        for (int u = 0; u < kMaxL / 32; ++u)
          if (lane + 32 * u < l) rown[u] = load(lane + 32 * u);
      }
      const double wv = fabs(dd_to_double(piv));
      if (kind == kUndecided) {
        if ((unsigned int)(win >> 32) >= 0x7f800000u) {
          if (cta == 0 && lane == 0) set_status(a.js, LRA_ENONFINITE);
          kind = kFailed;
        } else if (gepp_phase) {
          if (none || !(wv > 0.0)) {
            if (cta == 0 && lane == 0) set_status(a.js, LRA_ESINGULAR);
            kind = kFailed;
          } else {
            kind = LRA_TRACE_GEPP;
          }
        } else if (none || wv <= 1.0 + a.delta) {
          kind = LRA_TRACE_STOP;
        } else if (swaps >= a.max_swaps) {
          kind = LRA_TRACE_CAP;
        } else {
          kind = LRA_TRACE_SWAP;
        }
      }
      if (kind >= 0 && cta == 0 && lane == 0) {
        const int n = a.js->trace_len;
        if (n < a.js->trace_cap) {
          a.trace_i[4 * n + 0] = a.half_step;
          a.trace_i[4 * n + 1] = kind;
          a.trace_i[4 * n + 2] = (int)istar;
          a.trace_i[4 * n + 3] = jstar;
          a.trace_v[n] = wv;
          a.js->trace_len = n + 1;
        }
        if (kind == LRA_TRACE_STOP) {
          const int o = a.half_step & 1;
          a.js->stop_i[o] = (int)istar;
          a.js->stop_j[o] = jstar;
          a.js->stop_v[o] = wv;
        }
      }
      if (kind == LRA_TRACE_GEPP || kind == LRA_TRACE_SWAP) {
        // the update's row factor (W[i*, :] - e_j*^T) / W[i*, j*]
#pragma unroll
        for (int u = 0; u < kMaxL / 32; ++u) {
          const int t = lane + 32 * u;
          if (t < l) {
            dd rt = rown[u];
            if (t == jstar) rt = dd_add(rt, dd_make(-1.0f));
            rvec[t] = dd_div(rt, piv);
          }
        }
        if (lane == 0) {
          if (gepp_phase && istar >= row0 && istar < row0 + nrows) used[istar - row0] = 1;
          pos_s[jstar] = (int)istar;
        }
      }
      if (lane == 0) {
        ctl->kind = kind;
        ctl->istar = istar;
        ctl->jstar = jstar;
      }
    }
    __syncthreads();
    const int kind = ctl->kind;
    if (kind == kFailed) return;
    if (kind == LRA_TRACE_STOP || kind == LRA_TRACE_CAP) {
      capped = kind == LRA_TRACE_CAP;
      break;
    }
    const long long istar = ctl->istar;
    const int jstar = ctl->jstar;

    // ---- fused update + scan for the next decision; the pivot row becomes
    // e_j* exactly
    const bool next_gepp = gepp_phase && (step + 1 < l);
    const int next_col = step + 1;
    // the lane's entries of the row factor, the same for all its rows
    dd rv[NC];
#pragma unroll
    for (int cc = 0; cc < NC; ++cc) rv[cc] = rvec[min(gl + GS * cc, l - 1)];
    // running best: FP32 |hi| pattern + 1 (so that a zero entry counts) and
    // the row-major position in the chunk; entries are visited in increasing
    // position, so keeping the first of equal patterns keeps the smaller index
    unsigned int bk = 0u;
    int be = 0;
    for (int base = warp * kGpw; base < nrows; base += ngroups) {
      const int r = base + lane / GS;
      const bool act = r < nrows;
      dd* brow = B + (size_t)(act ? r : 0) * l;
      // the row's entry in column j* is read before its group writes the row
      const dd c = act ? brow[jstar] : dd_make(0.0f);
      __syncwarp();
      const bool piv_row = row0 + r == istar;
      const bool scan_row = act && !(next_gepp && used[act ? r : 0]);
#pragma unroll
      for (int cc = 0; cc < NC; ++cc) {
        const int t = gl + GS * cc;
        if (t < l) {
          dd v = dd_fnma(c, rv[cc], act ? brow[t] : dd_make(0.0f));
          if (piv_row) v = dd_make(t == jstar ? 1.0f : 0.0f);
          if (act) brow[t] = v;
          const unsigned int k1 = (__float_as_uint(v.hi) & 0x7fffffffu) + 1u;
          if (scan_row && (!next_gepp || t == next_col) && k1 > bk) {
            bk = k1;
            be = r * l + t;
          }
        }
      }
    }
    mine = bk ? ((unsigned long long)(bk - 1u) << 32) | (0xffffffffu - (unsigned int)(row0 * l + be)) : 0ull;
    if (gepp_phase) {
      if (++step == l) gepp_phase = false;
    } else {
      ++swaps;
    }
    buf ^= 1;
    ++dec;
  }

  // ---- epilogue: positions, counters, the job's decision counter, and the
  // barrier counter rounded up to a multiple of 256 for the next launch
  // (every CTA took the same decisions and has arrived at the last barrier
  // once CTA 0 passed it)
  if (cta == 0 && tid < l) a.pos[tid] = pos_s[tid];
  if (cta == 0 && tid == 0) {
    a.js->swaps_total += swaps;
    if (capped) a.js->converged = 0;
    // algorithmic flops: warm-start product S X^{-1} plus one rank-one
    // update of the N x l matrix W per GEPP step or swap
    const double upd = (double)(step + swaps) * 2.0 * (double)N * l;
    const double init = a.gepp ? 0.0 : 2.0 * (double)N * l * l;
    a.js->maxvol_flops += upd + init;
    if (a.count_sweep) a.js->sweeps_done += 1;
    if (a.fixed_point_exit) {
      // a warm-started half-step without a swap after another one: the
      // next half-step has the same strip, index set and cross as the one
      // before this, so it and all later ones repeat their decisions
      a.js->noswap_run = (a.gepp || swaps > 0 || capped) ? 0 : a.js->noswap_run + 1;
      if (a.js->noswap_run >= 2 && a.half_step + 1 < a.total_half_steps) {
        for (int h = a.half_step + 1; h < a.total_half_steps; ++h) {
          const int n = a.js->trace_len, o = h & 1;
          if (n < a.js->trace_cap) {
            a.trace_i[4 * n + 0] = h;
            a.trace_i[4 * n + 1] = LRA_TRACE_STOP;
            a.trace_i[4 * n + 2] = a.js->stop_i[o];
            a.trace_i[4 * n + 3] = a.js->stop_j[o];
            a.trace_v[n] = a.js->stop_v[o];
            a.js->trace_len = n + 1;
          }
        }
        a.js->sweeps_done = a.total_half_steps / 2;
        a.js->stop = 1;
      }
    }
    a.bar->seq = ctl->seq0 + dec + 1;   // the decisions taken, the final stop included
    const unsigned int pad = (256u - ((nbar * (unsigned)G) & 255u)) & 255u;
    if (pad) atomicAdd(&a.bar->count, pad);
  }
}

static size_t maxvol_smem(int rpc, int l, bool stage_xinv) {
  size_t b = (size_t)rpc * l * sizeof(dd) + kMaxL * sizeof(dd) +
             (stage_xinv ? (size_t)l * l * sizeof(dd) : 0) +
             2 * sizeof(unsigned long long) + sizeof(Ctl) + kMaxL * sizeof(int) +
             2 * kMaxL * sizeof(dd) + 2 * sizeof(unsigned long long) + (2 * kMaxL + 2) * sizeof(int) +
             3 * kMaxL * sizeof(float) + (size_t)rpc;
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

template <int GS, int NC, int L = 0>
static cudaError_t launch_gs(MaxvolArgs& a, const MaxvolPlan& plan, cudaStream_t st) {
  const void* k = (a.self_inverse && !a.gepp) ? reinterpret_cast<const void*>(maxvol_kernel<GS, NC, true, L>)
                                              : reinterpret_cast<const void*>(maxvol_kernel<GS, NC, false, L>);
  const cudaError_t e = smem_optin(k, 227 * 1024);
  if (e != cudaSuccess) return e;
  void* args[] = {&a};
  return cudaLaunchCooperativeKernel(k, dim3(plan.grid), dim3(plan.threads), args, plan.smem, st);
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
  if (a.self_inverse && !plan.stage_xinv) return cudaErrorInvalidValue;  // no room for X^{-1}
  a.rows_per_cta = plan.rows_per_cta;
  a.stage_xinv = plan.stage_xinv;
  // builds for the cross sizes of the served ranks (l = 1.5 k, k = 8 ... 64)
  switch (a.l) {
    case 12: return launch_gs<8, 2, 12>(a, plan, st);
    case 24: return launch_gs<8, 3, 24>(a, plan, st);
    case 48: return launch_gs<16, 3, 48>(a, plan, st);
    case 96: return launch_gs<32, 3, 96>(a, plan, st);
    default: break;
  }
  if (a.l <= 24) return launch_nc<8>(a, plan, st);
  if (a.l <= 48) return launch_nc<16>(a, plan, st);
  return launch_nc<32>(a, plan, st);
}

}  // namespace lra
