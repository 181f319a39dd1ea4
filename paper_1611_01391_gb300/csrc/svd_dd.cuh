// Singular value decomposition of a small square matrix (l <= 96) on one
// CTA, in double-float arithmetic: every value is an unevaluated pair
// hi + lo of FP32 numbers (Dekker, "A floating-point technique for extending
// the available precision", 1971; Knuth TAOCP vol. 2, 4.2.2; Hida, Li &
// Bailey, "Algorithms for quad-double precision", 2001), carrying about 48
// significant bits.  On this GPU the FP64 pipe issues 1/64 of the FP32 rate,
// so a double-float multiply-add (10 to 20 FP32 instructions) is several
// times cheaper than a native FP64 one.
//
// Method: Householder QR with column pivoting, then Hestenes' one-sided
// Jacobi on the transposed triangular factor (the preconditioned Jacobi SVD
// of Drmac & Veselic); dot products are compensated FP32 sums (Dot2).
#pragma once

#include <cooperative_groups.h>

#include <cfloat>

#include "dd_arith.cuh"
#include "lra_internal.cuh"

namespace lra {

// Plane rotation that annihilates the off-diagonal of the 2 x 2 Gram matrix
// [a g; g b] (Golub & Van Loan, Algorithm 8.5.1): zeta = (b - a) / (2 g),
// t = sign(zeta) / (|zeta| + sqrt(1 + zeta^2)).  t is needed to FP32
// accuracy only (any t gives an orthogonal rotation; t sets the speed of
// convergence), so it takes a short FP32 chain.  The cosine
// c = (1 + t^2)^{-1/2} must be accurate to double-float precision: the
// correctly rounded FP32 reciprocal square root y0 of x = 1 + t^2 (formed
// exactly as a pair) is refined by one Newton step y0 + y0 r / 2 with
// r = 1 - x y0^2; r is of order 2^-23 and its FMA-built FP32 value is
// accurate to about 2^-47.  Returns c; *t_out = t.
__device__ __forceinline__ dd rotation_cosine(dd a, dd b, dd g, float* t_out) {
  const dd d = two_sum(b.hi, -a.hi);
  const float diff = __fadd_rn(d.hi, __fadd_rn(d.lo, __fsub_rn(b.lo, a.lo)));
  const float zeta = __fdividef(diff, 2.0f * g.hi);
  float t;
  if (fabsf(zeta) > 1e18f) {
    t = __fdividef(0.5f, zeta);
  } else {
    const float q = fmaf(zeta, zeta, 1.0f);
    t = copysignf(__frcp_rn(fabsf(zeta) + q * __frsqrt_rn(q)), zeta);
  }
  *t_out = t;
  const float t2 = __fmul_rn(t, t);
  const float t2e = fmaf(t, t, -t2);             // t^2 = t2 + t2e exactly
  const dd xh = two_sum(1.0f, t2);
  const float xl = __fadd_rn(xh.lo, t2e);        // x = xh.hi + xl
  const float y0 = __frsqrt_rn(xh.hi);
  const float y2 = __fmul_rn(y0, y0);
  const float y2e = fmaf(y0, y0, -y2);           // y0^2 = y2 + y2e exactly
  float r = fmaf(-xh.hi, y2, 1.0f);
  r = fmaf(-xh.hi, y2e, r);
  r = fmaf(-xl, y2, r);
  return quick_two_sum(y0, __fmul_rn(__fmul_rn(0.5f, y0), r));
}


// c x + s y in double-float: both products with their FMA error terms, one
// TwoSum for the high parts.
__device__ __forceinline__ dd dd_lin2(dd c, dd x, dd s, dd y) {
  const float p1 = __fmul_rn(c.hi, x.hi);
  float e1 = fmaf(c.hi, x.hi, -p1);
  e1 = fmaf(c.hi, x.lo, e1);
  e1 = fmaf(c.lo, x.hi, e1);
  const float p2 = __fmul_rn(s.hi, y.hi);
  float e2 = fmaf(s.hi, y.hi, -p2);
  e2 = fmaf(s.hi, y.lo, e2);
  e2 = fmaf(s.lo, y.hi, e2);
  const dd t = two_sum(p1, p2);
  return two_sum(t.hi, __fadd_rn(t.lo, __fadd_rn(e1, e2)));
}

// sqrt and reciprocal: FP32 seed, one double-float Newton correction.
__device__ __forceinline__ dd dd_sqrt(dd a) {
  if (!(a.hi > 0.0f)) return dd{0.0f, 0.0f};
  const float y = sqrtf(a.hi);
  const dd r = dd_add(a, dd_neg(dd_mul(dd_make(y), dd_make(y))));
  return quick_two_sum(y, __fdiv_rn(r.hi, 2.0f * y));
}

__device__ __forceinline__ dd dd_recip(dd d) {
  const float r0 = __frcp_rn(d.hi);
  const dd e = dd_add(dd_make(1.0f), dd_neg(dd_mul(d, dd_make(r0))));
  return quick_two_sum(r0, __fmul_rn(r0, e.hi));
}

// for (i = first; i < l; i += STEP) body(i) with first >= 0.  With L > 0
// the trip count is fixed at ceil(L / STEP) (the iterations past l do
// nothing), so the loop unrolls and its shared-memory loads issue together
// instead of one iteration's latency after another; the iterations run in
// the same order either way.
template <int L, int STEP, typename F>
__device__ __forceinline__ void strided(int first, int l, F&& body) {
  if constexpr (L > 0) {
#pragma unroll
    for (int it = 0; it < (L + STEP - 1) / STEP; ++it) {
      const int i = first + STEP * it;
      if (i < l) body(i);
    }
  } else {
    for (int i = first; i < l; i += STEP) body(i);
  }
}

// Shared scratch of the SVD below.
struct SvdScratch {
  int perm[kMaxL];    // column c of X P is column perm[c] of X
  dd rdiag[kMaxL];    // diagonal of R
  dd beta[kMaxL];     // Householder scalars
  dd nrm[kMaxL];      // squared norms of the trailing columns
  int piv;
  int flag;
};

// Householder QR with column pivoting (Businger & Golub, 1965; Golub & Van
// Loan, Algorithm 5.4.1) of the l x l matrix A (column c at A[c*l, c*l+l)),
// in place: on exit the strictly upper part of R is in A (row j of column
// c > j), its diagonal in sc->rdiag, and the Householder vector v_j in rows
// j..l-1 of column j, with H_j = I - beta_j v_j v_j^T.  The pivot is the
// trailing column of largest norm (ties: the smaller column); the norms are
// recomputed from the updated columns at every step; a trailing column of
// squared norm at most 2^-100 is taken as zero (R's diagonal entry 0).
// L > 0 (every function below): a build for l == L exactly.
template <int NT, int L = 0>
__device__ void qrcp_dd(dd* A, int l_arg, SvdScratch* sc) {
  const int l = L > 0 ? L : l_arg;
  constexpr int G = 8, GPW = 32 / G, NG = NT / G;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, gl = lane & (G - 1);
  for (int c = tid; c < l; c += NT) sc->perm[c] = c;
  for (int base = warp * GPW; base < l; base += NG) {
    const int c = base + (lane / G);
    dacc a{0.f, 0.f};
    if (c < l) strided<L, G>(gl, l, [&](int i) { acc_fma(a, A[c * l + i], A[c * l + i]); });
    a = acc_group_sum<G>(a);
    if (c < l && gl == 0) sc->nrm[c] = acc_value(a);
  }
  __syncthreads();
  for (int j = 0; j < l; ++j) {
    if (warp == 0) {
      float best = -1.0f, bl = 0.0f;
      int bc = l;
      for (int c = j + lane; c < l; c += 32) {
        const dd v = sc->nrm[c];
        if (v.hi > best || (v.hi == best && v.lo > bl)) {
          best = v.hi;
          bl = v.lo;
          bc = c;
        }
      }
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) {
        const float ob = __shfl_xor_sync(0xffffffffu, best, off);
        const float ol = __shfl_xor_sync(0xffffffffu, bl, off);
        const int oc = __shfl_xor_sync(0xffffffffu, bc, off);
        if (ob > best || (ob == best && (ol > bl || (ol == bl && oc < bc)))) {
          best = ob;
          bl = ol;
          bc = oc;
        }
      }
      if (lane == 0) sc->piv = bc;
    }
    __syncthreads();
    const int pc = sc->piv;
    if (pc != j && pc < l) {
      for (int i = tid; i < l; i += NT) {
        const dd t = A[j * l + i];
        A[j * l + i] = A[pc * l + i];
        A[pc * l + i] = t;
      }
      if (tid == 0) {
        const int t = sc->perm[j];
        sc->perm[j] = sc->perm[pc];
        sc->perm[pc] = t;
        const dd u = sc->nrm[j];
        sc->nrm[j] = sc->nrm[pc];
        sc->nrm[pc] = u;
      }
    }
    __syncthreads();
    if (warp == 0) {  // reflector of rows j..l-1 of column j
      dacc a{0.f, 0.f};
      strided<L, 32>(j + lane, l, [&](int i) { acc_fma(a, A[j * l + i], A[j * l + i]); });
      a = acc_group_sum<32>(a);
      if (lane == 0) {
        const dd n2 = acc_value(a);
        // X is scaled to max |X| < 1: a trailing column of squared norm below
        // 2^-100 (norm 2^-50, under the pairs' 2^-48 rounding) is numerically
        // zero.  Below that the reflector's scalar 1 / (n2 + |x0| ||x||) can
        // overflow FP32 (repeated rows and columns of a sampled generator
        // leave such columns), so the step is skipped as for an exact zero.
        if (!(n2.hi > 0x1p-100f)) {
          sc->beta[j] = dd{0.f, 0.f};
          sc->rdiag[j] = dd{0.f, 0.f};
        } else {
          const dd nx = dd_sqrt(n2);
          const dd x0 = A[j * l + j];
          const dd alpha = x0.hi >= 0.0f ? dd_neg(nx) : nx;
          const dd ax0 = x0.hi >= 0.0f ? x0 : dd_neg(x0);
          A[j * l + j] = dd_add(x0, dd_neg(alpha));
          sc->beta[j] = dd_recip(dd_add(n2, dd_mul(ax0, nx)));
          sc->rdiag[j] = alpha;
        }
      }
    }
    __syncthreads();
    const dd bj = sc->beta[j];
    for (int base = j + 1 + warp * GPW; base < l; base += NG) {
      const int c = base + (lane / G);
      const bool act = c < l;
      dacc a{0.f, 0.f};
      if (act) strided<L, G>(j + gl, l, [&](int i) { acc_fma(a, A[j * l + i], A[c * l + i]); });
      a = acc_group_sum<G>(a);
      const dd sv = dd_mul(bj, acc_value(a));
      const dd nsv = dd_neg(sv);
      dacc nn{0.f, 0.f};
      if (act)
        strided<L, G>(j + gl, l, [&](int i) {
          const dd x = dd_lin2(dd_make(1.0f), A[c * l + i], nsv, A[j * l + i]);
          A[c * l + i] = x;
          if (i > j) acc_fma(nn, x, x);
        });
      nn = acc_group_sum<G>(nn);
      if (act && gl == 0) sc->nrm[c] = acc_value(nn);
    }
    __syncthreads();
  }
}

// One-sided Jacobi (Hestenes) on the columns of W, the rotations applied to
// the columns of Z as well when kAccumulate.  On exit W has orthogonal
// columns.  Columns are
// paired in round-robin order (l/2 independent pairs per round, G lanes per
// pair); a pair is rotated unless |w_p^T w_q| <= tol ||w_p|| ||w_q||.  The
// rotation tangent of the symmetric 2 x 2 problem (Golub & Van Loan,
// Algorithm 8.5.1) is taken to FP32 accuracy; c = (1 + t^2)^{-1/2} and
// s = c t are formed in double-float from that t, so every rotation is
// orthogonal to double-float accuracy and only the speed of convergence
// depends on t.
template <int NT, bool kAccumulate = true, int G = 8, int L = 0>
__device__ void jacobi_dd(dd* W, dd* Z, int l_arg, int* flag) {
  const int l = L > 0 ? L : l_arg;
  static_assert(G == 8 || G == 16, "lanes per pair");
  constexpr int kPairsPerWarp = 32 / G;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int np = (l + 1) & ~1;
  // about l * 2^-48; the test below runs on the FP32 high parts (relative
  // error 2^-24 of a threshold), keeping the FP64 pipe (1/64 rate) off the
  // inner loop
  const float tol = (float)l * 3.6e-15f;
  const int gl = lane & (G - 1), ngroups = (NT / 32) * kPairsPerWarp;
  for (int sweep = 0; sweep < 60; ++sweep) {
    if (tid == 0) *flag = 0;
    __syncthreads();
    for (int round = 0; round < np - 1; ++round) {
      for (int base = warp * kPairsPerWarp; base < np / 2; base += ngroups) {
        const int slot = base + lane / G;
        const int x0 = slot, x1 = np - 1 - slot;
        int p = (x0 == 0) ? 0 : ((x0 - 1 + round) % (np - 1)) + 1;
        int q = (x1 == 0) ? 0 : ((x1 - 1 + round) % (np - 1)) + 1;
        if (p > q) { const int t = p; p = q; q = t; }
        const bool act = slot < np / 2 && q < l;
        dd* wp = W + p * l;
        dd* wq = W + q * l;
        dacc sa{0.f, 0.f}, sb{0.f, 0.f}, sg{0.f, 0.f};
        if (act)
          strided<L, G>(gl, l, [&](int i) {
            const dd u = wp[i], v = wq[i];
            acc_fma(sa, u, u);
            acc_fma(sb, v, v);
            acc_fma(sg, u, v);
          });
        sa = acc_group_sum<G>(sa);
        sb = acc_group_sum<G>(sb);
        sg = acc_group_sum<G>(sg);
        if (!act) continue;
        const dd al = acc_value(sa), be = acc_value(sb), ga = acc_value(sg);
        if (!(al.hi > 0.0f) || !(be.hi > 0.0f) || fabsf(ga.hi) <= tol * sqrtf(al.hi) * sqrtf(be.hi)) continue;
        float tf_out;
        const dd c = rotation_cosine(al, be, ga, &tf_out);
        const float tf = tf_out;
        const dd s = dd_mul(c, dd_make(tf));
        const dd ns = dd_neg(s);
        strided<L, G>(gl, l, [&](int i) {
          const dd u = wp[i], v = wq[i];
          wp[i] = dd_lin2(c, u, ns, v);
          wq[i] = dd_lin2(s, u, c, v);
        });
        if (kAccumulate) {
          dd* zp = Z + p * l;
          dd* zq = Z + q * l;
          strided<L, G>(gl, l, [&](int i) {
            const dd xx = zp[i], yy = zq[i];
            zp[i] = dd_lin2(c, xx, ns, yy);
            zq[i] = dd_lin2(s, xx, c, yy);
          });
        }
        if (gl == 0) *flag = 1;
      }
      __syncthreads();
    }
    if (*flag == 0) break;
    __syncthreads();
  }
}

// jacobi_dd<NT, false, 8, L> on the CTAs of a cluster of NC.  The pairs of
// a round are slots s = 0 .. L/2 - 1 of the round-robin order, pairing the
// columns at positions s and L - 1 - s; CTA c takes slots c S .. c S + S - 1
// (S = L / (2 NC)), one warp per pair, and keeps the 2 S columns of those
// positions in its shared memory (cb: two buffers of 2 S columns).  From
// one round to the next a column moves from position x to x - 1 (position 1
// to L - 1, position 0 stays), so after its rotation a warp writes both
// columns straight into the buffer of the next round of the CTA that holds
// their next positions (distributed shared memory), and one cluster barrier
// per round ends the round.  Within a pair the three dot products run on
// three groups of 8 lanes (each in the lane order and summation tree of
// jacobi_dd's 8-lane group) and the column updates on all 32 lanes (the
// same operations per entry), so every rotation, and the result, is
// bitwise that of jacobi_dd.  W: the full L x L matrix in every CTA on
// entry; on exit every CTA holds the full result.  flags: two ints.
template <int NT, int L, int NC>
__device__ void jacobi_dd_cluster(cooperative_groups::cluster_group& cl, dd* W, dd* cb, int* flags) {
  static_assert(L % (2 * NC) == 0, "pairs per CTA");
  constexpr int S = L / (2 * NC);
  constexpr int NP = L;   // even: every position holds a column
  static_assert(S <= NT / 32, "one warp per pair");
  const int rank = (int)cl.block_rank();
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, grp = lane >> 3, gl = lane & 7;
  // column at position x in round r of a sweep
  auto colof = [](int x, int r) { return x == 0 ? 0 : ((x - 1 + r) % (NP - 1)) + 1; };
  // position x of slot k of this CTA: low half k, high half S + k
  auto posof = [&](int li) { return li < S ? rank * S + li : NP - 1 - (rank * S + li - S); };
  // CTA and local index of position x
  auto home = [](int x, int& cta, int& li) {
    if (x < NP / 2) {
      cta = x / S;
      li = x - cta * S;
    } else {
      const int s = NP - 1 - x;
      cta = s / S;
      li = S + s - cta * S;
    }
  };
  for (int e = tid; e < 2 * S * L; e += NT) {
    const int li = e / L, i = e - li * L;
    cb[e] = W[colof(posof(li), 0) * L + i];
  }
  if (tid < 2) flags[tid] = 0;
  __syncthreads();
  // about l * 2^-48, tested on the FP32 high parts as in jacobi_dd
  const float tol = (float)L * 3.6e-15f;
  int buf = 0;
  for (int sweep = 0; sweep < 60; ++sweep) {
    for (int round = 0; round < NP - 1; ++round) {
      if (warp < S) {
        const int xl = posof(warp), xh = posof(S + warp);
        const bool low_first = colof(xl, round) < colof(xh, round);   // p < q
        const int xp = low_first ? xl : xh, xq = low_first ? xh : xl;
        const dd* wp = cb + (size_t)buf * 2 * S * L + (low_first ? warp : S + warp) * L;
        const dd* wq = cb + (size_t)buf * 2 * S * L + (low_first ? S + warp : warp) * L;
        int cp, lp, cq, lq;
        home(xp == 0 ? 0 : (xp == 1 ? NP - 1 : xp - 1), cp, lp);
        home(xq == 0 ? 0 : (xq == 1 ? NP - 1 : xq - 1), cq, lq);
        dd* dp = cl.map_shared_rank(cb + (size_t)(buf ^ 1) * 2 * S * L + lp * L, cp);
        dd* dq = cl.map_shared_rank(cb + (size_t)(buf ^ 1) * 2 * S * L + lq * L, cq);
        // group 0: w_p^T w_p, group 1: w_q^T w_q, group 2: w_p^T w_q
        dacc a{0.f, 0.f};
        if (grp < 3)
          strided<L, 8>(gl, L, [&](int i) {
            const dd u = grp == 1 ? wq[i] : wp[i];
            const dd v = grp == 0 ? wp[i] : wq[i];
            acc_fma(a, u, v);
          });
        a = acc_group_sum<8>(a);
        const dacc sa{__shfl_sync(0xffffffffu, a.s, 0), __shfl_sync(0xffffffffu, a.c, 0)};
        const dacc sb{__shfl_sync(0xffffffffu, a.s, 8), __shfl_sync(0xffffffffu, a.c, 8)};
        const dacc sg{__shfl_sync(0xffffffffu, a.s, 16), __shfl_sync(0xffffffffu, a.c, 16)};
        const dd al = acc_value(sa), be = acc_value(sb), ga = acc_value(sg);
        const bool rot = (al.hi > 0.0f) && (be.hi > 0.0f) && !(fabsf(ga.hi) <= tol * sqrtf(al.hi) * sqrtf(be.hi));
        // the rotation is formed beside the test (its chain does not wait
        // for it) and used only when the test asks for it
        float tf;
        const dd c = rotation_cosine(al, be, ga, &tf);
        const dd s = dd_mul(c, dd_make(tf));
        const dd ns = dd_neg(s);
        if (rot) {
          strided<L, 32>(lane, L, [&](int i) {
            const dd u = wp[i], v = wq[i];
            dp[i] = dd_lin2(c, u, ns, v);
            dq[i] = dd_lin2(s, u, c, v);
          });
          if (lane == 0) flags[sweep & 1] = 1;
        } else {
          strided<L, 32>(lane, L, [&](int i) {
            dp[i] = wp[i];
            dq[i] = wq[i];
          });
        }
      }
      cl.sync();   // the round's columns are in place for the next round
      buf ^= 1;
    }
    // the sweep rotated somewhere in the cluster?
    int any = 0;
    if (tid < NC) any = *cl.map_shared_rank(&flags[sweep & 1], tid);
    any = __syncthreads_or(any);
    // the next sweep's flag (last read by the other CTAs before this sweep's rounds)
    if (tid == 0) flags[(sweep + 1) & 1] = 0;
    __syncthreads();
    if (!any) break;
  }
  // every sweep has NP - 1 rounds, so position x holds column colof(x, 0):
  // every CTA writes its columns into every CTA's W
  const dd* fin = cb + (size_t)buf * 2 * S * L;
  for (int d = 0; d < NC; ++d) {
    dd* dst = cl.map_shared_rank(W, d);
    for (int e = tid; e < 2 * S * L; e += NT) {
      const int li = e / L, i = e - li * L;
      dst[colof(posof(li), 0) * L + i] = fin[e];
    }
  }
  cl.sync();
}

// SVD of the l x l matrix X held in A (column c at A[c*l, c*l+l)), with Z an
// l x l work area: QR with column pivoting X P = Q R, then one-sided Jacobi
// on R^T (the preconditioning of Drmac & Veselic, "New fast and accurate
// Jacobi SVD algorithm I", SIAM J. Matrix Anal. Appl. 29, 2008: on the
// graded R^T the sweeps roughly halve).  With R^T V = W (orthogonal columns)
// this is X = (Q V) W^T P^T, so on exit (W in A)
//   sigma_b = ||W[:, b]||,  right singular vector b of X = P W[:, b] / sigma_b.
// The rotations are not accumulated: the left singular vectors needed later
// are u_b = X P W_b / sigma_b^2 (left_vectors), so Z keeps a copy of X.
template <int NT, int L = 0>
__device__ void svd_dd_precondition(dd* A, dd* Z, int l_arg, SvdScratch* sc);

template <int NT, int L = 0>
__device__ void svd_dd(dd* A, dd* Z, int l_arg, SvdScratch* sc) {
  const int l = L > 0 ? L : l_arg;
  svd_dd_precondition<NT, L>(A, Z, l, sc);
  jacobi_dd<NT, false, (NT >= 1024 ? 16 : 8), L>(A, nullptr, l, &sc->flag);
}

// The steps of svd_dd before the Jacobi sweeps: Z = X, the QR with column
// pivoting of X, and A = R^T.
template <int NT, int L>
__device__ void svd_dd_precondition(dd* A, dd* Z, int l_arg, SvdScratch* sc) {
  const int l = L > 0 ? L : l_arg;
  for (int e = threadIdx.x; e < l * l; e += NT) Z[e] = A[e];
  qrcp_dd<NT, L>(A, l, sc);
  // W = R^T in place: column j of W = row j of R (pivoted column order)
  constexpr int kPer = (kMaxL * kMaxL + NT - 1) / NT;
  dd v[kPer];
#pragma unroll
  for (int t = 0; t < kPer; ++t) {
    const int e = threadIdx.x + t * NT;
    v[t] = dd{0.f, 0.f};
    if (e < l * l) {
      const int j = e / l, c = e - j * l;
      if (c > j) v[t] = A[c * l + j];
      else if (c == j) v[t] = sc->rdiag[j];
    }
  }
  __syncthreads();
#pragma unroll
  for (int t = 0; t < kPer; ++t) {
    const int e = threadIdx.x + t * NT;
    if (e < l * l) A[e] = v[t];
  }
  __syncthreads();
}

// Left singular vectors of the kept triplets, in place of the copy of X in
// Z: u_r = X P W_{b_r} inv2[r] (b_r = order[r], inv2[r] = 1 / sigma_{b_r}^2)
// into column r of Z, r < ke.  One warp per row q of X: the warp holds the
// row in registers (l <= 96: three values per lane) before it overwrites
// that row's first ke positions, so rows are independent.
// Rows q0, q0 + qs, ... only when qs > 1 (the rows of one CTA of a cluster).
template <int NT, int L = 0>
__device__ void left_vectors(const dd* W, dd* Z, int l_arg, int ke, const int* order, const dd* inv2,
                             const int* perm, int q0 = 0, int qs = 1) {
  const int l = L > 0 ? L : l_arg;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int q = q0 + warp * qs; q < l; q += (NT / 32) * qs) {
    dd x[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const int c = lane + 32 * k;
      x[k] = c < l ? Z[perm[c] * l + q] : dd{0.f, 0.f};   // X[q][perm[c]]
    }
    __syncwarp();
    for (int r = 0; r < ke; ++r) {
      const dd* w = W + order[r] * l;
      dacc a{0.f, 0.f};
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        const int c = lane + 32 * k;
        if (c < l) acc_fma(a, x[k], w[c]);
      }
      a = acc_group_sum<32>(a);
      if (lane == 0) Z[r * l + q] = dd_mul(acc_value(a), inv2[r]);
    }
    __syncwarp();
  }
  __syncthreads();
}

// After jacobi_dd: sigma_b = ||W_b|| (double), order[rank] = column (sigma
// descending, ties to the smaller column).  sig, order: shared arrays.
template <int NT>
__device__ void jacobi_sigma(const dd* W, int l, double* sig, int* order) {
  const int tid = threadIdx.x;
  for (int b = tid; b < l; b += NT) {
    dd ss{0.f, 0.f};
    for (int i = 0; i < l; ++i) ss = dd_fma(W[b * l + i], W[b * l + i], ss);
    sig[b] = sqrt(dd_to_double(ss));
  }
  __syncthreads();
  for (int b = tid; b < l; b += NT) {
    int rk = 0;
    for (int c = 0; c < l; ++c) rk += (sig[c] > sig[b]) || (sig[c] == sig[b] && c < b);
    order[rk] = b;
  }
  __syncthreads();
}

// (X_k)^+ from svd_dd and left_vectors: U[perm[c]][q] = sum_{r < ke}
// W[b_r][c] u_r[q] inv2[r] with b_r = order[r], u_r = column r of Z and
// inv2[r] = 1 / sigma_{b_r}^2 (shared, computed once); out(e, value)
// receives the l*l entries, row-major e = p*l + q (p a column of X, q a row
// of X).
// With qs > 1 only the entries of rows q0, q0 + qs, ... of X (the rows of
// one CTA of a cluster).
template <int NT, int L = 0, typename Out>
__device__ void nucleus_from_svd(const dd* W, const dd* Z, const int* perm, int l_arg, int ke,
                                 const int* order, const dd* inv2, Out out, int q0 = 0, int qs = 1) {
  const int l = L > 0 ? L : l_arg;
  const int nq = (l - q0 + qs - 1) / qs;
  for (int e = threadIdx.x; e < l * nq; e += NT) {
    const int c = e / nq, q = q0 + (e - c * nq) * qs;
    dd acc{0.f, 0.f};
    for (int r = 0; r < ke; ++r) {
      const int b = order[r];
      acc = dd_fma(dd_mul(W[b * l + c], Z[r * l + q]), inv2[r], acc);
    }
    out(perm[c] * l + q, dd_to_double(acc));
  }
}

}  // namespace lra
