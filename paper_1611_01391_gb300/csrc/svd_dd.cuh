// One-sided Jacobi SVD of a small square matrix (l <= 96) on one CTA, in
// double-float arithmetic: every value is an unevaluated pair hi + lo of
// FP32 numbers (Dekker, "A floating-point technique for extending the
// available precision", 1971; Knuth TAOCP vol. 2, 4.2.2; Hida, Li & Bailey,
// "Algorithms for quad-double precision", 2001), carrying about 48
// significant bits.  On this GPU the FP64 pipe issues 1/64 of the FP32 rate,
// so a double-float FMA (about 15 FP32 instructions) is about 4x cheaper
// than a native FP64 one.
//
// Jacobi method: Hestenes' one-sided variant; the columns of W = X V are
// orthogonalised by plane rotations visited in round-robin order (l/2
// independent pairs per round, 8 lanes per pair).  The rotation tangent of
// the symmetric 2 x 2 Jacobi step (Golub & Van Loan, Algorithm 8.5.1) is
// taken to FP32 accuracy; c = (1 + t^2)^{-1/2} and s = c t are formed in
// double-float from that t, so every rotation is orthogonal to double-float
// accuracy and only the speed of convergence depends on t.
#pragma once

#include <cfloat>

namespace lra {

struct dd {
  float hi, lo;
};

__device__ __forceinline__ dd dd_make(float x) { return dd{x, 0.0f}; }

__device__ __forceinline__ dd dd_from_double(double x) {
  const float h = (float)x;
  return dd{h, (float)(x - (double)h)};
}

__device__ __forceinline__ double dd_to_double(dd a) { return (double)a.hi + (double)a.lo; }

// Knuth's TwoSum: s + e == a + b exactly.
__device__ __forceinline__ dd two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float z = __fsub_rn(s, a);
  return dd{s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, z)), __fsub_rn(b, z))};
}

// Dekker's FastTwoSum (|a| >= |b|): renormalise a pair.
__device__ __forceinline__ dd quick_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  return dd{s, __fsub_rn(b, __fsub_rn(s, a))};
}

__device__ __forceinline__ dd dd_add(dd a, dd b) {
  dd s = two_sum(a.hi, b.hi);
  const dd t = two_sum(a.lo, b.lo);
  s.lo = __fadd_rn(s.lo, t.hi);
  s = quick_two_sum(s.hi, s.lo);
  s.lo = __fadd_rn(s.lo, t.lo);
  return quick_two_sum(s.hi, s.lo);
}

__device__ __forceinline__ dd dd_neg(dd a) { return dd{-a.hi, -a.lo}; }

// TwoProduct through the FMA, plus the cross terms.
__device__ __forceinline__ dd dd_mul(dd a, dd b) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = fmaf(a.hi, b.hi, -p);
  e = fmaf(a.hi, b.lo, e);
  e = fmaf(a.lo, b.hi, e);
  return quick_two_sum(p, e);
}

__device__ __forceinline__ dd dd_fma(dd a, dd b, dd c) { return dd_add(dd_mul(a, b), c); }

// x^{-1/2} for x in [1, 2]: FP32 seed, one double-float Newton step
// y <- y + y (1 - x y^2) / 2.
__device__ __forceinline__ dd dd_rsqrt_1_2(dd x) {
  const float y0 = rsqrtf(x.hi);
  const dd y = dd_make(y0);
  const dd r = dd_add(dd_make(1.0f), dd_neg(dd_mul(x, dd_mul(y, y))));
  return dd_add(y, dd_mul(y, dd{0.5f * r.hi, 0.5f * r.lo}));
}

// W: column b at W[b*l .. b*l + l) (on entry the columns of X); V: identity
// on entry.  On exit W = X V with orthogonal columns.  Must be called by all
// NT threads of the CTA.  `flag` is a shared int.
template <int NT>
__device__ void jacobi_dd(dd* W, dd* V, int l, int* flag) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int np = (l + 1) & ~1;
  const double tol = (double)l * 3.6e-15;  // about l * 2^-48
  const int gl = lane & 7, ngroups = (NT / 32) * 4;
  for (int sweep = 0; sweep < 60; ++sweep) {
    if (tid == 0) *flag = 0;
    __syncthreads();
    for (int round = 0; round < np - 1; ++round) {
      for (int base = warp * 4; base < np / 2; base += ngroups) {
        const int slot = base + (lane >> 3);
        const int x0 = slot, x1 = np - 1 - slot;
        int p = (x0 == 0) ? 0 : ((x0 - 1 + round) % (np - 1)) + 1;
        int q = (x1 == 0) ? 0 : ((x1 - 1 + round) % (np - 1)) + 1;
        if (p > q) { const int t = p; p = q; q = t; }
        const bool act = slot < np / 2 && q < l;
        dd* wp = W + p * l;
        dd* wq = W + q * l;
        dd al{0.f, 0.f}, be{0.f, 0.f}, ga{0.f, 0.f};
        if (act)
          for (int i = gl; i < l; i += 8) {
            const dd u = wp[i], v = wq[i];
            al = dd_fma(u, u, al);
            be = dd_fma(v, v, be);
            ga = dd_fma(u, v, ga);
          }
#pragma unroll
        for (int off = 4; off > 0; off >>= 1) {
          al = dd_add(al, dd{__shfl_xor_sync(0xffffffffu, al.hi, off), __shfl_xor_sync(0xffffffffu, al.lo, off)});
          be = dd_add(be, dd{__shfl_xor_sync(0xffffffffu, be.hi, off), __shfl_xor_sync(0xffffffffu, be.lo, off)});
          ga = dd_add(ga, dd{__shfl_xor_sync(0xffffffffu, ga.hi, off), __shfl_xor_sync(0xffffffffu, ga.lo, off)});
        }
        if (!act) continue;
        const double a2 = dd_to_double(al), b2 = dd_to_double(be), g2 = dd_to_double(ga);
        if (a2 == 0.0 || b2 == 0.0 || g2 * g2 <= tol * tol * a2 * b2) continue;
        const float zeta = dd_add(be, dd_neg(al)).hi / (2.0f * ga.hi);
        const float tf = fabsf(zeta) > 1e18f
                             ? 0.5f / zeta
                             : (zeta >= 0.0f ? 1.0f : -1.0f) / (fabsf(zeta) + sqrtf(fmaf(zeta, zeta, 1.0f)));
        const dd x = dd_add(dd_make(1.0f), two_sum(__fmul_rn(tf, tf), fmaf(tf, tf, -__fmul_rn(tf, tf))));
        const dd c = dd_rsqrt_1_2(x);
        const dd s = dd_mul(c, dd_make(tf));
        const dd ns = dd_neg(s);
        dd* vp = V + p * l;
        dd* vq = V + q * l;
        for (int i = gl; i < l; i += 8) {
          const dd u = wp[i], v = wq[i];
          wp[i] = dd_fma(c, u, dd_mul(ns, v));
          wq[i] = dd_fma(s, u, dd_mul(c, v));
          const dd xx = vp[i], yy = vq[i];
          vp[i] = dd_fma(c, xx, dd_mul(ns, yy));
          vq[i] = dd_fma(s, xx, dd_mul(c, yy));
        }
        if (gl == 0) *flag = 1;
      }
      __syncthreads();
    }
    if (*flag == 0) break;
    __syncthreads();
  }
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

// U[p][q] = sum_{r < ke} V[b_r][p] W[b_r][q] / sigma_r^2 in double-float;
// inv2[r] = 1 / sigma_{b_r}^2 (shared, computed once); out(e, value)
// receives the l*l entries (row-major index e = p*l + q).
template <int NT, typename Out>
__device__ void nucleus_from_svd(const dd* W, const dd* V, int l, int ke, const int* order,
                                 const dd* inv2, Out out) {
  for (int e = threadIdx.x; e < l * l; e += NT) {
    const int p = e / l, q = e - p * l;
    dd acc{0.f, 0.f};
    for (int r = 0; r < ke; ++r) {
      const int b = order[r];
      acc = dd_fma(dd_mul(V[b * l + p], W[b * l + q]), inv2[r], acc);
    }
    out(e, dd_to_double(acc));
  }
}

}  // namespace lra
