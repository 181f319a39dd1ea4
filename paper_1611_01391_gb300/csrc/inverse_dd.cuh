// Cross inverse in double-float arithmetic on one CTA (the pairs of
// dd_arith.cuh carry about 48 significant bits, at the FP32 issue rate).
// Used by the maxvol kernel (every CTA inverts the cross for itself) and by
// the separate cross inverse kernel.
#pragma once

#include <cfloat>

#include "dd_arith.cuh"
#include "lra_internal.cuh"

namespace lra {

// Scratch of the in-kernel cross inverse (shared memory).
struct InvScratch {
  dd* rowt;                 // pivot row scaled by 1 / pivot (l)
  dd* colt;                 // column t before the step, after the interchange (l)
  dd* rowold;               // row t before the step (l)
  unsigned long long* pkey; // the next pivot's word, two steps deep
  int* swaps;               // pivot row of each step (l)
  int* at;                  // column map of the result (l)
  int* p_s;
};

__device__ __forceinline__ unsigned long long pivot_word(dd v, int r) {
  return ((unsigned long long)(__float_as_uint(v.hi) & 0x7fffffffu) << 32) | (0xffffffffu - (unsigned int)r);
}

// Inverse of the cross X = S[pos, :] of an N x l strip (element (i, t) at
// strip[i*si + t*st]) in double-float pairs, by one CTA: in-place
// Gauss-Jordan elimination (Golub & Van Loan, 3.4; l^3 multiply-adds) with partial pivoting on the rows (the pivot of
// step t+1 is found by a shared atomic max while step t updates column t+1;
// |hi| rounded to FP32 orders the candidates, ties to the smaller row).  A
// step interchanges rows t and p, scales the pivot row by 1/pivot and
// subtracts its multiples from every other row, column t taking the place
// of the eliminated unit column; the interchanges are undone at the end as
// a column map (X^{-1}[:, q] = A[:, at[q]]).  Every thread of the CTA calls
// it.  Returns false, with the job's status set by CTA 0 of the launch, on
// a non-finite or singular cross.
// NT = blockDim.x: each thread keeps the coordinates of its <= ceil(96^2 /
// NT) entries in registers for all steps.
// L > 0: a build for l == L exactly.
template <int NT, int L = 0>
__device__ __forceinline__ bool invert_cross(const float* __restrict__ strip, long long si, long long st, int l_arg,
                                    JobStatus* js, const int* pos, dd* A, const InvScratch& w) {
  const int l = L > 0 ? L : l_arg;
  constexpr int kPer = (kMaxL * kMaxL + NT - 1) / NT;
  const int ll = l * l;
  const int tid = threadIdx.x, nthr = NT, lane = tid & 31;
  int er[kPer], ec[kPer];
#pragma unroll
  for (int k = 0; k < kPer; ++k) {
    const int e = tid + k * NT;
    er[k] = e < ll ? e / l : -1;
    ec[k] = e < ll ? e - (e / l) * l : 0;
  }
  if (tid < 2) w.pkey[tid] = 0ull;
  __syncthreads();
  int bad = 0;
  for (int e = tid; e < ll; e += nthr) {
    const int r = e / l, c = e - r * l;
    const dd v = dd_make(strip[(long long)pos[r] * si + (long long)c * st]);
    if (!(fabsf(v.hi) <= FLT_MAX)) bad = 1;
    A[e] = v;
    if (c == 0) atomicMax(w.pkey, pivot_word(v, r));
  }
  if (__syncthreads_or(bad)) {
    if (blockIdx.x == 0 && tid == 0) set_status(js, LRA_ENONFINITE);
    return false;
  }
  for (int t = 0; t < l; ++t) {
    if (tid < 32) {
      const unsigned long long key = w.pkey[t & 1];
      const int p = (key >> 32) != 0ull ? (int)(0xffffffffu - (unsigned int)key) : -1;
      if (p >= 0) {
        const dd rp = dd_div(dd_make(1.0f), A[p * l + t]);
        for (int c = lane; c < l; c += 32) {
          w.rowt[c] = (c == t) ? rp : dd_mul(A[p * l + c], rp);
          w.rowold[c] = A[t * l + c];
          w.colt[c] = A[(c == p ? t : c) * l + t];
        }
      }
      if (lane == 0) {
        *w.p_s = p;
        w.swaps[t] = p;
        w.pkey[(t + 1) & 1] = 0ull;
      }
    }
    __syncthreads();
    const int p = *w.p_s;
    if (p < 0) {
      if (blockIdx.x == 0 && tid == 0) set_status(js, LRA_ESINGULAR);
      return false;
    }
#pragma unroll
    for (int k = 0; k < kPer; ++k) {
      const int r = er[k], c = ec[k];
      if (r < 0) break;   // this thread's entries end here
      const int e = r * l + c;
      dd v;
      if (r == t) {
        v = w.rowt[c];
      } else {
        // row r after the interchange is row t before it when r == p
        const dd av = (c == t) ? dd_make(0.0f) : (r == p ? w.rowold[c] : A[e]);
        v = dd_fnma(w.colt[r], w.rowt[c], av);
      }
      A[e] = v;
      if (c == t + 1 && r > t) atomicMax(&w.pkey[(t + 1) & 1], pivot_word(v, r));
    }
    __syncthreads();
  }
  if (tid == 0) {
    for (int q = 0; q < l; ++q) w.at[q] = q;
    for (int t = l - 1; t >= 0; --t) {
      const int p = w.swaps[t], x = w.at[t];
      w.at[t] = w.at[p];
      w.at[p] = x;
    }
  }
  __syncthreads();
  return true;
}

}  // namespace lra
