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
// S(g, c): entry c of strip row g (read or evaluated by the caller).
template <int NT, int L = 0, typename StripF>
__device__ __forceinline__ bool invert_cross(StripF S, int l_arg, JobStatus* js, const int* pos, dd* A,
                                             const InvScratch& w) {
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
    const dd v = dd_make(S((long long)pos[r], c));
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

// The same elimination with a one-step look-ahead.  While warps 1.. form step
// t's result in the other buffer, warp 0 forms column t+1 of it, picks the
// pivot of step t+1 (the largest |hi| below row t, ties to the smaller row),
// and prepares that step's scaled pivot row and interchanged column t+1 (in
// the buffers of step t+1's parity).  One block barrier per step instead of
// two, and the pivot's division no longer sits between the updates.  A0
// holds X on entry; returns the buffer that holds the result (A0 for even
// l, A1 for odd), or nullptr where invert_cross returns false (same
// arithmetic, results and failure rules).  The scratch is taken by value
// (its pointers stay in registers).
struct InvLaScratch {
  dd* rowt;      // scaled pivot row of the step of parity b at rowt + b * stride (l)
  dd* colt;      // column t after the interchange, same layout (l)
  int stride;    // >= l
  int* swaps;    // pivot row of each step (l)
  int* at;       // column map of the result (l)
  int* pinfo;    // 2: pivot row of the step of that parity (-1: singular)
};

template <int NT, int L = 0>
__device__ __forceinline__ dd* invert_cross_la(const float* __restrict__ strip, long long si, long long st,
                                               int l_arg, JobStatus* js, const int* pos, dd* A0, dd* A1,
                                               const InvLaScratch w) {
  const int l = L > 0 ? L : l_arg;
  const int ll = l * l;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  constexpr int kW = NT - 32;                          // threads of warps 1..
  constexpr int kPer = (kMaxL * kMaxL + kW - 1) / kW;  // their entries each
  constexpr int kLn = (kMaxL + 31) / 32;               // a column's entries per lane of warp 0
  int bad = 0;
  for (int e = tid; e < ll; e += NT) {
    const int r = e / l, c = e - r * l;
    const dd v = dd_make(strip[(long long)pos[r] * si + (long long)c * st]);
    if (!(fabsf(v.hi) <= FLT_MAX)) bad = 1;
    A0[e] = v;
  }
  if (__syncthreads_or(bad)) {
    if (blockIdx.x == 0 && tid == 0) set_status(js, LRA_ENONFINITE);
    return nullptr;
  }
  // warp 0: given column tn of the matrix that step tn works on (col.v, one
  // entry per row r = lane + 32 u) and a way to read that matrix's rows,
  // choose the pivot among rows >= tn and prepare step tn
  struct Col {
    dd v[kLn];
  };
  auto prepare = [&](int tn, Col col, auto&& row_entry) {
    const dd* v = col.v;
    unsigned long long key = 0ull;
#pragma unroll
    for (int u = 0; u < kLn; ++u) {
      const int r = lane + 32 * u;
      if (r < l && r >= tn) {
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
    const int nb = tn & 1;
    if (p >= 0) {
      // the pivot value and the entry of row tn, from the lanes that hold them
      dd vp = dd_make(0.0f), vt = dd_make(0.0f);
#pragma unroll
      for (int u = 0; u < kLn; ++u) {
        if (u == p / 32) vp = v[u];
        if (u == tn / 32) vt = v[u];
      }
      vp = dd{__shfl_sync(0xffffffffu, vp.hi, p & 31), __shfl_sync(0xffffffffu, vp.lo, p & 31)};
      vt = dd{__shfl_sync(0xffffffffu, vt.hi, tn & 31), __shfl_sync(0xffffffffu, vt.lo, tn & 31)};
      const dd rp = dd_div(dd_make(1.0f), vp);
#pragma unroll
      for (int u = 0; u < kLn; ++u) {
        const int c = lane + 32 * u;
        if (c < l) {
          w.rowt[nb * w.stride + c] = (c == tn) ? rp : dd_mul(row_entry(p, c), rp);
          w.colt[nb * w.stride + c] = (c == p) ? vt : v[u];   // c indexes rows here
        }
      }
    }
    if (lane == 0) {
      w.pinfo[nb] = p;
      if (p >= 0) w.swaps[tn] = p;
    }
  };
  if (warp == 0) {
    Col col;
#pragma unroll
    for (int u = 0; u < kLn; ++u) {
      const int r = lane + 32 * u;
      col.v[u] = r < l ? A0[r * l] : dd_make(0.0f);
    }
    prepare(0, col, [&](int r, int c) { return A0[r * l + c]; });
  }
  __syncthreads();
  dd* cur = A0;
  dd* nxt = A1;
  for (int t = 0; t < l; ++t) {
    const int pb = t & 1;
    const int p = w.pinfo[pb];
    if (p < 0) {
      if (blockIdx.x == 0 && tid == 0) set_status(js, LRA_ESINGULAR);
      return nullptr;
    }
    const dd* rowt = w.rowt + pb * w.stride;
    const dd* colt = w.colt + pb * w.stride;
    // entry (r, c) of the matrix after step t
    auto entry = [&](int r, int c) -> dd {
      if (r == t) return rowt[c];
      const dd av = (c == t) ? dd_make(0.0f) : cur[(r == p ? t : r) * l + c];
      return dd_fnma(colt[r], rowt[c], av);
    };
    const bool ahead = t + 1 < l;
    if (warp == 0) {
      if (ahead) {
        Col col;
#pragma unroll
        for (int u = 0; u < kLn; ++u) {
          const int r = lane + 32 * u;
          col.v[u] = dd_make(0.0f);
          if (r < l) {
            col.v[u] = entry(r, t + 1);
            nxt[r * l + t + 1] = col.v[u];
          }
        }
        prepare(t + 1, col, entry);
      }
    } else {
      // entry coordinates recomputed per step (a division by the
      // compile-time l is a multiply and a shift)
#pragma unroll
      for (int k = 0; k < kPer; ++k) {
        const int e = (tid - 32) + k * kW;
        if (e < ll) {
          const int r = e / l, c = e - r * l;
          if (!(ahead && c == t + 1)) nxt[e] = entry(r, c);   // column t+1 is warp 0's
        }
      }
    }
    __syncthreads();
    dd* tmp = cur;
    cur = nxt;
    nxt = tmp;
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
  return cur;
}

}  // namespace lra
