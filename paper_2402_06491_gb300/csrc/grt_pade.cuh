// grt_pade.cuh -- FP64 [L/M] Pade approximant of the series of per-order
// coefficients at eps = 1 (Sec. 2.1 end, Sec. 2.4) and compensated addition,
// shared by the binning kernel, the stand-alone Pade kernels and the plain
// one-launch-per-point FP64 path.
#pragma once

#include <climits>
#include <cstdint>
#include <cuda_runtime.h>

#include "grt_device.cuh"

namespace grt {

// Compensated (Kahan) addition; the explicit round-to-nearest intrinsics keep
// the compiler from reassociating the correction away.
__device__ __forceinline__ void kahan_add(float &s, float &c, float v) {
  const float y = __fsub_rn(v, c);
  const float t = __fadd_rn(s, y);
  c = __fsub_rn(__fsub_rn(t, s), y);
  s = t;
}
__device__ __forceinline__ void kahan_add(double &s, double &c, double v) {
  const double y = __dsub_rn(v, c);
  const double t = __dadd_rn(s, y);
  c = __dsub_rn(__dsub_rn(t, s), y);
  s = t;
}

// [L/M] Pade of sum a_n eps^n at eps = 1.  The series is first rescaled,
// c_n = a_n / rho^n with rho = 2^k, k = max_{j > m} ceil((e_j - e_m)/(j - m)),
// e_j the binary exponent of a_j and m the first nonzero term: this leaves the
// approximant unchanged (evaluated at w = rho), is exact in floating point,
// needs no transcendental function, and keeps every |c_j| within a factor of
// two of |c_m| or below in the Toeplitz system
// sum_{j=1..M} c_{L+i-j} beta_j = -c_{L+i}, i = 1..M.  Gaussian
// elimination with partial pivoting; a pivot at or below 1e-14 times the
// largest entry lowers the type to [L-1/M-1] (L not below 0) and sets
// PADE_SINGULAR.  |Q(1)| < 1e-8 sets PADE_POLE_NEAR.

// Integer forms of the Pade's comparisons and exponent steps (FP64 instructions are the
// evaluation's cost on this GPU): |v| compared through its bit pattern, which orders like |v|;
// ilogb and scalbn by the exponent field for normal numbers (exact), the library routines
// otherwise.  Every decision and value is the same as with the FP64 forms.
__device__ __forceinline__ uint64_t pd_abs_bits(double v) {
  return (uint64_t)__double_as_longlong(v) & 0x7FFFFFFFFFFFFFFFull;
}
// |v| as an integer key ordered like |v|; NaN -> 0 (loses every strict comparison, as in FP64)
__device__ __forceinline__ uint64_t pd_key(double v) {
  const uint64_t b = pd_abs_bits(v);
  return b > 0x7FF0000000000000ull ? 0ull : b;
}
__device__ __forceinline__ int pd_ilogb(double v) {
  const int e = (int)(((uint64_t)__double_as_longlong(v) >> 52) & 0x7FF);
  return (e == 0 || e == 0x7FF) ? ilogb(v) : e - 1023;
}
__device__ __forceinline__ double pd_scalbn(double v, int n) {
  const uint64_t b = (uint64_t)__double_as_longlong(v);
  const int e = (int)((b >> 52) & 0x7FF);
  if (e == 0 || e == 0x7FF || e + n <= 0 || e + n >= 0x7FF) return scalbn(v, n);
  return __longlong_as_double((long long)(b + ((uint64_t)(int64_t)n << 52)));
}
__device__ inline double pade_value(const double *a, int L, int M, int *status) {
  const int n = L + M;
  // growth rate of the series by the root test on its binary exponents,
  // rounded up to an integer: rho = 2^k, so the rescaling below is exact
  int first = 0;
  while (first <= n && pd_abs_bits(a[first]) == 0) ++first;
  int k = 0;
  bool any = false;
  for (int j = first + 1; j <= n; ++j) {
    if (pd_abs_bits(a[j]) == 0) continue;
    const int num = pd_ilogb(a[j]) - pd_ilogb(a[first]), den = j - first;
    const int q = num > 0 ? (num + den - 1) / den : -((-num) / den);  // ceil(num / den)
    k = any ? max(k, q) : q;
    any = true;
  }
  const double rho = scalbn(1.0, k);
  double c[kMaxK + 1];
  for (int i = 0; i <= n; ++i) c[i] = pd_scalbn(a[i], -k * i);

  int st = 0;
  int Lc = L, Mc = M;
  double beta[kMaxK + 1];
  beta[0] = 1.0;
  while (Mc > 0) {
    double T[kMaxK][kMaxK + 1];  // row r: coefficients of beta_1..beta_Mc, then the right side
    uint64_t bigk = 0;
    for (int r = 0; r < Mc; ++r) {
      for (int k = 0; k < Mc; ++k) {
        const int idx = Lc + r - k;  // c_{L+i-j} with i = r+1, j = k+1
        const double v = idx >= 0 ? c[idx] : 0.0;
        T[r][k] = v;
        bigk = max(bigk, pd_key(v));
      }
      T[r][Mc] = -c[Lc + r + 1];
    }
    bool ok = bigk > 0;
    const uint64_t tiny = pd_key(1e-14 * __longlong_as_double((long long)bigk));
    for (int k = 0; k < Mc && ok; ++k) {
      int pr = k;
      const uint64_t b0 = pd_abs_bits(T[k][k]);
      if (b0 <= 0x7FF0000000000000ull) {  // a NaN pivot candidate keeps its row, as the FP64 scan does
        uint64_t pvk = b0;
        for (int r = k + 1; r < Mc; ++r) {
          const uint64_t vk = pd_key(T[r][k]);
          if (vk > pvk) {
            pvk = vk;
            pr = r;
          }
        }
        if (pvk <= tiny) {
          ok = false;
          break;
        }
      }
      if (pr != k) {
        for (int j = k; j <= Mc; ++j) {
          const double tmp = T[k][j];
          T[k][j] = T[pr][j];
          T[pr][j] = tmp;
        }
      }
      const double inv = 1.0 / T[k][k];
      for (int r = k + 1; r < Mc; ++r) {
        const double m = T[r][k] * inv;
        if (pd_abs_bits(m) != 0)
          for (int j = k; j <= Mc; ++j) T[r][j] -= m * T[k][j];
      }
    }
    if (ok) {
      for (int r = Mc - 1; r >= 0; --r) {
        double s = T[r][Mc];
        for (int j = r + 1; j < Mc; ++j) s -= T[r][j] * beta[j + 1];
        beta[r + 1] = s / T[r][r];
      }
      break;
    }
    st |= 1;  // PADE_SINGULAR
    --Mc;
    if (Lc > 0) --Lc;
  }
  // Q(rho) and P(rho) by Horner; numerator coefficients alpha_i = sum_j beta_j c_{i-j}
  double Q = 0.0;
  for (int j = Mc; j >= 0; --j) Q = Q * rho + beta[j];
  double P = 0.0;
  for (int i = Lc; i >= 0; --i) {
    double al = 0.0;
    const int jm = i < Mc ? i : Mc;
    for (int j = 0; j <= jm; ++j) al += beta[j] * c[i - j];
    P = P * rho + al;
  }
  if (fabs(Q) < 1e-8) st |= 2;  // PADE_POLE_NEAR
  *status = st;
  return P / Q;
}

// The same [L/M] Pade, evaluated by all 32 lanes of a warp together (every lane gets the value and
// the status).  Lane r + 16 h holds row r of the Toeplitz system, columns 9h .. 9h+8 (M <= 16 rows,
// M + 1 <= 17 columns); an elimination step broadcasts the pivot row and each row's multiplier by
// shuffles, so its depth is one update instead of M - k of them.  The pivot search, the singularity
// rule, the back substitution and Horner read the same values in the same order as pade_value (every
// lane reads them through shuffles from the lanes that hold them) and apply the same operations.
// `a` [L+M+1] must be readable by every lane (shared memory).
__device__ inline double pade_value_warp(const double *a, int L, int M, int *status, int lane) {
  const int n = L + M;
  const int r = lane & 15, h = lane >> 4;
  // rescaling: the root test on the binary exponents, as in pade_value
  const bool nz = lane <= n && pd_abs_bits(a[lane <= n ? lane : 0]) != 0;
  const unsigned nzm = __ballot_sync(kFull, nz);
  const int first = nzm ? __ffs((int)nzm) - 1 : n + 1;
  int q = INT_MIN;
  if (nz && lane > first) {
    const int num = pd_ilogb(a[lane]) - pd_ilogb(a[first]), den = lane - first;
    q = num > 0 ? (num + den - 1) / den : -((-num) / den);
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) q = max(q, __shfl_xor_sync(kFull, q, off));
  const int k = q == INT_MIN ? 0 : q;
  const double rho = scalbn(1.0, k);
  const double cl = lane <= n ? pd_scalbn(a[lane], -k * lane) : 0.0;  // c_lane
  auto c_at = [&](int i) { return __shfl_sync(kFull, cl, i & 31); };  // c_i in every lane (uniform i)

  int st = 0;
  int Lc = L, Mc = M;
  double beta[kMaxK + 1];
  beta[0] = 1.0;
  while (Mc > 0) {
    double T[9];  // T[r][9h + e]
    uint64_t bigk = 0;
#pragma unroll
    for (int e = 0; e < 9; ++e) {
      const int j = 9 * h + e;
      const int idx = j < Mc ? Lc + r - j : Lc + r + 1;
      const double v = __shfl_sync(kFull, cl, idx < 0 ? 0 : (idx & 31));
      double t = 0.0;
      if (r < Mc && j < Mc) t = idx >= 0 ? v : 0.0;
      if (r < Mc && j == Mc) t = -v;
      T[e] = t;
      if (r < Mc && j < Mc) bigk = max(bigk, pd_key(t));
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) bigk = max(bigk, (uint64_t)__shfl_xor_sync(kFull, (unsigned long long)bigk, off));
    bool ok = bigk > 0;
    const uint64_t tiny = pd_key(1e-14 * __longlong_as_double((long long)bigk));
    auto elem = [&](int col) {  // this lane's T[r][col] (col in its half)
      double v = T[0];
#pragma unroll
      for (int e = 1; e < 9; ++e)
        if (e == col % 9) v = T[e];
      return v;
    };
    for (int kk = 0; kk < Mc && ok; ++kk) {
      const int hk = kk / 9;
      const double colk = elem(kk);
      // pivot search on column kk, rows kk .. Mc-1, in row order (every lane scans the same values)
      int pr = kk;
      const uint64_t b0 = pd_abs_bits(__shfl_sync(kFull, colk, kk + 16 * hk));
      if (b0 <= 0x7FF0000000000000ull) {  // a NaN pivot candidate keeps its row
        uint64_t pvk = b0;
        for (int rr = kk + 1; rr < Mc; ++rr) {
          const uint64_t vk = pd_key(__shfl_sync(kFull, colk, rr + 16 * hk));
          if (vk > pvk) {
            pvk = vk;
            pr = rr;
          }
        }
        if (pvk <= tiny) {
          ok = false;
          break;
        }
      }
      if (pr != kk) {  // swap rows kk and pr (whole rows: the entries left of kk are not read again)
        const int src = (r == kk ? pr : (r == pr ? kk : r)) + 16 * h;
#pragma unroll
        for (int e = 0; e < 9; ++e) T[e] = __shfl_sync(kFull, T[e], src);
      }
      const double inv = 1.0 / __shfl_sync(kFull, elem(kk), kk + 16 * hk);
      const double mine = elem(kk) * inv;             // the multiplier of this lane's row, in half hk
      const double m = __shfl_sync(kFull, mine, r + 16 * hk);
      double tk[9];                                   // the pivot row's entries of this half
#pragma unroll
      for (int e = 0; e < 9; ++e) tk[e] = __shfl_sync(kFull, T[e], kk + 16 * h);
      if (r > kk && r < Mc && pd_abs_bits(m) != 0) {
#pragma unroll
        for (int e = 0; e < 9; ++e) {
          const int j = 9 * h + e;
          if (j >= kk && j <= Mc) T[e] -= m * tk[e];
        }
      }
    }
    if (ok) {
      for (int rr = Mc - 1; rr >= 0; --rr) {
        double sv = __shfl_sync(kFull, elem(Mc), rr + 16 * (Mc / 9));
        for (int j = rr + 1; j < Mc; ++j) sv -= __shfl_sync(kFull, elem(j), rr + 16 * (j / 9)) * beta[j + 1];
        beta[rr + 1] = sv / __shfl_sync(kFull, elem(rr), rr + 16 * (rr / 9));
      }
      break;
    }
    st |= 1;  // PADE_SINGULAR
    --Mc;
    if (Lc > 0) --Lc;
  }
  double Q = 0.0;
  for (int j = Mc; j >= 0; --j) Q = Q * rho + beta[j];
  double P = 0.0;
  for (int i = Lc; i >= 0; --i) {
    double al = 0.0;
    const int jm = i < Mc ? i : Mc;
    for (int j = 0; j <= jm; ++j) al += beta[j] * c_at(i - j);
    P = P * rho + al;
  }
  if (fabs(Q) < 1e-8) st |= 2;  // PADE_POLE_NEAR
  *status = st;
  return P / Q;
}

}  // namespace grt
