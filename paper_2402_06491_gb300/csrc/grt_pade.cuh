// grt_pade.cuh -- FP64 [L/M] Pade approximant of the series of per-order
// coefficients at eps = 1 (Sec. 2.1 end, Sec. 2.4) and compensated addition,
// shared by the binning kernel, the stand-alone Pade kernels and the plain
// one-launch-per-point FP64 path.
#pragma once

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

}  // namespace grt
