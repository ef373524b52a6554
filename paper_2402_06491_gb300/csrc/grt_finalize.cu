// grt_finalize.cu -- per-point reduction of the item partials, series
// coefficients and standard errors (Sec. 2.4, Eq. simplecase_discrete), and
// the FP64 [L/M] Pade approximant at eps = 1 (Sec. 2.1 end, Sec. 2.4).
#include "grt_device.cuh"
#include "grt_launch.h"

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
// c_n = a_n / rho^n with rho = (|a_{L+M}| / |a_0|)^{1/(L+M)}, which leaves the
// approximant unchanged (evaluated at w = rho) and balances the Toeplitz
// system  sum_{j=1..M} c_{L+i-j} beta_j = -c_{L+i}, i = 1..M.  Gaussian
// elimination with partial pivoting; a pivot at or below 1e-14 times the
// largest entry lowers the type to [L-1/M-1] (L not below 0) and sets
// PADE_SINGULAR.  |Q(1)| < 1e-8 sets PADE_POLE_NEAR.
__device__ double pade_value(const double *a, int L, int M, int *status) {
  const int n = L + M;
  double rho = 1.0;
  if (n > 0 && a[0] != 0.0 && a[n] != 0.0) rho = pow(fabs(a[n]) / fabs(a[0]), 1.0 / (double)n);
  double c[kMaxK + 1];
  for (int i = 0; i <= n; ++i) c[i] = a[i] / pow(rho, (double)i);

  int st = 0;
  int Lc = L, Mc = M;
  double beta[kMaxK + 1];
  beta[0] = 1.0;
  while (Mc > 0) {
    double T[kMaxK][kMaxK + 1];  // row r: coefficients of beta_1..beta_Mc, then the right side
    double big = 0.0;
    for (int r = 0; r < Mc; ++r) {
      for (int k = 0; k < Mc; ++k) {
        const int idx = Lc + r - k;  // c_{L+i-j} with i = r+1, j = k+1
        const double v = idx >= 0 ? c[idx] : 0.0;
        T[r][k] = v;
        big = fmax(big, fabs(v));
      }
      T[r][Mc] = -c[Lc + r + 1];
    }
    bool ok = big > 0.0;
    for (int k = 0; k < Mc && ok; ++k) {
      int pr = k;
      double pv = fabs(T[k][k]);
      for (int r = k + 1; r < Mc; ++r) {
        const double v = fabs(T[r][k]);
        if (v > pv) {
          pv = v;
          pr = r;
        }
      }
      if (pv <= 1e-14 * big) {
        ok = false;
        break;
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
        if (m != 0.0)
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

// One warp per point.  Lane o (o <= K) adds S1, S2, S|W| of order o over the
// point's items in item order with Kahan compensation; lanes o <= K+2 add the
// counts (orders, pruned trees, nodes).
template <typename Acc>
__global__ void __launch_bounds__(32) finalize_kernel(const FinalizeParams f) {
  const int pt = blockIdx.x;
  const int lane = threadIdx.x;
  const int K = f.K;
  const uint32_t i0 = f.prefix[pt], i1 = f.prefix[pt + 1];
  const int pstride = 3 * (K + 1), cstride = K + 3;
  const Acc *part = reinterpret_cast<const Acc *>(f.part);
  Acc s1 = 0, c1 = 0, s2 = 0, c2 = 0, sa = 0, ca = 0;
  unsigned long long cn = 0;
  for (uint32_t it = i0; it < i1; ++it) {
    if (lane <= K) {
      const Acc *pp = part + (size_t)it * pstride;
      kahan_add(s1, c1, pp[lane]);
      kahan_add(s2, c2, pp[K + 1 + lane]);
      kahan_add(sa, ca, pp[2 * (K + 1) + lane]);
    }
    if (lane <= K + 2) cn += f.cnt[(size_t)it * cstride + lane];
  }
  __shared__ double a[kMaxK + 1];
  __shared__ unsigned long long pruned;
  const double N = (double)f.ntrees[pt];
  if (lane <= K) {
    const double S1 = (double)s1, S2 = (double)s2;
    const double an = N > 0.0 ? S1 / N : 0.0;
    const double var = N > 1.0 ? (S2 / N - an * an) / (N - 1.0) : 0.0;
    a[lane] = an;
    if (f.coef) f.coef[(size_t)pt * (K + 1) + lane] = an;
    if (f.se) f.se[(size_t)pt * (K + 1) + lane] = var > 0.0 ? sqrt(var) : 0.0;
  }
  if (lane == K + 1) {
    pruned = cn;
    if (f.pruned_pt) f.pruned_pt[pt] = cn;
  }
  if (lane == K + 2 && f.nodes_pt) f.nodes_pt[pt] = cn;
  // splitting events: n per kept tree of order n, K+1 per pruned tree
  unsigned long long sp = lane <= K + 1 ? (unsigned long long)lane * cn : 0ull;
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) sp += __shfl_xor_sync(kFull, sp, off);
  if (lane == 0 && f.splits_pt) f.splits_pt[pt] = sp;
  __syncwarp();
  if (lane == 0) {
    int st = 0;
    const double u = pade_value(a, f.L, f.M, &st);
    if (N > 0.0 && (double)pruned > 0.01 * N) st |= 8;  // HIGH_PRUNE
    f.u[pt] = u;
    if (f.status) f.status[pt] = st;
    if (pt == 0) *f.counter = 0u;  // the walk kernel that used it has finished
  }
}

__global__ void pade_kernel(int n, int K, int L, int M, const double *coef, double *u, int32_t *status) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double a[kMaxK + 1];
  for (int j = 0; j <= L + M; ++j) a[j] = coef[(size_t)i * (K + 1) + j];
  int st = 0;
  u[i] = pade_value(a, L, M, &st);
  if (status) status[i] = st;
}

cudaError_t launch_finalize(bool fp64, const FinalizeParams &f, cudaStream_t stream) {
  if (f.n <= 0) return cudaSuccess;
  if (fp64) finalize_kernel<double><<<f.n, 32, 0, stream>>>(f);
  else finalize_kernel<float><<<f.n, 32, 0, stream>>>(f);
  return cudaGetLastError();
}

cudaError_t launch_pade(int n, int K, int L, int M, const double *coef, double *u, int32_t *status,
                        cudaStream_t stream) {
  if (n <= 0) return cudaSuccess;
  pade_kernel<<<(n + 127) / 128, 128, 0, stream>>>(n, K, L, M, coef, u, status);
  return cudaGetLastError();
}

}  // namespace grt
