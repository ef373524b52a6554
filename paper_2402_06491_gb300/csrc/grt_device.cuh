// grt_device.cuh -- device-side building blocks of the random-tree walk.
//
// One node of a generalized random tree (Sec. 2.1 algorithm / Fig. 1 for
// Strategy A, Sec. 2.2 Eqs. probexpB1-probexpBclosed for Strategy B):
//   draw the node's Philox words, sample its Brownian segment exactly
//   (variance 2 D s per axis: Eqs. green, SDE with sigma^2 = 2D), decide
//   leaf / split, and return the factor it multiplies into the tree weight.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace grt {

constexpr int kMaxTerms = 16;     // powers 0..15 of f
constexpr int kMaxK = 16;         // highest series order
constexpr int kTile = 512;        // default trees per work-queue chunk
constexpr int kFinThreads = 64;   // threads of a finalize (binning) block
constexpr int kBinChunk = 8192;   // tree records binned by one finalize block
constexpr unsigned kFull = 0xFFFFFFFFu;

enum : int { kU0Const = 0, kU0Gauss = 1, kU0CosProd = 2, kU0TanhProd = 3, kU0Logistic = 4, kU0GaussAxes = 5,
             kU0Quadratic = 6 };
enum : int { kSdeHeat = 0, kSdeAffine = 1 };
// compile-time features of a walk instantiation
enum : int { kFeatEuler = 1, kFeatVarCoef = 2 };
enum : int { kCoefConst = 0, kCoefGaussOverT = 1, kCoefGauss = 2 };
enum : int { kStratA = 0, kStratB = 1 };

// Everything one walk launch needs, passed by value (constant bank).
struct WalkParams {
  // branching law
  int ncat_thr;              // number of finite thresholds used by the first categorical draw
  uint32_t thr[kMaxTerms + 1];
  int nterms;
  int arity[kMaxTerms];
  double term_factor[kMaxTerms];  // B: b_k / P(k);  A: b_k / (lambda P(k))
  double leaf_factor;             // B: 1 / P(leaf)
  float leaf_factorf;             // the same in binary32 (the FP32 walk converts nothing per node)
  // problem scalars
  int u0_kind;
  int K;
  double two_D;
  double inv_lambda;   // A
  double lam_minus_c;  // A
  double u0d[8];       // u0 constants (see make_u0_constants on the host)
  float u0f[8];
  float two_Df, inv_lambdaf, lam_minus_cf;
  // variable coefficients c_k(x, t) = b_k gamma(x, t) (kCoef*): gamma multiplies the
  // split factor of the categories in coef_cat_mask (bit = term index)
  int coef_kind;
  uint32_t coef_cat_mask;
  double cwd[3], cmd[3], ct0d;  // -w_i, centre m_i, t0
  float cwf[3], ct0f;           // -w_i log2 e, t0
  // path law: kSdeHeat (exact Gaussian segments) or kSdeAffine (Euler-Maruyama,
  // sde_steps steps per segment, per-axis beta, kappa, s, r)
  int sde_kind, sde_steps;
  double sded[12];
  float sdef[12];
  // Philox round keys: round r uses (k0 + r W0, k1 + r W1)
  uint32_t rk0[10], rk1[10];
  uint32_t point_base;
  // data
  const double *x;           // [n][dim]
  const double *t;           // [n]
  const uint32_t *ntrees;    // [n]
  const uint32_t *prefix;    // [n+1] first queue chunk of each point
  const unsigned long long *tree_prefix;  // [n+1] first record slot of each point (4-aligned segments)
  const uint32_t *tree_first;  // [n] first tree index walked for each point, or null (0): incremental solves
  const uint32_t *point_id;    // [n] random-stream point index of each point, or null (point_base + p)
  int n;
  uint32_t tile;             // trees per queue chunk
  uint32_t tile_small;       // trees per queue chunk of points small_from .. n-1 (0: every point uses tile)
  int small_from;
  uint32_t total_items;      // queue chunks: this launch takes items item_base .. total_items - 1
  uint32_t item_base;
  unsigned long long rec_base;  // record slot of rec_w[0] / rec_o[0] (the pointers are offset by it):
                                // a launch's records span fewer than 2^32 slots
  void *rec_w;               // [total trees] tree weights (float or double)
  uint8_t *rec_o;            // [total trees] tree orders (K+1 = pruned)
  unsigned long long *stats; // [0] nodes visited (added by the walk), [1] splits, [2] pruned trees (the binning)
  uint32_t *counter;         // work-queue head
};

// The compile-time features a problem needs (Euler paths, variable coefficients).
__host__ __device__ inline int walk_features(const WalkParams &p) {
  return (p.sde_kind == kSdeAffine ? kFeatEuler : 0) | (p.coef_kind != kCoefConst ? kFeatVarCoef : 0);
}

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11).  Each round multiplies
// words 0 and 2 by the two round constants (32x32 -> 64 bit), and the key of
// round r is the launch key advanced r times by the Weyl constants.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, const uint32_t (&rk0)[10], const uint32_t (&rk1)[10]) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)c.x;
    const uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)c.z;
    c = make_uint4((uint32_t)(p1 >> 32) ^ c.y ^ rk0[r], (uint32_t)p1, (uint32_t)(p0 >> 32) ^ c.w ^ rk1[r],
                   (uint32_t)p0);
  }
  return c;
}

// The same generator under a key given at the call (round keys formed on the fly).
__device__ __forceinline__ uint4 philox4x32_10_key(uint4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)c.x;
    const uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)c.z;
    c = make_uint4((uint32_t)(p1 >> 32) ^ c.y ^ k0, (uint32_t)p1, (uint32_t)(p0 >> 32) ^ c.w ^ k1, (uint32_t)p0);
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  return c;
}

// U(w) = ((w >> 9) + 1/2) 2^-23 in (0,1).  In binary32 it is formed exactly:
// the float 1 + (w>>9) 2^-23 minus (1 - 2^-24) is exact by Sterbenz' lemma.
template <typename Real> __device__ __forceinline__ Real uniform01(uint32_t w);
template <> __device__ __forceinline__ float uniform01<float>(uint32_t w) {
  return __fsub_rn(__uint_as_float(0x3F800000u | (w >> 9)), __uint_as_float(0x3F7FFFFFu));
}
template <> __device__ __forceinline__ double uniform01<double>(uint32_t w) {
  return __dadd_rn((double)(w >> 9), 0.5) * 0x1p-23;
}

template <typename Real> struct Math;
template <> struct Math<float> {
  static __device__ __forceinline__ float log(float v) { return logf(v); }
  static __device__ __forceinline__ float sqrt(float v) { return sqrtf(v); }
  static __device__ __forceinline__ float exp(float v) { return expf(v); }
  static __device__ __forceinline__ float cos(float v) { return cosf(v); }
  static __device__ __forceinline__ float tanh(float v) { return tanhf(v); }
  static __device__ __forceinline__ float abs(float v) { return fabsf(v); }
  static __device__ __forceinline__ void sincospi(float v, float *s, float *c) { sincospif(v, s, c); }
  static __device__ __forceinline__ float cospi(float v) { return cospif(v); }
};
template <> struct Math<double> {
  static __device__ __forceinline__ double log(double v) { return ::log(v); }
  static __device__ __forceinline__ double sqrt(double v) { return ::sqrt(v); }
  static __device__ __forceinline__ double exp(double v) { return ::exp(v); }
  static __device__ __forceinline__ double cos(double v) { return ::cos(v); }
  static __device__ __forceinline__ double tanh(double v) { return ::tanh(v); }
  static __device__ __forceinline__ double abs(double v) { return fabs(v); }
  static __device__ __forceinline__ void sincospi(double v, double *s, double *c) { ::sincospi(v, s, c); }
  static __device__ __forceinline__ double cospi(double v) { return ::cospi(v); }
};

// Node-body arithmetic.  The FP32 walk uses the special-function unit where
// its accuracy holds on the argument range:
//   sqrt(v)       = v * rsqrt(v), 0 for v = 0             (rsqrt.approx, ~2 ulp)
//   e^v           = 2^(v log2 e) by ex2.approx, the log2 e folded into the caller's constant
//   -2 ln U       = -2 ln 2 log2 U by lg2.approx for U <= 1/2, where |log2 U| >= 1 turns
//                   the SFU's small absolute error into a small relative one; for U > 1/2,
//                   where it would not, 4 atanh(z) with z = V / (2 - V), V = 1 - U (exact):
//                   -ln(1 - V) = 2 atanh(z), and z <= 1/3 makes the odd series to z^15
//                   exact to float precision (within 3.3 ulp over all 2^23 values of U)
// and sin / cos of 2 pi U an octant reduction on the bits of the Philox word
// with short near-minimax polynomials.  The FP64 walk uses the library functions.
template <typename Real> struct Node;
template <> struct Node<float> {
  static __device__ __forceinline__ float neg2ln(float u) {
    float l2;
    asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(l2) : "f"(u));
    const float lo = -1.38629436111989061883f * l2;  // -2 ln 2 log2 U
    const float v = 1.0f - u;                         // exact for U in (1/2, 1)
    const float d = 2.0f - v;
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(d));
    float z = v * r;
    z = fmaf(r, fmaf(-z, d, v), z);  // one residual correction of v / d
    const float z2 = z * z;
    float p = fmaf(z2, 1.0f / 15.0f, 1.0f / 13.0f);
    p = fmaf(z2, p, 1.0f / 11.0f);
    p = fmaf(z2, p, 1.0f / 9.0f);
    p = fmaf(z2, p, 1.0f / 7.0f);
    p = fmaf(z2, p, 1.0f / 5.0f);
    p = fmaf(z2, p, 1.0f / 3.0f);
    const float hi = 4.0f * fmaf(z * z2, p, z);  // 4 atanh z = 4 (z + z^3/3 + ... + z^15/15)
    return u <= 0.5f ? lo : hi;
  }
  // sin and cos of 2 pi U(w) from the bits of w: the top three bits pick the
  // octant, the next twenty the offset in it, so no floating-point range
  // reduction is needed.  With o = w >> 29 and rr the 20-bit offset (mirrored
  // in odd octants), v = (rr + 1/2) 2^-20 in (0, 1) is exact and phi = v pi/4;
  // sin phi = v P(v^2) and cos phi = Q(v^2) with P of degree 3 and Q of degree 4,
  // near-minimax in relative error on [0, 1] (fitted by Lawson's iteratively
  // reweighted least squares to sin(pi v/4)/v and cos(pi v/4); approximation
  // error below 0.06 and 0.001 ulp).  The octant's symmetries then swap and sign
  // the pair (bit 29 ^ bit 30: swap; bit 31: sign of sin; bit 31 ^ bit 30: sign
  // of cos).  Within 2 ulp of the exact values (sin 1.7, cos 1.0 over every w).
  static __device__ __forceinline__ void sincos_phi(uint32_t w, float *sp, float *cp) {
    const uint32_t hmask = (uint32_t)((int32_t)(w << 2) >> 31);
    const uint32_t rr = ((w >> 9) ^ hmask) & 0xFFFFFu;
    const float v = __fsub_rn(__uint_as_float(0x3F800004u | (rr << 3)), 1.0f);  // (rr + 1/2) 2^-20, exact
    const float y = v * v;
    float ps = fmaf(y, -3.59504520019982e-05f, 2.49000103212893e-03f);
    ps = fmaf(y, ps, -8.074543625116348e-02f);
    ps = fmaf(y, ps, 7.853981852531433e-01f);
    *sp = v * ps;
    float pc = fmaf(y, 3.52876168108196e-06f, -3.259365039411932e-04f);
    pc = fmaf(y, pc, 1.5854323282837868e-02f);
    pc = fmaf(y, pc, -3.084251284599304e-01f);
    *cp = fmaf(y, pc, 1.0f);
  }
  static __device__ __forceinline__ void sincos2pi_w(uint32_t w, float *s, float *c) {
    float sp, cp;
    sincos_phi(w, &sp, &cp);
    const uint32_t t = w ^ (w << 1);
    const bool swap = (t >> 30) & 1u;
    const float a = swap ? cp : sp, b = swap ? sp : cp;
    *s = __uint_as_float(__float_as_uint(a) ^ (w & 0x80000000u));
    *c = __uint_as_float(__float_as_uint(b) ^ (t & 0x80000000u));
  }
  static __device__ __forceinline__ float cos2pi_w(uint32_t w) {
    float sp, cp;
    sincos_phi(w, &sp, &cp);
    const uint32_t t = w ^ (w << 1);
    const float b = ((t >> 30) & 1u) ? sp : cp;
    return __uint_as_float(__float_as_uint(b) ^ (t & 0x80000000u));
  }
  // v rsqrt(v) by the PTX rsqrt.approx instruction on an argument kept normal (the library
  // rsqrtf adds a subnormal path the walk never needs); 0 for v = 0
  static __device__ __forceinline__ float sqrt_pos(float v) {
    float r;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(fmaxf(v, 1e-37f)));
    return v * r;
  }
  // 2^v by the PTX ex2.approx.ftz.f32 instruction (v already times log2 e; results
  // below the normal range flush to zero, which no weight of interest reaches)
  static __device__ __forceinline__ float exp_scaled(float v) {
    float r;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(v));
    return r;
  }
};
template <> struct Node<double> {
  static __device__ __forceinline__ double neg2ln(double u) { return -2.0 * ::log(u); }
  static __device__ __forceinline__ void sincos2pi_w(uint32_t w, double *s, double *c) {
    ::sincospi(2.0 * uniform01<double>(w), s, c);
  }
  static __device__ __forceinline__ double cos2pi_w(uint32_t w) { return ::cospi(2.0 * uniform01<double>(w)); }
  static __device__ __forceinline__ double sqrt_pos(double v) { return ::sqrt(v); }
  static __device__ __forceinline__ double exp_scaled(double v) { return ::exp(v); }  // v is the plain exponent
};

template <typename Real> __device__ __forceinline__ Real pconst(const WalkParams &p, int i);
template <> __device__ __forceinline__ float pconst<float>(const WalkParams &p, int i) { return p.u0f[i]; }
template <> __device__ __forceinline__ double pconst<double>(const WalkParams &p, int i) { return p.u0d[i]; }

// Per-point shifted origin of the initial data, formed once per point in FP64.
// The walk carries each particle's displacement D from its tree's root x_p, and
// g is evaluated at x_p + D through these offsets, so an FP32 walk keeps full
// relative accuracy near the initial data's centre, zeros and phases:
//   GAUSS, TANH_PROD, GAUSS_AXES  base_i = x_p,i - centre_i
//   LOGISTIC          base_0 = x_p,0 - centre
//   COS_PROD          base_i = omega_i x_p,i reduced to [-pi, pi]
template <typename Real, int DIM>
__device__ __forceinline__ void initial_data_base(const WalkParams &p, const double *xp, Real (&base)[DIM]) {
#pragma unroll
  for (int i = 0; i < DIM; ++i) {
    double b = 0.0;
    switch (p.u0_kind) {
    case kU0Gauss: b = xp[i] - p.u0d[3 + i]; break;
    case kU0TanhProd: b = xp[i] - p.u0d[2 + i]; break;
    case kU0Logistic: b = i == 0 ? xp[0] - p.u0d[2] : 0.0; break;
    case kU0GaussAxes: b = xp[i] - p.u0d[5 + i]; break;
    case kU0Quadratic: b = xp[i]; break;
    case kU0CosProd: b = remainder(p.u0d[2 + i] * xp[i], 6.283185307179586476925286766559); break;
    default: break;
    }
    base[i] = (Real)b;
  }
}

// Initial data g at x_p + D.  Constants (host-prepared; the exponent scales
// carry a factor log2 e in the FP32 copy, see Node<float>::exp_scaled):
//   GAUSS     c0, A, -1/(2 s^2), x0, y0, z0
//   COS_PROD  c0, A, w0, w1, w2
//   TANH_PROD c0, A, s0, s1, s2
//   LOGISTIC  c0, A, x0, -1/width
//   GAUSS_AXES c0, A, -w0, -w1, -w2, m0, m1, m2
//   QUADRATIC  c0, l0, l1, l2, q0, q1, q2
// U0 >= 0 fixes the kind at compile time (the switch folds to its one case);
// U0 = -1 reads it from the parameters.
template <typename Real, int DIM, int U0 = -1>
__device__ __forceinline__ Real initial_data(const WalkParams &p, const Real (&base)[DIM], const Real (&D)[DIM]) {
  using M = Math<Real>;
  const Real c0 = pconst<Real>(p, 0), A = pconst<Real>(p, 1);
  switch (U0 >= 0 ? U0 : p.u0_kind) {
  case kU0Gauss: {
    Real r2 = Real(0);
#pragma unroll
    for (int i = 0; i < DIM; ++i) {
      const Real e = base[i] + D[i];
      r2 += e * e;
    }
    return c0 + A * Node<Real>::exp_scaled(r2 * pconst<Real>(p, 2));
  }
  case kU0CosProd: {
    Real pr = Real(1);
#pragma unroll
    for (int i = 0; i < DIM; ++i) pr *= M::cos(base[i] + pconst<Real>(p, 2 + i) * D[i]);
    return c0 + A * pr;
  }
  case kU0TanhProd: {
    Real pr = Real(1);
#pragma unroll
    for (int i = 0; i < DIM; ++i) pr *= M::tanh(base[i] + D[i]);
    return c0 + A * pr;
  }
  case kU0Logistic:
    return c0 + A / (Real(1) + Node<Real>::exp_scaled((base[0] + D[0]) * pconst<Real>(p, 3)));
  case kU0Quadratic: {
    Real v = c0;
#pragma unroll
    for (int i = 0; i < DIM; ++i) {
      const Real e = base[i] + D[i];
      v += (pconst<Real>(p, 1 + i) + pconst<Real>(p, 4 + i) * e) * e;
    }
    return v;
  }
  case kU0GaussAxes: {
    Real r = Real(0);
#pragma unroll
    for (int i = 0; i < DIM; ++i) {
      const Real e = base[i] + D[i];
      r += pconst<Real>(p, 2 + i) * e * e;
    }
    return c0 + A * Node<Real>::exp_scaled(r);
  }
  default:
    return c0;
  }
}

// Variable-coefficient profile gamma at the root's point xp plus displacement y,
// at PDE time t (kinds as GRT_COEF_*):
//   GAUSS_OVER_T  exp(-sum_i w_i (x_i - m_i)^2) / (t + t0)
//   GAUSS         exp(-sum_i w_i (x_i - m_i)^2)
// The offset x_p - m is formed in FP64 and the displacement added in the walk's
// precision, as for the initial data.
template <typename Real, int DIM>
__device__ __forceinline__ Real coef_gamma(const WalkParams &p, const double *__restrict__ xp, const Real (&y)[DIM],
                                           Real t) {
  Real r = Real(0);
#pragma unroll
  for (int i = 0; i < DIM; ++i) {
    const Real e = (Real)(xp[i] - p.cmd[i]) + y[i];
    if constexpr (sizeof(Real) == 4) {
      r += p.cwf[i] * e * e;
    } else {
      r += p.cwd[i] * e * e;
    }
  }
  Real g = Node<Real>::exp_scaled(r);
  if (p.coef_kind == kCoefGaussOverT) {
    if constexpr (sizeof(Real) == 4) {
      g = g / (t + p.ct0f);
    } else {
      g = g / (t + p.ct0d);
    }
  }
  return g;
}

template <typename Real> struct Scalars;
template <> struct Scalars<float> {
  static __device__ __forceinline__ float leaf(const WalkParams &p) { return p.leaf_factorf; }
  static __device__ __forceinline__ float two_D(const WalkParams &p) { return p.two_Df; }
  static __device__ __forceinline__ float inv_lambda(const WalkParams &p) { return p.inv_lambdaf; }
  static __device__ __forceinline__ float lam_minus_c(const WalkParams &p) { return p.lam_minus_cf; }
};
template <> struct Scalars<double> {
  static __device__ __forceinline__ double leaf(const WalkParams &p) { return p.leaf_factor; }
  static __device__ __forceinline__ double two_D(const WalkParams &p) { return p.two_D; }
  static __device__ __forceinline__ double inv_lambda(const WalkParams &p) { return p.inv_lambda; }
  static __device__ __forceinline__ double lam_minus_c(const WalkParams &p) { return p.lam_minus_c; }
};

template <typename Real> __device__ __forceinline__ Real sdeconst(const WalkParams &p, int i);
template <> __device__ __forceinline__ float sdeconst<float>(const WalkParams &p, int i) { return p.sdef[i]; }
template <> __device__ __forceinline__ double sdeconst<double>(const WalkParams &p, int i) { return p.sded[i]; }

// Euler-Maruyama over a segment of length seg for dX_i = (beta_i - kappa_i X_i) dt
// + (s_i + r_i X_i) dW_i (the Euler scheme of Sec. 2.4 for the SDE of a general
// operator), sde_steps equal steps.  The walk carries displacements y from the
// root; X = x_p + y.  Normals come from Philox blocks at the node's counter with
// the sub bit set, block b under the key (k0 ^ (b+1) 0x2545F491, k1 ^ (b+1)
// 0x6C8E9CF5), Box-Muller on its word pairs: for d <= 2 block b serves steps 2b
// ((w0, w1)) and 2b + 1 ((w2, w3)); for d = 3 block b serves step b ((w0, w1) for
// n0, n1 and (w2, w3) for n2).
template <typename Real, int DIM>
__device__ __forceinline__ void euler_step(const WalkParams &p, const Real (&x0)[DIM], Real h, Real sh,
                                           const Real (&z)[3], Real (&y)[DIM]) {
#pragma unroll
  for (int i = 0; i < DIM; ++i) {
    const Real X = x0[i] + y[i];
    y[i] += (sdeconst<Real>(p, i) - sdeconst<Real>(p, 3 + i) * X) * h +
            (sdeconst<Real>(p, 6 + i) + sdeconst<Real>(p, 9 + i) * X) * sh * z[i];
  }
}

template <typename Real, int DIM>
__device__ __forceinline__ void euler_segment(const WalkParams &p, const double *__restrict__ xp, Real seg,
                                              uint32_t id_lo, uint32_t id_hi, uint32_t tree, uint32_t point,
                                              Real (&y)[DIM]) {
  using F = Node<Real>;
  const int m = p.sde_steps;
  const Real h = seg / (Real)m;
  const Real sh = F::sqrt_pos(h);
  Real x0[DIM];
#pragma unroll
  for (int i = 0; i < DIM; ++i) x0[i] = (Real)xp[i];
  const uint32_t k0 = p.rk0[0], k1 = p.rk1[0];
  const int nblocks = DIM <= 2 ? (m + 1) / 2 : m;
  for (int b = 0; b < nblocks; ++b) {
    const uint32_t bb = (uint32_t)(b + 1);
    const uint4 w = philox4x32_10_key(make_uint4(id_lo, id_hi, tree | 0x80000000u, point), k0 ^ (bb * 0x2545F491u),
                                      k1 ^ (bb * 0x6C8E9CF5u));
    Real z[3];
    {
      const Real r = F::sqrt_pos(F::neg2ln(uniform01<Real>(w.x)));
      Real sn, cs;
      F::sincos2pi_w(w.y, &sn, &cs);
      z[0] = r * cs;
      z[1] = r * sn;
    }
    if constexpr (DIM == 3) {
      z[2] = F::sqrt_pos(F::neg2ln(uniform01<Real>(w.z))) * F::cos2pi_w(w.w);
      euler_step<Real, DIM>(p, x0, h, sh, z, y);
    } else {
      z[2] = Real(0);
      euler_step<Real, DIM>(p, x0, h, sh, z, y);
      if (2 * b + 1 < m) {
        const Real r = F::sqrt_pos(F::neg2ln(uniform01<Real>(w.z)));
        Real sn, cs;
        F::sincos2pi_w(w.w, &sn, &cs);
        z[0] = r * cs;
        z[1] = r * sn;
        euler_step<Real, DIM>(p, x0, h, sh, z, y);
      }
    }
  }
}

// Index of the first category whose threshold exceeds w among the finite
// thresholds thr[first .. count-1] (the last category's threshold is 2^32 and
// is not stored): an early-exit scan, since the first categories carry most
// of the probability.  `thr` is the block-shared copy of the table.
__device__ __forceinline__ int categorical(const uint32_t *__restrict__ thr, uint32_t w, int first, int count) {
  int j = first;
  while (j < count && w >= thr[j]) ++j;
  return j;
}

// Result of one node.
template <typename Real, int DIM> struct NodeOut {
  Real y[DIM];   // end of the node's Brownian segment (displacement from the root)
  Real tau_c;    // remaining time of its children
  Real factor;   // multiplies the tree weight (includes g(y) at a leaf)
  int cat;       // term index (split) or -1 (leaf)
};

// One node: the draws, the segment, the decision and the factor.
//   Strategy B: leaf with probability q, weight g(x + sqrt(2 D tau) n) / q; else
//     term k with probability (1-q) p_k, split at tau S (S ~ U(0,1)), weight
//     tau b_k / ((1-q) p_k), children at remaining time tau (1 - S).
//   Strategy A: lifetime S = -ln(U)/lambda; S >= tau: leaf with weight
//     e^{(lambda-c) tau} g(x + sqrt(2 D tau) n); else split at S with weight
//     e^{(lambda-c) S} b_k / (lambda p_k), children at remaining time tau - S.
// A variable coefficient (coef_kind != 0, the term's bit in coef_cat_mask)
// multiplies the split factor by gamma at the split position and at the PDE
// time left to the children (Sec. 2.1, Eq. probexp1: c_j(beta(S), t - S)).
// `s_factor`, `s_thr` and the caller's arity table are block-shared copies of the tables;
// x is the displacement from the tree's root, `base` the root's shifted origin
// and xp the root's coordinates (read only by a variable coefficient).
template <typename Real, int DIM, int STRAT, int FEAT = 0, int U0 = -1>
__device__ __forceinline__ void node_step(const WalkParams &p, const Real *__restrict__ s_factor,
                                          const uint32_t *__restrict__ s_thr, const Real (&base)[DIM],
                                          const double *__restrict__ xp, const Real (&x)[DIM], Real tau,
                                          uint32_t id_lo, uint32_t id_hi, uint32_t tree, uint32_t point,
                                          NodeOut<Real, DIM> &o) {
  using M = Math<Real>;
  const uint4 w = philox4x32_10(make_uint4(id_lo, id_hi, tree, point), p.rk0, p.rk1);
  // Box-Muller on (w2, w3): n0 = r cos(2 pi U3), n1 = r sin(2 pi U3), r = sqrt(-2 ln U2); the
  // segment below scales them by sqrt(2 D s), taken together with r as one square root
  using F = Node<Real>;
  Real lg[DIM > 2 ? 2 : 1], cs[DIM];  // -2 ln U of each Box-Muller pair; cos / sin of its angle
  {
    lg[0] = F::neg2ln(uniform01<Real>(w.z));
    Real s, c;
    F::sincos2pi_w(w.w, &s, &c);
    cs[0] = c;
    if (DIM > 1) cs[DIM > 1 ? 1 : 0] = s;
  }
  if (DIM == 3) {
    const uint4 w2 = philox4x32_10(make_uint4(id_lo, id_hi, tree | 0x80000000u, point), p.rk0, p.rk1);
    lg[DIM > 2 ? 1 : 0] = F::neg2ln(uniform01<Real>(w2.x));
    cs[DIM - 1] = F::cos2pi_w(w2.y);
  }

  bool leaf;
  Real seg, S;
  if (STRAT == kStratB) {
    // joint draw: category 0 is the leaf (w < thr[0]), category j >= 1 is term j - 1
    // the first two thresholds come from the parameter bank (no shared-memory load): they
    // decide the leaf and the most probable term
    leaf = p.ncat_thr == 0 || w.x < p.thr[0];
    o.cat = leaf ? -1 : ((p.ncat_thr <= 1 || w.x < p.thr[1]) ? 0 : categorical(s_thr, w.x, 2, p.ncat_thr) - 1);
    S = uniform01<Real>(w.y);
    seg = leaf ? tau : tau * S;
    o.tau_c = tau * (Real(1) - S);
  } else {
    S = Real(0.5) * F::neg2ln(uniform01<Real>(w.x)) * Scalars<Real>::inv_lambda(p);
    leaf = (S >= tau) || (p.nterms == 0);
    seg = leaf ? tau : S;
    o.tau_c = tau - S;
    o.cat = leaf ? -1 : ((p.ncat_thr == 0 || w.y < p.thr[0]) ? 0 : categorical(s_thr, w.y, 1, p.ncat_thr));
  }
  if constexpr ((FEAT & kFeatEuler) != 0) {
#pragma unroll
    for (int i = 0; i < DIM; ++i) o.y[i] = x[i];
    euler_segment<Real, DIM>(p, xp, seg, id_lo, id_hi, tree, point, o.y);
  } else {
    // y = x + sqrt(2 D s) r (cos, sin): the two square roots as one
    const Real tds = Scalars<Real>::two_D(p) * seg;
    const Real R0 = F::sqrt_pos(tds * lg[0]);
#pragma unroll
    for (int i = 0; i < (DIM < 2 ? DIM : 2); ++i) o.y[i] = x[i] + R0 * cs[i];
    if constexpr (DIM == 3) o.y[2] = x[2] + F::sqrt_pos(tds * lg[1]) * cs[2];
  }

  // every lane evaluates g (a leaf uses it) and reads its term factor (a split uses it):
  // the warp runs one convergent body instead of two divergent ones
  const Real g = initial_data<Real, DIM, U0>(p, base, o.y);
  const Real tf = s_factor[leaf ? 0 : o.cat];
  if (STRAT == kStratB) {
    o.factor = leaf ? Scalars<Real>::leaf(p) * g : tau * tf;
  } else {
    const Real lmc = Scalars<Real>::lam_minus_c(p);
    const Real e = lmc == Real(0) ? Real(1) : F::exp_scaled(lmc * (leaf ? tau : S));
    o.factor = leaf ? ((p.nterms == 0) ? g : e * g) : e * tf;
  }
  if constexpr ((FEAT & kFeatVarCoef) != 0)
    if (!leaf && ((p.coef_cat_mask >> o.cat) & 1u)) o.factor *= coef_gamma<Real, DIM>(p, xp, o.y, o.tau_c);
}

}  // namespace grt
