// grt_pdd.cu -- the probabilistic-domain-decomposition stages after the point
// solve (Sec. 3): a tensor-product not-a-knot cubic spline of the interface
// values and independent Crank-Nicolson solves of the subdomains.
//
// GPU layout:
//   * spline: a weights kernel (one thread per target and nodal column: the
//     not-a-knot system of a unit data vector by elimination, then the cubic
//     at that target) and an axis-contraction kernel applied once per axis, FP64;
//   * local solver: a cluster of two thread blocks per subdomain (each owning
//     half of the rows, the peer's half read through distributed shared
//     memory) -- or one block when a half does not fit in shared memory --
//     runs every time step with an exact fast-diagonalisation solve per step
//     (DST-I along each axis as small dense FP64 contractions); the subdomains
//     share nothing, which is the decoupling the method is built on (Sec. 3,
//     "Local solver").
#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <cstring>
#include <string>
#include <vector>

#include "grt.h"
#include "grt_host.h"

namespace grt {

// ---------------------------------------------------------------------------
// spline weights: W[t][j] = s_j(target t), s_j the not-a-knot cubic spline of
// the unit vector e_j on n uniform nodes lo + i hn (Sec. 3, Interpolation).
// With uniform spacing the second derivatives M_i satisfy
//   M_{i-1} + 4 M_i + M_{i+1} = r_i = 6 (y_{i+1} - 2 y_i + y_{i-1}) / hn^2,  i = 1..n-2,
// and not-a-knot (s''' continuous at x_1, x_{n-2}) gives M_0 = 2 M_1 - M_2 and
// M_{n-1} = 2 M_{n-2} - M_{n-3}; substituted into rows 1 and n-2 these give
// M_1 = r_1 / 6 and M_{n-2} = r_{n-2} / 6, leaving a tridiagonal system for
// M_2..M_{n-3} (Thomas elimination).  On [x_i, x_{i+1}], A = (x_{i+1} - x)/hn,
// B = 1 - A: s = A y_i + B y_{i+1} + ((A^3 - A) M_i + (B^3 - B) M_{i+1}) hn^2 / 6.
// ---------------------------------------------------------------------------
// One thread per (target t, node j): the thread solves for the M_i of e_j (n is small: the
// spline's nodes on one axis) and evaluates that one target, so a launch is as long as one
// O(n) solve rather than a node's whole list of targets.
__global__ void spline_weights_kernel(int n, double lo, double hn, int m, const double *__restrict__ targets,
                                      double *__restrict__ W) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (long long)n * m) return;
  const int j = (int)(e % n), t = (int)(e / n);
  double M[GRT_SPLINE_MAX_NODES], cp[GRT_SPLINE_MAX_NODES];
  const double s6 = 6.0 / (hn * hn);
  auto r_at = [&](int i) -> double {  // 6 (y_{i+1} - 2 y_i + y_{i-1}) / hn^2 for y = e_j
    double v = 0.0;
    if (i + 1 == j || i - 1 == j) v += 1.0;
    if (i == j) v -= 2.0;
    return v * s6;
  };
  M[1] = r_at(1) / 6.0;
  M[n - 2] = r_at(n - 2) / 6.0;
  // M_2..M_{n-3}: diagonal 4, off-diagonals 1 (forward sweep, back substitution)
  const int first = 2, last = n - 3;
  for (int i = first; i <= last; ++i) {
    double rhs = r_at(i);
    if (i == first) rhs -= M[1];
    if (i == last) rhs -= M[n - 2];
    const double denom = (i == first) ? 4.0 : 4.0 - cp[i - 1];
    cp[i] = 1.0 / denom;
    M[i] = (i == first) ? rhs / denom : (rhs - M[i - 1]) / denom;
  }
  for (int i = last - 1; i >= first; --i) M[i] -= cp[i] * M[i + 1];
  M[0] = 2.0 * M[1] - M[2];
  M[n - 1] = 2.0 * M[n - 2] - M[n - 3];
  const double hh6 = hn * hn / 6.0;
  const double xt = targets[t];
  int i = (int)floor((xt - lo) / hn);
  i = i < 0 ? 0 : (i > n - 2 ? n - 2 : i);
  const double A = (lo + (double)(i + 1) * hn - xt) / hn, B = 1.0 - A;
  double v = 0.0;
  if (i == j) v += A;
  if (i + 1 == j) v += B;
  v += ((A * A * A - A) * M[i] + (B * B * B - B) * M[i + 1]) * hh6;
  W[(size_t)t * n + j] = v;
}

static void launch_spline_weights(int n, double lo, double hn, int m, const double *targets, double *W,
                                  cudaStream_t s) {
  const long long total = (long long)n * m;
  if (total <= 0) return;
  spline_weights_kernel<<<(unsigned)((total + 127) / 128), 128, 0, s>>>(n, lo, hn, m, targets, W);
}

// out[o][i][r] = sum_j W[i][j] in[o][j][r]: one axis of the tensor-product spline.
__global__ void axis_apply_kernel(const double *__restrict__ W, int m, int n, const double *__restrict__ in,
                                  double *__restrict__ out, long long outer, long long inner) {
  const long long total = outer * (long long)m * inner;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const long long r = e % inner;
    const long long oi = e / inner;
    const int i = (int)(oi % m);
    const long long o = oi / m;
    const double *src = in + (o * n) * inner + r;
    const double *w = W + (size_t)i * n;
    double acc = 0.0;
    for (int j = 0; j < n; ++j) acc = fma(w[j], src[(long long)j * inner], acc);
    out[e] = acc;
  }
}

// ---------------------------------------------------------------------------
// PDD device description
// ---------------------------------------------------------------------------
struct PddDev {
  int dim;
  int N[3], cells[3], sub[3], m[3];
  double lo[3], h[3], inv_h2[3];
  int nsteps;
  double dt, alpha;
  const double *B[3];        // per axis: [sub+1][nsteps][plane FD nodes] (levels t_1..t_N)
  long long plane_elems[3];  // FD nodes of one axis-a plane
  int f_deg;
  double f_coef[GRT_MAX_DEG + 1];
  uint32_t coef_pow_mask;    // powers k whose coefficient is b_k gamma(x, t)
  const double *S[3];        // per axis: the m x m orthonormal DST-I matrix
  const double *mu[3];       // per axis: eigenvalues of the 1-D Dirichlet second difference
  const double *inv_eig;     // [mloc] 1 / (1 - alpha sum_a mu_a(i_a)), subdomain-local row-major index
  double *work;              // [nsub][4][mloc] when the vectors do not fit in shared memory
  int mloc;
  int use_smem;
  int sub_first;             // first subdomain (row-major index) of this launch
  double *u_out;
};

// S[i][j] = sqrt(2/(m+1)) sin(pi (i+1)(j+1)/(m+1)) (symmetric, orthonormal, its own
// inverse) and mu[k] = -(4/h^2) sin^2(pi (k+1) / (2 (m+1))): the eigenvectors and
// eigenvalues of the second difference with zero Dirichlet ends.  The product
// (i+1)(j+1) is reduced modulo 2(m+1) in integers before the sine.
__global__ void dst_tables_kernel(int m, double h, double *__restrict__ S, double *__restrict__ mu) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= m * m) return;
  const int i = e / m, j = e % m;
  const int r = ((i + 1) * (j + 1)) % (2 * (m + 1));
  S[e] = sqrt(2.0 / (double)(m + 1)) * sinpi((double)r / (double)(m + 1));
  if (j == 0) {
    const double sv = sinpi((double)(i + 1) / (2.0 * (double)(m + 1)));
    mu[i] = -4.0 / (h * h) * sv * sv;
  }
}

// inv[l] = 1 / (1 - alpha sum_a mu_a(i_a)) for the subdomain-local row-major index l:
// the eigenvalues of I - alpha Lap_h, inverted once per solve instead of per step
__global__ void inv_eig_kernel(int dim, int m0, int m1, int m2, double alpha, const double *__restrict__ mu0,
                               const double *__restrict__ mu1, const double *__restrict__ mu2, double *__restrict__ inv) {
  const int n = m0 * m1 * m2;
  for (int l = blockIdx.x * blockDim.x + threadIdx.x; l < n; l += gridDim.x * blockDim.x) {
    const int i2 = l % m2, i1 = (l / m2) % m1, i0 = l / (m1 * m2);
    double lam = mu0[i0];
    if (dim > 1) lam += mu1[i1];
    if (dim > 2) lam += mu2[i2];
    inv[l] = 1.0 / (1.0 - alpha * lam);
  }
}

// initial data at a point (FP64, the walk's own formulas with zero displacement)
template <int DIM> __device__ __forceinline__ double u0_at(const WalkParams &p, const double (&x)[3]) {
  double base[DIM], zero[DIM];
  initial_data_base<double, DIM>(p, x, base);
#pragma unroll
  for (int i = 0; i < DIM; ++i) zero[i] = 0.0;
  return initial_data<double, DIM>(p, base, zero);
}

// f(u, x, t) = sum_k c_k(x, t) u^k (Horner on the constant and on the gamma-scaled powers)
template <int DIM>
__device__ __forceinline__ double f_at(const WalkParams &p, const PddDev &q, const double (&x)[3], double t,
                                       double u) {
  double fc = 0.0, fg = 0.0;
  const bool var = p.coef_kind != kCoefConst;
  for (int k = q.f_deg; k >= 0; --k) {
    const bool vk = var && ((q.coef_pow_mask >> k) & 1u);
    fc = fc * u + (vk ? 0.0 : q.f_coef[k]);
    fg = fg * u + (vk ? q.f_coef[k] : 0.0);
  }
  if (!var) return fc;
  double zero[DIM];
#pragma unroll
  for (int i = 0; i < DIM; ++i) zero[i] = 0.0;
  return fc + coef_gamma<double, DIM>(p, x, zero, t) * fg;
}

// Dirichlet value of the ring node next to interior node gi (global indices)
// across face `side` of axis a, at level n (0: initial data).
template <int DIM>
__device__ __forceinline__ double ring_value(const WalkParams &p, const PddDev &q, const int (&s)[3],
                                             const int (&gi)[3], int a, int side, int n) {
  int g[3] = {gi[0], gi[1], gi[2]};
  const int k = s[a] + side;
  g[a] = k * q.cells[a];
  if (n == 0) {
    double x[3] = {0.0, 0.0, 0.0};
#pragma unroll
    for (int b = 0; b < DIM; ++b) x[b] = q.lo[b] + (double)g[b] * q.h[b];
    return u0_at<DIM>(p, x);
  }
  long long off = 0;
#pragma unroll
  for (int b = 0; b < DIM; ++b)
    if (b != a) off = off * q.N[b] + g[b];
  return q.B[a][((long long)k * q.nsteps + (n - 1)) * q.plane_elems[a] + off];
}

template <int DIM> __device__ __forceinline__ void local_index(const PddDev &q, int l, int (&i)[3]) {
  i[0] = i[1] = i[2] = 0;
#pragma unroll
  for (int a = DIM - 1; a >= 0; --a) {
    i[a] = l % q.m[a];
    l /= q.m[a];
  }
}

// dst = S_ax applied along axis ax of src (one output per thread-iteration)
template <int DIM, int NT>
__device__ __forceinline__ void dst_axis(const PddDev &q, int ax, const int (&stride)[3], const double *src,
                                         double *dst) {
  const int m = q.m[ax], st = stride[ax];
  const double *__restrict__ S = q.S[ax];
  for (int l = threadIdx.x; l < q.mloc; l += NT) {
    int i[3];
    local_index<DIM>(q, l, i);
    const double *col = src + (l - i[ax] * st);
    const double *row = S + i[ax] * m;
    double acc = 0.0;
    for (int j = 0; j < m; ++j) acc = fma(__ldg(row + j), col[j * st], acc);
    dst[l] = acc;
  }
}

// One block per subdomain runs every Crank-Nicolson step.  Each step's system
// (I - alpha Lap_h) x = b is solved exactly by fast diagonalisation (Lynch,
// Rice and Thomas, Numer. Math. 6, 1964): the Dirichlet Laplacian of a box is
// diagonal in the tensor product of 1-D sine bases, so x = S (S b / (1 - alpha
// sum_a mu_a)) with S the DST-I along every axis -- 2 d small dense
// contractions per step, no iteration and no block-wide reduction.
template <int DIM, int NT>
__global__ void __launch_bounds__(NT) cn_subdomain_kernel(const WalkParams p, const PddDev q) {
  extern __shared__ double smem_vec[];
  const int sid = q.sub_first + (int)blockIdx.x;
  int s[3] = {0, 0, 0};
  {
    int r = sid;
#pragma unroll
    for (int a = DIM - 1; a >= 0; --a) {
      s[a] = r % q.sub[a];
      r /= q.sub[a];
    }
  }
  const int mloc = q.mloc;
  double *base = q.use_smem ? smem_vec : q.work + (size_t)sid * 4 * mloc;
  double *u = base, *up = u + mloc, *va = up + mloc, *vb = va + mloc;
  int stride[3] = {1, 1, 1};
#pragma unroll
  for (int a = DIM - 2; a >= 0; --a) stride[a] = stride[a + 1] * q.m[a + 1];

  auto node = [&](int l, int (&i)[3], int (&gi)[3], double (&xc)[3]) {
    local_index<DIM>(q, l, i);
    xc[0] = xc[1] = xc[2] = 0.0;
    gi[0] = gi[1] = gi[2] = 0;
#pragma unroll
    for (int a = 0; a < DIM; ++a) {
      gi[a] = s[a] * q.cells[a] + 1 + i[a];
      xc[a] = q.lo[a] + (double)gi[a] * q.h[a];
    }
  };

  for (int l = threadIdx.x; l < mloc; l += NT) {
    int i[3], gi[3];
    double xc[3];
    node(l, i, gi, xc);
    u[l] = u0_at<DIM>(p, xc);
    up[l] = u[l];
  }
  __syncthreads();

  for (int n = 0; n < q.nsteps; ++n) {
    // right-hand side b = u + alpha Lap_h u (ring at t_n) + alpha (ring part at t_{n+1}) + dt f(u*)
    const double th = ((double)n + 0.5) * q.dt;
    for (int l = threadIdx.x; l < mloc; l += NT) {
      int i[3], gi[3];
      double xc[3];
      node(l, i, gi, xc);
      const double c = u[l];
      double lap = 0.0, ring1 = 0.0;
#pragma unroll
      for (int a = 0; a < DIM; ++a) {
        const double left = i[a] > 0 ? u[l - stride[a]] : ring_value<DIM>(p, q, s, gi, a, 0, n);
        const double right = i[a] < q.m[a] - 1 ? u[l + stride[a]] : ring_value<DIM>(p, q, s, gi, a, 1, n);
        lap += (left + right - 2.0 * c) * q.inv_h2[a];
        double rn = 0.0;
        if (i[a] == 0) rn += ring_value<DIM>(p, q, s, gi, a, 0, n + 1);
        if (i[a] == q.m[a] - 1) rn += ring_value<DIM>(p, q, s, gi, a, 1, n + 1);
        ring1 += rn * q.inv_h2[a];
      }
      const double ustar = n == 0 ? c : 1.5 * c - 0.5 * up[l];
      va[l] = c + q.alpha * lap + q.alpha * ring1 + q.dt * f_at<DIM>(p, q, xc, th, ustar);
    }
    __syncthreads();
    double *src = va, *dst = vb;
#pragma unroll
    for (int a = 0; a < DIM; ++a) {  // into the sine basis
      dst_axis<DIM, NT>(q, a, stride, src, dst);
      __syncthreads();
      double *t = src;
      src = dst;
      dst = t;
    }
    for (int l = threadIdx.x; l < mloc; l += NT)  // divide by the eigenvalues of I - alpha Lap_h
      src[l] *= __ldg(q.inv_eig + l);
    __syncthreads();
#pragma unroll
    for (int a = 0; a < DIM; ++a) {  // back (S is its own inverse)
      dst_axis<DIM, NT>(q, a, stride, src, dst);
      __syncthreads();
      double *t = src;
      src = dst;
      dst = t;
    }
    // rotate: u^{n-1} <- u^n, u^n <- the solution; the two freed vectors are the next scratch
    double *old_up = up;
    up = u;
    u = src;
    va = old_up;
    vb = dst;
  }
  for (int l = threadIdx.x; l < mloc; l += NT) {
    int i[3], gi[3];
    double xc[3];
    node(l, i, gi, xc);
    long long off = 0;
#pragma unroll
    for (int a = 0; a < DIM; ++a) off = off * q.N[a] + gi[a];
    q.u_out[off] = u[l];
  }
}

// The same steps with each subdomain split between the two blocks of a
// cluster: block rank r owns the rows [r0, r1) of axis 0 (rank 0 the first
// ceil(m0/2)), keeps its four vectors in its own shared memory and reads the
// peer's rows through distributed shared memory for the axis-0 stencil and
// the axis-0 sine transform.  Twice the SMs work on the same subdomains.
// Order of a step: cluster barrier (the peer's u is final); right-hand side;
// transforms along the in-row axes (local); cluster barrier; axis-0 transform
// with the eigenvalue division; cluster barrier; axis-0 inverse transform;
// cluster barrier (every peer read of this step is done); inverse in-row
// transforms (local).
template <int DIM, int NT>
__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(NT) cn_pair_kernel(const WalkParams p, const PddDev q) {
  namespace cg = cooperative_groups;
  cg::cluster_group cl = cg::this_cluster();
  extern __shared__ double smem_vec[];
  const unsigned crank = cl.block_rank();
  const int sid = q.sub_first + (int)(blockIdx.x >> 1);
  int s[3] = {0, 0, 0};
  {
    int r = sid;
#pragma unroll
    for (int a = DIM - 1; a >= 0; --a) {
      s[a] = r % q.sub[a];
      r /= q.sub[a];
    }
  }
  const int m0 = q.m[0];
  const int h0 = (m0 + 1) >> 1;
  const int r0 = crank ? h0 : 0, r1 = crank ? m0 : h0;
  const int plane = q.mloc / m0;   // unknowns of one axis-0 row
  const int nloc = (r1 - r0) * plane;
  const int cap = h0 * plane;      // vector capacity: the larger half
  double *mine = smem_vec;
  double *peer = cl.map_shared_rank(smem_vec, (int)(crank ^ 1u));
  // roles -> vector slots (both blocks rotate identically)
  int ru = 0, rup = 1, ra = 2, rb = 3;
  // in-row strides (axis 1, 2 within a row of the local storage)
  int stride[3] = {plane, 1, 1};
#pragma unroll
  for (int a = DIM - 2; a >= 1; --a) stride[a] = stride[a + 1] * q.m[a + 1];
  // value of role `role` at row g0 (global within the subdomain), in-row offset w
  auto at = [&](int role, int g0, int w) -> double {
    return g0 >= r0 && g0 < r1 ? mine[role * cap + (g0 - r0) * plane + w]
                               : peer[role * cap + (g0 - (crank ? 0 : h0)) * plane + w];
  };
  auto node = [&](int l, int (&i)[3], int (&gi)[3], double (&xc)[3]) {
    i[0] = r0 + l / plane;
    int w = l % plane;
#pragma unroll
    for (int a = DIM - 1; a >= 1; --a) {
      i[a] = w % q.m[a];
      w /= q.m[a];
    }
    xc[0] = xc[1] = xc[2] = 0.0;
    gi[0] = gi[1] = gi[2] = 0;
#pragma unroll
    for (int a = 0; a < DIM; ++a) {
      gi[a] = s[a] * q.cells[a] + 1 + i[a];
      xc[a] = q.lo[a] + (double)gi[a] * q.h[a];
    }
  };
  // in-row transform along axis ax >= 1 (local)
  auto row_axis = [&](int ax, int rs, int rd) {
    const int m = q.m[ax], st = stride[ax];
    const double *__restrict__ S = q.S[ax];
    const double *src = mine + rs * cap;
    double *dst = mine + rd * cap;
    for (int l = threadIdx.x; l < nloc; l += NT) {
      int i[3], gi[3];
      double xc[3];
      node(l, i, gi, xc);
      const double *col = src + (l - i[ax] * st);
      const double *row = S + i[ax] * m;
      double acc = 0.0;
      for (int j = 0; j < m; ++j) acc = fma(__ldg(row + j), col[j * st], acc);
      dst[l] = acc;
    }
  };
  // axis-0 transform (reads both blocks' rows); with `scale` divides by 1 - alpha sum mu
  auto axis0 = [&](int rs, int rd, bool scale) {
    const double *__restrict__ S = q.S[0];
    for (int l = threadIdx.x; l < nloc; l += NT) {
      const int g0 = r0 + l / plane, w = l % plane;
      const double *row = S + g0 * m0;
      double acc = 0.0;
      for (int j = 0; j < m0; ++j) acc = fma(__ldg(row + j), at(rs, j, w), acc);
      if (scale) acc *= __ldg(q.inv_eig + r0 * plane + l);
      mine[rd * cap + l] = acc;
    }
  };

  for (int l = threadIdx.x; l < nloc; l += NT) {
    int i[3], gi[3];
    double xc[3];
    node(l, i, gi, xc);
    const double v = u0_at<DIM>(p, xc);
    mine[ru * cap + l] = v;
    mine[rup * cap + l] = v;
  }
  for (int n = 0; n < q.nsteps; ++n) {
    cl.sync();  // the peer's u is final
    const double th = ((double)n + 0.5) * q.dt;
    for (int l = threadIdx.x; l < nloc; l += NT) {
      int i[3], gi[3];
      double xc[3];
      node(l, i, gi, xc);
      const int w = l % plane;
      const double c = mine[ru * cap + l];
      double lap = 0.0, ring1 = 0.0;
#pragma unroll
      for (int a = 0; a < DIM; ++a) {
        double left, right;
        if (a == 0) {
          left = i[0] > 0 ? at(ru, i[0] - 1, w) : ring_value<DIM>(p, q, s, gi, 0, 0, n);
          right = i[0] < m0 - 1 ? at(ru, i[0] + 1, w) : ring_value<DIM>(p, q, s, gi, 0, 1, n);
        } else {
          left = i[a] > 0 ? mine[ru * cap + l - stride[a]] : ring_value<DIM>(p, q, s, gi, a, 0, n);
          right = i[a] < q.m[a] - 1 ? mine[ru * cap + l + stride[a]] : ring_value<DIM>(p, q, s, gi, a, 1, n);
        }
        lap += (left + right - 2.0 * c) * q.inv_h2[a];
        double rn = 0.0;
        if (i[a] == 0) rn += ring_value<DIM>(p, q, s, gi, a, 0, n + 1);
        if (i[a] == q.m[a] - 1) rn += ring_value<DIM>(p, q, s, gi, a, 1, n + 1);
        ring1 += rn * q.inv_h2[a];
      }
      const double ustar = n == 0 ? c : 1.5 * c - 0.5 * mine[rup * cap + l];
      mine[ra * cap + l] = c + q.alpha * lap + q.alpha * ring1 + q.dt * f_at<DIM>(p, q, xc, th, ustar);
    }
    __syncthreads();
    int x = ra, y = rb;  // data in x
#pragma unroll
    for (int a = DIM - 1; a >= 1; --a) {
      row_axis(a, x, y);
      __syncthreads();
      const int t = x;
      x = y;
      y = t;
    }
    cl.sync();          // the peer's rows are transformed along its in-row axes
    axis0(x, y, true);  // into the sine basis along axis 0, divided by the eigenvalues
    cl.sync();
    axis0(y, x, false);  // back along axis 0
    cl.sync();           // every read of the peer's rows in this step is done
#pragma unroll
    for (int a = 1; a < DIM; ++a) {
      row_axis(a, x, y);
      __syncthreads();
      const int t = x;
      x = y;
      y = t;
    }
    // rotate: u^{n-1} <- u^n, u^n <- the solution; the freed slots are the next scratch
    const int old_up = rup;
    rup = ru;
    ru = x;
    ra = old_up;
    rb = y;
  }
  for (int l = threadIdx.x; l < nloc; l += NT) {
    int i[3], gi[3];
    double xc[3];
    node(l, i, gi, xc);
    long long off = 0;
#pragma unroll
    for (int a = 0; a < DIM; ++a) off = off * q.N[a] + gi[a];
    q.u_out[off] = mine[ru * cap + l];
  }
  cl.sync();  // the peer may still read this block's shared memory until here
}

// Plane nodes of the output: the spline at T, the lowest axis's plane on edges.
template <int DIM> __global__ void pdd_planes_kernel(const PddDev q) {
  long long total = 1;
#pragma unroll
  for (int a = 0; a < DIM; ++a) total *= q.N[a];
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    int g[3] = {0, 0, 0};
    long long r = e;
#pragma unroll
    for (int a = DIM - 1; a >= 0; --a) {
      g[a] = (int)(r % q.N[a]);
      r /= q.N[a];
    }
    int a0 = -1;
#pragma unroll
    for (int a = DIM - 1; a >= 0; --a)
      if (g[a] % q.cells[a] == 0) a0 = a;
    if (a0 < 0) continue;
    long long off = 0;
#pragma unroll
    for (int b = 0; b < DIM; ++b)
      if (b != a0) off = off * q.N[b] + g[b];
    const int k = g[a0] / q.cells[a0];
    q.u_out[e] = q.B[a0][((long long)k * q.nsteps + (q.nsteps - 1)) * q.plane_elems[a0] + off];
  }
}

// Time levels of one axis's planes: level 0 = the initial data at the nodal
// points, levels 1..t_nodes = the probabilistic values.
template <int DIM>
__global__ void pdd_levels_kernel(const WalkParams p, int axis, double plane_lo, double plane_step, int nplanes,
                                  int t_nodes, int nb, int nc, double lob, double hb, double loc, double hc,
                                  const double *__restrict__ u_nodes, double *__restrict__ V) {
  const long long per = (long long)nb * nc;
  const long long total = (long long)nplanes * (t_nodes + 1) * per;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const long long in_plane = e % per;
    const int lev = (int)((e / per) % (t_nodes + 1));
    const int k = (int)(e / (per * (t_nodes + 1)));
    if (lev > 0) {
      V[e] = u_nodes[((long long)k * t_nodes + (lev - 1)) * per + in_plane];
      continue;
    }
    const int ib = (int)(in_plane / nc), ic = (int)(in_plane % nc);
    double x[3] = {0.0, 0.0, 0.0};
    int col = 0;
#pragma unroll
    for (int b = 0; b < DIM; ++b) {
      if (b == axis) {
        x[b] = plane_lo + (double)k * plane_step;
      } else {
        x[b] = col == 0 ? lob + (double)ib * hb : loc + (double)ic * hc;
        ++col;
      }
    }
    V[e] = u0_at<DIM>(p, x);
  }
}

}  // namespace grt

using grt::DevBuf;

namespace {

constexpr int kPddThreads = 512;
constexpr int kPddMaxAxis = 64;                   // interior nodes per axis of a subdomain (dense DST)
constexpr size_t kPddSmemBytes = 200u * 1024u;    // the four vectors in shared memory up to this size

int grid_for(long long total) {
  long long b = (total + 255) / 256;
  if (b > 152 * 16) b = 152 * 16;
  return (int)(b < 1 ? 1 : b);
}

int check_grid(grt_ctx *c, const grt_pdd_grid *g) {
  if (!g) return c ? c->set_error(GRT_EINVAL, "grid is NULL") : GRT_EINVAL;
  auto bad = [&](const char *m) { return c ? c->set_error(GRT_EINVAL, m) : GRT_EINVAL; };
  if (g->dim < 1 || g->dim > 3) return bad("grid dim must be 1, 2 or 3");
  if (c && g->dim != c->pb.dim) return bad("grid dim differs from the problem's");
  long long mloc = 1;
  for (int a = 0; a < g->dim; ++a) {
    if (!(std::isfinite(g->lo[a]) && std::isfinite(g->hi[a]) && g->hi[a] > g->lo[a]))
      return bad("need finite lo < hi on every axis");
    if (g->sub[a] < 1 || g->sub[a] > 4096) return bad("sub must be in [1, 4096]");
    if (g->cells[a] < 2 || g->cells[a] > kPddMaxAxis + 1) return bad("cells must be in [2, 65]");
    if (g->dim > 1 && (g->nodes[a] < 4 || g->nodes[a] > GRT_SPLINE_MAX_NODES))
      return bad("nodes must be in [4, 256] on every axis");
    mloc *= g->cells[a] - 1;
  }
  if (mloc > GRT_PDD_MAX_LOCAL) return bad("subdomain above GRT_PDD_MAX_LOCAL interior unknowns");
  if (g->t_nodes < 3 || g->t_nodes + 1 > GRT_SPLINE_MAX_NODES) return bad("t_nodes must be in [3, 255]");
  if (!(std::isfinite(g->T) && g->T > 0.0)) return bad("T must be finite and > 0");
  if (g->nsteps < 1 || g->nsteps > 1000000) return bad("nsteps must be in [1, 1e6]");
  return GRT_OK;
}

long long plane_nodal_points(const grt_pdd_grid *g, int a) {
  long long m = 1;
  for (int b = 0; b < g->dim; ++b)
    if (b != a) m *= g->nodes[b];
  return m;
}

}  // namespace

extern "C" {

int grt_pdd_points(const grt_pdd_grid *g, int64_t capacity, double *x, double *t, int64_t *n_out) {
  int rc = check_grid(nullptr, g);
  if (rc != GRT_OK) return rc;
  const int d = g->dim;
  long long total = 0;
  for (int a = 0; a < d; ++a) total += (long long)(g->sub[a] + 1) * g->t_nodes * plane_nodal_points(g, a);
  if (n_out) *n_out = total;
  if (capacity == 0 && !x && !t) return GRT_OK;
  if (capacity < total || !x || !t) return GRT_EINVAL;
  long long e = 0;
  for (int a = 0; a < d; ++a) {
    int others[2] = {0, 0}, no = 0;
    for (int b = 0; b < d; ++b)
      if (b != a) others[no++] = b;
    const long long m = plane_nodal_points(g, a);
    for (int k = 0; k <= g->sub[a]; ++k) {
      const double pa = g->lo[a] + k * (g->hi[a] - g->lo[a]) / g->sub[a];
      for (int j = 1; j <= g->t_nodes; ++j) {
        const double tj = g->T * j / g->t_nodes;
        for (long long i = 0; i < m; ++i) {
          long long r = i;
          double xi[3] = {0, 0, 0};
          xi[a] = pa;
          for (int o = no - 1; o >= 0; --o) {
            const int b = others[o];
            const long long ib = r % g->nodes[b];
            r /= g->nodes[b];
            xi[b] = g->lo[b] + ib * (g->hi[b] - g->lo[b]) / (g->nodes[b] - 1);
          }
          for (int b = 0; b < d; ++b) x[e * d + b] = xi[b];
          t[e] = tj;
          ++e;
        }
      }
    }
  }
  return GRT_OK;
}

int grt_spline_grid(grt_ctx *c, int ndim, const int32_t *n_nodes, const double *lo, const double *hi,
                    const int32_t *n_targets, const double *targets, int64_t batch, const double *d_values,
                    double *d_out, void *stream) {
  if (!c) return GRT_EINVAL;
  if (ndim < 1 || ndim > 4) return c->set_error(GRT_EINVAL, "ndim must be in [1, 4]");
  if (!n_nodes || !lo || !hi || !n_targets || !targets) return c->set_error(GRT_EINVAL, "NULL size or grid array");
  if (batch < 0) return c->set_error(GRT_EINVAL, "batch must be >= 0");
  long long nin = 1, nout = 1, ntot_t = 0, wsize = 0, stage = 0;
  for (int a = 0; a < ndim; ++a) {
    if (n_nodes[a] < 4 || n_nodes[a] > GRT_SPLINE_MAX_NODES)
      return c->set_error(GRT_EINVAL, "n_nodes must be in [4, 256]");
    if (n_targets[a] < 1 || n_targets[a] > (1 << 24)) return c->set_error(GRT_EINVAL, "n_targets must be >= 1");
    if (!(std::isfinite(lo[a]) && std::isfinite(hi[a]) && hi[a] > lo[a]))
      return c->set_error(GRT_EINVAL, "need finite lo < hi");
    nin *= n_nodes[a];
    nout *= n_targets[a];
    ntot_t += n_targets[a];
    wsize += (long long)n_targets[a] * n_nodes[a];
  }
  for (long long i = 0; i < ntot_t; ++i)
    if (!std::isfinite(targets[i])) return c->set_error(GRT_EINVAL, "targets must be finite");
  if (batch == 0) return GRT_OK;
  if (!d_values || !d_out) return c->set_error(GRT_EINVAL, "values and out must be non-NULL");
  // largest intermediate: axes 0..a mapped to targets, the rest still nodes
  {
    long long cur = nin;
    for (int a = 0; a < ndim; ++a) {
      cur = cur / n_nodes[a] * n_targets[a];
      stage = cur > stage ? cur : stage;
    }
  }
  cudaStream_t s = (cudaStream_t)stream;  // NULL: the legacy default stream, as for the solves
  GRT_CUDA(c, cudaSetDevice(c->device));
  const size_t bytes_w = (size_t)(wsize + ntot_t) * sizeof(double);
  const size_t bytes_stage = (size_t)stage * batch * sizeof(double);
  GRT_CUDA(c, c->pdd_scratch.ensure(bytes_w + 2 * bytes_stage + 1024));
  double *W = c->pdd_scratch.as<double>();
  double *dtg = W + wsize;
  double *st0 = dtg + ntot_t;
  double *st1 = st0 + stage * batch;
  GRT_CUDA(c, cudaMemcpyAsync(dtg, targets, ntot_t * sizeof(double), cudaMemcpyHostToDevice, s));
  long long woff = 0, toff = 0;
  std::vector<long long> wo(ndim), to(ndim);
  for (int a = 0; a < ndim; ++a) {
    wo[a] = woff;
    to[a] = toff;
    const double hn = (hi[a] - lo[a]) / (n_nodes[a] - 1);
    grt::launch_spline_weights(n_nodes[a], lo[a], hn, n_targets[a], dtg + toff, W + woff, s);
    woff += (long long)n_targets[a] * n_nodes[a];
    toff += n_targets[a];
  }
  GRT_CUDA(c, cudaGetLastError());
  // axis by axis: [batch * prod(before)] [n_a -> m_a] [prod(after)]
  const double *src = d_values;
  long long before = batch, after = nin;
  for (int a = 0; a < ndim; ++a) {
    after /= n_nodes[a];
    double *dst = (a == ndim - 1) ? d_out : ((a % 2 == 0) ? st0 : st1);
    const long long total = before * n_targets[a] * after;
    grt::axis_apply_kernel<<<grid_for(total), 256, 0, s>>>(W + wo[a], n_targets[a], n_nodes[a], src, dst, before,
                                                           after);
    src = dst;
    before *= n_targets[a];
  }
  GRT_CUDA(c, cudaGetLastError());
  return GRT_OK;
}

int grt_pdd_solve_range(grt_ctx *c, const grt_pdd_grid *g, int64_t sub_begin, int64_t sub_end,
                        const double *d_u_nodes, double *d_u_out, void *stream) {
  if (!c) return GRT_EINVAL;
  int rc = check_grid(c, g);
  if (rc != GRT_OK) return rc;
  long long nsub_all = 1;
  for (int a = 0; a < g->dim; ++a) nsub_all *= g->sub[a];
  if (sub_begin < 0 || sub_end > nsub_all || sub_begin > sub_end)
    return c->set_error(GRT_EINVAL, "need 0 <= sub_begin <= sub_end <= number of subdomains");
  if (c->pb.sde_kind != GRT_SDE_HEAT)
    return c->set_error(GRT_ENOTSUP, "the PDD local solver discretises D Lap: paths must be GRT_SDE_HEAT");
  if (!d_u_nodes || !d_u_out) return c->set_error(GRT_EINVAL, "u_nodes and u_out must be non-NULL");
  const int d = g->dim;
  cudaStream_t s = (cudaStream_t)stream;  // NULL: the legacy default stream, as for the solves
  GRT_CUDA(c, cudaSetDevice(c->device));

  grt::PddDev q{};
  q.dim = d;
  long long nsub = 1;
  q.mloc = 1;
  for (int a = 0; a < 3; ++a) {
    const bool on = a < d;
    q.sub[a] = on ? g->sub[a] : 1;
    q.cells[a] = on ? g->cells[a] : 2;
    q.N[a] = on ? g->sub[a] * g->cells[a] + 1 : 1;
    q.m[a] = on ? g->cells[a] - 1 : 1;
    q.lo[a] = on ? g->lo[a] : 0.0;
    q.h[a] = on ? (g->hi[a] - g->lo[a]) / (double)(g->sub[a] * g->cells[a]) : 1.0;
    q.inv_h2[a] = 1.0 / (q.h[a] * q.h[a]);
    if (on) {
      nsub *= g->sub[a];
      q.mloc *= q.m[a];
    }
  }
  q.nsteps = g->nsteps;
  q.dt = g->T / g->nsteps;
  q.alpha = 0.5 * q.dt * c->pb.D;
  q.f_deg = c->pb.f_deg;
  for (int k = 0; k <= GRT_MAX_DEG; ++k) q.f_coef[k] = k <= c->pb.f_deg ? c->pb.f_coef[k] : 0.0;
  q.coef_pow_mask = c->pb.coef_kind != GRT_COEF_CONST ? c->pb.coef_mask : 0u;

  // scratch layout: weights (time + one per axis), targets, two staging buffers,
  // the per-axis plane arrays, the DST tables, the subdomain vectors (when not in shared memory)
  const int tn = g->t_nodes + 1;
  long long wsz = (long long)g->nsteps * tn, tsz = g->nsteps, stage = 0, bsz = 0;
  long long woff_ax[3] = {0, 0, 0}, toff_ax[3] = {0, 0, 0}, boff[3] = {0, 0, 0};
  for (int a = 0; a < d; ++a) {
    woff_ax[a] = wsz;
    toff_ax[a] = tsz;
    wsz += (long long)q.N[a] * g->nodes[a];
    tsz += q.N[a];
  }
  for (int a = 0; a < d; ++a) {
    const long long np = g->sub[a] + 1;
    long long pn = 1, pf = 1;
    for (int b = 0; b < d; ++b)
      if (b != a) {
        pn *= g->nodes[b];
        pf *= q.N[b];
      }
    q.plane_elems[a] = pf;
    // stages: levels [np][tn][pn] -> [np][nsteps][pn] -> [np][nsteps][N_b][n_c]
    long long s0 = np * tn * pn, s1 = np * g->nsteps * pn, s2 = s1;
    if (d == 3) {
      int bs[2], nb = 0;
      for (int b = 0; b < d; ++b)
        if (b != a) bs[nb++] = b;
      s2 = np * g->nsteps * (long long)q.N[bs[0]] * g->nodes[bs[1]];
    }
    const long long mx = s0 > s1 ? (s0 > s2 ? s0 : s2) : (s1 > s2 ? s1 : s2);
    stage = mx > stage ? mx : stage;
    boff[a] = bsz;
    bsz += np * g->nsteps * pf;
  }
  long long dsz = 0, doff[3] = {0, 0, 0};
  for (int a = 0; a < d; ++a) {
    doff[a] = dsz;
    dsz += (long long)q.m[a] * q.m[a] + q.m[a];
  }
  const long long ioff = dsz;  // the inverse-eigenvalue table follows the DST tables
  dsz += q.mloc;
  const size_t vec_bytes = 4 * (size_t)q.mloc * sizeof(double);
  q.use_smem = vec_bytes <= kPddSmemBytes ? 1 : 0;
  const long long vsz = q.use_smem ? 0 : nsub * 4 * (long long)q.mloc;
  const size_t total = (size_t)(wsz + tsz + 2 * stage + bsz + dsz + vsz) * sizeof(double) + 256;
  GRT_CUDA(c, c->pdd_scratch.ensure(total));
  double *base = c->pdd_scratch.as<double>();
  double *W = base, *tg = W + wsz, *st0 = tg + tsz, *st1 = st0 + stage, *Bb = st1 + stage, *Dt = Bb + bsz;
  double *V = Dt + dsz;
  q.work = V;
  for (int a = 0; a < 3; ++a) {
    q.S[a] = a < d ? Dt + doff[a] : nullptr;
    q.mu[a] = a < d ? Dt + doff[a] + (long long)q.m[a] * q.m[a] : nullptr;
  }
  q.inv_eig = Dt + ioff;
  q.u_out = d_u_out;
  for (int a = 0; a < 3; ++a) q.B[a] = a < d ? Bb + boff[a] : nullptr;

  // target coordinates (host-built, one small copy): t_1..t_N, then each axis's FD nodes
  std::vector<double> ht((size_t)tsz);
  for (int n = 0; n < g->nsteps; ++n) ht[n] = q.dt * (n + 1);
  for (int a = 0; a < d; ++a)
    for (int i = 0; i < q.N[a]; ++i) ht[(size_t)toff_ax[a] + i] = q.lo[a] + i * q.h[a];
  GRT_CUDA(c, cudaMemcpyAsync(tg, ht.data(), ht.size() * sizeof(double), cudaMemcpyHostToDevice, s));
  for (int a = 0; a < d; ++a)
    grt::dst_tables_kernel<<<(q.m[a] * q.m[a] + 127) / 128, 128, 0, s>>>(q.m[a], q.h[a], Dt + doff[a],
                                                                          Dt + doff[a] + (long long)q.m[a] * q.m[a]);
  grt::inv_eig_kernel<<<grid_for(q.mloc), 256, 0, s>>>(d, q.m[0], d > 1 ? q.m[1] : 1, d > 2 ? q.m[2] : 1, q.alpha,
                                                      q.mu[0], d > 1 ? q.mu[1] : q.mu[0], d > 2 ? q.mu[2] : q.mu[0],
                                                      Dt + ioff);
  // weights: time axis (t_nodes + 1 uniform levels over [0, T]) and every space axis
  grt::launch_spline_weights(tn, 0.0, g->T / g->t_nodes, g->nsteps, tg, W, s);
  for (int a = 0; a < d; ++a)
    grt::launch_spline_weights(g->nodes[a], q.lo[a], (g->hi[a] - g->lo[a]) / (g->nodes[a] - 1), q.N[a],
                               tg + toff_ax[a], W + woff_ax[a], s);
  GRT_CUDA(c, cudaGetLastError());

  // spline every axis's planes
  long long in_off = 0;
  for (int a = 0; a < d; ++a) {
    const int np = g->sub[a] + 1;
    int bs[2] = {-1, -1}, nb = 0;
    for (int b = 0; b < d; ++b)
      if (b != a) bs[nb++] = b;
    const int nbn = nb > 0 ? g->nodes[bs[0]] : 1, ncn = nb > 1 ? g->nodes[bs[1]] : 1;
    const double lob = nb > 0 ? q.lo[bs[0]] : 0.0, hb = nb > 0 ? (g->hi[bs[0]] - g->lo[bs[0]]) / (nbn - 1) : 0.0;
    const double loc = nb > 1 ? q.lo[bs[1]] : 0.0, hc = nb > 1 ? (g->hi[bs[1]] - g->lo[bs[1]]) / (ncn - 1) : 0.0;
    const long long pn = (long long)nbn * ncn;
    const long long lev_total = (long long)np * tn * pn;
    const double pstep = (g->hi[a] - g->lo[a]) / g->sub[a];
    switch (d) {
    case 1:
      grt::pdd_levels_kernel<1><<<grid_for(lev_total), 256, 0, s>>>(c->base, a, q.lo[a], pstep, np, g->t_nodes,
                                                                      nbn, ncn, lob, hb, loc, hc, d_u_nodes + in_off,
                                                                      st0);
      break;
    case 2:
      grt::pdd_levels_kernel<2><<<grid_for(lev_total), 256, 0, s>>>(c->base, a, q.lo[a], pstep, np, g->t_nodes,
                                                                      nbn, ncn, lob, hb, loc, hc, d_u_nodes + in_off,
                                                                      st0);
      break;
    default:
      grt::pdd_levels_kernel<3><<<grid_for(lev_total), 256, 0, s>>>(c->base, a, q.lo[a], pstep, np, g->t_nodes,
                                                                      nbn, ncn, lob, hb, loc, hc, d_u_nodes + in_off,
                                                                      st0);
      break;
    }
    in_off += (long long)np * g->t_nodes * pn;
    double *Ba = Bb + boff[a];
    // time: [np][tn][pn] -> [np][nsteps][pn]
    double *dst = nb == 0 ? Ba : st1;
    grt::axis_apply_kernel<<<grid_for((long long)np * g->nsteps * pn), 256, 0, s>>>(W, g->nsteps, tn, st0, dst, np,
                                                                                    pn);
    if (nb >= 1) {
      // first in-plane axis: [np*nsteps][nbn][ncn] -> [np*nsteps][N_b][ncn]
      double *dst2 = nb == 1 ? Ba : st0;
      const long long outer = (long long)np * g->nsteps;
      grt::axis_apply_kernel<<<grid_for(outer * q.N[bs[0]] * ncn), 256, 0, s>>>(W + woff_ax[bs[0]], q.N[bs[0]], nbn,
                                                                                 st1, dst2, outer, ncn);
      if (nb == 2) {
        const long long outer2 = outer * q.N[bs[0]];
        grt::axis_apply_kernel<<<grid_for(outer2 * q.N[bs[1]]), 256, 0, s>>>(W + woff_ax[bs[1]], q.N[bs[1]], ncn,
                                                                             st0, Ba, outer2, 1);
      }
    }
  }
  GRT_CUDA(c, cudaGetLastError());

  // subdomain solves and the plane nodes of the output
  long long ntot = 1;
  for (int a = 0; a < d; ++a) ntot *= q.N[a];
  const size_t smem = q.use_smem ? vec_bytes : 0;
  q.sub_first = (int)sub_begin;
  const long long nrun = sub_end - sub_begin;  // subdomains solved by this call
  // a pair of blocks (a cluster) per subdomain when each half fits in shared memory
  const int h0 = (q.m[0] + 1) / 2;
  const size_t pair_bytes = 4 * (size_t)h0 * (q.mloc / q.m[0]) * sizeof(double);
  const bool pair = q.m[0] >= 2 && pair_bytes <= kPddSmemBytes;
#define GRT_CN_LAUNCH(D)                                                                                          \
  if (pair) {                                                                                                    \
    GRT_CUDA(c, cudaFuncSetAttribute(grt::cn_pair_kernel<D, kPddThreads>,                                        \
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kPddSmemBytes));          \
    if (nrun > 0)                                                                                                \
      grt::cn_pair_kernel<D, kPddThreads><<<(unsigned)(2 * nrun), kPddThreads, pair_bytes, s>>>(c->base, q);     \
  } else {                                                                                                       \
    GRT_CUDA(c, cudaFuncSetAttribute(grt::cn_subdomain_kernel<D, kPddThreads>,                                   \
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kPddSmemBytes));          \
    if (nrun > 0)                                                                                                \
      grt::cn_subdomain_kernel<D, kPddThreads><<<(unsigned)nrun, kPddThreads, smem, s>>>(c->base, q);            \
  }                                                                                                              \
  grt::pdd_planes_kernel<D><<<grid_for(ntot), 256, 0, s>>>(q);
  switch (d) {
  case 1: GRT_CN_LAUNCH(1) break;
  case 2: GRT_CN_LAUNCH(2) break;
  default: GRT_CN_LAUNCH(3) break;
  }
#undef GRT_CN_LAUNCH
  GRT_CUDA(c, cudaGetLastError());
  return GRT_OK;
}

int grt_pdd_solve(grt_ctx *c, const grt_pdd_grid *g, const double *d_u_nodes, double *d_u_out, void *stream) {
  if (!c) return GRT_EINVAL;
  int rc = check_grid(c, g);
  if (rc != GRT_OK) return rc;
  long long nsub_all = 1;
  for (int a = 0; a < g->dim; ++a) nsub_all *= g->sub[a];
  return grt_pdd_solve_range(c, g, 0, nsub_all, d_u_nodes, d_u_out, stream);
}

}  // extern "C"
