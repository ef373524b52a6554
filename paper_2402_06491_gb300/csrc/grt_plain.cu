// grt_plain.cu -- the plain FP64 point solve: one kernel launch per point.
//
// The straightforward GPU form of the method (Sec. 2.1 algorithm, Sec. 2.4
// binning and Pade), kept as the comparison path of the serving figures: for
// one point, thread g of the launch walks trees g, g + G, g + 2G, ... (G
// threads in the grid) one after another in FP64 with a local-memory stack,
// and adds each tree's weight to its own per-order sums (S1 = sum W, S2 =
// sum W^2, SA = sum |W|, order = number of splits; pruned trees, Ne > K, only
// counted).  The sums are then reduced by warp shuffles (a fixed butterfly),
// the warps' partials added in warp order into one partial per block, and the
// last block to finish (ticket) adds the block partials in block order, forms
// a_n = S1/N and SE_n = sqrt((S2/N - a_n^2)/(N - 1)) (Sec. 2.4, Eq.
// simplecase_discrete) and runs the FP64 Pade -- all within the point's one
// launch.  The assignment of trees to threads and every summation order are
// fixed, so a point's result depends only on its inputs and the launch's
// grid, which is a function of N alone.
#include "grt_device.cuh"
#include "grt_launch.h"
#include "grt_pade.cuh"

namespace grt {

template <int DIM, int STRAT, int FEAT>
__global__ void __launch_bounds__(kPlainThreads) plain_kernel(const WalkParams p, const PlainPoint q) {
  __shared__ double s_factor[kMaxTerms];
  __shared__ int s_arity[kMaxTerms];
  __shared__ uint32_t s_thr[kMaxTerms + 1];
  __shared__ double s_warp[kPlainThreads / 32][3][kMaxK + 2];
  __shared__ double s_tot[3][kMaxK + 2];
  __shared__ double s_a[kMaxK + 1];
  __shared__ bool s_last;
  if (threadIdx.x < kMaxTerms) {
    s_factor[threadIdx.x] = p.term_factor[threadIdx.x];
    s_arity[threadIdx.x] = p.arity[threadIdx.x];
  }
  if (threadIdx.x <= kMaxTerms) s_thr[threadIdx.x] = p.thr[threadIdx.x];
  __syncthreads();
  const int K = q.K, R = K + 2;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  double acc1[kMaxK + 1], acc2[kMaxK + 1], acc3[kMaxK + 1];
  for (int o = 0; o <= K; ++o) acc1[o] = acc2[o] = acc3[o] = 0.0;
  uint32_t pruned = 0;

  const double xin[3] = {q.x[0], q.x[1], q.x[2]};
  double base[DIM];
  initial_data_base<double, DIM>(p, xin, base);
  double sy[kMaxK][DIM], stau[kMaxK];
  uint64_t sbase[kMaxK];
  uint32_t snk[kMaxK];
  const uint32_t G = gridDim.x * blockDim.x;
  for (uint32_t tree = blockIdx.x * blockDim.x + threadIdx.x; tree < q.ntrees; tree += G) {
    double x[DIM];
#pragma unroll
    for (int d = 0; d < DIM; ++d) x[d] = 0.0;
    double tau = q.t, W = 1.0;
    uint64_t id = 0;
    int Ne = 0, depth = 0;
    bool cut = false;
    for (;;) {
      NodeOut<double, DIM> o;
      node_step<double, DIM, STRAT, FEAT>(p, s_factor, s_thr, base, xin, x, tau, (uint32_t)id, (uint32_t)(id >> 32),
                                          tree, q.point, o);
      W *= o.factor;
      bool descend = false;
      if (o.cat >= 0) {
        if (++Ne > K) {
          cut = true;
          break;
        }
        const int k = s_arity[o.cat];
        if (k > 0) {
          if (k > 1) {
#pragma unroll
            for (int d = 0; d < DIM; ++d) sy[depth][d] = o.y[d];
            stau[depth] = o.tau_c;
            sbase[depth] = id * 16u;
            snk[depth] = ((uint32_t)k << 8) | 2u;
            ++depth;
          }
#pragma unroll
          for (int d = 0; d < DIM; ++d) x[d] = o.y[d];
          tau = o.tau_c;
          id = id * 16u + 1u;
          descend = true;
        }
      }
      if (!descend) {
        if (depth == 0) break;
        const int at = depth - 1;
#pragma unroll
        for (int d = 0; d < DIM; ++d) x[d] = sy[at][d];
        tau = stau[at];
        const uint32_t nd = snk[at] & 0xFFu;
        id = sbase[at] + nd;
        if (nd == (snk[at] >> 8)) --depth;
        else snk[at] += 1u;
      }
    }
    if (cut) {
      ++pruned;
    } else {
      acc1[Ne] += W;
      acc2[Ne] += W * W;
      acc3[Ne] += fabs(W);
    }
  }

  // warp shuffles (fixed butterfly), then the warps' partials in warp order: one partial per block
  for (int o = 0; o <= K; ++o) {
    double a = acc1[o], b = acc2[o], c = acc3[o];
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
      a += __shfl_xor_sync(kFull, a, off);
      b += __shfl_xor_sync(kFull, b, off);
      c += __shfl_xor_sync(kFull, c, off);
    }
    if (lane == 0) {
      s_warp[warp][0][o] = a;
      s_warp[warp][1][o] = b;
      s_warp[warp][2][o] = c;
    }
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) pruned += __shfl_xor_sync(kFull, pruned, off);
  if (lane == 0) {
    s_warp[warp][0][K + 1] = (double)pruned;
    s_warp[warp][1][K + 1] = 0.0;
    s_warp[warp][2][K + 1] = 0.0;
  }
  __syncthreads();
  double *part = q.part + (size_t)blockIdx.x * 3 * R;
  for (int e = threadIdx.x; e < 3 * R; e += blockDim.x) {
    double s = 0.0;
    for (int w = 0; w < kPlainThreads / 32; ++w) s += s_warp[w][e / R][e % R];
    part[e] = s;
  }
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) s_last = atomicAdd(q.ticket, 1u) == gridDim.x - 1u;
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  // the last block: block partials in block order, coefficients, standard errors, Pade
  for (int e = threadIdx.x; e < 3 * R; e += blockDim.x) {
    double s = 0.0;
    for (uint32_t b = 0; b < gridDim.x; ++b) s += __ldcg(q.part + (size_t)b * 3 * R + e);
    s_tot[e / R][e % R] = s;
  }
  __syncthreads();
  const double N = (double)q.ntrees;
  if (threadIdx.x <= K) {
    const int n = threadIdx.x;
    const double an = N > 0.0 ? s_tot[0][n] / N : 0.0;
    const double var = N > 1.0 ? (s_tot[1][n] / N - an * an) / (N - 1.0) : 0.0;
    s_a[n] = an;
    if (q.coef) q.coef[n] = an;
    if (q.se) q.se[n] = var > 0.0 ? sqrt(var) : 0.0;
  }
  __syncthreads();
  if (threadIdx.x < 32) {  // the first warp evaluates the Pade together
    int st = 0;
    const double u = pade_value_warp(s_a, q.L, q.M, &st, threadIdx.x);
    if (threadIdx.x == 0) {
      if (N > 0.0 && s_tot[0][K + 1] > 0.01 * N) st |= 8;  // HIGH_PRUNE
      *q.u = u;
      if (q.status) *q.status = st;
    }
  }
}

template <int DIM, int STRAT>
static cudaError_t launch_plain_t(const WalkParams &p, const PlainPoint &q, unsigned blocks, cudaStream_t stream) {
  switch (walk_features(p)) {
  case 0: plain_kernel<DIM, STRAT, 0><<<blocks, kPlainThreads, 0, stream>>>(p, q); break;
  case kFeatEuler: plain_kernel<DIM, STRAT, kFeatEuler><<<blocks, kPlainThreads, 0, stream>>>(p, q); break;
  case kFeatVarCoef: plain_kernel<DIM, STRAT, kFeatVarCoef><<<blocks, kPlainThreads, 0, stream>>>(p, q); break;
  default:
    plain_kernel<DIM, STRAT, kFeatEuler | kFeatVarCoef><<<blocks, kPlainThreads, 0, stream>>>(p, q);
    break;
  }
  return cudaGetLastError();
}

cudaError_t launch_plain(int dim, int strategy, const WalkParams &p, const PlainPoint &q, unsigned blocks,
                         cudaStream_t stream) {
  if (blocks == 0) return cudaErrorInvalidValue;
#define GRT_PLAIN_CASE(D, S) \
  if (dim == D && strategy == S) return launch_plain_t<D, S>(p, q, blocks, stream);
  GRT_PLAIN_CASE(1, kStratA) GRT_PLAIN_CASE(2, kStratA) GRT_PLAIN_CASE(3, kStratA)
  GRT_PLAIN_CASE(1, kStratB) GRT_PLAIN_CASE(2, kStratB) GRT_PLAIN_CASE(3, kStratB)
#undef GRT_PLAIN_CASE
  return cudaErrorInvalidValue;
}

}  // namespace grt
