// grt_finalize.cu -- per-point reduction of the item partials, series
// coefficients and standard errors (Sec. 2.4, Eq. simplecase_discrete), and
// the FP64 [L/M] Pade approximant at eps = 1 (Sec. 2.1 end, Sec. 2.4).
#include "grt_device.cuh"
#include "grt_launch.h"
#include "grt_pade.cuh"
#include <math_constants.h>

namespace grt {

// Per-order accumulator slot of one binning thread, one 16-byte (float) or
// 32-byte (double) shared-memory access per record.
template <typename Acc> struct alignas(4 * sizeof(Acc)) Acc4 {
  Acc s1, c1, s2, sa;
};

// Four consecutive tree weights (16-byte aligned for float, 32 for double).
__device__ __forceinline__ void load4(const float *p, float (&w)[4]) {
  const float4 v = __ldcs(reinterpret_cast<const float4 *>(p));
  w[0] = v.x;
  w[1] = v.y;
  w[2] = v.z;
  w[3] = v.w;
}
__device__ __forceinline__ void load4(const double *p, double (&w)[4]) {
  const double2 a = __ldcs(reinterpret_cast<const double2 *>(p));
  const double2 b = __ldcs(reinterpret_cast<const double2 *>(p) + 1);
  w[0] = a.x;
  w[1] = a.y;
  w[2] = b.x;
  w[3] = b.y;
}

// a_n = S1_n / N and SE_n = sqrt((S2_n / N - a_n^2) / (N - 1)) (Sec. 2.4, Eq. simplecase_discrete)
// from one point's summed rows tot[stat][row] (S1, S2, S|W|, count; block-shared, complete), the
// FP64 [L/M] Pade at eps = 1, HIGH_PRUNE when more than 1 % of the N trees were pruned, and the
// bits `extra`.  All threads of the block call it (it synchronises).
__device__ __forceinline__ void finish_point(const double (*tot)[kMaxK + 2], double N, int K, int L, int M, double *u,
                                             double *coef, double *se, int32_t *status, int extra, int tid) {
  __shared__ double a[kMaxK + 1];
  if (tid <= K) {
    const double an = N > 0.0 ? tot[0][tid] / N : 0.0;
    const double var = N > 1.0 ? (tot[1][tid] / N - an * an) / (N - 1.0) : 0.0;
    a[tid] = an;
    if (coef) coef[tid] = an;
    if (se) se[tid] = var > 0.0 ? sqrt(var) : 0.0;
  }
  __syncthreads();
  if (tid < 32) {  // the first warp evaluates the Pade together
    int st = 0;
    const double v = pade_value_warp(a, L, M, &st, tid);
    if (tid == 0) {
      const double pruned = tot[3][K + 1];
      st |= extra;
      if (N > 0.0 && pruned > 0.01 * N) st |= 8;  // HIGH_PRUNE
      *u = v;
      if (status) *status = st;
    }
  }
}

// Completion of one point from its per-chunk sums (rows S1, S2, S|W|, count of K+2 entries each;
// chunk slots pstride doubles apart): the first nch chunk sums added in chunk order with
// compensation, then finish_point.  All T threads of the block call it (it synchronises).
__device__ __forceinline__ void complete_point(const double *part0, size_t pstride, uint32_t nch, double N, int K,
                                               int L, int M, double *u, double *coef, double *se, int32_t *status,
                                               int extra, int tid, int T) {
  const int R = K + 2;
  __shared__ double tot[4][kMaxK + 2];
  for (int e = tid; e < 4 * R; e += T) {  // entry (stat, row) adds the point's chunk sums in chunk order
    const double *pp = part0 + e;
    double s = 0.0, c = 0.0;
    for (uint32_t k = 0; k < nch; ++k) kahan_add(s, c, __ldcg(pp + (size_t)k * pstride));
    tot[e / R][e % R] = s - c;
  }
  __syncthreads();
  finish_point(tot, N, K, L, M, u, coef, se, status, extra, tid);
}

// Shape of the binning kernel: threads per block (one block per 8192-record chunk), record groups
// each thread loads before binning them, and the minimum resident blocks in its launch bounds.
constexpr int kBinThreads = 64;
constexpr int kBinGroups = 4;
constexpr int kFinMinBlocks = 16;

// Binning (Sec. 2.4: trees of order n give the n-th series coefficient).
// One block per chunk of kBinChunk consecutive tree records of one point.
// Thread j bins record groups 4j .. 4j+3, 4(j+T) .. 4(j+T)+3, ... of the chunk
// (T = kFinThreads) into its own shared-memory column of per-order sums (S1
// with Kahan compensation, S2, S|W|, count); the columns are added in a fixed order and
// the chunk's sums written to `part`.  A second kernel (complete_kernel, one
// block per point) then adds each point's chunk sums in chunk order, forms a_n
// and SE_n and runs the FP64 Pade: the binning blocks need few registers and
// stay many per SM.  Every result depends only on the records, not on block
// scheduling.
template <typename Acc, int T, int G>
__global__ void __launch_bounds__(T, kFinMinBlocks) finalize_kernel(const FinalizeParams f) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int K = f.K, R = K + 2;  // rows: orders 0..K and the pruned trees
  const uint32_t chunk = blockIdx.x;
  __shared__ int s_pt;
  if (warp == 0) {  // point owning this chunk: largest p with chunk_prefix[p] <= chunk (32-way search)
    int lo = 0, hi = f.n;
    while (hi - lo > 1) {
      const int step = (hi - lo + 31) >> 5;
      const int idx = lo + lane * step;
      const bool ok = (idx < hi) && (__ldg(f.chunk_prefix + idx) <= chunk);
      const int cnt = __popc(__ballot_sync(kFull, ok));
      lo = lo + (cnt - 1) * step;
      hi = min(lo + step, hi);
    }
    if (lane == 0) s_pt = lo;
  }
  // per-thread columns: acc[o * T + tid] = (S1, Kahan compensation of S1, S2, S|W|) for the kept
  // orders o = 0..K; pruned trees (order K+1, weight 0) are only counted, in a register
  Acc4<Acc> *acc = reinterpret_cast<Acc4<Acc> *>(smem);
  for (int r = 0; r <= K; ++r) acc[r * T + tid] = Acc4<Acc>{Acc(0), Acc(0), Acc(0), Acc(0)};
  __shared__ uint32_t s_pruned[T / 32];
  __syncthreads();
  const int pt = s_pt;
  // this chunk's records [r0, r1); r0 is a multiple of 4 (4-aligned point segments, 8192-record chunks)
  const unsigned long long seg = f.tree_prefix[pt];
  const unsigned long long r0 = seg + (unsigned long long)(chunk - f.chunk_prefix[pt]) * kBinChunk;
  const unsigned long long r1 = min(r0 + (unsigned long long)kBinChunk, seg + f.ntrees[pt]);
  const Acc *rw = reinterpret_cast<const Acc *>(f.rec_w);
  uint32_t npruned = 0, osum = 0;  // pruned trees; sum of the orders (= splits, K+1 for a pruned tree)
  auto bin1 = [&](int o, Acc w) {
    osum += (uint32_t)o;
    if (o <= K) {
      const int a = o * T + tid;
      Acc4<Acc> v = acc[a];
      kahan_add(v.s1, v.c1, w);
      v.s2 += w * w;
      v.sa += w < Acc(0) ? -w : w;
      acc[a] = v;
    } else {
      ++npruned;
    }
  };
  auto bin = [&](uint32_t o4, const Acc (&w4)[4], unsigned long long i) {
    if (i + 4 <= r1) {  // a full group (every group but possibly the chunk's last)
#pragma unroll
      for (int q = 0; q < 4; ++q) bin1((int)((o4 >> (8 * q)) & 0xFFu), w4[q]);
    } else {
#pragma unroll
      for (int q = 0; q < 4; ++q)
        if (i + q < r1) bin1((int)((o4 >> (8 * q)) & 0xFFu), w4[q]);
    }
  };
  // thread tid takes record groups r0 + 4 (tid + j T), j = 0, 1, ...: one 32-bit load of four orders
  // and one vector load of four weights per group, G groups loaded before any is binned (enough
  // loads in flight to cover the memory latency), binned in index order
#pragma unroll 1
  for (unsigned long long i0 = r0 + 4ull * tid; i0 < r1; i0 += 4ull * T * G) {
    uint32_t og[G];
    Acc wg[G][4];
#pragma unroll
    for (int g = 0; g < G; ++g) {
      const unsigned long long i = i0 + 4ull * T * g;
      og[g] = 0u;
      wg[g][0] = wg[g][1] = wg[g][2] = wg[g][3] = Acc(0);
      if (i < r1) {
        og[g] = __ldcs(reinterpret_cast<const uint32_t *>(f.rec_o + i));
        load4(rw + i, wg[g]);
      }
    }
#pragma unroll
    for (int g = 0; g < G; ++g) {
      const unsigned long long i = i0 + 4ull * T * g;
      if (i < r1) bin(og[g], wg[g], i);
    }
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    npruned += __shfl_xor_sync(kFull, npruned, off);
    osum += __shfl_xor_sync(kFull, osum, off);
  }
  if (lane == 0) {
    s_pruned[warp] = npruned;
    if (f.stats) {
      atomicAdd(f.stats + 1, (unsigned long long)osum);
      atomicAdd(f.stats + 2, (unsigned long long)npruned);
    }
  }
  __syncthreads();
  // rows in a fixed order: warp w takes rows w, w + T/32, ...; lane l adds
  // columns l, l+32, ... with compensation, then a fixed butterfly over lanes
  const size_t pstride = f.part_stride ? f.part_stride : (size_t)4 * R;
  const uint32_t cfirst = f.tree_first ? f.tree_first[pt] : 0u;
  const uint32_t slot0 = f.part_slot ? f.part_slot[pt] : f.chunk_prefix[pt];
  double *part = f.part + (size_t)(slot0 + cfirst / kBinChunk + (chunk - f.chunk_prefix[pt])) * pstride;
  for (int r = warp; r <= K; r += T / 32) {
    Acc a1 = 0, k1 = 0, a2 = 0, k2 = 0, a3 = 0, k3 = 0;
    for (int j = lane; j < T; j += 32) {
      const Acc4<Acc> v = acc[r * T + j];
      kahan_add(a1, k1, v.s1 - v.c1);
      kahan_add(a2, k2, v.s2);
      kahan_add(a3, k3, v.sa);
    }
    // butterfly in the walk's precision (FP64 arithmetic is scarce on this GPU:
    // it is used once per row, for the conversion)
    Acc d1 = a1 - k1, d2 = a2 - k2, d3 = a3 - k3;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
      d1 += __shfl_xor_sync(kFull, d1, off);
      d2 += __shfl_xor_sync(kFull, d2, off);
      d3 += __shfl_xor_sync(kFull, d3, off);
    }
    if (lane == 0) {
      part[r] = (double)d1;
      part[R + r] = (double)d2;
      part[2 * R + r] = (double)d3;
      part[3 * R + r] = 0.0;
    }
  }
  if (tid == 0) {  // the pruned row: a count only
    uint32_t c = 0;
#pragma unroll
    for (int w = 0; w < T / 32; ++w) c += s_pruned[w];
    part[K + 1] = 0.0;
    part[R + K + 1] = 0.0;
    part[2 * R + K + 1] = 0.0;
    part[3 * R + K + 1] = (double)c;
  }
}

// Completion of the points of a launch from their chunk sums: one block per point.
__global__ void __launch_bounds__(kFinThreads) complete_kernel(const CompleteParams c) {
  const int i = blockIdx.x;
  const int K = c.K;
  const uint32_t slot0 = c.part_slot ? c.part_slot[i] : c.chunk_prefix[i];
  uint32_t nch, N;
  if (c.nchunks) {  // a stopped solve: the chunks binned so far
    nch = c.nchunks[i];
    N = c.ntrees[i];
  } else {
    N = c.ntotal ? c.ntotal[i] : c.ntrees[i];
    const uint32_t first = c.tree_first ? c.tree_first[i] : 0u;
    if (first + c.ntrees[i] != N) return;  // more trees in a later launch: the sums stay resident
    nch = N == 0u ? 1u : (N + kBinChunk - 1) / kBinChunk;
  }
  const size_t pstride = c.part_stride ? c.part_stride : (size_t)4 * (K + 2);
  const size_t ostride = c.out_stride ? c.out_stride : (size_t)(K + 1);
  const size_t row = c.out_slot ? c.out_slot[i] : (size_t)i;
  complete_point(c.part + (size_t)slot0 * pstride, pstride, nch, (double)N, K, c.L, c.M, c.u + row,
                 c.coef ? c.coef + row * ostride : nullptr, c.se ? c.se + row * ostride : nullptr,
                 c.status ? c.status + row : nullptr, c.extra_status, threadIdx.x, kFinThreads);
}

cudaError_t launch_complete(const CompleteParams &c, cudaStream_t stream) {
  if (c.n <= 0) return cudaSuccess;
  complete_kernel<<<(unsigned)c.n, kFinThreads, 0, stream>>>(c);
  return cudaGetLastError();
}

// Serving, one block per (point, tree range) unit of a step.  A point's resident accumulator holds,
// for every entry (stat, row), the compensated sum (s, c) of the chunk sums added so far; the
// unit's chunk sums are added to it in chunk order.  A point's ranges start on its 8192-tree chunk
// boundaries and are walked in tree order, so its chunk sums meet the accumulator in chunk order:
// the same compensated additions, in the same order, as complete_point's loop over all of them, and
// the point's result is the same bits however its trees were split over steps.  A unit whose range
// ends the point's budget completes the point (finish_point) into output row `slot`; otherwise the
// accumulator is written back.
__global__ void __launch_bounds__(kFinThreads) fold_kernel(const FoldParams f) {
  __shared__ double tot[4][kMaxK + 2];
  const int i = blockIdx.x, tid = threadIdx.x;
  const int K = f.K, R = K + 2;
  const uint32_t slot = f.slot[i], first = f.tree_first[i], N = f.ntotal[i];
  const bool last = first + f.ntrees[i] == N;  // block-uniform
  double *as = f.acc + (size_t)slot * f.acc_stride, *ac = as + f.acc_stride / 2;
  const uint32_t c0 = f.part ? f.chunk_prefix[i] : 0u;
  const uint32_t nch = f.part ? f.chunk_prefix[i + 1] - c0 : 0u;
  for (int e = tid; e < 4 * R; e += kFinThreads) {
    double s = 0.0, c = 0.0;
    if (first != 0u) {  // the point's earlier ranges
      s = as[e];
      c = ac[e];
    }
    if (nch > 0u) {
      const double *pp = f.part + (size_t)c0 * f.part_stride + e;
      for (uint32_t k = 0; k < nch; ++k) kahan_add(s, c, __ldcg(pp + (size_t)k * f.part_stride));
    }
    if (last) {
      tot[e / R][e % R] = s - c;
    } else {
      as[e] = s;
      ac[e] = c;
    }
  }
  if (!last) return;
  __syncthreads();
  const size_t os = f.out_stride;
  finish_point(tot, (double)N, K, f.L, f.M, f.u + slot, f.coef ? f.coef + (size_t)slot * os : nullptr,
               f.se ? f.se + (size_t)slot * os : nullptr, f.status ? f.status + slot : nullptr, f.extra_status, tid);
}

cudaError_t launch_fold(const FoldParams &f, cudaStream_t stream) {
  if (f.n <= 0) return cudaSuccess;
  fold_kernel<<<(unsigned)f.n, kFinThreads, 0, stream>>>(f);
  return cudaGetLastError();
}

// One warp per series (pade_value_warp); 4 series per block.
__global__ void pade_kernel(int n, int K, int L, int M, const double *coef, double *u, int32_t *status) {
  __shared__ double s_a[4][kMaxK + 1];
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int i = blockIdx.x * 4 + w;
  if (i >= n) return;  // whole warps leave together
  if (lane <= L + M) s_a[w][lane] = coef[(size_t)i * (K + 1) + lane];
  __syncwarp();
  int st = 0;
  const double v = pade_value_warp(s_a[w], L, M, &st, lane);
  if (lane == 0) {
    u[i] = v;
    if (status) status[i] = st;
  }
}

// First-order statistical error of the Pade value: with the coefficients' standard errors
// SE_j, err = sqrt(sum_j (du/da_j SE_j)^2), du/da_j by central differences of the FP64
// approximant with steps h_j = 1e-6 max(|a_j|, 1e-12 max_i |a_i|) (the sensitivity the
// Wuytack bound of Sec. 2.4 speaks of, made per result).  +inf when an evaluation fails.
// One warp per result: lane j <= L+M forms the central difference of coefficient j, and lane 0
// adds the squared terms in order j = 0, 1, ...
__global__ void pade_error_kernel(int n, int K, int L, int M, const double *coef, const double *se, double *err) {
  const int i = (int)((blockIdx.x * (unsigned)blockDim.x + threadIdx.x) >> 5);
  const int lane = threadIdx.x & 31;
  if (i >= n) return;  // whole warps leave together
  const int nn = L + M;
  double a[kMaxK + 1];
  double amax = 0.0;
  for (int j = 0; j <= nn; ++j) {
    a[j] = coef[(size_t)i * (K + 1) + j];
    amax = fmax(amax, fabs(a[j]));
  }
  double d2 = 0.0;
  bool ok = true;
  if (lane <= nn) {
    const int j = lane;
    const double s = se[(size_t)i * (K + 1) + j];
    if (s != 0.0) {
      const double h = 1e-6 * fmax(fmax(fabs(a[j]), 1e-12 * amax), 1e-300);
      const double aj = a[j];
      int st = 0;
      a[j] = aj + h;
      const double up = pade_value(a, L, M, &st);
      a[j] = aj - h;
      const double um = pade_value(a, L, M, &st);
      const double d = (up - um) / (2.0 * h) * s;
      ok = isfinite(d);
      d2 = d * d;
    }
  }
  const bool all_ok = __all_sync(kFull, ok);
  double acc = 0.0;
  for (int j = 0; j <= nn; ++j) acc += __shfl_sync(kFull, d2, j);
  if (lane == 0) err[i] = all_ok ? sqrt(acc) : CUDART_INF;
}

// Cancellation factor kappa_n = SA_n / |S1_n| (Sec. 2.4: the Monte Carlo mean of a_n is a
// difference of weights of both signs) of each (point, order) from the resident per-chunk
// partial sums of a one-shot solve (part [chunk][4][K+2]: S1, S2, SA, count rows), summed over the
// point's chunks in chunk order with compensation exactly as the binning's last block sums S1.
// 0 where SA = 0 (no tree of that order), +inf where S1 = 0 < SA.
__global__ void kappa_kernel(int n, int K, const uint32_t *__restrict__ chunk_prefix,
                             const uint32_t *__restrict__ ntrees, const double *__restrict__ part,
                             double *__restrict__ kappa) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  const int R = K + 2;
  if (e >= n * (K + 1)) return;
  const int pt = e / (K + 1), r = e % (K + 1);
  const size_t pstride = (size_t)4 * R;
  const uint32_t nt = ntrees[pt];
  const uint32_t nch = nt == 0u ? 1u : (nt + kBinChunk - 1) / kBinChunk;
  const double *pp = part + (size_t)chunk_prefix[pt] * pstride;
  double s1 = 0.0, c1 = 0.0, sa = 0.0, ca = 0.0;
  for (uint32_t k = 0; k < nch; ++k) {
    kahan_add(s1, c1, pp[(size_t)k * pstride + r]);
    kahan_add(sa, ca, pp[(size_t)k * pstride + 2 * R + r]);
  }
  const double S1 = s1 - c1, SA = sa - ca;
  kappa[e] = SA == 0.0 ? 0.0 : (S1 == 0.0 ? CUDART_INF : SA / fabs(S1));
}

cudaError_t launch_kappa(int n, int K, const uint32_t *chunk_prefix, const uint32_t *ntrees, const double *part,
                         double *kappa, cudaStream_t stream) {
  const long long total = (long long)n * (K + 1);
  if (total <= 0) return cudaSuccess;
  kappa_kernel<<<(unsigned)((total + 127) / 128), 128, 0, stream>>>(n, K, chunk_prefix, ntrees, part, kappa);
  return cudaGetLastError();
}

cudaError_t launch_pade_error(int n, int K, int L, int M, const double *coef, const double *se, double *err,
                              cudaStream_t stream) {
  if (n <= 0) return cudaSuccess;
  pade_error_kernel<<<(unsigned)((n + 3) / 4), 128, 0, stream>>>(n, K, L, M, coef, se, err);  // 4 results per block
  return cudaGetLastError();
}

template <typename Acc> static cudaError_t launch_finalize_t(const FinalizeParams &f, cudaStream_t stream) {
  constexpr int T = kBinThreads, G = kBinGroups;
  const size_t smem = (size_t)(f.K + 1) * T * sizeof(Acc4<Acc>);
  auto kern = finalize_kernel<Acc, T, G>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  kern<<<f.total_chunks, T, smem, stream>>>(f);
  return cudaGetLastError();
}

cudaError_t launch_finalize(bool fp64, const FinalizeParams &f, cudaStream_t stream) {
  if (f.n <= 0) return cudaSuccess;
  return fp64 ? launch_finalize_t<double>(f, stream) : launch_finalize_t<float>(f, stream);
}

cudaError_t launch_pade(int n, int K, int L, int M, const double *coef, double *u, int32_t *status,
                        cudaStream_t stream) {
  if (n <= 0) return cudaSuccess;
  pade_kernel<<<(n + 3) / 4, 128, 0, stream>>>(n, K, L, M, coef, u, status);
  return cudaGetLastError();
}

}  // namespace grt
