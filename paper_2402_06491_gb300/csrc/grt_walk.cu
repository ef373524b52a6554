// grt_walk.cu -- the persistent random-tree walk kernel.
//
// Work decomposition: point p's N_p trees are cut into items of kTile
// consecutive trees (the last one ragged); items are numbered point by point
// (prefix[p] = first item of point p).  Persistent warps pull items from one
// global counter.  Inside an item every lane walks one tree at a time,
// depth-first, with an explicit stack in shared memory; a lane whose tree
// ends takes the next unstarted tree of the item at once (ballot + prefix
// count), so lanes never wait for a warp-mate's larger tree.
//
// Per-item sums (the series binning of Sec. 2.4): each finished tree leaves
// (order, weight) in a shared record indexed by its tree number; when the item
// is done the warp sums the records in a fixed order (lane l: trees l, l+32,
// ...; then a fixed sum over lanes), so the item's partial sums do not depend
// on which lane walked which tree.  Partials go to global memory; the
// finalize kernel adds them over items in a fixed order.
#include "grt_device.cuh"
#include "grt_launch.h"

namespace grt {

// Shared-memory layout of one warp (bytes).
struct WarpSmem {
  int levels;        // stack levels (max(K, 1))
  size_t stack_bytes, reduce_bytes, rec_w_off, rec_o_off, total;
};

template <typename Real, int DIM>
__host__ __device__ inline WarpSmem warp_smem_layout(int K) {
  WarpSmem L;
  L.levels = K > 0 ? K : 1;
  // stack: y[DIM], tau (Real) + base_lo, base_hi, (k << 8 | next digit) (u32), per level per lane
  L.stack_bytes = (size_t)L.levels * 32 * ((DIM + 1) * sizeof(Real) + 3 * sizeof(uint32_t));
  // reduction area (aliases the stack): 3 stats x (K+2) rows x 33 lanes (Real) + counts
  L.reduce_bytes = (size_t)(K + 2) * 33 * (3 * sizeof(Real) + sizeof(uint32_t));
  size_t a = L.stack_bytes > L.reduce_bytes ? L.stack_bytes : L.reduce_bytes;
  a = (a + 15) & ~(size_t)15;
  L.rec_w_off = a;
  L.rec_o_off = a + (size_t)kTile * sizeof(Real);
  L.total = (L.rec_o_off + (size_t)kTile + 15) & ~(size_t)15;
  return L;
}

// Point owning work item g: the largest p with prefix[p] <= g, found by a
// 32-way search (one probe per lane per round).
__device__ __forceinline__ int find_point(const uint32_t *__restrict__ prefix, int n, uint32_t g, int lane) {
  int lo = 0, hi = n;
  while (hi - lo > 1) {
    const int step = (hi - lo + 31) >> 5;
    const int idx = lo + lane * step;
    const bool ok = (idx < hi) && (__ldg(prefix + idx) <= g);
    const int cnt = __popc(__ballot_sync(kFull, ok));
    lo = lo + (cnt - 1) * step;
    hi = min(lo + step, hi);
  }
  return lo;
}

template <typename Real, int DIM, int STRAT>
__global__ void __launch_bounds__(kWarpsPerBlock * 32) walk_kernel(const WalkParams p) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ Real s_factor[kMaxTerms];
  __shared__ int s_arity[kMaxTerms];
  if (threadIdx.x < kMaxTerms) {
    s_factor[threadIdx.x] = (Real)p.term_factor[threadIdx.x];
    s_arity[threadIdx.x] = p.arity[threadIdx.x];
  }
  __syncthreads();

  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int K = p.K;
  const WarpSmem Lw = warp_smem_layout<Real, DIM>(K);
  unsigned char *wb = smem + (size_t)warp * Lw.total;
  const int lv = Lw.levels;
  Real *stk_y = reinterpret_cast<Real *>(wb);             // [DIM][lv][32]
  Real *stk_tau = stk_y + (size_t)DIM * lv * 32;          // [lv][32]
  uint32_t *stk_lo = reinterpret_cast<uint32_t *>(stk_tau + (size_t)lv * 32);
  uint32_t *stk_hi = stk_lo + lv * 32;
  uint32_t *stk_nk = stk_hi + lv * 32;
  Real *rec_w = reinterpret_cast<Real *>(wb + Lw.rec_w_off);
  uint8_t *rec_o = wb + Lw.rec_o_off;
  const unsigned lt_mask = (1u << lane) - 1u;
  const int cstride = K + 3;
  const int pstride = 3 * (K + 1);

  for (;;) {
    uint32_t item = 0;
    if (lane == 0) item = atomicAdd(p.counter, 1u);
    item = __shfl_sync(kFull, item, 0);
    if (item >= p.total_items) break;

    const int pt = find_point(p.prefix, p.n, item, lane);
    const uint32_t first = (item - __ldg(p.prefix + pt)) * (uint32_t)kTile;
    const uint32_t N = __ldg(p.ntrees + pt);
    const int ntr = (int)min((uint32_t)kTile, N - first);
    Real base[DIM];
    {
      double xp[DIM];
#pragma unroll
      for (int i = 0; i < DIM; ++i) xp[i] = __ldg(p.x + (size_t)pt * DIM + i);
      initial_data_base<Real, DIM>(p, xp, base);
    }
    const Real t0 = (Real)__ldg(p.t + pt);
    const uint32_t point = p.point_base + (uint32_t)pt;

    // lane state: the current node and the running tree
    int tree = lane;
    bool active = tree < ntr;
    Real x[DIM], tau = t0, W = Real(1);
    uint64_t id = 0;
    int Ne = 0, depth = 0;
#pragma unroll
    for (int i = 0; i < DIM; ++i) x[i] = Real(0);
    int next = 32;
    uint32_t nodes = 0;

    while (__any_sync(kFull, active)) {
      bool done = false, pruned = false;
      if (active) {
        ++nodes;
        NodeOut<Real, DIM> o;
        node_step<Real, DIM, STRAT>(p, s_factor, base, x, tau, id, first + (uint32_t)tree, point, o);
        W *= o.factor;
        bool descend = false;
        if (o.cat >= 0) {
          ++Ne;
          if (Ne > K) {
            pruned = true;
            done = true;
          } else {
            const int k = s_arity[o.cat];
            if (k > 0) {
              if (k > 1) {  // remember the remaining children k-1 .. k
                const int at = depth * 32 + lane;
#pragma unroll
                for (int i = 0; i < DIM; ++i) stk_y[(size_t)i * lv * 32 + at] = o.y[i];
                stk_tau[at] = o.tau_c;
                const uint64_t child0 = id * 16u;  // children of id are child0 + 1 .. child0 + k
                stk_lo[at] = (uint32_t)child0;
                stk_hi[at] = (uint32_t)(child0 >> 32);
                stk_nk[at] = ((uint32_t)k << 8) | 2u;
                ++depth;
              }
#pragma unroll
              for (int i = 0; i < DIM; ++i) x[i] = o.y[i];
              tau = o.tau_c;
              id = id * 16u + 1u;
              descend = true;
            }
          }
        }
        if (!descend && !done) {  // leaf (or arity-0 split): continue with the next pending sibling
          if (depth == 0) {
            done = true;
          } else {
            const int at = (depth - 1) * 32 + lane;
#pragma unroll
            for (int i = 0; i < DIM; ++i) x[i] = stk_y[(size_t)i * lv * 32 + at];
            tau = stk_tau[at];
            const uint32_t nk = stk_nk[at];
            const uint32_t nd = nk & 0xFFu;
            id = (((uint64_t)stk_hi[at] << 32) | stk_lo[at]) + nd;
            if (nd == (nk >> 8)) --depth;
            else stk_nk[at] = nk + 1u;
          }
        }
        if (done) {
          rec_w[tree] = pruned ? Real(0) : W;
          rec_o[tree] = (uint8_t)(pruned ? K + 1 : Ne);
        }
      }
      const unsigned dm = __ballot_sync(kFull, done);
      if (dm) {
        if (done) {
          tree = next + __popc(dm & lt_mask);
          active = tree < ntr;
          if (active) {
#pragma unroll
            for (int i = 0; i < DIM; ++i) x[i] = Real(0);
            tau = t0;
            W = Real(1);
            id = 0;
            Ne = 0;
            depth = 0;
          }
        }
        next += __popc(dm);
      }
    }
    __syncwarp();

    // ---- deterministic per-item order sums ---------------------------------
    Real *acc = reinterpret_cast<Real *>(wb);                 // [3][K+2][33]
    uint32_t *acn = reinterpret_cast<uint32_t *>(acc + (size_t)3 * (K + 2) * 33);  // [K+2][33]
    const int rows = (K + 2) * 33;
    for (int i = lane; i < 3 * rows; i += 32) acc[i] = Real(0);
    for (int i = lane; i < rows; i += 32) acn[i] = 0u;
    __syncwarp();
    for (int i = lane; i < ntr; i += 32) {
      const int o = rec_o[i];
      const Real wv = rec_w[i];
      const int a = o * 33 + lane;
      if (o <= K) {
        acc[a] += wv;
        acc[rows + a] += wv * wv;
        acc[2 * rows + a] += Math<Real>::abs(wv);
      }
      acn[a] += 1u;
    }
    __syncwarp();
    if (lane < K + 2) {
      Real s0 = Real(0), s1 = Real(0), s2 = Real(0);
      uint32_t c = 0;
      const int r = lane * 33;
#pragma unroll 8
      for (int l = 0; l < 32; ++l) {
        s0 += acc[r + l];
        s1 += acc[rows + r + l];
        s2 += acc[2 * rows + r + l];
        c += acn[r + l];
      }
      if (lane <= K) {
        Real *pp = reinterpret_cast<Real *>(p.part) + (size_t)item * pstride;
        pp[lane] = s0;
        pp[K + 1 + lane] = s1;
        pp[2 * (K + 1) + lane] = s2;
      }
      p.cnt[(size_t)item * cstride + lane] = c;
    }
    uint32_t tot = nodes;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) tot += __shfl_xor_sync(kFull, tot, off);
    if (lane == 0) p.cnt[(size_t)item * cstride + K + 2] = tot;
    __syncwarp();
  }
}

// One thread per tree: per-tree records (diagnostic form of the same streams).
template <typename Real, int DIM, int STRAT>
__global__ void trees_kernel(const WalkParams p, double x0_0, double x0_1, double x0_2, Real t0, uint32_t point,
                             uint32_t first_tree, uint32_t ntrees, int32_t *order, double *wout, uint32_t *nodes_out,
                             uint64_t *hash_out) {
  __shared__ Real s_factor[kMaxTerms];
  __shared__ int s_arity[kMaxTerms];
  if (threadIdx.x < kMaxTerms) {
    s_factor[threadIdx.x] = (Real)p.term_factor[threadIdx.x];
    s_arity[threadIdx.x] = p.arity[threadIdx.x];
  }
  __syncthreads();
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= ntrees) return;
  const int K = p.K;
  Real sy[kMaxK][DIM], stau[kMaxK];
  uint64_t sbase[kMaxK];
  uint32_t snk[kMaxK];
  const double xin[3] = {x0_0, x0_1, x0_2};
  Real base[DIM], x[DIM];
  initial_data_base<Real, DIM>(p, xin, base);
#pragma unroll
  for (int d = 0; d < DIM; ++d) x[d] = Real(0);
  Real tau = t0, W = Real(1);
  uint64_t id = 0, h = 0xCBF29CE484222325ull;
  int Ne = 0, depth = 0;
  uint32_t nodes = 0;
  bool pruned = false;
  const uint32_t tree = first_tree + i;
  for (;;) {
    ++nodes;
    NodeOut<Real, DIM> o;
    node_step<Real, DIM, STRAT>(p, s_factor, base, x, tau, id, tree, point, o);
    h = (h ^ (uint64_t)(o.cat + 1)) * 0x100000001B3ull;
    W *= o.factor;
    bool descend = false;
    if (o.cat >= 0) {
      if (++Ne > K) {
        pruned = true;
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
  if (order) order[i] = pruned ? K + 1 : Ne;
  if (wout) wout[i] = pruned ? 0.0 : (double)W;
  if (nodes_out) nodes_out[i] = nodes;
  if (hash_out) hash_out[i] = h;
}

// ---------------------------------------------------------------------------
// host-side launch helpers
// ---------------------------------------------------------------------------
template <typename Real, int DIM, int STRAT>
static cudaError_t launch_walk_t(const WalkParams &p, int num_sms, cudaStream_t stream, int *grid_out,
                                 size_t *smem_out) {
  const WarpSmem Lw = warp_smem_layout<Real, DIM>(p.K);
  const size_t smem = Lw.total * kWarpsPerBlock;
  auto kern = walk_kernel<Real, DIM, STRAT>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kWarpsPerBlock * 32, smem);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  long grid = (long)per_sm * num_sms;
  const long need = ((long)p.total_items + kWarpsPerBlock - 1) / kWarpsPerBlock;
  if (grid > need) grid = need;
  if (grid < 1) grid = 1;
  if (grid_out) *grid_out = (int)grid;
  if (smem_out) *smem_out = smem;
  kern<<<(unsigned)grid, kWarpsPerBlock * 32, smem, stream>>>(p);
  return cudaGetLastError();
}

cudaError_t launch_walk(bool fp64, int dim, int strategy, const WalkParams &p, int num_sms, cudaStream_t stream,
                        int *grid_out, size_t *smem_out) {
#define GRT_WALK_CASE(R, D, S) \
  if (dim == D && strategy == S) return launch_walk_t<R, D, S>(p, num_sms, stream, grid_out, smem_out);
  if (fp64) {
    GRT_WALK_CASE(double, 1, kStratA) GRT_WALK_CASE(double, 2, kStratA) GRT_WALK_CASE(double, 3, kStratA)
    GRT_WALK_CASE(double, 1, kStratB) GRT_WALK_CASE(double, 2, kStratB) GRT_WALK_CASE(double, 3, kStratB)
  } else {
    GRT_WALK_CASE(float, 1, kStratA) GRT_WALK_CASE(float, 2, kStratA) GRT_WALK_CASE(float, 3, kStratA)
    GRT_WALK_CASE(float, 1, kStratB) GRT_WALK_CASE(float, 2, kStratB) GRT_WALK_CASE(float, 3, kStratB)
  }
#undef GRT_WALK_CASE
  return cudaErrorInvalidValue;
}

template <typename Real, int DIM, int STRAT>
static cudaError_t launch_trees_t(const WalkParams &p, const double *x0, double t0, uint32_t point, uint32_t first,
                                  uint32_t ntrees, int32_t *order, double *w, uint32_t *nodes, uint64_t *hash,
                                  cudaStream_t stream) {
  const unsigned threads = 128;
  const unsigned blocks = (ntrees + threads - 1) / threads;
  if (blocks == 0) return cudaSuccess;
  trees_kernel<Real, DIM, STRAT><<<blocks, threads, 0, stream>>>(
      p, x0[0], DIM > 1 ? x0[1] : 0.0, DIM > 2 ? x0[2] : 0.0, (Real)t0, point, first, ntrees,
      order, w, nodes, hash);
  return cudaGetLastError();
}

cudaError_t launch_trees(bool fp64, int dim, int strategy, const WalkParams &p, const double *x0, double t0,
                         uint32_t point, uint32_t first, uint32_t ntrees, int32_t *order, double *w, uint32_t *nodes,
                         uint64_t *hash, cudaStream_t stream) {
#define GRT_TREES_CASE(R, D, S) \
  if (dim == D && strategy == S) \
    return launch_trees_t<R, D, S>(p, x0, t0, point, first, ntrees, order, w, nodes, hash, stream);
  if (fp64) {
    GRT_TREES_CASE(double, 1, kStratA) GRT_TREES_CASE(double, 2, kStratA) GRT_TREES_CASE(double, 3, kStratA)
    GRT_TREES_CASE(double, 1, kStratB) GRT_TREES_CASE(double, 2, kStratB) GRT_TREES_CASE(double, 3, kStratB)
  } else {
    GRT_TREES_CASE(float, 1, kStratA) GRT_TREES_CASE(float, 2, kStratA) GRT_TREES_CASE(float, 3, kStratA)
    GRT_TREES_CASE(float, 1, kStratB) GRT_TREES_CASE(float, 2, kStratB) GRT_TREES_CASE(float, 3, kStratB)
  }
#undef GRT_TREES_CASE
  return cudaErrorInvalidValue;
}

size_t walk_smem_per_block(bool fp64, int dim, int K) {
  const auto f = [&](auto real_tag) -> size_t {
    using R = decltype(real_tag);
    switch (dim) {
    case 1: return warp_smem_layout<R, 1>(K).total * kWarpsPerBlock;
    case 2: return warp_smem_layout<R, 2>(K).total * kWarpsPerBlock;
    default: return warp_smem_layout<R, 3>(K).total * kWarpsPerBlock;
    }
  };
  return fp64 ? f(double()) : f(float());
}

}  // namespace grt
