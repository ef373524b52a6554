// grt_walk.cuh -- the persistent random-tree walk kernel and the per-tree
// diagnostic kernel, as templates over the walk precision, the dimension, the
// strategy, the launch shape, the problem's features (kFeatEuler: Euler-
// Maruyama paths; kFeatVarCoef: variable coefficients) and optionally the kind
// of initial data.  Instantiated by grt_walk.cu (no feature: every launch
// shape), grt_walk_u0.cu (FP32, no feature, 4 warps with the stack in shared
// memory: one kernel per kind of initial data), grt_walk_feat.cu (features:
// 4 warps, stack in shared memory) and grt_trees.cu (the diagnostic kernel).
#pragma once
//
// Work decomposition: point p's N_p trees are cut into queue chunks of `tile`
// consecutive trees (the last one ragged; a plan cuts the points at the queue's
// end into shorter chunks, `tile_small`), numbered point by point
// (prefix[p] = first chunk of point p).  Persistent warps take chunks from
// one global counter; inside a warp every lane walks one tree at a time,
// depth-first, with an explicit stack in shared memory.  A lane whose tree
// ends takes the next unstarted tree of the warp's chunk at once (ballot +
// prefix count), and when the chunk is used up the warp fetches the next one
// while the other lanes keep walking: lanes never wait for a warp-mate's tree
// and no lane idles at chunk boundaries.
//
// Each finished tree writes its record (order Ne or K+1 if pruned, weight W)
// to its slot in HBM: rec_o / rec_w [tree_prefix[p] + tree - tree_first[p]],
// held as a 32-bit offset from the launch's rec_base (the host splits a plan
// whose records span 2^32 slots or more into several launches).
// (An incremental solve walks trees tree_first[p] .. tree_first[p] + ntrees[p] - 1
// of point p; a one-shot solve has tree_first = 0.)  The series
// binning of Sec. 2.4 is done from these records by the finalize kernel in a
// fixed order, so results do not depend on which lane walked which tree.
#include "grt_device.cuh"
#include "grt_launch.h"

namespace grt {

// Stack of pending frames, one per split with children still to walk:
// (y[DIM], tau, meta), meta = (tree depth F of the split node << 16) |
// (k << 8) | next digit.  The children's labels are not stored: node labels
// are paths (child j of label id is 16 id + j + 1), so the split node's label
// is the current label's first F hex digits, and its next child's label that
// prefix followed by the digit.  FP32 walks keep a frame as one vector laid
// out [level][lane] -- (y0, y1, tau, meta) for d <= 2; (y0, y1, y2, tau) plus
// a 32-bit meta array for d = 3 -- so a push or a pop is one 16-byte (and for
// d = 3 one 4-byte) shared access per lane, conflict-free across the warp
// whatever the lanes' depths.  FP64 walks lay the fields out field-major
// [field][level][lane].
// SLEV = 0 keeps every level (K of them) in shared memory; SLEV > 0 keeps the
// top SLEV levels there and deeper ones (rare: a frame is pushed only for
// splits of arity >= 2) in per-thread local memory, for more resident warps.
__host__ __device__ inline int smem_levels(int K, int slev) {
  const int k = K > 0 ? K : 1;
  return slev > 0 && slev < k ? slev : k;
}

template <typename Real, int DIM> __host__ __device__ constexpr size_t frame_bytes() {
  return sizeof(Real) == 4 ? (DIM <= 2 ? 16 : 20) : (DIM + 1) * sizeof(Real) + sizeof(uint32_t);
}

template <typename Real, int DIM>
__host__ __device__ inline size_t warp_stack_bytes(int K, int slev) {
  return (((size_t)smem_levels(K, slev) * 32 * frame_bytes<Real, DIM>()) + 15) & ~(size_t)15;
}

// Point owning queue chunk g: the largest p with prefix[p] <= g, found by a
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

// __launch_bounds__(threads, 1): without the minimum-blocks hint ptxas aims at more resident
// blocks and spills some shapes at 40 registers; with it the walk keeps its state in registers
// (48 for the 2-D FP32 kernels, up to 132 for the FP64 ones with features), which is worth more
// than the extra resident warps (measured in every workload)
template <typename Real, int DIM, int STRAT, int WARPS, int SLEV, int FEAT = 0, int U0 = -1>
__global__ void __launch_bounds__(WARPS * 32, 1) walk_kernel(const WalkParams p) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ Real s_factor[kMaxTerms];
  __shared__ int s_arity[kMaxTerms];
  __shared__ uint32_t s_thr[kMaxTerms + 1];
  if (threadIdx.x < kMaxTerms) {
    s_factor[threadIdx.x] = (Real)p.term_factor[threadIdx.x];
    s_arity[threadIdx.x] = p.arity[threadIdx.x];
  }
  if (threadIdx.x <= kMaxTerms) s_thr[threadIdx.x] = p.thr[threadIdx.x];
  __syncthreads();

  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int K = p.K;
  const int lv = smem_levels(K, SLEV);  // shared-memory levels
  unsigned char *wb = smem + (size_t)warp * warp_stack_bytes<Real, DIM>(K, SLEV);
  constexpr int LL = SLEV > 0 ? kMaxK : 1;  // local-memory levels (unused when SLEV = 0)
  Real ly[LL][DIM], ltau[LL];
  uint32_t lnk[LL];
  Real *stk_y = reinterpret_cast<Real *>(wb);             // [DIM][lv][32]
  Real *stk_tau = stk_y + (size_t)DIM * lv * 32;          // [lv][32]
  uint32_t *stk_nk = reinterpret_cast<uint32_t *>(stk_tau + (size_t)lv * 32);
  constexpr bool kVec = sizeof(Real) == 4;                 // FP32: vector frames
  float4 *fr_a = reinterpret_cast<float4 *>(wb);           // [lv][32]
  uint32_t *fr_m = reinterpret_cast<uint32_t *>(wb + (size_t)lv * 32 * sizeof(float4));  // d = 3: [lv][32] meta
  const unsigned lt_mask = (1u << lane) - 1u;

  // warp-uniform: the chunk trees are handed out from
  uint32_t c_next = 0, c_end = 0, c_point = 0, c_first = 0, c_pt = 0;
  uint32_t c_rec = 0;  // record slot of the chunk's first tree, relative to p.rec_base
  Real c_t = Real(0), c_base[DIM];
#pragma unroll
  for (int i = 0; i < DIM; ++i) c_base[i] = Real(0);
  bool exhausted = false;

  // lane: its tree and the tree's point
  bool active = false;
  uint32_t tree = 0, point = 0, pidx = 0;
  uint32_t rec = 0;    // the tree's record slot, relative to p.rec_base
  Real base[DIM];
  // lane: the current node (position, remaining time, label) and the running tree
  Real x[DIM], tau = Real(0), W = Real(1);
  uint32_t id_lo = 0, id_hi = 0;
  int Ne = 0, depth = 0;  // splits so far; pending frames
  uint32_t tdep = 0;      // tree depth of the current node (root 0)
#pragma unroll
  for (int i = 0; i < DIM; ++i) {
    base[i] = Real(0);
    x[i] = Real(0);
  }
  uint32_t nodes = 0;  // nodes this lane visited
  // this lane takes tree c_next + rank of the warp's current chunk
  auto start_tree = [&](uint32_t rank) {
    tree = c_first + c_next + rank;  // the tree's index in its point's stream
    point = c_point;
    pidx = c_pt;
    rec = c_rec + c_next + rank;
#pragma unroll
    for (int i = 0; i < DIM; ++i) {
      base[i] = c_base[i];
      x[i] = Real(0);
    }
    tau = c_t;
    W = Real(1);
    id_lo = 0;
    id_hi = 0;
    Ne = 0;
    depth = 0;
    tdep = 0;
    active = true;
  };

  for (;;) {
    // ---- hand unstarted trees to idle lanes ---------------------------------
    unsigned idle = __ballot_sync(kFull, !active);
    const uint32_t want0 = (uint32_t)__popc(idle);
    // common case: the current chunk has a tree for every idle lane (one pass, no chunk fetch);
    // otherwise the general loop below fetches chunks until every idle lane has a tree
    if (idle != 0u && c_end - c_next >= want0) {
      if (!active) start_tree((uint32_t)__popc(idle & lt_mask));
      c_next += want0;
    } else if (idle != 0u) {
      while (idle != 0u && !exhausted) {
        if (c_next >= c_end) {
          uint32_t item = 0;
          if (lane == 0) item = atomicAdd(p.counter, 1u) + p.item_base;
          item = __shfl_sync(kFull, item, 0);
          if (item >= p.total_items) {
            exhausted = true;
            break;
          }
          const int pt = find_point(p.prefix, p.n, item, lane);
          const uint32_t N = __ldg(p.ntrees + pt);
          const uint32_t tl = (p.tile_small != 0u && pt >= p.small_from) ? p.tile_small : p.tile;
          c_next = (item - __ldg(p.prefix + pt)) * tl;
          c_end = min(c_next + tl, N);
          c_point = p.point_id ? __ldg(p.point_id + pt) : p.point_base + (uint32_t)pt;
          c_first = p.tree_first ? __ldg(p.tree_first + pt) : 0u;
          c_rec = (uint32_t)(__ldg(p.tree_prefix + pt) - p.rec_base);
          c_t = (Real)__ldg(p.t + pt);
          c_pt = (uint32_t)pt;
          double xp[DIM];
#pragma unroll
          for (int i = 0; i < DIM; ++i) xp[i] = __ldg(p.x + (size_t)pt * DIM + i);
          initial_data_base<Real, DIM>(p, xp, c_base);
        }
        const uint32_t avail = c_end - c_next;
        const uint32_t want = (uint32_t)__popc(idle);
        const uint32_t rank = (uint32_t)__popc(idle & lt_mask);
        if (((idle >> lane) & 1u) && rank < avail) start_tree(rank);
        if (avail >= want) {  // every idle lane got a tree
          c_next += want;
          idle = 0u;
        } else {
          c_next = c_end;
          idle = __ballot_sync(kFull, !active);
        }
      }
      if (exhausted) {  // the queue is empty: finish the trees in flight
        if (!__any_sync(kFull, active)) break;
        if (!active) continue;
      }
    }

    // ---- one node -----------------------------------------------------------
    // Straight-line form: the next node is the first child (down), the next
    // pending sibling from the stack (up), or the tree is done.
    ++nodes;
    NodeOut<Real, DIM> o;
    node_step<Real, DIM, STRAT, FEAT, U0>(p, s_factor, s_thr, base, p.x + (size_t)pidx * DIM, x, tau, id_lo, id_hi,
                                          tree, point, o);
    W *= o.factor;
    const bool split = o.cat >= 0;
    Ne += split ? 1 : 0;
    const bool pruned = Ne > K;  // can only become true at a split
    const int k = (split && !pruned) ? s_arity[o.cat] : 0;
    const bool down = k > 0;
    if (k > 1) {  // remember the remaining children 2 .. k: labels 16 id + 2 .. 16 id + k
      const uint32_t meta = (tdep << 16) | ((uint32_t)k << 8) | 2u;
      if (SLEV == 0 || depth < lv) {
        const int at = depth * 32 + lane;
        if constexpr (kVec) {
          if constexpr (DIM <= 2) {
            fr_a[at] = make_float4((float)o.y[0], DIM > 1 ? (float)o.y[DIM - 1] : 0.0f, (float)o.tau_c,
                                   __uint_as_float(meta));
          } else {
            fr_a[at] = make_float4((float)o.y[0], (float)o.y[1], (float)o.y[DIM - 1], (float)o.tau_c);
            fr_m[at] = meta;
          }
        } else {
#pragma unroll
          for (int i = 0; i < DIM; ++i) stk_y[(size_t)i * lv * 32 + at] = o.y[i];
          stk_tau[at] = o.tau_c;
          stk_nk[at] = meta;
        }
      } else {
        const int at = depth - lv;
#pragma unroll
        for (int i = 0; i < DIM; ++i) ly[at][i] = o.y[i];
        ltau[at] = o.tau_c;
        lnk[at] = meta;
      }
      ++depth;
    }
    const bool up = !down && !pruned && depth > 0;
    if (down || up) {
      // the next node: the first child (down) or the next child of the frame on top (up); a frame
      // whose last child this is is popped (its digit is still advanced: the slot is free, and a
      // push overwrites all of it).  nk = (tree depth F of the parent << 16) | (k << 8) | digit:
      // a first child has parent depth tdep and digit 1
      uint32_t nk;
      if (up) {
        const int lvl = depth - 1;
        if (SLEV == 0 || lvl < lv) {
          const int at = lvl * 32 + lane;
          if constexpr (kVec) {
            const float4 a = fr_a[at];
            if constexpr (DIM <= 2) {
              x[0] = (Real)a.x;
              if (DIM > 1) x[DIM - 1] = (Real)a.y;
              tau = (Real)a.z;
              nk = __float_as_uint(a.w);
              reinterpret_cast<uint32_t *>(fr_a)[4 * at + 3] = nk + 1u;
            } else {
              x[0] = (Real)a.x;
              x[1] = (Real)a.y;
              x[DIM - 1] = (Real)a.z;
              tau = (Real)a.w;
              nk = fr_m[at];
              fr_m[at] = nk + 1u;
            }
          } else {
#pragma unroll
            for (int i = 0; i < DIM; ++i) x[i] = stk_y[(size_t)i * lv * 32 + at];
            tau = stk_tau[at];
            nk = stk_nk[at];
            stk_nk[at] = nk + 1u;
          }
        } else {
          const int at = lvl - lv;
#pragma unroll
          for (int i = 0; i < DIM; ++i) x[i] = ly[at][i];
          tau = ltau[at];
          nk = lnk[at];
          lnk[at] = nk + 1u;
        }
        if ((nk & 0xFFu) == ((nk >> 8) & 0xFFu)) --depth;
      } else {
#pragma unroll
        for (int i = 0; i < DIM; ++i) x[i] = o.y[i];
        tau = o.tau_c;
        nk = (tdep << 16) | 1u;
      }
      // the child's label: the parent's label (the current label without its last tdep - F
      // digits; for a first child the current label itself) followed by the child's digit
      const uint32_t F = nk >> 16;
      const uint32_t sh = 4u * (tdep - F);  // 0 .. 64; shr.b64 clamps 64 to an all-zero result
      uint64_t idF;
      asm("shr.b64 %0, %1, %2;" : "=l"(idF) : "l"(((uint64_t)id_hi << 32) | id_lo), "r"(sh));
      id_lo = ((uint32_t)idF << 4) | (nk & 0xFFu);
      id_hi = (uint32_t)(idF >> 28);
      tdep = F + 1u;
    }
    if (!down && !up) {  // leaf with nothing pending, or pruned
      reinterpret_cast<Real *>(p.rec_w)[rec] = pruned ? Real(0) : W;
      p.rec_o[rec] = (uint8_t)(pruned ? K + 1 : Ne);
      active = false;
    }
  }
  // nodes visited by this warp
  unsigned long long tot = nodes;
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) tot += __shfl_xor_sync(kFull, tot, off);
  if (lane == 0) atomicAdd(p.stats, tot);
}

// One thread per tree: per-tree records (diagnostic form of the same streams).
template <typename Real, int DIM, int STRAT, int FEAT>
__global__ void trees_kernel(const WalkParams p, double x0_0, double x0_1, double x0_2, Real t0, uint32_t point,
                             uint32_t first_tree, uint32_t ntrees, int32_t *order, double *wout, uint32_t *nodes_out,
                             uint64_t *hash_out) {
  __shared__ Real s_factor[kMaxTerms];
  __shared__ int s_arity[kMaxTerms];
  __shared__ uint32_t s_thr[kMaxTerms + 1];
  if (threadIdx.x < kMaxTerms) {
    s_factor[threadIdx.x] = (Real)p.term_factor[threadIdx.x];
    s_arity[threadIdx.x] = p.arity[threadIdx.x];
  }
  if (threadIdx.x <= kMaxTerms) s_thr[threadIdx.x] = p.thr[threadIdx.x];
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
    node_step<Real, DIM, STRAT, FEAT>(p, s_factor, s_thr, base, xin, x, tau, (uint32_t)id, (uint32_t)(id >> 32), tree,
                                point, o);
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

// Launch of one instantiation: grid = SMs x resident blocks (or the configured
// blocks per SM), no larger than the queue's warps.
template <typename Real, int DIM, int STRAT, int WARPS, int SLEV, int FEAT = 0, int U0 = -1>
inline cudaError_t launch_walk_t(const WalkParams &p, const WalkConfig &cfg, int num_sms, cudaStream_t stream) {
  const size_t smem = warp_stack_bytes<Real, DIM>(p.K, SLEV) * WARPS;
  auto kern = walk_kernel<Real, DIM, STRAT, WARPS, SLEV, FEAT, U0>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, WARPS * 32, smem);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  if (cfg.blocks_per_sm > 0 && cfg.blocks_per_sm < per_sm) per_sm = cfg.blocks_per_sm;
  long grid = (long)per_sm * num_sms;
  const long need = ((long)(p.total_items - p.item_base) + WARPS - 1) / WARPS;
  if (grid > need) grid = need;
  if (grid < 1) grid = 1;
  kern<<<(unsigned)grid, WARPS * 32, smem, stream>>>(p);
  return cudaGetLastError();
}

}  // namespace grt
