// grt_launch.h -- internal launch interface between the C-ABI host code and
// the kernels (not part of the public ABI).
#pragma once

#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

namespace grt {

struct WalkParams;

// The binning kernel: tree records -> per-chunk sums.
struct FinalizeParams {
  const void *rec_w;         // [total trees] tree weights (float or double)
  const uint8_t *rec_o;      // [total trees] tree orders (K+1 = pruned)
  const unsigned long long *tree_prefix;  // [n+1] first record slot of each point (multiples of 4)
  const uint32_t *ntrees;    // [n]
  const uint32_t *chunk_prefix;  // [n+1] first binning chunk of each point in this launch (every point has >= 1)
  uint32_t total_chunks;
  double *part;              // per-chunk sums S1, S2, S|W|, count: [slot][4][K+2], slot stride part_stride
  // incremental solves (null / 0 for a one-shot solve):
  const uint32_t *tree_first;  // [n] first tree of this launch's range (a multiple of kBinChunk), null: 0
  const uint32_t *part_slot;   // [n] first chunk slot of the point in `part`, null: chunk_prefix[p]
  size_t part_stride;          // doubles between chunk slots, 0: 4 (K+2)
  int n, K;
  unsigned long long *stats; // [1] splitting events (sum of record orders), [2] pruned trees: added here
};

// Launch shape of the walk kernel (results do not depend on it).
struct WalkConfig {
  int warps = 4;          // warps per block: 4 or 8
  int smem_levels = 0;    // stack levels in shared memory: 0 = all K, 3 = top three (rest local)
  int blocks_per_sm = 0;  // resident blocks per SM to launch (0 = as many as fit)
  uint32_t tile = 512;    // trees per work-queue chunk
};

cudaError_t launch_walk(bool fp64, int dim, int strategy, const WalkParams &p, const WalkConfig &cfg, int num_sms,
                        cudaStream_t stream);
// The FP32 featureless walk, one instantiation per kind of initial data, in each launch shape
// (w: warps per block, s: stack levels in shared memory, 0 = all); grt_walk_u0.cu.
#define GRT_U0_DECL(name)                                                                                  \
  cudaError_t name(int dim, int strategy, const WalkParams &p, const WalkConfig &cfg, int num_sms, \
                   cudaStream_t stream);
GRT_U0_DECL(launch_walk_u0_w4s0)
GRT_U0_DECL(launch_walk_u0_w4s3)
GRT_U0_DECL(launch_walk_u0_w8s0)
GRT_U0_DECL(launch_walk_u0_w8s3)
#undef GRT_U0_DECL
cudaError_t launch_kappa(int n, int K, const uint32_t *chunk_prefix, const uint32_t *ntrees, const double *part,
                         double *kappa, cudaStream_t stream);
cudaError_t launch_pade_error(int n, int K, int L, int M, const double *coef, const double *se, double *err,
                              cudaStream_t stream);
cudaError_t launch_walk_feat(bool fp64, int dim, int strategy, int feat, const WalkParams &p, const WalkConfig &cfg,
                             int num_sms, cudaStream_t stream);
cudaError_t launch_trees(bool fp64, int dim, int strategy, const WalkParams &p, const double *x0, double t0,
                         uint32_t point, uint32_t first, uint32_t ntrees, int32_t *order, double *w, uint32_t *nodes,
                         uint64_t *hash, cudaStream_t stream);
cudaError_t launch_finalize(bool fp64, const FinalizeParams &f, cudaStream_t stream);

// Completion of points from their chunk sums (after the binning, or for a stopped solve): one block
// per point adds the point's chunk sums in chunk order and forms a_n, SE_n and the Pade.
struct CompleteParams {
  int n, K, L, M;
  const double *part;        // chunk sums, slots part_stride doubles apart (0: 4 (K+2))
  size_t part_stride;
  const uint32_t *part_slot; // [n] first chunk slot of each point, or null: chunk_prefix[i]
  const uint32_t *chunk_prefix;  // [n+1] (when part_slot is null)
  const uint32_t *nchunks;   // [n] chunks to add (a stopped solve), or null: those of the whole budget
  const uint32_t *ntrees;    // [n] with nchunks: the trees those chunks hold; else the trees of the launch
  const uint32_t *ntotal;    // [n] whole budget, or null: ntrees
  const uint32_t *tree_first;  // [n] first tree of the launch's range, or null (0); a point whose
                               // range does not reach its budget is left for a later launch
  const uint32_t *out_slot;  // [n] output row, or null: i
  size_t out_stride;         // doubles between coef / se rows (0: K+1)
  double *u, *coef, *se;     // coef / se may be null
  int32_t *status;           // may be null
  int extra_status;          // bits added to every completed point's status
};
cudaError_t launch_complete(const CompleteParams &c, cudaStream_t stream);

// Serving: the chunk sums of one step's (point, tree range) units added to the points' resident
// accumulators, and the points whose budget the range ends completed (one block per unit).
struct FoldParams {
  int n, K, L, M;
  const double *part;            // the step's chunk sums (slots part_stride doubles apart), or null: none
  size_t part_stride;
  const uint32_t *chunk_prefix;  // [n+1] first chunk slot of each unit in part (read only with part)
  double *acc;                   // accumulators: slot k at acc + k acc_stride, compensated sums s [4 (K+2)]
  size_t acc_stride;             // then their compensations c at acc_stride / 2
  const uint32_t *slot;          // [n] accumulator slot = output row of each unit's point
  const uint32_t *tree_first;    // [n] trees already in the accumulator (0: start from zero sums)
  const uint32_t *ntrees;        // [n] trees of the unit's range
  const uint32_t *ntotal;        // [n] the point's N: it completes when tree_first + ntrees == ntotal
  size_t out_stride;             // doubles between coef / se rows
  double *u, *coef, *se;
  int32_t *status;
  int extra_status;              // bits added to every completed point's status
};
cudaError_t launch_fold(const FoldParams &f, cudaStream_t stream);

// The plain FP64 path (grt_plain.cu): one launch per point.
constexpr int kPlainThreads = 128;
struct PlainPoint {
  double x[3];             // the point (entries past dim unused)
  double t;
  uint32_t point;          // random-stream point index
  uint32_t ntrees;
  int K, L, M;
  double *part;            // [blocks][3][K+2] block partials (S1, S2, SA rows; the pruned count in S1's row K+1)
  uint32_t *ticket;        // zero before the launch
  double *u;               // this point's outputs: u, coef [K+1] and se [K+1] (may be null), status (may be null)
  double *coef, *se;
  int32_t *status;
};
cudaError_t launch_plain(int dim, int strategy, const WalkParams &p, const PlainPoint &q, unsigned blocks,
                         cudaStream_t stream);
cudaError_t launch_pade(int n, int K, int L, int M, const double *coef, double *u, int32_t *status,
                        cudaStream_t stream);

}  // namespace grt
