// grt_launch.h -- internal launch interface between the C-ABI host code and
// the kernels (not part of the public ABI).
#pragma once

#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

namespace grt {

struct WalkParams;

struct FinalizeParams {
  const void *part;          // [items][3][K+1] item sums (float or double)
  const uint32_t *cnt;       // [items][K+3]
  const uint32_t *prefix;    // [n+1]
  const uint32_t *ntrees;    // [n]
  int n, K, L, M;
  double *u;                 // [n]
  double *coef, *se;         // [n][K+1] or null
  int32_t *status;           // [n] or null
  unsigned long long *nodes_pt, *pruned_pt, *splits_pt;  // [n] or null
  uint32_t *counter;         // work-queue head, reset for the next walk
};

cudaError_t launch_walk(bool fp64, int dim, int strategy, const WalkParams &p, int num_sms, cudaStream_t stream,
                        int *grid_out, size_t *smem_out);
cudaError_t launch_trees(bool fp64, int dim, int strategy, const WalkParams &p, const double *x0, double t0,
                         uint32_t point, uint32_t first, uint32_t ntrees, int32_t *order, double *w, uint32_t *nodes,
                         uint64_t *hash, cudaStream_t stream);
cudaError_t launch_finalize(bool fp64, const FinalizeParams &f, cudaStream_t stream);
cudaError_t launch_pade(int n, int K, int L, int M, const double *coef, double *u, int32_t *status,
                        cudaStream_t stream);
size_t walk_smem_per_block(bool fp64, int dim, int K);

}  // namespace grt
