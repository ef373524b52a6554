// grt_trees.cu -- the per-tree diagnostic kernel (grt_trees): one thread per
// tree on the walk's streams, every feature combination.
#include "grt_walk.cuh"

namespace grt {

template <typename Real, int DIM, int STRAT>
static cudaError_t launch_trees_t(const WalkParams &p, const double *x0, double t0, uint32_t point, uint32_t first,
                                  uint32_t ntrees, int32_t *order, double *w, uint32_t *nodes, uint64_t *hash,
                                  cudaStream_t stream) {
  const unsigned threads = 128;
  const unsigned blocks = (ntrees + threads - 1) / threads;
  if (blocks == 0) return cudaSuccess;
  const double a = x0[0], b = DIM > 1 ? x0[1] : 0.0, c = DIM > 2 ? x0[2] : 0.0;
  switch (walk_features(p)) {
  case 0:
    trees_kernel<Real, DIM, STRAT, 0><<<blocks, threads, 0, stream>>>(p, a, b, c, (Real)t0, point, first, ntrees,
                                                                      order, w, nodes, hash);
    break;
  case kFeatEuler:
    trees_kernel<Real, DIM, STRAT, kFeatEuler><<<blocks, threads, 0, stream>>>(p, a, b, c, (Real)t0, point, first,
                                                                               ntrees, order, w, nodes, hash);
    break;
  case kFeatVarCoef:
    trees_kernel<Real, DIM, STRAT, kFeatVarCoef><<<blocks, threads, 0, stream>>>(p, a, b, c, (Real)t0, point, first,
                                                                                 ntrees, order, w, nodes, hash);
    break;
  default:
    trees_kernel<Real, DIM, STRAT, kFeatEuler | kFeatVarCoef><<<blocks, threads, 0, stream>>>(
        p, a, b, c, (Real)t0, point, first, ntrees, order, w, nodes, hash);
    break;
  }
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

}  // namespace grt
