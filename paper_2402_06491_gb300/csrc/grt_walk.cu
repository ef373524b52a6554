// grt_walk.cu -- walk launches: the featureless walk in every launch shape and
// the dispatch to the feature instantiations (grt_walk_feat.cu).
#include "grt_walk.cuh"

namespace grt {

template <typename Real, int DIM, int STRAT>
static cudaError_t launch_walk_cfg(const WalkParams &p, const WalkConfig &cfg, int num_sms, cudaStream_t stream) {
  if (cfg.warps == 8 && cfg.smem_levels == 3) return launch_walk_t<Real, DIM, STRAT, 8, 3>(p, cfg, num_sms, stream);
  if (cfg.warps == 8) return launch_walk_t<Real, DIM, STRAT, 8, 0>(p, cfg, num_sms, stream);
  if (cfg.smem_levels == 3) return launch_walk_t<Real, DIM, STRAT, 4, 3>(p, cfg, num_sms, stream);
  return launch_walk_t<Real, DIM, STRAT, 4, 0>(p, cfg, num_sms, stream);
}

cudaError_t launch_walk(bool fp64, int dim, int strategy, const WalkParams &p, const WalkConfig &cfg, int num_sms,
                        cudaStream_t stream) {
  const int feat = walk_features(p);
  if (feat != 0) return launch_walk_feat(fp64, dim, strategy, feat, p, cfg, num_sms, stream);
#define GRT_WALK_CASE(R, D, S) \
  if (dim == D && strategy == S) return launch_walk_cfg<R, D, S>(p, cfg, num_sms, stream);
  if (fp64) {  // the FP64 walk runs in the default configuration
    const WalkConfig dflt{};
    if (dim == 1 && strategy == kStratA) return launch_walk_t<double, 1, kStratA, 4, 0>(p, dflt, num_sms, stream);
    if (dim == 2 && strategy == kStratA) return launch_walk_t<double, 2, kStratA, 4, 0>(p, dflt, num_sms, stream);
    if (dim == 3 && strategy == kStratA) return launch_walk_t<double, 3, kStratA, 4, 0>(p, dflt, num_sms, stream);
    if (dim == 1 && strategy == kStratB) return launch_walk_t<double, 1, kStratB, 4, 0>(p, dflt, num_sms, stream);
    if (dim == 2 && strategy == kStratB) return launch_walk_t<double, 2, kStratB, 4, 0>(p, dflt, num_sms, stream);
    if (dim == 3 && strategy == kStratB) return launch_walk_t<double, 3, kStratB, 4, 0>(p, dflt, num_sms, stream);
  } else {
    GRT_WALK_CASE(float, 1, kStratA) GRT_WALK_CASE(float, 2, kStratA) GRT_WALK_CASE(float, 3, kStratA)
    GRT_WALK_CASE(float, 1, kStratB) GRT_WALK_CASE(float, 2, kStratB) GRT_WALK_CASE(float, 3, kStratB)
  }
#undef GRT_WALK_CASE
  return cudaErrorInvalidValue;
}

}  // namespace grt
