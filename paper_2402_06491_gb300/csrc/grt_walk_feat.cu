// grt_walk_feat.cu -- walk instantiations for problems with features
// (Euler-Maruyama paths, variable coefficients): 4 warps per block, the stack
// in shared memory; blocks per SM and queue chunk still follow the config.
#include "grt_walk.cuh"

namespace grt {

template <int FEAT>
static cudaError_t launch_feat_t(bool fp64, int dim, int strategy, const WalkParams &p, const WalkConfig &cfg,
                                 int num_sms, cudaStream_t stream) {
#define GRT_FEAT_CASE(R, D, S) \
  if (dim == D && strategy == S) return launch_walk_t<R, D, S, 4, 0, FEAT>(p, cfg, num_sms, stream);
  if (fp64) {
    const WalkConfig dflt{};
#define GRT_FEAT_CASE64(D, S) \
  if (dim == D && strategy == S) return launch_walk_t<double, D, S, 4, 0, FEAT>(p, dflt, num_sms, stream);
    GRT_FEAT_CASE64(1, kStratA) GRT_FEAT_CASE64(2, kStratA) GRT_FEAT_CASE64(3, kStratA)
    GRT_FEAT_CASE64(1, kStratB) GRT_FEAT_CASE64(2, kStratB) GRT_FEAT_CASE64(3, kStratB)
#undef GRT_FEAT_CASE64
  } else {
    GRT_FEAT_CASE(float, 1, kStratA) GRT_FEAT_CASE(float, 2, kStratA) GRT_FEAT_CASE(float, 3, kStratA)
    GRT_FEAT_CASE(float, 1, kStratB) GRT_FEAT_CASE(float, 2, kStratB) GRT_FEAT_CASE(float, 3, kStratB)
  }
#undef GRT_FEAT_CASE
  return cudaErrorInvalidValue;
}

cudaError_t launch_walk_feat(bool fp64, int dim, int strategy, int feat, const WalkParams &p, const WalkConfig &cfg,
                             int num_sms, cudaStream_t stream) {
  switch (feat) {
  case kFeatEuler: return launch_feat_t<kFeatEuler>(fp64, dim, strategy, p, cfg, num_sms, stream);
  case kFeatVarCoef: return launch_feat_t<kFeatVarCoef>(fp64, dim, strategy, p, cfg, num_sms, stream);
  case kFeatEuler | kFeatVarCoef:
    return launch_feat_t<kFeatEuler | kFeatVarCoef>(fp64, dim, strategy, p, cfg, num_sms, stream);
  default: return cudaErrorInvalidValue;
  }
}

}  // namespace grt
