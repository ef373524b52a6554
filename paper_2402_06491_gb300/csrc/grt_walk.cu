// grt_walk.cu -- walk launches: the FP64 walk (default launch shape), and the
// dispatch to the FP32 instantiations per kind of initial data and launch shape
// (grt_walk_u0.cu) and to the feature instantiations (grt_walk_feat.cu).
#include "grt_walk.cuh"

namespace grt {

// The FP32 walk takes the kernel built for its kind of initial data in the configured shape.
static cudaError_t launch_walk_fp32(int dim, int strategy, const WalkParams &p, const WalkConfig &cfg, int num_sms,
                                    cudaStream_t stream) {
  if (cfg.warps == 8 && cfg.smem_levels == 3) return launch_walk_u0_w8s3(dim, strategy, p, cfg, num_sms, stream);
  if (cfg.warps == 8) return launch_walk_u0_w8s0(dim, strategy, p, cfg, num_sms, stream);
  if (cfg.smem_levels == 3) return launch_walk_u0_w4s3(dim, strategy, p, cfg, num_sms, stream);
  return launch_walk_u0_w4s0(dim, strategy, p, cfg, num_sms, stream);
}

cudaError_t launch_walk(bool fp64, int dim, int strategy, const WalkParams &p, const WalkConfig &cfg, int num_sms,
                        cudaStream_t stream) {
  const int feat = walk_features(p);
  if (feat != 0) return launch_walk_feat(fp64, dim, strategy, feat, p, cfg, num_sms, stream);
  if (!fp64) return launch_walk_fp32(dim, strategy, p, cfg, num_sms, stream);
  const WalkConfig dflt{};  // the FP64 walk runs in the default configuration
#define GRT_WALK64_CASE(D, S) \
  if (dim == D && strategy == S) return launch_walk_t<double, D, S, 4, 0>(p, dflt, num_sms, stream);
  GRT_WALK64_CASE(1, kStratA) GRT_WALK64_CASE(2, kStratA) GRT_WALK64_CASE(3, kStratA)
  GRT_WALK64_CASE(1, kStratB) GRT_WALK64_CASE(2, kStratB) GRT_WALK64_CASE(3, kStratB)
#undef GRT_WALK64_CASE
  return cudaErrorInvalidValue;
}

}  // namespace grt
