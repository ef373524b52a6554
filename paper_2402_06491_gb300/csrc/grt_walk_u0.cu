// grt_walk_u0.cu -- the FP32 featureless walk with the kind of initial data
// fixed at compile time, in one launch shape per compilation: build.py
// compiles this file once per shape the walk offers (4 or 8 warps per block,
// the whole stack or its top three levels in shared memory), defining
// GRT_U0_FN (the launch function's name), GRT_U0_WARPS and GRT_U0_SLEV.
// With the kind known, g is straight-line code in the node body, without the
// dispatch on the kind (a few per cent of the walk's time).
#include "grt_walk.cuh"

#ifndef GRT_U0_FN
#define GRT_U0_FN launch_walk_u0_w4s0
#define GRT_U0_WARPS 4
#define GRT_U0_SLEV 0
#endif

namespace grt {

template <int DIM, int STRAT>
static cudaError_t launch_u0_t(const WalkParams &p, const WalkConfig &cfg, int num_sms, cudaStream_t stream) {
  constexpr int W = GRT_U0_WARPS, S = GRT_U0_SLEV;
  switch (p.u0_kind) {
  case kU0Const: return launch_walk_t<float, DIM, STRAT, W, S, 0, kU0Const>(p, cfg, num_sms, stream);
  case kU0Gauss: return launch_walk_t<float, DIM, STRAT, W, S, 0, kU0Gauss>(p, cfg, num_sms, stream);
  case kU0CosProd: return launch_walk_t<float, DIM, STRAT, W, S, 0, kU0CosProd>(p, cfg, num_sms, stream);
  case kU0TanhProd: return launch_walk_t<float, DIM, STRAT, W, S, 0, kU0TanhProd>(p, cfg, num_sms, stream);
  case kU0Logistic: return launch_walk_t<float, DIM, STRAT, W, S, 0, kU0Logistic>(p, cfg, num_sms, stream);
  case kU0GaussAxes: return launch_walk_t<float, DIM, STRAT, W, S, 0, kU0GaussAxes>(p, cfg, num_sms, stream);
  case kU0Quadratic: return launch_walk_t<float, DIM, STRAT, W, S, 0, kU0Quadratic>(p, cfg, num_sms, stream);
  default: return cudaErrorInvalidValue;  // kinds are validated when the context is created
  }
}

cudaError_t GRT_U0_FN(int dim, int strategy, const WalkParams &p, const WalkConfig &cfg, int num_sms,
                      cudaStream_t stream) {
#define GRT_U0_CASE(D, STR) \
  if (dim == D && strategy == STR) return launch_u0_t<D, STR>(p, cfg, num_sms, stream);
  GRT_U0_CASE(1, kStratA) GRT_U0_CASE(2, kStratA) GRT_U0_CASE(3, kStratA)
  GRT_U0_CASE(1, kStratB) GRT_U0_CASE(2, kStratB) GRT_U0_CASE(3, kStratB)
#undef GRT_U0_CASE
  return cudaErrorInvalidValue;
}

}  // namespace grt
