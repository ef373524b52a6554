// grt_host.h -- host-side types shared by the C-ABI translation units
// (context, device buffers, error plumbing).  Not part of the public ABI.
#pragma once

#include <cuda_runtime.h>

#include <cstddef>
#include <string>

#include "grt.h"
#include "grt_device.cuh"
#include "grt_launch.h"

namespace grt {

// A grow-only device allocation.
struct DevBuf {
  void *ptr = nullptr;
  size_t cap = 0;
  cudaError_t ensure(size_t bytes) {
    if (bytes <= cap && ptr) return cudaSuccess;
    if (ptr) cudaFree(ptr);
    ptr = nullptr;
    cap = 0;
    size_t want = bytes < 256 ? 256 : bytes;
    cudaError_t e = cudaMalloc(&ptr, want);
    if (e != cudaSuccess) {
      ptr = nullptr;
      return e;
    }
    cap = want;
    return cudaSuccess;
  }
  void release() {
    if (ptr) cudaFree(ptr);
    ptr = nullptr;
    cap = 0;
  }
  template <typename T> T *as() const { return reinterpret_cast<T *>(ptr); }
};

}  // namespace grt

struct grt_plan;

struct grt_ctx {
  grt_problem pb{};
  int device = 0;
  int num_sms = 0;
  grt::WalkParams base{};
  std::string err;
  cudaStream_t stream = nullptr;
  grt_plan *solve_plan = nullptr;
  grt::WalkConfig solve_cfg{};  // launch shape of grt_solve's walk (grt_set_solve_config)
  grt::DevBuf dx, dt, du, dcoef, dse, dstatus;
  grt::DevBuf pdd_scratch;  // spline weights, staging, plane data and subdomain vectors of the PDD stages
  grt::DevBuf plain_part, plain_ticket;  // block partials and per-point tickets of grt_solve_plain
  int set_error(int code, const std::string &msg) {
    err = msg;
    return code;
  }
  int cuda_error(cudaError_t e, const char *where) {
    err = std::string(where) + ": " + cudaGetErrorString(e);
    return GRT_EDEVICE;
  }
};

#define GRT_CUDA(ctx, expr)                                        \
  do {                                                             \
    cudaError_t e_ = (expr);                                       \
    if (e_ != cudaSuccess) return (ctx)->cuda_error(e_, #expr);    \
  } while (0)
