"""The FP32 walk's Box-Muller arithmetic against the device's FP64 library functions, over every
value U = ((w >> 9) + 1/2) 2^-23 the uniform map produces (2^23 of them):

  * -2 ln U: the special-function unit's log2 for U <= 1/2 (its absolute error is then a
    relative one, |log2 U| >= 1), the series 4 atanh(z), z = (1 - U) / (1 + U), above.
    Bound: 4 ulp of the float result everywhere.
  * sin and cos of 2 pi U from the bits of w (octant from the top three bits, near-minimax
    polynomials on [0, pi/4]) and the cosine alone (the third normal in 3-D).  Bound: 2 ulp.
  * the radius sqrt(-2 ln U) as the walk forms it (v rsqrt(v) of the value above).  Bound:
    4 ulp.
"""
import os
import shutil
import subprocess

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2402_06491_gb300", "csrc")

SRC = r"""
#include <cstdio>
#include <cmath>
#include "grt_device.cuh"
__device__ float ulp_err(float f, double ref) {
  const float rf = (float)ref;
  const double ulp = (double)nextafterf(fabsf(rf), INFINITY) - (double)fabsf(rf);
  return (float)(fabs((double)f - ref) / ulp);
}
// err[j][m]: j = 0 -2 ln U, 1 sin 2 pi U, 2 cos 2 pi U, 3 the cosine alone, 4 the radius
__global__ void k(float *err) {
  const unsigned m = blockIdx.x * blockDim.x + threadIdx.x;
  const unsigned n = 1u << 23;
  if (m >= n) return;
  const unsigned w = m << 9;
  const float u = grt::uniform01<float>(w);
  err[m] = ulp_err(grt::Node<float>::neg2ln(u), -2.0 * log((double)u));
  float s, c;
  grt::Node<float>::sincos2pi_w(w, &s, &c);
  double rs, rc;
  sincospi(2.0 * (double)u, &rs, &rc);
  err[n + m] = ulp_err(s, rs);
  err[2 * n + m] = ulp_err(c, rc);
  err[3 * n + m] = ulp_err(grt::Node<float>::cos2pi_w(w), rc);
  err[4 * n + m] = ulp_err(grt::Node<float>::sqrt_pos(grt::Node<float>::neg2ln(u)), sqrt(-2.0 * log((double)u)));
}
int main() {
  const unsigned n = 1u << 23;
  float *d;
  if (cudaMalloc(&d, 5ull * n * sizeof(float)) != cudaSuccess) return 2;
  k<<<n / 256, 256>>>(d);
  float *h = new float[5ull * n];
  if (cudaMemcpy(h, d, 5ull * n * sizeof(float), cudaMemcpyDeviceToHost) != cudaSuccess) return 3;
  for (int j = 0; j < 5; ++j) {
    double mx = 0, sum = 0;
    unsigned at = 0;
    for (unsigned i = 0; i < n; ++i) {
      const float e = h[(size_t)j * n + i];
      sum += e;
      if (e > mx) { mx = e; at = i; }
    }
    printf("%.6f %u %.6f\n", mx, at, sum / n);
  }
  return 0;
}
"""


def test_box_muller_arithmetic_for_every_uniform(tmp_path):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not found")
    src = tmp_path / "ln.cu"
    src.write_text(SRC)
    exe = tmp_path / "ln"
    subprocess.run([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-std=c++17",
                    "--expt-relaxed-constexpr", "-I" + os.path.join(ROOT, "include"), "-I" + CSRC,
                    "-o", str(exe), str(src)], check=True)
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stderr
    rows = [line.split() for line in r.stdout.strip().splitlines()]
    assert len(rows) == 5, r.stdout
    bounds = [("-2 ln U", 4.0), ("sin 2 pi U", 2.0), ("cos 2 pi U", 2.0), ("cos 2 pi U alone", 2.0),
              ("radius", 4.0)]
    for (name, bound), (mx, at, mean) in zip(bounds, rows):
        assert float(mx) <= bound, (name, mx, at)
        assert float(mean) <= 1.0, (name, mean)
