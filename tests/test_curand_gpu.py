"""Pin the oracle's Philox4x32-10 against cuRAND's Philox4_32_10 generator, run on the GPU.

curand_init(seed, subsequence, offset) starts the counter at
(offset/4 low, offset/4 high, subsequence low, subsequence high) under the key
(seed low, seed high); curand4() then returns the block of that counter.
"""
import os
import shutil
import subprocess

import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu

SRC = r"""
#include <cstdio>
#include <curand_kernel.h>
__global__ void k(const unsigned long long *seed, const unsigned long long *sub, const unsigned long long *off,
                  uint4 *out, int n) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  curandStatePhilox4_32_10_t s;
  curand_init(seed[i], sub[i], off[i], &s);
  out[i] = curand4(&s);
}
int main() {
  int n;
  if (scanf("%d", &n) != 1 || n <= 0 || n > 4096) return 2;
  unsigned long long *hs = new unsigned long long[3 * n];
  for (int i = 0; i < 3 * n; ++i) if (scanf("%llu", &hs[i]) != 1) return 3;
  unsigned long long *d; uint4 *o;
  if (cudaMalloc(&d, 3 * n * sizeof(unsigned long long)) != cudaSuccess) return 4;
  if (cudaMalloc(&o, n * sizeof(uint4)) != cudaSuccess) return 4;
  cudaMemcpy(d, hs, 3 * n * sizeof(unsigned long long), cudaMemcpyHostToDevice);
  k<<<(n + 127) / 128, 128>>>(d, d + n, d + 2 * n, o, n);
  uint4 *ho = new uint4[n];
  if (cudaMemcpy(ho, o, n * sizeof(uint4), cudaMemcpyDeviceToHost) != cudaSuccess) return 5;
  for (int i = 0; i < n; ++i) printf("%u %u %u %u\n", ho[i].x, ho[i].y, ho[i].z, ho[i].w);
  return 0;
}
"""


def test_philox_matches_curand(tmp_path):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not found")
    src = tmp_path / "cr.cu"
    src.write_text(SRC)
    exe = tmp_path / "cr"
    subprocess.run([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O2", "-o", str(exe), str(src)], check=True)
    rng = np.random.default_rng(2024)
    n = 256
    seeds = rng.integers(0, 2**63, size=n, dtype=np.uint64)
    seeds[0] = 0
    c = rng.integers(0, 2**32, size=(n, 4), dtype=np.uint64)
    c[:, 1] &= 0x3FFFFFFF  # offset = 4 (c1 << 32 | c0) must fit 64 bits
    sub = (c[:, 3] << np.uint64(32)) | c[:, 2]
    off = ((c[:, 1] << np.uint64(32)) | c[:, 0]) * np.uint64(4)
    inp = f"{n}\n" + " ".join(str(int(v)) for v in np.concatenate([seeds, sub, off])) + "\n"
    r = subprocess.run([str(exe)], input=inp, capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stderr
    got = np.array([[int(v) for v in line.split()] for line in r.stdout.strip().splitlines()], dtype=np.uint64)
    for i in range(n):
        key = [int(seeds[i]) & 0xFFFFFFFF, int(seeds[i]) >> 32]
        ref = oracle.philox4x32_10([int(v) for v in c[i]], key)
        assert np.array_equal(ref.astype(np.uint64), got[i]), (i, ref, got[i])
