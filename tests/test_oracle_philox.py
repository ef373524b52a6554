"""Pins of the oracle's counter-based generator (Philox4x32-10, Salmon et al. SC'11).

The paper does not name its generator; both the oracle and the GPU path key every node's draws by
(point, tree, node label) with Philox4x32-10.  The oracle's implementation is
pinned against an independent implementation of the same published
definition (Triton's, run by its CPU interpreter), and by statistics.
"""
import os
import subprocess
import sys
import textwrap

import numpy as np
import pytest


def test_uniform_map_is_exact_and_open(oracle_mod):
    # U(w) = ((w >> 9) + 1/2) 2^-23 lies in (0,1) and is exact in binary32.
    for w in [0, 1, 511, 512, 0x7FFFFFFF, 0x80000000, 0xFFFFFE00, 0xFFFFFFFF]:
        u = oracle_mod.uniform(w)
        assert 0.0 < u < 1.0
        assert float(np.float32(u)) == u
        assert u == ((w >> 9) + 0.5) / 2.0**23
    assert oracle_mod.uniform(0) == 2.0**-24
    assert oracle_mod.uniform(0xFFFFFFFF) == 1.0 - 2.0**-24


_TRITON_SCRIPT = textwrap.dedent(
    """
    import os, sys
    os.environ["TRITON_INTERPRET"] = "1"
    import numpy as np, torch, triton, triton.language as tl

    @triton.jit
    def k(c0p, c1p, c2p, c3p, o0, o1, o2, o3, seed, n: tl.constexpr):
        i = tl.arange(0, n)
        c0 = tl.load(c0p + i); c1 = tl.load(c1p + i); c2 = tl.load(c2p + i); c3 = tl.load(c3p + i)
        r0, r1, r2, r3 = tl.philox(seed, c0, c1, c2, c3)
        tl.store(o0 + i, r0); tl.store(o1 + i, r1); tl.store(o2 + i, r2); tl.store(o3 + i, r3)

    ctr = np.load(sys.argv[1]); seeds = np.load(sys.argv[2])
    n = ctr.shape[0]
    res = []
    for seed in seeds:
        c = [torch.from_numpy(ctr[:, j].astype(np.uint32).view(np.int32).copy()) for j in range(4)]
        o = [torch.zeros(n, dtype=torch.int32) for _ in range(4)]
        k[(1,)](*c, *o, int(seed), n)
        res.append(np.stack([x.numpy().view(np.uint32) for x in o], axis=1))
    np.save(sys.argv[3], np.stack(res))
    """
)


def test_philox_matches_triton_reference_implementation(oracle_mod, tmp_path):
    pytest.importorskip("triton")
    pytest.importorskip("torch")
    rng = np.random.default_rng(12345)
    n = 64
    ctr = rng.integers(0, 2**32, size=(n, 4), dtype=np.uint64)
    ctr[0] = 0
    ctr[1] = 0xFFFFFFFF
    seeds = np.array([0, 1, 0x123456789ABCDEF0, 2**64 - 1], dtype=np.uint64)
    script = tmp_path / "tri.py"
    script.write_text(_TRITON_SCRIPT)
    np.save(tmp_path / "ctr.npy", ctr)
    np.save(tmp_path / "seeds.npy", seeds)
    env = dict(os.environ, TRITON_INTERPRET="1")
    proc = subprocess.run([sys.executable, str(script), str(tmp_path / "ctr.npy"), str(tmp_path / "seeds.npy"),
                           str(tmp_path / "out.npy")], env=env, capture_output=True, text=True, timeout=600)
    if proc.returncode != 0:
        pytest.skip("triton interpreter unavailable: " + proc.stderr[-300:])
    ref = np.load(tmp_path / "out.npy")
    for si, seed in enumerate(seeds):
        key = [int(seed) & 0xFFFFFFFF, int(seed) >> 32]
        for i in range(n):
            got = oracle_mod.philox4x32_10([int(v) for v in ctr[i]], key)
            assert np.array_equal(got, ref[si, i]), (si, i, got, ref[si, i])


def test_philox_bit_balance_and_uniformity(oracle_mod):
    key = [0xDEADBEEF, 0x01234567]
    words = []
    for i in range(1 << 14):
        words.append(oracle_mod.philox4x32_10([i, 0, 7, 3], key))
    w = np.concatenate(words).astype(np.uint64)  # 2^16 words
    n = w.size
    bits = ((w[:, None] >> np.arange(32, dtype=np.uint64)) & 1).sum(axis=0)
    z = (bits - n / 2) / np.sqrt(n / 4)
    assert np.all(np.abs(z) < 5.0), z
    hist = np.bincount((w >> 24).astype(np.int64), minlength=256)
    e = n / 256
    chi2 = ((hist - e) ** 2 / e).sum()
    # chi-square with 255 dof: mean 255, sd ~22.6
    assert chi2 < 255 + 6 * 22.6
    # neighbouring counters must not be correlated
    u = w.astype(np.float64) / 2**32
    r = np.corrcoef(u[:-1], u[1:])[0, 1]
    assert abs(r) < 5 / np.sqrt(n)


def test_philox_key_and_counter_sensitivity(oracle_mod):
    base = oracle_mod.philox4x32_10([1, 2, 3, 4], [5, 6])
    for j in range(4):
        c = [1, 2, 3, 4]
        c[j] ^= 1
        out = oracle_mod.philox4x32_10(c, [5, 6])
        flips = sum(bin(int(a) ^ int(b)).count("1") for a, b in zip(base, out))
        assert 32 < flips < 96  # about half of 128 bits flip
    out = oracle_mod.philox4x32_10([1, 2, 3, 4], [5, 7])
    flips = sum(bin(int(a) ^ int(b)).count("1") for a, b in zip(base, out))
    assert 32 < flips < 96
