"""The C-ABI library loads, exports every call include/grt.h declares, and validates on the host."""
import ctypes
import os
import re

import numpy as np
import pytest

import workloads

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__

    __graft_entry__.build()
    from paper_2402_06491_gb300 import _binding

    return _binding._load()


def _declared():
    hdr = open(os.path.join(ROOT, "include", "grt.h")).read()
    return sorted(set(re.findall(r"\b(grt_[a-z_]+)\s*\(", hdr)))


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert "grt_solve" in names and "grt_create" in names
    for name in names:
        assert hasattr(lib, name), name
    import paper_2402_06491_gb300 as pkg

    for name in names:
        assert name in pkg.EXPORTED and callable(getattr(pkg, name)), name


def test_library_is_the_in_tree_build(lib):
    import paper_2402_06491_gb300 as pkg

    assert os.path.dirname(pkg.library_path()) == os.path.join(ROOT, "paper_2402_06491_gb300")
    assert os.path.exists(pkg.library_path())


@pytest.mark.parametrize("field,value,needle", [
    ("dim", 4, "dim"), ("D", -1.0, "D must"), ("q", 1.0, "0 < q < 1"), ("q", 0.0, "0 < q < 1"),
    ("strategy", "C", None), ("u0", ("gauss", (0.0, 1.0, 0.0)), "width"),
    ("coef", ("gauss_over_t", (1, 0, 0, 0, 0, 0, 0.0), [2]), "t0"),
    ("sde", (0, (0.0, 0.0), (0.0, 0.0), (1.0, 1.0), (0.0, 0.0)), "sde_steps"),
    ("sde", (5000, (0.0, 0.0), (0.0, 0.0), (1.0, 1.0), (0.0, 0.0)), "sde_steps"),
])
def test_invalid_problems_are_rejected_before_any_device_call(lib, field, value, needle):
    import paper_2402_06491_gb300 as pkg

    pb = workloads.problem_sin_2d()
    pb[field] = value
    if field == "strategy":
        with pytest.raises(KeyError):
            pkg.problem_struct(pb)
        return
    with pytest.raises(pkg.GrtError) as ei:
        pkg.grt_create(pb)
    assert ei.value.code == -1
    assert needle in str(ei.value)


def test_strategy_a_needs_positive_rate(lib):
    import paper_2402_06491_gb300 as pkg

    pb = workloads.problem_kpp_1d()
    pb["lam"] = 0.0
    with pytest.raises(pkg.GrtError) as ei:
        pkg.grt_create(pb)
    assert ei.value.code == -1 and "lambda" in str(ei.value)


def test_null_arguments(lib):
    out = ctypes.c_void_p()
    assert lib.grt_create(None, 0, ctypes.byref(out)) == -1
    assert out.value is None
    lib.grt_destroy(None)
    lib.grt_plan_destroy(None)
    assert lib.grt_solve(None, 0, None, None, None, 0, 0, 0, 0, 0, None, None, None, None) == -1
    assert lib.grt_plan_launches(None) == 0


def test_pdd_points_match_the_oracle_layout(lib):
    # grt_pdd_points is host-only: the nodal points and their order are the oracle's
    import paper_2402_06491_gb300 as pkg
    from oracle import pdd

    for g in (dict(dim=1, lo=[-1.0], hi=[2.0], sub=[3], cells=[4], nodes=[4], t_nodes=3, T=0.7, nsteps=5),
              dict(dim=2, lo=[0.0, -1.0], hi=[3.0, 1.0], sub=[3, 2], cells=[4, 6], nodes=[7, 5], t_nodes=4, T=1.0,
                   nsteps=8),
              dict(dim=3, lo=[0.0] * 3, hi=[4.0] * 3, sub=[4] * 3, cells=[8] * 3, nodes=[17] * 3, t_nodes=4, T=1.0,
                   nsteps=40)):
        x, t = pkg.grt_pdd_points(g)
        xo, to = pdd.points(g)
        assert x.shape == xo.shape and np.allclose(x, xo, rtol=0, atol=1e-14) and np.array_equal(t, to)
    with pytest.raises(pkg.GrtError):
        pkg.grt_pdd_points(dict(dim=2, lo=[0.0, 0.0], hi=[1.0, 1.0], sub=[2, 2], cells=[4, 4], nodes=[3, 5], t_nodes=4,
                                T=1.0, nsteps=4))


def test_host_arrays_pass_in_place_or_as_contiguous_copies(lib):
    # the binding hands the library plain addresses: an array that already has the layout is used in
    # place, anything else (strided, another dtype, a scalar to broadcast) becomes a contiguous copy
    from paper_2402_06491_gb300 import _binding as b

    a = np.arange(6, dtype=np.float64)
    assert b._vec(a, np.float64, 6) is a and b._ptr(a, ctypes.c_double) == a.ctypes.data
    v = b._vec(a[::2], np.float64, 3)
    assert v.flags.c_contiguous and np.array_equal(v, a[::2])
    w = b._vec(a.astype(np.float32), np.float64, 6)
    assert w.dtype == np.float64 and np.array_equal(w, a)
    assert np.array_equal(b._vec(0.5, np.float64, 4), np.full(4, 0.5))
    assert b._ptr(None, ctypes.c_double) is None


def test_server_memory_sizes(lib):
    # host-only: the step buffers grow with the step size, a point's resident state does not
    import paper_2402_06491_gb300 as pkg

    small, large = pkg.grt_server_sizes(1 << 16), pkg.grt_server_sizes(1 << 20)
    assert small["point_bytes"] == large["point_bytes"] == 1436
    assert large["step_bytes"] > small["step_bytes"] > 9 * (1 << 16)
    assert pkg.grt_server_sizes(0) == pkg.grt_server_sizes(1 << 27)
    for bad in (4096, (1 << 31) + 1):
        with pytest.raises(pkg.GrtError):
            pkg.grt_server_sizes(bad)
