"""CPU checks of the C ABI: the library builds for sm_103a, loads, exports
every symbol declared in include/rbe.h and validates arguments on the host."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    from paper_2204_13595_gb300 import build, rbe
    build.build()
    return rbe.lib()


def _declared():
    src = open(os.path.join(ROOT, "include", "rbe.h")).read()
    return sorted(set(re.findall(r"\b(rbe_[a-z_]+)\s*\(", src)))


def test_exports_every_declared_symbol(L):
    names = _declared()
    assert len(names) >= 15
    for n in names:
        assert hasattr(L, n), n
    from paper_2204_13595_gb300 import rbe
    assert sorted(rbe.EXPORTS) == names


def test_create_validates_parameters(L):
    h = ctypes.c_void_p()
    # r_s > L/2, r_c >= r_s, alpha <= 0, p < 1, P < 1 are rejected on the host
    for args in [(20.0, 0.3, 2.5, 10.5, 10, 100), (20.0, 0.3, 5.0, 5.0, 10, 100), (20.0, 0.0, 2.5, 5.0, 10, 100),
                 (20.0, 0.3, 2.5, 5.0, 0, 100), (20.0, 0.3, 2.5, 5.0, 10, 0)]:
        assert L.rbe_create(ctypes.byref(h), *args, 1) == -1
        assert not h.value
    assert L.rbe_create(ctypes.byref(h), 20.0, 0.3, 2.5, 5.0, 10, 100, 1) == 0
    info = (ctypes.c_double * 7)()
    assert L.rbe_get_info(h, info, 7) == 0
    # cells of edge >= r_c (Sec. 2.3), reach floor(r_s/w)+1, S = H^3 - 1
    assert info[0] == 8 and info[1] == 3
    import oracle
    assert info[3] == oracle.S(0.3, 20.0)
    assert L.rbe_set_precision(h, 7) == -1
    assert L.rbe_set_lj(h, 17, None, None, 0) == -1
    assert L.rbe_forces(h, 0, 0, None, None, None, None, None, None, None, None) == -1
    L.rbe_destroy(h)


def test_parameter_tables_match_oracle_definitions(L):
    """Cells per axis, stencil reach and S agree with the oracle's independent
    derivation for the configured workloads."""
    import oracle
    from paper_2204_13595_gb300 import systems
    for s in (systems.electrolyte(n=200, L=20.0), systems.water(1000, seed=1)):
        h = ctypes.c_void_p()
        assert L.rbe_create(ctypes.byref(h), s.L, s.alpha, s.r_c, s.r_s, s.p, s.P, 1) == 0
        info = (ctypes.c_double * 7)()
        L.rbe_get_info(h, info, 7)
        assert info[0] == oracle.n_cell(s.L, s.r_c)
        M, H, T = oracle.k_table(s.alpha, s.L)
        assert info[2] == M and info[3] == oracle.S(s.alpha, s.L)
        L.rbe_destroy(h)


def test_binding_argument_counts_match_header(L):
    """Every ctypes prototype set by the binding has as many arguments as the
    header's declaration (a mismatch would pass garbage through the ABI)."""
    src = open(os.path.join(ROOT, "include", "rbe.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    protos = dict(re.findall(r"\b(rbe_[a-z_]+)\s*\(([^;{)]*)\)\s*;", src))
    assert len(protos) >= 25
    for name, params in protos.items():
        params = params.strip()
        n = 0 if params in ("", "void") else params.count(",") + 1
        fn = getattr(L, name)
        assert fn.argtypes is not None, name
        assert len(fn.argtypes) == n, (name, len(fn.argtypes), n)


def test_batch_create_validates_contexts(L):
    hb = ctypes.c_void_p()
    assert L.rbe_batch_create(ctypes.byref(hb), 0, None) == -1
    h = ctypes.c_void_p()
    assert L.rbe_create(ctypes.byref(h), 20.0, 0.3, 2.5, 5.0, 10, 100, 1) == 0
    arr = (ctypes.c_void_p * 2)(h.value, h.value)
    assert L.rbe_batch_create(ctypes.byref(hb), 2, arr) == -1       # the same context twice
    arr1 = (ctypes.c_void_p * 1)(h.value)
    assert L.rbe_batch_create(ctypes.byref(hb), 1, arr1) == 0
    info = (ctypes.c_double * 7)()
    assert L.rbe_batch_info(hb, info, 7) == 0 and info[0] == 1
    assert L.rbe_batch_forces(hb, 0, None, None) == -1                 # not bound
    L.rbe_batch_destroy(hb)
    assert L.rbe_set_rbl_tiling(h, -1, 0) == -1
    assert L.rbe_set_rbl_tiling(h, 32, 2) == 0
    L.rbe_destroy(h)


def test_rho_noalloc_binding_rejects_bad_tensors():
    """The binding refuses, before any call into the library, tensors that
    rbe_rho_noalloc would read or write as the wrong type or size."""
    import torch

    from paper_2204_13595_gb300 import rbe
    n, P = 6, 4
    good = dict(pos=torch.zeros((n, 3), dtype=torch.float64), q=torch.zeros(n, dtype=torch.float64),
                m=torch.ones((P, 3), dtype=torch.int32), rho=torch.zeros((P, 2), dtype=torch.float64))
    bad = [
        dict(rho=torch.zeros((P, 2), dtype=torch.float32)),       # float32 rho
        dict(rho=torch.zeros((P - 1, 2), dtype=torch.float64)),   # fewer rows than k vectors
        dict(m=torch.ones((P, 3), dtype=torch.int64)),            # int64 m (torch.tensor of ints)
        dict(m=torch.ones((P, 2), dtype=torch.int32)),            # wrong m shape
        dict(pos=torch.zeros((n, 3), dtype=torch.float32)),       # float32 pos
        dict(pos=torch.zeros((3, n), dtype=torch.float64).t()),   # non-contiguous pos
        dict(q=torch.zeros(n - 1, dtype=torch.float64)),          # q and pos differ in length
        dict(q=torch.zeros((n, 1), dtype=torch.float64)),         # 2-D q
        dict(pos=[[0.0, 0.0, 0.0]] * n),                          # not a tensor
        {},                                                       # CPU tensors: not on a CUDA device
    ]
    for change in bad:
        args = dict(good, **change)
        with pytest.raises(rbe.RbeError) as e:
            rbe.rho_noalloc(args["pos"], args["q"], 10.0, args["m"], args["rho"])
        assert e.value.code == rbe.EINVAL, change
