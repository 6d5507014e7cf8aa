"""Host-side checks that need no GPU: the library builds, loads and exports
every entry point include/shs.h declares; argument validation; the generated
device tables are current and agree with the oracle's independent route."""

import ctypes
import os
import re
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER_DIR = os.path.join(ROOT, "include")


@pytest.fixture(scope="module")
def lib():
    from paper_2104_00359_gb300 import build, _lib
    build.build()
    return _lib.load()


def _declared_functions():
    names = []
    for fn in os.listdir(HEADER_DIR):
        if fn.endswith(".h"):
            text = open(os.path.join(HEADER_DIR, fn)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names += re.findall(r"\b(shs_\w+)\s*\(", text)
    return sorted(set(names))


def test_every_declared_symbol_is_exported(lib):
    names = _declared_functions()
    assert "shs_shade" in names and "shs_shade_backward" in names
    for n in names:
        assert hasattr(lib, n), f"{n} declared in include/ but not exported"


def test_binding_covers_header():
    from paper_2104_00359_gb300 import _lib
    assert set(_declared_functions()) <= set(_lib._SIGS), set(_declared_functions()) - set(_lib._SIGS)


def test_config_validation_without_gpu(lib):
    from paper_2104_00359_gb300._lib import ShsConfig
    cfg = ShsConfig()
    assert lib.shs_config_default(ctypes.byref(cfg)) == 0
    assert (cfg.n_bands, cfg.epsilon, cfg.exp_tau, cfg.exp_kmax, cfg.fixed_k) == (4, 3.0, 1.0, 16, -1)
    h = ctypes.c_void_p()
    for field, value, expect in (("n_bands", 9, 1), ("n_bands", 0, 1), ("exp_kmax", 17, 1),
                                 ("precision", 7, 1), ("precision", 2, 2), ("horizon_cull", 2, 1), ("exp_mode", 3, 1),
                                 ("exp_mode", -1, 1),
                                 ("exp_tau", 0.0, 1), ("deterministic", 2, 1)):
        bad = ShsConfig()
        lib.shs_config_default(ctypes.byref(bad))
        setattr(bad, field, value)
        st = lib.shs_scene_create(ctypes.byref(bad), 0, None, None, ctypes.c_void_p(16), None, ctypes.byref(h))
        assert st == expect, (field, value, st)
        assert lib.shs_last_error()
    st = lib.shs_scene_create(ctypes.byref(cfg), 2000, ctypes.c_void_p(16), ctypes.c_void_p(16),
                              ctypes.c_void_p(16), None, ctypes.byref(h))
    assert st == 1
    st = lib.shs_scene_create(ctypes.byref(cfg), 3, None, None, ctypes.c_void_p(16), None, ctypes.byref(h))
    assert st == 1
    assert lib.shs_saved_bytes(None, 100) == 0
    tab = (ctypes.c_float * 4)(1, 1, 1, 1)
    assert lib.shs_scene_set_ol_table(None, tab, 2, 1.0) == 1
    # the no-alloc backward has no scene to hold a table: refused before any CUDA call
    c2 = ShsConfig()
    lib.shs_config_default(ctypes.byref(c2))
    c2.exp_mode = 2
    assert lib.shs_shade_backward_noalloc(ctypes.byref(c2), 0, None, None, None, 0, *([None] * 11), None) == 2
    assert lib.shs_shade(None, 10, None, None, None, None, None, None) == 1
    assert lib.shs_shade_tail(None, 10, None, None, None, None, None) == 1
    assert lib.shs_status_string(5) == b"device wait timed out"


def test_generated_tables_are_current():
    sys.path.insert(0, os.path.join(ROOT, "paper_2104_00359_gb300", "csrc"))
    try:
        import gen_tables
        assert gen_tables.main(["--check"]) == 0
    finally:
        sys.path.pop(0)


@pytest.mark.parametrize("n", [4, 8])
def test_device_gaunt_route_agrees_with_oracle(n):
    """The CUDA side integrates monomials exactly; the oracle uses quadrature.
    The two independent routes must give the same triple-product tensor."""
    sys.path.insert(0, os.path.join(ROOT, "paper_2104_00359_gb300", "csrc"))
    try:
        import gen_tables
        g = gen_tables.gaunt_monomial(n)
        A = gen_tables.ahat(n)
        N = gen_tables.norms(n)
    finally:
        sys.path.pop(0)
    from oracle import shs_oracle as O
    C = O.gaunt_tensor(n)
    D = np.zeros_like(C)
    for (i, j, k), v in g.items():
        D[i, j, k] = v
        D[i, k, j] = v
    assert np.abs(C - D).max() < 1e-10
    R = O.zh_rotation_scale(n)[[l * l for l in range(n)]] * O.clamped_cosine_zh(n)
    np.testing.assert_allclose(A, R, atol=1e-14)
    d = np.array([[0.3, -0.5, 0.81]])
    d /= np.linalg.norm(d)
    ybar = [sum(float(c) * d[0, 0] ** a * d[0, 1] ** b * d[0, 2] ** e for (a, b, e), c in p.items())
            for p in gen_tables.ybar_polys(n)]
    np.testing.assert_allclose(np.array(N) * np.array(ybar), O.real_sh(n, d)[0], atol=1e-12)


def test_envmap_projection_argument_checks_without_gpu(lib):
    """Size query and argument validation of shs_project_envmap run on the host
    (no device call for a rejected request)."""
    assert lib.shs_envmap_workspace_bytes(0, 32, 4) == 0
    assert lib.shs_envmap_workspace_bytes(16, 0, 4) == 0
    assert lib.shs_envmap_workspace_bytes(16, 32, 9) == 0
    assert lib.shs_envmap_workspace_bytes(16, 32, 4) == 256 + 4 * 16 * 3 * 16
    assert lib.shs_envmap_workspace_bytes(100000, 32, 8) == 0
    assert lib.shs_envmap_workspace_bytes(4096, 8192, 8) == 8 * 8192 + 4 * 1216 * 3 * 64
    one = ctypes.c_void_p(16)
    need = lib.shs_envmap_workspace_bytes(16, 32, 4)
    for args in ((None, 16, 32, 4, one, one, need), (one, 16, 32, 4, None, one, need),
                 (one, 16, 32, 4, one, None, need), (one, 16, 32, 0, one, one, need),
                 (one, 16, 32, 9, one, one, need), (one, 0, 32, 4, one, one, need),
                 (one, 16, 0, 4, one, one, need), (one, 16, 65537, 4, one, one, need),
                 (one, 16, 32, 4, one, one, need - 4), (one, 16, 32, 4, one, ctypes.c_void_p(20), need)):
        assert lib.shs_project_envmap(*args, None) == 1, args
        assert lib.shs_last_error()


def test_chain_argument_checks_without_gpu(lib):
    """Size query and argument validation of the scene-chain calls run on the
    host (no device call for a rejected or empty request)."""
    assert lib.shs_chain_workspace_bytes(-1, 4) == 0
    assert lib.shs_chain_workspace_bytes(10, 0) == 0
    assert lib.shs_chain_workspace_bytes(10, 257) == 0
    assert lib.shs_chain_workspace_bytes(0, 60) == 4 * (60 + 12)           # one partial row
    assert lib.shs_chain_workspace_bytes(1000, 60) == 4 * 63 * (60 + 12)    # 63 blocks of 8 warps x 2 rows
    assert lib.shs_chain_workspace_bytes(50000, 60) == 4 * 608 * (60 + 12)  # capped at 608 partial rows
    assert lib.shs_chain_workspace_bytes(10 ** 7, 60) == 4 * 608 * (60 + 12)
    one = ctypes.c_void_p(16)
    for args in ((one, one, -1, 4, one, one, 0, None, one), (one, one, 5, 0, one, one, 0, None, one),
                 (one, one, 5, 257, one, one, 0, None, one), (one, one, 5, 4, None, one, 0, None, one),
                 (one, one, 5, 4, one, None, 0, None, one), (None, one, 5, 4, one, one, 0, None, one),
                 (one, one, 5, 4, one, one, 2, None, one), (one, one, 5, 4, one, one, 0, None, None)):
        assert lib.shs_chain_forward(*args, None) == 1, args
        assert lib.shs_last_error()
    assert lib.shs_chain_forward(None, None, 0, 4, one, one, 0, None, None, None) == 0
    need = lib.shs_chain_workspace_bytes(5, 4)
    for args in ((one, one, 5, 4, one, one, 0, None, one, one, one, need),
                 (one, one, 5, 4, one, one, 0, one, None, one, one, need),
                 (one, one, 5, 4, one, one, 0, one, one, one, None, need),
                 (one, one, 5, 4, one, one, 0, one, one, one, one, need - 4),
                 (one, one, 5, 4, one, one, 0, one, one, one, ctypes.c_void_p(20), need),
                 (one, one, 5, 4, one, one, 3, one, one, one, one, need)):
        assert lib.shs_chain_backward(*args, None) == 1, args
