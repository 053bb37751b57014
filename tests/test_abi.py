"""CPU checks of the C-ABI library: it is built, loads, exports every symbol
``include/rljsde.h`` declares, and rejects bad arguments before touching the
GPU."""
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def rl():
    from paper_2205_02646_gb300 import build, rljsde
    build.build()
    rljsde.load()
    return rljsde


def declared_functions():
    text = open(os.path.join(ROOT, "include", "rljsde.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(rljsde_[a-z0-9_]+)\s*\(", text)))


def test_exports_every_declared_symbol(rl):
    lib = rl.load()
    names = declared_functions()
    assert len(names) >= 12
    for n in names:
        assert hasattr(lib, n), n
    assert sorted(rl.EXPORTS) == names


def test_defaults_and_status_strings(rl):
    p = rl.default_params()
    assert (p.block, p.window, p.nu_max, p.gamma_odc, p.rho_decay, p.q_mode, p.precision, p.path, p.layout,
            p.pairs, p.c_supply) == \
        (4, 32, 100, 0.5, 0.7, 0, 0, 0, 0, 0, 0)
    lib = rl.load()
    for s in range(9):
        assert lib.rljsde_status_string(s)
    assert lib.rljsde_default_params(None) == 1


def _create(rl, mask, **kw):
    import ctypes
    lib = rl.load()
    p = rl.default_params(**kw)
    h = ctypes.c_void_p()
    m = np.ascontiguousarray(mask, dtype=np.uint8)
    return lib.rljsde_plan_create(ctypes.byref(h), m.ctypes.data, m.shape[0], m.shape[1], ctypes.byref(p))


def test_argument_errors_before_gpu(rl):
    ok = np.zeros((8, 8), np.uint8)
    assert _create(rl, np.zeros((7, 8), np.uint8)) == 2           # odd LR height
    assert _create(rl, np.zeros((2, 8), np.uint8)) == 2           # too small
    bad = ok.copy(); bad[3, 3] = 4
    assert _create(rl, bad) == 3                                   # code outside 0..3
    assert _create(rl, ok, block=8) == 8                           # B is fixed by the paper
    assert _create(rl, ok, window=16) == 8
    assert _create(rl, ok, nu_max=0) == 1
    assert _create(rl, ok, gamma_odc=2.0) == 1
    assert _create(rl, ok, rho_decay=0.0) == 1
    assert _create(rl, ok, precision=2) == 1
    assert _create(rl, ok, path=2, precision=1) == 8
    # sensor layouts: aperture codes 0..15; paths that cannot hold the mask's apertures
    assert _create(rl, ok, layout=2) == 1
    assert _create(rl, ok, pairs=2) == 1
    # stored Gram matrices: FP32 loop on host table sets only
    assert _create(rl, ok, c_supply=4) == 1
    assert _create(rl, ok, c_supply=3, precision=1) == 8
    qz = np.ones(1024); qz[5] = 0.0
    assert _create(rl, ok, c_supply=1, q_table=qz) == 8            # q = 0 somewhere: factored loop only
    assert _create(rl, ok, c_supply=1, precision=1) == 8
    assert _create(rl, ok, c_supply=1, path=2) == 8
    assert _create(rl, ok, c_supply=1, path=3) == 8
    assert _create(rl, np.full((8, 8), 16, np.uint8), layout=1) == 3
    quarter = np.tile(np.array([[1, 2], [4, 8]], np.uint8), (4, 4))
    assert _create(rl, quarter, layout=1, path=3) == 8            # in-kernel tables: three-quarter only
    many = np.arange(64, dtype=np.uint8).reshape(8, 8) % 15 + 1
    assert _create(rl, many, layout=1, path=1) == 8               # 15 apertures > 4 table slots
    assert _create(rl, many, layout=1, path=0, precision=1) == 8  # direct path is FP32
    lib = rl.load()
    assert lib.rljsde_plan_create(None, None, 8, 8, None) == 1
    assert lib.rljsde_reconstruct(None, None, 0, None, 0, None) == 1
    assert lib.rljsde_reconstruct_batch(None, None) == 1
    assert lib.rljsde_check(None, None) == 1
    lib.rljsde_plan_destroy(None)
