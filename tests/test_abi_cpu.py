"""C ABI checks that need no GPU: the library builds, loads, exports every
entry point declared in include/ccmsav.h, and validates arguments before it
touches the device."""
import math
import os
import re

import pytest

from paper_2601_10057_gb300 import build as B
from paper_2601_10057_gb300 import ccmsav as cc
from paper_2601_10057_gb300 import inputs as I

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    B.build()
    return cc.load()


def declared_functions():
    src = open(os.path.join(ROOT, "include", "ccmsav.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(ccmsav_[a-z_0-9]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ("ccmsav_create", "ccmsav_set_state", "ccmsav_step", "ccmsav_get_state",
                 "ccmsav_energy", "ccmsav_mass", "ccmsav_destroy"):
        assert must in names


def test_library_exports_every_declared_symbol(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_strerror_and_null_handles(lib):
    assert cc.ccmsav_strerror(0) == "ok"
    assert "invalid" in cc.ccmsav_strerror(cc.CCMSAV_EINVAL)
    assert cc.ccmsav_step(None, 1) == cc.CCMSAV_EINVAL
    assert cc.ccmsav_sync(None) == cc.CCMSAV_EINVAL
    assert cc.ccmsav_grid_size(None, 0) == cc.CCMSAV_EINVAL
    assert cc.ccmsav_set_group_points(None, 1 << 20) == cc.CCMSAV_EINVAL
    assert cc.ccmsav_group_points(None) == -1
    cc.ccmsav_destroy(None)


@pytest.mark.parametrize("N", [0, 4, 7, 12, 100, 16384])
def test_create_rejects_bad_grid_sizes(lib, N):
    st, h = cc.ccmsav_create(I.growth_params(), [N])
    assert st == cc.CCMSAV_EINVAL and not h.value


@pytest.mark.parametrize("field,value", [("eps", 0.0), ("dt", -1e-5), ("L", 0.0), ("lam", 0.0),
                                         ("M0", 1.0), ("M0", 0.0), ("theta", -1.0),
                                         ("gamma_area", math.nan), ("M_phi", 0.0)])
def test_create_rejects_bad_parameters(lib, field, value):
    p = I.growth_params().replace(**{field: value})
    st, h = cc.ccmsav_create(p, [64])
    assert st == cc.CCMSAV_EINVAL and not h.value


def test_create_rejects_bad_precision_and_flags(lib):
    assert cc.ccmsav_create(I.growth_params(), [64], precision=7)[0] == cc.CCMSAV_EINVAL
    assert cc.ccmsav_create(I.growth_params(), [64], flags=8)[0] == cc.CCMSAV_EINVAL
    assert cc.ccmsav_create(I.growth_params(), [])[0] == cc.CCMSAV_EINVAL


@pytest.mark.parametrize("N,bc,prec", [(4, 0, 0), (12, 0, 0), (16384, 0, 0), (64, 3, 0), (64, -1, 0), (64, 0, 5)])
def test_solver_create_rejects_bad_arguments(lib, N, bc, prec):
    st, h = cc.ccmsav_solver_create(N, 1.0, bc, prec)
    assert st == cc.CCMSAV_EINVAL and not h.value


def test_solver_calls_reject_null_handles(lib):
    assert cc.ccmsav_solver_create(64, 0.0, 0, 0)[0] == cc.CCMSAV_EINVAL
    assert cc.ccmsav_solver_solve(None, [1.0, 0.0, 0.0], 0, 0) == cc.CCMSAV_EINVAL
    assert cc.ccmsav_solver_smooth(None, 0.1, 0.01, 1e-6, 10, 0) == cc.CCMSAV_EINVAL
    assert cc.ccmsav_solver_sync(None) == cc.CCMSAV_EINVAL
    assert cc.ccmsav_solver_launch_count(None) == 0
    cc.ccmsav_solver_destroy(None)


def test_missing_library_fails_loudly(tmp_path):
    """Without the built library the binding raises at once: there is no CPU
    fallback for any call of the product path."""
    import subprocess
    import sys
    code = ("import sys\n"
            "from paper_2601_10057_gb300 import ccmsav as cc, inputs as I\n"
            f"cc.LIB_PATH = {str(tmp_path / 'libccmsav.so')!r}\n"
            "try:\n"
            "    cc.Simulation(I.growth_params(), 64, precision='fp32')\n"
            "except RuntimeError as e:\n"
            "    print('raised', 'missing' in str(e)); sys.exit(0)\n"
            "sys.exit(3)\n")
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, cwd=ROOT, timeout=300)
    assert r.returncode == 0, r.stdout + r.stderr
    assert "raised True" in r.stdout
