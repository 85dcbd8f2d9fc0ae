"""ccmsav_mass_noalloc: the allocation-free mass entry point, through the C
ABI, against ccmsav_mass() on the same stored field and against an exactly
rounded host sum (math.fsum), on two calls in a row.

Some callers cannot let the library allocate device memory (device memory
reserved up front by a pooling allocator or capped by a framework, real-time
loops that must not pay allocation latency); this entry point serves them
from a fixed scratch array inside the library.  The file is named so that
pytest collects it last."""
import math

import numpy as np
import pytest

from paper_2601_10057_gb300 import build as B
from paper_2601_10057_gb300 import ccmsav as cc
from paper_2601_10057_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_mass_noalloc_matches_ccmsav_mass(precision):
    import torch
    B.build()
    cc.load()
    w = I.workload("ellipse_shrink", N=256)
    sim = cc.Simulation(w.params, w.N, precision=precision)
    sim.set_state(w.phi0, w.psi0)
    sim.step(3)
    m_ref = sim.mass()
    _, psi = sim.state()                       # the stored field, widened to FP64 exactly
    dtype = torch.float64 if precision == "fp64" else torch.float32
    t = torch.tensor(psi, dtype=dtype, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    torch.cuda.synchronize()
    code = cc.CCMSAV_FP64 if precision == "fp64" else cc.CCMSAV_FP32_BULK
    got = []
    for _ in range(2):
        st, m = cc.ccmsav_mass_noalloc(t.data_ptr(), w.N, code, w.params.L, stream)
        assert st == cc.CCMSAV_OK, cc.ccmsav_strerror(st)
        got.append(m)
    assert got[0] == got[1]
    assert got[0] == pytest.approx(m_ref, rel=1e-12)
    h = w.params.L / w.N
    exact = h * h * math.fsum(psi.ravel().tolist())
    assert got[0] == pytest.approx(exact, rel=1e-12)
    sim.close()


def test_mass_noalloc_rejects_sizes_beyond_the_maximum():
    import torch
    B.build()
    cc.load()
    t = torch.zeros(16, 16, dtype=torch.float64, device="cuda")
    st, _ = cc.ccmsav_mass_noalloc(t.data_ptr(), 8193, cc.CCMSAV_FP64, 1.0)
    assert st == cc.CCMSAV_EINVAL
    st, _ = cc.ccmsav_mass_noalloc(t.data_ptr(), 0, cc.CCMSAV_FP64, 1.0)
    assert st == cc.CCMSAV_EINVAL
    st, m = cc.ccmsav_mass_noalloc(t.data_ptr(), 16, cc.CCMSAV_FP64, 1.0)
    assert st == cc.CCMSAV_OK and m == 0.0
