"""Failure detection on the GPU without a fault: a bounded device wait that nothing completes
gives up after about one second, reports it through its flag, and the device stays usable."""
import time

import numpy as np
import pytest

import synth
from oracle import chi0
from oracle.model import Model

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def W():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2203_05623_gb300 import build
    build.build()
    import paper_2203_05623_gb300 as W
    return W


def test_bounded_wait_gives_up_and_device_stays_usable(W, tiny):
    t0 = time.perf_counter()
    assert W.wgw_selftest_wait_timeout() == 1
    dt = time.perf_counter() - t0
    assert 0.9 < dt < 30.0
    # The same process keeps working: a tensor-core mixed apply matches the oracle.
    s = tiny
    ctx = W.wgw_setup(s.L, s.ecut, s.grid, s.vloc_G, s.psi_v, s.e_v,
                      W.wgw_default_options(precision=W.WGW_MIXED, cg_tol=1e-11))
    dV = synth.perturbations(s.miller_rho, s.L, 2, 71)
    drho, st, _ = W.wgw_apply_chi0(ctx, dV)
    ref = chi0.sos_drho(Model(s.L, s.ecut, s.grid, s.vloc_G, s.psi_v, s.e_v), dV, [0.0])
    assert np.max(np.abs(drho - ref)) < 1e-8 * np.max(np.abs(ref))
