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


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_iteration_cap_reports_noconv_with_per_system_flags(W, cfg24, prec):
    """A forced iteration cap: the apply returns WGW_ERR_NOCONV with drho still written, the
    statistics count the converged systems, and wgw_system_info flags exactly the systems whose
    final FP64 residual missed cg_tol.  With the cap lifted the same context converges."""
    s = cfg24
    opt = dict(precision=W.WGW_FP64, cg_tol=1e-12, max_cg_iter=6) if prec == "fp64" else \
        dict(precision=W.WGW_MIXED, cg_tol=1e-12, max_cg_iter=6, max_refine=1)
    ctx = W.wgw_setup(s.L, s.ecut, s.grid, s.vloc_G, s.psi_v, s.e_v, W.wgw_default_options(**opt))
    dV = synth.perturbations(s.miller_rho, s.L, 4, 77)
    drho, st, status = W.wgw_apply_chi0(ctx, dV, allow_noconv=True)
    assert status == W.WGW_ERR_NOCONV
    assert np.all(np.isfinite(drho)) and np.max(np.abs(drho)) > 0
    it, rr, conv = W.wgw_system_info(ctx, 16, with_flags=True)
    assert it.shape == (16,) and np.all(it <= (6 if prec == "fp64" else 6))
    assert np.array_equal(conv, (rr <= 1e-12 * (1 + 1e-6)).astype(np.int32))
    assert st["n_converged"] == int(conv.sum()) < 16
    W.wgw_set_options(ctx, W.wgw_default_options(precision=opt["precision"], cg_tol=1e-12))
    drho2, st2, status2 = W.wgw_apply_chi0(ctx, dV)
    assert status2 == W.WGW_OK and st2["n_converged"] == 16
    assert np.all(W.wgw_system_info(ctx, 16, with_flags=True)[2] == 1)


def test_cancel_a_queued_request(W, cfg24):
    """wgw_cancel on requests queued behind a running one: they complete with
    WGW_ERR_CANCELLED and their outputs stay untouched; the others are served normally."""
    s = cfg24
    ctx = W.wgw_setup(s.L, s.ecut, s.grid, s.vloc_G, s.psi_v, s.e_v, W.wgw_default_options(cg_tol=1e-12))
    first = W.wgw_submit(ctx, synth.perturbations(s.miller_rho, s.L, 8, 78), [0.0, 0.3, 0.9])
    later = [W.wgw_submit(ctx, synth.perturbations(s.miller_rho, s.L, 1, 79 + k), [0.0]) for k in range(3)]
    W.wgw_cancel(later[1])
    _, r0 = W.wgw_wait(first)
    assert r0["status"] == W.WGW_OK
    for k, t in enumerate(later):
        got, r = W.wgw_wait(t)
        if k == 1:
            assert r["status"] == W.WGW_ERR_CANCELLED and np.all(got == 0)
        else:
            assert r["status"] == W.WGW_OK and np.max(np.abs(got)) > 0
    with pytest.raises(W.WgwError):
        W.wgw_cancel(later[1])
