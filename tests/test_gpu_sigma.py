"""Exchange self-energy on the GPU against the oracle (Eq. sigmacIR): relative error 1e-10 on
both paths (the pair densities are transformed at FP64 accuracy either way)."""
import numpy as np
import pytest

import synth
from oracle import sigma
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


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_sigma_x_matches_oracle(W, cfg24, precision):
    s = cfg24
    m = Model(s.L, s.ecut, s.grid, s.vloc_G, s.psi_v, s.e_v)
    ref = sigma.sigma_x(m)
    opt = W.wgw_default_options(precision=W.WGW_MIXED if precision == "mixed" else W.WGW_FP64)
    ctx = W.wgw_setup(s.L, s.ecut, s.grid, s.vloc_G, s.psi_v, s.e_v, opt)
    got = W.wgw_sigma_x(ctx, list(range(s.n_v)))
    assert np.all(got < 0)
    assert np.max(np.abs(got - ref)) < 1e-10 * np.max(np.abs(ref))
    # A subset in another order gives the same numbers.
    sub = W.wgw_sigma_x(ctx, [3, 1])
    assert np.max(np.abs(sub - ref[[3, 1]])) < 1e-10 * np.max(np.abs(ref))


def test_sigma_x_many_states_in_batches(W):
    """70 occupied states: several batches of pair densities."""
    s = synth.make_system(synth.Config("nv70", L=10.0, ecut=5.0, grid=24, n_wells=16, well_seed=1, n_v=70))
    m = Model(s.L, s.ecut, s.grid, s.vloc_G, s.psi_v, s.e_v)
    states = [0, 17, 69, 68, 40, 5, 33, 12]
    ref = sigma.sigma_x(m, states)
    ctx = W.wgw_setup(s.L, s.ecut, s.grid, s.vloc_G, s.psi_v, s.e_v, W.wgw_default_options())
    got = W.wgw_sigma_x(ctx, states)
    assert np.max(np.abs(got - ref)) < 1e-10 * np.max(np.abs(ref))


def test_sigma_x_rejects_bad_state(W, tiny):
    s = tiny
    ctx = W.wgw_setup(s.L, s.ecut, s.grid, s.vloc_G, s.psi_v, s.e_v, W.wgw_default_options())
    with pytest.raises(W.WgwError):
        W.wgw_sigma_x(ctx, [s.n_v])


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_isr_matches_oracle(W, cfg24, precision):
    """I^SR of Eq. ISR: the GPU chains, resolvent and quadrature contraction against the oracle's
    (1e-10 of the largest value), with a Lambda that varies with the node and is not diagonal."""
    from oracle import sigma as osig
    s = cfg24
    m = Model(s.L, s.ecut, s.grid, s.vloc_G, s.psi_v, s.e_v)
    npd, n_steps = 4, 12
    phi = synth.perturbations(s.miller_rho, s.L, npd, 91)
    x, wts = np.polynomial.legendre.leggauss(8)
    nodes, weights = 5.0 * (x + 1.0), 5.0 * wts
    rng = np.random.default_rng(92)
    A = rng.standard_normal((npd, npd))
    lam = np.array([(A + A.T) / (1.0 + wp) for wp in nodes])
    states, omegas = [0, 3], [-0.4, 0.35]
    ref = osig.isr(m, phi, states, n_steps, omegas, lam, nodes, weights)
    opt = W.wgw_default_options(precision=W.WGW_MIXED if precision == "mixed" else W.WGW_FP64)
    ctx = W.wgw_setup(s.L, s.ecut, s.grid, s.vloc_G, s.psi_v, s.e_v, opt)
    got = W.wgw_isr(ctx, phi, states, n_steps, omegas, lam, nodes, weights)
    assert np.max(np.abs(got - ref)) < 1e-10 * np.max(np.abs(ref))
