"""Spin-polarised systems and KB with d channels on the GPU, against the oracle.

Spin: one context per spin channel (f_s = 1), combined by wgw_apply_channels; the oracle sums
the sum-over-states response of the channels.  Relative error of the whole result: FP64 path
1e-10, mixed path 1e-8 (as for one channel).
"""
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


def model_of(s, **kw):
    return Model(s.L, s.ecut, s.grid, s.vloc_G, s.psi_v, s.e_v, s.beta_G, s.d_proj, **kw)


def setup(W, s, precision, f_s):
    kb = s.beta_G.shape[1] > 0
    opt = W.wgw_default_options(precision=W.WGW_MIXED if precision == "mixed" else W.WGW_FP64,
                                cg_tol=1e-11 if precision == "mixed" else 1e-12, f_s=f_s)
    return W.wgw_setup(s.L, s.ecut, s.grid, s.vloc_G, s.psi_v, s.e_v, opt,
                       beta_G=s.beta_G if kb else None, d_proj=s.d_proj if kb else None)


def rel(a, b):
    return np.max(np.abs(a - b)) / np.max(np.abs(b))


@pytest.fixture(scope="module")
def spin24():
    return synth.make_spin_system("chi0_L10_24")


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_spin_channels_match_oracle(W, spin24, precision):
    up, dn = spin24
    assert up.psi_v.shape[1] == 4 and dn.psi_v.shape[1] == 3
    dV = synth.perturbations(up.miller_rho, up.L, 3, 51)
    oms = [0.0, 0.5]
    ref = chi0.sos_drho_channels([model_of(up, f_s=1.0), model_of(dn, f_s=1.0)], dV, oms)
    ctxs = [setup(W, up, precision, 1.0), setup(W, dn, precision, 1.0)]
    out, st, _ = W.wgw_apply_channels(ctxs, dV, oms)
    assert st["n_converged"] == st["n_systems"]
    assert rel(out, ref) < (1e-10 if precision == "fp64" else 1e-8)
    # The symmetrised form: v^1/2 (sum over channels) v^1/2.
    m = model_of(up)
    outb, _, _ = W.wgw_apply_channels(ctxs, dV[:, :2], [0.0], symmetrized=True)
    refb = m.vsqrt[:, None, None] * chi0.sos_drho_channels(
        [model_of(up, f_s=1.0), model_of(dn, f_s=1.0)], m.vsqrt[:, None] * dV[:, :2], [0.0])
    assert rel(outb, refb) < (1e-10 if precision == "fp64" else 1e-8)


def test_identical_channels_equal_unpolarised(W, cfg24):
    s = cfg24
    dV = synth.perturbations(s.miller_rho, s.L, 2, 52)
    one = setup(W, s, "fp64", 1.0)
    two = setup(W, s, "fp64", 1.0)
    both, _, _ = W.wgw_apply_channels([one, two], dV, [0.0, 1.0])
    ref, _, _ = W.wgw_apply_chi0(setup(W, s, "fp64", 2.0), dV, [0.0, 1.0])
    assert rel(both, ref) < 1e-13


def test_channels_reject_mismatched_grids(W, cfg24, tiny):
    a = setup(W, cfg24, "fp64", 1.0)
    b = setup(W, tiny, "fp64", 1.0)
    dV = synth.perturbations(cfg24.miller_rho, cfg24.L, 1, 53)
    with pytest.raises(W.WgwError):
        W.wgw_apply_channels([a, b], dV)
    with pytest.raises(W.WgwError):
        W.wgw_apply_channels([a, a], dV)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_kb_with_d_channels_matches_oracle(W, precision):
    """Nine KB channels per atom (s, p, d): chi0 against the oracle's sum over states."""
    s = synth.make_system(synth.Config("kbd", L=6.0, ecut=2.5, grid=12, n_wells=2, well_seed=7,
                                       n_v=2, kb=True, kb_dch=True))
    assert s.beta_G.shape[1] == 18
    dV = synth.perturbations(s.miller_rho, s.L, 2, 54)
    ref = chi0.sos_drho(model_of(s), dV, [0.0, 0.8])
    out, st, _ = W.wgw_apply_chi0(setup(W, s, precision, 2.0), dV, [0.0, 0.8])
    assert rel(out, ref) < (1e-10 if precision == "fp64" else 1e-8)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_spin_summed_davidson_matches_dense(W, spin24, precision):
    """PDEP eigenvalues of the spin-summed chibar0 against a dense diagonalisation of the
    oracle's sum of the two channels' chibar0 matrices."""
    up, dn = spin24
    X = sum(chi0.chibar0_matrix(model_of(c, f_s=1.0), 0.0) for c in (up, dn))
    w_ref = np.linalg.eigvalsh(0.5 * (X + X.conj().T))[:6]
    opt = dict(precision=W.WGW_FP64, cg_tol=1e-13, dav_tol=1e-12, f_s=1.0) if precision == "fp64" else \
        dict(precision=W.WGW_MIXED, cg_tol=1e-11, dav_tol=1e-11, f_s=1.0)
    ctxs = [W.wgw_setup(c.L, c.ecut, c.grid, c.vloc_G, c.psi_v, c.e_v, W.wgw_default_options(**opt))
            for c in (up, dn)]
    x0 = synth.perturbations(up.miller_rho, up.L, 6, 55)
    eig, basis, st, _ = W.wgw_pdep_davidson_channels(ctxs, 6, x0)
    assert st["n_converged"] == 6
    assert np.max(np.abs(eig - w_ref) / np.abs(w_ref)) < (1e-10 if precision == "fp64" else 1e-8)
    assert np.max(np.abs(basis.conj().T @ basis - np.eye(6))) < 1e-10
