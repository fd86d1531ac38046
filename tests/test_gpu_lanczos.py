"""GPU Lanczos chains (FP64) against the oracle's chains and the sum over states.

alpha, beta: element-wise relative error 1e-10 (FP64 path, as for the other FP64 results);
chi0_nm(i w): relative error of the whole matrix per frequency.
"""
import numpy as np
import pytest

import synth
from oracle import g0 as g0_oracle
from oracle import lanczos
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


def model_of(s):
    return Model(s.L, s.ecut, s.grid, s.vloc_G, s.psi_v, s.e_v)


def _setup_full(W, s, precision=None):
    kb = s.beta_G.shape[1] > 0
    opt = W.wgw_default_options(precision=W.WGW_MIXED if precision == "mixed" else W.WGW_FP64)
    return W.wgw_setup(s.L, s.ecut, s.grid, s.vloc_G, s.psi_v, s.e_v, opt,
                       beta_G=s.beta_G if kb else None, d_proj=s.d_proj if kb else None)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_lanczos_coefficients_and_chi0_match_oracle(W, cfg24, precision):
    s = cfg24
    phi = synth.perturbations(s.miller_rho, s.L, 6, 21)
    oms = [0.0, 0.5, 5.0]
    n_steps = 16
    ref_chi, ref_a, ref_b = lanczos.chi0_pdep(model_of(s), phi, oms, n_steps)
    ctx = _setup_full(W, s, precision)
    chi, a, b, st = W.wgw_lanczos(ctx, phi, n_steps, oms)
    assert st["n_systems"] == 6 * s.n_v
    assert np.max(np.abs(a - ref_a)) < 1e-10 * np.max(np.abs(ref_a))
    assert np.max(np.abs(b - ref_b) / np.maximum(np.abs(ref_b), 1e-30)) < 1e-10
    for k in range(len(oms)):
        assert np.max(np.abs(chi[:, :, k] - ref_chi[:, :, k].real)) < 1e-10 * np.max(np.abs(ref_chi[:, :, k]))
    assert np.max(np.abs(ref_chi.imag)) < 1e-14 * np.max(np.abs(ref_chi))


@pytest.mark.slow
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_lanczos_full_frequency_config_sizes(W, cfg24, precision):
    """The full-frequency configuration at its stated sizes: 32 basis vectors x 4 occupied states
    = 128 chains of 64 steps, chi0 in the basis at the 32 Gauss-Legendre frequencies on
    [0, 50 Ha].  alpha, beta element-wise and chi0_nm(i w_k) at every frequency against the
    oracle's chains (1e-10; both paths keep the chains at FP64 accuracy)."""
    s = cfg24
    phi = synth.perturbations(s.miller_rho, s.L, 32, 24)
    oms, _ = synth.gauss_legendre_omega(32, 50.0)
    n_steps = 64
    ref_chi, ref_a, ref_b = lanczos.chi0_pdep(model_of(s), phi, oms, n_steps)
    chi, a, b, st = W.wgw_lanczos(_setup_full(W, s, precision), phi, n_steps, oms)
    assert st["n_systems"] == 128 and a.shape == (s.n_v, 32, n_steps)
    assert np.max(np.abs(a - ref_a)) < 1e-10 * np.max(np.abs(ref_a))
    assert np.max(np.abs(b - ref_b) / np.maximum(np.abs(ref_b), 1e-30)) < 1e-10
    for k in range(len(oms)):
        assert np.max(np.abs(chi[:, :, k] - ref_chi[:, :, k].real)) < 1e-10 * np.max(np.abs(ref_chi[:, :, k])), k


def test_lanczos_exact_limit_equals_sum_over_states(W, tiny):
    s = tiny
    phi = synth.perturbations(s.miller_rho, s.L, 3, 22)
    oms = [0.0, 1.0]
    n_full = s.n_pw - s.n_v
    ctx = W.wgw_setup(s.L, s.ecut, s.grid, s.vloc_G, s.psi_v, s.e_v, W.wgw_default_options())
    chi, a, b, st = W.wgw_lanczos(ctx, phi, n_full, oms)
    ref = lanczos.chi0_pdep_sos(model_of(s), phi, oms).real
    assert np.max(np.abs(chi - ref)) < 1e-10 * np.max(np.abs(ref))


Z_G0 = np.array([-0.4 + 0.3j, 0.1 + 0.05j, 0.7 + 1.5j, 2.0 + 10.0j])


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_g0_lanczos_matches_oracle(W, cfg24, precision):
    """G0 chains of H (Eq. ISR): alpha, beta, d element-wise to 1e-10, residues and resolvent
    matrices to 1e-10 of their largest element, on two of the occupied states.  Both paths run
    the chains at FP64 accuracy (mixed: float-float FFT passes)."""
    s = cfg24
    phi = synth.perturbations(s.miller_rho, s.L, 5, 31)
    states, n_steps = [0, s.n_v - 1], 16
    ref = g0_oracle.g0_lanczos(Model(s.L, s.ecut, s.grid, s.vloc_G, s.psi_v, s.e_v, s.beta_G, s.d_proj),
                               phi, states, n_steps, Z_G0)
    out = W.wgw_g0_lanczos(_setup_full(W, s, precision), phi, states, n_steps, Z_G0)
    assert out["stats"]["n_systems"] == 5 * len(states)
    for key in ("alpha", "beta", "d"):
        assert np.max(np.abs(out[key] - ref[key])) < 1e-10 * np.max(np.abs(ref[key])), key
    assert np.max(np.abs(ref["C"].imag)) < 1e-12 * np.max(np.abs(ref["C"]))
    assert np.max(np.abs(out["C"] - ref["C"].real)) < 1e-10 * np.max(np.abs(ref["C"]))
    assert np.max(np.abs(out["g0"] - ref["g0"])) < 1e-10 * np.max(np.abs(ref["g0"]))


@pytest.mark.parametrize("kb", [False, True])
def test_g0_lanczos_exact_limit_equals_dense_resolvent(W, tiny, kb):
    """Chains that exhaust their Krylov spaces give <psi_i phi~_n|(H - z)^-1|psi_i phi~_m>
    of a dense solve, without and with KB projectors in H."""
    s = synth.make_system(synth.Config("kb", L=6.0, ecut=2.5, grid=12, n_wells=2, well_seed=7, n_v=2,
                                       kb=True)) if kb else tiny
    assert (s.beta_G.shape[1] > 0) == kb
    phi = synth.perturbations(s.miller_rho, s.L, 3, 32)
    m = Model(s.L, s.ecut, s.grid, s.vloc_G, s.psi_v, s.e_v, s.beta_G, s.d_proj)
    ref = g0_oracle.g0_exact(m, phi, [0, 1], Z_G0)
    out = W.wgw_g0_lanczos(_setup_full(W, s), phi, [0, 1], s.n_pw, Z_G0)
    assert np.max(np.abs(out["g0"] - ref)) < 1e-10 * np.max(np.abs(ref))


def test_g0_lanczos_rejects_bad_state(W, tiny):
    s = tiny
    phi = synth.perturbations(s.miller_rho, s.L, 1, 33)
    ctx = _setup_full(W, s)
    with pytest.raises(W.WgwError):
        W.wgw_g0_lanczos(ctx, phi, [s.n_v], 4, Z_G0)


def test_dyson_matches_oracle_and_closed_form(W):
    """(1 - chibar0)^-1 chibar0 per frequency: closed form on a known spectrum, the oracle's
    solve on non-symmetric input, n = 1 and a singular case."""
    from oracle import dyson
    rng = np.random.default_rng(31)
    n, nw = 64, 32
    A = np.zeros((nw, n, n))
    ref = np.zeros((nw, n, n))
    for k in range(nw):
        Q, _ = np.linalg.qr(rng.standard_normal((n, n)))
        lam = -rng.uniform(0.0, 8.0, n)
        A[k] = (Q * lam) @ Q.T
        ref[k] = (Q * (lam / (1.0 - lam))) @ Q.T
    X = W.wgw_dyson(A)
    assert np.max(np.abs(X - ref)) < 1e-12 * np.max(np.abs(ref))
    B = rng.standard_normal((3, 17, 17)) * 0.2
    assert np.max(np.abs(W.wgw_dyson(B) - dyson.chibar(B))) < 1e-12
    assert abs(W.wgw_dyson(np.array([[-3.0]]))[0, 0] + 0.75) < 1e-15
    with pytest.raises(W.WgwError):
        W.wgw_dyson(np.eye(4))


def test_dyson_on_lanczos_chi0(W, cfg24):
    """The Dyson step on the GPU's own chi0 in a basis (Lanczos, 4 frequencies) equals the
    oracle's solve of the same matrices."""
    from oracle import dyson
    s = cfg24
    phi = synth.perturbations(s.miller_rho, s.L, 8, 23)
    ctx = W.wgw_setup(s.L, s.ecut, s.grid, s.vloc_G, s.psi_v, s.e_v, W.wgw_default_options())
    chi, _, _, _ = W.wgw_lanczos(ctx, phi, 12, [0.0, 0.3, 1.0, 4.0])
    layout = np.ascontiguousarray(np.moveaxis(chi, 2, 0))     # (n_omega, n, n)
    got = W.wgw_dyson(layout)
    assert np.max(np.abs(got - dyson.chibar(layout))) < 1e-12 * max(1.0, np.max(np.abs(got)))
