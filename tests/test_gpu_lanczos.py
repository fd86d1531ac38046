"""GPU Lanczos chains (FP64) against the oracle's chains and the sum over states.

alpha, beta: element-wise relative error 1e-10 (FP64 path, as for the other FP64 results);
chi0_nm(i w): relative error of the whole matrix per frequency.
"""
import numpy as np
import pytest

import synth
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


def test_lanczos_coefficients_and_chi0_match_oracle(W, cfg24):
    s = cfg24
    phi = synth.perturbations(s.miller_rho, s.L, 6, 21)
    oms = [0.0, 0.5, 5.0]
    n_steps = 16
    ref_chi, ref_a, ref_b = lanczos.chi0_pdep(model_of(s), phi, oms, n_steps)
    ctx = W.wgw_setup(s.L, s.ecut, s.grid, s.vloc_G, s.psi_v, s.e_v, W.wgw_default_options())
    chi, a, b, st = W.wgw_lanczos(ctx, phi, n_steps, oms)
    assert st["n_systems"] == 6 * s.n_v
    assert np.max(np.abs(a - ref_a)) < 1e-10 * np.max(np.abs(ref_a))
    assert np.max(np.abs(b - ref_b) / np.maximum(np.abs(ref_b), 1e-30)) < 1e-10
    for k in range(len(oms)):
        assert np.max(np.abs(chi[:, :, k] - ref_chi[:, :, k].real)) < 1e-10 * np.max(np.abs(ref_chi[:, :, k]))
    assert np.max(np.abs(ref_chi.imag)) < 1e-14 * np.max(np.abs(ref_chi))


def test_lanczos_exact_limit_equals_sum_over_states(W, tiny):
    s = tiny
    phi = synth.perturbations(s.miller_rho, s.L, 3, 22)
    oms = [0.0, 1.0]
    n_full = s.n_pw - s.n_v
    ctx = W.wgw_setup(s.L, s.ecut, s.grid, s.vloc_G, s.psi_v, s.e_v, W.wgw_default_options())
    chi, a, b, st = W.wgw_lanczos(ctx, phi, n_full, oms)
    ref = lanczos.chi0_pdep_sos(model_of(s), phi, oms).real
    assert np.max(np.abs(chi - ref)) < 1e-10 * np.max(np.abs(ref))
