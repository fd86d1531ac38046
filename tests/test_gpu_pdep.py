"""PDEP Davidson and the dense Rayleigh-Ritz eigensolver on the GPU, against the oracle.

Eigenvalues: relative error |dlambda| / |lambda| per eigenvalue, FP64 path 1e-10 and
mixed path 1e-8.  Eigenvectors are compared through subspace angles (the PDEP vectors
are defined up to sign and rotation inside degenerate sets).
"""
import os

import numpy as np
import pytest

import synth
from oracle import pdep
from oracle.model import Model

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "pdep_L16_48.txt")


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
    return Model(s.L, s.ecut, s.grid, s.vloc_G, s.psi_v, s.e_v, s.beta_G, s.d_proj)


@pytest.mark.parametrize("n", [1, 2, 3, 17, 64, 200])
def test_symmetric_eigensolver(W, n):
    import torch
    rng = np.random.default_rng(n)
    A = rng.standard_normal((n, n))
    A = A + A.T
    if n >= 17:
        # A degenerate pair and a cluster, the cases the Rayleigh-Ritz matrices produce.
        Q, _ = np.linalg.qr(rng.standard_normal((n, n)))
        ev = np.sort(rng.standard_normal(n))
        ev[3] = ev[4]
        ev[7:10] = ev[7] + 1e-13 * np.arange(3)
        A = (Q * ev) @ Q.T
        A = 0.5 * (A + A.T)
    Ad = torch.from_numpy(A.copy()).cuda()
    w, Z = W.wgw_symm_eig_dev(Ad)
    torch.cuda.synchronize()
    w = w.cpu().numpy()
    Z = Z.cpu().numpy().T            # column-major on the device
    ref = np.linalg.eigvalsh(A)
    scale = max(1.0, np.max(np.abs(ref)))
    assert np.max(np.abs(w - ref)) < 1e-13 * scale * max(1, n) ** 0.5
    assert np.max(np.abs(Z.T @ Z - np.eye(n))) < 1e-12 * max(1, n) ** 0.5
    assert np.max(np.abs(A @ Z - Z * w)) < 1e-12 * scale * max(1, n) ** 0.5


@pytest.fixture(scope="module")
def dense24(cfg24):
    return pdep.pdep_dense(model_of(cfg24), 16)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_davidson_matches_dense_pdep(W, cfg24, dense24, prec):
    s = cfg24
    w_ref, U_ref = dense24
    n_pdep = 8
    opt = dict(precision=W.WGW_FP64, cg_tol=1e-13, dav_tol=1e-12) if prec == "fp64" else \
        dict(precision=W.WGW_MIXED, cg_tol=1e-11, dav_tol=1e-11)
    ctx = W.wgw_setup(s.L, s.ecut, s.grid, s.vloc_G, s.psi_v, s.e_v, W.wgw_default_options(**opt))
    x0 = synth.perturbations(s.miller_rho, s.L, n_pdep, 11)
    eig, basis, st, _ = W.wgw_pdep_davidson(ctx, n_pdep, x0)
    assert st["n_converged"] == n_pdep
    tol = 1e-10 if prec == "fp64" else 1e-8
    assert np.max(np.abs(eig - w_ref[:n_pdep]) / np.abs(w_ref[:n_pdep])) < tol
    # Orthonormal basis spanning the dense eigenvectors of the converged, separated part.
    assert np.max(np.abs(basis.conj().T @ basis - np.eye(n_pdep))) < 1e-10
    gap_ok = np.abs(w_ref[n_pdep] - w_ref[n_pdep - 1]) > 1e-6
    if gap_ok:
        sv = np.linalg.svd(U_ref[:, :n_pdep].conj().T @ basis, compute_uv=False)
        assert np.min(sv) > 1 - 1e-7


def test_davidson_without_start_block(W, cfg24, dense24):
    s = cfg24
    w_ref, _ = dense24
    ctx = W.wgw_setup(s.L, s.ecut, s.grid, s.vloc_G, s.psi_v, s.e_v,
                      W.wgw_default_options(cg_tol=1e-13, dav_tol=1e-12))
    eig, _, st, _ = W.wgw_pdep_davidson(ctx, 4, None, want_basis=False)
    assert np.max(np.abs(eig - w_ref[:4]) / np.abs(w_ref[:4])) < 1e-10


@pytest.mark.slow
def test_davidson_config48_matches_golden(W):
    """64 PDEP eigenvalues of the 48^3 model (mixed path) against the oracle's stored values."""
    ref = np.loadtxt(GOLDEN)
    s = synth.make_system("pdep_L16_48")
    ctx = W.wgw_setup(s.L, s.ecut, s.grid, s.vloc_G, s.psi_v, s.e_v,
                      W.wgw_default_options(precision=W.WGW_MIXED, cg_tol=1e-10, dav_tol=1e-10,
                                            max_cg_iter=200, dav_max_iter=250))
    x0 = synth.perturbations(s.miller_rho, s.L, 64, 11)
    eig, _, st, _ = W.wgw_pdep_davidson(ctx, 64, x0, want_basis=False)
    assert st["n_converged"] == 64
    assert np.max(np.abs(eig - ref) / np.abs(ref)) < 1e-8
