"""PDEP Davidson and the dense Rayleigh-Ritz eigensolver on the GPU, against the oracle.

Eigenvalues: relative error |dlambda| / |lambda| per eigenvalue, FP64 path 1e-10 and
mixed path 1e-8.  Eigenvectors are compared through subspace angles (the PDEP vectors
are defined up to sign and rotation inside degenerate sets).
"""
import numpy as np
import pytest

import synth
from oracle import pdep
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


def test_davidson_checkpoint_and_resume(W, cfg24, dense24, tmp_path):
    """Checkpoint and resume through the C ABI: a Davidson stopped after three iterations returns
    its current Ritz values and basis (status NOCONV); the basis, written to disk and read back,
    is the start block of a fresh context's solve, which converges to the dense PDEP eigenvalues in
    fewer iterations than the cold start from the original block."""
    s = cfg24
    w_ref, _ = dense24
    n_pdep = 8
    opt = dict(precision=W.WGW_FP64, cg_tol=1e-13, dav_tol=1e-12)
    x0 = synth.perturbations(s.miller_rho, s.L, n_pdep, 11)
    ctx = W.wgw_setup(s.L, s.ecut, s.grid, s.vloc_G, s.psi_v, s.e_v, W.wgw_default_options(dav_max_iter=3, **opt))
    eig1, basis1, st1, status = W.wgw_pdep_davidson(ctx, n_pdep, x0, allow_noconv=True)
    assert status == W.WGW_ERR_NOCONV and st1["max_iters"] == 3
    np.save(tmp_path / "pdep_basis.npy", basis1)
    np.save(tmp_path / "pdep_eig.npy", eig1)
    del ctx
    ctx2 = W.wgw_setup(s.L, s.ecut, s.grid, s.vloc_G, s.psi_v, s.e_v, W.wgw_default_options(**opt))
    eig2, basis2, st2, _ = W.wgw_pdep_davidson(ctx2, n_pdep, np.load(tmp_path / "pdep_basis.npy"))
    _, _, cold, _ = W.wgw_pdep_davidson(ctx2, n_pdep, x0, want_basis=False)
    assert st2["n_converged"] == n_pdep
    assert np.max(np.abs(eig2 - w_ref[:n_pdep]) / np.abs(w_ref[:n_pdep])) < 1e-10
    assert st2["max_iters"] < cold["max_iters"]


def _neg_index(miller):
    """Index of -G for every G of a sphere in canonical order."""
    where = {tuple(g): i for i, g in enumerate(np.asarray(miller))}
    return np.array([where[tuple(-g)] for g in np.asarray(miller)])


def _cluster_block(eig, lo, hi, rel_gap=1e-4):
    """[a, b) containing [lo, hi) whose ends fall on eigenvalue gaps > rel_gap |lambda|."""
    def gap(j):
        return abs(eig[j] - eig[j - 1]) > rel_gap * abs(eig[j])
    a, b = lo, hi
    while a > 0 and not gap(a):
        a -= 1
    while b < len(eig) and not gap(b):
        b += 1
    return a, b


@pytest.mark.slow
def test_davidson_config48_sampled_against_oracle(W):
    """The 48^3 model at full size (64 PDEP pairs, mixed path), checked on samples.

    The oracle applies chi0bar (static sum over states) to two blocks of the returned
    eigenvectors, each bounded by eigenvalue gaps: the leading block and the block around
    the middle.  The oracle's Rayleigh-Ritz values on each block equal the returned
    eigenvalues to 1e-8 (relative), and the oracle residual of each returned vector is
    within the Davidson stopping rule (sqrt(dav_tol)).  Every returned eigenvalue is negative
    and they ascend; the basis is orthonormal.  "Leading" is pinned independently of the
    Davidson: the six most negative eigenvalues of the oracle's static chi0bar, from ARPACK
    (implicitly restarted Lanczos, seeded start, no information from the GPU) on the oracle's
    operator in the real basis, equal the six lowest returned eigenvalues, so a Davidson run
    that missed a lower eigenvalue fails.
    """
    from oracle import chi0
    s = synth.make_system("pdep_L16_48")
    dav_tol = 1e-10
    ctx = W.wgw_setup(s.L, s.ecut, s.grid, s.vloc_G, s.psi_v, s.e_v,
                      W.wgw_default_options(precision=W.WGW_MIXED, cg_tol=1e-10, dav_tol=dav_tol,
                                            max_cg_iter=200, dav_max_iter=250))
    x0 = synth.perturbations(s.miller_rho, s.L, 64, 11)
    eig, basis, st, _ = W.wgw_pdep_davidson(ctx, 64, x0)
    assert st["n_converged"] == 64
    assert np.all(np.diff(eig) >= 0) and eig[-1] < 0
    assert np.max(np.abs(basis.conj().T @ basis - np.eye(64))) < 1e-10
    m = model_of(s)
    # Real in r (x(-G) = x(G)^*), the form the oracle's static sum over states takes.
    assert np.max(np.abs(basis - basis[_neg_index(m.mr)].conj())) < 1e-12
    states = chi0._states(m)
    for lo, hi in ((0, 4), (30, 34)):
        a, b = _cluster_block(eig, lo, hi)
        X = basis[:, a:b]
        Y = m.vsqrt[:, None] * chi0.sos_static_block(m, m.vsqrt[:, None] * X, states)
        T = X.conj().T @ Y
        ritz = np.linalg.eigvalsh(0.5 * (T + T.conj().T))
        assert np.max(np.abs(ritz - eig[a:b]) / np.abs(eig[a:b])) < 1e-8, (a, b)
        res = np.linalg.norm(Y - X * eig[a:b][None, :], axis=0)
        assert np.max(res) < np.sqrt(dav_tol), (a, b, res)
    # The most negative eigenvalues of the oracle's operator, found without the Davidson.
    k = 6
    lowest = _oracle_lowest_chibar0(m, states, k)
    assert np.max(np.abs(eig[:k] - lowest) / np.abs(lowest)) < 1e-8, (eig[:k], lowest)


def _oracle_lowest_chibar0(m, states, k):
    """The k most negative eigenvalues of the static chi0bar of the oracle (sum over states),
    by ARPACK on the real basis {G = 0, sqrt2 Re, sqrt2 Im of each +-G pair}: a vector y of
    that basis is the real-in-r function with coefficients c(G) = (y_re - i y_im)/sqrt2 at G and
    the conjugate at -G, on which chi0bar is real symmetric."""
    import scipy.sparse.linalg as sla
    from oracle import chi0
    i0, pos, neg = synth.real_basis_map(m.mr)
    n_rho = m.mr.shape[0]
    s2 = 1.0 / np.sqrt(2.0)

    def to_c(y):
        c = np.zeros((n_rho, y.shape[1]), np.complex128)
        c[i0] = y[0]
        c[pos] = (y[1::2] - 1j * y[2::2]) * s2
        c[neg] = (y[1::2] + 1j * y[2::2]) * s2
        return c

    def to_y(c):
        y = np.zeros((n_rho, c.shape[1]))
        y[0] = c[i0].real
        y[1::2] = np.sqrt(2.0) * c[pos].real
        y[2::2] = -np.sqrt(2.0) * c[pos].imag
        return y

    def mv(y):
        y = np.asarray(y).reshape(n_rho, -1)
        c = to_c(y)
        out = m.vsqrt[:, None] * chi0.sos_static_block(m, m.vsqrt[:, None] * c, states)
        return to_y(out)

    op = sla.LinearOperator((n_rho, n_rho), matvec=mv, matmat=mv, dtype=np.float64)
    v0 = np.random.default_rng(7).standard_normal(n_rho)
    w = sla.eigsh(op, k=k, which="SA", tol=1e-12, ncv=4 * k, v0=v0, return_eigenvectors=False)
    return np.sort(w)
