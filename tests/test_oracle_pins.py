"""Pins of the FP64 oracle against facts fixed by the paper and by the mathematics.

Each pin compares two different routes (or a route and a closed form), so that
a dropped term, a wrong sign or index, or a transposed operand in one of them
fails.  The planted-mistake tests at the end modify the oracle on the CPU and
check that a pin catches it.
"""
import math

import numpy as np
import pytest

import synth
from oracle import chi0, dyson, g0, lanczos, pdep, sigma
from oracle.model import Model, sphere


def model_of(s, **kw):
    return Model(s.L, s.ecut, s.grid, s.vloc_G, s.psi_v, s.e_v, s.beta_G, s.d_proj, **kw)


def rel(a, b):
    return np.max(np.abs(a - b)) / np.max(np.abs(b))


# ---------------------------------------------------------------- spheres and H
def test_sphere_enumeration_brute_force():
    """Both sphere enumerations equal a brute-force lattice count, in the documented order."""
    L, ecut = 10.0, 5.0
    b = 2 * math.pi / L
    count = sum(1 for h in range(-8, 9) for k in range(-8, 9) for l in range(-8, 9)
                if 0.5 * b * b * (h * h + k * k + l * l) <= ecut)
    a = sphere(L, ecut)
    c = synth.miller_sphere(L, ecut)
    assert a.shape[0] == count == 515
    assert np.array_equal(a, c)
    n2 = np.sum(a ** 2, axis=1)
    assert np.all(np.diff(n2) >= 0)
    assert synth.miller_sphere(L, 4 * ecut).shape[0] == 4337
    assert synth.miller_sphere(16.0, 7.75).shape[0] == 4169


def test_vloc_matches_real_space_gaussians(tiny):
    """V_loc(G) of the generator, taken to r, equals the Gaussian wells summed over images (band-limited)."""
    s = synth.make_system(synth.Config("g", L=6.0, ecut=12.0, grid=40, n_wells=2, well_seed=7, n_v=1,
                                       min_gap=-1.0))
    m = Model(s.L, s.ecut, s.grid, s.vloc_G, s.psi_v, s.e_v)
    v_r = m.vloc_r.real
    x = np.arange(s.grid) * s.L / s.grid
    X, Y, Z = np.meshgrid(x, x, x, indexing="ij")
    ref = np.zeros_like(X)
    for R in s.positions:
        for i in (-1, 0, 1):
            for j in (-1, 0, 1):
                for k in (-1, 0, 1):
                    d2 = (X - R[0] - i * s.L) ** 2 + (Y - R[1] - j * s.L) ** 2 + (Z - R[2] - k * s.L) ** 2
                    ref -= 2.0 * np.exp(-d2 / 2.0)
    # 4 * ecut = 48 Ha keeps Gaussians of width 1 bohr to ~1e-8 (exp(-w^2 G^2 / 2) at the cutoff).
    assert np.max(np.abs(v_r - ref)) < 1e-6


def test_fft_h_equals_dense_h(cfg24):
    m = model_of(cfg24)
    H = m.h_dense()
    assert np.max(np.abs(H - H.conj().T)) == 0.0
    rng = np.random.default_rng(0)
    x = rng.standard_normal((m.mw.shape[0], 3)) + 1j * rng.standard_normal((m.mw.shape[0], 3))
    assert rel(m.apply_h(x), H @ x) < 1e-13
    # The given occupied states are eigenvectors with the given eigenvalues.
    assert np.max(np.abs(H @ m.psi_v - m.psi_v * m.e_v)) < 1e-12


def test_fft_h_with_kb_equals_dense_h():
    s = synth.make_system(synth.Config("kb", L=6.0, ecut=2.5, grid=12, n_wells=2, well_seed=7,
                                       n_v=2, kb=True))
    m = model_of(s)
    assert s.beta_G.shape[1] == 8
    rng = np.random.default_rng(1)
    x = rng.standard_normal((m.mw.shape[0], 2)) + 1j * rng.standard_normal((m.mw.shape[0], 2))
    assert rel(m.apply_h(x), m.h_dense() @ x) < 1e-13


# ---------------------------------------------------------------- chi0 routes
@pytest.mark.parametrize("omegas", [[0.0], [0.35, 4.0]])
def test_sos_equals_sternheimer(tiny, omegas):
    m = model_of(tiny)
    dV = synth.perturbations(tiny.miller_rho, tiny.L, 3, 8)
    assert rel(chi0.sos_drho(m, dV, omegas), chi0.sternheimer_drho(m, dV, omegas)) < 1e-12


def test_static_block_sum_equals_sos(cfg24):
    m = model_of(cfg24)
    dV = synth.perturbations(cfg24.miller_rho, cfg24.L, 3, 4)
    assert rel(chi0.sos_static_block(m, dV), chi0.sos_drho(m, dV, [0.0])[:, :, 0]) < 1e-12


def test_sos_equals_sternheimer_complex_perturbation(tiny):
    m = model_of(tiny)
    dV = synth.perturbations(tiny.miller_rho, tiny.L, 2, 11, hermitian=False)
    assert rel(chi0.sos_drho(m, dV, [0.0, 0.8]), chi0.sternheimer_drho(m, dV, [0.0, 0.8])) < 1e-12


def test_sos_equals_sternheimer_config24(cfg24):
    m = model_of(cfg24)
    dV = synth.perturbations(cfg24.miller_rho, cfg24.L, 2, 2)
    assert rel(chi0.sos_drho(m, dV, [0.0, 1.5]), chi0.sternheimer_drho(m, dV, [0.0, 1.5])) < 1e-11


def test_static_response_is_density_derivative(tiny):
    """chi0(0) dV equals d n / d lambda of the ground state of H + lambda dV (no response formula used)."""
    m = model_of(tiny)
    dV = synth.perturbations(tiny.miller_rho, tiny.L, 2, 8)
    for p in range(2):
        fd = chi0.finite_difference_drho(m, dV[:, p], 1e-3)
        assert rel(chi0.sos_drho(m, dV[:, p], [0.0])[:, 0, 0], fd) < 1e-9


def test_static_response_derivative_with_kb():
    s = synth.make_system(synth.Config("kb", L=6.0, ecut=2.5, grid=12, n_wells=2, well_seed=7,
                                       n_v=2, kb=True))
    m = model_of(s)
    dV = synth.perturbations(s.miller_rho, s.L, 1, 3)[:, 0]
    fd = chi0.finite_difference_drho(m, dV, 1e-3)
    assert rel(chi0.sternheimer_drho(m, dV, [0.0])[:, 0, 0], fd) < 1e-9


def free_model(L=6.0, ecut=3.0, grid=16, n_occ=7):
    mw = sphere(L, ecut)
    mr = sphere(L, 4 * ecut)
    psi = np.zeros((mw.shape[0], n_occ), np.complex128)
    psi[np.arange(n_occ), np.arange(n_occ)] = 1.0
    b = 2 * math.pi / L
    e = 0.5 * b * b * np.sum(mw[:n_occ] ** 2, axis=1)
    return Model(L, ecut, grid, np.zeros(mr.shape[0], np.complex128), psi, e)


@pytest.mark.parametrize("n_occ", [1, 7, 19])
def test_free_electron_closed_form(n_occ):
    m = free_model(n_occ=n_occ)
    mr, diag = chi0.free_electron_chi0_diag(m.L, m.ecut, n_occ, [0.0, 0.6])
    assert np.array_equal(mr, m.mr)
    dV = synth.perturbations(m.mr, m.L, 2, 4)
    ref = diag[:, None, :] * dV[:, :, None]
    assert rel(chi0.sternheimer_drho(m, dV, [0.0, 0.6]), ref) < 1e-12
    assert rel(chi0.sos_drho(m, dV, [0.0, 0.6]), ref) < 1e-12


def test_free_electron_pdep_eigenvalues():
    m = free_model(n_occ=7)
    mr, diag = chi0.free_electron_chi0_diag(m.L, m.ecut, 7, [0.0])
    g2 = m.g2r
    lam = np.sort(np.where(g2 > 0, 4 * math.pi / np.where(g2 > 0, g2, 1) * diag[:, 0], 0.0))
    w, _ = pdep.pdep_dense(m, 20)
    assert np.max(np.abs(w - lam[:20])) < 1e-12 * np.max(np.abs(lam))


# ---------------------------------------------------------------- invariants
def test_chibar0_hermitian_negative_semidefinite(tiny):
    m = model_of(tiny)
    for om in (0.0, 0.9):
        X = chi0.chibar0_matrix(m, om)
        assert np.max(np.abs(X - X.conj().T)) < 1e-14
        assert np.max(np.linalg.eigvalsh(0.5 * (X + X.conj().T))) < 1e-12


def test_charge_conservation_and_linearity(tiny):
    m = model_of(tiny)
    dV = synth.perturbations(tiny.miller_rho, tiny.L, 2, 8)
    i0 = int(np.where(np.all(m.mr == 0, axis=1))[0][0])
    d = chi0.sos_drho(m, dV, [0.0, 0.4])
    assert np.max(np.abs(d[i0])) < 1e-15
    comb = chi0.sos_drho(m, 0.3 * dV[:, 0] - 1.7j * dV[:, 1], [0.0, 0.4])[:, 0, :]
    assert rel(comb, 0.3 * d[:, 0, :] - 1.7j * d[:, 1, :]) < 1e-13


def test_response_decays_monotonically_with_frequency(tiny):
    m = model_of(tiny)
    dV = synth.perturbations(tiny.miller_rho, tiny.L, 1, 8)[:, 0]
    oms = [0.0, 0.1, 0.5, 1.0, 3.0, 10.0]
    d = chi0.sos_drho(m, dV, oms)[:, 0, :]
    q = np.array([np.vdot(dV, d[:, k]).real for k in range(len(oms))])
    assert np.all(q < 0) and np.all(np.diff(q) > 0)


def test_frequency_integral_closed_form(tiny):
    """int_0^inf <a|chi0(iw)|c> dw, by quadrature of the sum over states, equals a form with no empty states."""
    m = model_of(tiny)
    dV = synth.perturbations(tiny.miller_rho, tiny.L, 2, 12)
    # w = s tan(t), t in [0, pi/2): Gauss-Legendre in t.
    x, wq = np.polynomial.legendre.leggauss(400)
    t = 0.25 * math.pi * (x + 1)
    s = 1.0
    oms = s * np.tan(t)
    jac = 0.25 * math.pi * wq * s / np.cos(t) ** 2
    d = chi0.sos_drho(m, dV[:, 1], oms)[:, 0, :]
    integral = np.sum(jac * (dV[:, 0].conj() @ d))
    ref = chi0.frequency_integral_closed_form(m, dV[:, 0], dV[:, 1])
    assert abs(integral - ref) < 1e-9 * abs(ref)


def test_cg_reaches_dense_solution(cfg24):
    m = model_of(cfg24)
    dV = synth.perturbations(cfg24.miller_rho, cfg24.L, 1, 2)
    out, iters = chi0.sternheimer_cg_drho(m, dV, tol=1e-13, return_iters=True)
    assert rel(out, chi0.sternheimer_drho(m, dV, [0.0])[:, :, 0]) < 1e-11
    assert max(iters) < 200


# ---------------------------------------------------------------- PDEP and Lanczos
def test_davidson_matches_dense(tiny):
    m = model_of(tiny)
    X = chi0.chibar0_matrix(m)
    w, U = pdep.pdep_dense(m, 8)
    rng = np.random.default_rng(3)
    th, V, it = pdep.davidson(lambda B: X @ B, X.shape[0], 8, rng.standard_normal((X.shape[0], 8)), tol=1e-12)
    assert np.max(np.abs(th - w)) < 1e-12
    assert np.max(np.abs(V.conj().T @ V - np.eye(8))) < 1e-12
    # Subspace check (eigenvectors are defined up to rotations inside degenerate sets).
    sv = np.linalg.svd(U.conj().T @ V, compute_uv=False)
    assert np.min(sv) > 1 - 1e-8


def test_lanczos_moments_orthogonality_and_exact_limit(tiny):
    m = model_of(tiny)
    rng = np.random.default_rng(5)
    b = rng.standard_normal(m.mw.shape[0]) + 1j * rng.standard_normal(m.mw.shape[0])
    n = 10
    alpha, beta, Q = lanczos.chain(m, b, n)
    assert np.max(np.abs(Q.conj().T @ Q - np.eye(n))) < 1e-13
    T = np.diag(alpha) + np.diag(beta[1:], 1) + np.diag(beta[1:], -1)
    P = np.eye(m.mw.shape[0]) - m.psi_v @ m.psi_v.conj().T
    A = P @ m.h_dense() @ P
    q1 = Q[:, 0]
    Ak, Tk = q1.copy(), np.eye(n)
    for k in range(1, 2 * n - 1):
        Ak = A @ Ak
        Tk = Tk @ T
        assert abs(np.vdot(q1, Ak) - Tk[0, 0]) < 1e-10 * abs(Tk[0, 0])
    # Exact limit: a chain spanning range(P_c) reproduces the spectrum of P_c H P_c there.
    nfull = m.mw.shape[0] - m.psi_v.shape[1]
    alpha, beta, Q = lanczos.chain(m, b, nfull)
    d, _ = lanczos.tridiag_eig(alpha, beta)
    ew = np.linalg.eigvalsh(P @ m.h_dense() @ P)
    ew = np.sort(ew[np.abs(ew) > 1e-9]) if nfull < ew.size else ew
    w_all, _ = np.linalg.eigh(m.h_dense())
    assert np.max(np.abs(np.sort(d) - w_all[m.psi_v.shape[1]:])) < 1e-10


def test_lanczos_chi0_pdep_exact_limit(tiny):
    m = model_of(tiny)
    w, U = pdep.pdep_dense(m, 3)
    oms = [0.0, 0.5, 5.0]
    n = m.mw.shape[0] - m.psi_v.shape[1]
    L, A, B = lanczos.chi0_pdep(m, U, oms, n)
    assert rel(L, lanczos.chi0_pdep_sos(m, U, oms)) < 1e-12
    # In the PDEP basis chi0(0) is diagonal with the PDEP eigenvalues.
    assert np.max(np.abs(L[:, :, 0] - np.diag(w))) < 1e-12


# ---------------------------------------------------------------- planted mistakes
def test_planted_wrong_eigenvalue_fails_sos_pin(tiny):
    """A Sternheimer solve with a shifted e_v (wrong diagonal of Eq. sternheimer) fails the SOS pin."""
    m = model_of(tiny)
    dV = synth.perturbations(tiny.miller_rho, tiny.L, 1, 8)
    good = chi0.sos_drho(m, dV, [0.0])
    m.e_v = m.e_v + 0.01
    assert rel(chi0.sternheimer_drho(m, dV, [0.0]), good) > 1e-3


def test_planted_transposed_grid_fails_dense_h_pin(cfg24, monkeypatch):
    """Placing coefficients on the grid with transposed axes fails the FFT-vs-dense H pin."""
    m = model_of(cfg24)
    H = m.h_dense()
    orig = Model.to_grid

    def transposed(self, c, miller):
        return orig(self, c, miller[:, ::-1]) if miller is self.mr else orig(self, c, miller)
    monkeypatch.setattr(Model, "to_grid", transposed)
    m._vloc_r = None
    x = np.random.default_rng(2).standard_normal(m.mw.shape[0]) + 0j
    assert rel(m.apply_h(x), H @ x) > 1e-3


def test_planted_wrong_spin_factor_fails_closed_form():
    m = free_model(n_occ=7)
    m.f_s = 1.0
    mr, diag = chi0.free_electron_chi0_diag(m.L, m.ecut, 7, [0.0])
    dV = synth.perturbations(m.mr, m.L, 1, 4)
    assert rel(chi0.sos_drho(m, dV, [0.0])[:, 0, 0], diag[:, 0] * dV[:, 0]) > 0.4


def test_planted_missing_projector_fails_sos_pin(tiny, monkeypatch):
    """Solving without P_c on the right-hand side gives a wrong answer that the SOS pin catches."""
    m = model_of(tiny)
    dV = synth.perturbations(tiny.miller_rho, tiny.L, 1, 8)
    monkeypatch.setattr(chi0, "_pc", lambda model, x: x)
    bad = chi0.sternheimer_cg_drho(m, dV, tol=1e-12, max_iter=300)
    monkeypatch.undo()
    assert rel(bad, chi0.sos_drho(m, dV, [0.0])[:, :, 0]) > 1e-3


def test_dyson_closed_form_on_the_spectrum():
    """(1 - A)^-1 A = Q diag(l/(1-l)) Q^T for A = Q diag(l) Q^T; X commutes with A and, for
    negative semidefinite A, has eigenvalues in (-1, 0] (epsilon^-1 - 1)."""
    rng = np.random.default_rng(8)
    n, nw = 12, 3
    A = np.zeros((nw, n, n))
    ref = np.zeros((nw, n, n))
    for k in range(nw):
        Q, _ = np.linalg.qr(rng.standard_normal((n, n)))
        lam = -rng.uniform(0.0, 6.0, n)
        A[k] = (Q * lam) @ Q.T
        ref[k] = (Q * (lam / (1.0 - lam))) @ Q.T
    X = dyson.chibar(A)
    assert np.max(np.abs(X - ref)) < 1e-12
    for k in range(nw):
        assert np.max(np.abs(X[k] @ A[k] - A[k] @ X[k])) < 1e-12
        w = np.linalg.eigvalsh(0.5 * (X[k] + X[k].T))
        assert np.all(w > -1.0) and np.all(w <= 1e-12)
    # Scalar case and a non-symmetric matrix: (1 - a)^-1 a, and (1 - A) X = A.
    assert abs(dyson.chibar(np.array([[-3.0]]))[0, 0] - (-0.75)) < 1e-15
    B = rng.standard_normal((5, 5)) * 0.1
    assert np.max(np.abs((np.eye(5) - B) @ dyson.chibar(B) - B)) < 1e-13


def test_planted_sign_error_fails_dyson_pin():
    """Plant (1 + A)^-1 A in place of (1 - A)^-1 A: the spectral pin must fail."""
    lam = np.array([-0.5, -2.0])
    A = np.diag(lam)
    wrong = np.linalg.solve(np.eye(2) + A, A)
    assert np.max(np.abs(wrong - np.diag(lam / (1.0 - lam)))) > 0.1


# ---------------------------------------------------------------- G0 Lanczos (Eq. ISR, Eq. lanczos)
Z_G0 = np.array([-0.4 + 0.3j, 0.1 + 0.05j, 0.7 + 1.5j, 2.0 + 10.0j])


def test_g0_lanczos_exact_limit_equals_dense_resolvent(tiny):
    """A chain that exhausts its Krylov space gives <b_n|(h - z)^-1|b_m> exactly (h with KB)."""
    m = model_of(tiny)
    phi = synth.perturbations(tiny.miller_rho, tiny.L, 3, 21)
    out = g0.g0_lanczos(m, phi, [0, 1], m.mw.shape[0], Z_G0)
    ref = g0.g0_exact(m, phi, [0, 1], Z_G0)
    assert rel(out["g0"], ref) < 1e-10
    # Real h and real-in-r start vectors: real residues, and a symmetric resolvent matrix.
    assert np.max(np.abs(out["C"].imag)) < 1e-12 * np.max(np.abs(out["C"]))
    assert rel(ref.transpose(0, 1, 3, 2), ref) < 1e-12


def test_g0_free_electron_resolvent_is_diagonal_sum(tiny):
    """V = 0, no projectors: h is diagonal in plane waves, so the dense solve reduces to
    sum_G b_n(G)^* b_m(G) / (|G|^2/2 - z), and the exhausted chain gives the same."""
    m = Model(tiny.L, tiny.ecut, tiny.grid, np.zeros_like(tiny.vloc_G), tiny.psi_v, tiny.e_v)
    phi = synth.perturbations(tiny.miller_rho, tiny.L, 2, 22)
    closed = []
    S = g0.start_vectors(m, phi, 1)
    kin = 0.5 * m.g2w
    for zk in Z_G0:
        closed.append(S.conj().T @ (S / (kin - zk)[:, None]))
    closed = np.asarray(closed)[None]
    assert rel(g0.g0_exact(m, phi, [1], Z_G0), closed) < 1e-12
    assert rel(g0.g0_lanczos(m, phi, [1], m.mw.shape[0], Z_G0)["g0"], closed) < 1e-10


def test_g0_chain_moments_and_orthonormality(tiny):
    """<q1|h^k|q1> = (T^k)_11 for k < 2 n_steps - 1, orthonormal q, unprojected h."""
    m = model_of(tiny)
    phi = synth.perturbations(tiny.miller_rho, tiny.L, 1, 23)
    b = g0.start_vectors(m, phi, 0)[:, 0]
    n = 8
    alpha, beta, Q = g0.chain(m, b, n)
    assert abs(beta[0] - np.linalg.norm(b)) < 1e-14 * beta[0]
    assert np.max(np.abs(Q.conj().T @ Q - np.eye(n))) < 1e-13
    T = np.diag(alpha) + np.diag(beta[1:], 1) + np.diag(beta[1:], -1)
    H = m.h_dense()
    q1 = Q[:, 0]
    hk, Tk = q1.copy(), np.eye(n)
    for k in range(1, 2 * n - 1):
        hk = H @ hk
        Tk = Tk @ T
        assert abs(np.vdot(q1, hk) - Tk[0, 0]) < 1e-10 * abs(Tk[0, 0])


def test_planted_transposed_tridiagonal_vectors_fail_g0_pin(tiny, monkeypatch):
    m = model_of(tiny)
    phi = synth.perturbations(tiny.miller_rho, tiny.L, 2, 24)
    real = g0.scipy.linalg.eigh_tridiagonal

    def transposed(a, b):
        d, U = real(a, b)
        return d, U.T

    monkeypatch.setattr(g0.scipy.linalg, "eigh_tridiagonal", transposed)
    out = g0.g0_lanczos(m, phi, [0], m.mw.shape[0], Z_G0)
    monkeypatch.undo()
    assert rel(out["g0"], g0.g0_exact(m, phi, [0], Z_G0)) > 1e-3


# ---------------------------------------------------------------- spin channels (sum over sigma, Eq. dfpt)
def test_spin_channels_identical_equal_unpolarised(tiny):
    """Two identical channels with f_s = 1 each give the spin-unpolarised response (f_s = 2)."""
    dV = synth.perturbations(tiny.miller_rho, tiny.L, 2, 41)
    one = model_of(tiny, f_s=1.0)
    both = chi0.sos_drho_channels([one, one], dV, [0.0, 0.7])
    assert rel(both, chi0.sos_drho(model_of(tiny), dV, [0.0, 0.7])) < 1e-14


def test_spin_channels_are_derivative_of_total_density():
    """chi0 dV of a spin-polarised model (split wells, N_up != N_down) equals the derivative of
    the total ground-state density of both channels under dV (no response formula used)."""
    up, dn = synth.make_spin_system("tiny_L6_12")
    assert up.psi_v.shape[1] == 2 and dn.psi_v.shape[1] == 1
    assert np.array_equal(up.positions, dn.positions)
    models = [model_of(up, f_s=1.0), model_of(dn, f_s=1.0)]
    dV = synth.perturbations(up.miller_rho, up.L, 1, 42)[:, 0]
    fd = sum(chi0.finite_difference_drho(m, dV, 1e-3) for m in models)
    assert rel(chi0.sos_drho_channels(models, dV, [0.0])[:, 0, 0], fd) < 1e-9


def test_static_response_derivative_with_d_channels():
    """KB with s, p and d channels (9 per atom): the static response still equals the density
    derivative, and the dense H still equals its FFT application."""
    s = synth.make_system(synth.Config("kbd", L=6.0, ecut=2.5, grid=12, n_wells=2, well_seed=7,
                                       n_v=2, kb=True, kb_dch=True))
    assert s.beta_G.shape[1] == 18
    m = model_of(s)
    rng = np.random.default_rng(3)
    x = rng.standard_normal((m.mw.shape[0], 2)) + 1j * rng.standard_normal((m.mw.shape[0], 2))
    assert rel(m.apply_h(x), m.h_dense() @ x) < 1e-13
    dV = synth.perturbations(s.miller_rho, s.L, 1, 43)[:, 0]
    fd = chi0.finite_difference_drho(m, dV, 1e-3)
    assert rel(chi0.sos_drho(m, dV, [0.0])[:, 0, 0], fd) < 1e-9


# ---------------------------------------------------------------- exchange self-energy (Eq. sigmacIR)
def _convolution_pair_density(m, ci, cj):
    """sum_G1 c_i(G1)^* c_j(G1 + G) on the density sphere (direct G-space route)."""
    where = {tuple(g): k for k, g in enumerate(m.mw.tolist())}
    out = np.zeros(m.mr.shape[0], np.complex128)
    for a, G in enumerate(m.mr.tolist()):
        acc = 0.0
        for k1, G1 in enumerate(m.mw.tolist()):
            k2 = where.get((G1[0] + G[0], G1[1] + G[1], G1[2] + G[2]))
            if k2 is not None:
                acc += np.conj(ci[k1]) * cj[k2]
        out[a] = acc
    return out


def test_pair_density_equals_convolution(tiny):
    m = model_of(tiny)
    for i, j in ((0, 0), (0, 1), (1, 0)):
        got = sigma.pair_density(m, m.psi_v[:, i], m.psi_v[:, j])
        ref = _convolution_pair_density(m, m.psi_v[:, i], m.psi_v[:, j])
        assert rel(got, ref) < 1e-13


def test_sigma_x_plane_waves_closed_form():
    """Plane-wave states e^{ik.r}: <i|Sigma_X|i> = -(1/Omega) sum_{j != i} 4 pi / |k_j - k_i|^2."""
    m = free_model(n_occ=7)
    got = sigma.sigma_x(m)
    k = m.b * m.mw[:7].astype(np.float64)
    ref = []
    for i in range(7):
        d2 = np.sum((k - k[i]) ** 2, axis=1)
        ref.append(-np.sum(4 * np.pi / d2[np.arange(7) != i]) / m.omega)
    assert np.max(np.abs(got - np.asarray(ref))) < 1e-12 * np.max(np.abs(ref))


def test_sigma_x_total_invariant_under_rotation(tiny):
    m = model_of(tiny)
    rng = np.random.default_rng(81)
    Q, _ = np.linalg.qr(rng.standard_normal((2, 2)) + 1j * rng.standard_normal((2, 2)))
    rot = Model(tiny.L, tiny.ecut, tiny.grid, tiny.vloc_G, tiny.psi_v @ Q, tiny.e_v)
    a, b = sigma.sigma_x(m), sigma.sigma_x(rot)
    assert abs(np.sum(a) - np.sum(b)) < 1e-13 * abs(np.sum(a))
    assert np.all(a < 0)


def test_planted_missing_conjugate_fails_pair_density_pin(tiny, monkeypatch):
    m = model_of(tiny)
    ci = m.psi_v[:, 0] * np.exp(0.7j)        # a phase makes the conjugate matter
    monkeypatch.setattr(sigma.np, "conj", lambda x: x)
    got = sigma.pair_density(m, ci, m.psi_v[:, 1])
    monkeypatch.undo()
    assert rel(got, _convolution_pair_density(m, ci, m.psi_v[:, 1])) > 1e-3


def test_isr_quadrature_converges_to_arctan_closed_form(tiny):
    """Lambda = c * identity at every node, exhausted chains: the folded quadrature over [0, W]
    of Eq. ISR approaches (c/Omega) sum_n <b_n|(1/pi) arctan(W/(h - w))|b_n>."""
    m = model_of(tiny)
    phi = synth.perturbations(tiny.miller_rho, tiny.L, 2, 82)
    W, c = 30.0, 0.37
    x, wts = np.polynomial.legendre.leggauss(400)
    # Composite Gauss-Legendre: [0, 2] resolves the peak of 2x/(x^2 + w'^2) near the spectrum.
    nodes = np.concatenate([(x + 1.0), 2.0 + 0.5 * (W - 2.0) * (x + 1.0)])
    weights = np.concatenate([wts, 0.5 * (W - 2.0) * wts])
    lam = np.broadcast_to(c * np.eye(2), (nodes.size, 2, 2))
    omegas = [0.23, -1.7]                       # away from the spectrum of h
    got = sigma.isr(m, phi, [1], m.mw.shape[0], omegas, lam, nodes, weights)
    e, U = np.linalg.eigh(m.h_dense())
    S = g0.start_vectors(m, phi, 1)
    Y = U.conj().T @ S
    ref = np.array([c / m.omega * np.sum(np.abs(Y) ** 2 * (np.arctan(W / (e - w)) / np.pi)[:, None])
                    for w in omegas])
    assert np.max(np.abs(got[0] - ref)) < 1e-9 * np.max(np.abs(ref))
    assert np.max(np.abs(got.imag)) < 1e-12 * np.max(np.abs(ref))


def _real_orthonormal_basis(s, n, seed):
    Q, _ = np.linalg.qr(synth.perturbations(s.miller_rho, s.L, n, seed))
    return Q


def test_isr_lanczos_equals_dense_resolvent(tiny):
    """I^SR with exhausted G0 chains equals I^SR with the exact resolvent of the dense h."""
    m = model_of(tiny)
    phi = _real_orthonormal_basis(tiny, 2, 83)
    x, wts = np.polynomial.legendre.leggauss(24)
    nodes, weights = 4.0 * (x + 1.0), 4.0 * wts
    lam = np.array([sigma.lam_basis(m, phi, 1j * wp).real for wp in nodes])
    omegas = [-0.9, 0.05, 0.6]
    a = sigma.isr(m, phi, [0], m.mw.shape[0], omegas, lam, nodes, weights)[0]
    b = sigma.isr_dense(m, phi, 0, omegas, lam, nodes, weights)
    assert np.max(np.abs(a - b)) < 1e-11 * np.max(np.abs(b))


@pytest.mark.parametrize("j_of", ["lumo", "homo"])
def test_contour_deformation_terms_continuous_across_a_pole(tiny, j_of):
    """Eq. sigmacIR: I(w) jumps by -(1/Omega) sum_nm Lambda_nm(0) <b_n|j><j|b_m> where w crosses an
    eigenvalue e_j of h, and the residue term R(w) (Eq. Rfac) jumps back: I + R is continuous."""
    m = model_of(tiny)
    phi = _real_orthonormal_basis(tiny, 2, 84)
    e = np.linalg.eigvalsh(m.h_dense())
    nv = tiny.n_v
    ej = e[nv] if j_of == "lumo" else e[nv - 1]
    e_fermi = 0.5 * (e[nv - 1] + e[nv])
    edges = [0.0, 1e-7, 1e-6, 1e-5, 1e-4, 1e-3, 1e-2, 0.1, 1.0, 10.0, 60.0]
    x, wts = np.polynomial.legendre.leggauss(60)
    nodes = np.concatenate([a + 0.5 * (b - a) * (x + 1.0) for a, b in zip(edges[:-1], edges[1:])])
    weights = np.concatenate([0.5 * (b - a) * wts for a, b in zip(edges[:-1], edges[1:])])
    lam = np.array([sigma.lam_basis(m, phi, 1j * wp) for wp in nodes])
    d = 1e-6
    om = [ej - d, ej + d]
    i_ = sigma.isr_dense(m, phi, 0, om, lam, nodes, weights)
    r_ = sigma.residue_term(m, phi, 0, om, e_fermi)
    _, Y = sigma._spectral_overlaps(m, phi, 0)
    jj = np.where(np.abs(e - ej) < 1e-9)[0]
    A = sum(np.outer(Y[j].conj(), Y[j]) for j in jj)
    jump = -np.sum(sigma.lam_basis(m, phi, 0.0) * A) / m.omega
    assert abs(jump) > 1e-8
    assert abs((i_[1] - i_[0]) - jump) < 1e-3 * abs(jump)
    assert abs((i_[1] + r_[1]) - (i_[0] + r_[0])) < 1e-3 * abs(jump)


def _half_line_quadrature(n=60):
    """Nodes and weights for int_0^inf: composite Gauss-Legendre panels on [0, 100] refined
    towards 0, and the tail [100, inf) mapped onto (0, 1] by w' = 100 / u."""
    edges = [0.0, 1e-4, 1e-3, 1e-2, 0.1, 1.0, 10.0, 100.0]
    x, wts = np.polynomial.legendre.leggauss(n)
    nodes = [a + 0.5 * (b - a) * (x + 1.0) for a, b in zip(edges[:-1], edges[1:])]
    weights = [0.5 * (b - a) * wts for a, b in zip(edges[:-1], edges[1:])]
    u = 0.5 * (x + 1.0)
    nodes.append(100.0 / u)
    weights.append(0.5 * wts * 100.0 / u ** 2)
    return np.concatenate(nodes), np.concatenate(weights)


@pytest.mark.parametrize("where", ["gap", "below", "inside_occupied", "above_lumo"])
def test_static_screening_gives_cohsex_closed_form(tiny, where):
    """Frequency-independent W_p (Lambda = c * identity at every frequency): I + R of Eq. sigmacIR
    is the static COHSEX self-energy (c/Omega) sum_j sum_n |<j|b_n>|^2 (1/2 - theta(e_F - e_j)),
    whatever w: a Coulomb hole of +1/2 over every eigenstate j of h and a screened exchange of -1
    over the occupied ones (the sign of the exchange sum of Sigma_X).  Pins the overall sign of the
    imaginary-axis integral of Eq. Ifac / Eq. ISR and of the residue term of Eq. Rfac."""
    m = model_of(tiny)
    phi = _real_orthonormal_basis(tiny, 2, 86)
    e = np.linalg.eigvalsh(m.h_dense())
    nv = tiny.n_v
    e_fermi = 0.5 * (e[nv - 1] + e[nv])
    w = {"gap": e_fermi, "below": e[0] - 0.5, "inside_occupied": 0.5 * (e[0] + e[1]),
         "above_lumo": 0.5 * (e[nv] + e[nv + 1])}[where]
    assert np.min(np.abs(e - w)) > 1e-3
    c = 0.3
    nodes, weights = _half_line_quadrature()
    lam = np.broadcast_to(c * np.eye(2), (nodes.size, 2, 2))
    i_ = sigma.isr_dense(m, phi, 0, [w], lam, nodes, weights)[0]
    r_ = sigma.residue_term(m, phi, 0, [w], e_fermi, lam_fn=lambda z: c * np.eye(2))[0]
    _, Y = sigma._spectral_overlaps(m, phi, 0)
    weight = np.where(e <= e_fermi, -0.5, 0.5)
    ref = c / m.omega * np.sum(np.abs(Y) ** 2 * weight[:, None])
    assert abs(ref) > 1e-6
    assert abs((i_ + r_) - ref) < 1e-8 * abs(ref), (i_, r_, ref)
    # The screened-exchange part alone carries the sign of Sigma_X: -(c/Omega) sum_occ |<j|b>|^2.
    sex = -c / m.omega * np.sum(np.abs(Y[:nv]) ** 2)
    coh = 0.5 * c / m.omega * np.sum(np.abs(Y) ** 2)
    assert abs((sex + coh) - ref) < 1e-12 * abs(ref) and sex < 0


def test_planted_integral_sign_error_fails_cohsex_pin(tiny, monkeypatch):
    m = model_of(tiny)
    phi = _real_orthonormal_basis(tiny, 2, 86)
    e = np.linalg.eigvalsh(m.h_dense())
    nv = tiny.n_v
    e_fermi = 0.5 * (e[nv - 1] + e[nv])
    c = 0.3
    nodes, weights = _half_line_quadrature()
    lam = np.broadcast_to(c * np.eye(2), (nodes.size, 2, 2))
    real = sigma.isr_dense
    monkeypatch.setattr(sigma, "isr_dense", lambda *a, **k: -real(*a, **k))
    i_ = sigma.isr_dense(m, phi, 0, [e_fermi], lam, nodes, weights)[0]
    monkeypatch.undo()
    r_ = sigma.residue_term(m, phi, 0, [e_fermi], e_fermi, lam_fn=lambda z: c * np.eye(2))[0]
    _, Y = sigma._spectral_overlaps(m, phi, 0)
    ref = c / m.omega * np.sum(np.abs(Y) ** 2 * np.where(e <= e_fermi, -0.5, 0.5)[:, None])
    assert abs((i_ + r_) - ref) > 0.1 * abs(ref)


def test_planted_residue_sign_error_breaks_continuity(tiny, monkeypatch):
    m = model_of(tiny)
    phi = _real_orthonormal_basis(tiny, 2, 84)
    e = np.linalg.eigvalsh(m.h_dense())
    nv = tiny.n_v
    ej, e_fermi = e[nv], 0.5 * (e[nv - 1] + e[nv])
    edges = [0.0, 1e-7, 1e-6, 1e-5, 1e-4, 1e-3, 1e-2, 0.1, 1.0, 10.0, 60.0]
    x, wts = np.polynomial.legendre.leggauss(60)
    nodes = np.concatenate([a + 0.5 * (b - a) * (x + 1.0) for a, b in zip(edges[:-1], edges[1:])])
    weights = np.concatenate([0.5 * (b - a) * wts for a, b in zip(edges[:-1], edges[1:])])
    lam = np.array([sigma.lam_basis(m, phi, 1j * wp) for wp in nodes])
    om = [ej - 1e-6, ej + 1e-6]
    real = sigma.residue_term
    monkeypatch.setattr(sigma, "residue_term", lambda *a, **k: -real(*a, **k))
    i_ = sigma.isr_dense(m, phi, 0, om, lam, nodes, weights)
    r_ = sigma.residue_term(m, phi, 0, om, e_fermi)
    monkeypatch.undo()
    jump = i_[1] - i_[0]
    assert abs((i_[1] + r_[1]) - (i_[0] + r_[0])) > 0.5 * abs(jump)


def test_qp_secant_solves_a_pole_model_exactly():
    """Sigma(E) = a + b / (E - c) (one pole): e_i + Re Sigma(E) - E = 0 is a quadratic whose root
    near e_i is known in closed form; the secant solve reaches it."""
    e_i, a, b, c = -0.3, -0.05, 0.02, 0.4
    E = sigma.qp_energy(e_i, lambda E: a + b / (E - c))
    # (e_i + a - E)(E - c) + b = 0  ->  E^2 - (e_i + a + c) E + c (e_i + a) - b = 0
    p, q = e_i + a + c, c * (e_i + a) - b
    roots = np.array([(p - np.sqrt(p * p - 4 * q)) / 2, (p + np.sqrt(p * p - 4 * q)) / 2])
    ref = roots[np.argmin(np.abs(roots - e_i))]
    assert abs(E - ref) < 1e-10
    assert abs(e_i + a + b / (E - c) - E) < 1e-10


def test_lanczos_chi0_at_complex_frequency(tiny):
    """chi0_pdep_z: z = i w reproduces chi0_pdep; with chains spanning range(P_c), z = w + i eta at a
    real w (inside and beyond the gap) equals the dense sum over states at that z."""
    m = model_of(tiny)
    phi = synth.perturbations(tiny.miller_rho, tiny.L, 2, 85)
    n_full = m.mw.shape[0] - m.psi_v.shape[1]
    a = lanczos.chi0_pdep_z(m, phi, [0.7j], 6)[:, :, 0]
    b = lanczos.chi0_pdep(m, phi, [0.7], 6)[0][:, :, 0]
    assert rel(a, b) < 1e-13
    pt = m.vsqrt[:, None] * phi
    for z in (0.1 + 0.01j, 1.3 + 0.05j):
        got = lanczos.chi0_pdep_z(m, phi, [z], n_full)[:, :, 0]
        ref = pt.conj().T @ sigma.chi0_z(m, z) @ pt
        assert rel(got, ref) < 1e-10, z
