"""G0 Lanczos chains for the short-range correlation integral I^SR (oracle, FP64).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Paper passages followed (Sec. 3, Eq. ISR, the Lanczos recurrence under it and
Eq. lanczos): the Green's-function factor of I^SR is the matrix element
<psi_i phi~_n | (h - z)^-1 | psi_i phi~_m> at the complex frequency
z = w + i w'.  For every PDEP index m one Lanczos chain of h (the Kohn-Sham
Hamiltonian itself, NOT projected) starts from psi_i phi~_m; with d, U the
eigenvalues / eigenvectors of the chain's tridiagonal matrix,
  <psi_i phi~_n | (h - z)^-1 | psi_i phi~_m>
      = beta_1 sum_{l,l'} <psi_i phi~_n | q^l_m> U_{l l'} U_{1 l'} / (d_l' - z),
so that the frequency enters only through 1 / (d - z) and one chain serves
every z.

Readings (the paper leaves these open):
  * phi~_m = v^1/2 phi_m with phi_m a PDEP vector on the density sphere; the
    product psi_i(r) phi~_m(r) is truncated to the wavefunction sphere, the
    space the chain (and h) lives in.
  * q^1 = b / ||b|| and beta_1 := ||b||, b = [psi_i phi~_m] (the paper writes
    q^1 = |psi phi~> without the normalisation); the factor beta_1 above
    restores it.
  * Full re-orthogonalisation, two classical Gram-Schmidt passes per step
    (the paper: new vectors are orthogonalised against the previous ones).
  * A chain whose new residual norm falls to <= 1e-14 beta_1 stops: its later
    vectors and beta are zero (the Krylov space is exhausted).
  * The frequency-independent part is returned as residues
    C[n, l', m] = beta_1,m U_{1 l'} sum_l <b_n | q^l_m> U_{l l'}, so that
    g0(z)[n, m] = sum_l' C[n, l', m] / (d_{m,l'} - z).

Pins (tests/test_oracle_pins.py): with the chain spanning the Krylov space
the result equals a dense solve of (h - z) x = b (g0_exact); for V = 0 the
dense solve itself reduces to the diagonal sum over plane waves
sum_G b_n(G)^* b_m(G) / (|G|^2/2 - z); the moment identity of the chain.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg

from .model import Model


def start_vectors(model: Model, phi: np.ndarray, i: int) -> np.ndarray:
    """b_m = [psi_i phi~_m] on the wavefunction sphere, phi~_m = v^1/2 phi_m; shape (N_pw, n_pdep)."""
    phi = np.asarray(phi, np.complex128)
    pi = model.to_r(model.psi_v[:, i], model.mw)
    return np.stack([model.to_G(model.to_r(model.vsqrt * phi[:, n], model.mr) * pi, model.mw)
                     for n in range(phi.shape[1])], axis=1)


def chain(model: Model, b: np.ndarray, n_steps: int):
    """Lanczos chain of h (unprojected) from b: alpha (n), beta (n; beta[0] = ||b||), Q (N_pw x n)."""
    b = np.asarray(b, np.complex128)
    alpha = np.zeros(n_steps)
    beta = np.zeros(n_steps)
    Q = np.zeros((b.size, n_steps), np.complex128)
    beta[0] = np.linalg.norm(b)
    q = b / beta[0]
    q_prev = np.zeros_like(q)
    for l in range(n_steps):
        Q[:, l] = q
        hq = model.apply_h(q)
        alpha[l] = np.vdot(q, hq).real
        r = hq - alpha[l] * q - (beta[l] * q_prev if l > 0 else 0.0)
        for _ in range(2):
            r = r - Q[:, : l + 1] @ (Q[:, : l + 1].conj().T @ r)
        if l + 1 < n_steps:
            nr = np.linalg.norm(r)
            if nr <= 1e-14 * beta[0]:
                q_prev, q = q, np.zeros_like(q)     # exhausted: beta and later q stay zero
            else:
                beta[l + 1] = nr
                q_prev, q = q, r / nr
    return alpha, beta, Q


def g0_lanczos(model: Model, phi: np.ndarray, states, n_steps: int, z=()):
    """Chains of every (i, m) and the resolvent matrices at the frequencies z.

    Returns a dict with alpha, beta, d (n_states, n_pdep, n_steps), the residues
    C (n_states, n_pdep, n_steps, n_pdep) as [i, n, l', m] (complex here; real when
    psi_i and phi are real in r, as at the Gamma point), and
    g0 (n_states, n_z, n_pdep, n_pdep) complex as [i, k, n, m].
    """
    phi = np.asarray(phi, np.complex128)
    z = np.asarray(z, np.complex128).ravel()
    npd = phi.shape[1]
    ns = len(states)
    A = np.zeros((ns, npd, n_steps))
    B = np.zeros((ns, npd, n_steps))
    D = np.zeros((ns, npd, n_steps))
    C = np.zeros((ns, npd, n_steps, npd), np.complex128)
    G = np.zeros((ns, z.size, npd, npd), np.complex128)
    for ii, i in enumerate(states):
        S = start_vectors(model, phi, i)
        for m in range(npd):
            alpha, beta, Q = chain(model, S[:, m], n_steps)
            d, U = scipy.linalg.eigh_tridiagonal(alpha, beta[1:])
            A[ii, m], B[ii, m], D[ii, m] = alpha, beta, d
            ov = S.conj().T @ Q                         # <b_n | q^l_m>
            C[ii, :, :, m] = beta[0] * (ov @ U) * U[0, :][None, :]
            for k, zk in enumerate(z):
                G[ii, k, :, m] = C[ii, :, :, m] @ (1.0 / (d - zk))
    return dict(alpha=A, beta=B, d=D, C=C, g0=G)


def g0_exact(model: Model, phi: np.ndarray, states, z) -> np.ndarray:
    """<b_n | (h - z)^-1 | b_m> by dense solves with the dense h; shape (n_states, n_z, n_pdep, n_pdep)."""
    z = np.asarray(z, np.complex128).ravel()
    H = model.h_dense()
    I = np.eye(H.shape[0])
    out = []
    for i in states:
        S = start_vectors(model, phi, i)
        out.append([S.conj().T @ np.linalg.solve(H - zk * I, S) for zk in z])
    return np.asarray(out)
