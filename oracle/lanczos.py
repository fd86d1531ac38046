"""Lanczos chains and chi0 in the PDEP basis at imaginary frequencies (oracle, FP64).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Paper passages followed (Sec. 3, the recurrence above Eq. lanczos and Eq. lanczos):
  q^{l+1} = [(h - alpha_l) q^l - beta_l q^{l-1}] / beta_{l+1},  q^0 = 0,
  alpha_l = <q^l|h|q^l>,  beta_{l+1} = || (h - alpha_l) q^l - beta_l q^{l-1} ||,
  new vectors orthogonalised against all previous ones;
  d, U = eigenvalues / eigenvectors of the tridiagonal matrix (alpha on the
  diagonal, beta off it), so that the frequency dependence is analytic.

Readings:
  * The chain runs on P_c h P_c (every new vector is re-projected with P_c) and
    starts from b = P_c [phi~_m psi_v] (phi~_m = v^1/2 phi_m), with
    q^1 = b / ||b|| and beta_1 := ||b|| (the paper writes q^1 = |psi phi~> without
    the normalisation).
  * chi0 in the PDEP basis follows by resolving P_c (h - e_v -/+ i w)^-1 P_c
    in the chain:
      chi0_nm(i w) = (f_s/Omega) sum_v beta_1 sum_{l,l'} <P_c phi~_n psi_v | q^l> U_{l l'} U_{1 l'}
                     [1/(e_v - d_l' - i w) + 1/(e_v - d_l' + i w)].
  * Full reorthogonalisation: two classical Gram-Schmidt passes per step.

chi0_pdep_z evaluates the same chains at complex frequencies z (z = w + i eta: a real
frequency with a broadening, as the residue term of Eq. Rfac needs).

Pins: the moment identity <q1|A^k|q1> = (T^k)_11 for k < 2 n_steps,
orthonormality of Q, eig(T) = eig of P_c h P_c on range(P_c) when the chain
spans it, and chi0_nm(Lanczos) = chi0_nm(sum over states) in that limit, at imaginary and
at complex frequencies inside and beyond the gap.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg

from .model import Model


def _pc(model: Model, x: np.ndarray) -> np.ndarray:
    P = model.psi_v
    return x - P @ (P.conj().T @ x)


def chain(model: Model, b: np.ndarray, n_steps: int):
    """One Lanczos chain on P_c H P_c from b.  Returns alpha (n), beta (n; beta[0] = ||b||), Q (N_pw x n)."""
    b = _pc(model, np.asarray(b, np.complex128))
    beta = np.zeros(n_steps)
    alpha = np.zeros(n_steps)
    Q = np.zeros((b.size, n_steps), np.complex128)
    beta[0] = np.linalg.norm(b)
    q = b / beta[0]
    q_prev = np.zeros_like(q)
    for l in range(n_steps):
        Q[:, l] = q
        hq = _pc(model, model.apply_h(q))
        alpha[l] = np.vdot(q, hq).real
        r = hq - alpha[l] * q - (beta[l] * q_prev if l > 0 else 0.0)
        for _ in range(2):
            r = _pc(model, r - Q[:, : l + 1] @ (Q[:, : l + 1].conj().T @ r))
        if l + 1 < n_steps:
            beta[l + 1] = np.linalg.norm(r)
            q_prev, q = q, r / beta[l + 1]
    return alpha, beta, Q


def tridiag_eig(alpha: np.ndarray, beta: np.ndarray):
    """d, U of the tridiagonal matrix with alpha on the diagonal and beta[1:] off it."""
    return scipy.linalg.eigh_tridiagonal(alpha, beta[1:])


def chi0_pdep(model: Model, phi: np.ndarray, omegas, n_steps: int):
    """chi0_nm(i w) in the PDEP basis phi (N_rho x n_pdep) from Lanczos chains of every (v, m).

    Returns (chi0 of shape (n_pdep, n_pdep, n_omega), alpha, beta of shape (n_v, n_pdep, n_steps)).
    """
    phi = np.asarray(phi, np.complex128)
    nv = model.psi_v.shape[1]
    npd = phi.shape[1]
    omegas = np.asarray(omegas, np.float64)
    out = np.zeros((npd, npd, omegas.size), np.complex128)
    A = np.zeros((nv, npd, n_steps))
    B = np.zeros((nv, npd, n_steps))
    for v in range(nv):
        pv = model.to_r(model.psi_v[:, v], model.mw)
        # P_c [phi~_n psi_v] for every n (the bras and the chain starts).
        S = np.stack([_pc(model, model.to_G(model.to_r(model.vsqrt * phi[:, n], model.mr) * pv, model.mw))
                      for n in range(npd)], axis=1)
        for m in range(npd):
            alpha, beta, Q = chain(model, S[:, m], n_steps)
            A[v, m], B[v, m] = alpha, beta
            d, U = tridiag_eig(alpha, beta)
            ov = S.conj().T @ Q                     # <P_c phi~_n psi_v | q^l>, (npd, n_steps)
            for k, om in enumerate(omegas):
                g = 1.0 / (model.e_v[v] - d - 1j * om) + 1.0 / (model.e_v[v] - d + 1j * om)
                out[:, m, k] += beta[0] * (ov @ (U @ (g * U[0, :])))
    return out * (model.f_s / model.omega), A, B


def chi0_pdep_sos(model: Model, phi: np.ndarray, omegas):
    """chi0_nm(i w) = <phi~_n| chi0(i w) |phi~_m> from the sum over states, for comparison."""
    from .chi0 import sos_drho
    phi = np.asarray(phi, np.complex128)
    drho = sos_drho(model, model.vsqrt[:, None] * phi, omegas)   # (N_rho, npd, n_omega)
    return np.einsum("gn,gmk->nmk", (model.vsqrt[:, None] * phi).conj(), drho)


def chi0_pdep_z(model: Model, phi: np.ndarray, zs, n_steps: int) -> np.ndarray:
    """chi0_nm(z) in the basis phi at complex frequencies z from the same chains as chi0_pdep:
    the i w of Eq. lanczos replaced by z, g = 1/(e_v - d - z) + 1/(e_v - d + z) (z = i w gives
    chi0_pdep; z = w + i eta gives the response at a real frequency w with a broadening eta).
    Returns shape (n_pdep, n_pdep, n_z)."""
    phi = np.asarray(phi, np.complex128)
    zs = np.asarray(zs, np.complex128).ravel()
    nv = model.psi_v.shape[1]
    npd = phi.shape[1]
    out = np.zeros((npd, npd, zs.size), np.complex128)
    for v in range(nv):
        pv = model.to_r(model.psi_v[:, v], model.mw)
        S = np.stack([_pc(model, model.to_G(model.to_r(model.vsqrt * phi[:, n], model.mr) * pv, model.mw))
                      for n in range(npd)], axis=1)
        for m in range(npd):
            alpha, beta, Q = chain(model, S[:, m], n_steps)
            d, U = tridiag_eig(alpha, beta)
            ov = S.conj().T @ Q
            for k, z in enumerate(zs):
                g = 1.0 / (model.e_v[v] - d - z) + 1.0 / (model.e_v[v] - d + z)
                out[:, m, k] += beta[0] * (ov @ (U @ (g * U[0, :])))
    return out * (model.f_s / model.omega)
