"""PDEP basis: leading eigenpairs of chi0bar(w = 0) (oracle, FP64).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Paper passages followed (Sec. 3): the PDEP basis is the set of N_PDEP leading
eigenvectors of the symmetrised response chi0bar at zero frequency, found with
the Davidson method: start from an orthonormal set of N_PDEP trial vectors,
apply chi0bar, expand the set with the residuals, repeat until the set holds
the N_PDEP leading eigenvectors; the subspace is at most 4 N_PDEP (Sec. 4.2).

Readings (the paper gives no preconditioner, start or stopping rule):
  * "leading" = most negative eigenvalues (chi0bar is negative semidefinite),
    returned in ascending order;
  * seeded random orthonormal start, unpreconditioned residual expansion,
    restart to the current Ritz vectors when the subspace would exceed
    4 N_PDEP;
  * converged when max |lambda_i^(k) - lambda_i^(k-1)| <= tol and every Ritz
    residual norm <= sqrt(tol).

Pins: pdep_dense is a plain eigendecomposition of the dense chi0bar; the
Davidson iteration is pinned to it (tests/test_oracle_pins.py), and on the
free-electron model the eigenvalues equal the sorted closed-form (4 pi/|G|^2) chi0_GG.
"""
from __future__ import annotations

import numpy as np

from .chi0 import chibar0_matrix
from .model import Model


def pdep_dense(model: Model, n_pdep: int):
    """Lowest n_pdep eigenpairs of the dense chi0bar(0) (eigenvalues ascending)."""
    X = chibar0_matrix(model, 0.0)
    X = 0.5 * (X + X.conj().T)
    w, U = np.linalg.eigh(X)
    return w[:n_pdep], U[:, :n_pdep]


def _orthonormalise(V: np.ndarray, against: np.ndarray | None = None) -> np.ndarray:
    """Two passes of classical Gram-Schmidt against `against`, then QR; drops nothing."""
    for _ in range(2):
        if against is not None and against.shape[1]:
            V = V - against @ (against.conj().T @ V)
    Q, R = np.linalg.qr(V)
    return Q


def davidson(apply, n: int, n_pdep: int, x0: np.ndarray, tol: float = 1e-10,
             max_iter: int = 200, factor: int = 4):
    """Block Davidson for the n_pdep lowest eigenpairs of a Hermitian operator.

    apply(V) returns the operator applied to the columns of V (shape n x k).
    x0: n x n_pdep start block (orthonormalised here).
    Returns (eigenvalues ascending, eigenvectors n x n_pdep, iterations).
    """
    V = _orthonormalise(np.asarray(x0, np.complex128))
    W = apply(V)
    prev = None
    for it in range(1, max_iter + 1):
        T = V.conj().T @ W
        T = 0.5 * (T + T.conj().T)
        theta, Y = np.linalg.eigh(T)
        theta, Y = theta[:n_pdep], Y[:, :n_pdep]
        X = V @ Y
        R = W @ Y - X * theta[None, :]
        rnorm = np.linalg.norm(R, axis=0)
        if prev is not None and np.max(np.abs(theta - prev)) <= tol and np.max(rnorm) <= np.sqrt(tol):
            return theta, X, it
        prev = theta
        if V.shape[1] + n_pdep > factor * n_pdep:
            # Restart from the Ritz vectors (and their images).
            V, W = X, W @ Y
        new = _orthonormalise(R, V)
        V = np.concatenate([V, new], axis=1)
        W = np.concatenate([W, apply(new)], axis=1)
    raise RuntimeError("Davidson did not converge")
