"""Dyson equation in the PDEP basis at imaginary frequencies (oracle, FP64).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Passage followed (Sec. 2, the screened response from the independent-particle one): with
chibar0 = v^1/2 chi0 v^1/2 the symmetrised independent-particle response, the symmetrised
reducible response is chibar = (1 - chibar0)^-1 chibar0 = epsilon^-1 - 1, evaluated in the
PDEP basis for every imaginary frequency.

Reading: the matrices are taken as given (no symmetrisation), so the result is the plain
solution of (1 - A) X = A per frequency, for A in the layout of the library's
chi0_pdep output (frequency-major, then row, then column).

Pins (tests/test_oracle_pins.py): for A = Q diag(l) Q^T with orthogonal Q the result is
Q diag(l / (1 - l)) Q^T (the closed form on the spectrum); X commutes with A; and for
negative semidefinite A the eigenvalues of X lie in (-1, 0].
"""
from __future__ import annotations

import numpy as np


def chibar(chi0bar: np.ndarray) -> np.ndarray:
    """(1 - A)^-1 A for each matrix A of chi0bar, shape (n_omega, n, n) (or (n, n))."""
    a = np.asarray(chi0bar, np.float64)
    single = a.ndim == 2
    a = a[None] if single else a
    n = a.shape[-1]
    eye = np.eye(n)
    out = np.stack([np.linalg.solve(eye - a[k], a[k]) for k in range(a.shape[0])])
    return out[0] if single else out
