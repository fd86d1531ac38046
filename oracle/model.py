"""Plane-wave model: spheres, grid maps and the Kohn-Sham Hamiltonian (oracle, FP64).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Paper passages followed:
  * Sec. 2.2: wavefunction sphere (N_psi = N_PW) and density sphere (N_rho ~ 8 N_psi).
  * Sec. 4.1: dual-space application of h_KS -- kinetic term in reciprocal
    space, local potential in direct space, one inverse and one forward FFT.
  * Sec. 3: norm-conserving (Kleinman-Bylander) nonlocal term.

Conventions: f(r_j) = sum_G f(G) e^{iG.r_j}; f(G) = (1/N_g) sum_j f(r_j) e^{-iG.r_j}
(numpy's ifftn / fftn up to the factor N_g).

Pins (tests/test_oracle_pins.py): the FFT application equals the dense matrix
product on alias-free grids; the sphere enumeration matches a brute-force
count of lattice points; H is Hermitian and the given psi_v are its lowest
eigenvectors.
"""
from __future__ import annotations

import math

import numpy as np


def sphere(L: float, ecut: float) -> np.ndarray:
    """Miller triples (h,k,l) with 0.5 (2pi/L)^2 (h^2+k^2+l^2) <= ecut.

    Ordered by h^2+k^2+l^2, then (h, k, l) lexicographically -- the ordering the
    library documents for its inputs and outputs.
    """
    b = 2.0 * math.pi / L
    m = int(math.sqrt(2.0 * ecut) / b) + 1
    pts = []
    for h in range(-m, m + 1):
        for k in range(-m, m + 1):
            for l in range(-m, m + 1):
                n2 = h * h + k * k + l * l
                if 0.5 * b * b * n2 <= ecut * (1.0 + 1e-12):
                    pts.append((n2, h, k, l))
    pts.sort()
    return np.array([p[1:] for p in pts], dtype=np.int64).reshape(-1, 3)


class Model:
    """The inputs of the response calculation, held in full-sphere complex form."""

    def __init__(self, L, ecut, grid, vloc_G, psi_v, e_v, beta_G=None, d_proj=None, f_s=2.0):
        self.L = float(L)
        self.omega = self.L ** 3
        self.ecut = float(ecut)
        self.N = int(grid)
        self.mw = sphere(L, ecut)            # wavefunction sphere
        self.mr = sphere(L, 4.0 * ecut)      # density sphere
        self.b = 2.0 * math.pi / self.L
        self.g2w = self.b ** 2 * np.sum(self.mw ** 2, axis=1).astype(np.float64)
        self.g2r = self.b ** 2 * np.sum(self.mr ** 2, axis=1).astype(np.float64)
        self.vloc_G = np.asarray(vloc_G, np.complex128)
        self.psi_v = np.asarray(psi_v, np.complex128)
        self.e_v = np.asarray(e_v, np.float64)
        n_pw = self.mw.shape[0]
        self.beta = (np.zeros((n_pw, 0), np.complex128) if beta_G is None
                     else np.asarray(beta_G, np.complex128))
        self.D = np.zeros(0) if d_proj is None else np.asarray(d_proj, np.float64)
        self.f_s = float(f_s)
        assert self.vloc_G.shape == (self.mr.shape[0],)
        assert self.psi_v.shape[0] == n_pw
        # Coulomb square root on the density sphere, zero at G = 0.
        g = np.sqrt(self.g2r)
        self.vsqrt = np.where(g > 0, math.sqrt(4.0 * math.pi) / np.where(g > 0, g, 1.0), 0.0)
        self._vloc_r = None
        self._dense = None

    # -- grid maps -----------------------------------------------------------------
    def to_grid(self, c: np.ndarray, miller: np.ndarray) -> np.ndarray:
        """Place sphere coefficients on the N^3 reciprocal grid (zero elsewhere)."""
        out = np.zeros((self.N,) * 3, np.complex128)
        idx = np.mod(miller, self.N)
        out[idx[:, 0], idx[:, 1], idx[:, 2]] = c
        return out

    def from_grid(self, g: np.ndarray, miller: np.ndarray) -> np.ndarray:
        idx = np.mod(miller, self.N)
        return g[idx[:, 0], idx[:, 1], idx[:, 2]]

    def to_r(self, c: np.ndarray, miller: np.ndarray) -> np.ndarray:
        """f(r_j) = sum_G c_G e^{iG.r_j} on the real-space grid."""
        return np.fft.ifftn(self.to_grid(c, miller)) * self.N ** 3

    def to_G(self, f_r: np.ndarray, miller: np.ndarray) -> np.ndarray:
        """c_G = (1/N_g) sum_j f(r_j) e^{-iG.r_j}, restricted to the given sphere."""
        return self.from_grid(np.fft.fftn(f_r) / self.N ** 3, miller)

    @property
    def vloc_r(self) -> np.ndarray:
        if self._vloc_r is None:
            self._vloc_r = self.to_r(self.vloc_G, self.mr)
        return self._vloc_r

    # -- Hamiltonian -----------------------------------------------------------------
    def h_dense(self) -> np.ndarray:
        """H_GG' = 0.5|G|^2 delta_GG' + V(G - G') + sum_p beta_p(G) D_p beta_p(G')^*."""
        if self._dense is None:
            n = self.mw.shape[0]
            # V(G - G'): look the difference vectors up in the density sphere through a dense
            # table indexed by Miller triples (every difference lies inside the density sphere).
            M = int(np.max(np.abs(self.mr)))
            box = np.full((2 * M + 1,) * 3, -1, np.int64)
            box[self.mr[:, 0] + M, self.mr[:, 1] + M, self.mr[:, 2] + M] = np.arange(self.mr.shape[0])
            H = np.zeros((n, n), np.complex128)
            for i in range(n):
                d = self.mw[i][None, :] - self.mw
                idx = box[d[:, 0] + M, d[:, 1] + M, d[:, 2] + M]
                assert np.all(idx >= 0)
                H[i, :] = self.vloc_G[idx]
            H[np.diag_indices(n)] += 0.5 * self.g2w
            if self.beta.shape[1]:
                H += self.beta @ np.diag(self.D) @ self.beta.conj().T
            self._dense = H
        return self._dense

    def apply_h(self, psi: np.ndarray) -> np.ndarray:
        """Dual-space H psi (Sec. 4.1): kinetic in G, V_loc in r, KB by projections."""
        psi = np.asarray(psi, np.complex128)
        one = psi.ndim == 1
        P = psi[:, None] if one else psi
        out = np.empty_like(P)
        for j in range(P.shape[1]):
            vpsi = self.to_G(self.vloc_r * self.to_r(P[:, j], self.mw), self.mw)
            out[:, j] = 0.5 * self.g2w * P[:, j] + vpsi
        if self.beta.shape[1]:
            out += self.beta @ (self.D[:, None] * (self.beta.conj().T @ P))
        return out[:, 0] if one else out

    def eigh(self):
        """All eigenpairs of the dense H (ascending)."""
        return np.linalg.eigh(self.h_dense())

    def multiply_r(self, dV_G: np.ndarray, psi: np.ndarray) -> np.ndarray:
        """[dV psi] on the wavefunction sphere: product on the grid, truncated to the sphere."""
        return self.to_G(self.to_r(dV_G, self.mr) * self.to_r(psi, self.mw), self.mw)
