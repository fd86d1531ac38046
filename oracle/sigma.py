"""Exchange self-energy of the occupied states (oracle, FP64).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Paper passages followed (Sec. 2, Eq. sigmacIR): the diagonal self-energy is
<psi_i|Sigma(w)|psi_i> = <psi_i|Sigma_X|psi_i> + I_i(w) + R_i(w), where the
exchange part Sigma_X is Eq. self_energy_gw with the screened W_0 replaced by
the bare Coulomb potential v:
  <psi_i|Sigma_X|psi_i> = - sum_{j occ} int int psi_i^*(r) psi_j(r) v(r - r')
                                              psi_j^*(r') psi_i(r') dr dr'.

Readings (the paper leaves these open):
  * One spin channel: the sum runs over the occupied states of the channel of
    psi_i (exchange couples equal spins only), so a spin-unpolarised system
    carries no factor 2 here.
  * Periodic cell at Gamma: v(G) = 4 pi / |G|^2 with the G = 0 term left out
    (the divergent head belongs to the long-range part Xi of Eq. Wp, out of
    scope), so with n_ij(G) = (1/Omega) int psi_i^* psi_j e^{-iG.r} dr
      <psi_i|Sigma_X|psi_i> = - Omega sum_j sum_{G != 0} v(G) |n_ij(G)|^2.
  * psi(r) = Omega^{-1/2} sum_G c(G) e^{iG.r} (the Model's convention); the
    pair densities are formed on the grid and taken to the density sphere,
    which holds every product of two wavefunction-sphere functions.

Pins (tests/test_oracle_pins.py): the pair densities equal the direct
G-space convolution sum_G1 c_i(G1)^* c_j(G1 + G); for plane-wave states the
result is the closed form -(1/Omega) sum_{j != i} 4 pi / |k_j - k_i|^2; the
total sum_i <psi_i|Sigma_X|psi_i> is invariant under a unitary rotation of the
occupied states.
"""
from __future__ import annotations

import numpy as np

from .model import Model


def pair_density(model: Model, ci: np.ndarray, cj: np.ndarray) -> np.ndarray:
    """n_ij(G) * Omega = FT[u_i^* u_j] on the density sphere, u = sum_G c(G) e^{iG.r}."""
    ui = model.to_r(np.asarray(ci, np.complex128), model.mw)
    uj = model.to_r(np.asarray(cj, np.complex128), model.mw)
    return model.to_G(np.conj(ui) * uj, model.mr)


def sigma_x(model: Model, states=None) -> np.ndarray:
    """<psi_i|Sigma_X|psi_i> for the occupied states i in `states` (default: all), in Ha."""
    nv = model.psi_v.shape[1]
    states = range(nv) if states is None else states
    v = model.vsqrt ** 2                       # 4 pi / |G|^2, zero at G = 0
    out = []
    for i in states:
        acc = 0.0
        for j in range(nv):
            n_ij = pair_density(model, model.psi_v[:, i], model.psi_v[:, j])
            acc += np.sum(v * np.abs(n_ij) ** 2)
        out.append(-acc / model.omega)
    return np.asarray(out)
