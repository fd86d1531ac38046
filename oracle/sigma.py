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

The short-range correlation integral of Eq. ISR,
  I^SR_i(w) = (1/Omega) sum_nm int dw'/(2 pi) Lambda_nm(i w') <psi_i phi~_n|(h - w - i w')^-1|psi_i phi~_m>,
is evaluated with the G0 Lanczos resolvent of oracle/g0.py (Eq. lanczos).
Readings: Lambda_nm(i w') is even in w' (it is built from chi0bar(i w'), which is), so the
integral over the whole imaginary axis is folded onto [0, inf):
  I^SR_i(w) = (1/Omega) int_0^inf dw'/(2 pi) sum_nm Lambda_nm(i w') [g0_nm(w + i w') + g0_nm(w - i w')],
and is taken by the quadrature (nodes, weights) the caller passes (e.g. Gauss-Legendre
on [0, w_max]); Lambda is supplied at the nodes (e.g. the Dyson step in the PDEP basis).

Pins (tests/test_oracle_pins.py): the pair densities equal the direct
G-space convolution sum_G1 c_i(G1)^* c_j(G1 + G); for plane-wave states the
result is the closed form -(1/Omega) sum_{j != i} 4 pi / |k_j - k_i|^2; the
total sum_i <psi_i|Sigma_X|psi_i> is invariant under a unitary rotation of the
occupied states.  For I^SR: with Lambda = c * identity at every node and exhausted chains, the
quadrature of the folded integrand over [0, W] converges to the closed form
(c/Omega) sum_n <b_n| (1/pi) arctan(W / (h - w)) |b_n> evaluated through the eigenpairs of h.
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


def isr(model: Model, phi: np.ndarray, states, n_steps: int, omegas, lam: np.ndarray, nodes, weights):
    """I^SR_i(w) for the listed states and real frequencies w: shape (n_states, n_omega), complex.

    lam: Lambda_nm(i w'_k) at the quadrature nodes, shape (n_nodes, n_pdep, n_pdep).
    nodes, weights: quadrature of [0, inf) (w'_k >= 0).
    """
    from . import g0
    omegas = np.asarray(omegas, np.float64).ravel()
    nodes = np.asarray(nodes, np.float64).ravel()
    weights = np.asarray(weights, np.float64).ravel()
    lam = np.asarray(lam, np.float64)
    z = np.array([[w + 1j * wp, w - 1j * wp] for w in omegas for wp in nodes]).ravel()
    G = g0.g0_lanczos(model, phi, states, n_steps, z)["g0"]          # (ns, nz, npd, npd)
    nw, nk = omegas.size, nodes.size
    G = G.reshape(len(states), nw, nk, 2, *G.shape[2:])
    out = np.zeros((len(states), nw), np.complex128)
    for k in range(nk):
        s = np.einsum("nm,iwnm->iw", lam[k], G[:, :, k, 0] + G[:, :, k, 1])
        out += weights[k] / (2.0 * np.pi) * s
    return out / model.omega
