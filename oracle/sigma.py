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
(c/Omega) sum_n <b_n| (1/pi) arctan(W / (h - w)) |b_n> evaluated through the eigenpairs of h;
with exhausted chains it equals isr_dense (the exact resolvent of the dense h).

The residue term of Eq. Rfac in the same basis,
  R_i(w) = (1/Omega) sum_j f_ij(w) sum_nm Lambda_nm(e_j - w) <b_n|j><j|b_m>,
  f_ij(w) = theta(e_j - e_F) theta(w - e_j) - theta(e_F - e_j) theta(e_j - w),
runs over the eigenstates j of h with Lambda (the Dyson step on chi0bar projected on the basis)
at the real frequency e_j - w (reading: the KS energies stand in for the QP energies in f).
Pin: I^SR jumps by -(1/Omega) sum_nm Lambda_nm(0) <b_n|j><j|b_m> where w crosses e_j, and R jumps
back, so I^SR + R is continuous there (an occupied and an empty j are tested); a sign error in R
breaks it.  Reading of the overall sign: Eq. Ifac carries a leading minus in front of G0 W_p, and
with G0(z) = (z - h)^-1 that minus makes -G0(z) = (h - z)^-1, the operator Eq. ISR writes without a
minus; the two equations agree and I^SR is evaluated with (h - z)^-1.  Pin of that sign: with a
frequency-independent W_p (Lambda = c * identity at every frequency) I + R is the static COHSEX
closed form (c/Omega) sum_j sum_n |<j|b_n>|^2 (1/2 - theta(e_F - e_j)), a Coulomb hole of +1/2 over
every state and a screened exchange of -1 over the occupied ones, the same sign as the exchange
sum -sum_{j occ} of Sigma_X; a sign error in I or in R breaks it.

The QP equation (Eq. e_qp) is solved by secant root finding (qp_energy); reading: the model
Hamiltonian has no exchange-correlation potential, so <v_xc> = 0 unless given.  Pin: a one-pole
self-energy whose QP equation is a quadratic with a closed-form root.
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


# ---------------------------------------------------------------- residues and dense references
def chi0_z(model: Model, z: complex) -> np.ndarray:
    """Dense chi0_GG'(z) on the density sphere at a complex frequency z (the sum over states of
    oracle/chi0.py with i w replaced by z): (f_s/Omega)[B diag(1/(d - z)) B^H + conj(B-) diag(1/(d + z)) B-^T],
    d_vc = e_v - e_c."""
    from .chi0 import _states, pair_densities
    w, U = _states(model)
    nv = model.psi_v.shape[1]
    B = pair_densities(model, U[:, :nv], U[:, nv:])
    d = (w[:nv, None] - w[None, nv:]).ravel()
    where = {tuple(m): i for i, m in enumerate(model.mr.tolist())}
    neg = np.array([where[(-h, -k, -l)] for h, k, l in model.mr.tolist()])
    Bm = B[neg]
    chi = (B / (d - z)) @ B.conj().T + (Bm.conj() / (d + z)) @ Bm.T
    return chi * (model.f_s / model.omega)


def lam_basis(model: Model, phi: np.ndarray, z: complex) -> np.ndarray:
    """Lambda(z) = (1 - chi0bar(z))^-1 chi0bar(z) with chi0bar projected on the basis phi
    (orthonormal columns on the density sphere): the Dyson step of Sec. 2 in that basis."""
    phi = np.asarray(phi, np.complex128)
    pt = model.vsqrt[:, None] * phi
    X = pt.conj().T @ chi0_z(model, z) @ pt
    return np.linalg.solve(np.eye(X.shape[0]) - X, X)


def _spectral_overlaps(model: Model, phi: np.ndarray, i: int):
    """Eigenpairs (e, U) of h and the overlaps Y[j, n] = <j | psi_i phi~_n> (b_n of oracle/g0.py)."""
    from . import g0
    e, U = np.linalg.eigh(model.h_dense())
    return e, U.conj().T @ g0.start_vectors(model, phi, i)


def isr_dense(model: Model, phi: np.ndarray, i: int, omegas, lam: np.ndarray, nodes, weights) -> np.ndarray:
    """I^SR_i(w) as sigma.isr, with the exact resolvent sum_j <b_n|j><j|b_m>/(e_j - z) of the
    dense h in place of the Lanczos chains."""
    e, Y = _spectral_overlaps(model, phi, i)
    out = []
    for w in np.asarray(omegas, np.float64).ravel():
        acc = 0.0 + 0.0j
        for k, (wp, wt) in enumerate(zip(np.asarray(nodes).ravel(), np.asarray(weights).ravel())):
            g = (Y.conj() / (e - w - 1j * wp)[:, None]).T @ Y + (Y.conj() / (e - w + 1j * wp)[:, None]).T @ Y
            acc += wt / (2.0 * np.pi) * np.sum(lam[k] * g)
        out.append(acc / model.omega)
    return np.asarray(out)


def residue_term(model: Model, phi: np.ndarray, i: int, omegas, e_fermi: float, eta: float = 0.0,
                 lam_fn=None) -> np.ndarray:
    """R_i(w) of Eq. Rfac in the basis: (1/Omega) sum_j f_ij(w) sum_nm Lambda_nm(e_j - w) <b_n|j><j|b_m>,
    f_ij(w) = theta(e_j - e_F) theta(w - e_j) - theta(e_F - e_j) theta(e_j - w), over every
    eigenstate j of h (Lambda at the real frequency e_j - w, plus i eta).  lam_fn(z) gives
    Lambda(z) in the basis; by default the Dyson step on the basis (lam_basis)."""
    if lam_fn is None:
        def lam_fn(z):
            return lam_basis(model, phi, z)
    e, Y = _spectral_overlaps(model, phi, i)
    out = []
    for w in np.asarray(omegas, np.float64).ravel():
        acc = 0.0 + 0.0j
        for j in range(e.size):
            f = (1.0 if (e[j] > e_fermi and w > e[j]) else 0.0) - (1.0 if (e[j] <= e_fermi and e[j] > w) else 0.0)
            if f != 0.0:
                A = np.outer(Y[j].conj(), Y[j])                 # <b_n|j><j|b_m>
                acc += f * np.sum(lam_fn(e[j] - w + 1j * eta) * A)
        out.append(acc / model.omega)
    return np.asarray(out)


# ---------------------------------------------------------------- quasiparticle equation (Eq. e_qp)
def secant(f, x0: float, x1: float, tol: float = 1e-10, max_iter: int = 100) -> float:
    """Root of f by the secant method from x0, x1 (Sec. 3: the QP equation is solved with a
    root-finding algorithm such as the secant method)."""
    f0, f1 = f(x0), f(x1)
    for _ in range(max_iter):
        if f1 == f0:
            break
        x2 = x1 - f1 * (x1 - x0) / (f1 - f0)
        x0, f0 = x1, f1
        x1, f1 = x2, f(x2)
        if abs(x1 - x0) <= tol * max(1.0, abs(x1)):
            return x1
    raise RuntimeError("secant did not converge")


def qp_energy(e_i: float, sigma_of_e, v_xc: float = 0.0, tol: float = 1e-10) -> float:
    """e^QP = e_i + Re <psi_i|Sigma(e^QP)|psi_i> - <psi_i|v_xc|psi_i> (Eq. e_qp), by secant from e_i.
    sigma_of_e(E) returns <psi_i|Sigma(E)|psi_i>."""
    return secant(lambda E: e_i + np.real(sigma_of_e(E)) - v_xc - E, e_i, e_i + 0.01, tol)
