"""Independent-particle density response chi0 (oracle, FP64).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Paper passages followed:
  * Sec. 2.1: chi0bar = v^1/2 chi0 v^1/2 (symmetrised response).
  * Sec. 2.2: Adler-Wiser sum over occupied and empty states (the "definition"
    the Sternheimer route reaches without empty states).
  * Sec. 3, Eq. sternheimer: (h - eps_i) P_c dpsi = -P_c v_pert psi_i with
    P_c = 1 - P_v, solved by preconditioned CG; Eq. dfpt: dn = sum_sigma sum_i
    [psi_i^* dpsi_i + dpsi_i^* psi_i].
  * Sec. 3 (Lanczos part): the response is needed at imaginary frequencies i w,
    which shifts the Sternheimer operator by +i w.

Readings of the paper used here (all listed in the design notes):
  * Spin-unpolarised, f_s = 2 (the sum over sigma of Eq. dfpt).
  * Frequency: the +i w shifted solve x_i solves P_c (H - e_i + i w) P_c x_i =
    -P_c dV psi_i on range(P_c); for a perturbation that is real in r the
    response is drho = f_s sum_i 2 Re(psi_i^* x_i) (the -i w partner is the
    complex conjugate).  A general complex dV is applied by linearity, as
    dV = A + i B with A, B real in r.
  * Truncations: dV psi_i is formed on the grid and truncated to the
    wavefunction sphere; drho is formed on the grid and truncated to the
    density sphere.
  * Units: psi(r) = Omega^-1/2 sum_G psi(G) e^{iGr}, so drho(G) carries 1/Omega;
    drho(G) = sum_G' chi0_GG' dV(G') with chi0_GG' = (1/Omega) FT_r FT_r' chi0(r, r').
  * Preconditioner: diagonal 1 / max(0.5|G|^2 - e_i, 1 Ha) (the paper says only
    "preconditioned"); it changes iteration counts, not the converged result.

Pins (tests/test_oracle_pins.py): sum over states == Sternheimer dense solves
== finite differences of the ground-state density (static), == the
free-electron closed form when V_loc = 0; Hermiticity and negative
semidefiniteness of chi0bar; charge conservation drho(G=0) = 0; linearity;
monotone decay with w; the frequency integral identity
int_0^inf chi0(iw) dw = -pi f_s P_v-weighted pair projector (a closed form that
needs no empty states).
"""
from __future__ import annotations

import math

import numpy as np
import scipy.linalg

from .model import Model


def hermitian_split(model: Model, dV: np.ndarray):
    """dV(G) = A(G) + i B(G) with A, B real in r: A(G) = (dV(G) + dV(-G)^*)/2, B = (dV(G) - dV(-G)^*)/(2i)."""
    where = {tuple(m): i for i, m in enumerate(model.mr.tolist())}
    neg = np.array([where[(-h, -k, -l)] for h, k, l in model.mr.tolist()])
    A = 0.5 * (dV + dV[neg].conj())
    B = (dV - dV[neg].conj()) / 2j
    return A, B


def _states(model: Model):
    """All eigenpairs of H; checks the occupied ones span the given psi_v."""
    w, U = model.eigh()
    nv = model.psi_v.shape[1]
    overlap = U[:, :nv].conj().T @ model.psi_v
    sv = np.linalg.svd(overlap, compute_uv=False)
    if np.min(sv) < 1.0 - 1e-8:
        raise ValueError("given psi_v do not span the lowest eigenvectors of H")
    return w, U


def sos_drho(model: Model, dV: np.ndarray, omegas=(0.0,)) -> np.ndarray:
    """Adler-Wiser sum over states.

    drho(r) = (f_s/Omega) sum_v sum_c [ psi_v^*(r) psi_c(r) <c|dV|v> / (e_v - e_c - i w)
                                        + psi_c^*(r) psi_v(r) <v|dV|c> / (e_v - e_c + i w) ]
    with tilde-orbitals psi(r) = sum_G psi(G) e^{iGr}.  dV: (N_rho,) or (N_rho, n_pert).
    Returns drho(G) on the density sphere, shape (N_rho, n_pert, n_omega).
    """
    dV = np.asarray(dV, np.complex128)
    dV = dV[:, None] if dV.ndim == 1 else dV
    w, U = _states(model)
    nv = model.psi_v.shape[1]
    occ, emp = U[:, :nv], U[:, nv:]
    ev, ec = w[:nv], w[nv:]
    out = np.zeros((model.mr.shape[0], dV.shape[1], len(omegas)), np.complex128)
    psi_r = [model.to_r(occ[:, v], model.mw) for v in range(nv)]
    for p in range(dV.shape[1]):
        dV_r = model.to_r(dV[:, p], model.mr)
        for v in range(nv):
            w1 = model.to_G(dV_r * psi_r[v], model.mw)             # dV psi_v on the sphere
            w2 = model.to_G(dV_r.conj() * psi_r[v], model.mw)      # dV^* psi_v
            M_cv = emp.conj().T @ w1                                # <c|dV|v>
            M_vc = (emp.conj().T @ w2).conj()                       # <v|dV|c>
            for k, om in enumerate(omegas):
                d = ev[v] - ec
                y1 = emp @ (M_cv / (d - 1j * om))
                y2 = emp @ (M_vc.conj() / (d - 1j * om))
                rho_r = psi_r[v].conj() * model.to_r(y1, model.mw) + psi_r[v] * model.to_r(y2, model.mw).conj()
                out[:, p, k] += model.to_G(rho_r, model.mr)
    return out * (model.f_s / model.omega)


def sos_drho_channels(models, dV: np.ndarray, omegas=(0.0,)) -> np.ndarray:
    """Spin-polarised response: the sum over spin channels sigma of Eq. dfpt, each channel a
    Model of its own (V_sigma, psi_sigma, e_sigma; f_s = 1 for a spin-polarised system)."""
    return sum(sos_drho(m, dV, omegas) for m in models)


def sos_static_block(model: Model, dV: np.ndarray, states=None) -> np.ndarray:
    """Static (w = 0) sum over states for a block of perturbations that are real in r.

    For such dV the two terms of the Adler-Wiser form are complex conjugates, so
    drho(r) = (f_s/Omega) sum_v 2 Re[ psi_v^*(r) y_v(r) ],  y_v = sum_c psi_c <c|dV|v> / (e_v - e_c).
    The same arithmetic as sos_drho, evaluated for all perturbations at once.
    `states` = (eigenvalues, eigenvectors) of H may be passed to reuse a diagonalisation.
    Returns drho(G) on the density sphere, shape (N_rho, n_pert).
    """
    dV = np.asarray(dV, np.complex128)
    w, U = _states(model) if states is None else states
    nv = model.psi_v.shape[1]
    occ, emp = U[:, :nv], U[:, nv:]
    N = model.N
    dV_r = np.stack([model.to_r(dV[:, p], model.mr) for p in range(dV.shape[1])], axis=-1)
    rho_r = np.zeros(dV_r.shape, np.float64)
    iw = np.mod(model.mw, N)
    for v in range(nv):
        pv = model.to_r(occ[:, v], model.mw)
        prod = np.fft.fftn(pv[..., None] * dV_r, axes=(0, 1, 2)) / N ** 3
        W = prod[iw[:, 0], iw[:, 1], iw[:, 2], :]                  # [dV psi_v] on the sphere
        Y = emp @ ((emp.conj().T @ W) / (w[v] - w[nv:])[:, None])
        grid = np.zeros((N, N, N, Y.shape[1]), np.complex128)
        grid[iw[:, 0], iw[:, 1], iw[:, 2], :] = Y
        y_r = np.fft.ifftn(grid, axes=(0, 1, 2)) * N ** 3
        rho_r += 2.0 * (pv.conj()[..., None] * y_r).real
    out = np.fft.fftn(rho_r, axes=(0, 1, 2)) / N ** 3
    ir = np.mod(model.mr, N)
    return out[ir[:, 0], ir[:, 1], ir[:, 2], :] * (model.f_s / model.omega)


def _pc(model: Model, x: np.ndarray) -> np.ndarray:
    """P_c x = x - sum_v psi_v <psi_v|x> (Sec. 3: P_c = 1 - P_v)."""
    P = model.psi_v
    return x - P @ (P.conj().T @ x)


def sternheimer_drho(model: Model, dV: np.ndarray, omegas=(0.0,)) -> np.ndarray:
    """Eq. sternheimer by dense linear solves on range(P_c), then Eq. dfpt.

    For each real-in-r part dV_s of dV and each occupied v:
      (P_c (H - e_v + i w) P_c + P_v) x = -P_c [dV_s psi_v]      (x lands in range(P_c))
      drho_s += (f_s/Omega) 2 Re(psi_v^*(r) x(r)).
    """
    dV = np.asarray(dV, np.complex128)
    dV = dV[:, None] if dV.ndim == 1 else dV
    H = model.h_dense()
    n = H.shape[0]
    Pv = model.psi_v @ model.psi_v.conj().T
    Pc = np.eye(n) - Pv
    nv = model.psi_v.shape[1]
    psi_r = [model.to_r(model.psi_v[:, v], model.mw) for v in range(nv)]
    out = np.zeros((model.mr.shape[0], dV.shape[1], len(omegas)), np.complex128)
    for k, om in enumerate(omegas):
        lu = [scipy.linalg.lu_factor(Pc @ (H - (model.e_v[v] - 1j * om) * np.eye(n)) @ Pc + Pv)
              for v in range(nv)]
        for p in range(dV.shape[1]):
            A, B = hermitian_split(model, dV[:, p])
            for part, scale in ((A, 1.0), (B, 1j)):
                if not np.any(part):
                    continue
                dV_r = model.to_r(part, model.mr)
                rho_r = np.zeros_like(dV_r)
                for v in range(nv):
                    b = -_pc(model, model.to_G(dV_r * psi_r[v], model.mw))
                    x = scipy.linalg.lu_solve(lu[v], b)
                    rho_r += 2.0 * (psi_r[v].conj() * model.to_r(x, model.mw)).real
                out[:, p, k] += scale * model.to_G(rho_r, model.mr)
    return out * (model.f_s / model.omega)


def sternheimer_cg_drho(model: Model, dV: np.ndarray, tol: float = 1e-12, max_iter: int = 2000,
                        systems=None, return_iters: bool = False):
    """Static (w = 0) Eq. sternheimer by preconditioned CG with FFT-applied H, then Eq. dfpt.

    The CG runs on range(P_c) with A = P_c (H - e_v) P_c and the diagonal
    preconditioner M^-1_G = 1 / max(0.5|G|^2 - e_v, 1); stop when
    ||b - A x|| <= tol ||b||.  dV must be real in r.  `systems` optionally
    restricts the sum to a list of (v, p) pairs (a bounded sample for timing);
    the result then holds only those systems' contributions.
    """
    dV = np.asarray(dV, np.complex128)
    dV = dV[:, None] if dV.ndim == 1 else dV
    nv = model.psi_v.shape[1]
    if systems is None:
        systems = [(v, p) for p in range(dV.shape[1]) for v in range(nv)]
    psi_r = {}
    dV_r = {}
    out = np.zeros((model.mr.shape[0], dV.shape[1]), np.complex128)
    iters = []
    for v, p in systems:
        if v not in psi_r:
            psi_r[v] = model.to_r(model.psi_v[:, v], model.mw)
        if p not in dV_r:
            dV_r[p] = model.to_r(dV[:, p], model.mr)
        x, it = sternheimer_cg_solve(model, dV_r[p], v, tol, max_iter, psi_r[v])
        iters.append(it)
        rho_r = 2.0 * (psi_r[v].conj() * model.to_r(x, model.mw)).real
        out[:, p] += model.to_G(rho_r, model.mr)
    out *= model.f_s / model.omega
    return (out, iters) if return_iters else out


def sternheimer_cg_solve(model: Model, dV_r: np.ndarray, v: int, tol: float = 1e-12, max_iter: int = 2000,
                         psi_r=None):
    """One static system of Eq. sternheimer by preconditioned CG: P_c (H - e_v) P_c x = -P_c [dV psi_v]
    on range(P_c), dV given in real space (dV_r, real in r), the diagonal preconditioner
    1 / max(0.5|G|^2 - e_v, 1), stop when ||b - A x|| <= tol ||b||.  Returns (x, iterations), x on
    the wavefunction sphere."""
    pv = model.to_r(model.psi_v[:, v], model.mw) if psi_r is None else psi_r
    ev = model.e_v[v]
    minv = 1.0 / np.maximum(0.5 * model.g2w - ev, 1.0)

    def A(x):
        return _pc(model, model.apply_h(x) - ev * x)

    b = -_pc(model, model.to_G(dV_r * pv, model.mw))
    bnorm = np.linalg.norm(b)
    x = np.zeros_like(b)
    r = b.copy()
    z = _pc(model, minv * r)
    d = z.copy()
    rz = np.vdot(r, z).real
    it = 0
    while np.linalg.norm(r) > tol * bnorm and it < max_iter:
        q = A(d)
        alpha = rz / np.vdot(d, q).real
        x += alpha * d
        r -= alpha * q
        z = _pc(model, minv * r)
        rz_new = np.vdot(r, z).real
        d = z + (rz_new / rz) * d
        rz = rz_new
        it += 1
    return x, it


def pair_densities(model: Model, occ: np.ndarray, emp: np.ndarray) -> np.ndarray:
    """b_vc(G) = (1/N_g) sum_r psi_v^*(r) psi_c(r) e^{-iGr} on the density sphere, columns (v, c)."""
    cols = []
    emp_r = [model.to_r(emp[:, c], model.mw) for c in range(emp.shape[1])]
    for v in range(occ.shape[1]):
        pv = model.to_r(occ[:, v], model.mw).conj()
        for c in range(emp.shape[1]):
            cols.append(model.to_G(pv * emp_r[c], model.mr))
    return np.stack(cols, axis=1)


def chi0_matrix(model: Model, omega: float = 0.0) -> np.ndarray:
    """Dense chi0_GG'(i w) on the density sphere from the sum over states.

    chi0 = (f_s/Omega) [ B diag(1/(d - i w)) B^H + conj(B-) diag(1/(d + i w)) B-^T ],
    B_(G,vc) = b_vc(G), B-_(G,vc) = b_vc(-G), d_vc = e_v - e_c.
    """
    w, U = _states(model)
    nv = model.psi_v.shape[1]
    B = pair_densities(model, U[:, :nv], U[:, nv:])
    d = (w[:nv, None] - w[None, nv:]).ravel()
    where = {tuple(m): i for i, m in enumerate(model.mr.tolist())}
    neg = np.array([where[(-h, -k, -l)] for h, k, l in model.mr.tolist()])
    Bm = B[neg]
    chi = (B / (d - 1j * omega)) @ B.conj().T + (Bm.conj() / (d + 1j * omega)) @ Bm.T
    return chi * (model.f_s / model.omega)


def chibar0_matrix(model: Model, omega: float = 0.0) -> np.ndarray:
    """chi0bar_GG' = v^1/2(G) chi0_GG' v^1/2(G') (Sec. 2.1)."""
    return model.vsqrt[:, None] * chi0_matrix(model, omega) * model.vsqrt[None, :]


def apply_chibar0(model: Model, phi: np.ndarray, omegas=(0.0,)) -> np.ndarray:
    """chi0bar phi = v^1/2 drho[dV = v^1/2 phi] by the sum over states."""
    phi = np.asarray(phi, np.complex128)
    phi = phi[:, None] if phi.ndim == 1 else phi
    drho = sos_drho(model, model.vsqrt[:, None] * phi, omegas)
    return model.vsqrt[:, None, None] * drho


def free_electron_chi0_diag(L: float, ecut: float, n_occ: int, omegas=(0.0,), f_s: float = 2.0):
    """Closed form of chi0_GG(i w) for V = 0 with closed shells (chi0 is diagonal in G).

    The occupied plane waves k are the n_occ lowest of the wavefunction sphere
    (n_occ must close a shell: 1, 7, 19, 27, 33, ...).  For each G of the density sphere
      chi0_GG = (f_s/Omega) sum_{k occ, k+G empty, 0.5|k+G|^2 <= ecut} 2 D / (D^2 + w^2),
      D = 0.5|k|^2 - 0.5|k+G|^2.
    Returns (miller_rho, chi0 of shape (N_rho, n_omega)).
    """
    from .model import sphere
    b = 2.0 * math.pi / L
    mw = sphere(L, ecut)
    mr = sphere(L, 4.0 * ecut)
    n2 = np.sum(mw ** 2, axis=1)
    if n_occ < len(n2) and n2[n_occ] == n2[n_occ - 1]:
        raise ValueError("n_occ must close a shell")
    occ = [tuple(k) for k in mw[:n_occ].tolist()]
    occ_set = set(occ)
    sphere_set = {tuple(k) for k in mw.tolist()}
    out = np.zeros((mr.shape[0], len(omegas)))
    for i, G in enumerate(mr.tolist()):
        for k in occ:
            q = (k[0] + G[0], k[1] + G[1], k[2] + G[2])
            if q in occ_set or q not in sphere_set:
                continue
            D = 0.5 * b * b * (k[0] ** 2 + k[1] ** 2 + k[2] ** 2 - q[0] ** 2 - q[1] ** 2 - q[2] ** 2)
            for j, om in enumerate(omegas):
                out[i, j] += 2.0 * D / (D * D + om * om)
    return mr, out * (f_s / L ** 3)


def density(model: Model, states: np.ndarray) -> np.ndarray:
    """n(G) = (f_s/Omega) FT[sum_v |psi_v(r)|^2] on the density sphere."""
    rho_r = np.zeros((model.N,) * 3)
    for v in range(states.shape[1]):
        rho_r += np.abs(model.to_r(states[:, v], model.mw)) ** 2
    return model.to_G(rho_r, model.mr) * (model.f_s / model.omega)


def finite_difference_drho(model: Model, dV: np.ndarray, lam: float = 1e-3) -> np.ndarray:
    """Static response as the derivative of the ground-state density.

    n(lam) = density of the lowest N_v eigenvectors of H + lam dV (dV real in r,
    its matrix dV(G - G') on the wavefunction sphere); drho = dn/dlam at 0 by the
    fourth-order central stencil [-n(2l) + 8 n(l) - 8 n(-l) + n(-2l)] / (12 l).
    """
    H = model.h_dense()
    where = {tuple(m): i for i, m in enumerate(model.mr.tolist())}
    n = model.mw.shape[0]
    dmat = np.zeros((n, n), np.complex128)
    for i in range(n):
        for j in range(n):
            d = tuple(model.mw[i] - model.mw[j])
            dmat[i, j] = dV[where[d]]
    nv = model.psi_v.shape[1]

    def n_of(l):
        w, U = np.linalg.eigh(H + l * dmat)
        return density(model, U[:, :nv])

    return (-n_of(2 * lam) + 8 * n_of(lam) - 8 * n_of(-lam) + n_of(-2 * lam)) / (12 * lam)


def frequency_integral_closed_form(model: Model, a: np.ndarray, c: np.ndarray) -> complex:
    """Closed form of <a| int_0^inf chi0(i w) dw |c> for real-in-r a, c (potentials on the density sphere).

    Since int_0^inf 2 D / (D^2 + w^2) dw = -pi for D < 0, the sum over empty
    states collapses through completeness (sum_c |c><c| = 1 - P_v on the
    wavefunction sphere):
      int chi0 = -pi (f_s/Omega) sum_v [ <a psi_v| Q |c psi_v> - sum_v' <a psi_v|psi_v'><psi_v'|c psi_v> ]
    where Q truncates to the wavefunction sphere and all products are taken on the grid.
    Needs no empty state.  Returns the value of Omega * sum_G a(G)^* [int chi0 c](G)
    divided by Omega (i.e. in the same units as sum_G a^* drho).
    """
    nv = model.psi_v.shape[1]
    total = 0.0 + 0.0j
    a_r = model.to_r(a, model.mr)
    c_r = model.to_r(c, model.mr)
    for v in range(nv):
        pv = model.to_r(model.psi_v[:, v], model.mw)
        ua = model.to_G(a_r * pv, model.mw)     # a psi_v truncated to the sphere
        uc = model.to_G(c_r * pv, model.mw)
        ov_a = model.psi_v.conj().T @ ua
        ov_c = model.psi_v.conj().T @ uc
        total += np.vdot(ua, uc) - np.vdot(ov_a, ov_c)
    # <a|X|c> in the sum_G a^* (Xc)(G) form picks up 1/Omega from drho(G).
    return -math.pi * model.f_s / model.omega * total
