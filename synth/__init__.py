"""Seeded synthetic inputs for the chi0 / Sternheimer path (Gamma point, cubic cell).

This module stands in for the ground-state DFT run that precedes a response
calculation (the paper takes psi_i, eps_i from Quantum ESPRESSO, Sec. 3 and
Fig. "workflow").  It draws random numbers (well positions, perturbation
coefficients) from seeded PCG64 generators, lays out the model potential and
projectors on the plane-wave spheres, and diagonalises the model Kohn-Sham
Hamiltonian densely on the host to give the occupied states.  It contains none
of the response method's arithmetic (no Sternheimer solve, no P_c, no density
response) and is shared by the tests, the benchmark and the library's users as
the source of inputs only.

Conventions (Hartree atomic units):
  * cubic cell of side L, volume Omega = L^3, reciprocal unit b = 2 pi / L;
  * G = b (h, k, l); wavefunction sphere 0.5 |G|^2 <= ecut, density sphere
    0.5 |G|^2 <= 4 ecut;
  * canonical order of a sphere: ascending h^2+k^2+l^2, ties broken by the
    Miller triple (h, k, l) compared lexicographically as signed integers;
  * plane-wave coefficients are dimensionless: f(r) = sum_G f(G) e^{iGr} for
    potentials and densities, psi(r) = Omega^{-1/2} sum_G psi(G) e^{iGr} with
    sum_G |psi(G)|^2 = 1 for orbitals.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np
import scipy.linalg

__all__ = [
    "Config", "CONFIGS", "System", "miller_sphere", "make_system", "make_spin_system",
    "perturbations", "gauss_legendre_omega", "real_basis_map",
]


@dataclasses.dataclass(frozen=True)
class Config:
    """One synthetic workload (a Gaussian-well model insulator at Gamma)."""
    name: str
    L: float                  # cubic cell side [bohr]
    ecut: float               # wavefunction cutoff [Ha]
    grid: int                 # FFT points per axis
    n_wells: int              # Gaussian wells, positions uniform in the cell
    well_seed: int
    n_v: int                  # doubly occupied states
    n_pert: int = 8
    pert_seed: int = 2
    well_depth: float = 2.0   # D_w [Ha]
    well_width: float = 1.0   # w [bohr]
    kb: bool = False          # one s + three p Gaussian KB projectors per atom
    kb_width: float = 0.8     # w_p [bohr]
    kb_d_s: float = 1.0       # D_s [Ha]
    kb_d_p: float = 0.5       # D_p [Ha]
    kb_dch: bool = False      # five more (d-type) KB projectors per atom
    kb_d_d: float = 0.3       # D_d [Ha]
    min_gap: float = 0.01     # reseed (seed + 1) while HOMO-LUMO gap < this [Ha]
    min_dist: float = 0.0     # hard core: redraw a centre closer than this to an earlier one [bohr]
    n_kb: int = -1            # with kb: only the first n_kb atoms carry projectors (-1: every atom)


CONFIGS = {
    # 24^3 grid, ~500 plane waves, 4 wells, N_v = 4, 8 perturbations.
    "chi0_L10_24": Config("chi0_L10_24", L=10.0, ecut=5.0, grid=24, n_wells=4,
                          well_seed=1, n_v=4, n_pert=8, pert_seed=2),
    # 48^3 grid, ~4k plane waves, 32 wells, N_v = 64, PDEP block of 64.
    # Seeds 3-8 give HOMO-LUMO gaps below 0.01 Ha; the reseeding rule lands on 9.
    "pdep_L16_48": Config("pdep_L16_48", L=16.0, ecut=7.75, grid=48, n_wells=32,
                          well_seed=9, n_v=64, n_pert=64, pert_seed=5),
    # 96^3 grid, ~30k plane waves, 64 atoms with wells + KB projectors, N_v = 256 = 4 per atom.
    # The wells are 6 Ha deep and 0.9 bohr wide and the atoms at least 4 bohr apart, so that each
    # atom binds an s and three p states below a gap (the 2 Ha, 1 bohr well of the smaller models
    # binds one state per atom, and 256 states would then fill a continuum with gaps of ~1e-3 Ha).
    "kb_L24_96": Config("kb_L24_96", L=24.0, ecut=12.75, grid=96, n_wells=64,
                        well_seed=4, n_v=256, n_pert=256, pert_seed=5, kb=True,
                        well_depth=6.0, well_width=0.9, min_dist=4.0),
    # Tiny case (12^3) for quick host checks.
    "tiny_L6_12": Config("tiny_L6_12", L=6.0, ecut=2.5, grid=12, n_wells=2,
                         well_seed=7, n_v=2, n_pert=3, pert_seed=8),
}


# The served mixed stream: one system per grid of SERVE_GRIDS.  On 32^3, 48^3 and 64^3: cell
# L = N/3 bohr at ecut 9 Ha (max Miller index 0.675 L, so each grid is alias-free for the
# iterative solver), wells 6 Ha deep and 0.9 bohr wide at least 4 bohr apart so that every well
# binds an s and three p states below a gap, N_v = 4 x wells drawn uniformly up to what the cell
# holds (SERVE_NV_CAP), and 0-8 of the atoms carrying s + p KB projectors.  On 96^3 the 96^3 KB
# model (kb_L24_96: N_v = 256, 64 KB atoms): the block solver of the ground state does not reach
# 1e-10 within its iteration limit on the L = 32 bohr cell of the same family.
SERVE_GRIDS = (32, 48, 64, 96)
SERVE_NV_CAP = {32: 32, 48: 96, 64: 160, 96: 256}


def serve_stream_configs(seed: int = 55) -> list:
    """The seeded systems of the served mixed stream, one Config per grid of SERVE_GRIDS."""
    rng = np.random.default_rng(seed)
    out = []
    for g in SERVE_GRIDS:
        if g == 96:
            out.append(CONFIGS["kb_L24_96"])
            continue
        n_wells = int(rng.integers(4, SERVE_NV_CAP[g] // 4 + 1))
        n_kb = int(min(rng.integers(0, 9), n_wells))
        out.append(Config(f"serve{g}", L=g / 3.0, ecut=9.0, grid=g, n_wells=n_wells,
                          well_seed=int(rng.integers(1, 1 << 30)), n_v=4 * n_wells, n_pert=128,
                          pert_seed=int(rng.integers(1, 1 << 30)), well_depth=6.0, well_width=0.9,
                          min_dist=4.0, kb=n_kb > 0, n_kb=n_kb if n_kb > 0 else -1))
    return out


def miller_sphere(L: float, ecut: float) -> np.ndarray:
    """Miller triples of the sphere 0.5 (2 pi / L)^2 (h^2+k^2+l^2) <= ecut, canonical order."""
    b = 2.0 * math.pi / L
    nmax_sq = 2.0 * ecut / (b * b)
    m = int(math.floor(math.sqrt(nmax_sq))) + 1
    rng = np.arange(-m, m + 1)
    h, k, l = np.meshgrid(rng, rng, rng, indexing="ij")
    h, k, l = h.ravel(), k.ravel(), l.ravel()
    n2 = h * h + k * k + l * l
    keep = 0.5 * b * b * n2 <= ecut * (1.0 + 1e-12)
    h, k, l, n2 = h[keep], k[keep], l[keep], n2[keep]
    order = np.lexsort((l, k, h, n2))   # last key is primary
    return np.stack([h[order], k[order], l[order]], axis=1).astype(np.int32)


def real_basis_map(miller: np.ndarray):
    """Pairs {G, -G} of a sphere in canonical order.

    Returns (i0, pos, neg): the index of G = 0 and, for each pair, the index of
    the member that is "positive" (h > 0, or h = 0 and k > 0, or h = k = 0 and
    l > 0) and of its mirror.  Pairs are listed in the canonical order of their
    positive member.
    """
    key = {tuple(g): i for i, g in enumerate(miller.tolist())}
    i0 = key[(0, 0, 0)]
    pos, neg = [], []
    for i, (h, k, l) in enumerate(miller.tolist()):
        if h > 0 or (h == 0 and (k > 0 or (k == 0 and l > 0))):
            pos.append(i)
            neg.append(key[(-h, -k, -l)])
    return i0, np.asarray(pos, dtype=np.int64), np.asarray(neg, dtype=np.int64)


@dataclasses.dataclass
class System:
    """Model ground state handed to the response code (what a DFT run would provide)."""
    cfg: Config
    L: float
    omega_cell: float
    ecut: float
    grid: int
    miller_wfc: np.ndarray       # (N_pw, 3) int32, canonical order
    miller_rho: np.ndarray       # (N_rho, 3) int32, canonical order
    vloc_G: np.ndarray           # (N_rho,) complex128, V_loc(G) on the density sphere
    beta_G: np.ndarray           # (N_pw, n_proj) complex128, KB projectors (may have 0 columns)
    d_proj: np.ndarray           # (n_proj,) float64, KB couplings [Ha]
    proj_atom: np.ndarray        # (n_proj,) int32, owning atom
    psi_v: np.ndarray            # (N_pw, n_v) complex128, occupied states, real in r
    e_v: np.ndarray              # (n_v,) float64, ascending
    e_lumo: float                # lowest unoccupied eigenvalue (gap check)
    positions: np.ndarray        # (n_wells, 3) well / atom centres [bohr]
    well_seed_used: int

    @property
    def n_pw(self) -> int:
        return self.miller_wfc.shape[0]

    @property
    def n_rho(self) -> int:
        return self.miller_rho.shape[0]

    @property
    def n_v(self) -> int:
        return self.psi_v.shape[1]

    @property
    def gap(self) -> float:
        return float(self.e_lumo - self.e_v[-1])


def _structure_factor(miller: np.ndarray, positions: np.ndarray, L: float) -> np.ndarray:
    """S_a(G) = exp(-i G . R_a) for every G (rows) and atom (columns)."""
    G = (2.0 * math.pi / L) * miller.astype(np.float64)
    return np.exp(-1j * (G @ positions.T))


def _positions(cfg: Config, seed: int) -> np.ndarray:
    """Centres uniform in the cell from a seeded PCG64; with cfg.min_dist > 0 a centre closer than
    min_dist (minimum image) to an earlier one is redrawn from the same stream."""
    rng = np.random.Generator(np.random.PCG64(seed))
    if cfg.min_dist <= 0:
        return rng.uniform(0.0, cfg.L, size=(cfg.n_wells, 3))
    pts = []
    while len(pts) < cfg.n_wells:
        p = rng.uniform(0.0, cfg.L, size=3)
        ok = True
        for q in pts:
            d = p - q
            d -= cfg.L * np.round(d / cfg.L)
            if np.dot(d, d) < cfg.min_dist ** 2:
                ok = False
                break
        if ok:
            pts.append(p)
    return np.asarray(pts)


def _gaussian_wells(cfg: Config, miller_rho: np.ndarray, positions: np.ndarray) -> np.ndarray:
    """V_loc(G) of V(r) = -D_w sum_a sum_images exp(-|r - R_a|^2 / (2 w^2)).

    (1/Omega) times the 3D Fourier integral of a Gaussian: (2 pi w^2)^{3/2} exp(-w^2 G^2 / 2).
    """
    b = 2.0 * math.pi / cfg.L
    G2 = (b * b) * np.sum(miller_rho.astype(np.float64) ** 2, axis=1)
    w = cfg.well_width
    form = -(cfg.well_depth / cfg.L ** 3) * (2.0 * math.pi * w * w) ** 1.5 * np.exp(-0.5 * w * w * G2)
    return form * _structure_factor(miller_rho, positions, cfg.L).sum(axis=1)


def _kb_projectors(cfg: Config, miller_wfc: np.ndarray, positions: np.ndarray):
    """Per atom: beta_s(G) = Omega^{-1/2} e^{-wp^2 G^2/2} e^{-iG.R}, beta_p,alpha = (-i G_alpha wp) beta_s,
    and with kb_dch five d-type beta_d,k = -wp^2 Q_k(G) beta_s, Q = (GxGy, GyGz, GzGx, (Gx^2 - Gy^2)/2,
    (3Gz^2 - G^2)/(2 sqrt 3)) (the transforms of the l = 2 real harmonics times a Gaussian)."""
    n_pw = miller_wfc.shape[0]
    if not cfg.kb or cfg.n_kb == 0:
        return (np.zeros((n_pw, 0), np.complex128), np.zeros(0), np.zeros(0, np.int32))
    b = 2.0 * math.pi / cfg.L
    G = b * miller_wfc.astype(np.float64)
    G2 = np.sum(G * G, axis=1)
    wp = cfg.kb_width
    radial = np.exp(-0.5 * wp * wp * G2) / math.sqrt(cfg.L ** 3)
    S = _structure_factor(miller_wfc, positions, cfg.L)
    cols, d, atom = [], [], []
    n_atoms = positions.shape[0] if cfg.n_kb < 0 else min(cfg.n_kb, positions.shape[0])
    for a in range(n_atoms):
        s = radial * S[:, a]
        cols.append(s); d.append(cfg.kb_d_s); atom.append(a)
        for alpha in range(3):
            cols.append(-1j * G[:, alpha] * wp * s); d.append(cfg.kb_d_p); atom.append(a)
        if cfg.kb_dch:
            gx, gy, gz = G[:, 0], G[:, 1], G[:, 2]
            for q in (gx * gy, gy * gz, gz * gx, 0.5 * (gx * gx - gy * gy),
                      (3.0 * gz * gz - G2) / (2.0 * math.sqrt(3.0))):
                cols.append(-wp * wp * q * s); d.append(cfg.kb_d_d); atom.append(a)
    return (np.stack(cols, axis=1), np.asarray(d, np.float64), np.asarray(atom, np.int32))


def _dense_h_real(cfg, miller_wfc, miller_rho, vloc_G, beta_G, d_proj):
    """Model Kohn-Sham Hamiltonian in the real basis {1, sqrt2 cos(G.r), sqrt2 sin(G.r)}.

    H_GG' = 0.5|G|^2 delta_GG' + V(G-G') + sum_p beta_p(G) D_p beta_p(G')^* on the
    wavefunction sphere, then rotated with the unitary map between the complex
    and real bases so that it is real symmetric (V and beta are real in r).
    """
    n = miller_wfc.shape[0]
    b = 2.0 * math.pi / cfg.L
    M = int(np.max(np.abs(miller_rho)))
    span = 2 * M + 1
    lookup = np.full(span ** 3, -1, np.int64)
    mr = miller_rho.astype(np.int64) + M
    lookup[(mr[:, 0] * span + mr[:, 1]) * span + mr[:, 2]] = np.arange(miller_rho.shape[0])
    mw = miller_wfc.astype(np.int64)
    H = np.empty((n, n), np.complex128)
    for i in range(n):
        d = mw[i][None, :] - mw + M
        idx = lookup[(d[:, 0] * span + d[:, 1]) * span + d[:, 2]]
        if np.any(idx < 0):
            raise ValueError("G - G' outside the density sphere")
        H[i] = vloc_G[idx]
    H[np.diag_indices(n)] += 0.5 * b * b * np.sum(miller_wfc.astype(np.float64) ** 2, axis=1)
    if beta_G.shape[1]:
        H += (beta_G * d_proj[None, :]) @ beta_G.conj().T
    i0, pos, neg = real_basis_map(miller_wfc)
    s = 1.0 / math.sqrt(2.0)
    HU = np.empty((n, n), np.complex128)
    HU[:, 0] = H[:, i0]
    HU[:, 1::2] = (H[:, pos] + H[:, neg]) * s
    HU[:, 2::2] = (-1j * H[:, pos] + 1j * H[:, neg]) * s
    Hr = np.empty((n, n), np.complex128)
    Hr[0, :] = HU[i0, :]
    Hr[1::2, :] = (HU[pos, :] + HU[neg, :]) * s
    Hr[2::2, :] = (1j * HU[pos, :] - 1j * HU[neg, :]) * s
    if np.max(np.abs(Hr.imag)) > 1e-10 * max(1.0, np.max(np.abs(Hr.real))):
        raise ValueError("model Hamiltonian is not real in the real basis")
    Hr = Hr.real
    return 0.5 * (Hr + Hr.T), (i0, pos, neg)


def _real_to_complex(y: np.ndarray, n: int, basis) -> np.ndarray:
    """Map real-basis coefficient columns back to complex plane-wave coefficients."""
    i0, pos, neg = basis
    s = 1.0 / math.sqrt(2.0)
    c = np.zeros((n, y.shape[1]), np.complex128)
    c[i0] = y[0]
    c[pos] = (y[1::2] - 1j * y[2::2]) * s
    c[neg] = (y[1::2] + 1j * y[2::2]) * s
    return c


# Above this many plane waves the ground state comes from the iterative block solver below
# (a dense real-symmetric diagonalisation of 30095^2 would take tens of minutes).
DENSE_MAX_PW = 9000


def make_system(cfg: Config | str, iterative: bool | None = None) -> System:
    """Build the model ground state of a configuration: dense host diagonalisation, or, for
    spheres above DENSE_MAX_PW plane waves (or iterative=True), the block solver of
    _iterative_ground_state started from a dense solve at a lower cutoff (cached on disk)."""
    if isinstance(cfg, str):
        cfg = CONFIGS[cfg]
    miller_wfc = miller_sphere(cfg.L, cfg.ecut)
    if iterative or (iterative is None and miller_wfc.shape[0] > DENSE_MAX_PW):
        return _make_system_iterative(cfg)
    miller_rho = miller_sphere(cfg.L, 4.0 * cfg.ecut)
    m_rho = int(np.max(np.abs(miller_rho)))
    if cfg.grid <= 2 * m_rho:
        raise ValueError(f"grid {cfg.grid} too small for density sphere (max Miller {m_rho})")
    seed = cfg.well_seed
    for _attempt in range(64):
        positions = _positions(cfg, seed)
        vloc_G = _gaussian_wells(cfg, miller_rho, positions)
        beta_G, d_proj, proj_atom = _kb_projectors(cfg, miller_wfc, positions)
        Hr, basis = _dense_h_real(cfg, miller_wfc, miller_rho, vloc_G, beta_G, d_proj)
        n = Hr.shape[0]
        evals, evecs = scipy.linalg.eigh(Hr, subset_by_index=[0, cfg.n_v], driver="evr")
        if evals[cfg.n_v] - evals[cfg.n_v - 1] >= cfg.min_gap:
            break
        seed += 1
    else:
        raise RuntimeError("no gapped model found")
    y = evecs[:, : cfg.n_v].copy()
    # Sign convention: the largest-magnitude real-basis component of each state is positive.
    piv = np.argmax(np.abs(y), axis=0)
    y *= np.sign(y[piv, np.arange(y.shape[1])])[None, :]
    psi_v = _real_to_complex(y, n, basis)
    return System(cfg=cfg, L=cfg.L, omega_cell=cfg.L ** 3, ecut=cfg.ecut, grid=cfg.grid,
                  miller_wfc=miller_wfc, miller_rho=miller_rho, vloc_G=vloc_G,
                  beta_G=beta_G, d_proj=d_proj, proj_atom=proj_atom, psi_v=psi_v,
                  e_v=evals[: cfg.n_v].copy(), e_lumo=float(evals[cfg.n_v]),
                  positions=positions, well_seed_used=seed)


def make_spin_system(cfg: Config | str, depth_split: float = 0.4, n_v_down: int | None = None):
    """Two spin channels of one model: the same cell, cutoff and well positions, wells deeper by
    depth_split/2 for spin up and shallower by depth_split/2 for spin down (a model exchange
    splitting).  Spin up holds n_v occupied states; spin down n_v_down, by default the largest
    count in n_v-1 .. n_v-4 whose gap to the next state is at least min_gap (else the count
    with the largest gap).  Returns (up, down) Systems; the down channel keeps the up channel's
    well seed."""
    if isinstance(cfg, str):
        cfg = CONFIGS[cfg]
    up = make_system(dataclasses.replace(cfg, well_depth=cfg.well_depth + 0.5 * depth_split))
    full = make_system(dataclasses.replace(cfg, well_depth=cfg.well_depth - 0.5 * depth_split,
                                           well_seed=up.well_seed_used, min_gap=-1.0))
    levels = np.append(full.e_v, full.e_lumo)
    if n_v_down is None:
        counts = list(range(cfg.n_v - 1, max(1, cfg.n_v - 4) - 1, -1))
        gaps = [levels[c] - levels[c - 1] for c in counts]
        ok = [c for c, g in zip(counts, gaps) if g >= cfg.min_gap]
        n_v_down = ok[0] if ok else counts[int(np.argmax(gaps))]
    down = dataclasses.replace(full, psi_v=full.psi_v[:, :n_v_down].copy(), e_v=full.e_v[:n_v_down].copy(),
                               e_lumo=float(levels[n_v_down]))
    return up, down


def perturbations(miller_rho: np.ndarray, L: float, n_pert: int, seed: int,
                  hermitian: bool = True) -> np.ndarray:
    """Seeded perturbations dV(G) on the density sphere, shape (N_rho, n_pert), complex128.

    N(0,1) + i N(0,1) coefficients on the positive half of the sphere, mirrored
    as dV(-G) = dV(G)^* (a real perturbation at Gamma) unless hermitian=False,
    dV(0) = 0, multiplied by v^{1/2}(G) = sqrt(4 pi)/|G|, and normalised to
    sum_G |dV(G)|^2 = 1.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    n = miller_rho.shape[0]
    i0, pos, neg = real_basis_map(miller_rho)
    out = np.zeros((n, n_pert), np.complex128)
    draws = rng.standard_normal((2, pos.size, n_pert)) + 1j * rng.standard_normal((2, pos.size, n_pert))
    out[pos] = draws[0]
    out[neg] = draws[0].conj() if hermitian else draws[1]
    out[i0] = 0.0
    b = 2.0 * math.pi / L
    g = b * np.sqrt(np.sum(miller_rho.astype(np.float64) ** 2, axis=1))
    vh = np.zeros(n)
    vh[g > 0] = math.sqrt(4.0 * math.pi) / g[g > 0]
    out *= vh[:, None]
    out /= np.linalg.norm(out, axis=0, keepdims=True)
    return out


def gauss_legendre_omega(n: int = 32, omega_max: float = 50.0):
    """Imaginary frequencies: n Gauss-Legendre nodes mapped linearly from [-1, 1] to [0, omega_max]."""
    x, w = np.polynomial.legendre.leggauss(n)
    half = 0.5 * omega_max
    return half * (x + 1.0), half * w


# ---------------------------------------------------------------- iterative ground state
# For the large configuration (96^3 grid, 30095 plane waves, 256 occupied states) the lowest
# eigenpairs of the model Hamiltonian come from a block LOBPCG iteration (Knyazev 2001) in the
# real basis {1, sqrt2 cos(G.r), sqrt2 sin(G.r)}, with H applied through real-to-complex FFTs
# (exact on these alias-free grids: grid > 4 x max Miller index of the wavefunction sphere), a
# Teter-Payne-Allan kinetic preconditioner, and a start block from a dense diagonalisation at a
# lower cutoff.  Ground-state diagonalisation only: no response arithmetic.

def _cache_dir() -> str:
    import os
    d = os.environ.get("WGW_SYNTH_CACHE") or os.path.join(os.path.dirname(os.path.dirname(
        os.path.abspath(__file__))), "_cache")
    os.makedirs(d, exist_ok=True)
    return d


def _to_real_basis(c: np.ndarray, basis) -> np.ndarray:
    """Complex coefficient columns of functions real in r -> real-basis columns (inverse of
    _real_to_complex)."""
    i0, pos, _neg = basis
    y = np.empty((c.shape[0], c.shape[1]))
    y[0] = c[i0].real
    y[1::2] = math.sqrt(2.0) * c[pos].real
    y[2::2] = -math.sqrt(2.0) * c[pos].imag
    return y


class _RealH:
    """The model Hamiltonian on real-basis columns: 0.5 G^2 y + FFT[V(r) FFT^-1 y] + B D B^T y."""

    def __init__(self, cfg, miller_wfc, miller_rho, vloc_G, beta_G, d_proj, workers=None):
        import os
        import scipy.fft
        self.fft = scipy.fft
        self.workers = workers or os.cpu_count()
        self.N = cfg.grid
        self.n = miller_wfc.shape[0]
        self.basis = real_basis_map(miller_wfc)
        b = 2.0 * math.pi / cfg.L
        g2 = (b * b) * np.sum(miller_wfc.astype(np.float64) ** 2, axis=1)
        i0, pos, _ = self.basis
        self.kin = np.empty(self.n)
        self.kin[0] = 0.5 * g2[i0]
        self.kin[1::2] = 0.5 * g2[pos]
        self.kin[2::2] = 0.5 * g2[pos]
        N = self.N
        # Half-spectrum positions (l >= 0) of the sphere members and of the positive members.
        mw = miller_wfc.astype(np.int64)
        self.half = np.where(mw[:, 2] >= 0)[0]
        self.h_idx = tuple(np.mod(mw[self.half].T, N))
        # Positive members with l >= 0 are read directly, those with l < 0 through their mirror
        # -G (l > 0) and a conjugation.
        self.pos_direct = np.where(mw[pos, 2] >= 0)[0]
        self.pos_mirror = np.where(mw[pos, 2] < 0)[0]
        self.pos_direct_idx = tuple(np.mod(mw[pos][self.pos_direct].T, N))
        self.pos_mirror_idx = tuple(np.mod(-mw[pos][self.pos_mirror].T, N))
        self.i0_idx = (0, 0, 0)
        mr = miller_rho.astype(np.int64)
        keep = mr[:, 2] >= 0
        grid = np.zeros((N, N, N // 2 + 1), np.complex128)
        grid[tuple(np.mod(mr[keep].T, N))] = vloc_G[keep]
        self.v_r = scipy.fft.irfftn(grid, s=(N, N, N), axes=(0, 1, 2), workers=self.workers) * N ** 3
        self.B = _to_real_basis(beta_G, self.basis) if beta_G.shape[1] else None
        self.D = np.asarray(d_proj, np.float64)

    def __call__(self, y: np.ndarray, chunk: int = 64) -> np.ndarray:
        out = self.kin[:, None] * y
        N = self.N
        s2 = 1.0 / math.sqrt(2.0)
        for j0 in range(0, y.shape[1], chunk):
            yb = y[:, j0:j0 + chunk]
            c = _real_to_complex(yb, self.n, self.basis)
            grid = np.zeros((yb.shape[1], N, N, N // 2 + 1), np.complex128)
            grid[(slice(None),) + self.h_idx] = c[self.half].T
            r = self.fft.irfftn(grid, s=(N, N, N), axes=(1, 2, 3), workers=self.workers) * N ** 3
            r *= self.v_r[None]
            g = self.fft.rfftn(r, axes=(1, 2, 3), workers=self.workers) / N ** 3
            vp = np.empty((yb.shape[1], self.pos_direct.size + self.pos_mirror.size), np.complex128)
            vp[:, self.pos_direct] = g[(slice(None),) + self.pos_direct_idx]   # value at +G
            vp[:, self.pos_mirror] = np.conj(g[(slice(None),) + self.pos_mirror_idx])
            out[0, j0:j0 + chunk] += g[(slice(None),) + self.i0_idx].real
            out[1::2, j0:j0 + chunk] += (2.0 * s2) * vp.real.T
            out[2::2, j0:j0 + chunk] += -(2.0 * s2) * vp.imag.T
        if self.B is not None:
            out += self.B @ (self.D[:, None] * (self.B.T @ y))
        return out

    def precondition(self, r: np.ndarray, x: np.ndarray) -> np.ndarray:
        """Teter-Payne-Allan preconditioner per column, scaled by the column's kinetic energy."""
        ek = np.sum(self.kin[:, None] * x * x, axis=0) / np.maximum(np.sum(x * x, axis=0), 1e-300)
        t = self.kin[:, None] / np.maximum(ek[None, :], 1e-3)
        num = 27.0 + t * (18.0 + t * (12.0 + 8.0 * t))
        return r * (num / (num + 16.0 * t ** 4))


def _orthonormalize(S: np.ndarray) -> np.ndarray:
    """Orthonormal columns spanning S (Cholesky QR twice, eigen-decomposition of the Gram matrix
    when it is too ill-conditioned), dropping directions below 1e-13 of the largest."""
    for _ in range(2):
        G = S.T @ S
        try:
            Lc = np.linalg.cholesky(G)
            if np.min(np.abs(np.diag(Lc))) < 1e-7 * np.max(np.abs(np.diag(Lc))):
                raise np.linalg.LinAlgError
            S = scipy.linalg.solve_triangular(Lc, S.T, lower=True).T
        except np.linalg.LinAlgError:
            w, U = np.linalg.eigh(0.5 * (G + G.T))
            keep = w > 1e-26 * w[-1]
            S = S @ (U[:, keep] / np.sqrt(w[keep]))
    return S


def _lobpcg(H: _RealH, X: np.ndarray, n_conv: int, tol: float, max_iter: int = 300, log=None, give_up=None):
    """Lowest eigenpairs of H by block LOBPCG from the columns of X.  Each step: residuals
    R = HX - X theta, preconditioned W = T R (converged columns left out), Rayleigh-Ritz on
    span[X, W, P] made orthonormal by whitening its Gram matrix (dropping near-dependent
    directions), P = the W, P part of the new X.  Converged when the first n_conv residual
    norms ||H x - theta x|| are <= tol.  Returns (theta, X, iterations), ascending, or None when
    give_up(theta, residual norms) says so first."""
    X = _orthonormalize(X)
    m = X.shape[1]
    HX = H(X)
    theta, C = np.linalg.eigh(0.5 * (X.T @ HX + HX.T @ X))
    X, HX = X @ C, HX @ C
    P = HP = None
    for it in range(max_iter):
        R = HX - X * theta[None, :]
        rn = np.linalg.norm(R, axis=0)
        if log:
            log(it, theta, rn)
        if np.all(rn[:n_conv] <= tol):
            return theta, X, it
        if give_up is not None and give_up(theta, rn):
            return None
        act = np.where(rn > 0.1 * tol)[0]
        Wb = H.precondition(R[:, act], X[:, act])
        Wb -= X @ (X.T @ Wb)
        Wb /= np.maximum(np.linalg.norm(Wb, axis=0), 1e-300)[None, :]
        HW = H(Wb)
        S = [X, Wb] + ([P] if P is not None else [])
        HS = [HX, HW] + ([HP] if P is not None else [])
        S = np.concatenate(S, axis=1)
        HS = np.concatenate(HS, axis=1)
        G = S.T @ S
        A = S.T @ HS
        g, U = np.linalg.eigh(0.5 * (G + G.T))
        keep = g > 1e-13 * g[-1]
        T = U[:, keep] / np.sqrt(g[keep])
        th, V = np.linalg.eigh(T.T @ (0.5 * (A + A.T)) @ T)
        Cm = (T @ V)[:, :m]
        theta = th[:m]
        P = S[:, m:] @ Cm[m:]
        HP = HS[:, m:] @ Cm[m:]
        X = X @ Cm[:m] + P
        HX = HX @ Cm[:m] + HP
        # Keep X orthonormal against rounding (a triangular change of basis, applied to HX too).
        Lc = np.linalg.cholesky(X.T @ X)
        X = scipy.linalg.solve_triangular(Lc, X.T, lower=True).T
        HX = scipy.linalg.solve_triangular(Lc, HX.T, lower=True).T
        nP = np.maximum(np.linalg.norm(P, axis=0), 1e-300)
        P, HP = P / nP[None, :], HP / nP[None, :]
        if it % 20 == 19:
            HX = H(X)                     # drop the rounding drift of the updated images
            theta, C = np.linalg.eigh(0.5 * (X.T @ HX + HX.T @ X))
            X, HX = X @ C, HX @ C
            P = HP = None
    raise RuntimeError("LOBPCG did not converge")


def _cache_key(cfg: Config) -> str:
    import hashlib
    fields = dataclasses.astuple(cfg)
    if cfg.n_kb < 0:             # the field came later: keys of configurations without it stay put
        fields = fields[:-1]
    return hashlib.sha256(repr(fields).encode() + b"lobpcg-v1").hexdigest()[:20]


def _make_system_iterative(cfg: Config, tol: float = 1e-10) -> System:
    import os
    miller_wfc = miller_sphere(cfg.L, cfg.ecut)
    miller_rho = miller_sphere(cfg.L, 4.0 * cfg.ecut)
    m_wfc = int(np.max(np.abs(miller_wfc)))
    if cfg.grid <= 4 * m_wfc:
        raise ValueError("the iterative ground state needs an alias-free grid (> 4 x max Miller)")
    path = os.path.join(_cache_dir(), f"gs_{cfg.name}_{_cache_key(cfg)}.npz")
    if os.path.exists(path):
        z = np.load(path)
        seed = int(z["seed"])
        positions = _positions(cfg, seed)
        vloc_G = _gaussian_wells(cfg, miller_rho, positions)
        beta_G, d_proj, proj_atom = _kb_projectors(cfg, miller_wfc, positions)
        return System(cfg=cfg, L=cfg.L, omega_cell=cfg.L ** 3, ecut=cfg.ecut, grid=cfg.grid,
                      miller_wfc=miller_wfc, miller_rho=miller_rho, vloc_G=vloc_G, beta_G=beta_G,
                      d_proj=d_proj, proj_atom=proj_atom, psi_v=z["psi_v"], e_v=z["e_v"],
                      e_lumo=float(z["e_lumo"]), positions=positions, well_seed_used=seed)
    n_want = cfg.n_v + 1                               # the occupied states and the LUMO
    m = n_want + max(16, cfg.n_v // 16)                # guard vectors
    seed = cfg.well_seed
    for _attempt in range(16):
        positions = _positions(cfg, seed)
        vloc_G = _gaussian_wells(cfg, miller_rho, positions)
        beta_G, d_proj, proj_atom = _kb_projectors(cfg, miller_wfc, positions)
        H = _RealH(cfg, miller_wfc, miller_rho, vloc_G, beta_G, d_proj)
        X0 = _low_cutoff_start(cfg, miller_wfc, positions, m, H.basis)

        def gap_too_small(theta, rn, nv=cfg.n_v):
            # Residuals below 1e-5 put the eigenvalues within ~1e-9 of their limits: a gap
            # clearly below min_gap by then will not open up, so the seed is dropped early.
            return np.max(rn[: nv + 1]) < 1e-5 and theta[nv] - theta[nv - 1] < cfg.min_gap - 1e-6

        res = _lobpcg(H, X0, n_want, tol, give_up=gap_too_small)
        if res is not None:
            theta, X, _ = res
            if theta[cfg.n_v] - theta[cfg.n_v - 1] >= cfg.min_gap:
                break
        seed += 1
    else:
        raise RuntimeError("no gapped model found")
    y = X[:, : cfg.n_v].copy()
    piv = np.argmax(np.abs(y), axis=0)
    y *= np.sign(y[piv, np.arange(y.shape[1])])[None, :]
    psi_v = _real_to_complex(y, miller_wfc.shape[0], H.basis)
    e_v = theta[: cfg.n_v].copy()
    np.savez(path + ".tmp.npz", psi_v=psi_v, e_v=e_v, e_lumo=theta[cfg.n_v], seed=seed)
    os.replace(path + ".tmp.npz", path)
    return System(cfg=cfg, L=cfg.L, omega_cell=cfg.L ** 3, ecut=cfg.ecut, grid=cfg.grid,
                  miller_wfc=miller_wfc, miller_rho=miller_rho, vloc_G=vloc_G, beta_G=beta_G,
                  d_proj=d_proj, proj_atom=proj_atom, psi_v=psi_v, e_v=e_v,
                  e_lumo=float(theta[cfg.n_v]), positions=positions, well_seed_used=seed)


def _low_cutoff_start(cfg: Config, miller_wfc, positions, m: int, basis) -> np.ndarray:
    """Start block: the m lowest eigenvectors of the same model at a cutoff with about 5000 plane
    waves (dense diagonalisation), placed in the full sphere's real basis."""
    n = miller_wfc.shape[0]
    ecut0 = min(cfg.ecut, cfg.ecut * (5000.0 / n) ** (2.0 / 3.0))
    lo = dataclasses.replace(cfg, ecut=ecut0)
    mw0 = miller_sphere(cfg.L, ecut0)
    mr0 = miller_sphere(cfg.L, 4.0 * ecut0)
    v0 = _gaussian_wells(lo, mr0, positions)
    b0, d0, _ = _kb_projectors(lo, mw0, positions)
    Hr, basis0 = _dense_h_real(lo, mw0, mr0, v0, b0, d0)
    _, vecs = scipy.linalg.eigh(Hr, subset_by_index=[0, min(m, Hr.shape[0]) - 1], driver="evr")
    c0 = _real_to_complex(vecs, mw0.shape[0], basis0)
    where = {tuple(g): i for i, g in enumerate(miller_wfc.tolist())}
    idx = np.array([where[tuple(g)] for g in mw0.tolist()])
    c = np.zeros((n, vecs.shape[1]), np.complex128)
    c[idx] = c0
    X = _to_real_basis(c, basis)
    if X.shape[1] < m:
        rng = np.random.default_rng(0)
        X = np.concatenate([X, rng.standard_normal((n, m - X.shape[1]))], axis=1)
    return X
