"""Parity on every grid size the library compiles kernels for, against the FP64 oracle.

The FFT kernels are instantiated per grid (compile-time radix plans): register-resident FP32
line kernels for N <= 64, register float-float kernels for N <= 32, shared-memory kernels for
the rest, native FP64 kernels for the FP64 path.  The 24^3 and 48^3 models of the other test
files cover N = 24 and 48; the models here put N = 32, 64 and 96 under the same parity bar:
FP64 path 1e-10, mixed path 1e-8 (relative error per perturbation and frequency), static and
at an imaginary frequency, with Kleinman-Bylander projectors on two of the grids.

Models (seeded Gaussian-well insulators; sizes chosen so that the oracle's sum over states
finishes in under a minute):
  g32  L = 32/3 bohr, ecut 9 Ha (the L = N/3, 9 Ha family of the served stream), 8 atoms with
       wells and s+p projectors, 16 occupied states: 1551 plane waves, max Miller 7.
  g64  L = 16 bohr, ecut 7.75 Ha (the 48^3 model's sphere) on a 64^3 grid, 32 wells, 16 states.
  g96  L = 24 bohr (the cell of the 96^3 KB configuration) at ecut 3.3 Ha on a 96^3 grid,
       64 atoms with wells and s+p projectors, 16 states: 3911 plane waves, max Miller 9.
"""
import numpy as np
import pytest

import synth
from oracle import chi0
from oracle.model import Model

pytestmark = pytest.mark.gpu

GRID_MODELS = {
    32: synth.Config("g32", L=32.0 / 3.0, ecut=9.0, grid=32, n_wells=8, well_seed=3, n_v=16, kb=True),
    64: synth.Config("g64", L=16.0, ecut=7.75, grid=64, n_wells=32, well_seed=3, n_v=16),
    96: synth.Config("g96", L=24.0, ecut=3.3, grid=96, n_wells=64, well_seed=3, n_v=16, kb=True),
}
OMEGAS = [0.0, 0.8]


@pytest.fixture(scope="module")
def W():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2203_05623_gb300 import build
    build.build()
    import paper_2203_05623_gb300 as W
    return W


def rel_err(got, ref):
    num = np.linalg.norm(got - ref, axis=0)
    den = np.linalg.norm(ref, axis=0)
    return float(np.max(num / np.where(den > 0, den, 1.0)))


@pytest.fixture(scope="module", params=sorted(GRID_MODELS))
def grid_case(request):
    s = synth.make_system(GRID_MODELS[request.param])
    m = Model(s.L, s.ecut, s.grid, s.vloc_G, s.psi_v, s.e_v, s.beta_G, s.d_proj)
    dV = synth.perturbations(s.miller_rho, s.L, 3, 40 + request.param)
    return s, dV, chi0.sos_drho(m, dV, OMEGAS)


def _ctx(W, s, **opt):
    kb = s.beta_G.shape[1] > 0
    return W.wgw_setup(s.L, s.ecut, s.grid, s.vloc_G, s.psi_v, s.e_v, W.wgw_default_options(**opt),
                       beta_G=s.beta_G if kb else None, d_proj=s.d_proj if kb else None)


@pytest.mark.parametrize("path", ["fp64", "mixed", "mixed_native64"])
def test_grid_parity(W, grid_case, path):
    """chi0(i w) dV on the grid's kernels: FP64 path, mixed path with float-float FP64-accuracy
    passes (the default), and mixed path with native FP64 passes."""
    s, dV, ref = grid_case
    if path == "fp64":
        ctx = _ctx(W, s, precision=W.WGW_FP64, cg_tol=1e-13)
        tol = 1e-10
    else:
        ctx = _ctx(W, s, precision=W.WGW_MIXED, cg_tol=1e-11, fp64_emulation=0 if path == "mixed_native64" else 1)
        tol = 1e-8
    drho, st, _ = W.wgw_apply_chi0(ctx, dV, OMEGAS)
    n_sys = dV.shape[1] * s.n_v * len(OMEGAS)
    assert st["n_systems"] == n_sys and st["n_converged"] == n_sys
    assert rel_err(drho.reshape(drho.shape[0], -1), ref.reshape(ref.shape[0], -1)) < tol


def test_grid_apply_h(W, grid_case):
    """H psi on the grid's kernels against the oracle's H: FP64-accuracy passes to 1e-12 and the
    FP32 kernels to 1e-5 of the largest element, and H psi_v = e_v psi_v on the given states."""
    import torch
    s, _, _ = grid_case
    m = Model(s.L, s.ecut, s.grid, s.vloc_G, s.psi_v, s.e_v, s.beta_G, s.d_proj)
    x = synth.perturbations(s.miller_wfc, s.L, 5, 73)
    ref = m.apply_h(x)
    ctx = _ctx(W, s, precision=W.WGW_MIXED)
    xd = torch.from_numpy(np.ascontiguousarray(x.T)).cuda()
    for fp32, tol in ((0, 1e-12), (1, 1e-5)):
        out = W.wgw_apply_h_dev(ctx, xd, fp32=bool(fp32)).cpu().numpy().T
        assert np.max(np.abs(out - ref)) < tol * np.max(np.abs(ref)), fp32
    pv = torch.from_numpy(np.ascontiguousarray(s.psi_v.T)).cuda()
    hv = W.wgw_apply_h_dev(ctx, pv).cpu().numpy().T
    assert np.max(np.abs(hv - s.psi_v * s.e_v[None, :])) < 1e-10 * np.max(np.abs(s.e_v))
