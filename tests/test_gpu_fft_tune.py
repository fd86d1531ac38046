"""Kernel choices of the FP32 FFT stages (G -> r planes, x-lines with V(r), r -> G planes; the
transforms of Sec. 4.1's H application) against the oracle.

Each stage runs the register-resident kernel (one line per thread), the same with packed FP32
butterflies, or the shared-memory kernel; all compute the same transforms, so a mixed-path apply
matches the oracle's sum over states within the path's 1e-8 whatever the choice, on every grid
with register-resident kernels (24, 32, 64, and 96 in FP32; 48 is the 48^3 model of the other
files).  The autotuner times every candidate of every stage on the first application to >= 256
systems and keeps the fastest; a fixed choice is bit-identical from one context to the next.
"""
import numpy as np
import pytest

import synth
from oracle import chi0
from oracle.model import Model

pytestmark = pytest.mark.gpu

MODELS = {
    24: "chi0_L10_24",
    32: synth.Config("g32", L=32.0 / 3.0, ecut=9.0, grid=32, n_wells=8, well_seed=3, n_v=16, kb=True),
    64: synth.Config("g64", L=16.0, ecut=7.75, grid=64, n_wells=32, well_seed=3, n_v=16),
    96: synth.Config("g96", L=24.0, ecut=3.3, grid=96, n_wells=64, well_seed=3, n_v=16, kb=True),
}
CHOICES = [(0, 0, 0), (1, 1, 1), (2, 2, 2), (2, 0, 1)]


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


def _model(s):
    return Model(s.L, s.ecut, s.grid, s.vloc_G, s.psi_v, s.e_v, s.beta_G, s.d_proj)


def _ctx(W, s, cg_tol=1e-10, **opt):
    kb = s.beta_G.shape[1] > 0
    return W.wgw_setup(s.L, s.ecut, s.grid, s.vloc_G, s.psi_v, s.e_v,
                       W.wgw_default_options(precision=W.WGW_MIXED, cg_tol=cg_tol, **opt),
                       beta_G=s.beta_G if kb else None, d_proj=s.d_proj if kb else None)


@pytest.fixture(scope="module", params=sorted(MODELS))
def case(request):
    s = synth.make_system(MODELS[request.param])
    dV = synth.perturbations(s.miller_rho, s.L, 2, 70 + request.param)
    return s, dV, chi0.sos_drho(_model(s), dV, [0.0])


@pytest.mark.parametrize("choice", CHOICES)
def test_every_fft_kernel_choice_matches_oracle(W, case, choice):
    s, dV, ref = case
    ctx = _ctx(W, s, fft_kernels=choice)
    drho, st, _ = W.wgw_apply_chi0(ctx, dV)
    assert st["n_converged"] == st["n_systems"]
    assert rel_err(drho, ref) < 1e-8
    rep = W.wgw_autotune_fft(ctx)
    names = [W.FFT_KERNEL_NAMES[k] for k in choice]
    assert [rep[st_]["choice"] for st_ in ("g2r", "xline", "r2g")] == names


def test_fft_autotuner_times_every_candidate(W):
    """280 systems: the first FP32 H application times the three candidates of each stage."""
    s = synth.make_system(synth.Config("nv70", L=10.0, ecut=5.0, grid=24, n_wells=16, well_seed=1, n_v=70))
    dV = synth.perturbations(s.miller_rho, s.L, 4, 64)
    ctx = _ctx(W, s, cg_tol=1e-11)
    assert all(v["choice"] == "untuned" for v in W.wgw_autotune_fft(ctx).values())
    drho, st, _ = W.wgw_apply_chi0(ctx, dV)
    rep = W.wgw_autotune_fft(ctx)
    for stage in ("g2r", "xline", "r2g"):
        assert rep[stage]["choice"] in ("register", "register, packed FP32", "shared memory")
        assert all(t > 0 for t in rep[stage]["ms"].values())
        # The kept candidate is the fastest one timed.
        assert rep[stage]["ms"][rep[stage]["choice"]] == min(rep[stage]["ms"].values())
    assert rel_err(drho, chi0.sos_drho(_model(s), dV, [0.0])) < 1e-8


def test_fixed_fft_choice_is_bit_identical_across_contexts(W):
    s = synth.make_system(synth.Config("nv70", L=10.0, ecut=5.0, grid=24, n_wells=16, well_seed=1, n_v=70))
    dV = synth.perturbations(s.miller_rho, s.L, 4, 65)
    outs = []
    for _ in range(2):
        ctx = _ctx(W, s, cg_tol=1e-11, fft_kernels=(2, 1, 0), fused_h=0, tc_split=4)
        outs.append(W.wgw_apply_chi0(ctx, dV)[0])
    assert np.array_equal(outs[0], outs[1])


def test_h_chunks_are_bit_identical(W):
    """The FP32 H pipeline run in chunks of pairs (ragged last chunk included) computes every pair
    exactly as the unchunked run: bit-identical results, and the oracle's within 1e-8."""
    s = synth.make_system(synth.Config("nv70", L=10.0, ecut=5.0, grid=24, n_wells=16, well_seed=1, n_v=70))
    dV = synth.perturbations(s.miller_rho, s.L, 4, 66)          # 280 systems = 140 pairs
    outs = []
    for chunk in (0, 16, 45):
        ctx = _ctx(W, s, cg_tol=1e-11, fft_kernels=(1, 1, 1), fused_h=0, tc_split=4, h_chunk_pairs=chunk)
        outs.append(W.wgw_apply_chi0(ctx, dV)[0])
        assert W.wgw_autotune_chunk(ctx)["chunk_pairs"] == chunk
    assert np.array_equal(outs[0], outs[1]) and np.array_equal(outs[0], outs[2])
    assert rel_err(outs[0], chi0.sos_drho(_model(s), dV, [0.0])) < 1e-8


def test_chunk_autotuner_times_its_candidates(W):
    """256 systems of the 48^3 model (128 pairs, 21 x 48^2 complex FP32 = 387,072 B each): no chunking
    and 32 MB chunks (86 pairs; 64 MB would exceed the list) are timed at the first FP32 H
    application and one is kept."""
    s = synth.make_system("pdep_L16_48")
    phi = synth.perturbations(s.miller_rho, s.L, 4, 67)
    ctx = _ctx(W, s, fused_h=0)
    assert W.wgw_autotune_chunk(ctx)["chunk_pairs"] == -1
    _, st, _ = W.wgw_apply_chibar0(ctx, phi)
    assert st["n_converged"] == st["n_systems"] == 256
    rep = W.wgw_autotune_chunk(ctx)
    assert sorted(rep["candidates_ms"]) == [0, 32 * 1048576 // (21 * 48 * 48 * 8)]
    assert all(t > 0 for t in rep["candidates_ms"].values())
    assert rep["chunk_pairs"] == min(rep["candidates_ms"], key=rep["candidates_ms"].get)
