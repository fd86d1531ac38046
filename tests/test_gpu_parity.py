"""Parity of the CUDA path (through the C ABI) with the FP64 oracle, on a GB300.

Tolerances: FP64 path 1e-10, mixed path 1e-8, as the relative error
||drho_gpu - drho_ref||_2 / ||drho_ref||_2 per perturbation (max over the batch).
"""
import numpy as np
import pytest

import synth
from oracle import chi0
from oracle.model import Model

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def W():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2203_05623_gb300 import build
    build.build()
    import paper_2203_05623_gb300 as W
    return W


def model_of(s):
    return Model(s.L, s.ecut, s.grid, s.vloc_G, s.psi_v, s.e_v, s.beta_G, s.d_proj)


def rel_err(got, ref):
    """max over perturbations (and frequencies) of ||got - ref|| / ||ref||."""
    num = np.linalg.norm(got - ref, axis=0)
    den = np.linalg.norm(ref, axis=0)
    return float(np.max(num / np.where(den > 0, den, 1.0)))


def setup(W, s, **opt):
    o = W.wgw_default_options(**opt)
    kb = s.beta_G.shape[1] > 0
    return W.wgw_setup(s.L, s.ecut, s.grid, s.vloc_G, s.psi_v, s.e_v, o,
                       beta_G=s.beta_G if kb else None, d_proj=s.d_proj if kb else None)


def test_gvectors_match_generator(W, cfg24):
    ctx = setup(W, cfg24)
    assert np.array_equal(W.wgw_get_gvectors(ctx, W.WGW_SPHERE_WFC), cfg24.miller_wfc)
    assert np.array_equal(W.wgw_get_gvectors(ctx, W.WGW_SPHERE_RHO), cfg24.miller_rho)


@pytest.fixture(scope="module")
def ref24(cfg24):
    dV = synth.perturbations(cfg24.miller_rho, cfg24.L, 8, 2)
    return dV, chi0.sos_drho(model_of(cfg24), dV, [0.0])


def test_chi0_fp64_matches_sum_over_states(W, cfg24, ref24):
    dV, ref = ref24
    ctx = setup(W, cfg24, precision=W.WGW_FP64, cg_tol=1e-13)
    drho, st, status = W.wgw_apply_chi0(ctx, dV)
    assert st["n_systems"] == 32 and st["n_converged"] == 32
    assert rel_err(drho, ref) < 1e-10


@pytest.mark.parametrize("emulate,tcores", [(1, 1), (0, 1), (1, 0)])
def test_chi0_mixed_matches_sum_over_states(W, cfg24, ref24, emulate, tcores):
    """Mixed path: FP64-accuracy passes in float-float (default) or native FP64; P_c of the FP32
    solves on the tcgen05 tensor cores (default) or CUDA cores."""
    dV, ref = ref24
    ctx = setup(W, cfg24, precision=W.WGW_MIXED, cg_tol=1e-11, fp64_emulation=emulate, tensor_cores=tcores)
    drho, st, status = W.wgw_apply_chi0(ctx, dV)
    assert st["refinements"] >= 2
    assert rel_err(drho, ref) < 1e-8


@pytest.mark.parametrize("n_v,n_wells", [(70, 16), (256, 48)])
def test_many_occupied_states_tensor_core_projector(W, n_v, n_wells):
    """P_c with more occupied states than one 64-wide MMA tile (70: a ragged tile; 256: the
    largest count the tensor-core projector takes), mixed path on both projector kinds."""
    s = synth.make_system(synth.Config(f"nv{n_v}", L=10.0, ecut=5.0, grid=24, n_wells=n_wells,
                                       well_seed=1, n_v=n_v))
    dV = synth.perturbations(s.miller_rho, s.L, 3, 61)
    ref = chi0.sos_drho(model_of(s), dV, [0.0])[:, :, 0]
    for tcores in (1, 0):
        ctx = setup(W, s, precision=W.WGW_MIXED, cg_tol=1e-11, tensor_cores=tcores)
        drho, st, _ = W.wgw_apply_chi0(ctx, dV)
        assert st["n_systems"] == 3 * n_v and st["n_converged"] == 3 * n_v
        assert rel_err(drho[:, :, 0], ref) < 1e-8, tcores


def test_complex_perturbation_by_linearity(W, tiny):
    dV = synth.perturbations(tiny.miller_rho, tiny.L, 3, 11, hermitian=False)
    ref = chi0.sos_drho(model_of(tiny), dV, [0.0])
    ctx = setup(W, tiny, cg_tol=1e-13)
    drho, st, _ = W.wgw_apply_chi0(ctx, dV)
    assert st["n_systems"] == 2 * 3 * tiny.n_v
    assert rel_err(drho, ref) < 1e-10


def test_odd_system_count_and_ragged_pairs(W):
    s = synth.make_system(synth.Config("odd", L=7.0, ecut=3.0, grid=16, n_wells=3, well_seed=21,
                                       n_v=3, min_gap=0.05))
    dV = synth.perturbations(s.miller_rho, s.L, 3, 5)       # 9 systems: the last pair is half empty
    ref = chi0.sos_drho(model_of(s), dV, [0.0])
    ctx = setup(W, s, cg_tol=1e-13)
    drho, st, _ = W.wgw_apply_chi0(ctx, dV)
    assert st["n_systems"] == 9
    assert rel_err(drho, ref) < 1e-10


def test_device_entry_point_matches_host_and_symmetrised(W, cfg24, ref24):
    import torch
    dV, ref = ref24
    ctx = setup(W, cfg24, cg_tol=1e-13)
    host, _, _ = W.wgw_apply_chi0(ctx, dV)
    x = torch.from_numpy(np.ascontiguousarray(dV.T)).cuda()
    out = torch.zeros((1, dV.shape[1], dV.shape[0]), dtype=torch.complex128, device="cuda")
    W.wgw_apply_chi0_dev(ctx, x, [0.0], out)
    torch.cuda.synchronize()
    dev = out.cpu().numpy().transpose(2, 1, 0)
    assert np.array_equal(dev, host)
    # chibar0 phi = v^1/2 chi0 (v^1/2 phi)
    m = model_of(cfg24)
    phi = synth.perturbations(cfg24.miller_rho, cfg24.L, 3, 17)
    o2 = torch.zeros((1, 3, dV.shape[0]), dtype=torch.complex128, device="cuda")
    W.wgw_apply_chibar0_dev(ctx, torch.from_numpy(np.ascontiguousarray(phi.T)).cuda(), [0.0], o2)
    torch.cuda.synchronize()
    got = o2.cpu().numpy().transpose(2, 1, 0)
    assert rel_err(got, chi0.apply_chibar0(m, phi, [0.0])) < 1e-10


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_imaginary_frequencies_match_sum_over_states(W, cfg24, prec):
    """chi0(i w) at several w, batched over frequencies (complex-shifted solves), incl. w = 0."""
    dV = synth.perturbations(cfg24.miller_rho, cfg24.L, 8, 2)
    oms = [0.35, 0.0, 4.0, 25.0]
    ref = chi0.sos_drho(model_of(cfg24), dV, oms)
    opt = dict(precision=W.WGW_FP64, cg_tol=1e-13) if prec == "fp64" else dict(precision=W.WGW_MIXED, cg_tol=1e-11)
    ctx = setup(W, cfg24, **opt)
    drho, st, _ = W.wgw_apply_chi0(ctx, dV, omega=oms)
    assert st["n_systems"] == 32 * len(oms)
    assert rel_err(drho.reshape(drho.shape[0], -1), ref.reshape(ref.shape[0], -1)) < (1e-10 if prec == "fp64" else 1e-8)


def test_imaginary_frequency_complex_perturbation(W, tiny):
    dV = synth.perturbations(tiny.miller_rho, tiny.L, 2, 13, hermitian=False)
    ref = chi0.sos_drho(model_of(tiny), dV, [0.7, 3.0])
    ctx = setup(W, tiny, cg_tol=1e-13)
    drho, st, _ = W.wgw_apply_chi0(ctx, dV, omega=[0.7, 3.0])
    assert rel_err(drho.reshape(drho.shape[0], -1), ref.reshape(ref.shape[0], -1)) < 1e-10


def test_gauss_legendre_frequency_batch(W, cfg24):
    """32 Gauss-Legendre frequencies on [0, 50 Ha] for 8 perturbations (1024 complex systems, mixed path)."""
    oms, _ = synth.gauss_legendre_omega(32, 50.0)
    phi = synth.perturbations(cfg24.miller_rho, cfg24.L, 8, 17)
    m = model_of(cfg24)
    ref = chi0.apply_chibar0(m, phi, oms)
    ctx = setup(W, cfg24, precision=W.WGW_MIXED, cg_tol=1e-11)
    import torch
    x = torch.from_numpy(np.ascontiguousarray(phi.T)).cuda()
    out = torch.zeros((32, 8, cfg24.n_rho), dtype=torch.complex128, device="cuda")
    st, _ = W.wgw_apply_chibar0_dev(ctx, x, oms, out)
    torch.cuda.synchronize()
    got = out.cpu().numpy().transpose(2, 1, 0)
    assert st["n_systems"] == 32 * 32 and st["n_converged"] == 32 * 32
    assert rel_err(got.reshape(got.shape[0], -1), ref.reshape(ref.shape[0], -1)) < 1e-8


@pytest.fixture(scope="module", params=["kb12", "kb24"])
def kbsys(request):
    if request.param == "kb12":
        cfg = synth.Config("kb12", L=6.0, ecut=2.5, grid=12, n_wells=2, well_seed=7, n_v=2, kb=True)
    else:
        cfg = synth.Config("kb24", L=10.0, ecut=5.0, grid=24, n_wells=4, well_seed=1, n_v=4, kb=True)
    return synth.make_system(cfg)


@pytest.mark.parametrize("prec", ["fp64", "mixed", "mixed_cuda_cores"])
def test_kb_projectors_match_sum_over_states(W, kbsys, prec):
    """H = T + V_loc + sum_p |beta_p> D_p <beta_p| (Kleinman-Bylander), static and at i w.  On the
    mixed path the KB products of the FP32 solves run on the tcgen05 tensor cores (default) or as
    CUDA-core GEMMs."""
    s = kbsys
    assert s.beta_G.shape[1] == 4 * s.cfg.n_wells
    dV = synth.perturbations(s.miller_rho, s.L, 3, 19)
    oms = [0.0, 0.6]
    ref = chi0.sos_drho(model_of(s), dV, oms)
    opt = dict(precision=W.WGW_FP64, cg_tol=1e-13) if prec == "fp64" else \
        dict(precision=W.WGW_MIXED, cg_tol=1e-11, tensor_cores=0 if prec == "mixed_cuda_cores" else 1)
    ctx = setup(W, s, **opt)
    drho, st, _ = W.wgw_apply_chi0(ctx, dV, omega=oms)
    assert rel_err(drho.reshape(drho.shape[0], -1), ref.reshape(ref.shape[0], -1)) < (1e-10 if prec == "fp64" else 1e-8)


def test_zero_and_empty_batches(W, tiny):
    ctx = setup(W, tiny)
    z = np.zeros((tiny.n_rho, 2), np.complex128)
    drho, st, _ = W.wgw_apply_chi0(ctx, z)
    assert np.all(drho == 0)
    drho, st, _ = W.wgw_apply_chi0(ctx, np.zeros((tiny.n_rho, 0), np.complex128))
    assert drho.shape == (tiny.n_rho, 0, 1)


def test_invalid_inputs_are_rejected(W, tiny):
    with pytest.raises(W.WgwError) as e:
        ctx = setup(W, tiny)
        W.wgw_apply_chi0(ctx, synth.perturbations(tiny.miller_rho, tiny.L, 1, 3), omega=[0.5, -0.5])
    assert e.value.status == W.WGW_ERR_ARG
    bad = tiny.psi_v.copy()
    bad[1, 0] += 0.3j          # no longer real in r
    with pytest.raises(W.WgwError) as e:
        W.wgw_setup(tiny.L, tiny.ecut, tiny.grid, tiny.vloc_G, bad, tiny.e_v)
    assert e.value.status == W.WGW_ERR_ARG
    with pytest.raises(W.WgwError) as e:
        W.wgw_setup(tiny.L, tiny.ecut, 6, tiny.vloc_G, tiny.psi_v, tiny.e_v)   # grid too small
    assert e.value.status == W.WGW_ERR_ARG


def test_static_response_matches_finite_differences(W, tiny):
    """Pins the GPU result to the derivative of the ground-state density (no response formula)."""
    dV = synth.perturbations(tiny.miller_rho, tiny.L, 1, 8)
    fd = chi0.finite_difference_drho(model_of(tiny), dV[:, 0], 1e-3)
    ctx = setup(W, tiny, cg_tol=1e-13)
    drho, _, _ = W.wgw_apply_chi0(ctx, dV)
    assert rel_err(drho[:, 0, 0][:, None], fd[:, None]) < 1e-9


@pytest.fixture(scope="module")
def cfg48():
    return synth.make_system("pdep_L16_48")


@pytest.mark.slow
def test_config48_full_batch_sampled_parity(W, cfg48):
    """The benchmarked workload (64 perturbations x 64 states, mixed path): eight perturbations
    spread over the batch (first, last and six between) against the oracle's sum over states."""
    import torch
    s = cfg48
    phi = synth.perturbations(s.miller_rho, s.L, 64, 5)
    ctx = setup(W, s, precision=W.WGW_MIXED, cg_tol=1e-10)
    x = torch.from_numpy(np.ascontiguousarray(phi.T)).cuda()
    out = torch.zeros((1, 64, s.n_rho), dtype=torch.complex128, device="cuda")
    st, _ = W.wgw_apply_chibar0_dev(ctx, x, [0.0], out)
    torch.cuda.synchronize()
    got = out.cpu().numpy().transpose(2, 1, 0)
    assert st["n_systems"] == 4096 and st["n_converged"] == 4096
    pick = [0, 9, 18, 27, 37, 45, 54, 63]
    m = model_of(s)
    ref = m.vsqrt[:, None] * chi0.sos_static_block(m, m.vsqrt[:, None] * phi[:, pick])
    assert rel_err(got[:, pick, 0], ref) < 1e-8


@pytest.mark.parametrize("kb", [False, True])
def test_apply_h_matches_oracle_and_eigenpairs(W, cfg24, kb):
    """H psi through wgw_apply_h_dev: random real-in-r vectors against the oracle's H (FP64
    accuracy 1e-12, FP32 kernels 1e-5 relative), and H psi_v = e_v psi_v on the given states."""
    import torch
    s = synth.make_system(synth.Config("kbd", L=6.0, ecut=2.5, grid=12, n_wells=2, well_seed=7, n_v=2,
                                       kb=True, kb_dch=True)) if kb else cfg24
    m = model_of(s)
    x = synth.perturbations(s.miller_wfc, s.L, 5, 72)
    ref = m.apply_h(x)
    ctx = setup(W, s, precision=W.WGW_MIXED)
    xd = torch.from_numpy(np.ascontiguousarray(x.T)).cuda()
    for fp32, tol in ((0, 1e-12), (1, 1e-5)):
        out = W.wgw_apply_h_dev(ctx, xd, fp32=bool(fp32)).cpu().numpy().T
        assert np.max(np.abs(out - ref)) < tol * np.max(np.abs(ref)), fp32
    pv = torch.from_numpy(np.ascontiguousarray(s.psi_v.T)).cuda()
    hv = W.wgw_apply_h_dev(ctx, pv).cpu().numpy().T
    assert np.max(np.abs(hv - s.psi_v * s.e_v[None, :])) < 1e-11 * np.max(np.abs(s.e_v))


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_cuda_graph_windows_give_identical_results(W, cfg24, ref24, prec):
    """The CG windows replayed as CUDA graphs launch the same kernels with the same arguments:
    bit-identical results with and without graphs (cuda_graphs 0 and 1).  The device-driven loop
    (cuda_graphs 2: windows and list compaction repeated by a conditional graph node) runs the same
    iterations on the same lists, with the K splits of the captured list: the same result to
    rounding (static and at an imaginary frequency).  Every variant within tolerance of the oracle."""
    dV, ref = ref24
    p = W.WGW_MIXED if prec == "mixed" else W.WGW_FP64
    tol = 1e-8 if prec == "mixed" else 1e-10
    outs = []
    for graphs in (0, 1, 2):
        ctx = setup(W, cfg24, precision=p, cg_tol=1e-11, check_every=3, cuda_graphs=graphs)
        drho, st, _ = W.wgw_apply_chi0(ctx, dV, [0.0, 0.7])
        outs.append(drho)
        assert st["n_converged"] == st["n_systems"]
        assert rel_err(drho[:, :, 0], ref[:, :, 0]) < tol
    assert np.array_equal(outs[0], outs[1])
    assert rel_err(outs[2].reshape(outs[2].shape[0], -1), outs[1].reshape(outs[1].shape[0], -1)) < tol


def test_autotuner_picks_a_candidate_and_results_stay_correct(W):
    """The tensor-core P_c K split is tuned at the first projection of >= 256 systems; the result
    of the apply is within tolerance whatever the choice."""
    s = synth.make_system(synth.Config("nv70", L=10.0, ecut=5.0, grid=24, n_wells=16, well_seed=1, n_v=70))
    dV = synth.perturbations(s.miller_rho, s.L, 4, 62)          # 280 systems
    ctx = setup(W, s, precision=W.WGW_MIXED, cg_tol=1e-11)
    assert W.wgw_autotune_info(ctx)["tc_split"] == 0
    drho, st, _ = W.wgw_apply_chi0(ctx, dV)
    info = W.wgw_autotune_info(ctx)
    assert info["tc_split"] in (2, 4, 8, 16)
    assert sorted(info["candidates_ms"]) == [2, 4, 8, 16]
    assert all(t > 0 for t in info["candidates_ms"].values())
    # The FP32 H kernel is tuned on the same first large list: both variants timed, one chosen.
    assert info["h_kernel"] in ("three kernels", "fused")
    assert info["h_ms"]["three_kernels"] > 0 and info["h_ms"]["fused"] > 0
    ref = chi0.sos_drho(model_of(s), dV, [0.0])
    assert rel_err(drho, ref) < 1e-8


@pytest.mark.parametrize("fused", [0, 1])
def test_fixed_tuning_choices_are_bit_identical_across_contexts(W, fused):
    """With the autotuned choices fixed (H kernel, tensor-core K split, FFT stage kernels) two
    contexts give bit-identical results for the same batch."""
    s = synth.make_system(synth.Config("nv70", L=10.0, ecut=5.0, grid=24, n_wells=16, well_seed=1, n_v=70))
    dV = synth.perturbations(s.miller_rho, s.L, 4, 63)
    outs = []
    for _ in range(2):
        ctx = setup(W, s, precision=W.WGW_MIXED, cg_tol=1e-11, fused_h=fused, tc_split=4, fft_kernels=(0, 1, 1))
        drho, st, _ = W.wgw_apply_chi0(ctx, dV, [0.0, 0.4])
        outs.append(drho)
        info = W.wgw_autotune_info(ctx)
        assert info["tc_split"] == 4 and info["h_kernel"] == "untuned"
    assert np.array_equal(outs[0], outs[1])
