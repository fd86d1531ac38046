"""The fused FP32 H application (one kernel per pair, the FFT intermediate in distributed shared
memory) against the three-kernel pipeline it replaces and the oracle.

Both run the same butterflies on the same data; the compiler contracts multiplies and adds into
FMAs differently in the two codes, so the results agree to FP32 rounding rather than bit for
bit.  Checked on every grid the fused kernel takes (24^3 in one CTA per pair, 32^3 in one CTA,
48^3 in a cluster of two CTAs), on the active-list launches of the CG (odd system counts, ragged
pairs): H psi within 1e-5 of the largest element of the three-kernel result and of the oracle's
H, and whole mixed-path chi0 applies within the path's 1e-8 of each other and of the oracle.
"""
import numpy as np
import pytest

import synth

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


MODELS = {
    24: "chi0_L10_24",
    32: synth.Config("g32", L=32.0 / 3.0, ecut=9.0, grid=32, n_wells=8, well_seed=3, n_v=16, kb=True),
    48: "pdep_L16_48",
}


@pytest.fixture(scope="module", params=sorted(MODELS))
def model(request):
    return synth.make_system(MODELS[request.param])


def _ctx(W, s, fused):
    kb = s.beta_G.shape[1] > 0
    return W.wgw_setup(s.L, s.ecut, s.grid, s.vloc_G, s.psi_v, s.e_v,
                       W.wgw_default_options(precision=W.WGW_MIXED, cg_tol=1e-10, fused_h=fused),
                       beta_G=s.beta_G if kb else None, d_proj=s.d_proj if kb else None)


def _model(s):
    from oracle.model import Model
    return Model(s.L, s.ecut, s.grid, s.vloc_G, s.psi_v, s.e_v, s.beta_G, s.d_proj)


def test_fused_h_matches_three_kernels_and_oracle(W, model):
    import torch
    s = model
    x = synth.perturbations(s.miller_wfc, s.L, 7, 91)      # 7 vectors: the last pair is half empty
    xd = torch.from_numpy(np.ascontiguousarray(x.T)).cuda()
    outs = [W.wgw_apply_h_dev(_ctx(W, s, f), xd, fp32=True).cpu().numpy() for f in (0, 1)]
    scale = np.max(np.abs(outs[0]))
    assert np.max(np.abs(outs[1] - outs[0])) < 1e-5 * scale
    ref = _model(s).apply_h(x).T
    assert np.max(np.abs(outs[1] - ref)) < 1e-5 * np.max(np.abs(ref))


def test_fused_chi0_apply_matches_three_kernels_and_oracle(W, model):
    from oracle import chi0
    s = model
    dV = synth.perturbations(s.miller_rho, s.L, 3, 92)
    outs = []
    for f in (0, 1):
        drho, st, _ = W.wgw_apply_chi0(_ctx(W, s, f), dV, [0.0, 0.5])
        assert st["n_converged"] == st["n_systems"]
        outs.append(drho.reshape(drho.shape[0], -1))

    def rel(a, b):
        return float(np.max(np.linalg.norm(a - b, axis=0) / np.linalg.norm(b, axis=0)))

    assert rel(outs[1], outs[0]) < 1e-8
    if s.n_pw < 5000:
        ref = chi0.sos_drho(_model(s), dV, [0.0, 0.5])
        assert rel(outs[1], ref.reshape(ref.shape[0], -1)) < 1e-8
