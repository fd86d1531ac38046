"""Serving entry points (wgw_submit / wgw_poll / wgw_wait) on a GB300.

Requests queued on one context are merged into batched applies; each request's
result must equal the oracle's within the path's tolerance (FP64 1e-10) and
its own synchronous wgw_apply_chi0 result, whatever it was batched with.
"""
import threading

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
    num = np.linalg.norm(got - ref, axis=0)
    den = np.linalg.norm(ref, axis=0)
    return float(np.max(num / np.where(den > 0, den, 1.0)))


def ctx_of(W, s):
    return W.wgw_setup(s.L, s.ecut, s.grid, s.vloc_G, s.psi_v, s.e_v,
                       W.wgw_default_options(precision=W.WGW_FP64, cg_tol=1e-13))


def test_queued_requests_match_oracle_and_sync(W, cfg24):
    s = cfg24
    ctx = ctx_of(W, s)
    m = model_of(s)
    # Ten requests of 1..4 perturbations: two frequency sets, so the worker forms separate batches.
    reqs = []
    for k in range(10):
        dV = synth.perturbations(s.miller_rho, s.L, 1 + k % 4, 100 + k)
        om = [0.0] if k % 3 else [0.0, 0.4]
        reqs.append((dV, om))
    tickets = [None] * len(reqs)

    def submit(i):
        tickets[i] = W.wgw_submit(ctx, *reqs[i])

    th = [threading.Thread(target=submit, args=(i,)) for i in range(len(reqs))]
    for t in th:
        t.start()
    for t in th:
        t.join()
    merged = 0
    for (dV, om), t in zip(reqs, tickets):
        got, res = W.wgw_wait(t)
        assert res["status"] == W.WGW_OK
        assert res["latency_s"] >= res["queue_s"] >= 0
        merged = max(merged, res["batch_requests"])
        ref = chi0.sos_drho(m, dV, om)
        assert rel_err(got, ref) < 1e-10
        alone, _, _ = W.wgw_apply_chi0(ctx, dV, om)
        assert rel_err(got, alone) < 1e-10
    assert merged >= 1


def test_queued_requests_mixed_path_alone_and_in_the_mix(W, cfg24):
    """Mixed path (FP32 inner CG on the tensor-core projector, float-float refinement): each
    request's result in a merged batch equals the oracle and its own result alone within the
    path's tolerance 1e-8, although the batch composition changes the list compaction and the
    projector's K split."""
    s = cfg24
    ctx = W.wgw_setup(s.L, s.ecut, s.grid, s.vloc_G, s.psi_v, s.e_v,
                      W.wgw_default_options(precision=W.WGW_MIXED, cg_tol=1e-11))
    m = model_of(s)
    reqs = [(synth.perturbations(s.miller_rho, s.L, 2 + k % 3, 200 + k), [0.0] if k % 2 else [0.0, 0.6])
            for k in range(8)]
    alone = [W.wgw_apply_chi0(ctx, dV, om)[0] for dV, om in reqs]
    tickets = [W.wgw_submit(ctx, dV, om) for dV, om in reqs]
    merged = 0
    for (dV, om), t, a in zip(reqs, tickets, alone):
        got, res = W.wgw_wait(t)
        assert res["status"] == W.WGW_OK
        merged = max(merged, res["batch_requests"])
        assert rel_err(got, chi0.sos_drho(m, dV, om)) < 1e-8
        assert rel_err(got, a) < 1e-8
    assert merged >= 2


def test_two_contexts_overlap_and_poll(W, cfg24, tiny):
    c1, c2 = ctx_of(W, cfg24), ctx_of(W, tiny)
    d1 = synth.perturbations(cfg24.miller_rho, cfg24.L, 3, 7)
    d2 = synth.perturbations(tiny.miller_rho, tiny.L, 2, 8)
    t1 = W.wgw_submit(c1, d1, [0.0, 0.3])
    t2 = W.wgw_submit(c2, d2, [0.0], kind=W.WGW_REQ_CHIBAR0)
    import time
    done2 = False
    for _ in range(6000):
        done2, res2 = W.wgw_poll(t2)
        if done2:
            break
        time.sleep(0.005)
    assert done2 and res2["status"] == W.WGW_OK
    got1, res1 = W.wgw_wait(t1)
    assert res1["status"] == W.WGW_OK
    assert rel_err(got1, chi0.sos_drho(model_of(cfg24), d1, [0.0, 0.3])) < 1e-10
    ref2, _, _ = W.wgw_apply_chibar0(c2, d2, [0.0])
    assert rel_err(t2.out.transpose(2, 1, 0), ref2) < 1e-10
    # A released ticket is unknown afterwards.
    with pytest.raises(W.WgwError):
        W.wgw_poll(t2)


def test_submit_rejects_bad_requests(W, tiny):
    ctx = ctx_of(W, tiny)
    d = synth.perturbations(tiny.miller_rho, tiny.L, 1, 3)
    with pytest.raises(W.WgwError):
        W.wgw_submit(ctx, d, [-0.1])
    with pytest.raises(W.WgwError):
        W.wgw_submit(ctx, d, [0.0], kind=7)


def test_continuous_batching_admits_requests_into_running_cg(W):
    """Mixed path, static requests: a request submitted while a long one is on the GPU is admitted
    at the next CG window (its queueing time is a fraction of the long request's run), the two share
    the slot pool, and each result equals the oracle and its own result alone within 1e-8."""
    import time
    s = synth.make_system("pdep_L16_48")
    ctx = W.wgw_setup(s.L, s.ecut, s.grid, s.vloc_G, s.psi_v, s.e_v,
                      W.wgw_default_options(precision=W.WGW_MIXED, cg_tol=1e-10))
    m = model_of(s)
    big = synth.perturbations(s.miller_rho, s.L, 16, 301)
    small = synth.perturbations(s.miller_rho, s.L, 2, 302)
    alone_small, _, _ = W.wgw_apply_chi0(ctx, small)
    t_big = W.wgw_submit(ctx, big, [0.0])
    time.sleep(0.02)                              # the big request is on the GPU
    t_small = W.wgw_submit(ctx, small, [0.0])
    got_small, r_small = W.wgw_wait(t_small)
    got_big, r_big = W.wgw_wait(t_big)
    assert r_small["status"] == W.WGW_OK and r_big["status"] == W.WGW_OK
    assert r_small["batch_requests"] >= 2 and r_big["batch_requests"] >= 2
    assert r_small["queue_s"] < 0.5 * r_big["latency_s"], (r_small, r_big)
    assert r_small["batch_systems"] == 2 * s.n_v and r_big["batch_systems"] == 16 * s.n_v
    assert rel_err(got_small, alone_small) < 1e-8
    states = chi0._states(m)
    ref_small = chi0.sos_static_block(m, small, states)
    assert rel_err(got_small[:, :, 0], ref_small) < 1e-8
    ref_big = chi0.sos_static_block(m, big[:, :4], states)
    assert rel_err(got_big[:, :4, 0], ref_big) < 1e-8


def test_continuous_batching_cancel_running_request(W, cfg24):
    """A running request of the continuous engine is dropped at the next window when cancelled;
    the requests around it are served normally."""
    s = cfg24
    ctx = W.wgw_setup(s.L, s.ecut, s.grid, s.vloc_G, s.psi_v, s.e_v,
                      W.wgw_default_options(precision=W.WGW_MIXED, cg_tol=1e-11))
    a = synth.perturbations(s.miller_rho, s.L, 4, 311)
    b = synth.perturbations(s.miller_rho, s.L, 4, 312)
    ta = W.wgw_submit(ctx, a, [0.0])
    tb = W.wgw_submit(ctx, b, [0.0])
    W.wgw_cancel(ta)
    got_a, ra = W.wgw_wait(ta)
    got_b, rb = W.wgw_wait(tb)
    assert ra["status"] == W.WGW_ERR_CANCELLED and np.all(got_a == 0)
    assert rb["status"] == W.WGW_OK
    alone_b, _, _ = W.wgw_apply_chi0(ctx, b)
    assert rel_err(got_b, alone_b) < 1e-8


def test_served_pdep_request_with_chibar0_requests(W, cfg24):
    """A PDEP Davidson submitted to the queue (its chibar0 block applications are queued requests,
    batched with whatever else is served) beside chibar0 requests: the eigenpairs equal the dense
    PDEP oracle's and the synchronous Davidson's within the mixed path's 1e-8, and every chibar0
    request equals its result alone."""
    from oracle import pdep
    s = cfg24
    ctx = W.wgw_setup(s.L, s.ecut, s.grid, s.vloc_G, s.psi_v, s.e_v,
                      W.wgw_default_options(precision=W.WGW_MIXED, cg_tol=1e-11, dav_tol=1e-11))
    n_pdep = 8
    x0 = synth.perturbations(s.miller_rho, s.L, n_pdep, 11)
    reqs = [synth.perturbations(s.miller_rho, s.L, 1 + k % 3, 320 + k) for k in range(6)]
    t_pdep = W.wgw_submit_pdep(ctx, n_pdep, x0)
    tickets = [W.wgw_submit(ctx, dV, [0.0], kind=W.WGW_REQ_CHIBAR0) for dV in reqs]
    (eig, basis), r = W.wgw_wait(t_pdep)
    assert r["status"] == W.WGW_OK, r
    assert r["batch_requests"] >= 2 and r["batch_systems"] >= n_pdep * s.n_v
    w_ref, U_ref = pdep.pdep_dense(model_of(s), 16)
    assert np.max(np.abs(eig - w_ref[:n_pdep]) / np.abs(w_ref[:n_pdep])) < 1e-8
    assert np.max(np.abs(basis.conj().T @ basis - np.eye(n_pdep))) < 1e-10
    if abs(w_ref[n_pdep] - w_ref[n_pdep - 1]) > 1e-6:
        sv = np.linalg.svd(U_ref[:, :n_pdep].conj().T @ basis, compute_uv=False)
        assert np.min(sv) > 1 - 1e-7
    eig_sync, _, _, _ = W.wgw_pdep_davidson(ctx, n_pdep, x0, want_basis=False)
    assert np.max(np.abs(eig - eig_sync) / np.abs(eig_sync)) < 1e-8
    for dV, t in zip(reqs, tickets):
        got, rr = W.wgw_wait(t)
        assert rr["status"] == W.WGW_OK
        alone, _, _ = W.wgw_apply_chibar0(ctx, dV)
        assert rel_err(got, alone) < 1e-8


def test_served_pdep_cancel_and_bad_request(W, cfg24):
    """A running PDEP request stops at its next block application when cancelled; one asking for
    more eigenpairs than the Davidson subspace holds is refused at submission."""
    s = cfg24
    ctx = W.wgw_setup(s.L, s.ecut, s.grid, s.vloc_G, s.psi_v, s.e_v,
                      W.wgw_default_options(precision=W.WGW_MIXED, cg_tol=1e-11, dav_tol=1e-11))
    t = W.wgw_submit_pdep(ctx, 8)
    W.wgw_cancel(t)
    _, r = W.wgw_wait(t)
    assert r["status"] == W.WGW_ERR_CANCELLED
    with pytest.raises(RuntimeError):
        W.wgw_submit_pdep(ctx, 4096)
    dV = synth.perturbations(s.miller_rho, s.L, 2, 330)
    got, rr = W.wgw_wait(W.wgw_submit(ctx, dV, [0.0]))
    alone, _, _ = W.wgw_apply_chi0(ctx, dV)
    assert rr["status"] == W.WGW_OK and rel_err(got, alone) < 1e-8


def test_mixed_grid_stream_of_chibar0_and_pdep_requests(W, cfg24):
    """The served mixed stream at test size: contexts on a 24^3 and a 32^3 system (the 32^3 one of
    the served-stream recipe: 8 deep wells, 32 states, 7 KB atoms), chibar0 and PDEP requests
    submitted from several threads and interleaved across the two.  Each chibar0 result equals its
    result alone and the oracle's sum over states within 1e-8; each PDEP request's eigenvalues
    equal the synchronous Davidson's within 1e-8 (and the dense PDEP oracle's on 24^3)."""
    from oracle import pdep
    s32 = synth.make_system(synth.serve_stream_configs()[0])
    assert s32.grid == 32 and s32.beta_G.shape[1] == 28
    opt = W.wgw_default_options(precision=W.WGW_MIXED, cg_tol=1e-11, dav_tol=1e-11)
    sy = {24: cfg24, 32: s32}
    ctx = {g: W.wgw_setup(s.L, s.ecut, s.grid, s.vloc_G, s.psi_v, s.e_v, opt,
                          beta_G=s.beta_G if s.beta_G.shape[1] else None,
                          d_proj=s.d_proj if s.beta_G.shape[1] else None) for g, s in sy.items()}
    plan = []
    for k in range(8):
        g = (24, 32)[k % 2]
        if k in (2, 5):
            plan.append(("pdep", g, 4, synth.perturbations(sy[g].miller_rho, sy[g].L, 4, 340 + k)))
        else:
            plan.append(("chibar0", g, 0, synth.perturbations(sy[g].miller_rho, sy[g].L, 1 + k % 3, 340 + k)))
    tickets = [None] * len(plan)

    def submit(i):
        kind, g, n, x = plan[i]
        tickets[i] = W.wgw_submit_pdep(ctx[g], n, x) if kind == "pdep" else \
            W.wgw_submit(ctx[g], x, [0.0], kind=W.WGW_REQ_CHIBAR0)

    th = [threading.Thread(target=submit, args=(i,)) for i in range(len(plan))]
    for t in th:
        t.start()
    for t in th:
        t.join()
    results = [W.wgw_wait(t) for t in tickets]
    dense24 = pdep.pdep_dense(model_of(cfg24), 8)[0]
    states = {g: chi0._states(model_of(s)) for g, s in sy.items()}
    for (kind, g, n, x), (out, r) in zip(plan, results):
        assert r["status"] == W.WGW_OK, (kind, g, r.get("error"))
        if kind == "pdep":
            eig, basis = out
            eig_sync, _, _, _ = W.wgw_pdep_davidson(ctx[g], n, x, want_basis=False)
            assert np.max(np.abs(eig - eig_sync) / np.abs(eig_sync)) < 1e-8
            assert np.max(np.abs(basis.conj().T @ basis - np.eye(n))) < 1e-10
            if g == 24:
                assert np.max(np.abs(eig - dense24[:n]) / np.abs(dense24[:n])) < 1e-8
        else:
            alone, _, _ = W.wgw_apply_chibar0(ctx[g], x)
            assert rel_err(out, alone) < 1e-8
            m = model_of(sy[g])
            ref = m.vsqrt[:, None] * chi0.sos_static_block(m, m.vsqrt[:, None] * x, states[g])
            assert rel_err(out[:, :, 0], ref) < 1e-8
