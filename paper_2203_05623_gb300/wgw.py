"""ctypes binding of libwgw (include/wgw.h): argument marshalling only.

Every step of the response calculation runs in the library's CUDA kernels;
this module converts numpy / torch arrays to the C layouts (interleaved
complex, column-major per perturbation) and raises WgwError on failure.  It
never computes a result itself and fails loudly when libwgw.so is missing.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

WGW_OK, WGW_ERR_ARG, WGW_ERR_NOMEM, WGW_ERR_NOCONV = 0, 1, 2, 3
WGW_ERR_CUDA, WGW_ERR_TIMEOUT, WGW_ERR_STATE, WGW_ERR_CANCELLED = 4, 5, 6, 7
WGW_FP64, WGW_MIXED = 0, 1
WGW_SPHERE_WFC, WGW_SPHERE_RHO = 0, 1
WGW_REQ_CHI0, WGW_REQ_CHIBAR0, WGW_REQ_PDEP = 0, 1, 2
WGW_PROF_KINDS = 18

_dp = ctypes.POINTER(ctypes.c_double)


class WgwError(RuntimeError):
    def __init__(self, status: int, where: str, msg: str):
        super().__init__(f"{where}: status {status} ({msg})")
        self.status = status


class Options(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int), ("cg_tol", ctypes.c_double),
                ("max_cg_iter", ctypes.c_int), ("max_refine", ctypes.c_int),
                ("inner_tol", ctypes.c_double), ("f_s", ctypes.c_double),
                ("check_every", ctypes.c_int), ("dav_tol", ctypes.c_double),
                ("dav_max_iter", ctypes.c_int), ("dav_factor", ctypes.c_int), ("seed", ctypes.c_int),
                ("fp64_emulation", ctypes.c_int), ("tensor_cores", ctypes.c_int), ("cuda_graphs", ctypes.c_int),
                ("max_batch_systems", ctypes.c_int), ("fused_h", ctypes.c_int),
                ("tc_split", ctypes.c_int), ("fft_kernels", ctypes.c_int * 3), ("h_chunk_pairs", ctypes.c_int)]


class SigmaParams(ctypes.Structure):
    _fields_ = [("n_steps_chi", ctypes.c_int), ("n_steps_g0", ctypes.c_int), ("nodes", _dp), ("weights", _dp),
                ("n_nodes", ctypes.c_int), ("e_fermi", ctypes.c_double), ("eta", ctypes.c_double)]


class Stats(ctypes.Structure):
    _fields_ = [("n_systems", ctypes.c_int), ("n_converged", ctypes.c_int),
                ("max_iters", ctypes.c_int), ("refinements", ctypes.c_int),
                ("max_rel_residual", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class Request(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("dV", _dp), ("n_pert", ctypes.c_int), ("omega", _dp),
                ("n_omega", ctypes.c_int), ("out", _dp)]


class Result(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("latency_s", ctypes.c_double), ("queue_s", ctypes.c_double),
                ("batch_requests", ctypes.c_int), ("batch_systems", ctypes.c_int)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_lib = None


def lib(path: str | None = None):
    """The loaded libwgw.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or _build.LIB
    if not os.path.exists(path):
        raise RuntimeError(f"libwgw.so not found at {path}: run paper_2203_05623_gb300.build.build() "
                           "(the CUDA library is required; there is no other execution path)")
    L = ctypes.CDLL(path)
    L.wgw_default_options.argtypes = [ctypes.POINTER(Options)]
    L.wgw_setup.argtypes = [ctypes.POINTER(ctypes.c_void_p), ctypes.c_double, ctypes.c_double,
                            ctypes.c_int, _dp, ctypes.c_int, _dp, _dp, _dp, _dp, ctypes.c_int,
                            ctypes.POINTER(Options)]
    L.wgw_sphere_size.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(ctypes.c_int)]
    L.wgw_get_gvectors.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(ctypes.c_int32)]
    L.wgw_set_options.argtypes = [ctypes.c_void_p, ctypes.POINTER(Options)]
    L.wgw_apply_chi0.argtypes = [ctypes.c_void_p, _dp, ctypes.c_int, _dp, ctypes.c_int, _dp,
                                 ctypes.POINTER(Stats)]
    L.wgw_apply_chi0_dev.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, _dp,
                                     ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p,
                                     ctypes.POINTER(Stats)]
    L.wgw_apply_chibar0_dev.argtypes = L.wgw_apply_chi0_dev.argtypes
    L.wgw_apply_chibar0.argtypes = L.wgw_apply_chi0.argtypes
    L.wgw_profile_enable.argtypes = [ctypes.c_void_p, ctypes.c_int]
    L.wgw_profile_classes.argtypes = [ctypes.c_void_p, ctypes.c_uint]
    L.wgw_profile_read.argtypes = [ctypes.c_void_p, ctypes.c_int, _dp, ctypes.POINTER(ctypes.c_long), _dp, _dp]
    L.wgw_profile_kind_name.restype = ctypes.c_char_p
    L.wgw_profile_kind_name.argtypes = [ctypes.c_int]
    L.wgw_pdep_davidson.argtypes = [ctypes.c_void_p, ctypes.c_int, _dp, _dp, _dp, ctypes.POINTER(Stats)]
    L.wgw_symm_eig_dev.argtypes = [ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    L.wgw_symm_eig_noalloc_dev.argtypes = L.wgw_symm_eig_dev.argtypes
    L.wgw_lanczos.argtypes = [ctypes.c_void_p, _dp, ctypes.c_int, ctypes.c_int, _dp, ctypes.c_int, _dp, _dp, _dp,
                              ctypes.POINTER(Stats)]
    L.wgw_system_info.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(ctypes.c_int), _dp,
                                  ctypes.POINTER(ctypes.c_int)]
    L.wgw_cancel.argtypes = [ctypes.c_void_p, ctypes.c_uint64]
    L.wgw_sample_solutions.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(ctypes.c_int)]
    L.wgw_read_samples.argtypes = [ctypes.c_void_p, ctypes.c_int, _dp]
    L.wgw_submit.argtypes = [ctypes.c_void_p, ctypes.POINTER(Request), ctypes.POINTER(ctypes.c_uint64)]
    L.wgw_poll.argtypes = [ctypes.c_void_p, ctypes.c_uint64, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(Result)]
    L.wgw_wait.argtypes = [ctypes.c_void_p, ctypes.c_uint64, ctypes.POINTER(Result)]
    L.wgw_dyson.argtypes = [ctypes.c_int, ctypes.c_int, _dp, _dp]
    L.wgw_pdep_davidson_channels.argtypes = [ctypes.POINTER(ctypes.c_void_p), ctypes.c_int, ctypes.c_int, _dp, _dp,
                                             _dp, ctypes.POINTER(Stats)]
    L.wgw_apply_h_dev.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_int,
                                  ctypes.c_void_p]
    L.wgw_isr.argtypes = [ctypes.c_void_p, _dp, ctypes.c_int, ctypes.POINTER(ctypes.c_int), ctypes.c_int, ctypes.c_int,
                          _dp, ctypes.c_int, _dp, _dp, _dp, ctypes.c_int, _dp, ctypes.POINTER(Stats)]
    L.wgw_sigma_x.argtypes = [ctypes.c_void_p, ctypes.POINTER(ctypes.c_int), ctypes.c_int, _dp]
    L.wgw_lanczos_z.argtypes = [ctypes.c_void_p, _dp, ctypes.c_int, ctypes.c_int, _dp, ctypes.c_int, _dp, _dp,
                                ctypes.POINTER(Stats)]
    L.wgw_sigma.argtypes = [ctypes.c_void_p, _dp, ctypes.c_int, ctypes.POINTER(ctypes.c_int), ctypes.c_int,
                            ctypes.POINTER(SigmaParams), _dp, ctypes.c_int, _dp, _dp, _dp, ctypes.POINTER(Stats)]
    L.wgw_qp.argtypes = [ctypes.c_void_p, _dp, ctypes.c_int, ctypes.POINTER(ctypes.c_int), ctypes.c_int,
                         ctypes.POINTER(SigmaParams), _dp, ctypes.c_double, ctypes.c_int, _dp, _dp,
                         ctypes.POINTER(ctypes.c_int), ctypes.POINTER(Stats)]
    L.wgw_autotune_info.argtypes = [ctypes.c_void_p, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                                    _dp, ctypes.c_int, ctypes.POINTER(ctypes.c_int), _dp]
    L.wgw_selftest_wait_timeout.argtypes = [ctypes.POINTER(ctypes.c_int)]
    L.wgw_autotune_fft.argtypes = [ctypes.c_void_p, ctypes.POINTER(ctypes.c_int), _dp]
    L.wgw_autotune_chunk.argtypes = [ctypes.c_void_p, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                                     _dp, ctypes.c_int]
    L.wgw_apply_channels.argtypes = [ctypes.POINTER(ctypes.c_void_p), ctypes.c_int, ctypes.c_int, _dp, ctypes.c_int,
                                     _dp, ctypes.c_int, _dp, ctypes.POINTER(Stats)]
    L.wgw_g0_lanczos.argtypes = [ctypes.c_void_p, _dp, ctypes.c_int, ctypes.POINTER(ctypes.c_int), ctypes.c_int,
                                 ctypes.c_int, _dp, ctypes.c_int, _dp, _dp, _dp, _dp, _dp, ctypes.POINTER(Stats)]
    L.wgw_destroy.argtypes = [ctypes.c_void_p]
    L.wgw_status_string.restype = ctypes.c_char_p
    L.wgw_status_string.argtypes = [ctypes.c_int]
    L.wgw_last_error.restype = ctypes.c_char_p
    _lib = L
    return L


def _check(status: int, where: str, allow=(WGW_OK,)):
    if status not in allow:
        raise WgwError(status, where, lib().wgw_last_error().decode())
    return status


def _interleave(a: np.ndarray) -> np.ndarray:
    """Complex array -> contiguous float64 (re, im) with the first axis fastest after re/im."""
    a = np.asarray(a, np.complex128)
    return np.ascontiguousarray(a.T).view(np.float64).ravel()


def wgw_default_options(**overrides) -> Options:
    o = Options()
    _check(lib().wgw_default_options(ctypes.byref(o)), "wgw_default_options")
    for k, v in overrides.items():
        if k == "fft_kernels":
            v = (ctypes.c_int * 3)(*[int(x) for x in v])
        setattr(o, k, v)
    return o


class Context:
    """Owner of a wgw_ctx*; destroyed with wgw_destroy."""

    def __init__(self, handle, n_pw, n_rho, n_v):
        self.handle, self.n_pw, self.n_rho, self.n_v = handle, n_pw, n_rho, n_v

    def __del__(self):
        if getattr(self, "handle", None):
            wgw_destroy(self)


def wgw_setup(L, ecut, grid, vloc_G, psi_v, e_v, opt: Options | None = None, beta_G=None,
              d_proj=None) -> Context:
    psi_v = np.asarray(psi_v, np.complex128)
    n_v = psi_v.shape[1]
    v = _interleave(vloc_G)
    ps = _interleave(psi_v)
    ev = np.ascontiguousarray(e_v, np.float64)
    n_proj = 0 if beta_G is None else np.asarray(beta_G).shape[1]
    bg = _interleave(beta_G) if n_proj else None
    dp = np.ascontiguousarray(d_proj, np.float64) if n_proj else None
    h = ctypes.c_void_p()
    _check(lib().wgw_setup(ctypes.byref(h), float(L), float(ecut), int(grid), v.ctypes.data_as(_dp),
                           n_proj, bg.ctypes.data_as(_dp) if n_proj else None,
                           dp.ctypes.data_as(_dp) if n_proj else None, ps.ctypes.data_as(_dp),
                           ev.ctypes.data_as(_dp), n_v, ctypes.byref(opt) if opt else None),
           "wgw_setup")
    n_pw, n_rho = ctypes.c_int(), ctypes.c_int()
    lib().wgw_sphere_size(h, WGW_SPHERE_WFC, ctypes.byref(n_pw))
    lib().wgw_sphere_size(h, WGW_SPHERE_RHO, ctypes.byref(n_rho))
    return Context(h, n_pw.value, n_rho.value, n_v)


def wgw_sphere_size(ctx: Context, which: int) -> int:
    n = ctypes.c_int()
    _check(lib().wgw_sphere_size(ctx.handle, which, ctypes.byref(n)), "wgw_sphere_size")
    return n.value


def wgw_get_gvectors(ctx: Context, which: int) -> np.ndarray:
    n = wgw_sphere_size(ctx, which)
    out = np.zeros((n, 3), np.int32)
    _check(lib().wgw_get_gvectors(ctx.handle, which, out.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))),
           "wgw_get_gvectors")
    return out


def wgw_set_options(ctx: Context, opt: Options):
    _check(lib().wgw_set_options(ctx.handle, ctypes.byref(opt)), "wgw_set_options")


def _host_call(fn, name, ctx, dV, omega, allow_noconv, out=None):
    dV = np.asarray(dV, np.complex128)
    dV = dV[:, None] if dV.ndim == 1 else dV
    n_pert = dV.shape[1]
    om = np.ascontiguousarray(omega, np.float64)
    buf = _interleave(dV)
    if out is None:
        out = np.zeros((len(om), n_pert, ctx.n_rho), np.complex128)
    st = Stats()
    s = fn(ctx.handle, buf.ctypes.data_as(_dp), n_pert, om.ctypes.data_as(_dp), len(om),
           out.view(np.float64).ctypes.data_as(_dp), ctypes.byref(st))
    _check(s, name, (WGW_OK, WGW_ERR_NOCONV) if allow_noconv else (WGW_OK,))
    return out.transpose(2, 1, 0), st.as_dict(), s


def wgw_apply_chi0(ctx: Context, dV, omega=(0.0,), allow_noconv=False, out=None):
    """Host arrays: dV (N_rho, n_pert) complex -> (drho (N_rho, n_pert, n_omega), stats dict, status).

    `out`, if given, is a C-contiguous complex128 array of shape (n_omega, n_pert, N_rho)
    (for example pinned host memory) that receives the result."""
    return _host_call(lib().wgw_apply_chi0, "wgw_apply_chi0", ctx, dV, omega, allow_noconv, out)


def wgw_apply_chibar0(ctx: Context, phi, omega=(0.0,), allow_noconv=False, out=None):
    """Host arrays: chibar0 phi = v^1/2 chi0 v^1/2 phi; layout as wgw_apply_chi0."""
    return _host_call(lib().wgw_apply_chibar0, "wgw_apply_chibar0", ctx, phi, omega, allow_noconv, out)


def wgw_apply_channels(ctxs, dV, omega=(0.0,), symmetrized=False, allow_noconv=False):
    """Spin-polarised response: the sum over the channels (one context each, normally f_s = 1)
    of chi0 dV (or chibar0 phi with symmetrized=True); layout as wgw_apply_chi0."""
    ctxs = list(ctxs)
    dV = np.asarray(dV, np.complex128)
    dV = dV[:, None] if dV.ndim == 1 else dV
    n_pert = dV.shape[1]
    om = np.ascontiguousarray(omega, np.float64)
    buf = _interleave(dV)
    out = np.zeros((len(om), n_pert, ctxs[0].n_rho), np.complex128)
    handles = (ctypes.c_void_p * len(ctxs))(*[c.handle for c in ctxs])
    st = Stats()
    s = lib().wgw_apply_channels(handles, len(ctxs), 1 if symmetrized else 0, buf.ctypes.data_as(_dp), n_pert,
                                 om.ctypes.data_as(_dp), len(om), out.view(np.float64).ctypes.data_as(_dp),
                                 ctypes.byref(st))
    _check(s, "wgw_apply_channels", (WGW_OK, WGW_ERR_NOCONV) if allow_noconv else (WGW_OK,))
    return out.transpose(2, 1, 0), st.as_dict(), s


def wgw_apply_h_dev(ctx: Context, psi_dev, out_dev=None, fp32=False, stream=None):
    """H psi on device: psi_dev a torch complex128 tensor (n_psi, N_pw) (row = one wavefunction,
    canonical order); returns out_dev of the same shape."""
    import torch
    assert psi_dev.is_cuda and psi_dev.dtype == torch.complex128 and psi_dev.is_contiguous()
    n_psi = psi_dev.shape[0]
    if out_dev is None:
        out_dev = torch.empty_like(psi_dev)
    if stream is None:
        stream = torch.cuda.current_stream(psi_dev.device).cuda_stream
    _check(lib().wgw_apply_h_dev(ctx.handle, ctypes.c_void_p(psi_dev.data_ptr()), n_psi,
                                 ctypes.c_void_p(out_dev.data_ptr()), 1 if fp32 else 0,
                                 ctypes.c_void_p(stream)), "wgw_apply_h_dev")
    return out_dev


def wgw_isr(ctx: Context, phi, states, n_steps: int, omega, lam, nodes, weights) -> np.ndarray:
    """I^SR_i(w) of Eq. ISR by quadrature; returns (n_states, n_omega) complex."""
    phi = np.asarray(phi, np.complex128)
    npd = phi.shape[1]
    sts = np.ascontiguousarray(states, np.int32)
    om = np.ascontiguousarray(omega, np.float64)
    lm = np.ascontiguousarray(lam, np.float64)
    nd = np.ascontiguousarray(nodes, np.float64)
    wt = np.ascontiguousarray(weights, np.float64)
    assert lm.shape == (nd.size, npd, npd) and wt.size == nd.size
    out = np.zeros((sts.size, om.size), np.complex128)
    st = Stats()
    pb = _interleave(phi)
    _check(lib().wgw_isr(ctx.handle, pb.ctypes.data_as(_dp), npd, sts.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
                         sts.size, n_steps, om.ctypes.data_as(_dp), om.size, lm.ctypes.data_as(_dp),
                         nd.ctypes.data_as(_dp), wt.ctypes.data_as(_dp), nd.size,
                         out.view(np.float64).ctypes.data_as(_dp), ctypes.byref(st)), "wgw_isr")
    return out


def wgw_lanczos_z(ctx: Context, phi, n_steps: int, z):
    """chi0bar and Lambda = (1 - chi0bar)^-1 chi0bar in the basis phi at complex frequencies z, from
    Lanczos chains of n_steps; returns (chi0 (n_z, n_pdep, n_pdep), lam (same)), element [k, m, n]."""
    phi = np.asarray(phi, np.complex128)
    npd = phi.shape[1]
    zz = np.ascontiguousarray(np.asarray(z, np.complex128).ravel())
    chi = np.zeros((zz.size, npd, npd), np.complex128)
    lam = np.zeros((zz.size, npd, npd), np.complex128)
    pb = _interleave(phi)
    st = Stats()
    _check(lib().wgw_lanczos_z(ctx.handle, pb.ctypes.data_as(_dp), npd, n_steps, zz.view(np.float64).ctypes.data_as(_dp),
                               zz.size, chi.view(np.float64).ctypes.data_as(_dp),
                               lam.view(np.float64).ctypes.data_as(_dp), ctypes.byref(st)), "wgw_lanczos_z")
    return chi, lam


def _sigma_params(n_steps_chi, n_steps_g0, nodes, weights, e_fermi, eta):
    nd = np.ascontiguousarray(nodes, np.float64)
    wt = np.ascontiguousarray(weights, np.float64)
    assert wt.size == nd.size
    p = SigmaParams(int(n_steps_chi), int(n_steps_g0), nd.ctypes.data_as(_dp), wt.ctypes.data_as(_dp), nd.size,
                    float(e_fermi), float(eta))
    return p, (nd, wt)


def wgw_sigma(ctx: Context, phi, states, omega, *, n_steps_chi: int, n_steps_g0: int, nodes, weights,
              e_fermi: float, eta: float):
    """Sigma_X, I^SR(w) and R(w) of the listed occupied states at real frequencies w <= e_fermi;
    returns (sigma_x (n_states), isr (n_states, n_omega) real, res (n_states, n_omega) complex)."""
    phi = np.asarray(phi, np.complex128)
    npd = phi.shape[1]
    sts = np.ascontiguousarray(states, np.int32)
    om = np.ascontiguousarray(omega, np.float64)
    p, keep = _sigma_params(n_steps_chi, n_steps_g0, nodes, weights, e_fermi, eta)
    sx = np.zeros(sts.size)
    isr = np.zeros((sts.size, om.size))
    res = np.zeros((sts.size, om.size), np.complex128)
    pb = _interleave(phi)
    st = Stats()
    _check(lib().wgw_sigma(ctx.handle, pb.ctypes.data_as(_dp), npd, sts.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
                           sts.size, ctypes.byref(p), om.ctypes.data_as(_dp), om.size, sx.ctypes.data_as(_dp),
                           isr.ctypes.data_as(_dp), res.view(np.float64).ctypes.data_as(_dp), ctypes.byref(st)),
           "wgw_sigma")
    del keep
    return sx, isr, res


def wgw_qp(ctx: Context, phi, states, *, n_steps_chi: int, n_steps_g0: int, nodes, weights, e_fermi: float,
           eta: float, v_xc=None, tol: float = 1e-10, max_iter: int = 100):
    """Quasiparticle energies of the listed occupied states (Eq. e_qp) by the secant method;
    returns (e_qp (n_states), sigma at e_qp (n_states) complex, secant steps (n_states))."""
    phi = np.asarray(phi, np.complex128)
    npd = phi.shape[1]
    sts = np.ascontiguousarray(states, np.int32)
    p, keep = _sigma_params(n_steps_chi, n_steps_g0, nodes, weights, e_fermi, eta)
    vx = None if v_xc is None else np.ascontiguousarray(v_xc, np.float64)
    eq = np.zeros(sts.size)
    sg = np.zeros(sts.size, np.complex128)
    it = np.zeros(sts.size, np.int32)
    pb = _interleave(phi)
    st = Stats()
    _check(lib().wgw_qp(ctx.handle, pb.ctypes.data_as(_dp), npd, sts.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
                        sts.size, ctypes.byref(p), vx.ctypes.data_as(_dp) if vx is not None else None, tol, max_iter,
                        eq.ctypes.data_as(_dp), sg.view(np.float64).ctypes.data_as(_dp),
                        it.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), ctypes.byref(st)), "wgw_qp")
    del keep
    return eq, sg, it


def wgw_sigma_x(ctx: Context, states) -> np.ndarray:
    """<psi_i|Sigma_X|psi_i> [Ha] for the listed occupied states."""
    sts = np.ascontiguousarray(states, np.int32)
    out = np.zeros(sts.size)
    _check(lib().wgw_sigma_x(ctx.handle, sts.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), sts.size,
                             out.ctypes.data_as(_dp)), "wgw_sigma_x")
    return out


def wgw_autotune_info(ctx: Context) -> dict:
    """The autotuner's choices: the tensor-core P_c K split with each candidate's median time, and
    the FP32 H kernel (-1 untuned, 0 three kernels, 1 fused) with both variants' median times."""
    choice = ctypes.c_int(0)
    splits = (ctypes.c_int * 16)()
    ms = np.zeros(16)
    fused = ctypes.c_int(-1)
    hms = np.zeros(2)
    k = lib().wgw_autotune_info(ctx.handle, ctypes.byref(choice), splits, ms.ctypes.data_as(_dp), 16,
                                ctypes.byref(fused), hms.ctypes.data_as(_dp))
    if k < 0:
        _check(-k, "wgw_autotune_info")
    return {"tc_split": choice.value, "candidates_ms": {int(splits[i]): float(ms[i]) for i in range(k)},
            "h_kernel": {-1: "untuned", 0: "three kernels", 1: "fused"}[fused.value],
            "h_ms": {"three_kernels": float(hms[0]), "fused": float(hms[1])}}


FFT_KERNEL_NAMES = {-1: "untuned", 0: "register", 1: "register, packed FP32", 2: "shared memory"}


def wgw_autotune_fft(ctx: Context) -> dict:
    """The FFT stage kernels in effect for the FP32 H application (G -> r, x-line, r -> G) and each
    candidate's median time [ms] from the autotuner (0 = not timed)."""
    ch = (ctypes.c_int * 3)()
    ms = np.zeros(9)
    _check(lib().wgw_autotune_fft(ctx.handle, ch, ms.ctypes.data_as(_dp)), "wgw_autotune_fft")
    stages = ("g2r", "xline", "r2g")
    return {st: {"choice": FFT_KERNEL_NAMES[ch[i]],
                 "ms": {FFT_KERNEL_NAMES[k]: float(ms[3 * i + k]) for k in range(3)}} for i, st in enumerate(stages)}


def wgw_autotune_chunk(ctx: Context) -> dict:
    """Pairs per chunk of the FP32 H pipeline in effect (0 none, -1 untuned) and each timed
    candidate's median time [ms]."""
    ch = ctypes.c_int(-1)
    cands = (ctypes.c_int * 8)()
    ms = np.zeros(8)
    k = lib().wgw_autotune_chunk(ctx.handle, ctypes.byref(ch), cands, ms.ctypes.data_as(_dp), 8)
    if k < 0:
        _check(-k, "wgw_autotune_chunk")
    return {"chunk_pairs": ch.value, "candidates_ms": {int(cands[i]): float(ms[i]) for i in range(k)}}


def wgw_selftest_wait_timeout() -> int:
    """Runs one bounded device wait that nothing completes; returns the flag it left (1 = gave up)."""
    t = ctypes.c_int(0)
    _check(lib().wgw_selftest_wait_timeout(ctypes.byref(t)), "wgw_selftest_wait_timeout")
    return t.value


class Ticket:
    """A submitted request; holds the output buffer until the library reports it done."""

    def __init__(self, ctx, ticket, out, n_pdep=0):
        self.ctx, self.ticket, self.out, self.n_pdep = ctx, ticket, out, n_pdep


def wgw_submit(ctx: Context, dV, omega=(0.0,), kind: int = WGW_REQ_CHI0) -> Ticket:
    """Queues chi0 (or chibar0) dV on the context's worker; returns at once."""
    dV = np.asarray(dV, np.complex128)
    dV = dV[:, None] if dV.ndim == 1 else dV
    n_pert = dV.shape[1]
    om = np.ascontiguousarray(omega, np.float64)
    buf = _interleave(dV)
    out = np.zeros((len(om), n_pert, ctx.n_rho), np.complex128)
    req = Request(kind, buf.ctypes.data_as(_dp), n_pert, om.ctypes.data_as(_dp), len(om),
                  out.view(np.float64).ctypes.data_as(_dp))
    t = ctypes.c_uint64()
    _check(lib().wgw_submit(ctx.handle, ctypes.byref(req), ctypes.byref(t)), "wgw_submit")
    return Ticket(ctx, t.value, out)


def wgw_submit_pdep(ctx: Context, n_pdep: int, x0=None) -> Ticket:
    """Queues a PDEP Davidson (n_pdep eigenpairs of chibar0, start block x0 (N_rho, n_pdep) or
    None); its chibar0 block applications are served through the same queue.  wgw_wait returns
    ((eigenvalues, basis (N_rho, n_pdep)), result dict)."""
    xb = _interleave(x0) if x0 is not None else None
    out = np.zeros(n_pdep + 2 * n_pdep * ctx.n_rho)
    req = Request(WGW_REQ_PDEP, xb.ctypes.data_as(_dp) if xb is not None else None, n_pdep, None, 0,
                  out.ctypes.data_as(_dp))
    t = ctypes.c_uint64()
    _check(lib().wgw_submit(ctx.handle, ctypes.byref(req), ctypes.byref(t)), "wgw_submit")
    return Ticket(ctx, t.value, out, n_pdep)


def _ticket_output(t: Ticket):
    if t.n_pdep:
        n = t.n_pdep
        return t.out[:n].copy(), t.out[n:].view(np.complex128).reshape(n, t.ctx.n_rho).T
    return t.out.transpose(2, 1, 0)


def wgw_cancel(t: Ticket) -> None:
    """Cancels a queued or running request (it then completes with WGW_ERR_CANCELLED)."""
    _check(lib().wgw_cancel(t.ctx.handle, t.ticket), "wgw_cancel")


def wgw_poll(t: Ticket):
    """(done, result dict or None); a finished ticket is released by the call that reports it."""
    done, res = ctypes.c_int(), Result()
    _check(lib().wgw_poll(t.ctx.handle, t.ticket, ctypes.byref(done), ctypes.byref(res)), "wgw_poll")
    if not done.value:
        return False, None
    d = res.as_dict()
    if d["status"] != WGW_OK:
        d["error"] = lib().wgw_last_error().decode()
    return True, d


def wgw_wait(t: Ticket):
    """Blocks until done -> (result (N_rho, n_pert, n_omega), result dict)."""
    res = Result()
    _check(lib().wgw_wait(t.ctx.handle, t.ticket, ctypes.byref(res)), "wgw_wait")
    d = res.as_dict()
    if d["status"] != WGW_OK:
        d["error"] = lib().wgw_last_error().decode()
    return _ticket_output(t), d


def wgw_dyson(chi0bar):
    """(1 - A)^-1 A for each A of chi0bar (n_omega, n, n) or (n, n), float64 -> same shape."""
    a = np.ascontiguousarray(chi0bar, np.float64)
    single = a.ndim == 2
    a3 = a[None] if single else a
    out = np.zeros_like(a3)
    n_om, n = a3.shape[0], a3.shape[-1]
    _check(lib().wgw_dyson(n, n_om, a3.ctypes.data_as(_dp), out.ctypes.data_as(_dp)), "wgw_dyson")
    return out[0] if single else out


def wgw_profile_enable(ctx: Context, on: bool = True):
    _check(lib().wgw_profile_enable(ctx.handle, int(on)), "wgw_profile_enable")


def wgw_profile_classes(ctx: Context, names=None):
    """Record only the named classes (None = all)."""
    if names is None:
        mask = (1 << WGW_PROF_KINDS) - 1
    else:
        idx = {lib().wgw_profile_kind_name(k).decode(): k for k in range(WGW_PROF_KINDS)}
        mask = sum(1 << idx[n] for n in names)
    _check(lib().wgw_profile_classes(ctx.handle, mask), "wgw_profile_classes")


def wgw_profile_read(ctx: Context) -> dict:
    """Per kernel class: {name: {ms, launches, bytes, flops}}."""
    out = {}
    for k in range(WGW_PROF_KINDS):
        ms, n, by, fl = ctypes.c_double(), ctypes.c_long(), ctypes.c_double(), ctypes.c_double()
        _check(lib().wgw_profile_read(ctx.handle, k, ctypes.byref(ms), ctypes.byref(n), ctypes.byref(by),
                                      ctypes.byref(fl)), "wgw_profile_read")
        out[lib().wgw_profile_kind_name(k).decode()] = {"ms": ms.value, "launches": n.value,
                                                        "bytes": by.value, "flops": fl.value}
    return out


def wgw_pdep_davidson(ctx: Context, n_pdep: int, x0=None, want_basis=True, allow_noconv=False):
    """PDEP eigenpairs: (eigenvalues (n_pdep,), basis (N_rho, n_pdep) complex or None, stats, status)."""
    eig = np.zeros(n_pdep)
    xb = _interleave(x0) if x0 is not None else None
    basis = np.zeros((n_pdep, ctx.n_rho), np.complex128) if want_basis else None
    st = Stats()
    s = lib().wgw_pdep_davidson(ctx.handle, n_pdep, xb.ctypes.data_as(_dp) if xb is not None else None,
                                eig.ctypes.data_as(_dp),
                                basis.view(np.float64).ctypes.data_as(_dp) if want_basis else None,
                                ctypes.byref(st))
    _check(s, "wgw_pdep_davidson", (WGW_OK, WGW_ERR_NOCONV) if allow_noconv else (WGW_OK,))
    return eig, (basis.T if want_basis else None), st.as_dict(), s


def wgw_pdep_davidson_channels(ctxs, n_pdep: int, x0=None, want_basis=True, allow_noconv=False):
    """PDEP eigenpairs of the spin-summed chibar0 (one context per channel); as wgw_pdep_davidson."""
    ctxs = list(ctxs)
    eig = np.zeros(n_pdep)
    xb = _interleave(x0) if x0 is not None else None
    basis = np.zeros((n_pdep, ctxs[0].n_rho), np.complex128) if want_basis else None
    st = Stats()
    handles = (ctypes.c_void_p * len(ctxs))(*[c.handle for c in ctxs])
    s = lib().wgw_pdep_davidson_channels(handles, len(ctxs), n_pdep, xb.ctypes.data_as(_dp) if xb is not None else None,
                                         eig.ctypes.data_as(_dp),
                                         basis.view(np.float64).ctypes.data_as(_dp) if want_basis else None,
                                         ctypes.byref(st))
    _check(s, "wgw_pdep_davidson_channels", (WGW_OK, WGW_ERR_NOCONV) if allow_noconv else (WGW_OK,))
    return eig, (basis.T if want_basis else None), st.as_dict(), s


def wgw_lanczos(ctx: Context, phi, n_steps: int, omega=()):
    """Lanczos chains for every (v, m): returns (chi0 (n_pdep, n_pdep, n_omega) as [n, m, k],
    alpha, beta (n_v, n_pdep, n_steps), stats)."""
    phi = np.asarray(phi, np.complex128)
    npd = phi.shape[1]
    om = np.ascontiguousarray(omega, np.float64)
    a = np.zeros((ctx.n_v, npd, n_steps))
    b = np.zeros((ctx.n_v, npd, n_steps))
    chi = np.zeros((max(len(om), 1), npd, npd))
    st = Stats()
    pb = _interleave(phi)
    _check(lib().wgw_lanczos(ctx.handle, pb.ctypes.data_as(_dp), npd, n_steps,
                             om.ctypes.data_as(_dp) if len(om) else None, len(om), a.ctypes.data_as(_dp),
                             b.ctypes.data_as(_dp), chi.ctypes.data_as(_dp) if len(om) else None,
                             ctypes.byref(st)), "wgw_lanczos")
    return chi[: len(om)].transpose(2, 1, 0), a, b, st.as_dict()


def wgw_g0_lanczos(ctx: Context, phi, states, n_steps: int, z=()):
    """G0 Lanczos chains of H from [psi_i phi~_m] for the listed occupied states i.

    Returns a dict: alpha, beta, d (n_states, n_pdep, n_steps); residues C (n_states, n_pdep,
    n_steps, n_pdep) as [i, n, l', m]; g0 (n_states, n_z, n_pdep, n_pdep) complex as [i, k, n, m]
    = <psi_i phi~_n|(H - z_k)^-1|psi_i phi~_m>; stats.
    """
    phi = np.asarray(phi, np.complex128)
    npd = phi.shape[1]
    sts = np.ascontiguousarray(states, np.int32)
    ns = sts.size
    zz = np.ascontiguousarray(np.asarray(z, np.complex128).ravel())
    nz = zz.size
    a = np.zeros((ns, npd, n_steps))
    b = np.zeros((ns, npd, n_steps))
    d = np.zeros((ns, npd, n_steps))
    C = np.zeros((ns, npd, n_steps, npd))
    g = np.zeros((ns, nz, npd, npd), np.complex128)
    st = Stats()
    pb = _interleave(phi)
    zb = zz.view(np.float64)
    _check(lib().wgw_g0_lanczos(ctx.handle, pb.ctypes.data_as(_dp), npd,
                                sts.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), ns, n_steps,
                                zb.ctypes.data_as(_dp) if nz else None, nz, a.ctypes.data_as(_dp),
                                b.ctypes.data_as(_dp), d.ctypes.data_as(_dp), C.ctypes.data_as(_dp),
                                g.view(np.float64).ctypes.data_as(_dp) if nz else None,
                                ctypes.byref(st)), "wgw_g0_lanczos")
    return dict(alpha=a, beta=b, d=d, C=C, g0=g, stats=st.as_dict())


def wgw_symm_eig_dev(A_dev, stream=None, w=None, Z=None, noalloc=False):
    """Symmetric eigensolver on device (torch float64 n x n, overwritten): returns (w, Z) torch tensors.

    noalloc=True calls wgw_symm_eig_noalloc_dev (library-side work space in a fixed device array,
    n <= 512); w and Z may then be passed in preallocated so that the call itself allocates nothing.
    """
    import torch
    n = A_dev.shape[0]
    assert A_dev.is_cuda and A_dev.dtype == torch.float64 and A_dev.is_contiguous()
    if w is None:
        w = torch.empty(n, dtype=torch.float64, device=A_dev.device)
    if Z is None:
        Z = torch.empty((n, n), dtype=torch.float64, device=A_dev.device)
    if stream is None:
        stream = torch.cuda.current_stream(A_dev.device).cuda_stream
    fn = lib().wgw_symm_eig_noalloc_dev if noalloc else lib().wgw_symm_eig_dev
    name = "wgw_symm_eig_noalloc_dev" if noalloc else "wgw_symm_eig_dev"
    _check(fn(n, ctypes.c_void_p(A_dev.data_ptr()), ctypes.c_void_p(w.data_ptr()),
              ctypes.c_void_p(Z.data_ptr()), ctypes.c_void_p(stream)), name)
    return w, Z


def wgw_system_info(ctx: Context, n_sys: int, with_flags: bool = False):
    """Per system of the last batched solve: (CG iterations, final FP64 relative residual) and,
    with with_flags, the converged flags (1 = met cg_tol)."""
    it = np.zeros(n_sys, np.int32)
    rr = np.zeros(n_sys, np.float64)
    cv = np.zeros(n_sys, np.int32)
    k = lib().wgw_system_info(ctx.handle, n_sys, it.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
                              rr.ctypes.data_as(_dp), cv.ctypes.data_as(ctypes.POINTER(ctypes.c_int)))
    return (it[:k], rr[:k], cv[:k]) if with_flags else (it[:k], rr[:k])


def wgw_sample_solutions(ctx: Context, systems) -> None:
    """Select static systems (s = r n_v + v) whose solutions the next applies keep."""
    sy = np.ascontiguousarray(np.asarray(systems, np.int32))
    _check(lib().wgw_sample_solutions(ctx.handle, sy.size, sy.ctypes.data_as(ctypes.POINTER(ctypes.c_int))),
           "wgw_sample_solutions")


def wgw_read_samples(ctx: Context, n: int) -> np.ndarray:
    """The kept solutions of the last static apply: (N_pw, n) complex, canonical order."""
    out = np.zeros((n, ctx.n_pw), np.complex128)
    _check(lib().wgw_read_samples(ctx.handle, n, out.ctypes.data_as(_dp)), "wgw_read_samples")
    return out.T.copy()


def _dev_call(fn, name, ctx, x, omega, out, stream, allow_noconv):
    """x, out: torch complex128 CUDA tensors of shape (n_pert, N_rho) / (n_omega, n_pert, N_rho)."""
    import torch
    assert x.is_cuda and x.dtype == torch.complex128 and x.is_contiguous()
    assert out.is_cuda and out.dtype == torch.complex128 and out.is_contiguous()
    n_pert = x.shape[0]
    om = np.ascontiguousarray(omega, np.float64)
    st = Stats()
    if stream is None:
        stream = torch.cuda.current_stream(x.device).cuda_stream
    s = fn(ctx.handle, ctypes.c_void_p(x.data_ptr()), n_pert, om.ctypes.data_as(_dp), len(om),
           ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(stream), ctypes.byref(st))
    _check(s, name, (WGW_OK, WGW_ERR_NOCONV) if allow_noconv else (WGW_OK,))
    return st.as_dict(), s


def wgw_apply_chi0_dev(ctx: Context, dV_dev, omega, drho_dev, stream=None, allow_noconv=False):
    return _dev_call(lib().wgw_apply_chi0_dev, "wgw_apply_chi0_dev", ctx, dV_dev, omega, drho_dev, stream,
                     allow_noconv)


def wgw_apply_chibar0_dev(ctx: Context, phi_dev, omega, out_dev, stream=None, allow_noconv=False):
    return _dev_call(lib().wgw_apply_chibar0_dev, "wgw_apply_chibar0_dev", ctx, phi_dev, omega, out_dev,
                     stream, allow_noconv)


def wgw_destroy(ctx: Context):
    if ctx.handle:
        lib().wgw_destroy(ctx.handle)
        ctx.handle = None
