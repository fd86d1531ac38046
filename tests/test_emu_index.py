"""Index logic of the CUDA kernel bodies, stepped on the CPU by the test-only harness tests/emu.

The harness compiles the library's own __host__ __device__ kernel bodies for
the host (one thread per block) and these tests compare them with numpy and
the oracle.  They check layouts, pairing, pruning and digit-reversed
positions; numerical parity on the GPU is in test_gpu_parity.py.
"""
import ctypes
import math
import os
import shutil
import subprocess

import numpy as np
import pytest

import synth
from oracle.model import Model

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(ROOT, "paper_2203_05623_gb300", "csrc")
EMU_SRC = os.path.join(HERE, "emu", "emu.cu")
EMU_LIB = os.path.join(HERE, "emu", "_build", "libwgw_emu.so")

dp = ctypes.POINTER(ctypes.c_double)
ip = ctypes.POINTER(ctypes.c_int)


@pytest.fixture(scope="module")
def emu():
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    deps = [EMU_SRC] + [os.path.join(CSRC, f) for f in os.listdir(CSRC)]
    if not os.path.exists(EMU_LIB) or any(os.path.getmtime(d) > os.path.getmtime(EMU_LIB) for d in deps):
        os.makedirs(os.path.dirname(EMU_LIB), exist_ok=True)
        cmd = [nvcc, "-std=c++17", "-O2", "-Xcompiler", "-fPIC", "-Xcompiler", "-ffp-contract=off",
               "-shared", "-I", CSRC,
               "-gencode", "arch=compute_103a,code=sm_103a", EMU_SRC, "-o", EMU_LIB]
        subprocess.run(cmd, check=True, capture_output=True)
    return ctypes.CDLL(EMU_LIB)


def P(a, t=np.float64):
    a = np.ascontiguousarray(a, dtype=t)
    return a, a.ctypes.data_as(dp if t == np.float64 else ip)


class Maps:
    def __init__(self, emu, L, ecut, N):
        n, npairs, m = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        emu.emu_sphere_size(ctypes.c_double(L), ctypes.c_double(ecut), N, ctypes.byref(n),
                            ctypes.byref(npairs), ctypes.byref(m))
        self.n, self.np_, self.m = n.value, npairs.value, m.value
        self.miller = np.zeros(3 * self.n, np.int32)
        self.pos = np.zeros(self.np_ + 1, np.int32)
        self.neg = np.zeros(self.np_ + 1, np.int32)
        self.i0 = emu.emu_sphere_maps(ctypes.c_double(L), ctypes.c_double(ecut), N,
                                      self.miller.ctypes.data_as(ip), self.pos.ctypes.data_as(ip),
                                      self.neg.ctypes.data_as(ip))
        self.miller = self.miller.reshape(-1, 3)
        self.nrb = 2 * self.np_ + 1

    def to_rb(self, c):
        """Real-basis form of a real-in-r function given by complex coefficients (columns)."""
        c = np.atleast_2d(c.T).T
        out = np.zeros((c.shape[1], self.nrb))
        out[:, 0] = c[self.i0].real
        out[:, 1::2] = math.sqrt(2) * c[self.pos[1:]].real.T
        out[:, 2::2] = math.sqrt(2) * c[self.pos[1:]].imag.T
        return out

    def to_c(self, x):
        x = np.atleast_2d(x)
        c = np.zeros((self.n, x.shape[0]), np.complex128)
        c[self.i0] = x[:, 0]
        zp = (x[:, 1::2] + 1j * x[:, 2::2]).T / math.sqrt(2)
        c[self.pos[1:]] = zp
        c[self.neg[1:]] = zp.conj()
        return c


def test_sphere_order_matches_generator(emu):
    for L, ecut in ((10.0, 5.0), (10.0, 20.0), (16.0, 7.75)):
        mp = Maps(emu, L, ecut, 48)
        assert np.array_equal(mp.miller, synth.miller_sphere(L, ecut))
        assert mp.np_ * 2 + 1 == mp.n


@pytest.mark.parametrize("N", [12, 16, 24, 32, 40, 48, 64, 96])
def test_line_fft_dif_dit(emu, N):
    rng = np.random.default_rng(N)
    x = rng.standard_normal(N) + 1j * rng.standard_normal(N)
    xin, xp = P(np.stack([x.real, x.imag], 1).ravel())
    out = np.zeros(2 * N)
    assert emu.emu_fft_line(N, 0, xp, out.ctypes.data_as(dp)) == 0
    y = out[0::2] + 1j * out[1::2]
    pos = np.array([emu.emu_fft_position(N, k) for k in range(N)])
    assert sorted(pos) == list(range(N))
    ref = np.fft.ifft(x) * N          # sum_j x_j e^{+2 pi i jk/N}
    assert np.max(np.abs(y[pos] - ref)) < 1e-12 * N
    # DIT: digit-reversed input, natural output, sign -1.
    z = rng.standard_normal(N) + 1j * rng.standard_normal(N)
    zin = np.zeros(N, np.complex128)
    zin[pos] = z
    zi, zp = P(np.stack([zin.real, zin.imag], 1).ravel())
    emu.emu_fft_line(N, 1, zp, out.ctypes.data_as(dp))
    w = out[0::2] + 1j * out[1::2]
    assert np.max(np.abs(w - np.fft.fft(z))) < 1e-12 * N


@pytest.mark.parametrize("N", [24, 32, 48, 64, 96])
def test_line_fft_compile_time_sizes(emu, N):
    rng = np.random.default_rng(N + 1)
    x = rng.standard_normal(N) + 1j * rng.standard_normal(N)
    xin, xp = P(np.stack([x.real, x.imag], 1).ravel())
    out = np.zeros(2 * N)
    assert emu.emu_fft_line_ct(N, 0, xp, out.ctypes.data_as(dp)) == 0
    pos = np.array([emu.emu_fft_position(N, k) for k in range(N)])
    y = out[0::2] + 1j * out[1::2]
    assert np.max(np.abs(y[pos] - np.fft.ifft(x) * N)) < 1e-12 * N
    zin = np.zeros(N, np.complex128)
    zin[pos] = x
    zi, zp = P(np.stack([zin.real, zin.imag], 1).ravel())
    emu.emu_fft_line_ct(N, 1, zp, out.ctypes.data_as(dp))
    assert np.max(np.abs(out[0::2] + 1j * out[1::2] - np.fft.fft(x))) < 1e-12 * N


def test_real_basis_roundtrip(emu):
    L, ecut, N = 10.0, 5.0, 24
    mp = Maps(emu, L, ecut, N)
    rng = np.random.default_rng(1)
    c = rng.standard_normal((mp.n, 3)) + 1j * rng.standard_normal((mp.n, 3))
    cin, cp = P(np.stack([c.real, c.imag], -1).transpose(1, 0, 2).ravel())
    rb = np.zeros(3 * mp.nrb)
    out = np.zeros(2 * 3 * mp.n)
    emu.emu_rb_roundtrip(ctypes.c_double(L), ctypes.c_double(ecut), N, 3, cp, rb.ctypes.data_as(dp),
                         out.ctypes.data_as(dp))
    back = out.reshape(3, mp.n, 2)
    back = (back[..., 0] + 1j * back[..., 1]).T
    assert np.max(np.abs(back - c)) < 1e-14
    # The Hermitian part's real basis equals the python map of (c(G) + c(-G)^*)/2.
    where = {tuple(g): i for i, g in enumerate(mp.miller.tolist())}
    negi = np.array([where[(-h, -k, -l)] for h, k, l in mp.miller.tolist()])
    A = 0.5 * (c + c[negi].conj())
    assert np.max(np.abs(rb.reshape(3, mp.nrb) - mp.to_rb(A))) < 1e-14
    # Inner product: Euclidean in the real basis = sum over the full sphere.
    assert abs(mp.to_rb(A)[0] @ mp.to_rb(A)[1] - np.vdot(A[:, 0], A[:, 1]).real) < 1e-12


def test_float_float_primitives_error_bounds(emu):
    """Float-float sum and product against the exact double results: the sloppy sum is within
    about 2^-47 (|a| + |b|), the product within about 2^-47 |a b| (Dekker; Hida, Li, Bailey)."""
    rng = np.random.default_rng(5)
    n = 20000
    a = rng.standard_normal(n) * 10.0 ** rng.integers(-6, 6, n)
    b = rng.standard_normal(n) * 10.0 ** rng.integers(-6, 6, n)
    b[:200] = -a[:200] * (1 + 1e-9 * rng.standard_normal(200))   # heavy cancellation
    ai, ap = P(a)
    bi, bp = P(b)
    out = np.zeros(n)
    # Inputs are first rounded to float-float: |x - ff(x)| <= 2^-48 |x|.
    emu.emu_ff_op(0, n, ap, bp, out.ctypes.data_as(dp))
    assert np.all(np.abs(out - (a + b)) <= 2.0 ** -45 * (np.abs(a) + np.abs(b)))
    emu.emu_ff_op(2, n, ap, bp, out.ctypes.data_as(dp))
    assert np.all(np.abs(out - (a - b)) <= 2.0 ** -45 * (np.abs(a) + np.abs(b)))
    emu.emu_ff_op(1, n, ap, bp, out.ctypes.data_as(dp))
    assert np.all(np.abs(out - a * b) <= 2.0 ** -45 * np.abs(a * b))
    # Far below FP32 accuracy: a float-rounded sum would miss by ~2^-24.
    assert np.max(np.abs(out - a * b) / np.abs(a * b)) < 1e-13


@pytest.mark.parametrize("N", [24, 48, 96])
def test_line_fft_float_float(emu, N):
    rng = np.random.default_rng(N + 2)
    x = rng.standard_normal(N) + 1j * rng.standard_normal(N)
    xin, xp = P(np.stack([x.real, x.imag], 1).ravel())
    out = np.zeros(2 * N)
    assert emu.emu_fft_line_ff(N, 0, xp, out.ctypes.data_as(dp)) == 0
    pos = np.array([emu.emu_fft_position(N, k) for k in range(N)])
    y = out[0::2] + 1j * out[1::2]
    ref = np.fft.ifft(x) * N
    err = np.max(np.abs(y[pos] - ref)) / np.max(np.abs(ref))
    assert err < 2e-13          # about 48-bit arithmetic; FP32 would give ~1e-7
    zin = np.zeros(N, np.complex128)
    zin[pos] = x
    zi, zp = P(np.stack([zin.real, zin.imag], 1).ravel())
    emu.emu_fft_line_ff(N, 1, zp, out.ctypes.data_as(dp))
    ref = np.fft.fft(x)
    assert np.max(np.abs(out[0::2] + 1j * out[1::2] - ref)) / np.max(np.abs(ref)) < 2e-13


@pytest.mark.parametrize("fp32", [0, 1, 2, 3, 4, 8, 9, 12])
def test_apply_h_bodies_equal_dense_h(emu, cfg24, fp32):
    s = cfg24
    m = Model(s.L, s.ecut, s.grid, s.vloc_G, s.psi_v, s.e_v)
    mp = Maps(emu, s.L, s.ecut, s.grid)
    rng = np.random.default_rng(2)
    n_sys = 3
    X = rng.standard_normal((n_sys, mp.nrb))
    shift = np.array([0.3, -0.7, 1.1])
    v_in, vp = P(np.stack([s.vloc_G.real, s.vloc_G.imag], 1).ravel())
    xin, xp = P(X.ravel())
    sh, shp = P(shift)
    out = np.zeros(n_sys * mp.nrb)
    emu.emu_apply_h(ctypes.c_double(s.L), ctypes.c_double(s.ecut), s.grid, vp, n_sys, xp, shp,
                    out.ctypes.data_as(dp), fp32)
    ref = m.h_dense() @ mp.to_c(X) + shift[None, :] * mp.to_c(X)
    got = mp.to_c(out.reshape(n_sys, mp.nrb))
    tol = 2e-6 if fp32 & 1 else 1e-12 if fp32 & 4 else 1e-13
    assert np.max(np.abs(got - ref)) < tol * np.max(np.abs(ref))


def test_apply_h_bodies_96_register_resident(emu):
    """The 96-point register-resident FP32 bodies (one line per thread; batched sphere scatter and
    gather) apply the local H of a 96^3 model as the dense H does, to FP32 accuracy."""
    s = synth.make_system(synth.Config("g96", L=24.0, ecut=3.3, grid=96, n_wells=64, well_seed=3, n_v=16, kb=True))
    m = Model(s.L, s.ecut, s.grid, s.vloc_G, s.psi_v, s.e_v)          # local part only, as the bodies
    mp = Maps(emu, s.L, s.ecut, s.grid)
    rng = np.random.default_rng(3)
    n_sys = 3
    X = rng.standard_normal((n_sys, mp.nrb))
    shift = np.array([0.2, -0.5, 0.9])
    v_in, vp = P(np.stack([s.vloc_G.real, s.vloc_G.imag], 1).ravel())
    xin, xp = P(X.ravel())
    sh, shp = P(shift)
    out = np.zeros(n_sys * mp.nrb)
    assert emu.emu_apply_h(ctypes.c_double(s.L), ctypes.c_double(s.ecut), s.grid, vp, n_sys, xp, shp,
                           out.ctypes.data_as(dp), 16 | 1) == 0
    ref = m.h_dense() @ mp.to_c(X) + shift[None, :] * mp.to_c(X)
    got = mp.to_c(out.reshape(n_sys, mp.nrb))
    assert np.max(np.abs(got - ref)) < 2e-6 * np.max(np.abs(ref))


@pytest.mark.parametrize("reg", [0, 1])
def test_products_bodies_equal_oracle(emu, cfg24, reg):
    """Right-hand-side products (FROM_REAL and TO_REAL x-line passes), shared-memory or
    register-resident x-line bodies."""
    emu.emu_set_reg_xline(reg)
    s = cfg24
    m = Model(s.L, s.ecut, s.grid, s.vloc_G, s.psi_v, s.e_v)
    mp = Maps(emu, s.L, s.ecut, s.grid)
    dV = synth.perturbations(s.miller_rho, s.L, 3, 2)
    a_idx = np.array([0, 3, 1, 2, 2], np.int32)
    b_idx = np.array([1, 0, 2, 2, 0], np.int32)
    psi_in, pp = P(np.stack([s.psi_v.real, s.psi_v.imag], -1).transpose(1, 0, 2).ravel())
    f_in, fp = P(np.stack([dV.real, dV.imag], -1).transpose(1, 0, 2).ravel())
    out = np.zeros(len(a_idx) * mp.nrb)
    emu.emu_products(ctypes.c_double(s.L), ctypes.c_double(s.ecut), s.grid, s.n_v, pp, 3, fp, len(a_idx),
                     a_idx.ctypes.data_as(ip), b_idx.ctypes.data_as(ip), out.ctypes.data_as(dp))
    got = mp.to_c(out.reshape(len(a_idx), mp.nrb))
    for k, (a, b) in enumerate(zip(a_idx, b_idx)):
        ref = m.multiply_r(dV[:, b], s.psi_v[:, a])
        assert np.max(np.abs(got[:, k] - ref)) < 1e-13 * np.max(np.abs(ref))
    emu.emu_set_reg_xline(0)


@pytest.mark.parametrize("reg", [0, 1])
def test_drho_bodies_equal_oracle(emu, cfg24, reg):
    emu.emu_set_reg_xline(reg)
    s = cfg24
    m = Model(s.L, s.ecut, s.grid, s.vloc_G, s.psi_v, s.e_v)
    mw = Maps(emu, s.L, s.ecut, s.grid)
    mr = Maps(emu, s.L, 4 * s.ecut, s.grid)
    rng = np.random.default_rng(4)
    n_pert = 3
    X = rng.standard_normal((n_pert * s.n_v, mw.nrb))
    psi_in, pp = P(np.stack([s.psi_v.real, s.psi_v.imag], -1).transpose(1, 0, 2).ravel())
    xin, xp = P(X.ravel())
    out = np.zeros(n_pert * mr.nrb)
    emu.emu_drho(ctypes.c_double(s.L), ctypes.c_double(s.ecut), s.grid, s.n_v, pp, n_pert, xp,
                 ctypes.c_double(0.75), out.ctypes.data_as(dp))
    got = mr.to_c(out.reshape(n_pert, mr.nrb))
    xc = mw.to_c(X)
    for p in range(n_pert):
        rho_r = sum(m.to_r(s.psi_v[:, v], m.mw) * m.to_r(xc[:, p * s.n_v + v], m.mw) for v in range(s.n_v))
        ref = 0.75 * m.to_G(rho_r, m.mr)
        assert np.max(np.abs(got[:, p] - ref)) < 1e-13 * np.max(np.abs(ref))
    emu.emu_set_reg_xline(0)


def test_projector_body(emu):
    rng = np.random.default_rng(5)
    n, nv, ns = 77, 5, 19
    Psi, _ = np.linalg.qr(rng.standard_normal((n, nv)))
    Y = rng.standard_normal((ns, n))
    ref = Y - (Y @ Psi) @ Psi.T
    pin, pp = P(Psi.T.ravel())
    yin, yp = P(Y.ravel())
    emu.emu_pc(n, nv, ns, pp, yp)
    assert np.max(np.abs(yin.reshape(ns, n) - ref)) < 1e-13
