"""Host logic of the serving entry points, without a GPU: the library's request queue
(csrc/serve_sched.h) built into a test-only harness with a fake device-memory reading.

Covers admission against the memory budget (the head request included, a request that can
never fit on an idle device fails with NOMEM), merging by kind and frequency set within the
budget, cancellation of queued and running requests, and the descriptor checks wgw_submit runs
before anything is copied.
"""
import ctypes
import os
import shutil
import subprocess

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(ROOT, "paper_2203_05623_gb300", "csrc")
SRC = os.path.join(HERE, "emu", "serve_host.cpp")
LIB = os.path.join(HERE, "emu", "_build", "libserve_host.so")

OK, ERR_ARG, ERR_NOMEM, ERR_CANCELLED = 0, 1, 2, 7
QUEUED, RUNNING, DONE, UNKNOWN = 1, 2, 3, 0
dp = ctypes.POINTER(ctypes.c_double)
u64p = ctypes.POINTER(ctypes.c_uint64)


@pytest.fixture(scope="module")
def H():
    cxx = shutil.which("g++")
    if not cxx:
        pytest.skip("g++ not available")
    deps = [SRC, os.path.join(CSRC, "serve_sched.h")]
    if not os.path.exists(LIB) or any(os.path.getmtime(d) > os.path.getmtime(LIB) for d in deps):
        os.makedirs(os.path.dirname(LIB), exist_ok=True)
        subprocess.run([cxx, "-std=c++17", "-O1", "-fPIC", "-shared", "-I", CSRC, SRC, "-o", LIB], check=True)
    L = ctypes.CDLL(LIB)
    L.sh_new.restype = ctypes.c_void_p
    L.sh_new.argtypes = [ctypes.c_double, ctypes.c_double]
    L.sh_free.argtypes = [ctypes.c_void_p]
    L.sh_validate.argtypes = [ctypes.c_int, dp, ctypes.c_int, dp, ctypes.c_int, dp, ctypes.c_long]
    L.sh_push.restype = ctypes.c_uint64
    L.sh_push.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, dp, ctypes.c_int]
    L.sh_take.argtypes = [ctypes.c_void_p, ctypes.c_double, ctypes.c_int, u64p, ctypes.c_int, u64p,
                          ctypes.POINTER(ctypes.c_int)]
    L.sh_take_running.argtypes = [ctypes.c_void_p, ctypes.c_double, u64p, ctypes.c_int]
    L.sh_finish_running.argtypes = [ctypes.c_void_p, ctypes.c_int, u64p, ctypes.c_int]
    L.sh_cancel.argtypes = [ctypes.c_void_p, ctypes.c_uint64]
    L.sh_state.argtypes = [ctypes.c_void_p, ctypes.c_uint64]
    L.sh_take_done.argtypes = [ctypes.c_void_p, ctypes.c_uint64]
    return L


class Q:
    def __init__(self, H, base, per_real):
        self.H, self.h = H, H.sh_new(base, per_real)

    def push(self, n_pert, omega=(0.0,), kind=0):
        om = np.ascontiguousarray(omega, np.float64)
        return self.H.sh_push(self.h, kind, n_pert, om.ctypes.data_as(dp), om.size)

    def take(self, budget, busy=False):
        b = (ctypes.c_uint64 * 64)()
        r = (ctypes.c_uint64 * 64)()
        nr = ctypes.c_int()
        n = self.H.sh_take(self.h, budget, int(busy), b, 64, r, ctypes.byref(nr))
        return list(b[:n]), list(r[:nr.value])

    def __del__(self):
        self.H.sh_free(self.h)


def test_head_request_is_held_to_the_budget(H):
    """Memory model: 100 bytes + 10 per resident real part (a request of p perturbations has up to
    2p parts).  A request whose least need (one part) exceeds the budget waits while the device
    is busy and fails with NOMEM on an idle device; the next request then runs."""
    q = Q(H, 100.0, 10.0)
    big, small = q.push(4), q.push(1)
    assert q.take(105.0, busy=True) == ([], [])            # head (needs 110) waits behind busy work
    assert H.sh_state(q.h, big) == QUEUED
    batch, rejected = q.take(105.0, busy=False)             # idle device: it can never fit
    assert batch == [] and rejected == [big, small]          # the small one needs 110 too
    assert H.sh_take_done(q.h, big) == ERR_NOMEM and H.sh_take_done(q.h, small) == ERR_NOMEM
    q2 = Q(H, 100.0, 10.0)
    t = q2.push(1)
    assert q2.take(115.0)[0] == [t]


def test_fake_allocator_with_no_free_memory(H):
    """Free memory reads 0: every request fails with NOMEM instead of running or hanging."""
    q = Q(H, 64.0, 8.0)
    ts = [q.push(2), q.push(1, omega=[0.0, 0.5])]
    batch, rejected = q.take(0.0)
    assert batch == [] and sorted(rejected) == sorted(ts)
    assert [H.sh_take_done(q.h, t) for t in ts] == [ERR_NOMEM, ERR_NOMEM]


def test_merging_by_kind_and_frequency_set_within_the_budget(H):
    q = Q(H, 100.0, 10.0)
    a = q.push(2)                          # 4 parts
    b = q.push(2, omega=[0.0, 0.3])        # other frequency set: not merged with a
    c = q.push(1)                          # 2 parts: a + c = 6 parts -> 160 bytes
    d = q.push(3)                          # a + c + d = 12 parts -> 220 bytes > budget 200
    e = q.push(1, kind=1)                  # other kind
    batch, _ = q.take(200.0)
    assert batch == [a, c]
    batch, _ = q.take(200.0)
    assert batch == [b]
    batch, _ = q.take(200.0)
    assert batch == [d]                     # alone: 160 bytes resident
    batch, _ = q.take(200.0)
    assert batch == [e]
    assert all(H.sh_take_done(q.h, t) == OK for t in (a, b, c, d, e))


def test_cancel_queued_and_running_requests(H):
    q = Q(H, 10.0, 1.0)
    a, b, c = q.push(1), q.push(1), q.push(1, omega=[0.2])
    assert H.sh_cancel(q.h, b) == OK
    assert H.sh_state(q.h, b) == DONE and H.sh_take_done(q.h, b) == ERR_CANCELLED
    run = (ctypes.c_uint64 * 8)()
    n = H.sh_take_running(q.h, 1e9, run, 8)
    assert list(run[:n]) == [a]                # b is gone; c has another frequency set
    assert H.sh_state(q.h, a) == RUNNING
    assert H.sh_cancel(q.h, a) == OK           # running: completes as cancelled at the batch end
    H.sh_finish_running(q.h, OK, run, n)
    assert H.sh_take_done(q.h, a) == ERR_CANCELLED
    assert H.sh_cancel(q.h, a) == ERR_ARG      # finished and released
    assert H.sh_cancel(q.h, 999) == ERR_ARG    # unknown
    assert q.take(1e9)[0] == [c]


def test_corrupted_descriptors_are_rejected(H):
    n_rho = 5
    dV = np.zeros(2 * n_rho * 2)
    out = np.zeros(2 * n_rho * 2)
    om = np.array([0.0, 1.0])

    def v(kind=0, d=dV, n_pert=2, o=om, n_om=2, ob=out):
        ptr = (lambda a: a.ctypes.data_as(dp) if a is not None else None)
        return H.sh_validate(kind, ptr(d), n_pert, ptr(o), n_om, ptr(ob), n_rho)

    assert v() == OK
    assert v(kind=5) == ERR_ARG
    assert v(n_pert=0) == ERR_ARG
    assert v(n_om=0) == ERR_ARG and v(n_om=5000) == ERR_ARG
    assert v(o=np.array([0.0, -1.0])) == ERR_ARG
    assert v(o=np.array([0.0, np.nan])) == ERR_ARG and v(o=np.array([np.inf, 0.0])) == ERR_ARG
    bad = dV.copy()
    bad[7] = np.nan
    assert v(d=bad) == ERR_ARG
    assert v(d=None) == ERR_ARG and v(ob=None) == ERR_ARG and v(o=None) == ERR_ARG


def test_pdep_descriptors(H):
    """A PDEP request (kind 2) takes no frequencies and an optional start block; its output buffer
    and a finite start block are still required."""
    n_rho = 5
    x0 = np.zeros(2 * n_rho * 2)
    out = np.zeros(2 + 2 * n_rho * 2)

    def v(d=x0, n_pert=2, ob=out):
        ptr = (lambda a: a.ctypes.data_as(dp) if a is not None else None)
        return H.sh_validate(2, ptr(d), n_pert, None, 0, ptr(ob), n_rho)

    assert v() == OK and v(d=None) == OK
    assert v(n_pert=0) == ERR_ARG and v(ob=None) == ERR_ARG
    bad = x0.copy()
    bad[3] = np.inf
    assert v(d=bad) == ERR_ARG
