"""Exchange self-energy on the GPU against the oracle (Eq. sigmacIR): relative error 1e-10 on
both paths (the pair densities are transformed at FP64 accuracy either way)."""
import numpy as np
import pytest

import synth
from oracle import sigma
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


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_sigma_x_matches_oracle(W, cfg24, precision):
    s = cfg24
    m = Model(s.L, s.ecut, s.grid, s.vloc_G, s.psi_v, s.e_v)
    ref = sigma.sigma_x(m)
    opt = W.wgw_default_options(precision=W.WGW_MIXED if precision == "mixed" else W.WGW_FP64)
    ctx = W.wgw_setup(s.L, s.ecut, s.grid, s.vloc_G, s.psi_v, s.e_v, opt)
    got = W.wgw_sigma_x(ctx, list(range(s.n_v)))
    assert np.all(got < 0)
    assert np.max(np.abs(got - ref)) < 1e-10 * np.max(np.abs(ref))
    # A subset in another order gives the same numbers.
    sub = W.wgw_sigma_x(ctx, [3, 1])
    assert np.max(np.abs(sub - ref[[3, 1]])) < 1e-10 * np.max(np.abs(ref))


def test_sigma_x_many_states_in_batches(W):
    """70 occupied states: several batches of pair densities."""
    s = synth.make_system(synth.Config("nv70", L=10.0, ecut=5.0, grid=24, n_wells=16, well_seed=1, n_v=70))
    m = Model(s.L, s.ecut, s.grid, s.vloc_G, s.psi_v, s.e_v)
    states = [0, 17, 69, 68, 40, 5, 33, 12]
    ref = sigma.sigma_x(m, states)
    ctx = W.wgw_setup(s.L, s.ecut, s.grid, s.vloc_G, s.psi_v, s.e_v, W.wgw_default_options())
    got = W.wgw_sigma_x(ctx, states)
    assert np.max(np.abs(got - ref)) < 1e-10 * np.max(np.abs(ref))


def test_sigma_x_rejects_bad_state(W, tiny):
    s = tiny
    ctx = W.wgw_setup(s.L, s.ecut, s.grid, s.vloc_G, s.psi_v, s.e_v, W.wgw_default_options())
    with pytest.raises(W.WgwError):
        W.wgw_sigma_x(ctx, [s.n_v])


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_isr_matches_oracle(W, cfg24, precision):
    """I^SR of Eq. ISR: the GPU chains, resolvent and quadrature contraction against the oracle's
    (1e-10 of the largest value), with a Lambda that varies with the node and is not diagonal."""
    from oracle import sigma as osig
    s = cfg24
    m = Model(s.L, s.ecut, s.grid, s.vloc_G, s.psi_v, s.e_v)
    npd, n_steps = 4, 12
    phi = synth.perturbations(s.miller_rho, s.L, npd, 91)
    x, wts = np.polynomial.legendre.leggauss(8)
    nodes, weights = 5.0 * (x + 1.0), 5.0 * wts
    rng = np.random.default_rng(92)
    A = rng.standard_normal((npd, npd))
    lam = np.array([(A + A.T) / (1.0 + wp) for wp in nodes])
    states, omegas = [0, 3], [-0.4, 0.35]
    ref = osig.isr(m, phi, states, n_steps, omegas, lam, nodes, weights)
    opt = W.wgw_default_options(precision=W.WGW_MIXED if precision == "mixed" else W.WGW_FP64)
    ctx = W.wgw_setup(s.L, s.ecut, s.grid, s.vloc_G, s.psi_v, s.e_v, opt)
    got = W.wgw_isr(ctx, phi, states, n_steps, omegas, lam, nodes, weights)
    assert np.max(np.abs(got - ref)) < 1e-10 * np.max(np.abs(ref))


def _model(s):
    return Model(s.L, s.ecut, s.grid, s.vloc_G, s.psi_v, s.e_v)


def _dyson(c):
    return np.linalg.solve(np.eye(c.shape[0]) - c, c)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_lanczos_z_matches_oracle(W, cfg24, precision):
    """chi0bar and Lambda at complex frequencies (real w + i eta, and one imaginary) from the GPU
    chains against the oracle's chains (chi0_pdep_z) and a dense Dyson solve: 1e-10 of the largest
    value.  The GPU returns element [k, m, n] (m = chain vector), the oracle [n, m, k]."""
    from oracle import lanczos
    s = cfg24
    m = _model(s)
    npd, n_steps = 4, 12
    phi = 3.0 * synth.perturbations(s.miller_rho, s.L, npd, 93)
    zs = np.array([0.3 + 0.05j, -0.5 + 0.1j, 0.7j, 1.5 + 0.02j])
    ref = lanczos.chi0_pdep_z(m, phi, zs, n_steps)
    opt = W.wgw_default_options(precision=W.WGW_MIXED if precision == "mixed" else W.WGW_FP64)
    ctx = W.wgw_setup(s.L, s.ecut, s.grid, s.vloc_G, s.psi_v, s.e_v, opt)
    chi, lam = W.wgw_lanczos_z(ctx, phi, n_steps, zs)
    for k in range(zs.size):
        c_ref = ref[:, :, k].T
        assert np.max(np.abs(chi[k] - c_ref)) < 1e-10 * np.max(np.abs(c_ref))
        l_ref = _dyson(ref[:, :, k]).T
        assert np.max(np.abs(lam[k] - l_ref)) < 1e-10 * np.max(np.abs(l_ref))
    # z = i w is the imaginary-frequency response of wgw_lanczos (real).
    assert np.max(np.abs(chi[2].imag)) < 1e-12 * np.max(np.abs(chi[2]))


class _OracleSigma:
    """The oracle's Sigma parts for one model and basis, with Lambda at complex frequencies from the
    oracle's chi0 chains (memoised per frequency) and at the quadrature nodes."""

    def __init__(self, m, phi, n_chi, n_g0, nodes, weights, e_fermi, eta):
        from oracle import lanczos
        self.m, self.phi, self.n_chi, self.n_g0 = m, phi, n_chi, n_g0
        self.nodes, self.weights, self.e_fermi, self.eta = nodes, weights, e_fermi, eta
        chi = lanczos.chi0_pdep(m, phi, nodes, n_chi)[0]
        self.lam_nodes = np.array([_dyson(chi[:, :, k]).real for k in range(nodes.size)])
        self.cache = {}

    def lam_fn(self, z):
        from oracle import lanczos
        if z not in self.cache:
            self.cache[z] = _dyson(lanczos.chi0_pdep_z(self.m, self.phi, [z], self.n_chi)[:, :, 0])
        return self.cache[z]

    def isr(self, i, omegas):
        return sigma.isr(self.m, self.phi, [i], self.n_g0, omegas, self.lam_nodes, self.nodes, self.weights)[0]

    def res(self, i, omegas):
        return sigma.residue_term(self.m, self.phi, i, omegas, self.e_fermi, self.eta, self.lam_fn)


def _sigma_setup(s):
    m = _model(s)
    e = np.linalg.eigvalsh(m.h_dense())
    e_fermi = 0.5 * (e[s.n_v - 1] + e[s.n_v])
    x, wts = np.polynomial.legendre.leggauss(8)
    nodes, weights = 5.0 * (x + 1.0), 5.0 * wts
    phi = 3.0 * synth.perturbations(s.miller_rho, s.L, 4, 94)
    return m, e_fermi, nodes, weights, phi


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_sigma_parts_match_oracle(W, cfg24, precision):
    """Sigma_X, I^SR(w) and the residue term R(w) of Eq. Rfac at real frequencies below e_F, with
    Lambda from the library's own chains, against the oracle with Lambda from the oracle's chains:
    each part within 1e-10 of its largest value."""
    s = cfg24
    m, e_fermi, nodes, weights, phi = _sigma_setup(s)
    n_chi, n_g0, eta = 12, 12, 0.1
    states = [0, s.n_v - 1]
    omegas = np.array([s.e_v[0] - 0.1, s.e_v[1] - 0.05, s.e_v[-1] - 0.02, e_fermi - 0.01])
    opt = W.wgw_default_options(precision=W.WGW_MIXED if precision == "mixed" else W.WGW_FP64)
    ctx = W.wgw_setup(s.L, s.ecut, s.grid, s.vloc_G, s.psi_v, s.e_v, opt)
    sx, isr, res = W.wgw_sigma(ctx, phi, states, omegas, n_steps_chi=n_chi, n_steps_g0=n_g0, nodes=nodes,
                               weights=weights, e_fermi=e_fermi, eta=eta)
    o = _OracleSigma(m, phi, n_chi, n_g0, nodes, weights, e_fermi, eta)
    sx_ref = sigma.sigma_x(m, states)
    isr_ref = np.array([o.isr(i, omegas) for i in states])
    res_ref = np.array([o.res(i, omegas) for i in states])
    assert np.max(np.abs(isr_ref.imag)) < 1e-12 * np.max(np.abs(isr_ref))
    assert np.max(np.abs(sx - sx_ref)) < 1e-10 * np.max(np.abs(sx_ref))
    assert np.max(np.abs(isr - isr_ref.real)) < 1e-10 * np.max(np.abs(isr_ref))
    assert np.max(np.abs(res_ref)) > 0
    assert np.max(np.abs(res - res_ref)) < 1e-10 * np.max(np.abs(res_ref))
    # Above the highest occupied energy no occupied state lies above w: R vanishes there.
    assert np.all(res[:, 3] == 0)
    with pytest.raises(W.WgwError):
        W.wgw_sigma(ctx, phi, states, [e_fermi + 0.05], n_steps_chi=n_chi, n_steps_g0=n_g0, nodes=nodes,
                    weights=weights, e_fermi=e_fermi, eta=eta)


def test_qp_energies_match_oracle(W, cfg24):
    """Eq. e_qp solved by the secant method on the library's Sigma_X + I^SR + R against the oracle's
    secant (qp_energy) on its own Sigma: within 1e-10 (FP64 path)."""
    s = cfg24
    m, e_fermi, nodes, weights, phi = _sigma_setup(s)
    n_chi, n_g0, eta = 12, 12, 0.1
    states = [0, s.n_v - 1]
    vxc = np.array([0.05, -0.02])
    ctx = W.wgw_setup(s.L, s.ecut, s.grid, s.vloc_G, s.psi_v, s.e_v, W.wgw_default_options(precision=W.WGW_FP64))
    eq, sg, it = W.wgw_qp(ctx, phi, states, n_steps_chi=n_chi, n_steps_g0=n_g0, nodes=nodes, weights=weights,
                          e_fermi=e_fermi, eta=eta, v_xc=vxc)
    o = _OracleSigma(m, phi, n_chi, n_g0, nodes, weights, e_fermi, eta)
    sx_ref = sigma.sigma_x(m, states)
    for k, i in enumerate(states):
        def sig(E, k=k, i=i):
            return sx_ref[k] + o.isr(i, [E])[0] + o.res(i, [E])[0]
        ref = sigma.qp_energy(s.e_v[i], sig, v_xc=vxc[k])
        assert abs(eq[k] - ref) < 1e-10 * max(1.0, abs(ref))
        assert 1 <= it[k] < 100
        # The returned Sigma is Sigma(e_qp): the QP equation holds with it.
        assert abs(s.e_v[i] + sg[k].real - vxc[k] - eq[k]) < 1e-9
