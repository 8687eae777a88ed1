"""Pins of the oracle's D3Q15-MRT flow model (Sec. 3.1.1: Eqs. 12-18, A1) against the lattice
definitions, the mathematics and closed forms; the same checks that pin its D3Q19 model."""
import itertools
import math

import numpy as np
import pytest

from lbm_inputs import paper_channel


def test_velocity_set_and_isotropy(orc):
    """Eq. 12: rest, 6 axis and 8 cube-corner vectors; the weights under Eq. 18 give the
    lattice tensors of an isotropic c_s^2 = 1/3 lattice up to fourth order."""
    t = orc.tables15()
    e, w = t["e15"], t["w15"]
    got = {tuple(int(v) for v in e[:, i]) for i in range(15)}
    want = {(0, 0, 0)} | {tuple(s * (a == k) for a in range(3)) for k in range(3) for s in (1, -1)}
    want |= set(itertools.product((1, -1), repeat=3))
    assert len(got) == 15 and got == want
    d = np.eye(3)
    assert w.sum() == pytest.approx(1.0, abs=1e-15)
    assert np.allclose(np.einsum("i,ai,bi->ab", w, e, e), d / 3, atol=1e-15)
    assert np.allclose(np.einsum("i,ai,bi,ci->abc", w, e, e, e), 0, atol=1e-15)
    four = np.einsum("i,ai,bi,ci,di->abcd", w, e, e, e, e)
    iso = (np.einsum("ab,cd->abcd", d, d) + np.einsum("ac,bd->abcd", d, d)
           + np.einsum("ad,bc->abcd", d, d)) / 9
    assert np.allclose(four, iso, atol=1e-15)


def test_matrix_rows_are_the_moment_polynomials(orc):
    """Eq. A1 = the D3Q15 moment polynomials (d'Humieres et al. 2002) on Eq. 12, in the
    moment order of Eq. 13; rows orthogonal; M M^-1 = I."""
    t = orc.tables15()
    ex, ey, ez = t["e15"]
    e2 = ex * ex + ey * ey + ez * ez
    rows = np.array([np.ones_like(ex), e2 - 2, (15 * e2 * e2 - 55 * e2 + 32) / 2,
                     ex, (5 * e2 - 13) * ex / 2, ey, (5 * e2 - 13) * ey / 2,
                     ez, (5 * e2 - 13) * ez / 2, 3 * ex * ex - e2, ey * ey - ez * ez,
                     ex * ey, ey * ez, ez * ex, ex * ey * ez])
    M = t["M"]
    assert np.array_equal(M, rows)
    gram = M @ M.T
    assert np.allclose(gram - np.diag(np.diag(gram)), 0, atol=0)
    assert np.allclose(M @ t["Minv"], np.eye(15), atol=1e-15)


@pytest.mark.parametrize("phi", [1.0, 0.55])
def test_equilibrium_moments(orc, phi):
    """M f_eq(Eq. 18) = the closed form of Eq. 15 with beta1 = 1, beta2 = -5; f_eq carries
    rho, rho0 u and c_s^2 rho I + rho0 u u / phi."""
    rng = np.random.default_rng(3)
    M = orc.tables15()["M"]
    e = orc.tables15()["e15"]
    for _ in range(5):
        rho, u = 1 + 0.02 * rng.uniform(-1, 1), 0.05 * rng.uniform(-1, 1, 3)
        feq = orc.feq15(rho, u, phi)
        assert np.allclose(M @ feq, orc.meq15_eq15(rho, u, phi), atol=2e-15)
        assert feq.sum() == pytest.approx(rho, abs=1e-15)
        assert np.allclose(e @ feq, u, atol=1e-16)
        assert np.allclose(np.einsum("i,ai,bi->ab", feq, e, e),
                           rho / 3 * np.eye(3) + np.outer(u, u) / phi, atol=1e-15)


def test_forcing_is_the_derivative_of_the_equilibrium(orc):
    """S~ of Eq. 17 = rho0 (d m_eq / d u) . F (the forcing of Eq. 9 in moment space); m_eq is
    quadratic in u, so the central difference along F is exact."""
    rng = np.random.default_rng(5)
    for phi in (1.0, 0.6):
        u, F = 0.04 * rng.uniform(-1, 1, 3), 1e-3 * rng.uniform(-1, 1, 3)
        h = 1.0
        d = (orc.meq15_eq15(1.0, u + h * F, phi) - orc.meq15_eq15(1.0, u - h * F, phi)) / (2 * h)
        assert np.allclose(orc.stilde15(u, F, phi), d, rtol=0, atol=1e-15)


def test_velocity_solves_eq26(orc):
    """Eq. 27 with the sum over all 15 velocities solves rho0 u = sum e f + phi F / 2 with F
    from Eq. 4 (Eq. 26)."""
    rng = np.random.default_rng(8)
    e = orc.tables15()["e15"]
    for _ in range(5):
        f = orc.feq15(1.0, 0.05 * rng.uniform(-1, 1, 3), 0.6) + 1e-3 * rng.uniform(-1, 1, 15)
        G = 1e-3 * rng.uniform(-1, 1, 3)
        phi, nu, K, Fphi = 0.6, 0.05, 2.0, 0.5
        u = orc.velocity15(f, G, phi, nu, K, Fphi)
        F = orc.force(u, G, phi, nu, K, Fphi)
        assert np.allclose(u, e @ f + 0.5 * F, atol=1e-16)


def _params(orc, **kw):
    pb = dict(nx=1, ny=1, nz=1, mapping="lattice", nu_e=0.08, alpha_f=0.05, phi=0.7, K=3.0,
              F_phi=0.4, gbeta=2e-3, gravity_axis=2, gravity_sign=-1, T0=0.5, q=15)
    pb.update(kw)
    return orc.map_problem(pb)


def test_collision_invariants(orc):
    """Equilibrium without force is a fixed point; the collision keeps the mass and gives
    post-collision momentum rho0 u + rho0 F / 2 for any s_j (Eqs. 9, 14, 26)."""
    lp = _params(orc, phi=1.0, K=0.0, Da=None, F_phi=0.0, gbeta=0.0)
    assert len(lp.s) == 15
    u = np.array([0.02, -0.03, 0.01])
    f, g = orc.feq15(1.003, u, 1.0), orc.geq7(0.7, u)
    fo, go, mac = orc.collide_site(lp, f, g)
    assert np.allclose(fo, f, atol=1e-16) and np.allclose(go, g, atol=1e-16)
    rng = np.random.default_rng(11)
    e = orc.tables15()["e15"]
    for s_j in (1.0, 0.7, 1.6):
        lp = _params(orc)
        s = list(lp.s)
        s[3] = s[5] = s[7] = s_j
        lp.s = s
        f = orc.feq15(1.01, 0.03 * rng.uniform(-1, 1, 3), lp.phi) + 2e-3 * rng.uniform(-1, 1, 15)
        g = orc.geq7(0.3, [0, 0, 0]) + 2e-3 * rng.uniform(-1, 1, 7)
        fo, go, mac = orc.collide_site(lp, f, g)
        assert fo.sum() == pytest.approx(f.sum(), abs=1e-15)
        u, T = mac[1:4], mac[4]
        F = orc.force(u, np.array(lp.buoy) * (T - lp.T0), lp.phi, lp.nu, lp.K, lp.F_phi)
        assert np.allclose(e @ fo, u + 0.5 * F, atol=1e-16)


def test_relaxation_rates_act_on_their_moments(orc):
    """Lambda of Eq. 16: a deviation in one non-conserved moment relaxes by (1 - s_k) alone."""
    lp = _params(orc, phi=1.0, K=0.0, Da=None, F_phi=0.0, gbeta=0.0)
    t = orc.tables15()
    M, Minv = t["M"], t["Minv"]
    f0 = orc.feq15(1.0, [0.0, 0.0, 0.0], 1.0)
    g = orc.geq7(0.5, [0, 0, 0])
    for k in (1, 2, 4, 9, 10, 11, 14):
        dm = np.zeros(15)
        dm[k] = 1e-4
        fo, _, _ = orc.collide_site(lp, f0 + Minv @ dm, g)
        got = M @ fo - M @ f0
        want = np.zeros(15)
        want[k] = (1 - lp.s[k]) * 1e-4
        assert np.allclose(got, want, rtol=0, atol=2e-15), k


def _steady_u(orc, pb, steps):
    o = orc.Oracle(orc.map_problem(pb))
    o.step(steps)
    return o.macros()[1]


@pytest.mark.parametrize("Fphi,a", [(0.3, 1e-4), (0.0, 1e-4)])
def test_uniform_darcy_forchheimer_flow(orc, Fphi, a):
    """Periodic box driven by a body force: (nu/K) u + (F_phi/sqrt K) u^2 = a (Eq. 4)."""
    nu, phi, K = 0.1, 0.5, 0.5
    pb = dict(nx=2, ny=2, nz=2, mapping="lattice", nu_e=nu, phi=phi, K=K, F_phi=Fphi,
              accel=[a, 0, 0], q=15)
    u = _steady_u(orc, pb, 2000)
    if Fphi > 0:
        c = Fphi / math.sqrt(K)
        ue = (-nu / K + math.sqrt((nu / K) ** 2 + 4 * c * a)) / (2 * c)
    else:
        ue = K * a / nu
    assert u[0].mean() == pytest.approx(ue, rel=1e-10)


def test_shear_wave_decay(orc):
    """u_x = A sin(k y) decays at nu_e k^2 + phi nu / K on the D3Q15 lattice (Eq. 32)."""
    N, phi, K = 32, 0.6, 200.0
    k = 2 * math.pi / N
    lp = orc.map_problem(dict(nx=1, ny=N, nz=1, mapping="lattice", nu_e=0.05, phi=phi, K=K,
                              F_phi=0.0, q=15))
    o = orc.Oracle(lp)
    uf = np.zeros((3, 1, N, 1))
    uf[0, 0, :, 0] = 1e-3 * np.sin(k * np.arange(N))
    o.init_equilibrium(0.5, None, uf)
    o.step(50)
    a1 = o.macros()[1][0, 0, :, 0]
    o.step(400)
    a2 = o.macros()[1][0, 0, :, 0]
    rate = -math.log(np.dot(a2, uf[0, 0, :, 0]) / np.dot(a1, uf[0, 0, :, 0])) / 400
    assert rate == pytest.approx(lp.nu_e * k * k + phi * lp.nu / K, rel=5e-3)


def test_paper_channel_second_order(orc):
    """The paper's channel (Sec. 4.1), which the paper runs on D3Q15 (Fig. 4): Eqs. 48-50
    approached at second order (Eq. 52)."""
    Re, Da, phi = 10.0, 1e-2, 0.6
    errs = []
    for ny in (16, 32, 64):
        pb = dict(paper_channel(ny, Re=Re, Da=Da), q=15)
        o = orc.Oracle(orc.map_problem(pb))
        o.step(int(40 * ny / (0.01 * Re)))
        _, u, T = o.macros()
        y = (np.arange(ny) + 0.5) / ny
        t1 = Re / (2 * phi)
        t2 = math.sqrt(Re * Re + 4 * phi ** 3 / Da) / (2 * phi)
        ua = 0.01 * np.exp(t1 * (y - 1)) * np.sinh(t2 * y) / math.sinh(t2)
        Ta = (np.exp(Re * y) - 1) / (math.exp(Re) - 1)
        ux, TT = u[0, 0, :, 0], T[0, :, 0]
        errs.append((math.sqrt(np.sum((ux - ua) ** 2) / np.sum(ua ** 2)),
                     math.sqrt(np.sum((TT - Ta) ** 2) / np.sum(Ta ** 2))))
    for (a0, b0), (a1, b1) in zip(errs, errs[1:]):
        assert math.log2(a0 / a1) > 1.8 and math.log2(b0 / b1) > 1.8
    assert errs[1][0] < 0.05
