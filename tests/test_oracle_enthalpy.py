"""Pins of the oracle's enthalpy-based D3Q7 model for solid-liquid phase change (App. B)."""
import math

import numpy as np
import pytest


def _params(orc, **kw):
    pb = dict(nx=1, ny=1, nz=1, mapping="lattice", nu_e=0.1, alpha_f=0.04, enthalpy=True,
              T_m=0.0, St=1.0, T0=0.0)
    pb.update(kw)
    return orc.map_problem(pb)


def test_enthalpy_state_relations(orc):
    """Eqs. B8-B9: T and f_l are continuous and piecewise linear in En_e, f_l in [0, 1], and
    the phase-pure enthalpy inverts B8 outside the mushy range."""
    lp = _params(orc, T_s=-0.1, T_l=0.2, sigma_s=1.5, sigma_l=0.8, St=2.0)
    Es = lp.sigma_s * lp.c_pl * lp.T_s
    El = lp.sigma_l * lp.c_pl * lp.T_l + lp.L_a
    for En, T, fl in ((Es - 1e-12, lp.T_s, 0.0), (Es + 1e-12, lp.T_s, 0.0),
                      (El - 1e-12, lp.T_l, 1.0), (El + 1e-12, lp.T_l, 1.0),
                      (0.5 * (Es + El), 0.5 * (lp.T_s + lp.T_l), 0.5)):
        t, f = orc.enthalpy_state(lp, En)
        assert t == pytest.approx(T, abs=1e-9) and f == pytest.approx(fl, abs=1e-9)
    for T in (-1.0, -0.3, 0.5, 2.0):
        t, f = orc.enthalpy_state(lp, orc.enthalpy_of(lp, T))
        assert t == pytest.approx(T, abs=1e-14) and f in (0.0, 1.0)


def test_latent_heat_scales_with_porosity(orc):
    """Eqs. B5 and B8: the effective enthalpy is sigma c_pl T + phi f_l L_a, only the pore
    fraction phi of a site melting, so at the melting point a site of porosity phi holding
    En_e = sigma c_pl T_m + phi f L_a is at T_m with liquid fraction f."""
    lp = _params(orc, T_s=0.5, T_l=0.5, St=0.5)
    for phi in (1.0, 0.4):
        for f in (0.25, 0.75):
            En = lp.sigma_s * lp.c_pl * 0.5 + phi * f * lp.L_a
            t, fl = orc.enthalpy_state(lp, En, phi)
            assert t == pytest.approx(0.5, abs=1e-12) and fl == pytest.approx(f, abs=1e-12)


def test_geq_b12_has_the_moments_of_b6(orc):
    """N g_eq (Eq. B12) = n_eq (Eq. B6)."""
    lp = _params(orc, c_pl=1.3, c_ps=0.7, varpi=0.4)
    N = orc.tables()["N"]
    u = np.array([0.02, -0.01, 0.03])
    for En, T in ((0.7, 0.2), (-0.4, -0.3)):
        n = N @ orc.geq7_enthalpy(lp, En, T, u)
        want = [En, lp.c_pl * T * u[0], lp.c_pl * T * u[1], lp.c_pl * T * u[2],
                lp.varpi * lp.c_ref * T, 0.0, 0.0]
        assert np.allclose(n, want, atol=1e-15)
    assert lp.c_ref == pytest.approx(2.0 / (1 / 1.3 + 1 / 0.7))  # Eq. B13


def test_enthalpy_collision_conserves_and_fixes_equilibrium(orc):
    lp = _params(orc, flow_off=True)
    rng = np.random.default_rng(4)
    f = orc.feq19(1.0, [0, 0, 0], 1.0)
    for T in (-0.5, 0.7):
        En = orc.enthalpy_of(lp, T)
        g = orc.geq7_enthalpy(lp, En, T, [0, 0, 0])
        fo, go, mac = orc.collide_site(lp, f, g)
        assert np.allclose(go, g, atol=1e-15) and mac[4] == pytest.approx(T)
        g2 = g + 1e-3 * rng.uniform(-1, 1, 7)
        _, go2, _ = orc.collide_site(lp, f, g2)
        assert go2.sum() == pytest.approx(g2.sum(), abs=1e-15)


def _eta(ratio, St=1.0, Th=1.0, Tm=0.0, Ti=-1.0):
    """Root of Eq. 59 with k_s/k_l = alpha_s/alpha_l (equal rho c_p), by bisection."""
    def F(e):
        r = ratio
        return (math.exp(-e * e) / math.erf(e)
                + (1.0 / r) * math.sqrt(r) * (Ti - Tm) / (Th - Tm) * math.exp(-e * e * r)
                / math.erfc(e * math.sqrt(r)) - e * math.sqrt(math.pi) / St)
    lo, hi = 1e-6, 5.0
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        lo, hi = (mid, hi) if F(mid) > 0 else (lo, mid)
    return 0.5 * (lo + hi)


@pytest.mark.parametrize("ratio", [1.0, 2.0, 4.0])
def test_two_region_melting(orc, ratio):
    """Sec. 4.3: a solid at T_i = -1 melts (T_m = 0, St = 1) from a wall held at T_h = 1; at
    Fo = 0.01 the temperature follows Eqs. 57-58 with eta from Eq. 59 (relative global error
    of Eq. 52 below 1.5 %) and the interface x_m = 2 eta sqrt(alpha_l t) is within half a
    spacing."""
    N, a_s = 100, 0.02
    pb = dict(nx=N, ny=1, nz=1, mapping="lattice", nu_e=0.1, alpha_f=ratio * a_s, enthalpy=True,
              flow_off=True, T_m=0.0, St=1.0, alpha_ratio=ratio, flow_bc=[1, 1, 0, 0, 0, 0],
              heat_bc=[2, 2, 0, 0, 0, 0], face_T=[1.0, -1.0, 0, 0, 0, 0], T_init=-1.0, T0=0.0)
    lp = orc.map_problem(pb)
    o = orc.Oracle(lp)
    t = int(0.01 * N * N / a_s)
    o.step(t)
    _, u, T = o.macros()
    T = T[0, 0, :]
    e = _eta(ratio)
    a_l = ratio * a_s
    x = np.arange(N) + 0.5  # halfway wall at x = 0
    xm = 2 * e * math.sqrt(a_l * t)
    Ta = np.where(x <= xm, 1.0 - np.vectorize(math.erf)(x / (2 * math.sqrt(a_l * t))) / math.erf(e),
                  -1.0 + np.vectorize(math.erfc)(x / (2 * math.sqrt(a_s * t)))
                  / math.erfc(e * math.sqrt(ratio)))
    assert math.sqrt(np.sum((T - Ta) ** 2) / np.sum(Ta ** 2)) < 1.5e-2
    _, g = o.populations()
    fl = np.clip(g.sum(axis=0)[0, 0, :] / lp.L_a, 0.0, 1.0)  # En = f_l L_a in the mushy cell
    assert abs(np.interp(0.5, fl[::-1], x[::-1]) - xm) < 0.5
    assert np.abs(u).max() == 0.0 and T.max() <= 1.0 + 1e-12 and T.min() >= -1.0 - 1e-12


def test_solid_cells_do_not_flow(orc):
    """Convection melting in a cavity: where f_l < 0.5 the velocity is zero."""
    pb = dict(nx=12, ny=6, nz=12, mapping="cavity", Ra=1e5, Pr=0.71, phi=1.0, enthalpy=True,
              T_m=0.5, St=1.0, flow_bc=[1] * 6, heat_bc=[2, 2, 1, 1, 1, 1],
              face_T=[1.0, 0.0, 0, 0, 0, 0], T_init=0.0, T0=0.5)
    lp = orc.map_problem(pb)
    o = orc.Oracle(lp)
    o.step(1500)
    _, u, T = o.macros()  # same time level: T below T_m means f_l = 0 (Eq. B9)
    solid = T < lp.T_s - 1e-9
    liquid = T > lp.T_l + 1e-9
    assert solid.any() and liquid.any()
    assert np.abs(u[:, solid]).max() == 0.0
    assert np.abs(u[:, liquid]).max() > 1e-5


def test_flow_gate_is_at_half_liquid(orc):
    """The flow gate of the enthalpy model (a reading: App. B gives the thermal model only) at
    one site: under a body force a mushy site with f_l just below 1/2 keeps no velocity and its
    flow populations rest at f_eq(rho, 0); just above 1/2 it flows."""
    lp = _params(orc, T_m=0.5, St=0.5, accel=[1e-4, 0.0, 0.0], K=10.0, phi=1.0)
    f = orc.feq19(1.0, np.zeros(3), 1.0, 1.0)
    for fl, flows in ((0.45, False), (0.55, True)):
        En = lp.sigma_s * lp.c_pl * 0.5 + fl * lp.L_a
        g = orc.geq7_enthalpy(lp, En, 0.5, np.zeros(3))
        fo, _, mac = orc.collide_site(lp, f, g)
        if flows:
            assert mac[1] > 1e-6
        else:
            assert np.abs(mac[1:4]).max() == 0.0 and np.allclose(fo, f, atol=1e-15)


def test_gate_margin_records_the_distance_of_f_l_from_one_half(orc):
    """Oracle.gate_margin: in a closed adiabatic box at rest with a uniform mushy enthalpy
    (f_l = 0.3 or 0.62 by Eq. B9) nothing changes, so after a step every site's margin is
    |f_l - 1/2|; phase-pure sites read 0.5; with flow_off there is no gate (0.5)."""
    pb = dict(nx=4, ny=3, nz=2, mapping="lattice", nu_e=0.1, alpha_f=0.04, enthalpy=True,
              T_m=0.0, St=1.0, T0=0.0, flow_bc=[1] * 6, heat_bc=[1] * 6)
    for flow_off in (False, True):
        lp = orc.map_problem(dict(pb, flow_off=flow_off))
        Es = lp.sigma_s * lp.c_pl * lp.T_s
        El = lp.sigma_l * lp.c_pl * lp.T_l + lp.L_a
        for fl, want in ((0.3, 0.2), (0.62, 0.12), (1.0, 0.5), (0.0, 0.5)):
            En = Es + fl * (El - Es) + (0.2 if fl == 1.0 else -0.2 if fl == 0.0 else 0.0)
            o = orc.Oracle(lp)
            f = np.broadcast_to(orc.feq19(1.0, [0, 0, 0], 1.0)[:, None, None, None],
                                (19,) + o.shape).copy()
            g = np.broadcast_to(orc.geq7_enthalpy(lp, En, 0.0, [0, 0, 0])[:, None, None, None],
                                (7,) + o.shape).copy()
            o.set_populations(f, g)
            o.step(1)
            m = o.gate_margin()
            assert np.allclose(m, 0.5 if flow_off else want, atol=1e-12), (fl, m.min(), m.max())
            o.reset_gate_margin()
            assert (o.gate_margin() == 0.5).all()
