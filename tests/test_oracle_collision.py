"""Pins of the oracle's one-site collision (Eqs. 9, 34) against its invariants."""
import math

import numpy as np
import pytest


def _params(orc, **kw):
    pb = dict(nx=1, ny=1, nz=1, mapping="lattice", nu_e=0.08, alpha_f=0.05, phi=0.7,
              K=3.0, F_phi=0.4, gbeta=2e-3, gravity_axis=2, gravity_sign=-1, T0=0.5)
    pb.update(kw)
    return orc.map_problem(pb)


def _state(orc, seed, phi=0.7):
    rng = np.random.default_rng(seed)
    f = orc.feq19(1 + 0.01 * rng.uniform(-1, 1), 0.04 * rng.uniform(-1, 1, 3), phi)
    f = f + 2e-3 * rng.uniform(-1, 1, 19)
    g = orc.geq7(rng.uniform(0, 1), 0.04 * rng.uniform(-1, 1, 3)) + 2e-3 * rng.uniform(-1, 1, 7)
    return f, g


def test_equilibrium_is_a_fixed_point(orc):
    """With no force (no medium, no buoyancy) f = f_eq and g = g_eq are unchanged."""
    lp = _params(orc, phi=1.0, K=0.0, Da=None, F_phi=0.0, gbeta=0.0)
    assert math.isinf(lp.K)
    u = np.array([0.02, -0.03, 0.01])
    f = orc.feq19(1.003, u, 1.0)
    g = orc.geq7(0.7, u)
    fo, go, mac = orc.collide_site(lp, f, g)
    assert np.allclose(fo, f, atol=1e-16) and np.allclose(go, g, atol=1e-16)
    assert np.allclose(mac[1:4], u, atol=1e-17)


@pytest.mark.parametrize("seed", range(4))
def test_collision_conserves_mass_and_heat(orc, seed):
    lp = _params(orc)
    f, g = _state(orc, seed)
    fo, go, _ = orc.collide_site(lp, f, g)
    assert fo.sum() == pytest.approx(f.sum(), abs=1e-15)
    assert go.sum() == pytest.approx(g.sum(), abs=1e-15)


@pytest.mark.parametrize("s_j", [1.0, 0.7, 1.6])
def test_post_collision_momentum(orc, s_j):
    """sum e f* = rho0 u + rho0 F / 2 for any s_j (Eqs. 9, 14, 26)."""
    lp = _params(orc)
    s = list(lp.s)
    s[3] = s[5] = s[7] = s_j
    lp.s = s
    f, g = _state(orc, 7)
    fo, go, mac = orc.collide_site(lp, f, g)
    u = mac[1:4]
    T = mac[4]
    G = np.array(lp.buoy) * (T - lp.T0)
    F = orc.force(u, G, lp.phi, lp.nu, lp.K, lp.F_phi)
    e = orc.tables()["e19"]
    assert np.allclose(e @ fo, u + 0.5 * F, atol=1e-16)


def test_temperature_equilibrium_fixed_point(orc):
    """g = g_eq(T, u) with u the flow's own velocity is a fixed point of Eq. 34."""
    lp = _params(orc, gbeta=0.0, K=0.0, Da=None, phi=1.0, F_phi=0.0)
    u = np.array([0.01, 0.02, -0.03])
    f = orc.feq19(1.0, u, 1.0)
    g = orc.geq7(0.3, u) * 1.0
    fo, go, mac = orc.collide_site(lp, f, g)
    assert np.allclose(go, g, atol=1e-16)


def test_relaxation_rates_act_on_their_moments(orc):
    """A non-equilibrium part in one moment relaxes by exactly (1 - s_k): perturb the
    energy-squared moment and the temperature moment n5 and check both decays."""
    lp = _params(orc, gbeta=0.0, K=0.0, Da=None, phi=1.0, F_phi=0.0, s_eps=0.6, zeta_nu=1.3)
    t = orc.tables()
    u = np.zeros(3)
    f = orc.feq19(1.0, u, 1.0) + 1e-3 * t["Minv"][:, 2]
    g = orc.geq7(0.5, u) + 1e-3 * t["Ninv"][:, 5]
    fo, go, _ = orc.collide_site(lp, f, g)
    m_neq = t["M"] @ (fo - orc.feq19(1.0, u, 1.0))
    n_neq = t["N"] @ (go - orc.geq7(0.5, u))
    assert m_neq[2] == pytest.approx(1e-3 * (1 - 0.6), rel=1e-12)
    assert n_neq[5] == pytest.approx(1e-3 * (1 - 1.3), rel=1e-12)
    assert np.allclose(np.delete(m_neq, 2), 0, atol=5e-15)
    assert np.allclose(np.delete(n_neq, 5), 0, atol=5e-15)
