"""FP16 / BF16 population storage (FP32 arithmetic) against the FP64 oracle.

Stored values are (f_i - w_i rho0) / w_i and (g_i - omega_i sigma T_x) / omega_i with the
site temperature T_x in an FP32 plane, rounded to nearest.  Bounds:
 - one step from the same (already rounded) state: every population within the rounding of
   its own stored value, u_r |stored| (u_r = 2^-11 FP16, 2^-8 BF16), plus 2e-6 of the largest
   deviation for the FP32 arithmetic;
 - long runs: the errors measured on GB300 with a margin of 2-3x, stated per format
   (velocity and temperature field-normalised, Nusselt relative).
"""
import numpy as np
import pytest

from lbm_inputs import cavity_problem, channel_problem, random_macros, uniform

pytestmark = pytest.mark.gpu

UNIT_ROUNDOFF = {"fp16": 2.0 ** -11, "bf16": 2.0 ** -8}
# field-normalised u error, T error, Nu relative error after the long runs below
LONG_RUN_TOL = {"fp16": (1e-2, 1.5e-3, 1e-3), "bf16": (1.5e-1, 5e-2, 8e-2)}


@pytest.fixture(scope="module")
def gb():
    import paper_1611_03329_gb300 as gb

    gb.build.build()
    gb.lib()
    return gb


def _weights(orc, lp):
    w = orc.tables()["w19"].reshape(19, 1, 1, 1)
    om = np.array([1 - lp.varpi] + [lp.varpi / 6] * 6).reshape(7, 1, 1, 1)
    return w, om


CASES = {
    "cavity": dict(cavity_problem(13, Ra=1e4, Da=1e-2, phi=0.6, Pr=0.71), ny=11, nz=9),
    "channel": channel_problem(19, 10, 7, Da=1e-2),
    "periodic_sigma": dict(nx=21, ny=6, nz=5, mapping="lattice", nu_e=0.05, alpha_f=0.03,
                           gbeta=2e-3, phi=0.5, K=2.0, F_phi=0.4, sigma=1.7,
                           accel=[2e-4, -1e-4, 5e-5]),
}


@pytest.mark.parametrize("storage", ["fp16", "bf16"])
@pytest.mark.parametrize("name", sorted(CASES))
def test_single_step_within_rounding(gb, orc, storage, name):
    pb = dict(CASES[name], storage=storage)
    lp = orc.map_problem(pb)
    o = orc.Oracle(lp)
    rho, u, T = random_macros(lp.nx, lp.ny, lp.nz, 11, u_amp=0.03)
    o.init_equilibrium(0.5, T, u)
    f, g = o.populations()
    f = f + 3e-4 * uniform(f.shape, 12)
    g = g + 3e-4 * uniform(g.shape, 13)
    lat = gb.Lattice(pb)
    lat.set_populations(f, g)
    fq, gq = lat.populations()  # the rounded state both sides start from
    w, om = _weights(orc, lp)
    ur = UNIT_ROUNDOFF[storage]
    # round trip: each value within the rounding of its stored form
    Tq = gq.sum(axis=0, keepdims=True) / lp.sigma
    sub = 3e-8  # half the spacing of FP16 subnormals (stored units)
    assert np.all(np.abs(fq - f) <= ur * np.abs(f - w * lp.rho0) * 1.001 + sub * w)
    assert np.all(np.abs(gq - g) <= ur * np.abs(g - om * lp.sigma * Tq) * 1.001 + 1e-6 * om)
    o.set_populations(fq, gq)
    lat.step(1)
    o.step(1)
    fa, ga = lat.populations()
    fb, gb_ = o.populations()
    Tb = gb_.sum(axis=0, keepdims=True) / lp.sigma
    dev_f = np.abs(fb - w * lp.rho0)
    dev_g = np.abs(gb_ - om * lp.sigma * Tb)
    assert np.all(np.abs(fa - fb) <= ur * dev_f + 2e-6 * dev_f.max() + sub * w)
    assert np.all(np.abs(ga - gb_) <= ur * dev_g + 2e-6 * np.abs(gb_ - om * lp.sigma * lp.T0).max())


def _long_run(gb, orc, pb, steps, storage):
    lat = gb.Lattice(dict(pb, storage=storage))
    lat.step(steps)
    o = orc.Oracle(orc.map_problem(pb))
    o.step(steps)
    _, ug, Tg = lat.macros()
    _, uo, To = o.macros()
    return lat, o, orc.field_error(ug, uo), orc.field_error(Tg, To), To


@pytest.mark.parametrize("storage", ["fp16", "bf16"])
@pytest.mark.parametrize("Ra,phi", [(1e3, 0.6), (1e5, 0.8)])
def test_cavity_32_5000_steps(gb, orc, storage, Ra, phi):
    pb = cavity_problem(32, Ra=Ra, Da=1e-2, phi=phi, Pr=1.0 if Ra == 1e3 else 0.71)
    lat, o, eu, eT, To = _long_run(gb, orc, pb, 5000, storage)
    tu, tT, tnu = LONG_RUN_TOL[storage]
    assert eu < tu and eT < tT, (eu, eT)
    nu_g = lat.nusselt(0)[0]
    nu_o = orc.nusselt(To, 0, 1.0, 32)[0]
    assert abs(nu_g - nu_o) / nu_o < tnu, (nu_g, nu_o)


@pytest.mark.parametrize("storage", ["fp16", "bf16"])
def test_channel_64x16x16_2000_steps(gb, orc, storage):
    _, _, eu, eT, _ = _long_run(gb, orc, channel_problem(64, 16, 16), 2000, storage)
    tu, tT, _ = LONG_RUN_TOL[storage]
    assert eu < tu and eT < tT, (eu, eT)


@pytest.mark.parametrize("storage", ["fp16", "bf16"])
def test_closed_cavity_mass_and_heat(gb, storage):
    """Bounce-back keeps the total mass to the rounding of the stored deviations; the sums
    agree with the host-side totals of the same state."""
    pb = dict(cavity_problem(16, Ra=1e5, Da=1e-2, phi=0.8, Pr=0.71), storage=storage)
    lat = gb.Lattice(pb)
    lat.step(500)
    m, h = lat.sums()
    f, g = lat.populations()
    assert m == pytest.approx(f.sum() - f[0].size, abs=1e-6 * f[0].size)
    assert h == pytest.approx(g.sum() - g[0].size * 0.5, abs=1e-6 * g[0].size)
    assert abs(m) < 1e-3 * f[0].size
