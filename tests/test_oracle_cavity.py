"""Pins of the oracle on the porous cavity of Sec. 4.2: conservation, mirror symmetries and
the wall heat balance."""
import numpy as np
import pytest

from lbm_inputs import cavity_problem, porosity_field


def test_closed_cavity_conserves_mass(orc):
    """Halfway bounce-back closes the cavity: sum rho is constant to round-off (Eq. 29)."""
    pb = cavity_problem(8, Ra=1e4, Da=1e-2, phi=0.8, Pr=0.71)
    o = orc.Oracle(orc.map_problem(pb))
    m0 = o.macros()[0].sum()
    o.step(300)
    rho, u, T = o.macros()
    assert abs(rho.sum() - m0) < 1e-11
    assert np.abs(u).max() > 1e-4  # the flow is not trivial


def test_adiabatic_box_conserves_heat(orc):
    """With every face adiabatic, sum sigma T is constant (Eq. 39) while the flow stirs a
    non-uniform initial temperature field."""
    pb = cavity_problem(8, Ra=1e4, Da=1e-2, phi=0.7, heat_bc=[1] * 6, sigma=1.5)
    lp = orc.map_problem(pb)
    o = orc.Oracle(lp)
    z = np.arange(8).reshape(8, 1, 1) * np.ones((8, 8, 8))
    o.init_equilibrium(0.5, 0.2 + 0.6 * (z[..., ::-1] / 7) * (np.arange(8) / 7), None)
    h0 = o.macros()[2].sum()
    o.step(300)
    _, u, T = o.macros()
    assert abs(T.sum() - h0) < 1e-11
    assert np.abs(u).max() > 1e-5


def _cavity(orc, steps, **kw):
    pb = cavity_problem(10, Ra=1e4, Da=1e-2, phi=0.8, Pr=0.71)
    pb.update(ny=8)
    pb.update(kw)
    o = orc.Oracle(orc.map_problem(pb))
    o.step(steps)
    return o.macros()


def test_y_mirror_symmetry(orc):
    """Gravity along z, hot/cold along x: the solution is even in y (u_y odd)."""
    _, u, T = _cavity(orc, 400)
    assert np.abs(T - T[:, ::-1, :]).max() < 1e-13
    assert np.abs(u[1] + u[1][:, ::-1, :]).max() < 1e-15
    assert np.abs(u[0] - u[0][:, ::-1, :]).max() < 1e-15
    assert np.abs(u).max() > 1e-3


def test_x_mirror_symmetry(orc):
    """Both x walls hot: the solution is even in x (u_x odd)."""
    _, u, T = _cavity(orc, 400, face_T=[1.0, 1.0, 0, 0, 0, 0])
    assert np.abs(T - T[:, :, ::-1]).max() < 1e-13
    assert np.abs(u[0] + u[0][:, :, ::-1]).max() < 1e-15
    assert np.abs(u[2] - u[2][:, :, ::-1]).max() < 1e-15
    assert np.abs(u).max() > 1e-3


def test_z_mirror_symmetry(orc):
    """Gravity along y: the solution is even in z (u_z odd)."""
    _, u, T = _cavity(orc, 400, gravity_axis=1)
    assert np.abs(T - T[::-1]).max() < 1e-13
    assert np.abs(u[2] + u[2][::-1]).max() < 1e-15
    assert np.abs(u[0] - u[0][::-1]).max() < 1e-15


def test_steady_wall_heat_balance(orc):
    """At steady state the heat entering at the hot wall leaves at the cold wall
    (Nu_hot = -Nu_cold up to the one-sided derivative's truncation), and Nu exceeds the
    conduction value 1 once buoyancy drives a flow."""
    pb = cavity_problem(12, Ra=2e4, Da=1e-2, phi=0.8, Pr=0.71)
    lp = orc.map_problem(pb)
    o = orc.Oracle(lp)
    o.step(6000)
    _, _, T = o.macros()
    nh = orc.nusselt(T, 0, 1.0, lp.L)[0]
    nc = orc.nusselt(T, 1, 0.0, lp.L)[0]
    assert nh > 1.05
    assert abs(nh + nc) / nh < 2e-2


def test_heterogeneous_medium_conserves_mass(orc):
    """A seeded porosity field (Kozeny-Carman K(phi), Ergun F_phi(phi), Eq. 6) keeps the
    closed-cavity mass invariant and changes the flow relative to the mean porosity."""
    n = 8
    phi = porosity_field(n, n, n, seed=7)
    pb = cavity_problem(n, Ra=1e5, Da=1e-2, phi=0.6, Pr=0.71, phi_field=phi, phi_ref=0.6)
    o = orc.Oracle(orc.map_problem(pb))
    m0 = o.macros()[0].sum()
    o.step(200)
    rho, u, _ = o.macros()
    assert abs(rho.sum() - m0) < 1e-11
    pb2 = cavity_problem(n, Ra=1e5, Da=1e-2, phi=0.6, Pr=0.71)
    o2 = orc.Oracle(orc.map_problem(pb2))
    o2.step(200)
    u2 = o2.macros()[1]
    assert np.abs(u - u2).max() > 1e-3 * np.abs(u2).max()


def test_hot_fluid_rises(orc):
    """Buoyancy (Eq. 5) lifts warm fluid against gravity: in the cavity heated from the x-low
    wall, with gravity along -z, the fluid next to the hot wall moves up and the fluid next to
    the cold wall moves down (the mirror symmetries and the Nusselt numbers are the same for
    either sign, so this is the pin on it)."""
    pb = cavity_problem(10, Ra=1e4, Da=1e-2, phi=0.8, Pr=0.71)
    o = orc.Oracle(orc.map_problem(pb))
    o.step(600)
    _, u, T = o.macros()  # u[3][z][y][x]
    uz = u[2]
    assert uz[:, :, 0].mean() > 1e-5 and uz[:, :, -1].mean() < -1e-5, (uz[:, :, 0].mean(),
                                                                      uz[:, :, -1].mean())
