"""The oracle against the closed form of the paper's porous channel (Sec. 4.1, Eqs. 44-50):
moving hot upper plate, injection through the cold lower plate and withdrawal through the upper
one, periodic in x and z.  At steady state u_x follows Eq. 48 with Eq. 50, u_y = u1 and T
follows Eq. 49; the relative global error E of Eq. 52 falls at second order with the grid, as
the paper states for its model."""
import math

import numpy as np
import pytest

from lbm_inputs import paper_channel


def exact(ny, Re, Da, phi=0.6, u0=0.01, Pr=1.0, J=1.0):
    """Eqs. 48-50 at the nodes of a lattice with halfway walls: y = (j + 1/2) / H, H = ny."""
    y = (np.arange(ny) + 0.5) / ny
    t1 = Re / (2.0 * phi * J)
    t2 = math.sqrt(Re * Re + 4.0 * phi ** 3 * J / Da) / (2.0 * phi * J)
    ux = u0 * np.exp(t1 * (y - 1.0)) * np.sinh(t2 * y) / math.sinh(t2)
    T = (np.exp(Pr * Re * y) - 1.0) / (math.exp(Pr * Re) - 1.0)
    return ux, T


def E(a, ref):
    """Relative global error, Eq. 52."""
    return math.sqrt(float(np.sum((a - ref) ** 2)) / float(np.sum(ref ** 2)))


_STEADY = {}


def steady(orc, ny, Re, Da, full=False):
    if (ny, Re, Da) not in _STEADY:
        o = orc.Oracle(orc.map_problem(paper_channel(ny, Re=Re, Da=Da)))
        o.step(max(2000, int(40 * ny / (0.01 * Re))))  # 40 advective times of the injection
        _STEADY[(ny, Re, Da)] = o.macros()
    _, u, T = _STEADY[(ny, Re, Da)]
    return T if full else (u[:, 0, :, 0], T[0, :, 0])


@pytest.mark.parametrize("Re,Da", [(10.0, 1e-2), (5.0, 1e-1)])
def test_second_order_convergence(orc, Re, Da):
    errs = []
    for ny in (16, 32, 64):
        u, T = steady(orc, ny, Re, Da)
        ua, Ta = exact(ny, Re, Da)
        assert np.abs(u[1] - 0.01).max() < 1e-8  # u_y = u1 (Eq. 48)
        assert np.abs(u[2]).max() < 1e-12
        errs.append((E(u[0], ua), E(T, Ta)))
    assert errs[1][0] < 0.05 and errs[1][1] < 0.02
    for (eu0, et0), (eu1, et1) in zip(errs, errs[1:]):
        assert math.log2(eu0 / eu1) > 1.8 and math.log2(et0 / et1) > 1.8


def test_closed_form_is_a_solution():
    """Eq. 48 solves Eq. 44 and Eq. 49 solves Eq. 46 (finite differences), and both meet the
    plate conditions: the pin above tests the oracle against the right function."""
    Re, Da, phi, J, H, u0, u1 = 10.0, 1e-2, 0.6, 1.0, 1.0, 1.0, 1.0
    nu = u1 * H / Re
    K = Da * H * H
    y = np.linspace(0.0, 1.0, 20001)
    h = y[1] - y[0]
    t1 = Re / (2 * phi * J)
    t2 = math.sqrt(Re * Re + 4 * phi ** 3 * J / Da) / (2 * phi * J)
    ux = u0 * np.exp(t1 * (y - 1)) * np.sinh(t2 * y) / math.sinh(t2)
    d1 = (ux[2:] - ux[:-2]) / (2 * h)
    d2 = (ux[2:] - 2 * ux[1:-1] + ux[:-2]) / h ** 2
    res = u1 / phi * d1 - (J * nu * d2 - phi * nu / K * ux[1:-1])
    assert np.abs(res).max() < 1e-5 * np.abs(phi * nu / K * ux).max()
    assert ux[0] == 0.0 and ux[-1] == pytest.approx(u0)
    T = (np.exp(Re * y) - 1) / (math.exp(Re) - 1)  # Pr_e = 1
    alpha = nu
    rT = u1 * (T[2:] - T[:-2]) / (2 * h) - alpha * (T[2:] - 2 * T[1:-1] + T[:-2]) / h ** 2
    assert np.abs(rT).max() < 1e-5 * u1 * np.abs(np.gradient(T, h)).max()



def _exact_flux(pe):
    """Heat flux into the fluid at the hot plate, in units of dT / H, of Eq. 49's profile
    T = (exp(Pe y) - 1) / (exp(Pe) - 1), Pe = Pr Re."""
    return pe * math.exp(pe) / (math.exp(pe) - 1.0)


def test_wall_heat_flux_formula_second_order(orc):
    """Eq. 53's discretisations, applied to Eq. 49's exact temperatures at the nodes of a
    halfway-wall lattice (y = (j + 1/2) / H) and of a node-wall lattice (y = j / H), converge
    to the plate's exact heat flux at second order.  The profile is exponential, so a formula
    that is exact only for linear profiles (a one-sided first-order difference) fails."""
    pe = 10.0
    for node in (False, True):
        errs = []
        for H in (32, 64, 128):
            ny = H + 1 if node else H
            y = np.arange(ny) / H if node else (np.arange(ny) + 0.5) / H
            T = ((np.exp(pe * y) - 1.0) / (math.exp(pe) - 1.0)).reshape(1, ny, 1)
            T = np.broadcast_to(T, (2, ny, 3))
            nu = orc.nusselt(T, 3, 1.0, H, node_wall=node)[0]
            errs.append(abs(nu / _exact_flux(pe) - 1.0))
        for e0, e1 in zip(errs, errs[1:]):
            assert math.log2(e0 / e1) > 1.8, (node, errs)


def test_node_wall_heat_flux_converges(orc):
    """The paper's channel with node walls (the paper's boundary scheme): the hot plate's heat
    flux from the oracle's steady field approaches Eq. 49's at second order on the last
    halving (H = 32 -> 64)."""
    Re, Da = 10.0, 1e-2
    errs = []
    for H in (16, 32, 64):
        ny = H + 1
        o = orc.Oracle(orc.map_problem(paper_channel(ny, Re=Re, Da=Da, walls="nee")))
        o.step(max(2000, int(40 * ny / (0.01 * Re))))
        _, _, T = o.macros()
        errs.append(abs(orc.nusselt(T, 3, 1.0, H, node_wall=True)[0] / _exact_flux(Re) - 1.0))
    assert errs[0] > errs[1] > errs[2] and errs[2] < 0.05, errs
    assert math.log2(errs[1] / errs[2]) > 1.8, errs
