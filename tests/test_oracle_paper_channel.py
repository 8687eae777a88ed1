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


def steady(orc, ny, Re, Da):
    o = orc.Oracle(orc.map_problem(paper_channel(ny, Re=Re, Da=Da)))
    o.step(max(2000, int(40 * ny / (0.01 * Re))))  # 40 advective times of the injection
    _, u, T = o.macros()
    return u[:, 0, :, 0], T[0, :, 0]


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
