"""The paper's porous channel (Sec. 4.1) on the GPU: parity with the oracle on the paper's
6 x 32 x 6 grid, and the closed form of Eqs. 48-50 approached at second order up to
H = 128 (Eq. 52)."""
import math

import numpy as np
import pytest

from lbm_inputs import paper_channel

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gb():
    import paper_1611_03329_gb300 as gb

    gb.build.build()
    gb.lib()
    return gb


def _exact(ny, Re, Da, phi=0.6, u0=0.01, Pr=1.0, J=1.0):
    y = (np.arange(ny) + 0.5) / ny
    t1 = Re / (2.0 * phi * J)
    t2 = math.sqrt(Re * Re + 4.0 * phi ** 3 * J / Da) / (2.0 * phi * J)
    ux = u0 * np.exp(t1 * (y - 1.0)) * np.sinh(t2 * y) / math.sinh(t2)
    T = (np.exp(Pr * Re * y) - 1.0) / (math.exp(Pr * Re) - 1.0)
    return ux, T


def _E(a, ref):
    return math.sqrt(float(np.sum((a - ref) ** 2)) / float(np.sum(ref ** 2)))


def test_paper_grid_matches_oracle(gb, orc):
    pb = paper_channel(32, Re=10.0, Da=1e-2, nx=6, nz=6)
    steps = 12800
    lat = gb.Lattice(pb)
    lat.step(steps)
    o = orc.Oracle(orc.map_problem(pb))
    o.step(steps)
    _, ug, Tg = lat.macros()
    _, uo, To = o.macros()
    assert orc.field_error(ug, uo) < 1e-5 and orc.field_error(Tg, To) < 1e-5


@pytest.mark.parametrize("Re,Da", [(10.0, 1e-2), (5.0, 1e-1)])
def test_second_order_to_h128(gb, Re, Da):
    errs = []
    for ny in (16, 32, 64, 128):
        lat = gb.Lattice(paper_channel(ny, Re=Re, Da=Da))
        lat.step(max(2000, int(40 * ny / (0.01 * Re))))
        _, u, T = lat.macros()
        ua, Ta = _exact(ny, Re, Da)
        assert np.abs(u[1, 0, :, 0] - 0.01).max() < 1e-6
        errs.append((_E(u[0, 0, :, 0], ua), _E(T[0, :, 0], Ta)))
        lat.close()
    for (eu0, et0), (eu1, et1) in zip(errs, errs[1:]):
        assert math.log2(eu0 / eu1) > 1.8 and math.log2(et0 / et1) > 1.8
    assert errs[-1][0] < 3e-3 and errs[-1][1] < 1e-3
