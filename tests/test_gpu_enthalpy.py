"""The enthalpy-based phase-change model (App. B) on the GPU against the FP64 oracle."""

import numpy as np
import pytest

from lbm_inputs import random_macros, uniform

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gb():
    import paper_1611_03329_gb300 as gb

    gb.build.build()
    gb.lib()
    return gb


def _melting(ratio=2.0, N=100):
    return dict(nx=N, ny=1, nz=1, mapping="lattice", nu_e=0.1, alpha_f=0.02 * ratio,
                enthalpy=True, flow_off=True, T_m=0.0, St=1.0, alpha_ratio=ratio,
                flow_bc=[1, 1, 0, 0, 0, 0], heat_bc=[2, 2, 0, 0, 0, 0],
                face_T=[1.0, -1.0, 0, 0, 0, 0], T_init=-1.0, T0=0.0)


def _convection(n=16):
    return dict(nx=n, ny=n // 2, nz=n, mapping="cavity", Ra=1e5, Pr=0.71, phi=1.0, enthalpy=True,
                T_m=0.5, St=1.0, flow_bc=[1] * 6, heat_bc=[2, 2, 1, 1, 1, 1],
                face_T=[1.0, 0.0, 0, 0, 0, 0], T_init=0.0, T0=0.5)


def test_single_step_mixed_phases(gb, orc):
    pb = _convection(12)
    lp = orc.map_problem(pb)
    o = orc.Oracle(lp)
    _, u, T = random_macros(lp.nx, lp.ny, lp.nz, 21, u_amp=0.02, T_lo=0.2, T_hi=0.8)
    o.init_equilibrium(0.5, T, u)
    f, g = o.populations()
    f = f + 2e-4 * uniform(f.shape, 22)
    g = g + 0.3 * uniform(g.shape, 23)  # enthalpies across solid, mushy and liquid
    lat = gb.Lattice(pb)
    lat.set_populations(f, g)
    o.set_populations(f, g)
    _, ug, Tg = lat.macros()
    _, uo, To = o.macros()
    assert orc.field_error(Tg, To) < 1e-5 and orc.field_error(ug, uo) < 1e-5
    lat.step(1)
    o.step(1)
    fa, ga = lat.populations()
    fb, gbo = o.populations()
    w = orc.tables()["w19"].reshape(19, 1, 1, 1)
    assert np.abs(fa - fb).max() < 1e-5 * np.abs(fb - w).max()
    assert np.abs(ga - gbo).max() < 1e-5 * np.abs(gbo).max()


def test_two_region_melting_matches_oracle(gb, orc):
    pb = _melting(2.0)
    t = int(0.01 * 100 * 100 / 0.02)
    lat = gb.Lattice(pb)
    lat.step(t)
    o = orc.Oracle(orc.map_problem(pb))
    o.step(t)
    _, ug, Tg = lat.macros()
    _, _, To = o.macros()
    assert orc.field_error(Tg, To) < 1e-5
    assert np.abs(ug).max() == 0.0
    m, h = lat.sums()  # total enthalpy of the stored populations
    _, g = o.populations()
    assert h == pytest.approx(g.sum(), rel=1e-5)


def test_convection_melting_cavity(gb, orc):
    pb = _convection(16)
    lat = gb.Lattice(pb)
    lat.step(2000)
    o = orc.Oracle(orc.map_problem(pb))
    o.step(2000)
    _, ug, Tg = lat.macros()
    _, uo, To = o.macros()
    assert orc.field_error(Tg, To) < 1e-4
    assert orc.field_error(ug, uo) < 1e-3
    nu_g = lat.nusselt(0)[0]
    nu_o = orc.nusselt(To, 0, 1.0, 16)[0]
    assert nu_g == pytest.approx(nu_o, rel=1e-4)


def test_enthalpy_lattice_in_a_batch(gb):
    from lbm_inputs import cavity_problem

    pbs = [_convection(12), cavity_problem(12, Ra=1e4, Da=1e-2, phi=0.7, Pr=0.71), _melting(1.0, 40)]
    alone = [gb.Lattice(pb) for pb in pbs]
    batched = [gb.Lattice(pb) for pb in pbs]
    batch = gb.Batch(batched)
    batch.step(301)
    for a in alone:
        a.step(301)
    for a, b in zip(alone, batched):
        fa, ga = a.populations()
        fb, gbb = b.populations()
        assert np.array_equal(fa, fb) and np.array_equal(ga, gbb)
    batch.close()


def test_enthalpy_rejects_unsupported_setups(gb):
    with pytest.raises(gb.LbmError):
        gb.derive_lattice(dict(_melting(), storage="fp16"))
    lat = gb.Lattice(_melting())
    with pytest.raises(gb.LbmError):
        lat.set_medium(np.full((1, 1, 100), 0.5, np.float32))
