"""Node walls by non-equilibrium extrapolation (the paper's boundary scheme [50], Sec. 4) on
the GPU, through the C ABI, against the FP64 oracle: one and twenty steps from random states
on walled, transpiring, moving, heterogeneous, D3Q15 and corner-heavy lattices (wall sites
included), a long cavity run with the node-wall Nusselt number, exact conduction, the
paper's channel converging on the GPU, and the combinations the library declines."""
import math
import zlib

import numpy as np
import pytest

from lbm_inputs import cavity_problem, paper_channel, porosity_field, random_macros, uniform

pytestmark = pytest.mark.gpu

NEE, NEE_T, NEE_A = 4, 4, 5


@pytest.fixture(scope="module")
def gb():
    import paper_1611_03329_gb300 as gb

    gb.build.build()
    gb.lib()
    return gb


def nee_cavity(n, q=19, **kw):
    pb = cavity_problem(n, Ra=1e4, Da=1e-2, phi=0.8, Pr=0.71, L=n - 1, q=q, **kw)
    pb.update(flow_bc=[NEE] * 6, heat_bc=[NEE_T, NEE_T, NEE_A, NEE_A, NEE_A, NEE_A])
    return pb


CASES = {
    "cavity_ragged": dict(nee_cavity(13), ny=11, nz=9),
    "cavity_d3q15": dict(nee_cavity(12, q=15), ny=10, nz=9),
    "transpiring": paper_channel(12, nx=5, nz=4, walls="nee"),
    "transpiring_d3q15": dict(paper_channel(12, nx=5, nz=4, walls="nee"), q=15),
    "moving_hetero": dict(nx=9, ny=10, nz=7, mapping="lattice", nu_e=0.06, alpha_f=0.04, L=9,
                          gbeta=2e-3, gravity_axis=1, gravity_sign=-1, K=40.0, F_phi=0.3,
                          phi_field=porosity_field(9, 10, 7, seed=4).astype(np.float32)
                          .astype(np.float64), flow_bc=[0, 0, NEE, NEE, 0, 0],
                          heat_bc=[0, 0, NEE_T, NEE_A, 0, 0], face_T=[0, 0, 1.0, 0, 0, 0],
                          face_u=[(0, 0, 0), (0, 0, 0), (0, 0, 0), (0.03, 0, -0.01),
                                  (0, 0, 0), (0, 0, 0)]),
    "corners_3x4x3": dict(nee_cavity(3), ny=4),
}


def _state(orc, pb, seed):
    lp = orc.map_problem(pb)
    o = orc.Oracle(lp)
    _, u, T = random_macros(lp.nx, lp.ny, lp.nz, seed, u_amp=0.03)
    o.init_equilibrium(0.5, T, u)
    f, g = o.populations()
    return lp, o, f + 3e-4 * uniform(f.shape, seed + 1), g + 3e-4 * uniform(g.shape, seed + 2)


@pytest.mark.parametrize("name", sorted(CASES))
@pytest.mark.parametrize("steps", [1, 20])
def test_steps_from_random_state(gb, orc, name, steps):
    pb = CASES[name]
    lp, o, f, g = _state(orc, pb, zlib.crc32(name.encode()) % 1000)
    lat = gb.Lattice(pb)
    lat.set_populations(f, g)
    o.set_populations(f, g)
    rg, ug, Tg = lat.macros()
    ro, uo, To = o.macros()
    assert orc.field_error(ug, uo) < 1e-5 and orc.field_error(Tg, To) < 1e-5
    assert np.abs(rg - ro).max() < 1e-6
    lat.step(steps)
    o.step(steps)
    fa, ga = lat.populations()
    fb, gbo = o.populations()
    w = (orc.tables15()["w15"] if lp.q == 15 else orc.tables()["w19"]).reshape(-1, 1, 1, 1)
    om = np.array([1 - lp.varpi] + [lp.varpi / 6] * 6).reshape(7, 1, 1, 1) * lp.sigma * lp.T0
    tol = 1e-5 if steps == 1 else 4e-5
    assert np.abs(fa - fb).max() < tol * np.abs(fb - w).max()
    assert np.abs(ga - gbo).max() < tol * np.abs(gbo - om).max()


def test_cavity_long_run_and_nusselt(gb, orc):
    pb = nee_cavity(25)
    lat = gb.Lattice(pb)
    lat.step(3000)
    o = orc.Oracle(orc.map_problem(pb))
    o.step(3000)
    _, ug, Tg = lat.macros()
    _, uo, To = o.macros()
    assert orc.field_error(ug, uo) < 1e-5 and orc.field_error(Tg, To) < 1e-5
    # the node-wall stencil L (3 T_w - 4 T_1 + T_2) / 2 turns a temperature error e into up to
    # 2.5 L e = 60 e on Nu (L = 24): with e ~ 1e-6 (FP32 state), 1e-4 relative
    for face, Tw in ((0, 1.0), (1, 0.0)):
        nu_g, prof_g, mp_g = lat.nusselt(face)
        nu_o, prof_o, mp_o = orc.nusselt(To, face, Tw, 24, node_wall=True)
        assert nu_g == pytest.approx(nu_o, rel=1e-4) and mp_g == pytest.approx(mp_o, rel=1e-4)
        assert np.allclose(prof_g, prof_o, rtol=1e-4)


def test_conduction_is_exact(gb):
    N = 16
    pb = dict(nx=N, ny=6, nz=3, mapping="lattice", nu_e=0.1, alpha_f=0.2, gbeta=0.0, L=N - 1,
              flow_bc=[NEE, NEE, NEE, NEE, 0, 0], heat_bc=[NEE_T, NEE_T, NEE_A, NEE_A, 0, 0],
              face_T=[1.0, 0.0, 0, 0, 0, 0], T_init=0.5)
    lat = gb.Lattice(pb)
    lat.step(8000)
    _, u, T = lat.macros()
    assert np.abs(T - (1.0 - np.arange(N) / (N - 1))[None, None, :]).max() < 2e-6
    assert lat.nusselt(0)[0] == pytest.approx(1.0, abs=1e-4)


@pytest.mark.parametrize("q", [19, 15])
def test_paper_channel_converges_to_h128(gb, q):
    Re, Da, phi = 10.0, 1e-2, 0.6
    errs = []
    for ny in (17, 33, 65, 129):
        H = ny - 1
        uw = 0.16 / H
        lat = gb.Lattice(dict(paper_channel(ny, Re=Re, Da=Da, u0=uw, u1=uw, walls="nee"), q=q))
        lat.step(int(40 * H / (uw * Re)))
        _, u, T = lat.macros()
        y = np.arange(ny) / H
        t1 = Re / (2 * phi)
        t2 = math.sqrt(Re * Re + 4 * phi ** 3 / Da) / (2 * phi)
        ua = uw * np.exp(t1 * (y - 1)) * np.sinh(t2 * y) / math.sinh(t2)
        Ta = (np.exp(Re * y) - 1) / (math.exp(Re) - 1)
        errs.append((math.sqrt(np.sum((u[0, 0, :, 0] - ua) ** 2) / np.sum(ua ** 2)),
                     math.sqrt(np.sum((T[0, :, 0] - Ta) ** 2) / np.sum(Ta ** 2))))
        lat.close()
    for (a0, b0), (a1, b1) in zip(errs, errs[1:]):
        assert a1 < a0 and b1 < b0, errs
    (a0, b0), (a1, b1) = errs[-2], errs[-1]
    assert math.log2(a0 / a1) > 1.6 and math.log2(b0 / b1) > 1.6, errs


def test_declined_combinations(gb):
    pb = nee_cavity(8)
    for bad in (dict(pb, storage="fp16"),
                dict(pb, heat_bc=[2, 2, NEE_A, NEE_A, NEE_A, NEE_A]),
                dict(pb, enthalpy=True),
                dict(nee_cavity(8), flow_bc=[2, 3, NEE, NEE, NEE, NEE],
                     heat_bc=[2, 3, NEE_A, NEE_A, NEE_A, NEE_A]),
                dict(nee_cavity(8), nz=2)):
        with pytest.raises(gb.LbmError):
            gb.derive_lattice(bad)
    lat = gb.Lattice(pb)
    assert lat.lattice()["node_walls"] == 1
    lat.close()
