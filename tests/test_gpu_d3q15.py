"""The D3Q15-MRT flow lattice (Sec. 3.1.1) on the GPU, through the C ABI, against the FP64
oracle: one step from random near-equilibrium states on every boundary kind, long runs, the
paper's channel (Sec. 4.1, which the paper runs on D3Q15) up to H = 128, diagnostics, and the
combinations the library declines.  Tolerances as for D3Q19 (FP32 storage of deviations)."""
import math
import zlib

import numpy as np
import pytest

from lbm_inputs import (cavity_problem, channel_problem, paper_channel, porosity_field,
                        random_macros, uniform)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gb():
    import paper_1611_03329_gb300 as gb

    gb.build.build()
    gb.lib()
    return gb


def q15(pb):
    return dict(pb, q=15)


CASES = {
    "cavity_ragged": q15(dict(cavity_problem(13, Ra=1e4, Da=1e-2, phi=0.6, Pr=0.71), ny=11, nz=9)),
    "channel_ragged": q15(channel_problem(19, 10, 7, Da=1e-2)),
    "periodic_forced": q15(dict(nx=37, ny=5, nz=3, mapping="lattice", nu_e=0.05, alpha_f=0.03,
                                gbeta=2e-3, phi=0.5, K=2.0, F_phi=0.4,
                                accel=[2e-4, -1e-4, 5e-5])),
    "moving_lid": q15(dict(cavity_problem(9, Ra=1e4, Da=None, phi=1.0, Pr=0.71), nz=7,
                           flow_bc=[1, 1, 1, 1, 1, 2],
                           face_u=[(0, 0, 0)] * 5 + [(0.02, -0.01, 0.0)])),
    "paper_channel": q15(paper_channel(12, nx=5, nz=4)),
    "hetero_phi": q15(dict(cavity_problem(12, Ra=1e5, Da=1e-2, phi=0.6, Pr=0.71,
                                          phi_field=porosity_field(12, 10, 8, seed=11)
                                          .astype(np.float32).astype(np.float64),
                                          alpha_m=0.02), ny=10, nz=8)),
    "tiny_3": q15(cavity_problem(3, Ra=1e4, Da=1e-2, phi=0.6)),
}


def _state(orc, pb, seed):
    lp = orc.map_problem(pb)
    o = orc.Oracle(lp)
    _, u, T = random_macros(lp.nx, lp.ny, lp.nz, seed, u_amp=0.03)
    o.init_equilibrium(0.5, T, u)
    f, g = o.populations()
    assert f.shape[0] == 15
    f = f + 3e-4 * uniform(f.shape, seed + 1)
    g = g + 3e-4 * uniform(g.shape, seed + 2)
    return lp, o, f, g


def _dev_err(orc, lp, fa, ga, fb, gb_):
    w = orc.tables15()["w15"].reshape(15, 1, 1, 1) * lp.rho0
    om = (np.array([1 - lp.varpi] + [lp.varpi / 6] * 6) * lp.sigma * lp.T0).reshape(7, 1, 1, 1)
    return (np.abs(fa - fb).max() / np.abs(fb - w).max(),
            np.abs(ga - gb_).max() / np.abs(gb_ - om).max())


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
    fb, gb_ = o.populations()
    ef, eg = _dev_err(orc, lp, fa, ga, fb, gb_)
    tol = 1e-5 if steps == 1 else 4e-5
    assert ef < tol and eg < tol, (ef, eg)


def test_cavity_long_run(gb, orc):
    pb = q15(cavity_problem(24, Ra=1e4, Da=1e-2, phi=0.8, Pr=0.71))
    lat = gb.Lattice(pb)
    lat.step(3000)
    o = orc.Oracle(orc.map_problem(pb))
    o.step(3000)
    _, ug, Tg = lat.macros()
    _, uo, To = o.macros()
    assert orc.field_error(ug, uo) < 1e-5 and orc.field_error(Tg, To) < 1e-5
    nu_g = lat.nusselt(0)[0]
    assert nu_g == pytest.approx(orc.nusselt(To, 0, 1.0, 24)[0], rel=1e-5)
    m_g, h_g = lat.sums()
    fo, go = o.populations()
    assert m_g == pytest.approx(fo.sum() - lp_ns(pb), abs=1e-3)


def lp_ns(pb):
    return pb["nx"] * pb["ny"] * pb["nz"]  # rho0 = 1


def test_paper_grid_matches_oracle(gb, orc):
    pb = q15(paper_channel(32, Re=10.0, Da=1e-2, nx=6, nz=6))
    lat = gb.Lattice(pb)
    lat.step(12800)
    o = orc.Oracle(orc.map_problem(pb))
    o.step(12800)
    _, ug, Tg = lat.macros()
    _, uo, To = o.macros()
    assert orc.field_error(ug, uo) < 1e-5 and orc.field_error(Tg, To) < 1e-5


def test_paper_channel_second_order_to_h128(gb):
    Re, Da, phi = 10.0, 1e-2, 0.6
    errs = []
    for ny in (16, 32, 64, 128):
        lat = gb.Lattice(q15(paper_channel(ny, Re=Re, Da=Da)))
        lat.step(int(40 * ny / (0.01 * Re)))
        _, u, T = lat.macros()
        y = (np.arange(ny) + 0.5) / ny
        t1 = Re / (2 * phi)
        t2 = math.sqrt(Re * Re + 4 * phi ** 3 / Da) / (2 * phi)
        ua = 0.01 * np.exp(t1 * (y - 1)) * np.sinh(t2 * y) / math.sinh(t2)
        Ta = (np.exp(Re * y) - 1) / (math.exp(Re) - 1)
        ux, TT = u[0, 0, :, 0], T[0, :, 0]
        errs.append((math.sqrt(np.sum((ux - ua) ** 2) / np.sum(ua ** 2)),
                     math.sqrt(np.sum((TT - Ta) ** 2) / np.sum(Ta ** 2))))
        lat.close()
    for (a0, b0), (a1, b1) in zip(errs, errs[1:]):
        assert math.log2(a0 / a1) > 1.8 and math.log2(b0 / b1) > 1.8


def test_declined_combinations(gb):
    pb = q15(cavity_problem(8, Ra=1e4, Da=1e-2, phi=0.7))
    for bad in (dict(pb, storage="fp16"), dict(pb, q=17),
                dict(pb, enthalpy=True, heat_bc=[2, 2, 1, 1, 1, 1])):
        with pytest.raises(gb.LbmError):
            gb.derive_lattice(bad)
    assert gb.derive_lattice(pb)["q"] == 15
    srv = gb.Server(chunk=100)  # the serving loop takes it and steps it alone
    rid = srv.submit(pb, tol=1e-14, max_steps=200)
    done = []
    for _ in range(10):
        na, nq = srv.advance()
        done += srv.poll()
        if na == 0 and nq == 0:
            break
    srv.close()
    assert [r["id"] for r in done] == [rid] and done[0]["status"] == "max_steps"
