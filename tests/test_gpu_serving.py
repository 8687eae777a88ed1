"""Serving loop: requests admitted by device footprint, advanced together in chunks, retired
at steady state; each request's result is the same alone and in the mix."""
import math

import numpy as np
import pytest

from lbm_inputs import cavity_problem, channel_problem

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gb():
    import paper_1611_03329_gb300 as gb

    gb.build.build()
    gb.lib()
    return gb


def _requests():
    return [
        cavity_problem(16, Ra=1e4, Da=1e-2, phi=0.8, Pr=0.71),
        dict(cavity_problem(20, Ra=1e5, Da=1e-2, phi=0.6, Pr=0.71), storage="fp16"),
        channel_problem(48, 12, 12, Da=1e-2),
        dict(cavity_problem(12, Ra=1e3, Da=1e-1, phi=0.7, Pr=1.0), ny=10),
        cavity_problem(24, Ra=5e4, Da=1e-3, phi=0.5, Pr=0.71),
        dict(cavity_problem(14, Ra=1e4, Da=1e-2, phi=0.6, Pr=0.71), storage="bf16"),
    ]


KEYS = ("status", "steps", "r_u", "r_T", "nu_avg", "nu_mp", "mass_dev", "heat_dev")


def _drain(srv, limit=10000):
    out = []
    for _ in range(limit):
        na, nq = srv.advance()
        out += srv.poll()
        if na == 0 and nq == 0:
            break
    return out


def _same(a, b):
    for k in KEYS:
        va, vb = a[k], b[k]
        if isinstance(va, float) and math.isnan(va):
            assert math.isnan(vb), k
        else:
            assert va == vb, (k, va, vb)


def test_result_is_the_same_alone_and_in_the_mix(gb):
    pbs = _requests()
    srv = gb.Server(chunk=100)
    ids = [srv.submit(pb, tol=1e-6, max_steps=2500) for pb in pbs[:3]]
    done = []
    for _ in range(3):  # three rounds with the first arrivals, then the rest arrive
        srv.advance()
        done += srv.poll()
    ids += [srv.submit(pb, tol=1e-6, max_steps=2500) for pb in pbs[3:]]
    done += _drain(srv)
    srv.close()
    assert sorted(r["id"] for r in done) == sorted(ids)
    mixed = {r["id"]: r for r in done}
    for rid, pb in zip(ids, pbs):
        solo = gb.Server(chunk=100)
        solo.submit(pb, tol=1e-6, max_steps=2500)
        (r,) = _drain(solo)
        solo.close()
        _same(mixed[rid], r)
        assert r["status"] in ("converged", "max_steps")
        assert r["steps"] % 100 == 0 and 200 <= r["steps"] <= 2500
        assert mixed[rid]["t_done"] >= mixed[rid]["t_admit"] >= mixed[rid]["t_submit"]


def test_admission_respects_the_budget(gb):
    pbs = [cavity_problem(24, Ra=1e4, Da=1e-2, phi=0.8, Pr=0.71) for _ in range(5)]
    fp = gb.footprint(pbs[0])
    srv = gb.Server(budget_bytes=2 * fp + fp // 2, chunk=50)
    ids = [srv.submit(pb, tol=1e-12, max_steps=300) for pb in pbs]
    seen = 0
    done = []
    for _ in range(1000):
        na, nq = srv.advance()
        seen = max(seen, na)
        assert na <= 2
        done += srv.poll()
        if na == 0 and nq == 0:
            break
    srv.close()
    assert seen == 2
    assert [r["id"] for r in sorted(done, key=lambda r: r["t_admit"])] == ids  # FIFO
    assert all(r["status"] == "max_steps" and r["steps"] == 300 for r in done)
    with pytest.raises(gb.LbmError):
        gb.Server(budget_bytes=fp // 2).submit(pbs[0])


def test_conduction_request_converges(gb):
    pb = dict(nx=10, ny=4, nz=4, mapping="lattice", nu_e=0.1, alpha_f=0.2, gbeta=0.0,
              flow_bc=[1] * 6, heat_bc=[2, 2, 1, 1, 1, 1], face_T=[1, 0, 0, 0, 0, 0], T_init=0.5)
    srv = gb.Server(chunk=100)
    srv.submit(pb, tol=1e-6, max_steps=50000)
    (r,) = _drain(srv)
    srv.close()
    assert r["status"] == "converged" and r["r_T"] < 1e-6
    assert r["nu_avg"] == pytest.approx(1.0, abs=1e-3)  # exact conduction value at steady state


def test_unstable_request_is_reported_alone(gb):
    # near-inviscid walled box driven by a huge wall temperature difference: blows up
    bad = dict(nx=8, ny=8, nz=8, mapping="lattice", nu_e=1e-4, alpha_f=1e-4, gbeta=1.0,
               flow_bc=[1] * 6, heat_bc=[2, 2, 1, 1, 1, 1], face_T=[100.0, -100.0, 0, 0, 0, 0],
               T_init=0.0, T0=0.0)
    good = cavity_problem(12, Ra=1e4, Da=1e-2, phi=0.8, Pr=0.71)
    srv = gb.Server(chunk=100)
    ib = srv.submit(bad, tol=1e-9, max_steps=3000)
    ig = srv.submit(good, tol=1e-9, max_steps=600)
    res = {r["id"]: r for r in _drain(srv)}
    srv.close()
    assert res[ib]["status"] == "unstable"
    assert res[ig]["status"] == "max_steps" and np.isfinite(res[ig]["nu_avg"])
