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


KEYS = ("status", "steps", "r_u", "r_T", "nu_avg", "nu_mp", "mass_dev", "heat_dev", "storage")


def _tol(pb):
    """A tolerance each storage format can reach (above the 16-bit residual floors), so the
    16-bit requests stay 16-bit."""
    return {"fp16": 5e-4, "bf16": 5e-3}.get(pb.get("storage", "fp32"), 1e-6)


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
    ids = [srv.submit(pb, tol=_tol(pb), max_steps=2500) for pb in pbs[:3]]
    done = []
    for _ in range(3):  # three rounds with the first arrivals, then the rest arrive
        srv.advance()
        done += srv.poll()
    ids += [srv.submit(pb, tol=_tol(pb), max_steps=2500) for pb in pbs[3:]]
    done += _drain(srv)
    srv.close()
    assert sorted(r["id"] for r in done) == sorted(ids)
    mixed = {r["id"]: r for r in done}
    for rid, pb in zip(ids, pbs):
        solo = gb.Server(chunk=100)
        solo.submit(pb, tol=_tol(pb), max_steps=2500)
        (r,) = _drain(solo)
        solo.close()
        _same(mixed[rid], r)
        assert r["storage"] == pb.get("storage", "fp32")
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


def test_tolerance_below_a_16bit_floor_is_served_in_fp32(gb):
    """A 16-bit request whose tolerance lies below its format's residual floor is stored in
    FP32 (it could not converge otherwise); above the floor it keeps its format."""
    base = cavity_problem(12, Ra=1e4, Da=1e-2, phi=0.7, Pr=0.71)
    cases = [("fp16", 1e-6, "fp32"), ("fp16", 5e-4, "fp16"), ("bf16", 1e-3, "fp32"),
             ("bf16", 5e-3, "bf16"), ("fp32", 1e-6, "fp32")]
    assert gb.RESIDUAL_FLOOR["fp16"] == 2e-4 and gb.RESIDUAL_FLOOR["bf16"] == 2e-3
    srv = gb.Server(chunk=100)
    ids = {srv.submit(dict(base, storage=st), tol=tol, max_steps=200): want
           for st, tol, want in cases}
    res = _drain(srv)
    srv.close()
    for r in res:
        assert r["storage"] == ids[r["id"]], r


@pytest.mark.parametrize("policy", ["fifo", "backfill"])
def test_backfill_lets_small_requests_pass(gb, policy):
    """With a fill cap that the first request fills, a large second request waits; under
    BACKFILL a small third request that fits is admitted ahead of it, under FIFO it is not.
    Results do not depend on the policy."""
    a = cavity_problem(16, Ra=1e4, Da=1e-2, phi=0.8, Pr=0.71)
    big = cavity_problem(20, Ra=1e4, Da=1e-2, phi=0.8, Pr=0.71)
    small = cavity_problem(8, Ra=1e4, Da=1e-2, phi=0.8, Pr=0.71)
    srv = gb.Server(chunk=100, max_active_sites=16 ** 3 + 8 ** 3, policy=policy)
    ia = srv.submit(a, tol=1e-12, max_steps=400)
    ib = srv.submit(big, tol=1e-12, max_steps=200)
    ic = srv.submit(small, tol=1e-12, max_steps=200)
    res = {r["id"]: r for r in _drain(srv)}
    srv.close()
    assert res[ia]["t_admit"] < res[ib]["t_admit"]
    if policy == "backfill":
        assert res[ic]["t_admit"] < res[ib]["t_admit"]
    else:
        assert res[ic]["t_admit"] >= res[ib]["t_admit"]
    for r in res.values():
        assert r["status"] == "max_steps"


NEE, NEE_T, NEE_A = 4, 4, 5


def _variant_requests():
    nee = cavity_problem(11, Ra=1e4, Da=1e-2, phi=0.8, Pr=0.71, L=10)
    nee.update(ny=10, nz=9, flow_bc=[NEE] * 6, heat_bc=[NEE_T, NEE_T, NEE_A, NEE_A, NEE_A, NEE_A])
    return [
        dict(cavity_problem(12, Ra=1e4, Da=1e-2, phi=0.8, Pr=0.71), q=15, ny=10),  # D3Q15
        nee,                                                                         # node walls
        dict(cavity_problem(14, Ra=1e5, Da=1e-2, phi=0.6, Pr=0.71), ny=12, scheme="aa"),
        cavity_problem(16, Ra=1e4, Da=1e-2, phi=0.8, Pr=0.71),
        channel_problem(40, 10, 10, Da=1e-2),
    ]


def test_d3q15_node_wall_and_aa_requests_are_served(gb):
    """D3Q15, node-wall and AA lattices batch in groups of their own: each result is the same
    alone and in the mix, and the AA request holds one population copy."""
    pbs = _variant_requests()
    srv = gb.Server(chunk=100)
    ids = [srv.submit(pb, tol=1e-6, max_steps=1500) for pb in pbs]
    done = _drain(srv)
    srv.close()
    assert sorted(r["id"] for r in done) == sorted(ids)
    mixed = {r["id"]: r for r in done}
    for rid, pb in zip(ids, pbs):
        solo = gb.Server(chunk=100)
        solo.submit(pb, tol=1e-6, max_steps=1500)
        (r,) = _drain(solo)
        solo.close()
        _same(mixed[rid], r)
        assert r["status"] in ("converged", "max_steps"), r["status"]
    aa, pp = mixed[ids[2]], None
    solo = gb.Server(chunk=100)
    solo.submit(dict(pbs[2], scheme="pingpong"), tol=1e-6, max_steps=1500)
    (pp,) = _drain(solo)
    solo.close()
    assert aa["bytes"] < pp["bytes"]
    _same(aa, {**pp, "storage": aa["storage"]})  # the AA scheme changes no result


def test_aa_request_the_scheme_does_not_take_is_rejected(gb):
    srv = gb.Server(chunk=100)
    with pytest.raises(gb.LbmError):  # an outflow face: AA does not apply
        srv.submit(dict(channel_problem(40, 10, 10, Da=1e-2), scheme="aa"), tol=1e-6)
    with pytest.raises(gb.LbmError):  # 16-bit storage kept (tolerance above its floor)
        srv.submit(dict(cavity_problem(12, Ra=1e4, Da=1e-2, phi=0.8, Pr=0.71), scheme="aa",
                        storage="fp16"), tol=1e-3)
    srv.close()


def test_served_residuals_equal_lbm_residual(gb):
    """The server takes the residuals of its batched lattices in one launch per kernel variant
    (uniform and field media, outflow, 16-bit storage, the enthalpy model), and those of its
    batched D3Q15 and node-wall lattices one at a time: each equals, bit for bit, what
    lbm_residual gives for the same lattice after the same chunks."""
    from lbm_inputs import porosity_field

    phi = porosity_field(12, 10, 8, seed=9).astype(np.float32).astype(np.float64)
    melt = dict(nx=12, ny=6, nz=12, mapping="cavity", Ra=1e5, Pr=0.71, phi=1.0, enthalpy=True,
                T_m=0.5, St=1.0, flow_bc=[1] * 6, heat_bc=[2, 2, 1, 1, 1, 1],
                face_T=[1.0, 0.0, 0, 0, 0, 0], T_init=0.0, T0=0.5)
    pbs = [cavity_problem(12, Ra=1e5, Da=1e-2, phi=0.8, Pr=0.71),
           dict(cavity_problem(12, Ra=1e5, Da=1e-2, phi=0.6, Pr=0.71, phi_field=phi), ny=10, nz=8),
           channel_problem(32, 8, 6, Da=1e-2),
           dict(cavity_problem(14, Ra=1e4, Da=1e-2, phi=0.7, Pr=0.71), storage="fp16"),
           melt,
           dict(cavity_problem(11, Ra=1e4, Da=1e-2, phi=0.7, Pr=0.71), q=15),
           dict(cavity_problem(11, Ra=1e4, Da=1e-2, phi=0.8, Pr=0.71, L=10),
                flow_bc=[4] * 6, heat_bc=[4, 4, 5, 5, 5, 5])]
    steps = 300
    srv = gb.Server(chunk=100)
    # tolerances none of them reaches in 300 steps; the FP16 one above its format's residual
    # floor, so that it is served in FP16
    ids = [srv.submit(pb, tol=2.5e-4 if pb.get("storage") == "fp16" else 1e-14, max_steps=steps)
           for pb in pbs]
    done = {r["id"]: r for r in _drain(srv)}
    srv.close()
    for rid, pb in zip(ids, pbs):
        lat = gb.Lattice(pb)
        for _ in range(steps // 100):
            lat.step(100)
            ru, rT = lat.residual()
        lat.close()
        r = done[rid]
        assert r["steps"] == steps and r["storage"] == pb.get("storage", "fp32")
        assert r["r_u"] == ru and r["r_T"] == rT, (pb.get("storage"), r["r_u"], ru, r["r_T"], rT)
