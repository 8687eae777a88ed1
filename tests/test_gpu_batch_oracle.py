"""Batched and served lattices against the FP64 oracle.

The batched launch (lbm_batch_step) and the serving loop (lbm_server_*) run their own
kernels (one flat grid over the blocks of many lattices, per-lattice parameter tables, graph
replays), so they are checked against the oracle directly, not only against the same lattice
stepped alone on the GPU.  Tolerances are those of the single-lattice parity tests:
 - one step from the same state: every population within 1e-5 of the largest population
   deviation (4e-5 after 20 steps), FP16 storage within the rounding of each stored value;
 - runs from the initial state: u and T within 1e-5 field-normalised;
 - the enthalpy model: sites whose f_l lies within the FP32 band of the flow gate at 1/2 are
   counted and left out (see tests/test_gpu_enthalpy.py for the band).
"""
import numpy as np
import pytest

from lbm_inputs import (cavity_problem, channel_problem, paper_channel, porosity_field,
                        random_macros,
                        uniform)

pytestmark = pytest.mark.gpu

TOL_STEP = 1e-5
TOL_FIELD = 1e-5
GATE_BAND_STEP = 1e-5


@pytest.fixture(scope="module")
def gb():
    import paper_1611_03329_gb300 as gb

    gb.build.build()
    gb.lib()
    return gb


def _hetero(n=12):
    phi = porosity_field(n, n - 2, n - 4, seed=11).astype(np.float32).astype(np.float64)
    return dict(cavity_problem(n, Ra=1e5, Da=1e-2, phi=0.6, Pr=0.71, phi_field=phi),
                ny=n - 2, nz=n - 4)


def _melting(n=12):
    return dict(nx=n, ny=n // 2, nz=n, mapping="cavity", Ra=1e5, Pr=0.71, phi=1.0, enthalpy=True,
                T_m=0.5, St=1.0, flow_bc=[1] * 6, heat_bc=[2, 2, 1, 1, 1, 1],
                face_T=[1.0, 0.0, 0, 0, 0, 0], T_init=0.0, T0=0.5)


# ragged lattices of every kernel variant that batches: uniform and field media, the outflow
# channel, a forced periodic box, a moving lid, and one-copy (AA) lattices in their own group
STEP_CASES = {
    "cavity_ragged": dict(cavity_problem(13, Ra=1e4, Da=1e-2, phi=0.6, Pr=0.71), ny=11, nz=9),
    "channel_ragged": channel_problem(19, 10, 7, Da=1e-2),
    "channel_T_out": dict(channel_problem(21, 8, 5, Da=1e-2), heat_bc=[2, 3, 2, 2, 0, 0]),
    "hetero_phi": _hetero(),
    "periodic_forced": dict(nx=37, ny=5, nz=3, mapping="lattice", nu_e=0.05, alpha_f=0.03,
                            gbeta=2e-3, phi=0.5, K=2.0, F_phi=0.4, accel=[2e-4, -1e-4, 5e-5]),
    "moving_lid": dict(cavity_problem(9, Ra=1e4, Da=None, phi=1.0, Pr=0.71), nz=7,
                       flow_bc=[1, 1, 1, 1, 1, 2], face_u=[(0, 0, 0)] * 5 + [(0.02, -0.01, 0.0)]),
    "aa_cavity": dict(cavity_problem(11, Ra=1e4, Da=1e-2, phi=0.7, Pr=0.71), ny=9, nz=8,
                      scheme="aa"),
    "aa_hetero": dict(_hetero(10), scheme="aa"),
}


def _weights(orc, lp):
    w = orc.tables()["w19"].reshape(19, 1, 1, 1) * lp.rho0
    om = (np.array([1 - lp.varpi] + [lp.varpi / 6] * 6) * lp.sigma * lp.T0).reshape(7, 1, 1, 1)
    return w, om


def _random_state(orc, pb, seed, g_noise=3e-4):
    lp = orc.map_problem(pb)
    o = orc.Oracle(lp)
    _, u, T = random_macros(lp.nx, lp.ny, lp.nz, seed, u_amp=0.03)
    o.init_equilibrium(0.5, T, u)
    f, g = o.populations()
    f = f + 3e-4 * uniform(f.shape, seed + 1)
    g = g + g_noise * uniform(g.shape, seed + 2)
    return lp, o, f, g


def _step_errors(orc, lp, lat, o):
    fa, ga = lat.populations()
    fb, gbo = o.populations()
    w, om = _weights(orc, lp)
    return (np.abs(fa - fb).max() / np.abs(fb - w).max(),
            np.abs(ga - gbo).max() / np.abs(gbo - om).max())


def test_batch_steps_match_oracle(gb, orc):
    """Eight lattices of six kernel variants in one batch, each from its own seeded random
    state: every population after one batched step, and after 19 more (two graph replays of
    different length), against the oracle."""
    names = sorted(STEP_CASES)
    lats, runs = [], []
    for k, name in enumerate(names):
        lp, o, f, g = _random_state(orc, STEP_CASES[name], seed=40 + 7 * k)
        lat = gb.Lattice(STEP_CASES[name])
        lat.set_populations(f, g)
        o.set_populations(f, g)
        lats.append(lat)
        runs.append((lp, o))
    assert [l.lattice()["scheme"] for l in lats].count(1) == 2  # the AA lattices
    batch = gb.Batch(lats)
    batch.step(1)
    for name, lat, (lp, o) in zip(names, lats, runs):
        o.step(1)
        ef, eg = _step_errors(orc, lp, lat, o)
        assert ef < TOL_STEP and eg < TOL_STEP, (name, ef, eg)
    batch.step(12)
    batch.step(7)
    for name, lat, (lp, o) in zip(names, lats, runs):
        o.step(19)
        ef, eg = _step_errors(orc, lp, lat, o)
        assert ef < 4 * TOL_STEP and eg < 4 * TOL_STEP, (name, ef, eg)
        assert lat.steps == 20
    batch.close()


def _node_walls(pb):
    nee, nee_t, nee_a = 4, 4, 5  # LBM_FLOW_NEE, LBM_HEAT_NEE_DIRICHLET, LBM_HEAT_NEE_ADIABATIC
    return dict(pb, flow_bc=[nee] * 6, heat_bc=[nee_t, nee_t, nee_a, nee_a, nee_a, nee_a])


# the paper-fidelity lattices of Secs. 3.1.1 and 4: D3Q15 with halfway walls (a field medium,
# the outflow channel), node walls by non-equilibrium extrapolation on D3Q19 and D3Q15 (a
# ragged cavity, the paper's transpiring channel, a field medium), beside a D3Q19 lattice
VARIANT_CASES = {
    "d3q15_hetero": dict(cavity_problem(12, Ra=1e5, Da=1e-2, phi=0.6, Pr=0.71,
                                        phi_field=porosity_field(12, 10, 8, seed=5)
                                        .astype(np.float32).astype(np.float64)),
                         ny=10, nz=8, q=15),
    "d3q15_channel": dict(channel_problem(19, 10, 7, Da=1e-2), q=15),
    "nee_cavity": dict(_node_walls(cavity_problem(13, Ra=1e4, Da=1e-2, phi=0.8, Pr=0.71, L=12)),
                       ny=11, nz=9),
    "nee_d3q15_channel": dict(paper_channel(12, nx=5, nz=4, walls="nee"), q=15),
    "nee_hetero": dict(_node_walls(cavity_problem(10, Ra=1e5, Da=1e-2, phi=0.6, Pr=0.71, L=9,
                                                  phi_field=porosity_field(10, 9, 8, seed=6)
                                                  .astype(np.float32).astype(np.float64))),
                       ny=9, nz=8),
    "d3q19_cavity": dict(cavity_problem(11, Ra=1e4, Da=1e-2, phi=0.7, Pr=0.71), ny=9, nz=8),
}


def test_batch_d3q15_and_node_walls_match_oracle(gb, orc):
    """D3Q15 and node-wall lattices advance in the batched launch (groups of their own): every
    population after one batched step and after 19 more (two graph replays) against the oracle,
    and bit for bit the same as the lattice stepped alone by lbm_step."""
    names = sorted(VARIANT_CASES)
    lats, solos, runs = [], [], []
    for k, name in enumerate(names):
        pb = VARIANT_CASES[name]
        lp, o, f, g = _random_state(orc, pb, seed=90 + 5 * k)
        lat, solo = gb.Lattice(pb), gb.Lattice(pb)
        for x in (lat, solo):
            x.set_populations(f, g)
        o.set_populations(f, g)
        lats.append(lat)
        solos.append(solo)
        runs.append((lp, o))
    assert sum(l.lattice()["q"] == 15 for l in lats) == 3
    assert sum(l.lattice()["node_walls"] == 1 for l in lats) == 3
    batch = gb.Batch(lats)

    def errors(lp, lat, o):
        fa, ga = lat.populations()
        fb, gbo = o.populations()
        w = (orc.tables15()["w15"] if lp.q == 15 else orc.tables()["w19"]).reshape(-1, 1, 1, 1)
        _, om = _weights(orc, lp)
        return (np.abs(fa - fb).max() / np.abs(fb - w * lp.rho0).max(),
                np.abs(ga - gbo).max() / np.abs(gbo - om).max())

    batch.step(1)
    for name, lat, (lp, o) in zip(names, lats, runs):
        o.step(1)
        ef, eg = errors(lp, lat, o)
        assert ef < TOL_STEP and eg < TOL_STEP, (name, ef, eg)
    batch.step(12)
    batch.step(7)
    for name, lat, solo, (lp, o) in zip(names, lats, solos, runs):
        o.step(19)
        ef, eg = errors(lp, lat, o)
        assert ef < 4 * TOL_STEP and eg < 4 * TOL_STEP, (name, ef, eg)
        assert lat.steps == 20
        solo.step(20)
        fa, ga = lat.populations()
        fs, gs = solo.populations()
        assert np.array_equal(fa, fs) and np.array_equal(ga, gs), name
    batch.close()
    for x in lats + solos:
        x.close()


def test_batch_enthalpy_and_fp16_one_step(gb, orc):
    """An enthalpy lattice whose random state spans solid, mushy and liquid cells, an FP16
    lattice and an FP32 lattice in one batch, one step: the enthalpy lattice at 1e-5 outside
    the gate band, the FP16 lattice within the rounding of each stored value."""
    # enthalpy lattice: a random mixed-phase state
    pe = _melting(12)
    lpe, oe, fe, ge = _random_state(orc, pe, seed=21, g_noise=0.3)
    le = gb.Lattice(pe)
    le.set_populations(fe, ge)
    oe.set_populations(fe, ge)
    # FP16 lattice: both sides start from the rounded state the GPU holds
    p16 = dict(cavity_problem(13, Ra=1e4, Da=1e-2, phi=0.6, Pr=0.71), ny=11, nz=9, storage="fp16")
    lp16, o16, f16, g16 = _random_state(orc, p16, seed=33)
    l16 = gb.Lattice(p16)
    l16.set_populations(f16, g16)
    fq, gq = l16.populations()
    o16.set_populations(fq, gq)
    # FP32 companion
    p32 = STEP_CASES["channel_ragged"]
    lp32, o32, f32, g32 = _random_state(orc, p32, seed=34)
    l32 = gb.Lattice(p32)
    l32.set_populations(f32, g32)
    o32.set_populations(f32, g32)

    batch = gb.Batch([le, l16, l32])
    batch.step(1)
    for o in (oe, o16, o32):
        o.reset_gate_margin()
        o.step(1)
    # enthalpy: sites inside the band are counted and left out
    fa, ga = le.populations()
    fb, gbo = oe.populations()
    w = orc.tables()["w19"].reshape(19, 1, 1, 1)
    keep = oe.gate_margin() >= GATE_BAND_STEP
    assert (~keep).sum() <= keep.size // 100
    assert np.abs(fa - fb)[:, keep].max() < TOL_STEP * np.abs(fb - w).max()
    assert np.abs(ga - gbo)[:, keep].max() < TOL_STEP * np.abs(gbo).max()
    # FP16: the rounding of each stored value (u_r = 2^-11) plus the FP32 arithmetic
    fa, ga = l16.populations()
    fb, gbo = o16.populations()
    w16, _ = _weights(orc, lp16)
    om16 = np.array([1 - lp16.varpi] + [lp16.varpi / 6] * 6).reshape(7, 1, 1, 1)
    Tb = gbo.sum(axis=0, keepdims=True) / lp16.sigma
    ur, sub = 2.0 ** -11, 3e-8
    dev_f = np.abs(fb - w16)
    dev_g = np.abs(gbo - om16 * lp16.sigma * Tb)
    assert np.all(np.abs(fa - fb) <= ur * dev_f + 2e-6 * dev_f.max() + sub * w16 / lp16.rho0)
    assert np.all(np.abs(ga - gbo) <= ur * dev_g +
                  2e-6 * np.abs(gbo - om16 * lp16.sigma * lp16.T0).max())
    # FP32
    ef, eg = _step_errors(orc, lp32, l32, o32)
    assert ef < TOL_STEP and eg < TOL_STEP
    batch.close()


def test_batch_runs_match_oracle(gb, orc):
    """Four lattices from their initial states for 1,300 batched steps: a convection cavity, a
    field-medium cavity, the outflow channel and a convection-melting cavity (whose gate
    decisions all stay at least 1.8e-3 from 1/2 over this run, so both sides gate alike): u and
    T within 1e-5 of the oracle."""
    pbs = {"cavity": cavity_problem(16, Ra=1e5, Da=1e-2, phi=0.8, Pr=0.71),
           "hetero": _hetero(14),
           "channel": channel_problem(48, 12, 8, Da=1e-2),
           "melting": _melting(16)}
    steps = 1300
    lats = {k: gb.Lattice(pb) for k, pb in pbs.items()}
    batch = gb.Batch(list(lats.values()))
    batch.tune()
    batch.step(steps)
    for k, pb in pbs.items():
        o = orc.Oracle(orc.map_problem(pb))
        o.step(steps)
        if k == "melting":
            assert o.gate_margin().min() > 1e-4
        _, ug, Tg = lats[k].macros()
        _, uo, To = o.macros()
        assert orc.field_error(ug, uo) < TOL_FIELD, k
        assert orc.field_error(Tg, To) < TOL_FIELD, k
    batch.close()


def test_served_requests_match_oracle(gb, orc):
    """Requests served in a staggered mix (continuous batching, two arrival waves, chunks of
    100 steps) each hand back their final u and T (lbm_server_set_output); every one equals an
    oracle run of the same problem for the same number of steps, within 1e-5."""
    mix = [cavity_problem(12, Ra=1e5, Da=1e-2, phi=0.8, Pr=0.71),
           channel_problem(32, 8, 6, Da=1e-2),
           _hetero(12),
           _melting(12),
           dict(cavity_problem(10, Ra=1e4, Da=1e-3, phi=0.5, Pr=0.71), ny=8)]
    limits = [600, 400, 500, 700, 300]
    srv = gb.Server(chunk=100)
    outs, ids = {}, {}

    def submit(k):
        pb = mix[k]
        ns = int(pb["nx"]) * int(pb["ny"]) * int(pb["nz"])
        rid = srv.submit(pb, tol=1e-14, max_steps=limits[k])  # unreachable: run to the limit
        u = np.zeros(3 * ns, np.float32)
        T = np.zeros(ns, np.float32)
        srv.set_output(rid, u, T)
        outs[rid] = (u, T)
        ids[rid] = k

    for k in (0, 1, 2):
        submit(k)
    srv.advance()
    srv.advance()
    for k in (3, 4):  # the second wave joins while the first is on the GPU
        submit(k)
    results = []
    for _ in range(100):
        na, nq = srv.advance()
        results += srv.poll()
        if na == 0 and nq == 0:
            break
    results += srv.poll()
    srv.close()
    assert sorted(r["id"] for r in results) == sorted(ids)
    for r in results:
        k = ids[r["id"]]
        pb = mix[k]
        assert r["status"] == "max_steps" and r["steps"] == limits[k]
        o = orc.Oracle(orc.map_problem(pb))
        o.step(r["steps"])
        _, uo, To = o.macros()
        u, T = outs[r["id"]]
        ug = u.reshape(uo.shape)
        Tg = T.reshape(To.shape)
        assert orc.field_error(ug, uo) < TOL_FIELD, k
        assert orc.field_error(Tg, To) < TOL_FIELD, k


def test_served_variants_match_oracle(gb, orc):
    """A D3Q15 cavity, a node-wall cavity and an AA cavity (each batched in a group of its
    own), served together with a ping-pong cavity: each request's final
    u and T equal an oracle run of the same problem for the same steps, within 1e-5."""
    nee = cavity_problem(11, Ra=1e4, Da=1e-2, phi=0.8, Pr=0.71, L=10)
    nee.update(ny=10, nz=9, flow_bc=[4] * 6, heat_bc=[4, 4, 5, 5, 5, 5])
    mix = [dict(cavity_problem(12, Ra=1e4, Da=1e-2, phi=0.8, Pr=0.71), q=15, ny=10),
           nee,
           dict(cavity_problem(12, Ra=1e5, Da=1e-2, phi=0.6, Pr=0.71), ny=10, scheme="aa"),
           cavity_problem(10, Ra=1e4, Da=1e-2, phi=0.8, Pr=0.71)]
    limits = [400, 300, 500, 300]
    srv = gb.Server(chunk=100)
    outs, ids = {}, {}
    for k, pb in enumerate(mix):
        ns = int(pb["nx"]) * int(pb["ny"]) * int(pb["nz"])
        rid = srv.submit(pb, tol=1e-14, max_steps=limits[k])
        u = np.zeros(3 * ns, np.float32)
        T = np.zeros(ns, np.float32)
        srv.set_output(rid, u, T)
        outs[rid] = (u, T)
        ids[rid] = k
    results = []
    for _ in range(100):
        na, nq = srv.advance()
        results += srv.poll()
        if na == 0 and nq == 0:
            break
    results += srv.poll()
    srv.close()
    assert sorted(r["id"] for r in results) == sorted(ids)
    for r in results:
        k = ids[r["id"]]
        assert r["status"] == "max_steps" and r["steps"] == limits[k]
        o = orc.Oracle(orc.map_problem(mix[k]))
        o.step(r["steps"])
        _, uo, To = o.macros()
        u, T = outs[r["id"]]
        assert orc.field_error(u.reshape(uo.shape), uo) < TOL_FIELD, k
        assert orc.field_error(T.reshape(To.shape), To) < TOL_FIELD, k
