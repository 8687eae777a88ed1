"""The AA scheme (one population copy updated in place) against the ping-pong scheme and the
FP64 oracle.

The AA pull step gathers exactly the values the ping-pong pull gathers, and its local step
reads back exactly what the pull pushed (the face rules applied on the same operands), so the
populations, the macroscopic fields, the totals and the Nusselt numbers must agree bit for bit
after any number of steps, odd counts included (the state is then rearranged, without
arithmetic, before it is read).  Cases: walls on every face, periodic faces of extent 1, 3 and
5, a moving lid, a velocity face, a heterogeneous medium, sigma != 1."""
import numpy as np
import pytest

from lbm_inputs import cavity_problem, channel_problem, porosity_field, random_macros, uniform

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gb():
    import paper_1611_03329_gb300 as gb

    gb.build.build()
    gb.lib()
    return gb


def _hetero(n=12):
    phi = porosity_field(n, n - 2, n - 4, seed=11).astype(np.float32).astype(np.float64)
    pb = cavity_problem(n, Ra=1e5, Da=1e-2, phi=0.6, Pr=0.71, phi_field=phi, alpha_m=0.02)
    pb.update(ny=n - 2, nz=n - 4)
    return pb


CASES = {
    "cavity_ragged": dict(cavity_problem(13, Ra=1e4, Da=1e-2, phi=0.6, Pr=0.71), ny=11, nz=9),
    "periodic_forced": dict(nx=37, ny=5, nz=3, mapping="lattice", nu_e=0.05, alpha_f=0.03,
                            gbeta=2e-3, phi=0.5, K=2.0, F_phi=0.4, accel=[2e-4, -1e-4, 5e-5]),
    "moving_lid": dict(cavity_problem(9, Ra=1e4, Da=None, phi=1.0, Pr=0.71), nz=7,
                       flow_bc=[1, 1, 1, 1, 1, 2],
                       face_u=[(0, 0, 0)] * 5 + [(0.02, -0.01, 0.0)]),
    # velocity face on x-low (inflow with a transverse component), wall on x-high
    "velocity_face": dict(cavity_problem(10, Ra=1e4, Da=1e-2, phi=0.7, Pr=0.71), ny=8, nz=6,
                          flow_bc=[2, 1, 1, 1, 0, 0], heat_bc=[2, 2, 1, 1, 0, 0],
                          face_u=[(0.01, 0.003, 0.0)] + [(0, 0, 0)] * 5),
    "hetero_phi": _hetero(),
    "sigma_gamma": dict(cavity_problem(8, Ra=2e4, Da=1e-2, phi=0.7, Pr=0.71, J=1.4,
                                       sigma=1.6, Gamma=1.3), ny=6),
    "line_1xNx1": dict(nx=1, ny=17, nz=1, mapping="lattice", nu_e=0.1, phi=0.6, K=5.0,
                       F_phi=0.3, accel=[1e-4, 0, 0], flow_bc=[0, 0, 1, 1, 0, 0],
                       heat_bc=[0, 0, 2, 2, 0, 0], face_T=[0, 0, 1, 0, 0, 0]),
}


def _state(orc, pb, seed):
    lp = orc.map_problem(pb)
    o = orc.Oracle(lp)
    _, u, T = random_macros(lp.nx, lp.ny, lp.nz, seed, u_amp=0.03)
    o.init_equilibrium(0.5, T, u)
    f, g = o.populations()
    return lp, o, f + 3e-4 * uniform(f.shape, seed + 1), g + 3e-4 * uniform(g.shape, seed + 2)


def _pair(gb, pb, f=None, g=None):
    pp = gb.Lattice(dict(pb, scheme="pingpong"))
    aa = gb.Lattice(dict(pb, scheme="aa"))
    assert pp.lattice()["scheme"] == 0 and aa.lattice()["scheme"] == 1
    if f is not None:
        pp.set_populations(f, g)
        aa.set_populations(f, g)
    return pp, aa


def _same_state(pp, aa, pb):
    fa, ga = pp.populations()
    fb, gb_ = aa.populations()
    assert np.array_equal(fa, fb) and np.array_equal(ga, gb_)
    for a, b in zip(pp.macros(), aa.macros()):
        assert np.array_equal(a, b)
    assert pp.sums() == aa.sums()
    heat = pb.get("heat_bc", [0] * 6)
    for face in range(6):
        if heat[face] == 2 and [pb["nx"], pb["ny"], pb["nz"]][face // 2] >= 2:
            a, b = pp.nusselt(face), aa.nusselt(face)
            assert a[0] == b[0] and a[2] == b[2] and np.array_equal(a[1], b[1])


@pytest.mark.parametrize("name", sorted(CASES))
def test_bit_identical_to_pingpong(gb, orc, name):
    pb = CASES[name]
    _, _, f, g = _state(orc, pb, 23)
    pp, aa = _pair(gb, pb, f, g)
    for n in (1, 1, 2, 5):  # odd and even counts; reads in between rearrange the AA copy
        pp.step(n)
        aa.step(n)
        _same_state(pp, aa, pb)


def test_long_run_without_reads(gb, orc):
    """500 steps from the equilibrium start with no read in between (the AA copy alternates
    layouts 500 times), then 1 more: identical to ping-pong both times."""
    pb = dict(cavity_problem(24, Ra=1e5, Da=1e-2, phi=0.6, Pr=0.71), ny=20, nz=17)
    pp, aa = _pair(gb, pb)
    for n in (500, 1):
        pp.step(n)
        aa.step(n)
        fa, ga = pp.populations()
        fb, gb_ = aa.populations()
        assert np.array_equal(fa, fb) and np.array_equal(ga, gb_)


def test_twenty_steps_match_oracle(gb, orc):
    """AA directly against the FP64 oracle: 20 steps from a seeded random state, every
    population within 4e-5 of the largest deviation (the ping-pong parity bound)."""
    pb = CASES["hetero_phi"]
    lp, o, f, g = _state(orc, pb, 5)
    aa = gb.Lattice(dict(pb, scheme="aa"))
    aa.set_populations(f, g)
    o.set_populations(f, g)
    aa.step(20)
    o.step(20)
    fa, ga = aa.populations()
    fb, gb_ = o.populations()
    wf = orc.tables()["w19"].reshape(19, 1, 1, 1) * lp.rho0
    om = (np.array([1 - lp.varpi] + [lp.varpi / 6] * 6) * lp.sigma * lp.T0).reshape(7, 1, 1, 1)
    assert np.abs(fa - fb).max() < 4e-5 * np.abs(fb - wf).max()
    assert np.abs(ga - gb_).max() < 4e-5 * np.abs(gb_ - om).max()


def test_cavity_128_bit_identical(gb):
    """The 128^3 cavity with a porosity field (the precision-sweep workload at the smaller
    edge): 25 steps, AA and ping-pong identical."""
    phi = porosity_field(128, 128, 128, seed=20161110).astype("float32")
    pb = cavity_problem(128, Ra=1e5, Da=1e-2, phi=0.6, Pr=0.71, phi_field=phi, phi_ref=0.6)
    pp, aa = _pair(gb, pb)
    pp.step(25)
    aa.step(25)
    for a, b in zip(pp.macros(), aa.macros()):
        assert np.array_equal(a, b)


def test_scheme_rules(gb):
    from paper_1611_03329_gb300 import LbmError

    with pytest.raises(LbmError):  # outflow face
        gb.Lattice(dict(channel_problem(32, 8, 4), scheme="aa"))
    with pytest.raises(LbmError):  # 16-bit storage
        gb.Lattice(dict(cavity_problem(8, Ra=1e4, Da=1e-2, phi=0.6), storage="fp16", scheme="aa"))
    with pytest.raises(LbmError):  # D3Q15
        gb.Lattice(dict(cavity_problem(8, Ra=1e4, Da=1e-2, phi=0.6), q=15, scheme="aa"))
    pb = dict(cavity_problem(64, Ra=1e4, Da=1e-2, phi=0.6), ny=8, nz=8, scheme="auto")
    # AUTO: ping-pong while two copies fit, AA when the memory cap leaves room for one only
    assert gb.Lattice(pb).lattice()["scheme"] == 0
    one_copy = gb.footprint(dict(pb, scheme="aa"))
    cav = gb.Lattice(dict(pb, auto_mem_limit=one_copy + 1024))
    assert cav.lattice()["scheme"] == 1
    ch = gb.Lattice(dict(channel_problem(64, 8, 4), scheme="auto",
                         auto_mem_limit=one_copy + 1024))  # outflow: ping-pong
    assert ch.lattice()["scheme"] == 0
    with pytest.raises(LbmError):  # the TMA kernel runs ping-pong copies
        cav.set_step_kernel("tma")


def test_batch_with_aa_lattices(gb):
    """AA lattices batched beside ping-pong lattices (their own group, one launch per step for
    both phases): after 1, 3 and 2 batched steps every lattice is bit-identical to the same
    problem stepped alone with ping-pong copies.  One AA lattice enters the batch after an odd
    step count (streamed layout), so the first batched launch mixes pull and local steps; the
    tuner runs first and must leave every state unchanged."""
    names = ["cavity_ragged", "hetero_phi", "moving_lid", "periodic_forced"]
    aa = [gb.Lattice(dict(CASES[k], scheme="aa")) for k in names]
    pp = [gb.Lattice(dict(CASES[k], scheme="pingpong")) for k in names[:2]]
    ref = [gb.Lattice(dict(CASES[k], scheme="pingpong")) for k in names + names[:2]]
    aa[0].step(1)
    ref[0].step(1)
    batch = gb.Batch(aa + pp)
    batch.tune()
    for n in (1, 3, 2):
        batch.step(n)
        for r in ref:
            r.step(n)
        for a, r in zip(aa + pp, ref):
            fa, ga = a.populations()
            fr, gr = r.populations()
            assert np.array_equal(fa, fr) and np.array_equal(ga, gr)
    batch.close()


def test_batch_of_aa_lattices_only(gb):
    """A batch of AA lattices alone: the tuner sets its shape without launching anything, and
    the batched steps match the lattices stepped one at a time."""
    names = ["cavity_ragged", "velocity_face", "sigma_gamma"]
    aa = [gb.Lattice(dict(CASES[k], scheme="aa")) for k in names]
    solo = [gb.Lattice(dict(CASES[k], scheme="aa")) for k in names]
    batch = gb.Batch(aa)
    assert tuple(batch.tune()) == (32, 4)
    batch.step(7)
    for s_ in solo:
        s_.step(7)
    for a, s_ in zip(aa, solo):
        assert np.array_equal(a.populations()[0], s_.populations()[0])
        assert np.array_equal(a.populations()[1], s_.populations()[1])
    batch.close()


def test_batch_moves_lattices_to_aa(gb):
    """lbm_batch_set_scheme("aa"): the eligible ping-pong members move to the one-copy scheme
    (their current copy permuted into the second, the first freed); an outflow channel stays
    ping-pong.  Every lattice keeps stepping bit-identically to the same problem stepped alone
    with ping-pong copies."""
    pbs = [dict(cavity_problem(12, Ra=1e4, Da=1e-2, phi=0.7, Pr=0.71), ny=10, nz=9),
           _hetero(10), channel_problem(24, 8, 6, Da=1e-2)]
    alone = [gb.Lattice(pb) for pb in pbs]
    batched = [gb.Lattice(pb) for pb in pbs]
    for a, b in zip(alone, batched):
        a.step(3)
        b.step(3)
    batch = gb.Batch(batched)
    batch.step(2)
    batch.set_scheme("aa")
    assert [b.lattice()["scheme"] for b in batched] == [1, 1, 0]
    batch.step(5)
    batch.step(4)
    for a in alone:
        a.step(11)
    for a, b in zip(alone, batched):
        fa, ga = a.populations()
        fb, gbb = b.populations()
        assert np.array_equal(fa, fb) and np.array_equal(ga, gbb)
    batch.close()


def test_tuner_chooses_the_scheme_by_timing(gb):
    """lbm_batch_tune times eligible ping-pong groups both ways (AA on scratch copies) and
    keeps ping-pong unless AA is more than 3 % faster; the state is untouched either way."""
    pbs = [cavity_problem(24, Ra=1e5, Da=1e-2, phi=0.8, Pr=0.71) for _ in range(3)]
    alone = [gb.Lattice(pb) for pb in pbs]
    batched = [gb.Lattice(pb) for pb in pbs]
    batch = gb.Batch(batched)
    batch.step(7)
    for a in alone:
        a.step(7)
    batch.tune()
    pp, aa = batch.scheme_times()
    assert pp > 0.0 and aa > 0.0
    want = 1 if aa < 0.97 * pp else 0
    assert all(b.lattice()["scheme"] == want for b in batched)
    batch.step(9)
    for a in alone:
        a.step(9)
    for a, b in zip(alone, batched):
        fa, ga = a.populations()
        fb, gbb = b.populations()
        assert np.array_equal(fa, fb) and np.array_equal(ga, gbb)
    batch.close()
