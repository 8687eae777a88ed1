"""Batched launches: a lattice advanced inside a batch gives exactly the same populations as
the same lattice advanced alone (the batch runs the same site update), across storage
formats, media, boundary kinds and sizes, graph replays of odd and even step counts, and
interleaved individual steps; the autotuner leaves the state untouched."""
import numpy as np
import pytest

from lbm_inputs import cavity_problem, channel_problem, porosity_field

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gb():
    import paper_1611_03329_gb300 as gb

    gb.build.build()
    gb.lib()
    return gb


def _problems():
    phi = porosity_field(14, 12, 10, seed=3).astype(np.float32)
    return [
        cavity_problem(20, Ra=1e5, Da=1e-2, phi=0.8, Pr=0.71),
        dict(cavity_problem(13, Ra=1e4, Da=1e-3, phi=0.5, Pr=0.71), ny=11, nz=9),
        channel_problem(33, 10, 7, Da=1e-2),
        dict(cavity_problem(14, Ra=1e5, Da=1e-2, phi=0.6, Pr=0.71, phi_field=phi), ny=12, nz=10),
        dict(cavity_problem(16, Ra=1e4, Da=1e-2, phi=0.7, Pr=0.71), storage="fp16"),
        dict(nx=37, ny=5, nz=3, mapping="lattice", nu_e=0.05, alpha_f=0.03, gbeta=2e-3, phi=0.5,
             K=2.0, F_phi=0.4, accel=[2e-4, -1e-4, 5e-5]),
        dict(cavity_problem(12, Ra=1e4, Da=1e-2, phi=0.7, Pr=0.71), storage="bf16"),
    ]


def _pair(gb):
    alone = [gb.Lattice(pb) for pb in _problems()]
    batched = [gb.Lattice(pb) for pb in _problems()]
    for a, b in zip(alone, batched):  # a few individual steps first so copies differ
        a.step(3)
        b.step(3)
    return alone, batched


def _same(alone, batched):
    for a, b in zip(alone, batched):
        fa, ga = a.populations()
        fb, gb_ = b.populations()
        assert np.array_equal(fa, fb) and np.array_equal(ga, gb_)
        assert a.steps == b.steps


def test_batch_equals_individual_steps(gb):
    alone, batched = _pair(gb)
    batch = gb.Batch(batched)
    batch.step(137)
    for a in alone:
        a.step(137)
    _same(alone, batched)
    batch.step(100)  # a second graph, even length
    batch.step(137)  # the first graph replayed from the other parity
    for a in alone:
        a.step(237)
    _same(alone, batched)
    batched[2].step(5)  # one lattice moves on its own in between
    alone[2].step(5)
    batch.step(1)
    for a in alone:
        a.step(1)
    _same(alone, batched)
    batch.close()


def test_tune_keeps_state(gb):
    alone, batched = _pair(gb)
    batch = gb.Batch(batched)
    before = [b.populations() for b in batched]
    bt, rows = batch.tune()
    assert bt in (32, 64, 128, 256) and rows in (1, 2, 4)
    for (f0, g0), b in zip(before, batched):
        f1, g1 = b.populations()
        assert np.array_equal(f0, f1) and np.array_equal(g0, g1)
    for threads, rows in ((32, 1), (128, 2), (256, 3), (64, 4)):
        batch.set_block(threads, rows)
        batch.step(11)
        for a in alone:
            a.step(11)
        _same(alone, batched)
    batch.close()


def test_per_lattice_launch_equals_individual_steps(gb):
    """Groups stepped by each lattice's own kernel (lbm_batch_set_launch_mode): the same
    populations as the lattices stepped alone, across graph-free odd and even step counts, a
    switch back to the fused launch and an individual step in between."""
    alone, batched = _pair(gb)
    batch = gb.Batch(batched)
    batch.set_launch_mode("per_lattice")
    nf, ns = batch.launch_groups()
    assert nf == 0 and ns >= 4  # every group is a ping-pong group here
    batch.step(37)
    batch.step(20)
    for a in alone:
        a.step(57)
    _same(alone, batched)
    batched[1].step(3)
    alone[1].step(3)
    batch.set_launch_mode("fused")
    assert batch.launch_groups() == (ns, 0)
    batch.step(9)
    batch.set_launch_mode("per_lattice")
    batch.step(4)
    for a in alone:
        a.step(13)
    _same(alone, batched)
    batch.close()


def test_tuner_chooses_the_launch_by_timing_and_keeps_state(gb):
    """Stage 3 of the tuner times every ping-pong group fused and per lattice without changing
    the state; large lattices (which fill the GPU alone) and small ones batch differently,
    and either way the populations follow the individual steps."""
    pbs = [dict(cavity_problem(96, Ra=1e5, Da=1e-2, phi=0.8, Pr=0.71), storage="fp16"),
           dict(cavity_problem(128, Ra=1e4, Da=1e-3, phi=0.6, Pr=0.71), storage="fp16")]
    batched = [gb.Lattice(pb) for pb in pbs]
    alone = [gb.Lattice(pb) for pb in pbs]
    batch = gb.Batch(batched)
    before = [b.populations() for b in batched]
    batch.tune()
    for (f0, g0), b in zip(before, batched):
        f1, g1 = b.populations()
        assert np.array_equal(f0, f1) and np.array_equal(g0, g1)
    nf, ns = batch.launch_groups()
    assert nf + ns == 1  # one FP16 paired group
    batch.step(7)
    for a in alone:
        a.step(7)
    _same(alone, batched)
    batch.close()


def test_batch_diagnostics_follow_the_contexts(gb):
    """After batched steps every per-context call sees the new state."""
    pb = cavity_problem(16, Ra=1e5, Da=1e-2, phi=0.8, Pr=0.71)
    a, b = gb.Lattice(pb), gb.Lattice(pb)
    batch = gb.Batch([b])
    batch.step(400)
    a.step(400)
    assert a.nusselt(0) [0] == b.nusselt(0)[0]
    assert a.sums() == b.sums()
    ra, Ta = a.macros()[1:]
    rb, Tb = b.macros()[1:]
    assert np.array_equal(ra, rb) and np.array_equal(Ta, Tb)


def test_batch_rejects_bad_lists(gb):
    lat = gb.Lattice(cavity_problem(8, Ra=1e4, Da=1e-2, phi=0.6))
    with pytest.raises(gb.LbmError):
        gb.Batch([lat, lat])
    with pytest.raises(gb.LbmError):
        gb.Batch([])
