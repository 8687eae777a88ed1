"""Raw state save / load (lbm_state_bytes, lbm_save_state, lbm_load_state): a restart from a
saved blob continues bit for bit like the run that was never interrupted, in the same or a
new context, for every storage format, with the outflow history and the 16-bit temperature
plane, and under the AA scheme after an odd step count; the blob holds the stored deviations
themselves; blobs of another lattice, format or scheme are refused."""
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


CASES = {
    "channel_fp32": channel_problem(48, 12, 6, Da=1e-2),
    "channel_fp16": dict(channel_problem(48, 12, 6, Da=1e-2), storage="fp16"),
    "channel_bf16": dict(channel_problem(48, 12, 6, Da=1e-2), storage="bf16"),
    "cavity_aa": dict(cavity_problem(14, Ra=1e5, Da=1e-2, phi=0.6, Pr=0.71), ny=12, nz=9,
                      scheme="aa"),
    "d3q15_channel": dict(channel_problem(40, 10, 6, Da=1e-2), q=15),
}


@pytest.mark.parametrize("name", sorted(CASES))
def test_restart_is_exact(gb, name):
    pb = CASES[name]
    a = gb.Lattice(pb)
    a.step(101)  # odd: the AA copy is saved after its rearrangement
    blob = a.save_state()
    assert blob.size == a.state_bytes()
    a.step(37)
    fa, ga = a.populations()
    ua = a.macros()
    a.load_state(blob)
    assert a.steps == 101
    a.step(37)
    fb, gb_ = a.populations()
    assert np.array_equal(fa, fb) and np.array_equal(ga, gb_)
    b = gb.Lattice(pb)  # a fresh context of the same problem
    b.load_state(blob)
    b.step(37)
    fc, gc = b.populations()
    assert np.array_equal(fa, fc) and np.array_equal(ga, gc)
    for x, y in zip(ua, b.macros()):
        assert np.array_equal(x, y)
    assert b.steps == 138


def test_blob_holds_the_stored_deviations(gb, orc):
    """FP32 blob: 128-byte header, then 26 planes of sq floats; plane q at site s plus the
    plane's rest value (w_i rho0, omega_i sigma T0) is the population lbm_get_populations
    returns."""
    pb = dict(cavity_problem(10, Ra=1e4, Da=1e-2, phi=0.7), ny=9, nz=7)
    lat = gb.Lattice(pb)
    lat.step(20)
    blob = lat.save_state()
    assert bytes(blob[:8]) == b"LBMSTATE"
    ns = 10 * 9 * 7
    sq = (ns + 63) // 64 * 64
    dev = blob[128:128 + 26 * sq * 4].view(np.float32).reshape(26, sq)[:, :ns]
    f, g = lat.populations()
    lp = orc.map_problem(pb)
    w = orc.tables()["w19"] * lp.rho0
    om = np.array([1 - lp.varpi] + [lp.varpi / 6] * 6) * lp.sigma * lp.T0
    assert np.array_equal(dev[:19].astype(np.float64) + w[:, None], f.reshape(19, ns))
    assert np.array_equal(dev[19:].astype(np.float64) + om[:, None], g.reshape(7, ns))


def test_foreign_blobs_refused(gb):
    from paper_1611_03329_gb300 import LbmError

    ch = gb.Lattice(channel_problem(48, 12, 6, Da=1e-2))
    blob = ch.save_state()
    for other in (dict(channel_problem(48, 12, 7, Da=1e-2)),
                  dict(channel_problem(48, 12, 6, Da=1e-2), storage="fp16"),
                  dict(cavity_problem(12, Ra=1e4, Da=1e-2, phi=0.6), scheme="aa")):
        with pytest.raises(LbmError):
            gb.Lattice(other).load_state(blob)
    with pytest.raises(LbmError):  # truncated
        ch.load_state(blob[: blob.size - 4])
    bad = blob.copy()
    bad[0] = ord("X")
    with pytest.raises(LbmError):
        ch.load_state(bad)
