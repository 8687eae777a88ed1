"""The TMA-staged step kernel against the per-thread-load kernel and the FP64 oracle.

Both kernels load the same stored values and run the same arithmetic on them, so the
populations after any number of steps must agree bit for bit, in every storage format; the
cases cover walled, velocity and outflow x faces (staged loads, then the face rule), periodic
x faces (global-memory path), ragged y extents (partial tiles) and y / z boundary rows, and a
heterogeneous medium.  One-step parity with the oracle uses the FP32 bound of the parity tests
(1e-5 of the largest deviation)."""
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


def _hetero(nx, ny, nz):
    phi = porosity_field(nx, ny, nz, seed=5).astype(np.float32).astype(np.float64)
    pb = cavity_problem(nx, Ra=1e5, Da=1e-2, phi=0.6, Pr=0.71, phi_field=phi, alpha_m=0.02)
    pb.update(ny=ny, nz=nz)
    return pb


CASES = {
    # velocity inlet / anchored outflow on x, walls on y, periodic z; ny not a multiple of 4
    "channel_128x10x7": channel_problem(128, 10, 7, Da=1e-2),
    # walls on every face (x faces: staged loads then the bounce-back rule)
    "cavity_64x9x6": dict(cavity_problem(64, Ra=1e4, Da=1e-2, phi=0.6, Pr=0.71), ny=9, nz=6),
    # periodic box: x-face warps take the global path with the wrap
    "periodic_64x6x5": dict(nx=64, ny=6, nz=5, mapping="lattice", nu_e=0.05, alpha_f=0.03,
                            gbeta=2e-3, phi=0.5, K=2.0, F_phi=0.4, sigma=1.7,
                            accel=[2e-4, -1e-4, 5e-5]),
    "moving_lid_64x8x7": dict(cavity_problem(64, Ra=1e4, Da=None, phi=1.0, Pr=0.71), ny=8,
                              nz=7, flow_bc=[1, 1, 1, 1, 1, 2],
                              face_u=[(0, 0, 0)] * 5 + [(0.02, -0.01, 0.0)]),
    "hetero_64x12x6": _hetero(64, 12, 6),
    # sigma != 1 and Gamma != 1 (heat-capacity ratio and viscosity ratio of Eqs. 3, 32)
    "sigma_gamma_64x8x6": dict(cavity_problem(64, Ra=2e4, Da=1e-2, phi=0.7, Pr=0.71, J=1.4,
                                              sigma=1.6, Gamma=1.3), ny=8, nz=6),
}


def _state(orc, pb, seed):
    lp = orc.map_problem(pb)
    o = orc.Oracle(lp)
    _, u, T = random_macros(lp.nx, lp.ny, lp.nz, seed, u_amp=0.03)
    o.init_equilibrium(0.5, T, u)
    f, g = o.populations()
    return lp, o, f + 3e-4 * uniform(f.shape, seed + 1), g + 3e-4 * uniform(g.shape, seed + 2)


def _pair(gb, pb, f, g):
    plain, tma = gb.Lattice(pb), gb.Lattice(pb)
    plain.set_step_kernel("plain")
    tma.set_step_kernel("tma")
    assert plain.step_kernel == "plain" and tma.step_kernel == "tma"
    plain.set_populations(f, g)
    tma.set_populations(f, g)
    return plain, tma


@pytest.mark.parametrize("storage", ["fp32", "fp16", "bf16"])
@pytest.mark.parametrize("name", sorted(CASES))
def test_bit_identical_to_plain_kernel(gb, orc, name, storage):
    pb = dict(CASES[name], storage=storage)
    _, _, f, g = _state(orc, pb, 31)
    plain, tma = _pair(gb, pb, f, g)
    for n in (1, 6):
        plain.step(n)
        tma.step(n)
        tma.sync()
        fa, ga = plain.populations()
        fb, gb_ = tma.populations()
        assert np.array_equal(fa, fb) and np.array_equal(ga, gb_), (name, storage, n)


@pytest.mark.parametrize("name", ["channel_128x10x7", "cavity_64x9x6", "hetero_64x12x6"])
def test_one_step_matches_oracle(gb, orc, name):
    lp, o, f, g = _state(orc, CASES[name], 17)
    lat = gb.Lattice(CASES[name])
    lat.set_step_kernel("tma")
    lat.set_populations(f, g)
    o.set_populations(f, g)
    lat.step(1)
    o.step(1)
    fa, ga = lat.populations()
    fb, gb_ = o.populations()
    wf = orc.tables()["w19"].reshape(19, 1, 1, 1) * lp.rho0
    om = (np.array([1 - lp.varpi] + [lp.varpi / 6] * 6) * lp.sigma * lp.T0).reshape(7, 1, 1, 1)
    assert np.abs(fa - fb).max() < 1e-5 * np.abs(fb - wf).max()
    assert np.abs(ga - gb_).max() < 1e-5 * np.abs(gb_ - om).max()


@pytest.mark.parametrize("storage", ["fp32", "fp16"])
def test_full_size_channel_bit_identical(gb, orc, storage):
    """The 256 x 64 x 64 channel in the benchmark's launch configuration: 20 steps from the
    equilibrium start agree bit for bit with the plain kernel (whose parity with the oracle
    at this size is tested in the parity tests)."""
    pb = dict(channel_problem(256, 64, 64), storage=storage)
    plain, tma = gb.Lattice(pb), gb.Lattice(pb)
    tma.set_step_kernel("tma")
    plain.step(20)
    tma.step(20)
    tma.sync()
    fa, ga = plain.populations()
    fb, gb_ = tma.populations()
    assert np.array_equal(fa, fb) and np.array_equal(ga, gb_)
    _, u, T = tma.macros()
    assert np.isfinite(u).all() and np.isfinite(T).all()


def test_selection_rules(gb):
    from paper_1611_03329_gb300 import LbmError

    with pytest.raises(LbmError):  # nx not a multiple of 64
        gb.Lattice(channel_problem(100, 8, 4)).set_step_kernel("tma")
    with pytest.raises(LbmError):  # D3Q15 flow lattice
        gb.Lattice(dict(channel_problem(64, 8, 4), q=15)).set_step_kernel("tma")
    lat = gb.Lattice(channel_problem(64, 8, 4))
    lat.set_step_kernel("tma")
    lat.set_step_kernel("plain")
    assert lat.step_kernel == "plain"


@pytest.mark.parametrize("reader", ["sync", "macros", "residual"])
def test_wait_timeout_is_reported(gb, reader):
    """Failure detection of the bounded waits: with every stage told to wait for 16 bytes its
    loads never bring (lbm_test_tma_extra_wait), each wait runs out after about a second, the
    kernel sets its flag and stops, and the next call that synchronises the stream -- lbm_sync,
    or a reader of the state such as lbm_macros or lbm_residual -- reports LBM_ETIMEOUT instead
    of results from the step that stopped early; the context then refuses further steps.
    Nothing faults or hangs: a new context on the same device steps normally and matches the
    plain kernel."""
    from paper_1611_03329_gb300 import LbmError

    pb = channel_problem(64, 8, 6)
    lat = gb.Lattice(pb)
    lat.set_step_kernel("tma")
    lat.test_tma_extra_wait(16)
    lat.step(1)
    with pytest.raises(LbmError) as ei:
        {"sync": lat.sync, "macros": lat.macros, "residual": lat.residual}[reader]()
    assert ei.value.status == gb.LBM_ETIMEOUT
    with pytest.raises(LbmError):
        lat.step(1)
    lat.close()
    ok, ref = gb.Lattice(pb), gb.Lattice(pb)
    ok.set_step_kernel("tma")
    ok.step(3)
    ref.step(3)
    assert np.array_equal(ok.populations()[0], ref.populations()[0])
