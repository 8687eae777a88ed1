"""The paired step kernel (two x-adjacent sites per thread, paired FP32 instructions) against
the one-site kernel and the FP64 oracle.

Both kernels read the same stored values and run the same explicitly rounded operations on
them (the collision is one template over one site or a pair), so the populations after any
number of steps agree bit for bit, in every storage format.  The cases cover walled,
velocity, outflow and periodic faces on every axis (interior pairs, x-face pairs, y/z-face
rows), ragged extents, a porosity field and sigma, Gamma != 1."""
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
    "channel_34x10x7": channel_problem(34, 10, 7, Da=1e-2),
    "channel_T_out_22x8x5": dict(channel_problem(22, 8, 5, Da=1e-2), heat_bc=[2, 3, 2, 2, 0, 0]),
    "cavity_14x11x9": dict(cavity_problem(14, Ra=1e4, Da=1e-2, phi=0.6, Pr=0.71), ny=11, nz=9),
    "periodic_38x5x3": dict(nx=38, ny=5, nz=3, mapping="lattice", nu_e=0.05, alpha_f=0.03,
                            gbeta=2e-3, phi=0.5, K=2.0, F_phi=0.4, sigma=1.7,
                            accel=[2e-4, -1e-4, 5e-5]),
    "moving_lid_10x8x7": dict(cavity_problem(10, Ra=1e4, Da=None, phi=1.0, Pr=0.71), ny=8, nz=7,
                              flow_bc=[1, 1, 1, 1, 1, 2],
                              face_u=[(0, 0, 0)] * 5 + [(0.02, -0.01, 0.0)]),
    "hetero_16x12x6": _hetero(16, 12, 6),
    "sigma_gamma_12x8x6": dict(cavity_problem(12, Ra=2e4, Da=1e-2, phi=0.7, Pr=0.71, J=1.4,
                                              sigma=1.6, Gamma=1.3), ny=8, nz=6),
    "narrow_2x17x4": dict(nx=2, ny=17, nz=4, mapping="lattice", nu_e=0.1, phi=0.6, K=5.0,
                          F_phi=0.3, accel=[1e-4, 0, 0], flow_bc=[0, 0, 1, 1, 1, 1],
                          heat_bc=[0, 0, 2, 2, 1, 1], face_T=[0, 0, 1, 0, 0, 0]),
}


def _state(orc, pb, seed):
    lp = orc.map_problem(pb)
    o = orc.Oracle(lp)
    _, u, T = random_macros(lp.nx, lp.ny, lp.nz, seed, u_amp=0.03)
    o.init_equilibrium(0.5, T, u)
    f, g = o.populations()
    return lp, o, f + 3e-4 * uniform(f.shape, seed + 1), g + 3e-4 * uniform(g.shape, seed + 2)


@pytest.mark.parametrize("storage", ["fp32", "fp16", "bf16"])
@pytest.mark.parametrize("name", sorted(CASES))
def test_paired_kernel_is_bit_identical(gb, orc, name, storage):
    pb = dict(CASES[name], storage=storage)
    lp, o, f, g = _state(orc, pb, seed=len(name))
    one, two = gb.Lattice(pb), gb.Lattice(pb)
    one.set_step_kernel("plain")
    two.set_step_kernel("paired")
    assert one.step_kernel == "plain" and two.step_kernel == "paired"
    for lat in (one, two):
        lat.set_populations(f, g)
    for n in (1, 2, 17):
        one.step(n)
        two.step(n)
        fa, ga = one.populations()
        fb, gb_ = two.populations()
        assert np.array_equal(fa, fb) and np.array_equal(ga, gb_), (name, storage, n)
    if storage == "fp32":  # and the oracle, one step from the same state
        one.set_populations(f, g)
        o.set_populations(f, g)
        two.set_populations(f, g)
        two.step(1)
        o.step(1)
        fa, ga = two.populations()
        fb, gb_ = o.populations()
        w = orc.tables()["w19"].reshape(19, 1, 1, 1) * lp.rho0
        om = (np.array([1 - lp.varpi] + [lp.varpi / 6] * 6) * lp.sigma * lp.T0).reshape(7, 1, 1, 1)
        assert np.abs(fa - fb).max() < 1e-5 * np.abs(fb - w).max()
        assert np.abs(ga - gb_).max() < 1e-5 * np.abs(gb_ - om).max()


def test_paired_kernel_long_channel_run_matches_oracle(gb, orc):
    """The 64 x 16 x 16 channel from rest for 2,000 steps on the paired kernel: u and T within
    1e-5 of the oracle, and bit-identical to the one-site kernel."""
    pb = channel_problem(64, 16, 16)
    one, two = gb.Lattice(pb), gb.Lattice(pb)
    one.set_step_kernel("plain")
    two.set_step_kernel("paired")
    one.step(2000)
    two.step(2000)
    assert np.array_equal(one.populations()[0], two.populations()[0])
    o = orc.Oracle(orc.map_problem(pb))
    o.step(2000)
    _, ug, Tg = two.macros()
    _, uo, To = o.macros()
    assert orc.field_error(ug, uo) < 1e-5 and orc.field_error(Tg, To) < 1e-5


def test_paired_kernel_is_the_default_where_it_applies(gb):
    assert gb.Lattice(channel_problem(34, 10, 7, Da=1e-2)).step_kernel == "paired"
    assert gb.Lattice(dict(cavity_problem(9, Ra=1e4, Da=1e-2, phi=0.6), ny=8)).step_kernel == "plain"
    assert gb.Lattice(dict(cavity_problem(8, Ra=1e4, Da=1e-2, phi=0.6), q=15)).step_kernel == "plain"
    assert gb.Lattice(dict(cavity_problem(8, Ra=1e4, Da=1e-2, phi=0.6), scheme="aa")).step_kernel == "plain"


def test_paired_kernel_rules(gb):
    with pytest.raises(gb.LbmError):  # odd nx
        gb.Lattice(dict(cavity_problem(9, Ra=1e4, Da=1e-2, phi=0.6), ny=8)).set_step_kernel("paired")
    with pytest.raises(gb.LbmError):  # D3Q15
        gb.Lattice(dict(cavity_problem(8, Ra=1e4, Da=1e-2, phi=0.6), q=15)).set_step_kernel("paired")
    with pytest.raises(gb.LbmError):  # AA scheme
        gb.Lattice(dict(cavity_problem(8, Ra=1e4, Da=1e-2, phi=0.6), scheme="aa")).set_step_kernel("paired")
