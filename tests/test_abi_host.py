"""Host-side checks of the C ABI (no GPU): the library loads and exports every symbol that
include/lbm.h declares, the parameter mapping matches the oracle's own mapping of Eq. 56 /
Eq. 51 / Eq. 41, and invalid problem statements are rejected with LBM_EINVAL."""
import ctypes as C
import math
import os
import re

import numpy as np
import pytest

from lbm_inputs import cavity_problem, channel_problem

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def gb():
    import paper_1611_03329_gb300 as gb

    gb.build.build()
    gb.lib()
    return gb


def _declared_symbols():
    text = open(os.path.join(ROOT, "include", "lbm.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(lbm_[a-z_]+)\s*\(", text)))


def test_header_symbols_are_exported(gb):
    names = _declared_symbols()
    assert len(names) >= 19
    assert set(names) == set(gb.ABI_SYMBOLS)
    for n in names:
        assert hasattr(gb.lib(), n), n


def test_struct_sizes_match_header(gb):
    p = gb.LbmParams()
    assert gb.lib().lbm_params_default(C.byref(p)) == 0
    assert p.rho0 == 1.0 and p.varpi == 0.5 and p.s_m == 1.2 and p.zeta_e == 1.2


PROBLEMS = [
    cavity_problem(32, Ra=1e3, Da=1e-2, phi=0.6, Pr=1.0),
    cavity_problem(64, Ra=1e5, Da=1e-3, phi=0.8, Pr=0.71, J=1.3, sigma=1.4, Gamma=0.8),
    cavity_problem(20, Ra=1e4, Da=1e-2, phi=0.8, Pr=0.71, gravity_axis=1, gravity_sign=1),
    channel_problem(256, 64, 64),
    channel_problem(64, 16, 16, Re=5, Ri=0.5, Pr=1.0),
    dict(nx=4, ny=16, nz=1, mapping="lattice", nu_e=0.07, alpha_f=0.03, gbeta=1e-4,
         accel=[1e-5, 0, 2e-6], flow_bc=[0, 0, 1, 1, 0, 0], heat_bc=[0, 0, 2, 2, 0, 0]),
]


@pytest.mark.parametrize("pb", PROBLEMS)
def test_mapping_matches_oracle(gb, orc, pb):
    got = gb.derive_lattice(pb)
    want = orc.map_problem({k: v for k, v in pb.items() if k not in ("phi", "F_phi")})
    for k in ("s_nu", "zeta_alpha", "nu", "nu_e", "alpha_f", "gbeta", "L", "U_out"):
        assert got[k] == pytest.approx(getattr(want, k), rel=1e-14, abs=1e-300), k
    assert np.allclose(got["s"], want.s, rtol=1e-14)
    assert np.allclose(got["buoy"], want.buoy, rtol=1e-14, atol=0)
    assert np.allclose(got["accel"], want.accel, rtol=1e-14, atol=0)
    if pb.get("Da") is not None:
        assert got["K"] == pytest.approx(want.K, rel=1e-14)
    else:
        assert math.isinf(got["K"])


def test_cavity_workload_numbers(gb):
    """32^3 cavity with phi = 0.6, Da = 1e-2, Ra = 1e3, Pr = 1: 1/s_nu = 0.6753 (Eq. 56),
    1/zeta_alpha = 0.8505, g beta = 1.042e-4, K = 10.24."""
    d = gb.derive_lattice(PROBLEMS[0])
    assert 1 / d["s_nu"] == pytest.approx(0.5 + 0.1 * 32 * math.sqrt(3) / math.sqrt(1e3), rel=1e-15)
    assert 1 / d["s_nu"] == pytest.approx(0.6753, abs=5e-5)
    assert 1 / d["zeta_alpha"] == pytest.approx(0.8505, abs=5e-5)
    assert d["gbeta"] == pytest.approx(0.01 / 3 / 32, rel=1e-15)
    assert d["K"] == pytest.approx(10.24, rel=1e-15)


BAD = [
    dict(nx=0),
    dict(varpi=1.0),
    dict(rho0=0.0),
    dict(Ra=-1.0),
    dict(flow_bc=[3, 1, 1, 1, 1, 1], heat_bc=[3, 2, 1, 1, 1, 1]),   # outflow on x-low
    dict(flow_bc=[0, 1, 1, 1, 1, 1]),                                 # unpaired periodic face
    dict(heat_bc=[0, 2, 1, 1, 1, 1]),                                 # periodic heat, wall flow
    dict(heat_bc=[2, 3, 1, 1, 1, 1]),                                 # thermal outflow w/o flow
    dict(s_e=2.5),
    dict(gravity_axis=3),
]


@pytest.mark.parametrize("bad", BAD)
def test_invalid_problems_rejected(gb, bad):
    pb = cavity_problem(8, Ra=1e3, Da=1e-2, phi=0.6)
    pb.update(bad)
    with pytest.raises(gb.LbmError) as ei:
        gb.derive_lattice(pb)
    assert ei.value.status == gb.LBM_EINVAL


def test_relaxation_rate_bound(gb):
    """Large and tiny viscosities map to rates inside (0, 2) (Eq. 32); a problem without a
    usable Prandtl number is rejected."""
    pb = dict(nx=4, ny=4, nz=4, mapping="lattice", nu_e=50.0)
    d = gb.derive_lattice(pb)
    assert 0 < d["s_nu"] < 2
    pb = dict(nx=4, ny=4, nz=4, mapping="lattice", nu_e=1e-7, alpha_f=1e-7)
    d = gb.derive_lattice(pb)
    assert d["s_nu"] == pytest.approx(1 / (0.5 + 3e-7), rel=1e-12)
    pb = dict(nx=4, ny=4, nz=4, mapping="lattice", nu_e=0.1, alpha_f=-0.0, Pr=-1.0)
    with pytest.raises(gb.LbmError):
        gb.derive_lattice(pb)


def test_aa_scheme_resolution_and_footprint(gb):
    """The AA scheme applies to FP32, D3Q19 lattices without outflow, node walls or the
    enthalpy model and is rejected elsewhere; LBM_SCHEME_AUTO derives as ping-pong (the
    device-memory test that may switch it to AA happens at lbm_create); an AA lattice holds
    one population copy instead of two (26 planes of sq = ceil(ns / 64) * 64 floats fewer)."""
    from lbm_inputs import channel_problem

    cav = cavity_problem(20, Ra=1e4, Da=1e-2, phi=0.6)
    assert gb.derive_lattice(dict(cav, scheme="aa"))["scheme"] == 1
    assert gb.derive_lattice(dict(cav, scheme="auto"))["scheme"] == 0
    assert gb.derive_lattice(dict(cav, scheme="pingpong"))["scheme"] == 0
    assert gb.derive_lattice(dict(cav, scheme="auto", storage="bf16"))["scheme"] == 0
    ch = channel_problem(32, 8, 4)
    assert gb.derive_lattice(dict(ch, scheme="auto"))["scheme"] == 0
    for bad in (dict(ch, scheme="aa"), dict(cav, scheme="aa", storage="fp16"),
                dict(cav, scheme="aa", q=15)):
        with pytest.raises(gb.LbmError):
            gb.derive_lattice(bad)
    ns = 20 ** 3
    sq = (ns + 63) // 64 * 64
    assert gb.footprint(dict(cav, scheme="pingpong")) - gb.footprint(dict(cav, scheme="aa")) \
        == 26 * 4 * sq


def test_algorithmic_bytes_per_site(gb):
    """The roofline's bytes per site update: the populations read and written in their storage
    format, the FP32 temperature plane of the 16-bit formats (read and written), and the FP32
    porosity of a heterogeneous medium."""
    import numpy as np
    from lbm_inputs import channel_problem

    ch = channel_problem(16, 8, 4)
    assert gb.algorithmic_bytes_per_site(ch) == 26 * 4 * 2
    assert gb.algorithmic_bytes_per_site(dict(ch, storage="fp16")) == 26 * 2 * 2 + 8
    assert gb.algorithmic_bytes_per_site(dict(ch, storage="bf16")) == 26 * 2 * 2 + 8
    assert gb.algorithmic_bytes_per_site(dict(ch, q=15)) == 22 * 4 * 2
    het = cavity_problem(8, Ra=1e4, Da=1e-2, phi=0.6, phi_field=np.full((8, 8, 8), 0.6))
    assert gb.algorithmic_bytes_per_site(het) == 26 * 4 * 2 + 4
