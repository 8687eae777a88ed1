"""The bounds-checked build (-DLBM_BOUNDS_CHECK): every site index of a population,
temperature-plane, porosity or outflow-history access is checked.  Across boundary kinds,
media, storage formats, the one-site and paired kernels and a batch, no access leaves its
buffer, and the checked build computes exactly what the ordinary one does."""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

# Runs with either library (LBM_LIBRARY): steps every case and writes the populations.
SCRIPT = r"""
import json, sys
import numpy as np
sys.path.insert(0, ROOT)
import paper_1611_03329_gb300 as gb
from lbm_inputs import cavity_problem, channel_problem, porosity_field
phi = porosity_field(12, 10, 8, seed=3).astype(np.float32)
cases = {
    "channel": channel_problem(34, 10, 7, Da=1e-2),
    "channel_fp16": dict(channel_problem(34, 10, 7, Da=1e-2), storage="fp16"),
    "cavity_odd": dict(cavity_problem(13, Ra=1e4, Da=1e-2, phi=0.6, Pr=0.71), ny=11, nz=9),
    "hetero_bf16": dict(cavity_problem(12, Ra=1e5, Da=1e-2, phi=0.6, Pr=0.71, phi_field=phi),
                        ny=10, nz=8, storage="bf16"),
    "periodic": dict(nx=38, ny=5, nz=3, mapping="lattice", nu_e=0.05, alpha_f=0.03, gbeta=2e-3,
                     phi=0.5, K=2.0, F_phi=0.4, accel=[2e-4, -1e-4, 5e-5]),
    "moving_lid": dict(cavity_problem(10, Ra=1e4, Da=None, phi=1.0, Pr=0.71), ny=8, nz=7,
                       flow_bc=[1, 1, 1, 1, 1, 2], face_u=[(0, 0, 0)] * 5 + [(0.02, -0.01, 0.0)]),
    "aa": dict(cavity_problem(12, Ra=1e4, Da=1e-2, phi=0.7, Pr=0.71), ny=9, nz=8, scheme="aa"),
}
out = {}
for name, pb in cases.items():
    for kern in ("plain", "auto"):
        lat = gb.Lattice(pb)
        if kern == "plain":
            lat.set_step_kernel("plain")
        lat.step(7)
        f, g = lat.populations()
        out[f"{name}_{kern}"] = np.concatenate([f.ravel(), g.ravel()])
lats = [gb.Lattice(cases[k]) for k in ("channel", "cavity_odd", "hetero_bf16", "aa")]
batch = gb.Batch(lats)
batch.step(5)
for k, l in zip(("channel", "cavity_odd", "hetero_bf16", "aa"), lats):
    f, g = l.populations()
    out["batch_" + k] = np.concatenate([f.ravel(), g.ravel()])
np.savez(sys.argv[1], **out)
try:
    print(json.dumps({"first_bad": gb.bounds_report()}))
except gb.LbmError:
    print(json.dumps({"first_bad": None}))
"""


def _run(lib, out):
    env = dict(os.environ, LBM_LIBRARY=lib)
    r = subprocess.run([sys.executable, "-c", "ROOT = %r\n" % ROOT + SCRIPT, out],
                       capture_output=True, text=True, env=env, cwd=ROOT, timeout=900)
    assert r.returncode == 0, r.stderr[-3000:]
    return json.loads(r.stdout.strip().splitlines()[-1])["first_bad"], np.load(out)


def test_checked_build_stays_in_bounds_and_matches(tmp_path):
    from paper_1611_03329_gb300 import build

    checked = build.build(checked=True)
    plain = build.build()
    bad, got = _run(checked, str(tmp_path / "checked.npz"))
    assert bad == -1, f"out-of-range site index {bad}"
    none, ref = _run(plain, str(tmp_path / "plain.npz"))
    assert none is None  # the ordinary build checks nothing and says so
    assert sorted(got.files) == sorted(ref.files)
    for k in ref.files:
        assert np.array_equal(got[k], ref[k]), k
