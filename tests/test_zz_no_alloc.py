"""The allocation-free residual entry point against the existing one.

lbm_residual_noalloc serves callers that cannot allocate device memory (an application that
hands the library a fixed arena and forbids cudaMalloc after start-up, or a loop in which an
allocation would stall); it keeps its partial sums in a static device array.  This file runs
last so that a failure here leaves every other test already run; it also passes on its own in
a fresh process.
"""
import pytest

from lbm_inputs import cavity_problem

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch

    import paper_1611_03329_gb300 as gb

    gb.build.build()
    gb.lib()
    assert torch.cuda.is_available()
    torch.cuda.set_device(0)
    return gb, torch


def test_noalloc_residual_matches_lbm_residual(env):
    """Two calls in a row, each checked against lbm_residual on the same pair of fields."""
    gb, torch = env
    pb = cavity_problem(20, Ra=1e5, Da=1e-2, phi=0.8, Pr=0.71)
    stream = torch.cuda.current_stream()
    lat = gb.Lattice(pb, stream=stream.cuda_stream)
    ns = lat.ns
    u = [torch.empty(3 * ns, device="cuda") for _ in range(3)]
    T = [torch.empty(ns, device="cuda") for _ in range(3)]
    out = torch.full((3,), -1.0, dtype=torch.float64, device="cuda")

    lat.step(300)
    lat.residual()  # snapshot for lbm_residual
    lat.macros_device(0, u[0].data_ptr(), T[0].data_ptr())
    for k in (1, 2):
        lat.step(100)
        ru, rT = lat.residual()
        lat.macros_device(0, u[k].data_ptr(), T[k].data_ptr())
        gb.residual_noalloc(u[k].data_ptr(), T[k].data_ptr(), u[k - 1].data_ptr(),
                            T[k - 1].data_ptr(), ns, out.data_ptr(), stream.cuda_stream)
        r = out.cpu().tolist()
        assert r[0] == pytest.approx(ru, rel=1e-5)
        assert r[1] == pytest.approx(rT, rel=1e-5)
        assert r[2] == 0.0
        assert 0.0 < r[0] < 1.0 and 0.0 < r[1] < 1.0
    lat.close()


def test_noalloc_rejects_sizes_beyond_the_maximum(env):
    gb, torch = env
    buf = torch.zeros(3 * 8, device="cuda")
    out = torch.zeros(3, dtype=torch.float64, device="cuda")
    p = buf.data_ptr()
    for ns in (0, -5, gb.NOALLOC_MAX_SITES + 1):
        with pytest.raises(gb.LbmError) as ei:
            gb.residual_noalloc(p, p, p, p, ns, out.data_ptr())
        assert ei.value.status == gb.LBM_EINVAL
    with pytest.raises(gb.LbmError):
        gb.residual_noalloc(0, p, p, p, 8, out.data_ptr())


def test_noalloc_reports_non_finite_fields(env):
    """A NaN or Inf in a field is counted in out[2] and makes both residuals NaN, so a caller
    that tests r < tol never takes a blown-up solve for a converged one; the next call on
    finite fields is unaffected (the shared array keeps nothing that matters)."""
    gb, torch = env
    ns = 5000
    stream = torch.cuda.current_stream()
    u = torch.linspace(0.1, 0.2, 3 * ns, device="cuda")
    up = u * 0.999
    T = torch.linspace(0.0, 1.0, ns, device="cuda")
    Tp = T.clone()
    out = torch.zeros(3, dtype=torch.float64, device="cuda")
    for bad, where in ((float("nan"), "u"), (float("inf"), "T")):
        ub, Tb = u.clone(), T.clone()
        (ub if where == "u" else Tb)[1234] = bad
        gb.residual_noalloc(ub.data_ptr(), Tb.data_ptr(), up.data_ptr(), Tp.data_ptr(), ns,
                            out.data_ptr(), stream.cuda_stream)
        r = out.cpu().tolist()
        assert r[2] == 1.0
        assert r[0] != r[0] and r[1] != r[1]  # NaN
        assert not (r[0] < 1e-6) and not (r[1] < 1e-6)
    gb.residual_noalloc(u.data_ptr(), T.data_ptr(), up.data_ptr(), Tp.data_ptr(), ns,
                        out.data_ptr(), stream.cuda_stream)
    r = out.cpu().tolist()
    want_u = float(torch.linalg.vector_norm(u.double() - up.double()) /
                   torch.linalg.vector_norm(u.double()))
    assert r[2] == 0.0 and r[1] == 0.0
    assert r[0] == pytest.approx(want_u, rel=1e-5)


def test_noalloc_keeps_the_current_device(env):
    """The call runs on its stream's device and leaves the thread's current device as it was."""
    gb, torch = env
    ns = 64
    buf = torch.ones(3 * ns, device="cuda")
    out = torch.zeros(3, dtype=torch.float64, device="cuda")
    before = torch.cuda.current_device()
    gb.residual_noalloc(buf.data_ptr(), buf.data_ptr(), buf.data_ptr(), buf.data_ptr(), ns,
                        out.data_ptr(), torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    assert torch.cuda.current_device() == before
