"""Pins of the oracle's full time stepping (streaming, walls, forcing) against closed-form
solutions of the macroscopic equations (Eqs. 1-5)."""
import math

import numpy as np
import pytest


def _run(orc, pb, steps):
    o = orc.Oracle(orc.map_problem(pb))
    o.step(steps)
    return o


@pytest.mark.parametrize("sigma,nu_e,alpha", [(1.0, 0.1, 0.05), (2.0, 0.05, 0.2)])
def test_conduction_profile_is_exact(orc, sigma, nu_e, alpha):
    """Pure conduction between a hot (T=1) and a cold (T=0) Dirichlet wall: the
    anti-bounce-back steady state is T(x) = 1 - (x + 1/2)/N exactly, and the wall Nusselt
    numbers of Eq. 53 are +1 and -1."""
    N = 8
    pb = dict(nx=N, ny=4, nz=3, mapping="lattice", nu_e=nu_e, alpha_f=alpha, sigma=sigma,
              gbeta=0.0, flow_bc=[1] * 6, heat_bc=[2, 2, 1, 1, 1, 1],
              face_T=[1, 0, 0, 0, 0, 0], T_init=0.5)
    o = _run(orc, pb, int(40 * N * N * sigma / alpha))
    _, u, T = o.macros()
    x = np.arange(N)
    assert np.abs(T - (1 - (x + 0.5) / N)).max() < 1e-12
    assert np.abs(u).max() < 1e-14
    assert orc.nusselt(T, 0, 1.0, N)[0] == pytest.approx(1.0, abs=1e-10)
    assert orc.nusselt(T, 1, 0.0, N)[0] == pytest.approx(-1.0, abs=1e-10)


@pytest.mark.parametrize("Fphi,a", [(0.3, 1e-4), (0.0, 1e-4), (1.2, 5e-4)])
def test_uniform_darcy_forchheimer_flow(orc, Fphi, a):
    """Periodic box driven by a body force a: the steady velocity solves
    (nu/K) u + (F_phi/sqrt K) u^2 = a (Eq. 4 with F = 0)."""
    nu_e, phi, K = 0.1, 0.5, 0.5
    pb = dict(nx=2, ny=2, nz=2, mapping="lattice", nu_e=nu_e, phi=phi, K=K, F_phi=Fphi,
              accel=[a, 0, 0])
    o = _run(orc, pb, 2000)
    _, u, _ = o.macros()
    nu = nu_e
    if Fphi > 0:
        c = Fphi / math.sqrt(K)
        ue = (-nu / K + math.sqrt((nu / K) ** 2 + 4 * c * a)) / (2 * c)
    else:
        ue = K * a / nu
    assert u[0].mean() == pytest.approx(ue, rel=1e-10)
    assert np.abs(u[1:]).max() < 1e-14


def _poiseuille_error(orc, N, Da=0.0375, phi=0.6, nu_e=0.1, a=1e-5):
    K = Da * N * N
    pb = dict(nx=1, ny=N, nz=1, mapping="lattice", nu_e=nu_e, phi=phi, K=K, F_phi=0.0,
              accel=[a, 0, 0], flow_bc=[0, 0, 1, 1, 0, 0], heat_bc=[0, 0, 1, 1, 0, 0])
    lp = orc.map_problem(pb)
    o = orc.Oracle(lp)
    o.step(int(25 * K / (phi * lp.nu)))
    _, u, _ = o.macros()
    ux = u[0, 0, :, 0]
    y = np.arange(N)
    r = math.sqrt(phi / K)  # J = 1
    ua = (K * a / lp.nu) * (1 - np.cosh(r * (y - (N - 1) / 2)) / np.cosh(r * N / 2))
    return math.sqrt(np.sum((ux - ua) ** 2) / np.sum(ua ** 2))  # Eq. 52


def test_brinkman_poiseuille_second_order(orc):
    """Brinkman-Darcy channel (F_phi = 0) between halfway walls: the relative global error
    of Eq. 52 against u(y) = (K a / nu)[1 - cosh(r (y - y_c)) / cosh(r N / 2)],
    r = sqrt(phi / (J K)), falls at second order in the grid spacing (Sec. 4.1)."""
    E = [_poiseuille_error(orc, N) for N in (16, 32, 64)]
    slopes = [math.log2(E[i] / E[i + 1]) for i in range(2)]
    assert E[0] < 5e-3
    assert all(1.8 < s < 2.2 for s in slopes), (E, slopes)


def test_couette_flow_is_exact(orc):
    """Moving top wall, resting bottom wall, no medium: u_x = u_w (y + 1/2) / N exactly."""
    N = 12
    pb = dict(nx=1, ny=N, nz=1, mapping="lattice", nu_e=0.1, flow_bc=[0, 0, 1, 2, 0, 0],
              heat_bc=[0, 0, 1, 1, 0, 0],
              face_u=[(0, 0, 0)] * 3 + [(0.01, 0, 0)] + [(0, 0, 0)] * 2)
    o = _run(orc, pb, 12000)
    _, u, _ = o.macros()
    assert np.abs(u[0, 0, :, 0] - 0.01 * (np.arange(N) + 0.5) / N).max() < 1e-13


def test_brinkman_couette(orc):
    """Moving wall over a Brinkman medium: u = u_w sinh(r (y + 1/2)) / sinh(r N)."""
    N, phi, K = 24, 0.8, 20.0
    pb = dict(nx=1, ny=N, nz=1, mapping="lattice", nu_e=0.1, phi=phi, K=K, F_phi=0.0,
              flow_bc=[0, 0, 1, 2, 0, 0], heat_bc=[0, 0, 1, 1, 0, 0],
              face_u=[(0, 0, 0)] * 3 + [(0.01, 0, 0)] + [(0, 0, 0)] * 2)
    o = _run(orc, pb, 6000)
    _, u, _ = o.macros()
    r = math.sqrt(phi / K)
    ua = 0.01 * np.sinh(r * (np.arange(N) + 0.5)) / np.sinh(r * N)
    ux = u[0, 0, :, 0]
    assert math.sqrt(np.sum((ux - ua) ** 2) / np.sum(ua ** 2)) < 2e-3


@pytest.mark.parametrize("phi,K", [(1.0, math.inf), (0.6, 200.0)])
def test_shear_wave_decay(orc, phi, K):
    """u_x = A sin(k y) decays at nu_e k^2 + phi nu / K (Eq. 2 with Eq. 4, nu_e from
    Eq. 32); the lattice reproduces it to O(k^2)."""
    N = 32
    k = 2 * math.pi / N
    pb = dict(nx=1, ny=N, nz=1, mapping="lattice", nu_e=0.05, phi=phi,
              K=K if K < math.inf else 0.0, Da=None, F_phi=0.0)
    lp = orc.map_problem(pb)
    o = orc.Oracle(lp)
    uf = np.zeros((3, 1, N, 1))
    uf[0, 0, :, 0] = 1e-3 * np.sin(k * np.arange(N))
    o.init_equilibrium(0.5, None, uf)
    o.step(50)
    a1 = o.macros()[1][0, 0, :, 0]
    o.step(400)
    a2 = o.macros()[1][0, 0, :, 0]
    rate = -math.log(np.dot(a2, uf[0, 0, :, 0]) / np.dot(a1, uf[0, 0, :, 0])) / 400
    want = lp.nu_e * k * k + (phi * lp.nu / K if K < math.inf else 0.0)
    assert rate == pytest.approx(want, rel=5e-3)


@pytest.mark.parametrize("sigma,ux,phi,alpha_m", [(1.0, 0.0, 1.0, -1.0), (2.0, 0.02, 1.0, -1.0),
                                                  (1.5, 0.0, 0.4, 0.01)])
def test_temperature_wave(orc, sigma, ux, phi, alpha_m):
    """sigma dT/dt + u.grad T = alpha_e lap T (Eq. 3): a cosine mode decays at
    alpha_e k^2 / sigma and travels at u / sigma, with alpha_e from Eq. 41; with a solid
    matrix of diffusivity alpha_m, alpha_e = phi alpha_f + (1 - phi) alpha_m (Sec. 2)."""
    N = 32
    k = 2 * math.pi / N
    pb = dict(nx=N, ny=1, nz=1, mapping="lattice", nu_e=0.05, alpha_f=0.04, sigma=sigma,
              phi=phi, alpha_m=alpha_m)
    lp = orc.map_problem(pb)
    o = orc.Oracle(lp)
    x = np.arange(N)
    uf = np.zeros((3, 1, 1, N))
    uf[0] = ux
    o.init_equilibrium(0.5, (0.5 + 1e-2 * np.cos(k * x)).reshape(1, 1, N), uf)
    o.step(20)
    T1 = o.macros()[2][0, 0, :] - 0.5
    o.step(300)
    T2 = o.macros()[2][0, 0, :] - 0.5
    z1, z2 = np.sum(T1 * np.exp(-1j * k * x)), np.sum(T2 * np.exp(-1j * k * x))
    rate = -math.log(abs(z2) / abs(z1)) / 300
    speed = -np.angle(z2 / z1) / 300 / k
    alpha_e = phi * 0.04 + (1.0 - phi) * alpha_m if alpha_m >= 0 else 0.04
    assert rate == pytest.approx(alpha_e * k * k / sigma, rel=5e-3)
    assert speed == pytest.approx(ux / sigma, abs=1e-5)


def test_uniform_stream_through_inlet_and_outflow(orc):
    """A uniform stream u0 entering through the velocity inlet and leaving through the
    convective outflow is an exact steady state (Eq. 24 populations are kept)."""
    pb = dict(nx=8, ny=3, nz=2, mapping="channel", Re=10, u0=0.01, Pr=0.71, Ri=0.0,
              flow_bc=[2, 3, 0, 0, 0, 0], heat_bc=[2, 3, 0, 0, 0, 0],
              face_u=[(0.01, 0, 0)] + [(0, 0, 0)] * 5, face_T=[0.3] + [0] * 5)
    o = orc.Oracle(orc.map_problem(pb))
    uf = np.zeros((3, 2, 3, 8))
    uf[0] = 0.01
    o.init_equilibrium(0.3, None, uf)
    o.step(200)
    rho, u, T = o.macros()
    assert np.abs(u[0] - 0.01).max() < 1e-13 and np.abs(u[1:]).max() < 1e-13
    assert np.abs(rho - 1).max() < 1e-13 and np.abs(T - 0.3).max() < 1e-13


def test_channel_outflow_mass_balance(orc):
    """Walled porous channel with inlet and anchored convective outflow reaches a steady
    state in which the flux through every cross-section is the same and the outlet density
    equals rho0 (continuity, Eq. 1)."""
    from lbm_inputs import channel_problem

    pb = channel_problem(32, 8, 2, Da=1e-2)
    o = orc.Oracle(orc.map_problem(pb))
    o.step(6000)
    rho, u, _ = o.macros()
    flux = u[0].sum(axis=(0, 1))
    assert np.ptp(flux) / flux.mean() < 1e-6
    assert np.abs(rho[:, :, -1] - 1.0).max() < 1e-12


@pytest.mark.parametrize("p,Fphi", [(0.45, 0.0), (0.8, -1.0)])
def test_porosity_field_medium(orc, p, Fphi):
    """A porosity field sets each site's medium from Eq. 6: K = K_ref [p^3 / (1 - p)^2] /
    [p_ref^3 / (1 - p_ref)^2] (Kozeny-Carman about the reference porosity) and, for Ergun's
    inertia, F_phi = 1.75 / sqrt(150 p^3).  A field uniform at p in a forced periodic box
    must then flow at the uniform Darcy-Forchheimer velocity of that K and F_phi."""
    nu_e, K_ref, p_ref, a = 0.1, 0.5, 0.6, 2e-4
    field = np.full((2, 2, 2), p)
    pb = dict(nx=2, ny=2, nz=2, mapping="lattice", nu_e=nu_e, phi=p_ref, K=K_ref, F_phi=Fphi,
              accel=[a, 0, 0], phi_field=field, phi_ref=p_ref)
    o = _run(orc, pb, 3000)
    _, u, _ = o.macros()
    K = K_ref * (p ** 3 / (1 - p) ** 2) / (p_ref ** 3 / (1 - p_ref) ** 2)
    nu = nu_e
    if Fphi < 0:
        c = 1.75 / math.sqrt(150 * p ** 3) / math.sqrt(K)
        ue = (-nu / K + math.sqrt((nu / K) ** 2 + 4 * c * a)) / (2 * c)
    else:
        ue = K * a / nu
    assert u[0].mean() == pytest.approx(ue, rel=1e-9)
