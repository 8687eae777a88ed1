"""Seeded synthetic inputs shared by the oracle tests, the GPU tests and the benchmark.

This module holds no arithmetic of the lattice Boltzmann method: it only draws seeded
random numbers and shapes them into the problem inputs that the paper's workloads use
(porosity fields, perturbation fields, problem statements).  Both sides receive the same
arrays from here; neither side's arithmetic lives here.
"""
from __future__ import annotations

import math

import numpy as np

FACES = ("x-", "x+", "y-", "y+", "z-", "z+")


def gaussian_field(shape, seed: int, corr: float) -> np.ndarray:
    """Zero-mean, unit-variance Gaussian random field on a [z][y][x] grid.

    White noise from PCG64(seed), smoothed by a separable periodic Gaussian kernel of
    standard deviation ``corr`` lattice spacings along each axis (FFT convolution), then
    rescaled to unit variance.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    w = rng.standard_normal(shape)
    out = np.fft.fftn(w)
    for ax, n in enumerate(shape):
        k = np.fft.fftfreq(n)
        kern = np.exp(-0.5 * (2 * math.pi * k * corr) ** 2)
        sh = [1] * len(shape)
        sh[ax] = n
        out = out * kern.reshape(sh)
    f = np.real(np.fft.ifftn(out))
    f -= f.mean()
    sd = f.std()
    return f / sd if sd > 0 else f


def porosity_field(nx: int, ny: int, nz: int, seed: int = 20161110, mean: float = 0.6,
                   std: float = 0.05, lo: float = 0.4, hi: float = 0.9,
                   corr: float | None = None) -> np.ndarray:
    """Heterogeneous porosity phi(x) [z][y][x]: Gaussian field, mean 0.6, std 0.05, clipped
    to [0.4, 0.9]; correlation length L/16 with L the largest edge."""
    if corr is None:
        corr = max(nx, ny, nz) / 16.0
    g = gaussian_field((nz, ny, nx), seed, corr)
    return np.clip(mean + std * g, lo, hi)


def uniform(shape, seed: int, lo: float = -1.0, hi: float = 1.0) -> np.ndarray:
    """Seeded uniform random numbers (PCG64)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return rng.uniform(lo, hi, size=shape)


def random_macros(nx: int, ny: int, nz: int, seed: int, u_amp: float = 0.03,
                  rho_amp: float = 0.01, T_lo: float = 0.0, T_hi: float = 1.0):
    """Random density, velocity and temperature fields for single-step parity checks:
    rho in 1 +- rho_amp, |u_a| <= u_amp, T in [T_lo, T_hi]; shapes [z][y][x] / [3][z][y][x]."""
    rng = np.random.Generator(np.random.PCG64(seed))
    rho = 1.0 + rho_amp * rng.uniform(-1, 1, size=(nz, ny, nx))
    u = u_amp * rng.uniform(-1, 1, size=(3, nz, ny, nx))
    T = rng.uniform(T_lo, T_hi, size=(nz, ny, nx))
    return rho, u, T


def cavity_problem(n: int, Ra: float, Da: float, phi: float, Pr: float = 1.0,
                   F_phi: float = -1.0, J: float = 1.0, sigma: float = 1.0, **kw) -> dict:
    """Porous cavity of Sec. 4.2: hot x-low wall (T=1), cold x-high wall (T=0), the other
    four walls adiabatic, no-slip everywhere, gravity along -z, initial T = 0.5.
    ``F_phi=-1`` selects Ergun's inertia coefficient (Eq. 6)."""
    pb = dict(nx=n, ny=n, nz=n, mapping="cavity", Ra=Ra, Da=Da, Pr=Pr, J=J, sigma=sigma,
              phi=phi, F_phi=F_phi, flow_bc=[1] * 6, heat_bc=[2, 2, 1, 1, 1, 1],
              face_T=[1.0, 0.0, 0.0, 0.0, 0.0, 0.0], T_init=0.5, T0=0.5,
              gravity_axis=2, gravity_sign=-1)
    pb.update(kw)
    return pb


def channel_problem(nx: int, ny: int, nz: int, Re: float = 10.0, u0: float = 0.01,
                    Pr: float = 0.71, Ri: float = 1.0, Da: float = 1e-3, phi: float = 0.7,
                    F_phi: float = -1.0, **kw) -> dict:
    """Porous channel: velocity inlet u0 at T=0 on x-low, convective outflow on x-high,
    no-slip walls at y-low (T=0) and y-high (T=1), periodic in z, gravity along -y; the
    channel height ny is the length scale of Re, Ri and Da."""
    pb = dict(nx=nx, ny=ny, nz=nz, mapping="channel", Re=Re, u0=u0, Pr=Pr, Ri=Ri, Da=Da,
              phi=phi, F_phi=F_phi, flow_bc=[2, 3, 1, 1, 0, 0], heat_bc=[2, 3, 2, 2, 0, 0],
              face_T=[0.0, 0.0, 0.0, 1.0, 0.0, 0.0],
              face_u=[(u0, 0.0, 0.0)] + [(0.0, 0.0, 0.0)] * 5,
              T_init=0.0, T0=0.5, gravity_axis=1, gravity_sign=-1)
    pb.update(kw)
    return pb


def paper_channel(ny: int, Re: float = 10.0, Da: float = 1e-2, phi: float = 0.6,
                  u0: float = 0.01, u1: float = 0.01, Pr: float = 1.0, Ra: float = 100.0,
                  nx: int = 1, nz: int = 1, walls: str = "halfway") -> dict:
    """The porous channel of Sec. 4.1: plates at y-low (cold, T = 0) and y-high (hot, T = 1, moving
    along x at u0), fluid injected through the lower plate and withdrawn through the upper one at
    u1, periodic in x and z, Brinkman-Darcy medium (F_phi = 0), H = ny for Re = H u1 / nu, Da and
    Ra (Ri = Ra / (Re^2 Pr)), gravity along -y.  The external force of Eq. 47 enters through its
    uniform part nu u1 / K = u1^2 / (Re Da H); its y-dependent part only offsets the buoyancy's,
    which in this one-dimensional flow a pressure gradient balances as well.  walls="halfway":
    plates half a spacing outside the first and last rows (H = ny); walls="nee": the first and
    last rows are the plates, by non-equilibrium extrapolation (H = ny - 1)."""
    H = ny if walls == "halfway" else ny - 1
    kind = 2 if walls == "halfway" else 4
    return dict(nx=nx, ny=ny, nz=nz, mapping="channel", L=H, Re=Re, u0=u1, Pr=Pr,
                Ri=Ra / (Re * Re * Pr), Da=Da, phi=phi, F_phi=0.0,
                flow_bc=[0, 0, kind, kind, 0, 0], heat_bc=[0, 0, kind, kind, 0, 0],
                face_T=[0.0, 0.0, 0.0, 1.0, 0.0, 0.0],
                face_u=[(0.0, 0.0, 0.0), (0.0, 0.0, 0.0), (0.0, u1, 0.0), (u0, u1, 0.0),
                        (0.0, 0.0, 0.0), (0.0, 0.0, 0.0)],
                accel=[0.0, u1 * u1 / (Re * Da * H), 0.0], T_init=0.5, T0=0.5,
                gravity_axis=1, gravity_sign=-1)


def batch_cavities(n: int = 64, seed: int = 2016, sizes=(32, 48, 64, 96, 128),
                   phi_range=(0.4, 0.9), log_da=(-5.0, -1.0), log_ra=(3.0, 6.0),
                   Pr: float = 0.71) -> list:
    """n independent porous cavities: edge drawn uniformly from `sizes`, porosity uniform in
    phi_range, log10 Da and log10 Ra uniform in their ranges (PCG64(seed)); Ergun F_phi."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for _ in range(n):
        edge = int(rng.choice(sizes))
        phi = float(rng.uniform(*phi_range))
        Da = float(10.0 ** rng.uniform(*log_da))
        Ra = float(10.0 ** rng.uniform(*log_ra))
        out.append(cavity_problem(edge, Ra=Ra, Da=Da, phi=phi, Pr=Pr))
    return out


def serving_mix(n: int = 24, seed: int = 5, rate: float = 20.0,
                edges=(32, 48, 64, 96, 128, 160, 192), widths=(32, 64),
                p_channel: float = 0.4, p_fp16: float = 0.5, p_melt: float = 0.1) -> list:
    """Seeded stream of solve requests: (arrival time in s, problem).  Poisson arrivals of
    mean `rate` per second; a request is, with probability p_melt, a melting cavity (clear
    fluid, edge from `edges`, solid at T = 0 below a melting point of 0.5, Stefan number 1,
    log10 Ra in [4, 6], FP32: the enthalpy model of App. B), else with probability
    p_channel a porous channel of length 4W and section W x W (W from `widths`, porosity
    0.7, log10 Da in [-3, -2]), else a porous cavity (edge from `edges`, porosity in
    [0.4, 0.9], log10 Da in [-5, -1], log10 Ra in [3, 6]); storage of the last two FP16
    with probability p_fp16, else FP32."""
    rng = np.random.Generator(np.random.PCG64(seed))
    t = 0.0
    out = []
    for _ in range(n):
        t += float(rng.exponential(1.0 / rate))
        storage = "fp16" if rng.uniform() < p_fp16 else "fp32"
        kind = rng.uniform()
        if kind < p_melt:
            edge = int(rng.choice(edges))
            pb = cavity_problem(edge, Ra=float(10.0 ** rng.uniform(4.0, 6.0)), Da=None,
                                phi=1.0, Pr=0.71, enthalpy=True, T_m=0.5, St=1.0, T_init=0.0)
            storage = "fp32"
        elif kind < p_melt + (1.0 - p_melt) * p_channel:
            w = int(rng.choice(widths))
            pb = channel_problem(4 * w, w, w, Da=float(10.0 ** rng.uniform(-3.0, -2.0)))
        else:
            edge = int(rng.choice(edges))
            pb = cavity_problem(edge, Ra=float(10.0 ** rng.uniform(3.0, 6.0)),
                                Da=float(10.0 ** rng.uniform(-5.0, -1.0)),
                                phi=float(rng.uniform(0.4, 0.9)), Pr=0.71)
        pb["storage"] = storage
        out.append((t, pb))
    return out
