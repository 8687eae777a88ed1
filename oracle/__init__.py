"""FP64 CPU oracle of the 3D DDF-MRT lattice Boltzmann model for porous-media convection
(Liu & He, arXiv:1611.03329).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` may import this package.  It shares no code with the CUDA
library: the arithmetic lives in ``lbm_oracle.c`` (plain loops, dense matrices, FP64) and
in the few plain definitions below (parameter mapping, Nusselt numbers, residual).

Pins: every function here is checked by ``tests/test_oracle_*.py`` against the lattice
definitions, closed forms, invariants and symmetries that the paper and the mathematics
fix, and against the cavity Nusselt numbers the paper prints; ``tests/test_oracle_mutants.py``
plants 41 plausible slips in a copy of the oracle and checks that a pin rejects each.  The
Nusselt discretisation (Eq. 53) is pinned by the exact conduction value and, at second order,
by the exponential temperature profile of the paper's channel.  Parity unpinned, in part:
the advection speed of the convective outflow (a reading; the paper has no outflow).  Its
steady states, which the pins check, are the same for every speed; and the corner convention
of node walls (which face's velocity a corner site takes), which the paper leaves open.
"""
from __future__ import annotations

import ctypes as C
import math
from dataclasses import dataclass, field
from typing import Optional, Sequence

import numpy as np

from . import build as _build

Q19, Q15, Q7 = 19, 15, 7
CS2 = 1.0 / 3.0  # c_s^2 with c = 1 (Sec. 3.1.2)

# face order: x-low, x-high, y-low, y-high, z-low, z-high
BC_PERIODIC, BC_WALL, BC_VELOCITY, BC_OUTFLOW, BC_NEE = 0, 1, 2, 3, 4
HT_PERIODIC, HT_ADIABATIC, HT_DIRICHLET, HT_OUTFLOW, HT_NEE_DIRICHLET, HT_NEE_ADIABATIC = range(6)

# Free relaxation rates of the D3Q19 and D3Q7 models chosen in Sec. 4.
PAPER_RATES = dict(s_e=1.1, s_eps=1.1, s_q=1.1, s_pi=1.1, s_m=1.2,
                   zeta_T=1.0, zeta_e=1.2, zeta_nu=1.2)


class _Lattice(C.Structure):
    _fields_ = [
        ("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int),
        ("rho0", C.c_double), ("T0", C.c_double), ("sigma", C.c_double), ("varpi", C.c_double),
        ("s", C.c_double * Q19),
        ("zeta_T", C.c_double), ("zeta_e", C.c_double), ("zeta_nu", C.c_double),
        ("alpha_f", C.c_double), ("alpha_m", C.c_double), ("Gamma", C.c_double),
        ("nu", C.c_double),
        ("phi", C.c_double), ("K", C.c_double), ("F_phi", C.c_double),
        ("phi_ref", C.c_double),
        ("buoy", C.c_double * 3), ("accel", C.c_double * 3),
        ("flow_bc", C.c_int * 6), ("heat_bc", C.c_int * 6),
        ("face_T", C.c_double * 6), ("face_u", (C.c_double * 3) * 6),
        ("U_out", C.c_double),
        ("enthalpy", C.c_int), ("flow_off", C.c_int),
        ("c_pl", C.c_double), ("c_ref", C.c_double),
        ("sigma_s", C.c_double), ("sigma_l", C.c_double),
        ("T_s", C.c_double), ("T_l", C.c_double), ("L_a", C.c_double),
        ("alpha_s", C.c_double), ("alpha_l", C.c_double),
        ("q", C.c_int),
    ]


_lib = None


def lib():
    """Load (building if needed) the oracle shared library."""
    global _lib
    if _lib is None:
        path = _build.build()
        L = C.CDLL(path)
        dp = C.POINTER(C.c_double)
        L.orc_create.restype = C.c_void_p
        L.orc_create.argtypes = [C.POINTER(_Lattice), dp]
        L.orc_destroy.argtypes = [C.c_void_p]
        L.orc_init_equilibrium.argtypes = [C.c_void_p, C.c_double, dp, dp]
        L.orc_set_populations.argtypes = [C.c_void_p, dp, dp]
        L.orc_get_populations.argtypes = [C.c_void_p, dp, dp]
        L.orc_step.argtypes = [C.c_void_p, C.c_int]
        L.orc_macros.argtypes = [C.c_void_p, dp, dp, dp]
        L.orc_steps_done.restype = C.c_long
        L.orc_steps_done.argtypes = [C.c_void_p]
        L.orc_set_threads.argtypes = [C.c_int]
        L.orc_gate_margin.argtypes = [C.c_void_p, dp]
        L.orc_gate_margin_reset.argtypes = [C.c_void_p]
        L.orc_max_threads.restype = C.c_int
        L.orc_sizeof_lattice.restype = C.c_int
        L.orc_tables.argtypes = [dp] * 7
        L.orc_feq19.argtypes = [C.c_double, dp, C.c_double, C.c_double, dp]
        L.orc_meq19_eq21.argtypes = [C.c_double, dp, C.c_double, C.c_double, dp]
        L.orc_stilde19.argtypes = [dp, dp, C.c_double, C.c_double, dp]
        L.orc_geq7.argtypes = [C.c_double, dp, C.c_double, C.c_double, dp]
        L.orc_neq7.argtypes = [C.c_double, dp, C.c_double, C.c_double, dp]
        L.orc_force.argtypes = [dp, dp, C.c_double, C.c_double, C.c_double, C.c_double, dp]
        L.orc_velocity.argtypes = [dp, dp, C.c_double, C.c_double, C.c_double, C.c_double,
                                   C.c_double, dp]
        L.orc_collide_site.argtypes = [C.POINTER(_Lattice), dp, dp, C.c_double, C.c_double,
                                       C.c_double, C.c_double, dp, dp, dp]
        L.orc_enthalpy_state.argtypes = [C.POINTER(_Lattice), C.c_double, C.c_double, dp, dp]
        L.orc_enthalpy_of.argtypes = [C.POINTER(_Lattice), C.c_double, C.c_double]
        L.orc_enthalpy_of.restype = C.c_double
        L.orc_geq7_enthalpy.argtypes = [C.POINTER(_Lattice), C.c_double, C.c_double, dp, dp]
        L.orc_tables15.argtypes = [dp] * 4
        L.orc_feq15.argtypes = [C.c_double, dp, C.c_double, C.c_double, dp]
        L.orc_meq15_eq15.argtypes = [C.c_double, dp, C.c_double, C.c_double, dp]
        L.orc_stilde15.argtypes = [dp, dp, C.c_double, C.c_double, dp]
        L.orc_velocity15.argtypes = [dp, dp, C.c_double, C.c_double, C.c_double, C.c_double,
                                     C.c_double, dp]
        if L.orc_sizeof_lattice() != C.sizeof(_Lattice):
            raise RuntimeError("oracle struct layout mismatch")
        _lib = L
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _vec(v) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(v, dtype=np.float64))


def set_threads(n: int) -> None:
    lib().orc_set_threads(int(n))


def max_threads() -> int:
    return int(lib().orc_max_threads())


# ---- tables and pointwise formulas ------------------------------------------------------

def tables() -> dict:
    """e19 (3x19, Eq. 19), w19, M (Eq. A2), M^-1 (Gauss-Jordan), e7 (Eq. 12), N (Eq. 36),
    N^-1 (as printed in Eq. 43)."""
    e19 = np.zeros((3, Q19)); w19 = np.zeros(Q19); m = np.zeros((Q19, Q19))
    minv = np.zeros((Q19, Q19)); e7 = np.zeros((3, Q7)); n7 = np.zeros((Q7, Q7))
    ninv = np.zeros((Q7, Q7))
    lib().orc_tables(_p(e19), _p(w19), _p(m), _p(minv), _p(e7), _p(n7), _p(ninv))
    return dict(e19=e19, w19=w19, M=m, Minv=minv, e7=e7, N=n7, Ninv=ninv)


def tables15() -> dict:
    """e15 (3x15, Eq. 12), w15 (under Eq. 18), M (Eq. A1), M^-1 (Gauss-Jordan)."""
    e15 = np.zeros((3, Q15)); w15 = np.zeros(Q15); m = np.zeros((Q15, Q15))
    minv = np.zeros((Q15, Q15))
    lib().orc_tables15(_p(e15), _p(w15), _p(m), _p(minv))
    return dict(e15=e15, w15=w15, M=m, Minv=minv)


def feq15(rho, u, phi, rho0=1.0) -> np.ndarray:
    out = np.zeros(Q15)
    lib().orc_feq15(float(rho), _p(_vec(u)), float(phi), float(rho0), _p(out))
    return out


def meq15_eq15(rho, u, phi, rho0=1.0) -> np.ndarray:
    out = np.zeros(Q15)
    lib().orc_meq15_eq15(float(rho), _p(_vec(u)), float(phi), float(rho0), _p(out))
    return out


def stilde15(u, F, phi, rho0=1.0) -> np.ndarray:
    out = np.zeros(Q15)
    lib().orc_stilde15(_p(_vec(u)), _p(_vec(F)), float(phi), float(rho0), _p(out))
    return out


def velocity15(f, G, phi, nu, K, Fphi, rho0=1.0) -> np.ndarray:
    out = np.zeros(3)
    lib().orc_velocity15(_p(_vec(f)), _p(_vec(G)), float(phi), float(nu), float(K),
                         float(Fphi), float(rho0), _p(out))
    return out


def feq19(rho, u, phi, rho0=1.0) -> np.ndarray:
    out = np.zeros(Q19)
    lib().orc_feq19(float(rho), _p(_vec(u)), float(phi), float(rho0), _p(out))
    return out


def meq19_eq21(rho, u, phi, rho0=1.0) -> np.ndarray:
    out = np.zeros(Q19)
    lib().orc_meq19_eq21(float(rho), _p(_vec(u)), float(phi), float(rho0), _p(out))
    return out


def stilde19(u, F, phi, rho0=1.0) -> np.ndarray:
    out = np.zeros(Q19)
    lib().orc_stilde19(_p(_vec(u)), _p(_vec(F)), float(phi), float(rho0), _p(out))
    return out


def geq7(T, u, sigma=1.0, varpi=0.5) -> np.ndarray:
    out = np.zeros(Q7)
    lib().orc_geq7(float(T), _p(_vec(u)), float(sigma), float(varpi), _p(out))
    return out


def neq7(T, u, sigma=1.0, varpi=0.5) -> np.ndarray:
    out = np.zeros(Q7)
    lib().orc_neq7(float(T), _p(_vec(u)), float(sigma), float(varpi), _p(out))
    return out


def force(u, G, phi, nu, K, Fphi) -> np.ndarray:
    out = np.zeros(3)
    lib().orc_force(_p(_vec(u)), _p(_vec(G)), float(phi), float(nu), float(K), float(Fphi),
                    _p(out))
    return out


def velocity(f, G, phi, nu, K, Fphi, rho0=1.0) -> np.ndarray:
    out = np.zeros(3)
    lib().orc_velocity(_p(_vec(f)), _p(_vec(G)), float(phi), float(nu), float(K),
                       float(Fphi), float(rho0), _p(out))
    return out


# ---- parameter mapping (Sec. 2 and Sec. 4) ----------------------------------------------

@dataclass
class LatticeParams:
    """Lattice-unit parameters of one problem (dt = dx = 1, c = 1)."""
    nx: int
    ny: int
    nz: int
    rho0: float = 1.0
    T0: float = 0.5
    sigma: float = 1.0
    varpi: float = 0.5
    s: Sequence[float] = ()
    zeta_T: float = 1.0
    zeta_e: float = 1.2
    zeta_nu: float = 1.2
    alpha_f: float = 0.0
    alpha_m: float = -1.0
    Gamma: float = 1.0
    nu: float = 0.0
    nu_e: float = 0.0
    phi: float = 1.0
    K: float = math.inf
    F_phi: float = 0.0
    phi_ref: float = 1.0
    buoy: Sequence[float] = (0.0, 0.0, 0.0)
    accel: Sequence[float] = (0.0, 0.0, 0.0)
    flow_bc: Sequence[int] = (0,) * 6
    heat_bc: Sequence[int] = (0,) * 6
    face_T: Sequence[float] = (0.0,) * 6
    face_u: Sequence[Sequence[float]] = ((0.0, 0.0, 0.0),) * 6
    U_out: float = 0.0
    s_nu: float = 1.0
    zeta_alpha: float = 1.0
    gbeta: float = 0.0
    L: float = 1.0
    dT: float = 1.0
    T_init: float = 0.5
    enthalpy: bool = False
    flow_off: bool = False
    c_pl: float = 1.0
    c_ref: float = 1.0
    sigma_s: float = 1.0
    sigma_l: float = 1.0
    T_s: float = 0.0
    T_l: float = 0.0
    L_a: float = 1.0
    alpha_s: float = 0.0
    alpha_l: float = 0.0
    q: int = 19
    phi_field: Optional[np.ndarray] = field(default=None, repr=False)

    def to_c(self) -> _Lattice:
        c = _Lattice()
        c.nx, c.ny, c.nz = self.nx, self.ny, self.nz
        c.rho0, c.T0, c.sigma, c.varpi = self.rho0, self.T0, self.sigma, self.varpi
        for k in range(len(self.s)):
            c.s[k] = self.s[k]
        c.zeta_T, c.zeta_e, c.zeta_nu = self.zeta_T, self.zeta_e, self.zeta_nu
        c.alpha_f, c.alpha_m, c.Gamma = self.alpha_f, self.alpha_m, self.Gamma
        c.nu = self.nu
        c.phi, c.K, c.F_phi, c.phi_ref = self.phi, self.K, self.F_phi, self.phi_ref
        for a in range(3):
            c.buoy[a] = self.buoy[a]
            c.accel[a] = self.accel[a]
        for k in range(6):
            c.flow_bc[k] = self.flow_bc[k]
            c.heat_bc[k] = self.heat_bc[k]
            c.face_T[k] = self.face_T[k]
            for a in range(3):
                c.face_u[k][a] = self.face_u[k][a]
        c.U_out = self.U_out
        c.enthalpy = int(self.enthalpy)
        c.flow_off = int(self.flow_off)
        c.c_pl, c.c_ref = self.c_pl, self.c_ref
        c.sigma_s, c.sigma_l = self.sigma_s, self.sigma_l
        c.T_s, c.T_l, c.L_a = self.T_s, self.T_l, self.L_a
        c.alpha_s, c.alpha_l = self.alpha_s, self.alpha_l
        c.q = int(self.q)
        return c


def relaxation_vector(s_nu, s_e=1.1, s_eps=1.1, s_q=1.1, s_pi=1.1, s_m=1.2):
    """Diagonal of Lambda in the moment order of Eq. 20 (Eq. 22), s_rho = s_j = 1."""
    s_rho = s_j = 1.0
    return [s_rho, s_e, s_eps, s_j, s_q, s_j, s_q, s_j, s_q,
            s_nu, s_pi, s_nu, s_pi, s_nu, s_nu, s_nu, s_m, s_m, s_m]


def relaxation_vector15(s_nu, s_e=1.1, s_eps=1.1, s_q=1.1, s_m=1.2):
    """Diagonal of Lambda in the moment order of Eq. 13 (Eq. 16), s_rho = s_j = 1."""
    s_rho = s_j = 1.0
    return [s_rho, s_e, s_eps, s_j, s_q, s_j, s_q, s_j, s_q,
            s_nu, s_nu, s_nu, s_nu, s_nu, s_m]


def ergun_F(phi: float) -> float:
    """Eq. 6: F_phi = 1.75 / sqrt(150 phi^3)."""
    return 1.75 / math.sqrt(150.0 * phi ** 3)


def map_problem(pb: dict) -> LatticeParams:
    """Dimensionless problem statement -> lattice parameters.

    cavity  : Eq. 56 (1/s_nu and 1/zeta_alpha), u_c = Ma c_s = sqrt(g beta dT L), Da = K/L^2.
    channel : Eq. 51 read with 1/s_nu on the left (nu_e = J H u0 / Re), g beta from the
              Richardson number Ri = g beta dT H / u0^2, Da = K/H^2.
    lattice : nu_e, alpha_f and gbeta given directly in lattice units.
    Then nu = nu_e / J (Eq. 7), alpha_e = Gamma alpha_f (Eq. 7) or phi alpha_f + (1-phi)
    alpha_m (Sec. 2), 1/zeta_alpha = 1/2 + alpha_e / (sigma c_sT^2) (Eq. 41, c_sT^2 = varpi/3).
    """
    nx, ny, nz = int(pb["nx"]), int(pb["ny"]), int(pb["nz"])
    mapping = pb.get("mapping", "cavity")
    J = float(pb.get("J", 1.0)); sigma = float(pb.get("sigma", 1.0))
    Gamma = float(pb.get("Gamma", 1.0)); Pr = float(pb.get("Pr", 1.0))
    varpi = float(pb.get("varpi", 0.5)); dT = float(pb.get("dT", 1.0))
    rates = {k: float(pb.get(k, v)) for k, v in PAPER_RATES.items()}
    if mapping == "cavity":
        L = float(pb.get("L", nx))
        Ra = float(pb["Ra"]); Ma = float(pb.get("Ma", 0.1))
        inv_s_nu = 0.5 + Ma * J * L * math.sqrt(3.0 * Pr) / math.sqrt(Ra)
        nu_e = CS2 * (inv_s_nu - 0.5)                      # Eq. 32
        nu = nu_e / J
        alpha_f = nu / Pr
        gbeta = (Ma * math.sqrt(CS2)) ** 2 / (dT * L)
    elif mapping == "channel":
        L = float(pb.get("L", ny))
        Re = float(pb["Re"]); u0 = float(pb["u0"]); Ri = float(pb.get("Ri", 0.0))
        inv_s_nu = 0.5 + J * L * u0 / (CS2 * Re)
        nu_e = CS2 * (inv_s_nu - 0.5)
        nu = nu_e / J
        alpha_f = nu / Pr
        gbeta = Ri * u0 * u0 / (dT * L)
    elif mapping == "lattice":
        L = float(pb.get("L", nx))
        nu_e = float(pb["nu_e"])
        inv_s_nu = 0.5 + nu_e / CS2
        nu = nu_e / J
        alpha_f = float(pb.get("alpha_f", nu / Pr))
        gbeta = float(pb.get("gbeta", 0.0))
    else:
        raise ValueError(f"unknown mapping {mapping!r}")
    s_nu = 1.0 / inv_s_nu
    phi = float(pb.get("phi", 1.0))
    K = float(pb.get("K", 0.0))
    Da = pb.get("Da", None)
    if K <= 0:
        K = float(Da) * L * L if Da is not None else math.inf
    F_phi = float(pb.get("F_phi", 0.0))
    alpha_m = float(pb.get("alpha_m", -1.0))
    phi_field = pb.get("phi_field", None)
    phi_ref = float(pb.get("phi_ref", float(np.mean(phi_field)) if phi_field is not None else phi))
    csT2 = varpi / 3.0
    alpha_e = Gamma * alpha_f if alpha_m < 0 else phi * alpha_f + (1 - phi) * alpha_m
    zeta_alpha = 1.0 / (0.5 + alpha_e / (sigma * csT2))
    gaxis = int(pb.get("gravity_axis", 2)); gsign = int(pb.get("gravity_sign", -1))
    buoy = [0.0, 0.0, 0.0]
    buoy[gaxis] = -gsign * gbeta   # G = -g beta (T - T0) with g pointing along gsign*axis
    u0 = float(pb.get("u0", 0.0))
    U_out = float(pb.get("U_out", 0.0))
    if U_out <= 0:
        U_out = u0
    face_u = [tuple(float(v) for v in fu) for fu in pb.get("face_u", [(0.0, 0.0, 0.0)] * 6)]
    # enthalpy model (App. B): melting point T_m (T_s = T_l unless given), Stefan number
    # St = c_pl dT / L_a, c_ref the harmonic mean of c_pl and c_ps (Eq. B13), liquid
    # diffusivity = alpha_f, solid diffusivity alpha_f / alpha_ratio (alpha_l / alpha_s).
    ent = {}
    if pb.get("enthalpy", False):
        c_pl = float(pb.get("c_pl", 1.0)); c_ps = float(pb.get("c_ps", 1.0))
        T_m = float(pb.get("T_m", 0.5))
        ent = dict(enthalpy=True, flow_off=bool(pb.get("flow_off", False)), c_pl=c_pl,
                   c_ref=2.0 / (1.0 / c_pl + 1.0 / c_ps),
                   sigma_s=float(pb.get("sigma_s", sigma)), sigma_l=float(pb.get("sigma_l", sigma)),
                   T_s=float(pb.get("T_s", T_m)), T_l=float(pb.get("T_l", T_m)),
                   L_a=c_pl * dT / float(pb.get("St", 1.0)),
                   alpha_l=float(pb.get("alpha_l", alpha_f)),
                   alpha_s=float(pb.get("alpha_s", float(pb.get("alpha_l", alpha_f))
                                        / float(pb.get("alpha_ratio", 1.0)))))
    q = int(pb.get("q", Q19))  # flow lattice: D3Q19 (Sec. 3.1.2) or D3Q15 (Sec. 3.1.1)
    if q not in (Q15, Q19):
        raise ValueError(f"flow lattice D3Q{q}")
    return LatticeParams(
        **ent,
        nx=nx, ny=ny, nz=nz, rho0=float(pb.get("rho0", 1.0)), T0=float(pb.get("T0", 0.5)),
        sigma=sigma, varpi=varpi,
        s=(relaxation_vector15(s_nu, rates["s_e"], rates["s_eps"], rates["s_q"], rates["s_m"])
           if q == Q15 else
           relaxation_vector(s_nu, rates["s_e"], rates["s_eps"], rates["s_q"], rates["s_pi"],
                             rates["s_m"])),
        q=q,
        zeta_T=rates["zeta_T"], zeta_e=rates["zeta_e"], zeta_nu=rates["zeta_nu"],
        alpha_f=alpha_f, alpha_m=alpha_m, Gamma=Gamma, nu=nu, nu_e=nu_e,
        phi=phi, K=K, F_phi=F_phi, phi_ref=phi_ref,
        buoy=buoy, accel=[float(a) for a in pb.get("accel", (0.0, 0.0, 0.0))],
        flow_bc=list(pb.get("flow_bc", [BC_PERIODIC] * 6)),
        heat_bc=list(pb.get("heat_bc", [HT_PERIODIC] * 6)),
        face_T=[float(t) for t in pb.get("face_T", [0.0] * 6)], face_u=face_u,
        U_out=U_out, s_nu=s_nu, zeta_alpha=zeta_alpha, gbeta=gbeta, L=L, dT=dT,
        T_init=float(pb.get("T_init", pb.get("T0", 0.5))),
        phi_field=None if phi_field is None else np.asarray(phi_field, dtype=np.float64),
    )


# ---- the lattice state ---------------------------------------------------------------------

class Oracle:
    """One lattice advanced by the FP64 oracle.  Arrays are [q][z][y][x] (x fastest)."""

    def __init__(self, lp: LatticeParams):
        self.lp = lp
        self.shape = (lp.nz, lp.ny, lp.nx)
        self.ns = lp.nx * lp.ny * lp.nz
        self.q = int(lp.q)
        self._c = lp.to_c()
        phi = None
        if lp.phi_field is not None:
            self._phi = np.ascontiguousarray(lp.phi_field.reshape(-1), dtype=np.float64)
            phi = _p(self._phi)
        self._h = lib().orc_create(C.byref(self._c), phi)
        if not self._h:
            raise MemoryError("oracle allocation failed")
        self.init_equilibrium(lp.T_init)

    def close(self):
        if getattr(self, "_h", None):
            lib().orc_destroy(self._h)
            self._h = None

    def __del__(self):
        self.close()

    def init_equilibrium(self, T=0.5, T_field=None, u_field=None):
        tp = None
        up = None
        if T_field is not None:
            self._tf = np.ascontiguousarray(T_field, dtype=np.float64).reshape(-1)
            tp = _p(self._tf)
        if u_field is not None:
            self._uf = np.ascontiguousarray(u_field, dtype=np.float64).reshape(-1)
            up = _p(self._uf)
        lib().orc_init_equilibrium(self._h, float(T), tp, up)

    def set_populations(self, f: np.ndarray, g: np.ndarray):
        f = np.ascontiguousarray(f, dtype=np.float64)
        g = np.ascontiguousarray(g, dtype=np.float64)
        assert f.size == self.q * self.ns and g.size == Q7 * self.ns
        lib().orc_set_populations(self._h, _p(f), _p(g))

    def populations(self):
        f = np.zeros((self.q,) + self.shape)
        g = np.zeros((Q7,) + self.shape)
        lib().orc_get_populations(self._h, _p(f), _p(g))
        return f, g

    def step(self, n: int = 1):
        lib().orc_step(self._h, int(n))

    @property
    def steps(self) -> int:
        return int(lib().orc_steps_done(self._h))

    def gate_margin(self) -> np.ndarray:
        """Enthalpy model: per site, the smallest |f_l - 1/2| the flow gate met in the steps
        since the last reset (0.5 for a site that stayed in one phase, and everywhere without
        the model), shaped [z][y][x].  A site whose margin is below the resolution of a
        lower-precision implementation's f_l may legitimately be gated differently there."""
        out = np.zeros(self.shape)
        lib().orc_gate_margin(self._h, _p(out))
        return out

    def reset_gate_margin(self):
        lib().orc_gate_margin_reset(self._h)

    def macros(self):
        """(rho, u[3], T) at the current time, each shaped [z][y][x]."""
        rho = np.zeros(self.shape)
        u = np.zeros((3,) + self.shape)
        T = np.zeros(self.shape)
        lib().orc_macros(self._h, _p(rho), _p(u), _p(T))
        return rho, u, T


def enthalpy_state(lp: LatticeParams, En: float, phi: float = 1.0):
    """(T, f_l) from the effective enthalpy (Eqs. B8, B9)."""
    T, fl = C.c_double(), C.c_double()
    c = lp.to_c()
    lib().orc_enthalpy_state(C.byref(c), float(phi), float(En), C.byref(T), C.byref(fl))
    return T.value, fl.value


def enthalpy_of(lp: LatticeParams, T: float, phi: float = 1.0) -> float:
    c = lp.to_c()
    return lib().orc_enthalpy_of(C.byref(c), float(phi), float(T))


def geq7_enthalpy(lp: LatticeParams, En: float, T: float, u) -> np.ndarray:
    """Eq. B12."""
    out = np.zeros(Q7)
    c = lp.to_c()
    lib().orc_geq7_enthalpy(C.byref(c), float(En), float(T), _p(_vec(u)), _p(out))
    return out


def collide_site(lp: LatticeParams, f, g, phi=None, K=None, Fphi=None, zeta_alpha=None):
    """One-site collision (steps 2-11 of the module header).  Returns f*, g*, macros."""
    c = lp.to_c()
    phi = lp.phi if phi is None else phi
    K = lp.K if K is None else K
    if Fphi is None:
        Fphi = ergun_F(phi) if lp.F_phi < 0 else lp.F_phi
    za = lp.zeta_alpha if zeta_alpha is None else zeta_alpha
    fo = np.zeros(lp.q); go = np.zeros(Q7); mac = np.zeros(5)
    lib().orc_collide_site(C.byref(c), _p(_vec(f)), _p(_vec(g)), float(phi), float(K),
                           float(Fphi), float(za), _p(fo), _p(go), _p(mac))
    return fo, go, mac


# ---- diagnostics: plain definitions ---------------------------------------------------------

def nusselt(T: np.ndarray, face: int, T_wall: float, L: float, dT: float = 1.0,
            node_wall: bool = False):
    """Wall heat flux of Eq. 53 on a halfway wall, normalised as a Nusselt number.

    The wall sits half a spacing outside the first node; -d(theta)/dn at the wall is taken
    from the quadratic through (wall, node 0, node 1): (8 T_w - 9 T_0 + T_1) / 3.  Positive
    values are heat flowing from the wall into the fluid.  On a node wall (non-equilibrium
    extrapolation) the first node is the wall and the one-sided second-order gradient over
    (wall, node 1, node 2) gives (3 T_w - 4 T_1 + T_2) / 2.  Returns (Nu_3D, profile, Nu_mp):
    the profile runs along the first tangential axis (y for x-faces, x otherwise) averaged
    over the second one (Eq. 54, midpoint rule), Nu_3D is its mean (Eq. 55) and Nu_mp the
    profile at the centre (mean of the two middle entries for an even count).
    """
    T = np.asarray(T, dtype=np.float64)  # [z][y][x]
    axis = face // 2
    hi = face % 2 == 1
    arr = np.moveaxis(T, 2 - axis, 0)  # normal axis first
    if node_wall:
        t1 = arr[-2] if hi else arr[1]
        t2 = arr[-3] if hi else arr[2]
        q = (3.0 * T_wall - 4.0 * t1 + t2) / 2.0 * L / dT
    else:
        t0 = arr[-1] if hi else arr[0]
        t1 = arr[-2] if hi else arr[1]
        q = (8.0 * T_wall - 9.0 * t0 + t1) / 3.0 * L / dT
    # remaining axes of q, in [z][y][x] order minus the normal one
    if axis == 0:      # q[z][y]: profile over y, mean over z
        prof = q.mean(axis=0)
    elif axis == 1:    # q[z][x]: profile over x, mean over z
        prof = q.mean(axis=0)
    else:              # q[y][x]: profile over x, mean over y
        prof = q.mean(axis=0)
    n = prof.shape[0]
    mp = 0.5 * (prof[n // 2 - 1] + prof[n // 2]) if n % 2 == 0 else prof[n // 2]
    return float(prof.mean()), prof, float(mp)


def residual(new: np.ndarray, old: np.ndarray) -> float:
    """Relative change ||new - old||_2 / ||new||_2 (steady-state test); 0 for a field that
    is zero and unchanged."""
    new = np.asarray(new, dtype=np.float64)
    old = np.asarray(old, dtype=np.float64)
    den = math.sqrt(float(np.sum(new * new)))
    num = math.sqrt(float(np.sum((new - old) ** 2)))
    if den > 0:
        return num / den
    return math.inf if num > 0 else 0.0


def field_error(a: np.ndarray, ref: np.ndarray) -> float:
    """max|a - ref| / max|ref|, the field-normalised error used for parity."""
    ref = np.asarray(ref, dtype=np.float64)
    scale = float(np.max(np.abs(ref)))
    return float(np.max(np.abs(np.asarray(a, dtype=np.float64) - ref))) / (scale if scale > 0 else 1.0)
