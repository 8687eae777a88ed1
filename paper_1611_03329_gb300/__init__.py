"""GB300 (sm_103a) library for the 3D DDF-MRT lattice Boltzmann model of convection heat
transfer in porous media at the REV scale (Liu & He, arXiv:1611.03329).

This module is a thin ctypes binding of the C ABI in ``include/lbm.h``: it marshals
arguments and owns nothing but host buffers.  Every step of the computation runs in the
CUDA library ``_lib/liblbm_gb300.so``; when that library is missing the binding raises
instead of falling back to anything else.
"""
from __future__ import annotations

import ctypes as C
import math
import os
from typing import Optional

import numpy as np

from . import build as _build

Q19, Q7 = 19, 7

LBM_OK, LBM_EINVAL, LBM_ENOMEM, LBM_ECUDA, LBM_EUNSTABLE, LBM_ESTATE, LBM_ETIMEOUT = range(7)
FLOW_PERIODIC, FLOW_WALL, FLOW_VELOCITY, FLOW_OUTFLOW = range(4)
HEAT_PERIODIC, HEAT_ADIABATIC, HEAT_DIRICHLET, HEAT_OUTFLOW = range(4)
MAP_CAVITY, MAP_CHANNEL, MAP_LATTICE = range(3)
_MAPPINGS = {"cavity": MAP_CAVITY, "channel": MAP_CHANNEL, "lattice": MAP_LATTICE}
STORE_FP32, STORE_FP16_DEV, STORE_BF16_DEV = range(3)
_STORAGE = {"fp32": STORE_FP32, "fp16": STORE_FP16_DEV, "bf16": STORE_BF16_DEV}
STORAGE_BYTES = {"fp32": 4, "fp16": 2, "bf16": 2}

# Every symbol that include/lbm.h declares.
ABI_SYMBOLS = (
    "lbm_params_default", "lbm_derive_lattice", "lbm_create", "lbm_destroy", "lbm_set_medium",
    "lbm_step", "lbm_init_equilibrium", "lbm_set_populations", "lbm_get_populations",
    "lbm_macros", "lbm_macros_device", "lbm_nusselt", "lbm_sums", "lbm_residual",
    "lbm_get_lattice", "lbm_steps_done", "lbm_sync", "lbm_last_error", "lbm_status_string",
    "lbm_residual_noalloc", "lbm_batch_create", "lbm_batch_step", "lbm_batch_tune",
    "lbm_batch_set_block", "lbm_batch_last_error", "lbm_batch_destroy", "lbm_footprint",
    "lbm_server_create", "lbm_server_submit", "lbm_server_advance", "lbm_server_poll",
    "lbm_server_clock", "lbm_server_destroy", "lbm_server_set_fill", "lbm_set_step_kernel",
    "lbm_get_step_kernel", "lbm_state_bytes", "lbm_save_state", "lbm_load_state",
    "lbm_set_launch", "lbm_test_tma_extra_wait", "lbm_server_set_output",
    "lbm_server_set_policy", "lbm_batch_set_scheme", "lbm_batch_scheme_times",
    "lbm_batch_set_launch_mode", "lbm_batch_launch_groups",
    "lbm_bounds_report",
)

ADMIT_POLICIES = {"fifo": 0, "backfill": 1}
RESIDUAL_FLOOR = {"fp16": 2e-4, "bf16": 2e-3}  # LBM_RESIDUAL_FLOOR_FP16 / _BF16

# Population schemes (LBM_SCHEME_*).
SCHEMES = {"pingpong": 0, "aa": 1, "auto": 2}
BATCH_LAUNCH = {"fused": 0, "per_lattice": 1}  # LBM_BATCH_FUSED / _PER_LATTICE

# Step kernels (LBM_KERNEL_*).
STEP_KERNELS = {"plain": 0, "tma": 1, "paired": 2}

REQ_CONVERGED, REQ_MAX_STEPS, REQ_UNSTABLE, REQ_FAILED = range(4)
REQ_STATUS = {0: "converged", 1: "max_steps", 2: "unstable", 3: "failed"}

NOALLOC_MAX_SITES = 33554432  # LBM_NOALLOC_MAX_SITES


class LbmParams(C.Structure):
    """Mirror of ``lbm_params`` (include/lbm.h)."""
    _fields_ = [
        ("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int),
        ("storage", C.c_int), ("mapping", C.c_int),
        ("L", C.c_double),
        ("Ra", C.c_double), ("Da", C.c_double), ("Pr", C.c_double), ("J", C.c_double),
        ("sigma", C.c_double), ("Gamma", C.c_double), ("Ma", C.c_double),
        ("Re", C.c_double), ("Ri", C.c_double), ("u0", C.c_double),
        ("dT", C.c_double),
        ("T0", C.c_double), ("rho0", C.c_double), ("varpi", C.c_double),
        ("s_e", C.c_double), ("s_eps", C.c_double), ("s_q", C.c_double), ("s_pi", C.c_double),
        ("s_m", C.c_double), ("zeta_T", C.c_double), ("zeta_e", C.c_double),
        ("zeta_nu", C.c_double),
        ("nu_e", C.c_double), ("alpha_f", C.c_double), ("gbeta", C.c_double),
        ("gravity_axis", C.c_int), ("gravity_sign", C.c_int),
        ("accel", C.c_double * 3),
        ("flow_bc", C.c_int * 6), ("heat_bc", C.c_int * 6),
        ("face_T", C.c_double * 6), ("face_u", (C.c_double * 3) * 6),
        ("T_init", C.c_double), ("U_out", C.c_double),
        ("enthalpy", C.c_int), ("flow_off", C.c_int),
        ("T_m", C.c_double), ("T_s", C.c_double), ("T_l", C.c_double), ("St", C.c_double),
        ("c_pl", C.c_double), ("c_ps", C.c_double), ("sigma_s", C.c_double),
        ("sigma_l", C.c_double), ("alpha_ratio", C.c_double),
        ("q_flow", C.c_int), ("scheme", C.c_int),
        ("auto_mem_limit", C.c_ulonglong),
    ]


class LbmLattice(C.Structure):
    """Mirror of ``lbm_lattice`` (include/lbm.h)."""
    _fields_ = [
        ("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int),
        ("L", C.c_double), ("rho0", C.c_double), ("T0", C.c_double), ("sigma", C.c_double),
        ("varpi", C.c_double), ("dT", C.c_double),
        ("s", C.c_double * 19),
        ("zeta_T", C.c_double), ("zeta_e", C.c_double), ("zeta_nu", C.c_double),
        ("zeta_alpha", C.c_double),
        ("s_nu", C.c_double), ("nu_e", C.c_double), ("nu", C.c_double), ("alpha_f", C.c_double),
        ("alpha_m", C.c_double), ("Gamma", C.c_double),
        ("gbeta", C.c_double), ("buoy", C.c_double * 3), ("accel", C.c_double * 3),
        ("phi", C.c_double), ("K", C.c_double), ("F_phi", C.c_double), ("phi_ref", C.c_double),
        ("has_phi_field", C.c_int),
        ("U_out", C.c_double),
        ("enthalpy", C.c_int), ("flow_off", C.c_int),
        ("c_pl", C.c_double), ("c_ref", C.c_double), ("sigma_s", C.c_double),
        ("sigma_l", C.c_double), ("T_s", C.c_double), ("T_l", C.c_double), ("L_a", C.c_double),
        ("alpha_s", C.c_double), ("alpha_l", C.c_double),
        ("node_walls", C.c_int), ("q", C.c_int), ("scheme", C.c_int),
    ]

    def as_dict(self) -> dict:
        out = {}
        for name, _ in self._fields_:
            v = getattr(self, name)
            out[name] = list(v) if hasattr(v, "__len__") else v
        return out


class LbmMedium(C.Structure):
    """Mirror of ``lbm_medium`` (include/lbm.h)."""
    _fields_ = [("phi_field", C.POINTER(C.c_float)), ("phi", C.c_double), ("K", C.c_double),
                ("F_phi", C.c_double), ("alpha_m", C.c_double), ("phi_ref", C.c_double)]


class LbmResult(C.Structure):
    """Mirror of ``lbm_result`` (include/lbm.h)."""
    _fields_ = [("id", C.c_longlong), ("status", C.c_int), ("steps", C.c_longlong),
                ("r_u", C.c_double), ("r_T", C.c_double), ("nu_avg", C.c_double),
                ("nu_mp", C.c_double), ("mass_dev", C.c_double), ("heat_dev", C.c_double),
                ("t_submit", C.c_double), ("t_admit", C.c_double), ("t_done", C.c_double),
                ("bytes", C.c_ulonglong), ("sites", C.c_longlong), ("storage", C.c_int)]

    def as_dict(self) -> dict:
        d = {name: getattr(self, name) for name, _ in self._fields_}
        d["status"] = REQ_STATUS.get(self.status, str(self.status))
        d["storage"] = {v: k for k, v in _STORAGE.items()}.get(self.storage, str(self.storage))
        return d


class LbmError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(msg)
        self.status = status


_lib = None


def library_path() -> str:
    """The shared library the binding loads: ``LBM_LIBRARY`` if set, else the in-tree build."""
    return os.environ.get("LBM_LIBRARY") or _build.LIB


def lib():
    """Load the CUDA library; raises if it has not been built."""
    global _lib
    if _lib is None:
        path = library_path()
        if not os.path.exists(path):
            raise RuntimeError(f"CUDA library not built ({path}); run "
                               "`python -c 'import __graft_entry__ as g; g.build()'`")
        L = C.CDLL(path)
        vp, dp, fp = C.c_void_p, C.POINTER(C.c_double), C.POINTER(C.c_float)
        pp = C.POINTER(LbmParams)
        L.lbm_params_default.argtypes = [pp]
        L.lbm_derive_lattice.argtypes = [pp, C.POINTER(LbmLattice)]
        L.lbm_create.argtypes = [pp, vp, C.POINTER(vp)]
        L.lbm_destroy.argtypes = [vp]
        L.lbm_destroy.restype = None
        L.lbm_set_medium.argtypes = [vp, fp, C.c_double, C.c_double, C.c_double, C.c_double,
                                     C.c_double]
        L.lbm_step.argtypes = [vp, C.c_int]
        L.lbm_set_step_kernel.argtypes = [vp, C.c_int]
        L.lbm_state_bytes.argtypes = [vp, C.POINTER(C.c_ulonglong)]
        L.lbm_save_state.argtypes = [vp, vp, C.c_ulonglong]
        L.lbm_load_state.argtypes = [vp, vp, C.c_ulonglong]
        L.lbm_get_step_kernel.argtypes = [vp]
        L.lbm_set_launch.argtypes = [vp, C.c_int, C.c_int]
        L.lbm_test_tma_extra_wait.argtypes = [vp, C.c_int]
        L.lbm_init_equilibrium.argtypes = [vp, dp, dp, C.c_double]
        L.lbm_set_populations.argtypes = [vp, dp, dp]
        L.lbm_get_populations.argtypes = [vp, dp, dp]
        L.lbm_macros.argtypes = [vp, fp, fp, fp]
        L.lbm_macros_device.argtypes = [vp, vp, vp, vp]
        L.lbm_nusselt.argtypes = [vp, C.c_int, dp, dp, dp]
        L.lbm_sums.argtypes = [vp, dp, dp]
        L.lbm_residual.argtypes = [vp, dp, dp]
        L.lbm_get_lattice.argtypes = [vp, C.POINTER(LbmLattice)]
        L.lbm_steps_done.argtypes = [vp]
        L.lbm_steps_done.restype = C.c_longlong
        L.lbm_sync.argtypes = [vp]
        L.lbm_last_error.argtypes = [vp]
        L.lbm_last_error.restype = C.c_char_p
        L.lbm_status_string.argtypes = [C.c_int]
        L.lbm_status_string.restype = C.c_char_p
        L.lbm_residual_noalloc.argtypes = [vp, vp, vp, vp, C.c_longlong, vp, vp]
        L.lbm_batch_create.argtypes = [C.POINTER(vp), C.c_int, vp, C.POINTER(vp)]
        L.lbm_batch_step.argtypes = [vp, C.c_int]
        L.lbm_batch_tune.argtypes = [vp, C.POINTER(C.c_int), C.POINTER(C.c_int)]
        L.lbm_batch_set_block.argtypes = [vp, C.c_int, C.c_int]
        L.lbm_batch_set_scheme.argtypes = [vp, C.c_int]
        L.lbm_batch_scheme_times.argtypes = [vp, dp, dp]
        L.lbm_batch_set_launch_mode.argtypes = [vp, C.c_int]
        L.lbm_batch_launch_groups.argtypes = [vp, C.POINTER(C.c_int), C.POINTER(C.c_int)]
        L.lbm_batch_last_error.argtypes = [vp]
        L.lbm_batch_last_error.restype = C.c_char_p
        L.lbm_batch_destroy.argtypes = [vp]
        L.lbm_batch_destroy.restype = None
        L.lbm_footprint.argtypes = [pp, C.c_int, C.POINTER(C.c_ulonglong)]
        L.lbm_server_create.argtypes = [C.c_ulonglong, C.c_int, vp, C.POINTER(vp)]
        L.lbm_server_submit.argtypes = [vp, pp, C.POINTER(LbmMedium), C.c_double, C.c_longlong,
                                        C.POINTER(C.c_longlong)]
        L.lbm_server_advance.argtypes = [vp, C.POINTER(C.c_int), C.POINTER(C.c_int)]
        L.lbm_server_poll.argtypes = [vp, C.POINTER(LbmResult), C.c_int, C.POINTER(C.c_int)]
        L.lbm_server_set_output.argtypes = [vp, C.c_longlong, fp, fp]
        L.lbm_server_set_policy.argtypes = [vp, C.c_int]
        L.lbm_bounds_report.argtypes = [C.POINTER(C.c_longlong)]
        L.lbm_server_set_fill.argtypes = [vp, C.c_longlong]
        L.lbm_server_clock.argtypes = [vp]
        L.lbm_server_clock.restype = C.c_double
        L.lbm_server_destroy.argtypes = [vp]
        L.lbm_server_destroy.restype = None
        _lib = L
    return _lib


def _dp(a: np.ndarray):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _fp(a: np.ndarray):
    return a.ctypes.data_as(C.POINTER(C.c_float))


def params_from_problem(pb: dict) -> LbmParams:
    """Marshal a problem dictionary (the keys of ``lbm_params``) into the C struct."""
    p = LbmParams()
    lib().lbm_params_default(C.byref(p))
    p.nx, p.ny, p.nz = int(pb["nx"]), int(pb["ny"]), int(pb["nz"])
    p.mapping = _MAPPINGS[pb.get("mapping", "cavity")]
    p.storage = _STORAGE[pb.get("storage", "fp32")]
    scalars = ("L", "Ra", "Pr", "J", "sigma", "Gamma", "Ma", "Re", "Ri", "u0", "dT", "T0",
               "rho0", "varpi", "s_e", "s_eps", "s_q", "s_pi", "s_m", "zeta_T", "zeta_e",
               "zeta_nu", "nu_e", "alpha_f", "gbeta", "T_init", "U_out")
    for k in scalars:
        if k in pb and pb[k] is not None:
            setattr(p, k, float(pb[k]))
    if pb.get("Da") is not None:
        p.Da = float(pb["Da"])
    if "T_init" not in pb:
        p.T_init = p.T0
    p.q_flow = int(pb.get("q", 19))
    p.scheme = SCHEMES[pb.get("scheme", "pingpong")]
    p.auto_mem_limit = int(pb.get("auto_mem_limit", 0))
    p.enthalpy = int(bool(pb.get("enthalpy", False)))
    p.flow_off = int(bool(pb.get("flow_off", False)))
    for k in ("T_m", "T_s", "T_l", "St", "c_pl", "c_ps", "sigma_s", "sigma_l", "alpha_ratio"):
        if k in pb and pb[k] is not None:
            setattr(p, k, float(pb[k]))
    p.gravity_axis = int(pb.get("gravity_axis", 2))
    p.gravity_sign = int(pb.get("gravity_sign", -1))
    for a, v in enumerate(pb.get("accel", (0.0, 0.0, 0.0))):
        p.accel[a] = float(v)
    for f in range(6):
        p.flow_bc[f] = int(pb.get("flow_bc", [0] * 6)[f])
        p.heat_bc[f] = int(pb.get("heat_bc", [0] * 6)[f])
        p.face_T[f] = float(pb.get("face_T", [0.0] * 6)[f])
        fu = pb.get("face_u", [(0.0, 0.0, 0.0)] * 6)[f]
        for a in range(3):
            p.face_u[f][a] = float(fu[a])
    return p


def derive_lattice(pb: dict) -> dict:
    """Lattice parameters of a problem (host only, no GPU needed)."""
    out = LbmLattice()
    st = lib().lbm_derive_lattice(C.byref(params_from_problem(pb)), C.byref(out))
    if st != LBM_OK:
        raise LbmError(st, "lbm_derive_lattice: invalid problem")
    return out.as_dict()


class Lattice:
    """One lattice on the current CUDA device, driven through the C ABI.

    ``pb`` is a problem dictionary; its medium keys (phi, K, F_phi, alpha_m, phi_field,
    phi_ref) go to ``lbm_set_medium``.  ``stream`` is a cudaStream_t handle (int) or None.
    """

    def __init__(self, pb: dict, stream: Optional[int] = None):
        self.pb = dict(pb)
        self.nx, self.ny, self.nz = int(pb["nx"]), int(pb["ny"]), int(pb["nz"])
        self.shape = (self.nz, self.ny, self.nx)
        self.ns = self.nx * self.ny * self.nz
        self.q = 15 if int(pb.get("q", 19)) == 15 else 19  # flow lattice
        self._h = C.c_void_p()
        self._params = params_from_problem(pb)
        st = lib().lbm_create(C.byref(self._params), C.c_void_p(stream or 0), C.byref(self._h))
        if st != LBM_OK:
            raise LbmError(st, f"lbm_create failed: {lib().lbm_status_string(st).decode()}")
        self.set_medium(pb.get("phi_field"), pb.get("phi", 1.0), pb.get("K", 0.0),
                        pb.get("F_phi", 0.0), pb.get("alpha_m", -1.0), pb.get("phi_ref", 0.0))

    # -- plumbing
    def _check(self, st: int, what: str):
        if st != LBM_OK:
            msg = lib().lbm_last_error(self._h).decode()
            raise LbmError(st, f"{what}: {lib().lbm_status_string(st).decode()}: {msg}")

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            lib().lbm_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def handle(self) -> int:
        return self._h.value

    # -- calls
    def set_medium(self, phi_field=None, phi=1.0, K=0.0, F_phi=0.0, alpha_m=-1.0, phi_ref=0.0):
        fptr = None
        if phi_field is not None:
            self._phi = np.ascontiguousarray(np.asarray(phi_field, dtype=np.float32).reshape(-1))
            assert self._phi.size == self.ns
            fptr = _fp(self._phi)
        K = float(K) if K is not None else 0.0
        self._check(lib().lbm_set_medium(self._h, fptr, float(phi), K, float(F_phi),
                                         float(alpha_m), float(phi_ref)), "lbm_set_medium")

    def step(self, n: int = 1):
        self._check(lib().lbm_step(self._h, int(n)), "lbm_step")

    def sync(self):
        self._check(lib().lbm_sync(self._h), "lbm_sync")

    def state_bytes(self) -> int:
        n = C.c_ulonglong()
        self._check(lib().lbm_state_bytes(self._h, C.byref(n)), "lbm_state_bytes")
        return int(n.value)

    def save_state(self, out: Optional[np.ndarray] = None, sync: bool = True) -> np.ndarray:
        """The raw state blob (lbm_save_state) into `out` (a C-contiguous uint8 array of at
        least state_bytes(), ideally pinned) or a new array."""
        n = self.state_bytes()
        if out is None:
            out = np.empty(n, dtype=np.uint8)
        assert out.dtype == np.uint8 and out.flags.c_contiguous and out.size >= n
        self._check(lib().lbm_save_state(self._h, out.ctypes.data_as(C.c_void_p), out.size),
                    "lbm_save_state")
        if sync:
            self.sync()
        return out

    def load_state(self, blob: np.ndarray, sync: bool = True):
        """Restore a blob of save_state (lbm_load_state); asynchronous unless `sync`."""
        assert blob.dtype == np.uint8 and blob.flags.c_contiguous
        self._check(lib().lbm_load_state(self._h, blob.ctypes.data_as(C.c_void_p), blob.size),
                    "lbm_load_state")
        if sync:
            self.sync()

    def set_step_kernel(self, kernel: str):
        """Select the step kernel: "plain" (one thread per site) or "tma" (populations staged
        into shared memory by the Tensor Memory Accelerator); both give the same populations."""
        self._check(lib().lbm_set_step_kernel(self._h, STEP_KERNELS[kernel]), "lbm_set_step_kernel")

    def set_launch(self, block_threads: int = 0, dependent_launch: int = -1):
        """lbm_set_launch: block size (0 keeps) and programmatic dependent launch (-1 keeps)."""
        self._check(lib().lbm_set_launch(self._h, int(block_threads), int(dependent_launch)),
                    "lbm_set_launch")

    def test_tma_extra_wait(self, nbytes: int):
        """lbm_test_tma_extra_wait (test only): TMA stages wait for nbytes more than arrive."""
        self._check(lib().lbm_test_tma_extra_wait(self._h, int(nbytes)), "lbm_test_tma_extra_wait")

    @property
    def step_kernel(self) -> str:
        k = int(lib().lbm_get_step_kernel(self._h))
        return {v: n for n, v in STEP_KERNELS.items()}[k]

    @property
    def steps(self) -> int:
        return int(lib().lbm_steps_done(self._h))

    def init_equilibrium(self, T=0.5, T_field=None, u_field=None):
        tp = up = None
        if T_field is not None:
            self._tf = np.ascontiguousarray(T_field, dtype=np.float64).reshape(-1)
            tp = _dp(self._tf)
        if u_field is not None:
            self._uf = np.ascontiguousarray(u_field, dtype=np.float64).reshape(-1)
            up = _dp(self._uf)
        self._check(lib().lbm_init_equilibrium(self._h, tp, up, float(T)), "lbm_init_equilibrium")

    def set_populations(self, f: np.ndarray, g: np.ndarray):
        f = np.ascontiguousarray(f, dtype=np.float64)
        g = np.ascontiguousarray(g, dtype=np.float64)
        assert f.size == self.q * self.ns and g.size == Q7 * self.ns
        self._check(lib().lbm_set_populations(self._h, _dp(f), _dp(g)), "lbm_set_populations")

    def populations(self):
        f = np.zeros((self.q,) + self.shape)
        g = np.zeros((Q7,) + self.shape)
        self._check(lib().lbm_get_populations(self._h, _dp(f), _dp(g)), "lbm_get_populations")
        return f, g

    def macros(self):
        """(rho, u[3], T) as float32 arrays shaped [z][y][x]."""
        rho = np.zeros(self.shape, np.float32)
        u = np.zeros((3,) + self.shape, np.float32)
        T = np.zeros(self.shape, np.float32)
        self._check(lib().lbm_macros(self._h, _fp(rho), _fp(u), _fp(T)), "lbm_macros")
        return rho, u, T

    def macros_into(self, rho, u, T):
        """Host-buffer variant writing into caller-owned float32 arrays (any may be None)."""
        args = [None if a is None else _fp(a) for a in (rho, u, T)]
        self._check(lib().lbm_macros(self._h, *args), "lbm_macros")

    def macros_device(self, rho_ptr: int, u_ptr: int, T_ptr: int):
        """Device-pointer variant (e.g. torch tensors' data_ptr()); asynchronous."""
        self._check(lib().lbm_macros_device(self._h, C.c_void_p(rho_ptr or 0),
                                            C.c_void_p(u_ptr or 0), C.c_void_p(T_ptr or 0)),
                    "lbm_macros_device")

    def nusselt(self, face: int):
        """(Nu_3D, profile, Nu_mp) on a Dirichlet face (Eqs. 53-55)."""
        axis = face // 2
        n1 = self.ny if axis == 0 else self.nx
        prof = np.zeros(n1)
        avg, mp = C.c_double(), C.c_double()
        self._check(lib().lbm_nusselt(self._h, int(face), C.byref(avg), _dp(prof), C.byref(mp)),
                    "lbm_nusselt")
        return avg.value, prof, mp.value

    def sums(self):
        m, h = C.c_double(), C.c_double()
        self._check(lib().lbm_sums(self._h, C.byref(m), C.byref(h)), "lbm_sums")
        return m.value, h.value

    def residual(self):
        ru, rT = C.c_double(), C.c_double()
        self._check(lib().lbm_residual(self._h, C.byref(ru), C.byref(rT)), "lbm_residual")
        return ru.value, rT.value

    def lattice(self) -> dict:
        out = LbmLattice()
        self._check(lib().lbm_get_lattice(self._h, C.byref(out)), "lbm_get_lattice")
        return out.as_dict()


def residual_noalloc(u_ptr: int, T_ptr: int, u_prev_ptr: int, T_prev_ptr: int, ns: int,
                     out_ptr: int, stream: Optional[int] = None) -> None:
    """Allocation-free residual of caller-held device fields (``lbm_residual_noalloc``):
    writes r_u, r_T and the non-finite count to the 3 device doubles at ``out_ptr``,
    asynchronously on ``stream``.  For callers that cannot allocate device memory."""
    st = lib().lbm_residual_noalloc(C.c_void_p(u_ptr), C.c_void_p(T_ptr), C.c_void_p(u_prev_ptr),
                                    C.c_void_p(T_prev_ptr), C.c_longlong(ns),
                                    C.c_void_p(out_ptr), C.c_void_p(stream or 0))
    if st != LBM_OK:
        raise LbmError(st, f"lbm_residual_noalloc: {lib().lbm_status_string(st).decode()}")


class Batch:
    """Many lattices advanced by one fused launch per time step (``lbm_batch_*``)."""

    def __init__(self, lattices, stream: Optional[int] = None):
        self.lattices = list(lattices)
        arr = (C.c_void_p * len(self.lattices))(*[l.handle for l in self.lattices])
        self._h = C.c_void_p()
        st = lib().lbm_batch_create(arr, len(self.lattices), C.c_void_p(stream or 0),
                                    C.byref(self._h))
        if st != LBM_OK:
            raise LbmError(st, f"lbm_batch_create: {lib().lbm_status_string(st).decode()}")

    def _check(self, st: int, what: str):
        if st != LBM_OK:
            raise LbmError(st, f"{what}: {lib().lbm_status_string(st).decode()}: "
                               f"{lib().lbm_batch_last_error(self._h).decode()}")

    def step(self, n: int = 1):
        self._check(lib().lbm_batch_step(self._h, int(n)), "lbm_batch_step")

    def tune(self):
        """Autotune the block shape; returns (threads per block, z-planes per block)."""
        bt, rows = C.c_int(), C.c_int()
        self._check(lib().lbm_batch_tune(self._h, C.byref(bt), C.byref(rows)), "lbm_batch_tune")
        return bt.value, rows.value

    def set_block(self, threads: int, rows: int = 1):
        self._check(lib().lbm_batch_set_block(self._h, int(threads), int(rows)),
                    "lbm_batch_set_block")

    def set_scheme(self, scheme: str):
        """lbm_batch_set_scheme: move the members that can run AA to it ("aa")."""
        self._check(lib().lbm_batch_set_scheme(self._h, SCHEMES[scheme]), "lbm_batch_set_scheme")

    def scheme_times(self):
        """(ping-pong ms, AA ms) per step of the tuner's last scheme trial."""
        pp, aa = C.c_double(), C.c_double()
        self._check(lib().lbm_batch_scheme_times(self._h, C.byref(pp), C.byref(aa)),
                    "lbm_batch_scheme_times")
        return pp.value, aa.value

    def set_launch_mode(self, mode: str):
        """lbm_batch_set_launch_mode: "fused" (one launch per step for a group) or
        "per_lattice" (each lattice's own step kernel)."""
        self._check(lib().lbm_batch_set_launch_mode(self._h, BATCH_LAUNCH[mode]),
                    "lbm_batch_set_launch_mode")

    def launch_groups(self):
        """(fused groups, per-lattice groups): lbm_batch_launch_groups."""
        nf, ns = C.c_int(), C.c_int()
        self._check(lib().lbm_batch_launch_groups(self._h, C.byref(nf), C.byref(ns)),
                    "lbm_batch_launch_groups")
        return nf.value, ns.value

    def sync(self):
        for l in self.lattices:
            l.sync()

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            lib().lbm_batch_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def footprint(pb: dict) -> int:
    """Device bytes a lattice for problem pb holds while it is solved (host only)."""
    out = C.c_ulonglong()
    st = lib().lbm_footprint(C.byref(params_from_problem(pb)),
                             int(pb.get("phi_field") is not None), C.byref(out))
    if st != LBM_OK:
        raise LbmError(st, "lbm_footprint: invalid problem")
    return out.value


class Server:
    """Continuous-batching serving loop (``lbm_server_*``): submit problems as they arrive,
    call advance() repeatedly, poll() finished results."""

    def __init__(self, budget_bytes: int = 0, chunk: int = 100, stream: Optional[int] = None,
                 max_active_sites: int = 0, policy: str = "fifo"):
        self._h = C.c_void_p()
        st = lib().lbm_server_create(C.c_ulonglong(budget_bytes), int(chunk),
                                     C.c_void_p(stream or 0), C.byref(self._h))
        if st != LBM_OK:
            raise LbmError(st, f"lbm_server_create: {lib().lbm_status_string(st).decode()}")
        if max_active_sites:
            st = lib().lbm_server_set_fill(self._h, C.c_longlong(max_active_sites))
            if st != LBM_OK:
                raise LbmError(st, "lbm_server_set_fill")
        st = lib().lbm_server_set_policy(self._h, ADMIT_POLICIES[policy])
        if st != LBM_OK:
            raise LbmError(st, "lbm_server_set_policy")

    def submit(self, pb: dict, tol: float = 1e-6, max_steps: int = 50000) -> int:
        m = LbmMedium()
        m.phi = float(pb.get("phi", 1.0))
        m.K = float(pb.get("K", 0.0) or 0.0)
        m.F_phi = float(pb.get("F_phi", 0.0))
        m.alpha_m = float(pb.get("alpha_m", -1.0))
        m.phi_ref = float(pb.get("phi_ref", 0.0))
        keep = None
        if pb.get("phi_field") is not None:
            keep = np.ascontiguousarray(np.asarray(pb["phi_field"], dtype=np.float32).reshape(-1))
            m.phi_field = keep.ctypes.data_as(C.POINTER(C.c_float))
        rid = C.c_longlong()
        st = lib().lbm_server_submit(self._h, C.byref(params_from_problem(pb)), C.byref(m),
                                     float(tol), int(max_steps), C.byref(rid))
        del keep
        if st != LBM_OK:
            raise LbmError(st, f"lbm_server_submit: {lib().lbm_status_string(st).decode()}")
        return rid.value

    def set_output(self, rid: int, u: Optional[np.ndarray], T: Optional[np.ndarray]):
        """lbm_server_set_output: float32 host arrays (u: 3 x ns, T: ns) that receive the
        request's final fields; the caller keeps them alive until the result is polled."""
        for a in (u, T):
            assert a is None or (a.dtype == np.float32 and a.flags["C_CONTIGUOUS"])
        st = lib().lbm_server_set_output(self._h, int(rid), None if u is None else _fp(u),
                                         None if T is None else _fp(T))
        if st != LBM_OK:
            raise LbmError(st, "lbm_server_set_output")

    def advance(self):
        """One scheduling round; returns (admitted, queued)."""
        na, nq = C.c_int(), C.c_int()
        st = lib().lbm_server_advance(self._h, C.byref(na), C.byref(nq))
        if st != LBM_OK:
            raise LbmError(st, f"lbm_server_advance: {lib().lbm_status_string(st).decode()}")
        return na.value, nq.value

    def poll(self, max_results: int = 1024) -> list:
        buf = (LbmResult * max_results)()
        n = C.c_int()
        st = lib().lbm_server_poll(self._h, buf, max_results, C.byref(n))
        if st != LBM_OK:
            raise LbmError(st, "lbm_server_poll")
        return [buf[k].as_dict() for k in range(n.value)]

    def clock(self) -> float:
        return lib().lbm_server_clock(self._h)

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            lib().lbm_server_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def medium_args(pb: dict) -> dict:
    """The medium part of a problem dictionary with defaults made explicit."""
    return dict(phi=pb.get("phi", 1.0), K=pb.get("K", 0.0), F_phi=pb.get("F_phi", 0.0),
                alpha_m=pb.get("alpha_m", -1.0), phi_ref=pb.get("phi_ref", 0.0),
                has_field=pb.get("phi_field") is not None)


def algorithmic_bytes_per_site(pb: dict) -> int:
    """Bytes one time step must move per site: the Q + 7 populations (26 for D3Q19, 22 for
    D3Q15) read and written in the storage format (4 or 2 bytes each), the FP32 temperature
    plane of the 16-bit formats (read and written: the thermal populations are stored against
    it), plus the FP32 porosity of a heterogeneous medium."""
    npop = (15 if int(pb.get("q", 19)) == 15 else 19) + 7
    storage = pb.get("storage", "fp32")
    return (npop * 2 * STORAGE_BYTES[storage] + (8 if storage != "fp32" else 0)
            + (4 if pb.get("phi_field") is not None else 0))


def nan_safe(x: float) -> float:
    return x if math.isfinite(x) else float("nan")


def bounds_report():
    """lbm_bounds_report: the first out-of-range site index the bounds-checked library met
    (-1: none); raises LbmError(LBM_EINVAL) on the ordinary build."""
    v = C.c_longlong(-1)
    st = lib().lbm_bounds_report(C.byref(v))
    if st != LBM_OK:
        raise LbmError(st, "lbm_bounds_report: not a bounds-checked build")
    return v.value
