"""Thin ctypes binding of ``libtled`` (include/tled.h).

Argument marshalling only: every step of the method runs in the library's
CUDA kernels.  PyTorch supplies the device workspace (a ``torch.uint8``
tensor) and the CUDA stream.  There is no CPU fallback: if the library or a
CUDA device is missing, construction raises.
"""
from __future__ import annotations

import ctypes as C
import os
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libtled.so")

OK, E_ARG, E_MESH, E_STATE, E_CUDA, E_UNSTABLE, E_INVERTED, E_TIMEOUT, E_NOMEM, E_FORMAT = 0, -1, -2, -3, -4, -5, -6, -7, -8, -9
T4, H8 = 4, 8
HOST, DEVICE = 0, 1
EXPANSION, TEMP_DEP, COMPENSATED, CEM43, GENERAL_H8, STREAMED = 1, 2, 4, 8, 16, 32


def default_flags(prob):
    """Step flags a workloads.Problem asks for: compensated accumulation, and
    thermal expansion, temperature-dependent c and k, CEM43 as it sets them."""
    return (COMPENSATED | (EXPANSION if prob.expansion else 0) | (TEMP_DEP if prob.temp_dep else 0) |
            (CEM43 if getattr(prob, "cem43", False) else 0))
SRC_GAUSSIAN, SRC_SPHERE = 0, 1
FIX_X, FIX_Y, FIX_Z, FIX_T = 1, 2, 4, 8

_dp = C.POINTER(C.c_double)


class Material(C.Structure):
    _fields_ = [("rho", C.c_double), ("mu", C.c_double), ("kappa", C.c_double), ("k1", C.c_double),
                ("k2", C.c_double), ("a0", C.c_double * 3), ("n_prony", C.c_int32), ("pad", C.c_int32),
                ("prony_g", C.c_double * 4), ("prony_tau", C.c_double * 4), ("alpha", C.c_double),
                ("k", C.c_double), ("c", C.c_double), ("beta_k", C.c_double), ("beta_c", C.c_double),
                ("T_ref", C.c_double), ("wb_cb", C.c_double), ("Qm", C.c_double), ("T0", C.c_double),
                ("Ta", C.c_double), ("lnA", C.c_double), ("Ea", C.c_double), ("alpha_fibre_ratio", C.c_double),
                ("k_fibre_ratio", C.c_double)]


class Source(C.Structure):
    _fields_ = [("c0", C.c_double * 3), ("vel", C.c_double * 3), ("sigma", C.c_double), ("power", C.c_double),
                ("t_on", C.c_double), ("t_off", C.c_double), ("shape", C.c_int32), ("pad", C.c_int32)]


class Params(C.Structure):
    _fields_ = [("dt", C.c_double), ("dt_safety", C.c_double), ("gamma", C.c_double), ("mass_scale", C.c_double),
                ("kappa_hg", C.c_double), ("kappa_hgT", C.c_double), ("flags", C.c_uint32),
                ("tile_elems", C.c_int32), ("n_sub", C.c_int32), ("pad", C.c_int32)]


class Stats(C.Structure):
    _fields_ = [("step", C.c_int64), ("t", C.c_double), ("dt", C.c_double), ("T_max", C.c_double),
                ("T_min", C.c_double), ("u_max", C.c_double), ("damage_volume", C.c_double),
                ("heat_content", C.c_double), ("kinetic_energy", C.c_double), ("strain_energy", C.c_double),
                ("hourglass_energy", C.c_double), ("status", C.c_uint32),
                ("pad", C.c_int32)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_ if k != "pad"}


class TledError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"libtled error {code}: {msg}")
        self.code = code


_lib = None

_SIGS = {
    "tled_version": ([], C.c_int),
    "tled_status_string": ([C.c_int], C.c_char_p),
    "tled_create": ([C.POINTER(C.c_void_p), C.c_int, C.c_void_p], C.c_int),
    "tled_destroy": ([C.c_void_p], C.c_int),
    "tled_last_error": ([C.c_void_p], C.c_char_p),
    "tled_set_mesh": ([C.c_void_p, C.c_int, C.c_int64, _dp, C.c_int64, C.POINTER(C.c_int32)], C.c_int),
    "tled_set_material": ([C.c_void_p, C.POINTER(Material), _dp, _dp], C.c_int),
    "tled_set_bcs": ([C.c_void_p, C.POINTER(C.c_uint8), _dp, C.c_double], C.c_int),
    "tled_set_heat_sources": ([C.c_void_p, C.c_int32, C.POINTER(Source)], C.c_int),
    "tled_set_params": ([C.c_void_p, C.POINTER(Params)], C.c_int),
    "tled_workspace_size": ([C.c_void_p, C.POINTER(C.c_int64)], C.c_int),
    "tled_init": ([C.c_void_p, C.c_void_p, C.c_int64], C.c_int),
    "tled_get_dt": ([C.c_void_p, _dp, _dp, _dp], C.c_int),
    "tled_step": ([C.c_void_p, C.c_int64], C.c_int),
    "tled_sync": ([C.c_void_p], C.c_int),
    "tled_get_displacement": ([C.c_void_p, C.c_void_p, C.c_int], C.c_int),
    "tled_get_temperature": ([C.c_void_p, C.c_void_p, C.c_int], C.c_int),
    "tled_get_damage": ([C.c_void_p, C.c_void_p, C.c_int], C.c_int),
    "tled_get_cem43": ([C.c_void_p, C.c_void_p, C.c_int], C.c_int),
    "tled_get_isotherm_volume": ([C.c_void_p, C.c_double, C.POINTER(C.c_double)], C.c_int),
    "tled_set_state": ([C.c_void_p, _dp, _dp, _dp, _dp, _dp, C.c_double, C.c_int64], C.c_int),
    "tled_get_state": ([C.c_void_p, _dp, _dp, _dp, _dp, _dp, _dp, C.POINTER(C.c_int64)], C.c_int),
    "tled_get_stats": ([C.c_void_p, C.POINTER(Stats)], C.c_int),
    "tled_step_timed": ([C.c_void_p, C.c_int64, _dp], C.c_int),
    "tled_get_stats_noalloc": ([C.c_void_p, C.c_int32, C.c_void_p], C.c_int),
    "tled_plan_info": ([C.c_void_p, C.POINTER(C.c_int64)], C.c_int),
    "tled_l2_window": ([C.c_void_p, C.POINTER(C.c_int64)], C.c_int),
    "tled_set_probes": ([C.c_void_p, C.c_int64, _dp], C.c_int),
    "tled_get_probes": ([C.c_void_p, C.c_void_p, C.c_int], C.c_int),
    "tled_batch_create": ([C.POINTER(C.c_void_p), C.c_int, C.c_void_p], C.c_int),
    "tled_batch_add": ([C.c_void_p, C.c_void_p, C.c_int64, C.POINTER(C.c_int32)], C.c_int),
    "tled_batch_run": ([C.c_void_p, C.POINTER(C.c_int64)], C.c_int),
    "tled_scenario_info": ([C.c_void_p, C.c_int32, C.POINTER(C.c_int64)], C.c_int),
    "tled_scenario_dt": ([C.c_void_p, C.c_int32, _dp], C.c_int),
    "tled_stable_dt": ([C.c_void_p, _dp, _dp], C.c_int),
    "tled_get_mass_scale": ([C.c_void_p, C.c_int32, _dp], C.c_int),
    "tled_autotune": ([C.c_void_p, C.c_void_p, C.c_int64, C.c_int32, C.POINTER(C.c_int32)], C.c_int),
    "tled_get_mode": ([C.c_void_p, C.POINTER(C.c_int32)], C.c_int),
    "tled_selftest_wait": ([C.c_void_p, C.c_int32], C.c_int),
    "tled_save_state": ([C.c_void_p, C.c_void_p, C.POINTER(C.c_int64)], C.c_int),
    "tled_load_state": ([C.c_void_p, C.c_void_p, C.c_int64], C.c_int),
}


def lib():
    """Load libtled.so (built in-tree).  Raises if it is missing."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"libtled.so not built ({LIB_PATH}); run `python -m paper_2009_10400_b300.build`")
        L = C.CDLL(LIB_PATH)
        for name, (args, res) in _SIGS.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = res
        _lib = L
    return _lib


def exported_symbols():
    return list(_SIGS)


def _p(a):
    return None if a is None else a.ctypes.data_as(_dp)


def material_from_problem(prob) -> Material:
    m = Material()
    m.rho = float(prob.rho[0])
    for f, src in (("mu", prob.mu), ("kappa", prob.kappa), ("k1", prob.k1), ("k2", prob.k2), ("alpha", prob.alpha),
                   ("k", prob.kc)):
        setattr(m, f, float(src[0]))
    for i in range(3):
        m.a0[i] = float(prob.a0[0, i])
    m.n_prony = len(prob.prony_g)
    for i in range(m.n_prony):
        m.prony_g[i] = prob.prony_g[i]
        m.prony_tau[i] = prob.prony_tau[i]
    m.c = prob.c_heat
    m.beta_k, m.beta_c, m.T_ref = prob.beta_k, prob.beta_c, prob.T_ref
    m.wb_cb, m.Qm, m.T0, m.Ta, m.lnA, m.Ea = prob.wbcb, prob.Qm, prob.T0, prob.Ta, prob.lnA, prob.Ea
    m.alpha_fibre_ratio = getattr(prob, "aniso_alpha", 1.0)
    m.k_fibre_ratio = getattr(prob, "aniso_k", 1.0)
    return m


def sources_array(rows) -> tuple:
    rows = np.asarray(rows, np.float64)
    rows = rows.reshape(-1, rows.shape[-1] if rows.size else 11)  # 10 columns: Gaussian; 11th: shape
    arr = (Source * max(len(rows), 1))()
    for i, r in enumerate(rows):
        for j in range(3):
            arr[i].c0[j] = r[j]
            arr[i].vel[j] = r[3 + j]
        arr[i].sigma, arr[i].power, arr[i].t_on, arr[i].t_off = r[6], r[7], r[8], r[9]
        arr[i].shape = int(r[10]) if len(r) > 10 else SRC_GAUSSIAN
    return len(rows), arr


def plan_info(h, check) -> dict:
    info = (C.c_int64 * 8)()
    check(lib().tled_plan_info(h, info))
    return dict(n_tiles=info[0], n_interior=info[1], n_shared=info[2], n_partials=info[3], workspace=info[4],
                npe=info[5], n_scenarios=info[6], ctas=info[7])


class HostPlanner:
    """Host-only context (device -1): validates a problem and sizes/plans it
    without a GPU."""

    def __init__(self):
        L = lib()
        h = C.c_void_p()
        rc = L.tled_create(C.byref(h), -1, None)
        if rc != OK:
            raise TledError(rc, L.tled_status_string(rc).decode())
        self.h = h

    def _check(self, rc):
        if rc != OK:
            raise TledError(rc, lib().tled_last_error(self.h).decode())
        return rc

    def close(self):
        if getattr(self, "h", None):
            lib().tled_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    set_mesh = lambda self, *a, **k: Solver.set_mesh(self, *a, **k)  # noqa: E731
    set_material = lambda self, *a, **k: Solver.set_material(self, *a, **k)  # noqa: E731
    set_bcs = lambda self, *a, **k: Solver.set_bcs(self, *a, **k)  # noqa: E731
    set_heat_sources = lambda self, *a, **k: Solver.set_heat_sources(self, *a, **k)  # noqa: E731
    set_params = lambda self, *a, **k: Solver.set_params(self, *a, **k)  # noqa: E731
    set_probes = lambda self, *a, **k: Solver.set_probes(self, *a, **k)  # noqa: E731
    setup_from = lambda self, *a, **k: Solver.setup_from(self, *a, **k)  # noqa: E731
    workspace_size = lambda self: Solver.workspace_size(self)  # noqa: E731

    def plan_info(self):
        return plan_info(self.h, self._check)

    def stable_dt(self):
        a, b = C.c_double(), C.c_double()
        self._check(lib().tled_stable_dt(self.h, C.byref(a), C.byref(b)))
        return a.value, b.value

    def init(self, ptr=1 << 20, n=1 << 30):
        self._check(lib().tled_init(self.h, C.c_void_p(ptr), n))

    def mass_scale(self, index=0):
        return Solver.mass_scale(self, index)


class Solver:
    """One coupled TLED problem on one GPU (a libtled context + its workspace)."""

    def __init__(self, device: int = 0, stream=None):
        import torch

        if not torch.cuda.is_available():
            raise RuntimeError("libtled needs a CUDA device; there is no CPU fallback")
        self._torch = torch
        self.device = device
        self.stream = stream if stream is not None else torch.cuda.current_stream(device)
        L = lib()
        h = C.c_void_p()
        self._check(L.tled_create(C.byref(h), device, C.c_void_p(self.stream.cuda_stream)), h)
        self.h = h
        self.ws = None
        self.nn = self.ne = 0

    # -- error handling ----------------------------------------------------
    def _check(self, rc, h=None):
        if rc != OK:
            hh = h if h is not None else getattr(self, "h", None)
            msg = lib().tled_last_error(hh).decode() if hh else lib().tled_status_string(rc).decode()
            raise TledError(rc, msg or lib().tled_status_string(rc).decode())
        return rc

    def close(self):
        if getattr(self, "h", None):
            lib().tled_destroy(self.h)
            self.h = None
        self.ws = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- set-up ------------------------------------------------------------
    def set_mesh(self, elem_type, X, conn):
        X = np.ascontiguousarray(X, np.float64)
        conn = np.ascontiguousarray(conn, np.int32)
        self.nn, self.ne, self.npe = X.shape[0], conn.shape[0], elem_type
        self._check(lib().tled_set_mesh(self.h, elem_type, self.nn, _p(X), self.ne,
                                        conn.ctypes.data_as(C.POINTER(C.c_int32))))

    def set_material(self, m: Material, per_elem=None, fibre=None):
        pe = None if per_elem is None else np.ascontiguousarray(per_elem, np.float64)
        fb = None if fibre is None else np.ascontiguousarray(fibre, np.float64)
        self.n_prony = m.n_prony
        self._check(lib().tled_set_material(self.h, C.byref(m), _p(pe), _p(fb)))

    def set_bcs(self, mask, ubar=None, ramp_time=0.0):
        mask = np.ascontiguousarray(mask, np.uint8)
        ub = None if ubar is None else np.ascontiguousarray(ubar, np.float64)
        self._check(lib().tled_set_bcs(self.h, mask.ctypes.data_as(C.POINTER(C.c_uint8)), _p(ub), float(ramp_time)))

    def set_heat_sources(self, rows):
        n, arr = sources_array(rows)
        self._check(lib().tled_set_heat_sources(self.h, n, arr))

    def set_probes(self, xyz):
        xyz = np.ascontiguousarray(xyz, np.float64).reshape(-1, 3)
        self.n_probes = xyz.shape[0]
        self._check(lib().tled_set_probes(self.h, xyz.shape[0], _p(xyz)))

    def set_params(self, dt=0.0, dt_safety=0.8, gamma=0.0, mass_scale=1.0, kappa_hg=0.1, kappa_hgT=0.1,
                   flags=EXPANSION | COMPENSATED, tile_elems=0, n_sub=1):
        p = Params(dt, dt_safety, gamma, mass_scale, kappa_hg, kappa_hgT, flags, tile_elems, n_sub, 0)
        self._check(lib().tled_set_params(self.h, C.byref(p)))

    def workspace_size(self) -> int:
        b = C.c_int64()
        self._check(lib().tled_workspace_size(self.h, C.byref(b)))
        return b.value

    def init(self):
        torch = self._torch
        n = self.workspace_size()
        if self.ws is None or self.ws.numel() < n + 256:
            self.ws = torch.empty(n + 256, dtype=torch.uint8, device=f"cuda:{self.device}")
        base = self.ws.data_ptr()
        ptr = (base + 255) & ~255
        self._check(lib().tled_init(self.h, C.c_void_p(ptr), n))

    @classmethod
    def from_problem(cls, prob, device=0, stream=None, dt=None, flags=None, tile_elems=0, probes=None,
                     init=True):
        s = cls(device, stream)
        s.setup_from(prob, dt=dt, flags=flags, tile_elems=tile_elems, probes=probes)
        if init:
            s.init()
        return s

    def setup_from(self, prob, dt=None, flags=None, tile_elems=0, probes=None):
        """Set-up calls for a workloads.Problem (no init)."""
        s = self
        s.set_mesh(prob.npe, prob.X, prob.conn)
        per = np.stack([prob.mu, prob.kappa, prob.k1, prob.k2, prob.kc, prob.alpha], 1) if prob.per_element else None
        fib = prob.a0 if prob.per_element else None
        s.set_material(material_from_problem(prob), per, fib)
        s.set_bcs(prob.mask, prob.ubar, prob.ramp_time)
        s.set_heat_sources(prob.sources)
        if flags is None:
            flags = default_flags(prob)
        s.set_params(dt=float(prob.dt if dt is None else dt), dt_safety=prob.dt_safety, gamma=prob.gamma,
                     mass_scale=prob.mass_scale, kappa_hg=prob.kappa_hg, kappa_hgT=prob.kappa_hgT, flags=flags,
                     tile_elems=tile_elems, n_sub=prob.n_sub)
        if probes is not None:
            s.set_probes(probes)
        return s

    def mass_scale(self, index=0) -> float:
        """Mechanical mass multiplier in use for scenario `index` (the automatic
        R17 choice when the set-up asked for mass_scale < 0)."""
        a = C.c_double()
        self._check(lib().tled_get_mass_scale(self.h, int(index), C.byref(a)))
        return a.value

    # -- stepping ----------------------------------------------------------
    def get_dt(self):
        a, b, c = C.c_double(), C.c_double(), C.c_double()
        self._check(lib().tled_get_dt(self.h, C.byref(a), C.byref(b), C.byref(c)))
        return a.value, b.value, c.value

    def step(self, n=1):
        self._check(lib().tled_step(self.h, int(n)))

    def sync(self):
        self._check(lib().tled_sync(self.h))

    def step_timed(self, n):
        """n steps with per-kernel CUDA events: (ms tile kernel, ms shared-node kernel)."""
        ms = (C.c_double * 2)()
        self._check(lib().tled_step_timed(self.h, int(n), ms))
        return ms[0], ms[1]

    def plan_info(self) -> dict:
        return plan_info(self.h, self._check)

    def l2_window(self) -> dict:
        """The streamed step's persisting-L2 window: bytes, the context's set-aside, hit ratio."""
        out = (C.c_int64 * 3)()
        self._check(lib().tled_l2_window(self.h, out))
        return {"window_bytes": int(out[0]), "set_aside_bytes": int(out[1]), "hit_ratio": out[2] / 1e6}

    def selftest_wait(self, which: int) -> int:
        """Run the bounded-wait self-test (0: mbarrier, 1: grid barrier); returns the
        library status code (E_TIMEOUT expected)."""
        return lib().tled_selftest_wait(self.h, int(which))

    def _mode(self) -> int:
        m = C.c_int32()
        self._check(lib().tled_get_mode(self.h, C.byref(m)))
        return m.value

    @property
    def resident(self) -> bool:
        """True when the steps run in the resident mode (each scenario held by one CTA)."""
        return bool(self._mode() & 1)

    @property
    def grid_resident(self) -> bool:
        """True when the steps run in the grid-resident mode (one cooperative launch per chunk)."""
        return bool(self._mode() & 4)

    @property
    def brick(self) -> bool:
        """True when the H8 brick instance (axis-aligned boxes: no reference hourglass
        projections, diagonal J0^-1) runs."""
        return bool(self._mode() & 2)

    # -- read-back ---------------------------------------------------------
    def _read(self, fn, shape, out=None):
        if out is None:
            a = np.empty(shape, np.float64)
            self._check(fn(self.h, a.ctypes.data_as(C.c_void_p), HOST))
            return a
        # a torch tensor: device memory (enqueued only) or host memory (pinned or not; synchronises)
        where = DEVICE if out.is_cuda else HOST
        self._check(fn(self.h, C.c_void_p(out.data_ptr()), where))
        return out

    def displacement(self, out=None):
        return self._read(lib().tled_get_displacement, (self.nn, 3), out)

    def temperature(self, out=None):
        return self._read(lib().tled_get_temperature, (self.nn,), out)

    def damage(self, out=None):
        return self._read(lib().tled_get_damage, (self.nn,), out)

    def cem43(self, out=None):
        """CEM43 thermal dose per node, equivalent minutes at 43 C (needs the CEM43 flag)."""
        return self._read(lib().tled_get_cem43, (self.nn,), out)

    def isotherm_volume(self, T_iso=60.0):
        """Volume (m^3) of the nodes at or above T_iso (C)."""
        v = C.c_double()
        self._check(lib().tled_get_isotherm_volume(self.h, float(T_iso), C.byref(v)))
        return v.value

    def set_state(self, u, v, T, Omega, visc=None, t=0.0, step=0):
        arrs = [np.ascontiguousarray(a, np.float64) for a in (u, v, T, Omega)]
        vs = None if visc is None else np.ascontiguousarray(visc, np.float64)
        self._check(lib().tled_set_state(self.h, *[_p(a) for a in arrs], _p(vs), float(t), int(step)))

    def get_state(self):
        nn, ne = self.nn, self.ne
        u, v, T, Om = np.empty((nn, 3)), np.empty((nn, 3)), np.empty(nn), np.empty(nn)
        vs = np.empty((ne, max(self.n_prony, 1), 6))
        t, st = C.c_double(), C.c_int64()
        self._check(lib().tled_get_state(self.h, _p(u), _p(v), _p(T), _p(Om), _p(vs), C.byref(t), C.byref(st)))
        return dict(u=u, v=v, T=T, Omega=Om, visc=vs, t=t.value, step=st.value)

    def stats(self) -> dict:
        s = Stats()
        self._check(lib().tled_get_stats(self.h, C.byref(s)))
        return s.as_dict()

    def probes(self, out=None):
        """(temperature, damage) at the probe points."""
        n = getattr(self, "n_probes", 0)
        if out is None:
            a = np.empty((2, n), np.float64)
            if n:
                self._check(lib().tled_get_probes(self.h, a.ctypes.data_as(C.c_void_p), HOST))
            return a
        self._check(lib().tled_get_probes(self.h, C.c_void_p(out.data_ptr()), DEVICE if out.is_cuda else HOST))
        return out

    def autotune(self, trial_steps=20, workspace_bytes=None):
        """Pick the fastest tiling by timing (see tled_autotune); re-initialises the state."""
        torch = self._torch
        if self.ws is None or (workspace_bytes and self.ws.numel() < workspace_bytes):
            n = workspace_bytes or int(self.workspace_size() * 1.6) + (1 << 20)
            self.ws = torch.empty(n + 256, dtype=torch.uint8, device=f"cuda:{self.device}")
        base = (self.ws.data_ptr() + 255) & ~255
        ch = (C.c_int32 * 3)()
        self._check(lib().tled_autotune(self.h, C.c_void_p(base), self.ws.numel() - 256, int(trial_steps), ch))
        return dict(tile_elems=ch[0], ctas=ch[1], cached=bool(ch[2]))

    def stats_noalloc(self, out, n_blocks=0):
        """Allocation-free diagnostics into a device float64 tensor of 6 entries
        (enqueued on the solver's stream, no synchronisation)."""
        assert out.is_cuda and out.dtype.is_floating_point and out.element_size() == 8 and out.numel() >= 6
        self._check(lib().tled_get_stats_noalloc(self.h, int(n_blocks), C.c_void_p(out.data_ptr())))
        return out

    def save_state(self) -> bytes:
        n = C.c_int64()
        self._check(lib().tled_save_state(self.h, None, C.byref(n)))
        buf = C.create_string_buffer(n.value)
        self._check(lib().tled_save_state(self.h, buf, C.byref(n)))
        return buf.raw

    def load_state(self, blob: bytes):
        buf = C.create_string_buffer(blob, len(blob))
        self._check(lib().tled_load_state(self.h, buf, len(blob)))


class Batch(Solver):
    """Many independent scenarios advanced together (tled_batch_*).

    ``add(problem, n_steps)`` copies a scenario's set-up; after ``init()``,
    ``run()`` steps every scenario to its own n_steps in the same launches;
    field read-backs return all scenarios concatenated (see ``scenario``)."""

    def __init__(self, device: int = 0, stream=None):
        import torch

        if not torch.cuda.is_available():
            raise RuntimeError("libtled needs a CUDA device; there is no CPU fallback")
        self._torch = torch
        self.device = device
        self.stream = stream if stream is not None else torch.cuda.current_stream(device)
        h = C.c_void_p()
        self._check(lib().tled_batch_create(C.byref(h), device, C.c_void_p(self.stream.cuda_stream)), h)
        self.h = h
        self.ws = None
        self.n_scn = 0
        self.n_probes = 0

    def add(self, prob, n_steps, dt=None, flags=None, probes=None):
        one = HostPlanner()  # set-up only: the batch copies it
        one.setup_from(prob, dt=dt, flags=flags, probes=probes)
        idx = C.c_int32()
        self._check(lib().tled_batch_add(self.h, one.h, int(n_steps), C.byref(idx)))
        one.close()
        self.n_scn += 1
        self.n_prony = len(prob.prony_g)
        self.n_probes += 0 if probes is None else len(probes)
        return idx.value

    def init(self):
        super().init()
        info = self.plan_info()
        tot = [self.scenario(i) for i in range(self.n_scn)]
        self.nn = sum(t["nodes"] for t in tot)
        self.ne = sum(t["elements"] for t in tot)
        return info

    def run(self):
        n = C.c_int64()
        self._check(lib().tled_batch_run(self.h, C.byref(n)))
        return n.value

    def scenario(self, i) -> dict:
        info = (C.c_int64 * 8)()
        self._check(lib().tled_scenario_info(self.h, int(i), info))
        return dict(node_off=info[0], nodes=info[1], elem_off=info[2], elements=info[3], n_steps=info[4],
                    steps=info[5], probe_off=info[6], probes=info[7])

    def scenario_dt(self, i) -> float:
        d = C.c_double()
        self._check(lib().tled_scenario_dt(self.h, int(i), C.byref(d)))
        return d.value
