"""Python handle on the FP64 CPU oracle (ctypes over ``liboracle.so``).

TEST INFRASTRUCTURE ONLY: the oracle exists to check the CUDA library.  Only
the test-suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package; the library never does.

The oracle consumes any object with the fields of ``workloads.Problem`` (duck
typed, nothing imported from the library package).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_SRC = os.path.join(_HERE, "tled_oracle.c")
MAX_PRONY = 4

_dp = C.POINTER(C.c_double)
_ip = C.POINTER(C.c_int32)


class _Model(C.Structure):
    _fields_ = [
        ("npe", C.c_int32), ("pad0", C.c_int32), ("nn", C.c_int64), ("ne", C.c_int64),
        ("X", _dp), ("conn", _ip),
        ("rho", _dp), ("mu", _dp), ("kappa", _dp), ("k1", _dp), ("k2", _dp), ("kc", _dp),
        ("alpha", _dp), ("a0", _dp),
        ("n_prony", C.c_int32), ("pad1", C.c_int32),
        ("prony_g", C.c_double * MAX_PRONY), ("prony_tau", C.c_double * MAX_PRONY),
        ("c_heat", C.c_double), ("beta_c", C.c_double), ("beta_k", C.c_double), ("T_ref", C.c_double),
        ("wbcb", C.c_double), ("Qm", C.c_double), ("T0", C.c_double), ("Ta", C.c_double),
        ("lnA", C.c_double), ("Ea", C.c_double),
        ("expansion", C.c_int32), ("temp_dep", C.c_int32),
        ("gamma", C.c_double), ("mass_scale", C.c_double), ("kappa_hg", C.c_double),
        ("kappa_hgT", C.c_double), ("dt", C.c_double),
        ("n_src", C.c_int32), ("pad2", C.c_int32), ("src", _dp),
        ("mask", C.POINTER(C.c_uint8)), ("ubar", _dp), ("ramp_time", C.c_double),
        ("aniso_alpha", C.c_double), ("aniso_k", C.c_double),
        ("dhdX", _dp), ("V0", _dp), ("hg_gamma", _dp), ("khg", _dp), ("khgT", _dp),
        ("M", _dp), ("Cth", _dp), ("Vn", _dp),
    ]


class _State(C.Structure):
    _fields_ = [("u", _dp), ("u_prev", _dp), ("T", _dp), ("Omega", _dp), ("visc", _dp),
                ("t", C.c_double), ("step", C.c_int64), ("cem", _dp)]


def build(force: bool = False) -> str:
    """Compile the oracle with the system C compiler (plain IEEE FP64, no fast-math)."""
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-o", _LIB_PATH, _SRC,
                               "-lm"])
    return _LIB_PATH


_lib = None


def lib():
    global _lib
    if _lib is None:
        build()
        L = C.CDLL(_LIB_PATH)
        L.ora_setup.argtypes = [C.POINTER(_Model)]
        L.ora_step.argtypes = [C.POINTER(_Model), C.POINTER(_State), _dp, _dp]
        L.ora_element.argtypes = [C.POINTER(_Model), C.c_int64, _dp, _dp, _dp, _dp, _dp, _dp]
        L.ora_element.restype = C.c_double
        L.ora_element_energy.argtypes = [C.POINTER(_Model), C.c_int64, _dp, _dp]
        L.ora_element_energy.restype = C.c_double
        L.ora_element_thermal_energy.argtypes = [C.POINTER(_Model), C.c_int64, _dp, _dp, C.c_double]
        L.ora_element_thermal_energy.restype = C.c_double
        L.ora_step_nodes.argtypes = [C.POINTER(_Model), C.POINTER(_State), C.POINTER(C.c_int64), C.c_int64,
                                     _dp, _dp, _dp]
        L.ora_stable_dt.argtypes = [C.POINTER(_Model), C.c_double, _dp, _dp]
        L.ora_stable_dt.restype = C.c_double
        _i64p = C.POINTER(C.c_int64)
        L.ora_probe.argtypes = [C.POINTER(_Model), C.POINTER(_State), _dp, C.c_int64, _dp, _dp]
        L.ora_incidence.argtypes = [C.POINTER(_Model), _i64p, _i64p]
        L.ora_step_parallel.argtypes = [C.POINTER(_Model), C.POINTER(_State), _i64p, _i64p, _dp, _dp, _dp]
        L.ora_threads.restype = C.c_int
        L.ora_step_subcycled.argtypes = [C.POINTER(_Model), C.POINTER(_State), C.c_int, _dp, _dp]
        _lib = L
    return _lib


def _p(a):
    return a.ctypes.data_as(_dp) if a is not None else None


class OracleState:
    """FP64 state: u(t), u(t - dt) (Eq. 27), absolute T, Omega, Prony state, and
    the CEM43 thermal dose (equivalent minutes at 43 C) of every node."""

    def __init__(self, nn, ne, n_prony, T0):
        self.u = np.zeros((nn, 3))
        self.u_prev = np.zeros((nn, 3))
        self.T = np.full(nn, float(T0))
        self.Omega = np.zeros(nn)
        self.visc = np.zeros((ne, max(n_prony, 1), 6))
        self.cem = np.zeros(nn)
        self.t = 0.0
        self.step = 0

    def _c(self):
        return _State(_p(self.u), _p(self.u_prev), _p(self.T), _p(self.Omega), _p(self.visc),
                      self.t, self.step, _p(self.cem))

    def copy(self):
        s = OracleState.__new__(OracleState)
        for k in ("u", "u_prev", "T", "Omega", "visc", "cem"):
            setattr(s, k, getattr(self, k).copy())
        s.t, s.step = self.t, self.step
        return s


class OracleModel:
    """Precomputed oracle model of a problem (shape derivatives, volumes, masses)."""

    def __init__(self, prob, dt=None):
        L = lib()
        self.prob = prob
        npe, nn, ne = prob.npe, prob.nn, prob.ne
        self.n_prony = len(prob.prony_g)
        assert self.n_prony <= MAX_PRONY
        self.dhdX = np.zeros((ne, npe, 3))
        self.V0 = np.zeros(ne)
        self.hg_gamma = np.zeros((ne, 8, 4)) if npe == 8 else None
        self.khg = np.zeros(ne)
        self.khgT = np.zeros(ne)
        self.M = np.zeros(nn)
        self.Cth = np.zeros(nn)
        self.Vn = np.zeros(nn)
        src = np.asarray(prob.sources, np.float64).reshape(-1, np.shape(prob.sources)[-1] if np.size(prob.sources) else 11)
        if src.shape[1] == 10:  # rows without a shape column are Gaussian
            src = np.concatenate([src, np.zeros((len(src), 1))], 1)
        self._src = np.ascontiguousarray(src)
        self._keep = [prob.X, prob.conn, prob.a0, self._src, prob.mask, prob.ubar]
        m = _Model()
        m.npe, m.nn, m.ne = npe, nn, ne
        m.X = _p(prob.X)
        m.conn = prob.conn.ctypes.data_as(_ip)
        for f in ("rho", "mu", "kappa", "k1", "k2", "kc", "alpha", "a0"):
            setattr(m, f, _p(getattr(prob, f)))
        m.n_prony = self.n_prony
        for i in range(self.n_prony):
            m.prony_g[i] = prob.prony_g[i]
            m.prony_tau[i] = prob.prony_tau[i]
        for f in ("c_heat", "beta_c", "beta_k", "T_ref", "wbcb", "Qm", "T0", "Ta", "lnA", "Ea", "gamma",
                  "mass_scale", "kappa_hg", "kappa_hgT", "ramp_time", "aniso_alpha", "aniso_k"):
            setattr(m, f, float(getattr(prob, f)))
        self.n_sub = max(1, int(getattr(prob, "n_sub", 1)))
        if prob.mass_scale < 0:  # R17: scaled so that the fixed (sub)step is the safe mechanical step
            m.mass_scale = mass_scale_for(prob, prob.dt / self.n_sub, prob.dt_safety)
        self.mass_scale = m.mass_scale
        m.expansion = int(bool(prob.expansion))
        m.temp_dep = int(bool(prob.temp_dep))
        m.n_src = self._src.shape[0]
        m.src = _p(self._src) if m.n_src else None
        m.mask = prob.mask.ctypes.data_as(C.POINTER(C.c_uint8))
        m.ubar = _p(prob.ubar)
        m.dhdX, m.V0, m.hg_gamma = _p(self.dhdX), _p(self.V0), _p(self.hg_gamma)
        m.khg, m.khgT, m.M, m.Cth, m.Vn = _p(self.khg), _p(self.khgT), _p(self.M), _p(self.Cth), _p(self.Vn)
        self._m = m
        rc = L.ora_setup(C.byref(m))
        if rc != 0:
            raise ValueError(f"oracle: non-positive reference Jacobian in element {-rc - 1}")
        if dt is None:  # with subcycling dt is the thermal step, n_sub mechanical substeps long
            if prob.dt > 0:
                dt = prob.dt
            else:
                self.stable_dt(prob.dt_safety)
                dt = prob.dt_safety * min(self.n_sub * self.dt_mech, self.dt_th)
        m.dt = float(dt)
        self.dt = float(dt)
        self._f = np.zeros((nn, 3))
        self._fT = np.zeros(nn)

    def stable_dt(self, safety=0.8):
        a, b = C.c_double(), C.c_double()
        dt = lib().ora_stable_dt(C.byref(self._m), safety, C.byref(a), C.byref(b))
        self.dt_mech, self.dt_th = a.value, b.value
        return dt

    def init_state(self):
        return OracleState(self.prob.nn, self.prob.ne, self.n_prony, self.prob.T0)

    def state_from(self, u, v, T, Omega, visc, t=0.0, step=0):
        """State from (u, v): u(t - dt) = u - dt v (velocity form of Eq. 27)."""
        s = self.init_state()
        s.u[:] = u
        s.u_prev[:] = u - self.dt * v
        s.T[:] = T
        s.Omega[:] = Omega
        if self.n_prony:
            s.visc[:] = visc
        s.t, s.step = t, step
        return s

    def step(self, s: OracleState, n=1):
        L = lib()
        for _ in range(n):
            cs = s._c()
            L.ora_step(C.byref(self._m), C.byref(cs), _p(self._f), _p(self._fT))
            s.t, s.step = cs.t, cs.step
        return s

    def step_thermal(self, s: OracleState, n=1):
        """n thermal steps of self.dt, each of prob.n_sub mechanical substeps
        (ora_step_subcycled)."""
        L = lib()
        for _ in range(n):
            cs = s._c()
            L.ora_step_subcycled(C.byref(self._m), C.byref(cs), self.n_sub, _p(self._f), _p(self._fT))
            s.t, s.step = cs.t, cs.step
        return s

    def step_parallel(self, s: OracleState, n=1):
        """The same steps on all host cores (OpenMP threads, OMP_NUM_THREADS):
        bitwise the result of step()."""
        L = lib()
        if not hasattr(self, "_inc_off"):
            npe = self.prob.npe
            self._inc_off = np.zeros(self.prob.nn + 1, np.int64)
            self._inc_slot = np.zeros(self.prob.ne * npe, np.int64)
            self._elem_out = np.zeros((self.prob.ne, npe, 4))
            ip = C.POINTER(C.c_int64)
            if L.ora_incidence(C.byref(self._m), self._inc_off.ctypes.data_as(ip), self._inc_slot.ctypes.data_as(ip)):
                raise MemoryError("oracle: allocation failed")
        ip = C.POINTER(C.c_int64)
        for _ in range(n):
            cs = s._c()
            L.ora_step_parallel(C.byref(self._m), C.byref(cs), self._inc_off.ctypes.data_as(ip),
                                self._inc_slot.ctypes.data_as(ip), _p(self._elem_out), _p(self._f), _p(self._fT))
            s.t, s.step = cs.t, cs.step
        return s

    def probe(self, s: OracleState, xyz):
        """Temperature (C) and damage fraction at points xyz [k][3] (reference
        coordinates), interpolated with the shape functions of the element
        that contains each point."""
        xyz = np.ascontiguousarray(xyz, float).reshape(-1, 3)
        k = xyz.shape[0]
        T, d = np.zeros(k), np.zeros(k)
        cs = s._c()
        rc = lib().ora_probe(C.byref(self._m), C.byref(cs), _p(xyz), k, _p(T), _p(d))
        if rc:
            raise ValueError(f"oracle: probe {-rc - 1} lies outside the mesh")
        return T, d

    def forces(self):
        """Assembled nodal forces and thermal loads from the last step."""
        return self._f.copy(), self._fT.copy()

    def element(self, e, u, T, visc=None):
        npe = self.prob.npe
        vin = np.zeros((max(self.n_prony, 1), 6)) if visc is None else np.ascontiguousarray(visc, float)
        vout = np.zeros_like(vin)
        fe = np.zeros((npe, 3))
        fTe = np.zeros(npe)
        u = np.ascontiguousarray(u, float)
        T = np.ascontiguousarray(T, float)
        detF = lib().ora_element(C.byref(self._m), int(e), _p(u), _p(T), _p(vin), _p(vout), _p(fe), _p(fTe))
        return fe, fTe, vout, detF

    def energy(self, e, u, T):
        u = np.ascontiguousarray(u, float)
        T = np.ascontiguousarray(T, float)
        return lib().ora_element_energy(C.byref(self._m), int(e), _p(u), _p(T))

    def thermal_energy(self, e, u, T, Tk):
        u = np.ascontiguousarray(u, float)
        T = np.ascontiguousarray(T, float)
        return lib().ora_element_thermal_energy(C.byref(self._m), int(e), _p(u), _p(T), float(Tk))

    def step_nodes(self, s: OracleState, nodes):
        nodes = np.ascontiguousarray(nodes, np.int64)
        k = nodes.size
        ou, oT, oO = np.zeros((k, 3)), np.zeros(k), np.zeros(k)
        cs = s._c()
        rc = lib().ora_step_nodes(C.byref(self._m), C.byref(cs), nodes.ctypes.data_as(C.POINTER(C.c_int64)),
                                  k, _p(ou), _p(oT), _p(oO))
        if rc:
            raise MemoryError("oracle: allocation failed")
        return ou, oT, oO


def threads() -> int:
    """Threads the oracle's parallel step uses on this host."""
    return int(lib().ora_threads())


def mass_scale_for(prob, dt, safety=0.8):
    """R17 mass scaling: the mechanical mass multiplier s_m >= 1 that makes dt
    the safe mechanical step, s_m = (dt / (safety dt_mech))^2, with dt_mech the
    oracle's own CFL bound of the unscaled mesh (R16)."""
    import copy

    q = copy.copy(prob)
    q.mass_scale = 1.0
    m = OracleModel(q, dt=dt)
    m.stable_dt(safety)
    return max(1.0, (dt / (safety * m.dt_mech)) ** 2)


def damage_fraction(Omega):
    """Fraction of necrotised tissue 1 - exp(-Omega) of the Arrhenius integral."""
    return -np.expm1(-np.asarray(Omega))
