"""Seeded synthetic inputs for the coupled thermo-visco-hyperelastic TLED step.

This module only *builds inputs*: meshes, material fields, heat sources and
boundary masks, drawn with ``numpy.random.default_rng(seed)``.  It holds none
of the method's arithmetic (no shape functions, stresses, lumping or time
steps), so both the CUDA library and the FP64 CPU oracle can consume the same
:class:`Problem` without sharing any computation.

Workloads (sizes and materials follow the paper's liver models, Section 6.3,
Table 5; the paper's own meshes come from a clinical dataset that is not
available, so synthetic shapes stand in):

* :func:`cube_h8`      -- 5 cm cube of n^3 hexahedra (n = 8: 729 nodes), bottom fixed.
* :func:`ellipsoid_t4` -- 15 x 10 x 8 cm ellipsoid "liver" of linear tetrahedra from a
  seeded Delaunay of a jittered BCC lattice, per-element von Mises-Fisher fibres,
  a Gaussian source moving along a straight needle track.
* :func:`block_h8`     -- 12.8 cm block of n^3 hexahedra (n = 128: 2.1M elements) with
  +-10 % per-element material noise and four Gaussian sources.
"""
from __future__ import annotations

import dataclasses
from typing import Optional

import numpy as np

# Arrhenius constants for liver (a common literature set), J/mol and 1/s.
ARRHENIUS_A = 7.39e39
ARRHENIUS_EA = 2.577e5
# Perfusion: w_b c_b = rho_b * omega * c_b with blood density and heat capacity
# of the paper's Table 5 (1060 kg/m^3, 3617 J/(kg K)) and omega = 0.0064 1/s.
BLOOD_RHO = 1060.0
BLOOD_CB = 3617.0

MASK_UX, MASK_UY, MASK_UZ, MASK_T = 1, 2, 4, 8
MASK_U = MASK_UX | MASK_UY | MASK_UZ


@dataclasses.dataclass
class Problem:
    """One coupled thermo-mechanical problem, SI units, temperatures in C."""

    name: str
    npe: int                      # 4 = linear tetrahedron, 8 = hexahedron
    X: np.ndarray                 # (nn, 3) float64 reference coordinates
    conn: np.ndarray              # (ne, npe) int32, VTK corner order
    rho: np.ndarray               # (ne,) density
    mu: np.ndarray                # (ne,) shear modulus
    kappa: np.ndarray             # (ne,) bulk modulus
    k1: np.ndarray                # (ne,) fibre stiffness
    k2: np.ndarray                # (ne,) fibre exponent
    kc: np.ndarray                # (ne,) conductivity at T_ref
    alpha: np.ndarray             # (ne,) thermal expansion
    a0: np.ndarray                # (ne, 3) unit fibre direction
    per_element: bool             # True if mu..alpha or a0 vary per element
    prony_g: tuple = (0.5,)
    prony_tau: tuple = (0.5,)
    c_heat: float = 3600.0
    beta_c: float = 0.0           # relative slope of c(T), 1/K
    beta_k: float = 0.0           # relative slope of k(T), 1/K
    T_ref: float = 37.0
    wbcb: float = BLOOD_RHO * 0.0064 * BLOOD_CB
    Qm: float = 0.0
    T0: float = 37.0
    Ta: float = 37.0
    lnA: float = float(np.log(ARRHENIUS_A))
    Ea: float = ARRHENIUS_EA
    expansion: bool = True
    temp_dep: bool = False
    cem43: bool = False           # track the CEM43 thermal dose
    aniso_alpha: float = 1.0      # thermal expansion along the fibre / transverse (Eq. 11)
    aniso_k: float = 1.0          # conductivity along the current fibre / transverse
    gamma: float = 0.0
    mass_scale: float = 1.0       # mechanical mass multiplier >= 1; < 0: chosen so that dt is the safe
                                  # mechanical step (R17 mass scaling, needs a fixed dt)
    kappa_hg: float = 0.1
    kappa_hgT: float = 0.1
    dt: float = 0.0               # 0 = use the stable step (with n_sub > 1: the thermal step)
    n_sub: int = 1                # mechanical substeps per thermal step (subcycling)
    dt_safety: float = 0.8
    sources: np.ndarray = dataclasses.field(default_factory=lambda: np.zeros((0, 11)))
    mask: Optional[np.ndarray] = None     # (nn,) uint8
    ubar: Optional[np.ndarray] = None     # (nn, 3) float64
    ramp_time: float = 0.0
    n_steps: int = 100

    @property
    def nn(self) -> int:
        return int(self.X.shape[0])

    @property
    def ne(self) -> int:
        return int(self.conn.shape[0])

    def __post_init__(self):
        self.X = np.ascontiguousarray(self.X, dtype=np.float64)
        self.conn = np.ascontiguousarray(self.conn, dtype=np.int32)
        for f in ("rho", "mu", "kappa", "k1", "k2", "kc", "alpha"):
            setattr(self, f, np.ascontiguousarray(getattr(self, f), dtype=np.float64))
        self.a0 = np.ascontiguousarray(self.a0, dtype=np.float64)
        src = np.asarray(self.sources, dtype=np.float64)
        src = src.reshape(-1, src.shape[-1] if src.size else 11)
        if src.shape[1] == 10:  # rows without a shape column are Gaussian
            src = np.concatenate([src, np.zeros((len(src), 1))], 1)
        self.sources = np.ascontiguousarray(src)
        if self.mask is None:
            self.mask = np.zeros(self.nn, np.uint8)
        self.mask = np.ascontiguousarray(self.mask, dtype=np.uint8)
        if self.ubar is not None:
            self.ubar = np.ascontiguousarray(self.ubar, dtype=np.float64)


def source(c0, power, sigma=5e-3, vel=(0.0, 0.0, 0.0), t_on=0.0, t_off=1e30, sphere=False):
    """One source row: centre, velocity, sigma (Gaussian) or radius (uniform
    sphere), peak W/m^3, on/off times, shape (0 Gaussian, 1 uniform sphere)."""
    return [*map(float, c0), *map(float, vel), float(sigma), float(power), float(t_on), float(t_off),
            1.0 if sphere else 0.0]


# ---------------------------------------------------------------------------
# meshes
# ---------------------------------------------------------------------------
def hex_grid(n, size, origin=(0.0, 0.0, 0.0), jitter=0.0, rng=None):
    """Structured grid of hexahedra. Node (i,j,k) -> i + (nx+1)(j + (ny+1)k)."""
    nx, ny, nz = n
    xs = [np.linspace(origin[d], origin[d] + size[d], (nx, ny, nz)[d] + 1) for d in range(3)]
    Z, Y, Xg = np.meshgrid(xs[2], xs[1], xs[0], indexing="ij")
    X = np.stack([Xg.ravel(), Y.ravel(), Z.ravel()], axis=1)
    if jitter > 0:
        h = np.array([size[d] / (nx, ny, nz)[d] for d in range(3)])
        X = X + rng.uniform(-jitter, jitter, X.shape) * h
    i, j, k = np.meshgrid(np.arange(nx), np.arange(ny), np.arange(nz), indexing="ij")
    i, j, k = (a.transpose(2, 1, 0).ravel() for a in (i, j, k))  # x fastest
    nid = lambda a, b, c: a + (nx + 1) * (b + (ny + 1) * c)
    conn = np.stack([nid(i, j, k), nid(i + 1, j, k), nid(i + 1, j + 1, k), nid(i, j + 1, k),
                     nid(i, j, k + 1), nid(i + 1, j, k + 1), nid(i + 1, j + 1, k + 1), nid(i, j + 1, k + 1)],
                    axis=1).astype(np.int32)
    return X, conn


def _orient_tets(X, conn):
    """Swap two corners of negatively oriented tetrahedra (input preparation)."""
    p = X[conn]
    d = np.einsum("ij,ij->i", np.cross(p[:, 1] - p[:, 0], p[:, 2] - p[:, 0]), p[:, 3] - p[:, 0])
    conn = conn.copy()
    neg = d < 0
    conn[neg, 1], conn[neg, 2] = conn[neg, 2].copy(), conn[neg, 1].copy()
    return conn


def kuhn_tets(n, size, origin=(0.0, 0.0, 0.0), jitter=0.0, rng=None):
    """Six-tetrahedron (Kuhn) split of every cell of a structured grid: no slivers."""
    X, hexes = hex_grid(n, size, origin, jitter, rng)
    split = [(0, 1, 2, 6), (0, 2, 3, 6), (0, 3, 7, 6), (0, 7, 4, 6), (0, 4, 5, 6), (0, 5, 1, 6)]
    conn = np.concatenate([hexes[:, list(s)] for s in split], axis=0)
    conn = conn.reshape(6, -1, 4).transpose(1, 0, 2).reshape(-1, 4)  # keep a cell's tets together
    return X, _orient_tets(X, conn.astype(np.int32))


def _tet_quality(X, conn):
    """Normalised volume / rms-edge^3 ratio (1 for the regular tetrahedron)."""
    p = X[conn]
    vol = np.abs(np.einsum("ij,ij->i", np.cross(p[:, 1] - p[:, 0], p[:, 2] - p[:, 0]), p[:, 3] - p[:, 0])) / 6
    edges = [(0, 1), (0, 2), (0, 3), (1, 2), (1, 3), (2, 3)]
    l2 = sum(((p[:, a] - p[:, b]) ** 2).sum(1) for a, b in edges) / 6.0
    return vol / (l2 ** 1.5) * 6.0 * np.sqrt(2.0)


def tet_ellipsoid(semi_axes, spacing, jitter=0.1, rng=None, min_quality=0.1):
    """Seeded Delaunay tetrahedralisation of jittered BCC lattice points inside an
    ellipsoid; tetrahedra of low quality or with a centroid outside are peeled."""
    from scipy.spatial import Delaunay

    a, b, c = semi_axes
    h = spacing
    g = [np.arange(-s, s + h, h) for s in (a, b, c)]
    P = np.stack(np.meshgrid(*g, indexing="ij"), -1).reshape(-1, 3)
    P = np.concatenate([P, P + h / 2])  # body-centred cubic
    P = P + rng.uniform(-jitter, jitter, P.shape) * h
    inside = (P[:, 0] / a) ** 2 + (P[:, 1] / b) ** 2 + (P[:, 2] / c) ** 2 <= 1.0
    P = P[inside]
    tri = Delaunay(P)
    conn = tri.simplices.astype(np.int32)
    cen = P[conn].mean(1)
    keep = ((cen[:, 0] / a) ** 2 + (cen[:, 1] / b) ** 2 + (cen[:, 2] / c) ** 2 <= 1.0)
    keep &= _tet_quality(P, conn) >= min_quality
    conn = conn[keep]
    used = np.unique(conn)
    remap = -np.ones(P.shape[0], np.int64)
    remap[used] = np.arange(used.size)
    X = P[used]
    conn = remap[conn].astype(np.int32)
    return X, _orient_tets(X, conn)


def boundary_nodes_t4(conn):
    """Nodes on faces that belong to exactly one tetrahedron."""
    faces = np.concatenate([conn[:, [1, 2, 3]], conn[:, [0, 2, 3]], conn[:, [0, 1, 3]], conn[:, [0, 1, 2]]])
    fs = np.sort(faces, axis=1)
    _, idx, cnt = np.unique(fs, axis=0, return_index=True, return_counts=True)
    return np.unique(fs[idx[cnt == 1]])


def vmf_directions(n, kappa, mean, rng):
    """Unit vectors from a von Mises-Fisher distribution on the sphere (3-D inverse CDF)."""
    xi = rng.uniform(size=n)
    w = 1.0 + np.log(xi + (1.0 - xi) * np.exp(-2.0 * kappa)) / kappa
    phi = rng.uniform(0.0, 2.0 * np.pi, n)
    s = np.sqrt(np.clip(1.0 - w * w, 0.0, None))
    v = np.stack([w, s * np.cos(phi), s * np.sin(phi)], 1)  # around +x
    mean = np.asarray(mean, float) / np.linalg.norm(mean)
    # rotate +x onto mean (Rodrigues); the default mean is +x
    ex = np.array([1.0, 0.0, 0.0])
    k = np.cross(ex, mean)
    sk = np.linalg.norm(k)
    if sk < 1e-12:
        return v if mean[0] > 0 else -v
    k /= sk
    ck = float(ex @ mean)
    Kx = np.array([[0, -k[2], k[1]], [k[2], 0, -k[0]], [-k[1], k[0], 0]])
    Rm = np.eye(3) + sk * Kx + (1 - ck) * Kx @ Kx
    return v @ Rm.T


# ---------------------------------------------------------------------------
# materials
# ---------------------------------------------------------------------------
LIVER = dict(rho=1000.0, mu=3.0e3, kappa=3.0e5, k1=1.0e3, k2=10.0, kc=0.5, alpha=1.0e-4)


def _material(ne, rng=None, noise=0.0, fibre=None, **over):
    m = dict(LIVER)
    m.update(over)
    out = {}
    for key in ("rho", "mu", "kappa", "k1", "k2", "kc", "alpha"):
        v = np.full(ne, m[key], np.float64)
        if noise > 0 and key != "rho":
            v = v * rng.uniform(1.0 - noise, 1.0 + noise, ne)
        out[key] = v
    out["a0"] = np.tile([1.0, 0.0, 0.0], (ne, 1)) if fibre is None else fibre
    out["per_element"] = bool(noise > 0 or fibre is not None)
    return out


# ---------------------------------------------------------------------------
# workloads
# ---------------------------------------------------------------------------
def cube_h8(n=8, seed=1, n_steps=2000, side=0.05, power=5e6, jitter=0.0):
    """5 cm cube of n^3 H8 (n = 8: 512 elements, 729 nodes); z = 0 face fixed;
    one Gaussian source (sigma 5 mm) at the centre; liver-like material."""
    rng = np.random.default_rng(seed)
    X, conn = hex_grid((n, n, n), (side, side, side), jitter=jitter, rng=rng)
    mask = np.where(np.isclose(X[:, 2], 0.0), MASK_U, 0).astype(np.uint8)
    return Problem(name=f"cube_h8_{n}", npe=8, X=X, conn=conn, **_material(conn.shape[0]),
                   sources=[source((side / 2,) * 3, power)], mask=mask, n_steps=n_steps)


def block_h8(n=128, seed=3, n_steps=5000, h=1e-3, noise=0.1, n_sources=4):
    """Block of n^3 H8 of edge h (n = 128, h = 1 mm: 2,097,152 elements and
    2,146,689 nodes); bottom fixed; mu, kappa, k1, k2, k, alpha x U(0.9, 1.1) per
    element; Gaussian sources at positions uniform in the inner half, peak
    power U(2, 8) MW/m^3, sigma 5 mm."""
    rng = np.random.default_rng(seed)
    L = n * h
    X, conn = hex_grid((n, n, n), (L, L, L))
    mat = _material(conn.shape[0], rng, noise=noise)
    src = [source(rng.uniform(L / 4, 3 * L / 4, 3), rng.uniform(2e6, 8e6)) for _ in range(n_sources)]
    mask = np.where(np.isclose(X[:, 2], 0.0), MASK_U, 0).astype(np.uint8)
    name = f"block_h8_{n}" if h == 1e-3 else f"block_h8_{n}_h{h * 1e3:g}mm"
    return Problem(name=name, npe=8, X=X, conn=conn, **mat, sources=src, mask=mask, n_steps=n_steps)


def ellipsoid_t4(seed=2, spacing=3.7e-3, semi_axes=(0.075, 0.05, 0.04), n_steps=10000,
                 kappa_vmf=5.0, track=0.03, track_time=0.6, power=5e6, fix_below=-0.035):
    """Ellipsoid 'liver' of T4 (semi-axes 7.5 x 5 x 4 cm, spacing 3.7 mm: ~25k nodes,
    ~120k tets); vMF(kappa = 5) fibres about x; a Gaussian source that moves
    along a straight needle track of 3 cm over `track_time` seconds; surface nodes
    below z = -3.5 cm fixed."""
    rng = np.random.default_rng(seed)
    X, conn = tet_ellipsoid(semi_axes, spacing, 0.1, rng)
    fib = vmf_directions(conn.shape[0], kappa_vmf, (1, 0, 0), rng)
    mat = _material(conn.shape[0], fibre=fib)
    a = np.asarray(semi_axes)
    while True:  # entry point uniform in the inner half of the ellipsoid
        c0 = rng.uniform(-a / 2, a / 2)
        if ((c0 / (a / 2)) ** 2).sum() <= 1.0:
            break
    d = rng.normal(size=3)
    d /= np.linalg.norm(d)
    src = [source(c0, power, vel=d * track / track_time)]
    bnd = boundary_nodes_t4(conn)
    mask = np.zeros(X.shape[0], np.uint8)
    mask[bnd[X[bnd, 2] < fix_below]] = MASK_U
    return Problem(name="ellipsoid_t4", npe=4, X=X, conn=conn, **mat, sources=src, mask=mask,
                   n_steps=n_steps)


def cube_t4(n=6, seed=7, side=0.05, power=5e6, jitter=0.15, n_steps=500):
    """Small Kuhn-split tetrahedral cube with jittered nodes and vMF fibres (tests)."""
    rng = np.random.default_rng(seed)
    X, conn = kuhn_tets((n, n, n), (side, side, side), jitter=0.0, rng=rng)
    interior = np.all((X > 1e-9) & (X < side - 1e-9), axis=1)
    X[interior] += rng.uniform(-jitter, jitter, (interior.sum(), 3)) * (side / n)
    fib = vmf_directions(conn.shape[0], 5.0, (1, 0, 0), rng)
    mat = _material(conn.shape[0], rng, noise=0.1, fibre=fib)
    mask = np.where(np.isclose(X[:, 2], 0.0), MASK_U, 0).astype(np.uint8)
    src = [source((side / 2, side / 2, side / 2), power, vel=(0.01, 0.0, 0.0))]
    return Problem(name=f"cube_t4_{n}", npe=4, X=X, conn=conn, **mat, sources=src, mask=mask,
                   n_steps=n_steps)


def random_state(prob: Problem, seed: int, u_scale=1e-3, v_scale=1e-3, theta_scale=5.0,
                 visc_scale=50.0, n_prony=None):
    """A seeded, smooth-plus-noise mid-run state (u, v, T, Omega, Prony) used to
    compare single steps at full size.  Returns float64 arrays."""
    rng = np.random.default_rng(seed)
    X = prob.X
    L = np.ptp(X, axis=0).max()
    k = rng.uniform(1.0, 3.0, 3) * np.pi / L
    smooth = np.sin(k[0] * X[:, 0]) * np.cos(k[1] * X[:, 1]) * np.sin(k[2] * X[:, 2] + 0.3)
    u = u_scale * (smooth[:, None] * rng.uniform(-1, 1, 3) + 0.05 * rng.uniform(-1, 1, (prob.nn, 3)))
    v = v_scale * rng.uniform(-1, 1, (prob.nn, 3))
    T = prob.T0 + theta_scale * (0.5 + 0.5 * smooth) + 0.1 * rng.uniform(-1, 1, prob.nn)
    Om = rng.uniform(0.0, 0.5, prob.nn)
    npr = len(prob.prony_g) if n_prony is None else n_prony
    visc = visc_scale * rng.uniform(-1, 1, (prob.ne, npr, 6))
    fixed = prob.mask & MASK_U
    for d in range(3):
        sel = (fixed & (1 << d)) != 0
        u[sel, d] = 0.0 if prob.ubar is None else prob.ubar[sel, d]
        v[sel, d] = 0.0
    return dict(u=u, v=v, T=T, Omega=Om, visc=visc)


# ---------------------------------------------------------------------------
# treatment-planning scenarios for the batched solver and the surrogate
# ---------------------------------------------------------------------------
SURROGATE_INPUTS = ("power", "x", "y", "z", "duration", "mu", "kappa", "k", "c", "perfusion", "alpha", "fibre_angle")


def surrogate_ranges(side=0.05):
    """Sampling ranges of the 12 scenario inputs: source peak power (W/m^3),
    position (inner half of the cube), heating duration (s), shear and bulk
    modulus and conductivity (+-20 %), heat capacity and expansion (+-20 %),
    perfusion rate omega (x U(0.5, 1.5) of 0.0064 1/s), fibre angle in the
    x-y plane (rad)."""
    lo = np.array([1e6, side / 4, side / 4, side / 4, 60.0, 0.8 * 3e3, 0.8 * 3e5, 0.8 * 0.5, 0.8 * 3600.0,
                   0.5 * 0.0064, 0.8e-4, 0.0])
    hi = np.array([1e7, 3 * side / 4, 3 * side / 4, 3 * side / 4, 600.0, 1.2 * 3e3, 1.2 * 3e5, 1.2 * 0.5,
                   1.2 * 3600.0, 1.5 * 0.0064, 1.2e-4, np.pi])
    return lo, hi


def sample_scenarios(n, seed=5, side=0.05, duration=None):
    """n x 12 scenario inputs drawn uniformly in `surrogate_ranges` (seeded);
    `duration` = (lo, hi) overrides the heating-time range."""
    rng = np.random.default_rng(seed)
    lo, hi = surrogate_ranges(side)
    if duration is not None:
        lo[4], hi[4] = duration
    return lo + (hi - lo) * rng.uniform(size=(n, 12))


def scenario_problem(q, n=16, side=0.05, dt=0.01, gamma=5.0, sigma=5e-3):
    """Problem of one scenario row q (see SURROGATE_INPUTS) on an n^3 H8 cube,
    bottom fixed, fixed time step dt and damping gamma, with the mechanical
    mass scaled so that dt is the safe mechanical step (R17); its probes are
    the n^3 element centroids."""
    X, conn = hex_grid((n, n, n), (side, side, side))
    ne = conn.shape[0]
    ang = q[11]
    mat = _material(ne, mu=q[5], kappa=q[6], kc=q[7], alpha=q[10])
    mat["a0"] = np.tile([np.cos(ang), np.sin(ang), 0.0], (ne, 1))
    mat["per_element"] = False
    mask = np.where(np.isclose(X[:, 2], 0.0), MASK_U, 0).astype(np.uint8)
    p = Problem(name=f"scenario_h8_{n}", npe=8, X=X, conn=conn, **mat, c_heat=q[8],
                wbcb=BLOOD_RHO * q[9] * BLOOD_CB, sources=[source(q[1:4], q[0], sigma=sigma)], mask=mask,
                dt=dt, gamma=gamma, mass_scale=-1.0, n_steps=int(round(q[4] / dt)))
    return p


def centroids(prob):
    return prob.X[prob.conn].mean(1)


def planning_scenarios(n=256, seed=4, side=0.05, dt=0.01, gamma=5.0, ne_range=(2000, 60000),
                       duration=(60.0, 600.0)):
    """Batched treatment planning: n scenarios, each a hexahedral (jittered n^3
    H8) or tetrahedral (Kuhn-split jittered grid) mesh of the 5 cm cube with a
    log-uniform element count, one Gaussian source of U(1, 10) MW/m^3 in the
    inner half, heating time U(60, 600) s at a fixed dt, shear modulus and
    conductivity x U(0.8, 1.2), bottom fixed, mechanical mass scaled so that dt
    is the safe mechanical step (R17).  Returns a list of Problems (n_steps =
    heating time / dt)."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n):
        ne = float(np.exp(rng.uniform(np.log(ne_range[0]), np.log(ne_range[1]))))
        hexa = rng.uniform() < 0.5
        if hexa:
            m = max(2, int(round(ne ** (1.0 / 3.0))))
            X, conn = hex_grid((m, m, m), (side, side, side))
        else:
            m = max(2, int(round((ne / 6.0) ** (1.0 / 3.0))))
            X, conn = kuhn_tets((m, m, m), (side, side, side))
        interior = np.all((X > 1e-9) & (X < side - 1e-9), axis=1)
        X[interior] += rng.uniform(-0.1, 0.1, (interior.sum(), 3)) * (side / m)
        if not hexa:
            conn = _orient_tets(X, conn)
        mat = _material(conn.shape[0], mu=3e3 * rng.uniform(0.8, 1.2), kc=0.5 * rng.uniform(0.8, 1.2))
        mask = np.where(np.isclose(X[:, 2], 0.0), MASK_U, 0).astype(np.uint8)
        T = rng.uniform(*duration)
        src = [source(rng.uniform(side / 4, 3 * side / 4, 3), rng.uniform(1e6, 1e7))]
        out.append(Problem(name=f"plan_{'h8' if hexa else 't4'}_{i}", npe=8 if hexa else 4, X=X, conn=conn, **mat,
                           sources=src, mask=mask, dt=dt, gamma=gamma, mass_scale=-1.0,
                           n_steps=int(round(T / dt))))
    return out


def liver_f2(spacing=7.3e-3, seed=6, semi_axes=(0.075, 0.05, 0.04), duration=25.0, margin=2e-5):
    """The paper's liver heating case (Section 6.3) on the synthetic ellipsoid:
    temperature-dependent c and k linear through (37 C: 3600 J/kgK, 0.53 W/mK)
    and (90 C: 4300, 0.75), metabolic heat 33.8 kW/m^3, perfusion w_b c_b =
    26.6 x 3617 W/m^3K, three touching uniform spherical sources of 1 cm
    diameter at 9.70536 MW/m^3 along a needle, CEM43 tracked; 25 s of heating.
    The spacing gives about the paper's model size (3234 nodes, 17227 tets, flat
    boundary tets below quality 0.3 peeled).  The sources'
    common centre is nudged (0.1 mm steps) until no node lies within `margin`
    of a sphere surface, so that which nodes are heated is unambiguous.  The
    time step is the stable step of this mesh (the paper's 2e-4 s is above the
    mechanical limit of the synthetic tets)."""
    rng = np.random.default_rng(seed)
    X, conn = tet_ellipsoid(semi_axes, spacing, 0.1, rng, min_quality=0.3)
    fib = vmf_directions(conn.shape[0], 5.0, (1, 0, 0), rng)
    mat = _material(conn.shape[0], fibre=fib, kc=0.53)
    r = 0.005
    c = np.zeros(3)
    for _ in range(200):
        centres = [c + np.array([dx, 0.0, 0.0]) for dx in (-2 * r, 0.0, 2 * r)]
        gap = min(np.min(np.abs(np.linalg.norm(X - cc, axis=1) - r)) for cc in centres)
        if gap > margin:
            break
        c = c + np.array([0.0, 1e-4, 0.0])
    else:
        raise RuntimeError("no source placement clear of the nodes")
    src = [source(cc, 9.70536e6, sigma=r, sphere=True) for cc in centres]
    mask = np.zeros(X.shape[0], np.uint8)
    bnd = boundary_nodes_t4(conn)
    mask[bnd[X[bnd, 2] < -0.035]] = MASK_U  # surface below z = -3.5 cm held
    p = Problem(name="liver_f2", npe=4, X=X, conn=conn, **mat, sources=src, mask=mask, c_heat=3600.0,
                beta_c=(4300.0 / 3600.0 - 1.0) / 53.0, beta_k=(0.75 / 0.53 - 1.0) / 53.0, T_ref=37.0,
                temp_dep=True, Qm=33800.0, wbcb=26.6 * 3617.0, cem43=True, dt=0.0)
    p.n_steps = 0  # set by the driver from the stable step and `duration`
    p.duration = duration
    return p
