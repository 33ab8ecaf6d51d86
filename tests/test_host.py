"""CPU-only tests of the library boundary: the shared object loads and exports
every symbol include/tled.h declares, and the host-side validation and
planning (host-only context, device -1) behave."""
import os
import re

import numpy as np
import pytest

from paper_2009_10400_b300 import tled
from paper_2009_10400_b300 import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", f)).read()
            names |= set(re.findall(r"^\s*(?:int|const char \*|int64_t)\s*(tled_\w+)\s*\(", txt, re.M))
    return names


def test_library_exports_every_declared_symbol():
    L = tled.lib()
    names = _declared()
    assert len(names) >= 24
    for n in names:
        assert hasattr(L, n), n
    from paper_2009_10400_b300 import mlp
    assert set(names) <= set(tled.exported_symbols()) | set(mlp.exported_symbols()) | {"tled_version"}
    hdr = open(os.path.join(ROOT, "include", "tled.h")).read()
    assert L.tled_version() == int(re.search(r"#define TLED_VERSION (\d+)", hdr).group(1))


def _planner(prob, **kw):
    p = tled.HostPlanner()
    p.set_mesh(prob.npe, prob.X, prob.conn)
    per = np.stack([prob.mu, prob.kappa, prob.k1, prob.k2, prob.kc, prob.alpha], 1) if prob.per_element else None
    p.set_material(tled.material_from_problem(prob), per, prob.a0 if prob.per_element else None)
    p.set_bcs(prob.mask)
    p.set_heat_sources(prob.sources)
    p.set_params(**kw)
    return p


def test_plan_counts_structured_block():
    prob = W.block_h8(n=16, h=3e-3)
    p = _planner(prob)
    info = p.plan_info()
    # Morton order cuts 16^3 into sixteen 8x8x4 tiles of 256 elements
    assert info["n_tiles"] == 16
    assert info["n_interior"] + info["n_shared"] == prob.nn
    # shared nodes are exactly those on the internal planes i = 8, j = 8, k = 4, 8, 12
    idx = np.arange(17)
    on_plane = lambda v, planes: np.isin(v, planes)
    I, J, K = np.meshgrid(idx, idx, idx, indexing="ij")
    shared = on_plane(I, [8]) | on_plane(J, [8]) | on_plane(K, [4, 8, 12])
    assert info["n_shared"] == int(shared.sum())
    assert info["workspace"] > 0


def test_plan_single_tile_has_no_shared_nodes():
    prob = W.cube_h8(n=6)
    info = _planner(prob).plan_info()
    assert info["n_tiles"] == 1 and info["n_shared"] == 0 and info["n_interior"] == 343


def test_plan_tile_size_parameter():
    prob = W.cube_t4(n=4)
    info = _planner(prob, tile_elems=50).plan_info()
    assert info["n_tiles"] == -(-prob.ne // 50)


def test_rejects_bad_mesh():
    X, conn = W.hex_grid((1, 1, 1), (0.01, 0.01, 0.01))
    p = tled.HostPlanner()
    bad = conn.copy()
    bad[0, 3] = 99
    with pytest.raises(tled.TledError) as e:
        p.set_mesh(8, X, bad)
    assert e.value.code == tled.E_MESH
    inv = conn[:, [4, 5, 6, 7, 0, 1, 2, 3]]  # mirrored: det J0 < 0
    with pytest.raises(tled.TledError) as e:
        p.set_mesh(8, X, inv)
    assert e.value.code == tled.E_MESH and "element 0" in str(e.value)
    with pytest.raises(tled.TledError) as e:
        p.set_mesh(5, X, conn)
    assert e.value.code == tled.E_ARG


def test_rejects_unreferenced_node():
    X, conn = W.hex_grid((1, 1, 1), (0.01, 0.01, 0.01))
    X2 = np.vstack([X, [[1.0, 1.0, 1.0]]])
    prob = W.cube_h8(n=1)
    p = tled.HostPlanner()
    p.set_mesh(8, X2, conn)
    p.set_material(tled.material_from_problem(prob))
    with pytest.raises(tled.TledError) as e:
        p.workspace_size()
    assert e.value.code == tled.E_MESH


def test_rejects_bad_material_and_params():
    prob = W.cube_h8(n=2)
    p = tled.HostPlanner()
    p.set_mesh(8, prob.X, prob.conn)
    m = tled.material_from_problem(prob)
    m.rho = float("nan")
    with pytest.raises(tled.TledError) as e:
        p.set_material(m)
    assert e.value.code == tled.E_ARG
    m = tled.material_from_problem(prob)
    m.n_prony, m.prony_g[0] = 1, 1.5
    with pytest.raises(tled.TledError):
        p.set_material(m)
    with pytest.raises(tled.TledError):
        p.set_params(mass_scale=0.5)
    with pytest.raises(tled.TledError):
        p.set_heat_sources(np.zeros((17, 10)) + 1)
    fib = np.tile([1.0, 1.0, 0.0], (prob.ne, 1))
    with pytest.raises(tled.TledError):
        p.set_material(tled.material_from_problem(prob), None, fib)


def test_call_order_errors():
    p = tled.HostPlanner()
    with pytest.raises(tled.TledError) as e:
        p.workspace_size()
    assert e.value.code == tled.E_STATE
    prob = W.cube_h8(n=2)
    p2 = _planner(prob)
    with pytest.raises(tled.TledError) as e:
        p2.init()
    assert e.value.code == tled.E_STATE


def test_batch_planning_keeps_scenarios_apart():
    """Host-only batch: tiles never span scenarios (nor element types), so the
    tile count is the sum of the per-scenario counts, and shared nodes never join
    two scenarios."""
    import ctypes as C
    probs = [W.cube_h8(n=6), W.cube_h8(n=9, seed=2), W.cube_h8(n=5, seed=3)]
    h = C.c_void_p()
    assert tled.lib().tled_batch_create(C.byref(h), -1, None) == 0
    singles = []
    for i, p in enumerate(probs):
        one = _planner(p)
        singles.append(one.plan_info())
        idx = C.c_int32()
        assert tled.lib().tled_batch_add(h, one.h, 100 * (i + 1), C.byref(idx)) == 0, tled.lib().tled_last_error(h)
        assert idx.value == i
    info = (C.c_int64 * 8)()
    assert tled.lib().tled_plan_info(h, info) == 0
    assert info[6] == 3
    assert info[0] == sum(s["n_tiles"] for s in singles)
    assert info[1] + info[2] == sum(p.nn for p in probs)
    sinfo = (C.c_int64 * 8)()
    assert tled.lib().tled_scenario_info(h, 1, sinfo) == 0
    assert (sinfo[0], sinfo[1], sinfo[2], sinfo[3], sinfo[4]) == (probs[0].nn, probs[1].nn, probs[0].ne, probs[1].ne, 200)
    assert info[5] == 8
    # a tetrahedral scenario joins the hexahedral ones: tiles hold one element type
    # each, so the count is still the per-scenario sum; the plan reports type 0 (mixed)
    t4p = W.cube_t4(n=4)
    t4 = _planner(t4p)
    n_t4 = t4.plan_info()["n_tiles"]
    assert tled.lib().tled_batch_add(h, t4.h, 10, None) == 0, tled.lib().tled_last_error(h)
    assert tled.lib().tled_plan_info(h, info) == 0
    assert info[6] == 4 and info[5] == 0
    assert info[0] == sum(s["n_tiles"] for s in singles) + n_t4
    assert info[1] + info[2] == sum(p.nn for p in probs) + t4p.nn
    tled.lib().tled_destroy(h)


def test_surrogate_spread_threshold_rule():
    """Calibration (the library's host rule, tled_sur_spread_threshold) picks
    the longest prefix (by spread) whose errors meet the tolerance at the
    requested coverage, never above the tolerance itself."""
    from paper_2009_10400_b300.surrogate import spread_threshold
    f32 = lambda v: float(np.float32(v))  # the rule works on float32 arrays
    spread = [0.1, 0.2, 0.3, 0.4, 0.5, 0.6]
    err = [0.5, 0.8, 1.5, 0.9, 2.0, 0.7]
    assert spread_threshold(spread, err, tol=1.0, coverage=1.0) == (f32(0.2), f32(2 / 6))
    assert spread_threshold(spread, err, tol=1.0, coverage=0.75) == (f32(0.4), f32(4 / 6))
    assert spread_threshold(spread, [2.0] + err[1:], tol=1.0, coverage=1.0) == (-1.0, 0.0)
    tau, frac = spread_threshold([0.5, 2.0, 3.0], [0.1, 0.1, 0.1], tol=1.0)
    assert tau == 1.0 and frac == f32(1 / 3)


def test_cem43_is_refused_in_a_batch():
    """The dose needs a per-node time step: batches refuse scenarios that ask for it."""
    import ctypes as C
    h = C.c_void_p()
    assert tled.lib().tled_batch_create(C.byref(h), -1, None) == 0
    prob = W.cube_h8(n=3)
    one = _planner(prob)
    one.set_params(flags=tled.EXPANSION | tled.COMPENSATED | tled.CEM43)
    assert tled.lib().tled_batch_add(h, one.h, 10, None) == tled.E_ARG
    tled.lib().tled_destroy(h)


def test_binding_constants_match_the_header():
    """Flag, status and mode values of the Python binding are the C header's."""
    hdr = open(os.path.join(ROOT, "include", "tled.h")).read()

    def val(name):
        m = re.search(r"#define %s \((\d+)u << (\d+)\)" % name, hdr)
        if m:
            return int(m.group(1)) << int(m.group(2))
        m = re.search(r"#define %s \(?(-?\d+)u?\)?(?:\s|/|$)" % name, hdr, re.M)
        assert m, name
        return int(m.group(1))

    for py, c in (("EXPANSION", "TLED_EXPANSION"), ("TEMP_DEP", "TLED_TEMP_DEP"), ("COMPENSATED", "TLED_COMPENSATED"),
                  ("CEM43", "TLED_CEM43"), ("GENERAL_H8", "TLED_GENERAL_H8"), ("STREAMED", "TLED_STREAMED"),
                  ("E_FORMAT", "TLED_E_FORMAT"), ("E_MESH", "TLED_E_MESH"), ("E_ARG", "TLED_E_ARG")):
        assert getattr(tled, py) == val(c), (py, c)
    assert val("TLED_MODE_RESIDENT") == 1 and val("TLED_MODE_BRICK") == 2



def test_bench_graph_launch_count():
    """A call of n steps replays the cached graphs of 32 steps and of the binary
    digits of the rest: the bench's launch count follows that decomposition."""
    import bench
    assert bench.graph_chunks(0) == 0
    assert bench.graph_chunks(1) == 1
    assert bench.graph_chunks(20) == 2     # 16 + 4
    assert bench.graph_chunks(32) == 1
    assert bench.graph_chunks(69) == 4     # 32 + 32 + 4 + 1
    assert bench.graph_chunks(500) == 15 + 2  # 15 x 32, then 20 = 16 + 4
    for n in range(1, 200):
        full, rest = divmod(n, 32)
        assert bench.graph_chunks(n) == full + bin(rest).count("1")


def test_bench_probe_points_lie_in_the_mesh():
    """On a block the bench probes a lattice inside the box; on any other mesh it
    probes element centroids (a lattice over the box would leave the mesh)."""
    import bench
    blk = W.block_h8(n=8)
    q = bench.probe_lattice(blk, 4)
    lo, hi = blk.X.min(0), blk.X.max(0)
    assert q.shape == (64, 3) and np.all(q > lo) and np.all(q < hi)
    cube = W.cube_t4(n=4)
    q = bench.probe_lattice(cube, 4)
    assert q.shape == (min(64, cube.ne), 3)
    cen = cube.X[cube.conn].mean(1)
    assert all(np.min(np.abs(cen - p).sum(1)) < 1e-12 for p in q)
