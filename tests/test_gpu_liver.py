"""The paper's liver heating case (uniform spherical sources, temperature-
dependent c and k, metabolic heat, perfusion) with the CEM43 dose and the
isotherm read-out, against the oracle."""
import numpy as np
import pytest

import oracle
from helpers import TOL_DAMAGE, TOL_E, compare, rel_l2
from paper_2009_10400_b300 import workloads as W

pytestmark = pytest.mark.gpu


def test_liver_f2_matches_oracle_with_cem43_and_isotherm():
    from paper_2009_10400_b300 import tled
    p = W.liver_f2()
    for r in p.sources:  # which nodes the spheres heat is unambiguous (margin from the generator)
        assert r[10] == 1.0
        assert np.min(np.abs(np.linalg.norm(p.X - r[:3], axis=1) - r[6])) > 2e-5
    m = oracle.OracleModel(p)
    s = m.init_state()
    g = tled.Solver.from_problem(p)
    assert g.get_dt()[0] == pytest.approx(m.dt, rel=1e-12)
    for k in range(2):
        m.step(s, 1000)
        g.step(1000)
        g.sync()
        c = compare(g.displacement(), g.temperature(), g.damage(), s.u, s.T, s.Omega, p.T0)
        assert c["e_u"] <= TOL_E and c["e_theta"] <= TOL_E and c["d_abs"] <= TOL_DAMAGE, (k, c)
        cem = g.cem43()
        assert rel_l2(cem, s.cem) <= 1e-5, rel_l2(cem, s.cem)
    T = g.temperature()
    assert (T - p.T0).max() > 0.2  # the spheres heated (0.137 s of heating)
    T_iso = float(np.quantile(T, 0.95))
    vol = g.isotherm_volume(T_iso)
    np.testing.assert_allclose(vol, m.Vn[T >= T_iso].sum(), rtol=1e-6)  # definition, on the GPU's own field
    assert 0 < vol < m.Vn.sum()


def test_cem43_survives_checkpoint_bitwise():
    from paper_2009_10400_b300 import tled
    p = W.liver_f2()
    g = tled.Solver.from_problem(p)
    g.step(200)
    blob = g.save_state()
    g.step(300)
    ref = g.cem43()
    g.load_state(blob)
    g.step(300)
    np.testing.assert_array_equal(g.cem43(), ref)
