"""GPU relaxing (Sec. 2.4) against the oracle: the particles a split
introduced are shuffled towards the reference set (the particles before the
split) with the same step, cap and stopping rule; positions agree within
1e-8 h (FP64) / 1e-4 h (FP32) after three shuffles."""
import numpy as np
import pytest

import apr_synth
import oracle
from gpu_util import sim

pytestmark = pytest.mark.gpu


def _both(precision, make=apr_synth.c1_lattice):
    w = make()
    n = len(w["p"]["x"])
    cap = 4 * n
    o = oracle.Oracle(w, capacity=cap)
    o.density_force()
    ref_o = o.copy()
    g = sim(w, precision, capacity=cap)
    g.density()
    g.force()
    ref_g = g.snapshot()
    o.init()
    g.init()
    assert g.n == o.n
    return o, ref_o, g, ref_g


def _by_id(o, g, f):
    so, sg = np.argsort(o["id"]), np.argsort(g.get("id"))
    return o[f][so], g.get(f)[sg]


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_relax_matches_oracle(precision):
    o, ref_o, g, ref_g = _both(precision)
    new = int(np.count_nonzero(g.get("flags") & apr_synth.FLAG_NEW))
    assert new == int(np.count_nonzero(o["flags"] & oracle.FLAG_NEW)) > 400
    it_o, r_o = o.relax(ref_o, 3, 0.0)
    it_g, r_g = g.relax(ref_g, 3, 0.0)
    assert it_o == it_g == 3
    assert r_g == pytest.approx(r_o, rel=1e-6 if precision == "fp64" else 2e-2)
    h, _ = _by_id(o, g, "h")
    tol = 1e-8 if precision == "fp64" else 1e-4
    for f in ("x", "y", "z"):
        a, b = _by_id(o, g, f)
        d = a - b
        d -= np.round(d)  # periodic unit box
        assert np.abs(d).max() < tol * h.min(), f
    assert not np.any(g.get("flags") & apr_synth.FLAG_NEW)
    ro, rg = _by_id(o, g, "rho")
    assert np.abs(rg / ro - 1.0).max() < (1e-10 if precision == "fp64" else 2e-5)


def test_relax_stopping_rule_and_capacity():
    o, ref_o, g, ref_g = _both("fp64")
    it_o, r_o = o.relax(ref_o, 50, 0.8)
    it_g, r_g = g.relax(ref_g, 50, 0.8)
    assert it_g == it_o < 50 and r_g <= 0.8
    # the reference set must fit in the spare capacity
    import paper_2409_11470_gb300.binding as B
    w = apr_synth.c1_lattice()
    small = sim(w, "fp64", capacity=len(w["p"]["x"]) + 10)
    small.density()
    small.force()
    ref = small.snapshot()
    with pytest.raises(B.AprError) as e:
        small.relax(ref, 1, 0.0)
    assert e.value.status == 2
