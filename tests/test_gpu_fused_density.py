"""The first density pass fused into the list build (FP32-mixed): it evaluates
the density kernel's terms in the same order, so whole steps with it
(``fused_density`` 1) give the same bits as steps whose every pass runs in the
density kernel (the default), on workloads with density retries, list overflow into
the per-particle walks, periodic boxes, mixed masses and the Wendland kernel."""
import copy

import numpy as np
import pytest

import apr_synth
from gpu_util import sim

pytestmark = pytest.mark.gpu

FIELDS = ("x", "y", "z", "vx", "vy", "vz", "u", "h", "rho", "omega", "ax", "ay", "az", "dudt",
          "vsig", "dnn", "pres", "cs", "level", "flags")


def _by_id(g):
    ids = g.get("id")
    o = np.argsort(ids)
    return ids[o], {f: g.get(f)[o] for f in FIELDS}


def _workloads():
    return [
        ("sod", apr_synth.sod(12), 4, 0, 0.0),
        ("disc", apr_synth.disc_planet(20000), 4, 2048, 0.02),
        ("wendland", apr_synth.wendland_lattice(16), 3, 0, 0.0),
        ("flyby", apr_synth.flyby(60000), 2, 2048, 0.0),
    ]


@pytest.mark.parametrize("idx", range(4), ids=["sod", "disc", "wendland", "flyby"])
def test_fused_first_pass_bit_identical(idx):
    name, w, capf, mn, dt = _workloads()[idx]
    n0 = len(w["p"]["x"])
    runs = []
    for fused in (1, 0):
        wc = copy.deepcopy(w)
        wc["cfg"]["fused_density"] = fused
        g = sim(wc, "fp32", capacity=capf * n0 + 1024, max_neigh=mn)
        g.init()
        g.profile_enable(True)
        for _ in range(2):
            g.step(dt)
        runs.append((_by_id(g), g.profile(), g.n))
        g.close()
    (ia, fa), pa, na = runs[0]
    (ib, fb), pb, nb = runs[1]
    assert na == nb
    assert np.array_equal(ia, ib)
    for f in FIELDS:
        assert np.array_equal(fa[f].view(np.uint8), fb[f].view(np.uint8)), (name, f)
    # the same retries in both
    assert pa["uncovered"] == pb["uncovered"]
    assert pa["density_attempts"] == pb["density_attempts"]
