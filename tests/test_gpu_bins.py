"""Individual time steps in bins (Sec. 2.5) on the GPU: one bin is the global
step bit for bit, with and without point masses; with several bins the bins,
the split/merge/accretion counts and the number of force updates equal the
oracle's (FP64), and the fields agree within 1e-8 relative."""
import numpy as np
import pytest

import apr_synth
import oracle
from gpu_util import sim

pytestmark = pytest.mark.gpu


def _by_id(o, g, f):
    so, sg = np.argsort(o["id"]), np.argsort(g.get("id"))
    return o[f][so], g.get(f)[sg]


def test_one_bin_is_the_global_step_on_the_gpu():
    w = apr_synth.sod(8)
    cap = 4 * len(w["p"]["x"])
    a = sim(w, "fp64", capacity=cap)
    b = sim(w, "fp64", capacity=cap)
    a.init()
    b.init()
    dt = 0.5 * a.timestep()
    for _ in range(2):
        _, _, ca = a.step(dt)
        cb, upd, sat, _ = b.step_bins(dt, 0, init_bins=True)
        assert upd == b.n and sat == 0
        assert list(ca.n_split) == list(cb.n_split) and list(ca.n_merge) == list(cb.n_merge)
    for f in ("x", "vx", "u", "rho", "h", "level", "id"):
        assert np.array_equal(a.get(f), b.get(f)), f


@pytest.mark.parametrize("B", [2, 3])
def test_bins_match_oracle(B):
    w = apr_synth.sod(8)
    cap = 4 * len(w["p"]["x"])
    o = oracle.Oracle(w, capacity=cap)
    g = sim(w, "fp64", capacity=cap)
    o.init()
    g.init()
    # not a power of two times the smallest limit: no particle sits on a bin boundary
    dt_max = 1.37 * 2 ** (B - 1) * o.timestep()
    for first in (True, False):
        co, uo, so = o.step_bins(dt_max, B, init_bins=first)
        cg, ug, sg, _ = g.step_bins(dt_max, B, init_bins=first)
        assert (ug, sg) == (uo, so)
        assert list(cg.n_split) == list(co.n_split) and list(cg.n_merge) == list(co.n_merge)
        assert g.n == o.n
        bo, bg = _by_id(o, g, "bin")
        assert np.array_equal(bo, bg)
    assert len(np.unique(g.get("bin"))) >= 2 and ug < (1 << B) * g.n
    h, _ = _by_id(o, g, "h")
    for f, floor in (("x", 0.01), ("vx", 0.05), ("rho", 0.0), ("u", 0.0)):
        a, b = _by_id(o, g, f)
        assert np.max(np.abs(a - b) / (np.abs(a) + floor)) < 1e-8, f


def test_bins_fp32_close_to_fp64():
    w = apr_synth.sod(8)
    cap = 4 * len(w["p"]["x"])
    g64 = sim(w, "fp64", capacity=cap)
    g32 = sim(w, "fp32", capacity=cap)
    g64.init()
    g32.init()
    dt_max = 2 * g64.timestep()
    _, u64, _, s64 = g64.step_bins(dt_max, 2, init_bins=True)
    _, u32, _, s32 = g32.step_bins(dt_max, 2, init_bins=True)
    assert s32.mass == pytest.approx(s64.mass, rel=1e-13)
    if g32.n == g64.n and u32 == u64:
        a, b = g64.get("x"), g32.get("x")
        assert np.abs(a - b).max() < 1e-4 * g64.get("h").min()


def _disc(n=2000, racc_star=1.02, zone=True):
    # the inner edge of the disc (R = 1) falls inside a star radius of 1.02
    w = apr_synth.disc_planet(n)
    w["sinks"][0]["racc"] = racc_star
    if not zone:
        w["regions"] = []
    return w, 4 * n


def test_one_bin_is_the_global_step_with_point_masses_on_the_gpu():
    w, cap = _disc()
    a = sim(w, "fp64", capacity=cap)
    b = sim(w, "fp64", capacity=cap)
    a.init()
    b.init()
    dt = 0.5 * a.timestep()
    acc = 0
    for _ in range(3):
        _, _, ca = a.step(dt)
        cb, upd, _, _ = b.step_bins(dt, 0, init_bins=True)
        assert upd == b.n and ca.n_accreted == cb.n_accreted
        assert list(ca.n_split) == list(cb.n_split) and list(ca.n_merge) == list(cb.n_merge)
        acc += cb.n_accreted
    assert acc > 0
    for f in ("x", "vx", "rho", "h", "ax", "level", "id"):
        assert np.array_equal(a.get(f), b.get(f)), f
    assert a.sinks() == b.sinks()


@pytest.mark.parametrize("zone", [False, True])
def test_bins_with_point_masses_match_oracle(zone):
    w, cap = _disc(zone=zone)
    o = oracle.Oracle(w, capacity=cap)
    g = sim(w, "fp64", capacity=cap)
    o.init()
    g.init()
    B = 3
    dt_max = 1.37 * 2 ** (B - 1) * o.timestep()
    acc = 0
    for first in (True, False):
        co, uo, so = o.step_bins(dt_max, B, init_bins=first)
        cg, ug, sg, _ = g.step_bins(dt_max, B, init_bins=first)
        assert (ug, sg) == (uo, so)
        assert list(cg.n_split) == list(co.n_split) and list(cg.n_merge) == list(co.n_merge)
        assert cg.n_accreted == co.n_accreted
        acc += cg.n_accreted
        assert g.n == o.n
        bo, bg = _by_id(o, g, "bin")
        assert np.array_equal(bo, bg)
    assert acc > 0 and len(np.unique(g.get("bin"))) >= 3
    for f, floor in (("x", 0.01), ("vx", 0.05), ("rho", 0.0), ("ax", 0.01)):
        a, b = _by_id(o, g, f)
        assert np.max(np.abs(a - b) / (np.abs(a) + floor)) < 1e-8, f
    for ko, kg in zip(o.sinks_state(), g.sinks()):
        assert np.allclose(ko["x"], kg["x"], rtol=0, atol=1e-10)
        assert np.allclose(ko["v"], kg["v"], rtol=0, atol=1e-10)
        assert ko["m"] == pytest.approx(kg["m"], rel=1e-14)


def test_bins_with_point_masses_conserve_mass_fp32():
    w, cap = _disc()
    g = sim(w, "fp32", capacity=cap)
    g.init()
    m0 = g.stats().mass
    acc = 0
    for first in (True, False):
        c, _, _, st = g.step_bins(8 * g.timestep(), 3, init_bins=first)
        acc += c.n_accreted
    assert acc > 0 and st.mass == pytest.approx(m0, rel=1e-14)
