"""The periodic sound-wave box of the paper's appendix tests on the GPU: steps
against the oracle (a small box, the circular zone active from the start), and
the two quantities the paper reports for it, the density blip at the zone and
the width of the mixed-level transition.

The paper's bound (a blip below 5% of the initial density) is asserted at 32
particles across, where the FP64 oracle meets it too (3.8%).  At the paper's 64
across neither the oracle (8.2%, or 7.3% with the children r_sep apart instead
of each r_sep from its parent) nor the GPU (about 7.4%) does; there the test
guards against regressions only, with a bound of twice the paper's."""
import numpy as np
import pytest

import apr_synth
import oracle
from gpu_util import need_gpu, sim

pytestmark = pytest.mark.gpu


def _compare_by_id(o, g, fields, tol):
    io, ig = o["id"], g.get("id")
    so, sg = np.argsort(io), np.argsort(ig)
    assert np.array_equal(io[so], ig[sg])
    for f, t in zip(fields, tol):
        a, b = g.get(f)[sg], o[f][so]
        assert np.max(np.abs(a - b) / (np.abs(b) + t[1])) < t[0], f


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_sound_wave_steps_match_oracle(precision):
    w = apr_synth.sound_wave_box(16)
    w["regions"] = list(w["regions_at"][1])
    cap = 4 * len(w["p"]["x"])
    o = oracle.Oracle(w, capacity=cap)
    g = sim(w, precision, capacity=cap)
    o.init()
    g.init()
    assert g.n == o.n and g.n > len(w["p"]["x"])
    dt = 0.5 * o.timestep()
    for _ in range(3):
        co, so = o.step(dt)
        _, sg, cg = g.step(dt)
        assert list(cg.n_split) == list(co.n_split) and list(cg.n_merge) == list(co.n_merge)
        assert g.n == o.n
        assert sg.mass == pytest.approx(so.mass, rel=1e-13)
    tol = 1e-9 if precision == "fp64" else 2e-5
    _compare_by_id(o, g, ("x", "vx", "rho", "u"), [(10 * tol, 0.01), (100 * tol, 0.01),
                                                  (10 * tol, 0.0), (10 * tol, 0.0)])


def run_wave(w, t_end, zone):
    """Steps to t_end (the zone switched on at its time); returns the final state."""
    g = sim(w, "fp32", capacity=2 * len(w["p"]["x"]))
    g.init()
    t_on, regs = w["regions_at"]
    rho0 = float(np.mean(g.get("rho")))
    t, on = 0.0, False
    while t < t_end - 1e-12:
        if zone and not on and t >= t_on - 1e-12:
            g.set_regions(regs)
            on = True
        dt = min(g.timestep(), t_end - t, (t_on - t) if (zone and not on) else 1e9)
        g.step(dt)
        t += dt
    return g, rho0


def test_sound_wave_blip_at_32_across_within_the_paper_bound():
    need_gpu()
    w = apr_synth.sound_wave_box(32)
    ref, rho_ic = run_wave(w, 2.0, zone=False)
    apr, _ = run_wave(w, 2.0, zone=True)
    assert apr.n > ref.n
    _, pr = apr_synth.wave_profile(ref.get("x"), ref.get("y"), ref.get("rho"), w["Ly"], nbins=32)
    _, pa = apr_synth.wave_profile(apr.get("x"), apr.get("y"), apr.get("rho"), w["Ly"], nbins=32)
    assert np.max(np.abs(pa - pr)) / rho_ic < 0.05


@pytest.mark.slow
def test_sound_wave_blip_and_transition_width():
    need_gpu()
    w = apr_synth.sound_wave_box()
    ref, rho_ic = run_wave(w, 2.0, zone=False)
    apr, _ = run_wave(w, 2.0, zone=True)
    assert apr.n > ref.n  # the zone holds split particles
    _, pr = apr_synth.wave_profile(ref.get("x"), ref.get("y"), ref.get("rho"), w["Ly"])
    _, pa = apr_synth.wave_profile(apr.get("x"), apr.get("y"), apr.get("rho"), w["Ly"])
    blip = np.max(np.abs(pa - pr)) / rho_ic
    assert blip < 0.10  # regression guard: twice the paper's bound (see above)
    fuzz = apr_synth.zone_fuzz(apr.get("x"), apr.get("y"), apr.get("level"), apr.get("h"))
    assert fuzz < 0.5
    # away from the zone the wave is that of the run without it
    xs = (np.arange(64) + 0.5) / 64
    far = np.abs(xs - 0.5) > 0.2
    basis = np.stack([np.ones(far.sum()), np.sin(2 * np.pi * xs[far])], 1)
    cr = np.linalg.lstsq(basis, pr[far] / rho_ic, rcond=None)[0]
    ca = np.linalg.lstsq(basis, pa[far] / rho_ic, rcond=None)[0]
    assert abs(ca[1] - cr[1]) < 0.003
