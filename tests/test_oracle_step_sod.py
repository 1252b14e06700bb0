"""Pins of the oracle's time stepping, point masses and the Sod shock tube (not GPU)."""
import math

import numpy as np
import pytest

import apr_synth
import oracle
from conftest import read_golden
from oracle import riemann

SOD = dict(rhoL=1.0, uL=0.0, pL=1.0, rhoR=0.125, uR=0.0, pR=0.1, g=1.4)


def test_exact_riemann_star_state_textbook():
    gold = {r[0]: float(r[1]) for r in read_golden("sod_star_state.txt")}
    p, u = riemann.star_state(1.0, 0.0, 1.0, 0.125, 0.0, 0.1, 1.4)
    assert round(p, 5) == gold["p_star"] and round(u, 5) == gold["u_star"]
    # densities either side of the contact, sampled just left/right of u*
    rl, _, _ = riemann.sample([u - 1e-9], *SOD.values())
    rr, _, _ = riemann.sample([u + 1e-9], *SOD.values())
    assert round(rl[0], 5) == gold["rho_star_L"] and round(rr[0], 5) == gold["rho_star_R"]


def test_exact_solution_conserves_mass_momentum_energy():
    t = 0.2
    x = np.linspace(-0.5, 0.5, 400001)
    r, u, p = riemann.sample(x / t, *SOD.values())
    dx = x[1] - x[0]
    mass0 = 0.5 * 1.0 + 0.5 * 0.125
    e0 = 0.5 * 1.0 / 0.4 + 0.5 * 0.1 / 0.4
    assert abs(np.sum(r) * dx - mass0) < 1e-4
    # momentum grows by the pressure difference at the two ends: (pL - pR) t
    assert abs(np.sum(r * u) * dx - (1.0 - 0.1) * t) < 1e-4
    assert abs(np.sum(p / 0.4 + 0.5 * r * u * u) * dx - e0) < 1e-4


def _run_sod(nL, slab, tend):
    w = apr_synth.sod(nL, slab=slab)
    o = oracle.Oracle(w, capacity=4 * len(w["p"]["x"]))
    o.init()
    t = 0.0
    m0 = o.stats().mass
    while t < tend - 1e-12:
        dt = min(o.timestep(), tend - t)
        o.step(dt)
        t += dt
    return o, t, m0


def _l1(o, t):
    x = o["x"]
    sel = np.abs(x) < 0.4
    r, u, p = riemann.sample(x[sel] / t, *SOD.values())
    return (np.mean(np.abs(o["rho"][sel] - r)), np.mean(np.abs(o["vx"][sel] - u)),
            np.mean(np.abs(o["pres"][sel] - p)))


def test_sod_tube_matches_closed_form():
    o, t, m0 = _run_sod(12, (), 0.2)
    l1r, l1v, l1p = _l1(o, t)
    assert l1r < 0.025 and l1v < 0.045 and l1p < 0.02
    # the star state between the rarefaction tail and the shock
    gold = {r[0]: float(r[1]) for r in read_golden("sod_star_state.txt")}
    x = o["x"]
    left_star = (x > 0.0) & (x < 0.1)
    right_star = (x > 0.22) & (x < 0.3)
    assert abs(o["pres"][left_star].mean() / gold["p_star"] - 1) < 0.03
    assert abs(o["pres"][right_star].mean() / gold["p_star"] - 1) < 0.03
    assert abs(o["vx"][left_star].mean() / gold["u_star"] - 1) < 0.03
    assert abs(o["rho"][left_star].mean() / gold["rho_star_L"] - 1) < 0.03
    assert abs(o["rho"][right_star].mean() / gold["rho_star_R"] - 1) < 0.03
    # the shock front: rightmost moving particle with rho above the mid value behind it
    p, u = riemann.star_state(1.0, 0.0, 1.0, 0.125, 0.0, 0.1, 1.4)
    aR = math.sqrt(1.4 * 0.1 / 0.125)
    S = aR * math.sqrt(2.4 / 2.8 * p / 0.1 + 0.4 / 2.8)
    rho2 = riemann.sample([S - 1e-9], *SOD.values())[0][0]
    mid = 0.5 * (rho2 + 0.125)
    x = o["x"]
    free = (o["flags"] & oracle.FLAG_FIXED) == 0
    xs = x[free & (o["rho"] > mid) & (x > 0.1)].max()
    assert abs(xs - S * t) < 0.03
    assert o.stats().mass == pytest.approx(m0, rel=1e-14)


@pytest.mark.slow
def test_sod_tube_with_two_level_slab():
    o, t, m0 = _run_sod(12, (0.15, 0.10), 0.2)
    l1r, l1v, l1p = _l1(o, t)
    assert l1r < 0.025 and l1v < 0.045 and l1p < 0.02
    assert o.stats().mass == pytest.approx(m0, rel=1e-14)
    lev = o["level"]
    assert lev.max() == 2 and np.sum(lev == 2) > 1000
    # outside the slab only level-0 particles and at most a thin fuzzy boundary remain
    far = np.abs(o["x"]) > 0.2
    assert np.mean(lev[far] > 0) < 0.05


def _periodic_box(seed=3):
    w = apr_synth.lattice_box(10, jitter=0.1, sphere_R=(0.3,), seed=seed)
    rng = np.random.default_rng(seed)
    n = len(w["p"]["x"])
    for f in ("vx", "vy", "vz"):
        w["p"][f] = rng.normal(0, 0.2, n)
    w["cfg"]["alpha_u"] = 1.0
    return w


def test_step_conserves_mass_momentum_and_energy():
    w = _periodic_box()
    o = oracle.Oracle(w, capacity=8000)
    o.init()
    s0 = o.stats()
    e0 = s0.ekin + s0.etherm
    dt = 0.2 * o.timestep()
    for _ in range(6):
        cnt, s = o.step(dt)
    assert s.mass == pytest.approx(s0.mass, rel=1e-14)
    scale = s0.mass * 0.2
    for k in range(3):
        assert abs(s.mom[k] - s0.mom[k]) < 1e-13 * scale
    assert abs(s.ekin + s.etherm - e0) < 2e-4 * e0


def test_two_body_orbit_and_accretion():
    w = apr_synth.lattice_box(2, jitter=0.0, sphere_R=())
    w["p"] = {k: v[:0] for k, v in w["p"].items()}
    w["cfg"]["periodic"] = [0, 0, 0]
    w["cfg"]["box_lo"] = [-4.0] * 3
    w["cfg"]["box_hi"] = [4.0] * 3
    w["cfg"]["delta"] = 2.0 ** -27
    mp = 1e-3
    vrel = math.sqrt(1.0 + mp)  # circular relative orbit of radius 1 about the centre of mass
    w["sinks"] = [dict(x=[-mp / (1 + mp), 0, 0], v=[0, -vrel * mp / (1 + mp), 0], m=1.0, racc=0.1),
                  dict(x=[1 / (1 + mp), 0, 0], v=[0, vrel / (1 + mp), 0], m=mp, racc=0.05)]
    o = oracle.Oracle(w, capacity=16)
    o.init()
    s0 = o.stats()

    def energy(ss):
        a, b = ss
        r = np.linalg.norm(np.array(a["x"]) - np.array(b["x"]))
        ke = sum(0.5 * s["m"] * np.dot(s["v"], s["v"]) for s in ss)
        return ke - a["m"] * b["m"] / r

    E0 = energy(o.sinks_state())
    nstep = 2000
    dt = 2 * math.pi / math.sqrt(1 + mp) / nstep
    for _ in range(nstep):
        o.step(dt)
    ss = o.sinks_state()
    assert abs(energy(ss) / E0 - 1) < 1e-5
    assert np.linalg.norm(np.array(ss[1]["x"]) - [1 / (1 + mp), 0, 0]) < 1e-3
    s1 = o.stats()
    for k in range(3):
        assert abs(s1.mom[k] - s0.mom[k]) < 1e-15


def test_accretion_conserves_mass_and_momentum():
    w = _periodic_box()
    w["cfg"]["periodic"] = [0, 0, 0]
    w["cfg"]["box_lo"] = [-1.0] * 3
    w["cfg"]["box_hi"] = [2.0] * 3
    w["cfg"]["delta"] = 2.0 ** -28
    w["regions"] = []
    w["sinks"] = [dict(x=[0.5, 0.5, 0.5], v=[0.1, 0, 0], m=0.01, racc=0.15)]
    o = oracle.Oracle(w, capacity=4000)
    s0 = o.stats()
    p = np.stack([o["x"], o["y"], o["z"]], 1)
    inside = int(np.sum(np.linalg.norm(p - 0.5, axis=1) < 0.15))
    na = o.accrete()
    assert na == inside > 0
    o.compact()
    s1 = o.stats()
    assert s1.mass == pytest.approx(s0.mass, rel=1e-15)
    for k in range(3):
        assert s1.mom[k] == pytest.approx(s0.mom[k], rel=1e-12, abs=1e-16)
    assert o.sinks_state()[0]["m"] == pytest.approx(0.01 + inside * w["cfg"]["m0"], rel=1e-14)
