"""Pins of the oracle's SPH force and energy equations (not GPU).

The paper cites, and does not print, the momentum and energy equations; the
oracle takes the standard grad-h form with signal-velocity artificial viscosity
and conductivity.  These tests pin that reading to what mathematics fixes:
pairwise antisymmetry (total momentum), exact energy exchange, zero force on a
perfect lattice, the continuum pressure gradient, and compression heating.
"""
import math

import numpy as np

import apr_synth
import oracle


def _randomised(n_side=12, seed=7, split=True, conductivity=1.0):
    w = apr_synth.lattice_box(n_side, jitter=0.1, sphere_R=(0.3,), seed=seed)
    w["cfg"]["alpha_u"] = conductivity
    rng = np.random.default_rng(seed)
    n = len(w["p"]["x"])
    for f in ("vx", "vy", "vz"):
        w["p"][f] = rng.normal(0.0, 0.3, n)
    w["p"]["u"] = 1.0 + 0.5 * rng.uniform(size=n)
    o = oracle.Oracle(w, capacity=4 * n)
    o.density()
    if split:
        o.split_pass(0, 3)
        o.density()
    o.force()
    return o


def test_total_momentum_conserved_with_mixed_masses():
    o = _randomised()
    assert len(np.unique(o["level"])) == 2
    m = o.mass()
    for f in ("ax", "ay", "az"):
        scale = np.sum(m * np.abs(o[f]))
        assert abs(np.sum(m * o[f])) < 1e-13 * scale


def test_energy_exchange_exact():
    o = _randomised()
    m = o.mass()
    work = m * (o["vx"] * o["ax"] + o["vy"] * o["ay"] + o["vz"] * o["az"])
    heat = m * o["dudt"]
    scale = np.sum(np.abs(work)) + np.sum(np.abs(heat))
    assert abs(np.sum(work) + np.sum(heat)) < 1e-12 * scale


def test_perfect_lattice_has_no_force():
    w = apr_synth.lattice_box(12, jitter=0.0, sphere_R=())
    o = oracle.Oracle(w)
    o.density()
    o.force()
    a = np.sqrt(o["ax"] ** 2 + o["ay"] ** 2 + o["az"] ** 2)
    # the scale of one pairwise pressure term
    scale = o["pres"].max() / o["rho"].min() / o["h"].min()
    assert a.max() < 1e-11 * scale
    assert np.abs(o["dudt"]).max() < 1e-11 * scale


def test_pressure_gradient_of_a_sine_wave():
    # uniform density, u = u0 (1 + A sin 2 pi x): a_x = -(gamma-1) u0 A 2 pi cos 2 pi x
    n_side, A, u0 = 24, 0.01, 1.0
    w = apr_synth.lattice_box(n_side, jitter=0.0, sphere_R=())
    w["cfg"]["alpha_av"] = 0.0
    w["p"]["u"] = u0 * (1.0 + A * np.sin(2 * math.pi * w["p"]["x"]))
    o = oracle.Oracle(w)
    o.density()
    o.force()
    g = w["cfg"]["gamma"]
    exact = -(g - 1.0) * u0 * A * 2 * math.pi * np.cos(2 * math.pi * o["x"])
    amp = (g - 1.0) * u0 * A * 2 * math.pi
    assert np.abs(o["ax"] - exact).max() < 0.03 * amp
    assert np.abs(o["ay"]).max() < 1e-3 * amp and np.abs(o["az"]).max() < 1e-3 * amp


def test_compression_heats():
    w = apr_synth.lattice_box(12, jitter=0.0, sphere_R=())
    x = w["p"]["x"]
    w["p"]["vx"] = -0.2 * np.sin(2 * math.pi * (x - 0.5))  # converging on x = 0.5
    o = oracle.Oracle(w)
    o.density()
    o.force()
    core = np.abs(o["x"] - 0.5) < 0.15
    assert np.all(o["dudt"][core] > 0.0)
    # and viscosity on alone (no pressure work) also only heats
    w["p"]["u"] = np.zeros_like(x) + 1e-12
    o = oracle.Oracle(w)
    o.density()
    o.force()
    assert np.all(o["dudt"][core] > 0.0)
