"""GPU steps of the whole hot path against the oracle: initial refinement and
kick-drift-kick steps on a shock tube with a two-level slab and on a disc with
a planet; conservation on the GPU; sampled checks at the full shock-tube size."""
import numpy as np
import pytest

import apr_synth
import oracle
from gpu_util import rel, sim, with_velocities

pytestmark = pytest.mark.gpu


def _compare_by_id(o, g, fields, tol):
    io, ig = o["id"], g.get("id")
    so, sg = np.argsort(io), np.argsort(ig)
    assert np.array_equal(io[so], ig[sg])
    for f, t in zip(fields, tol):
        a, b = g.get(f)[sg], o[f][so]
        assert np.max(np.abs(a - b) / (np.abs(b) + t[1])) < t[0], f


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_sod_init_and_steps(precision):
    w = apr_synth.sod(12)
    cap = 4 * len(w["p"]["x"])
    o = oracle.Oracle(w, capacity=cap)
    g = sim(w, precision, capacity=cap)
    po, pg = o.init(), g.init()
    assert g.n == o.n and po == pg
    assert np.array_equal(np.bincount(g.get("level")), np.bincount(o["level"]))
    tol = 1e-9 if precision == "fp64" else 2e-5
    _compare_by_id(o, g, ("x", "rho", "h"), [(tol, 0.0)] * 3)
    dt = 0.5 * o.timestep()
    for k in range(3):
        co, so = o.step(dt)
        _, sg, cg = g.step(dt)
        assert list(cg.n_split) == list(co.n_split) and list(cg.n_merge) == list(co.n_merge)
        assert g.n == o.n
        assert sg.mass == pytest.approx(so.mass, rel=1e-13)
    _compare_by_id(o, g, ("x", "vx", "rho", "u"), [(10 * tol, 0.01), (100 * tol, 0.05),
                                                  (10 * tol, 0.0), (10 * tol, 0.0)])


def test_disc_planet_steps_with_accretion():
    w = apr_synth.disc_planet(20000)
    cap = 4 * 20000
    o = oracle.Oracle(w, capacity=cap)
    g = sim(w, "fp64", capacity=cap)
    o.init()
    g.init()
    assert g.n == o.n
    dt = 0.02
    for _ in range(2):
        co, so = o.step(dt)
        _, sg, cg = g.step(dt)
        assert cg.n_accreted == co.n_accreted
        assert g.n == o.n
        assert sg.mass == pytest.approx(so.mass, rel=1e-13)
        for k in range(3):
            assert sg.mom[k] == pytest.approx(so.mom[k], rel=1e-9, abs=1e-15)
    ks, kg = o.sinks_state(), g.sinks()
    for a, b in zip(ks, kg):
        assert np.allclose(a["x"], b["x"], rtol=1e-12, atol=1e-14)
        assert a["m"] == pytest.approx(b["m"], rel=1e-14)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("which", ["sod", "disc"])
def test_timestep_matches_oracle(precision, which):
    """apr_timestep against the oracle's orc_timestep after the initial refinement
    and after one step.  dt = min(0.3 h / v_sig, 0.25 sqrt(h / |a|)), so its relative
    error is at most that of h plus v_sig, or half that of h plus |a|: the FP64 path
    keeps 1e-9, the FP32-mixed path 1e-4 (its force tolerance)."""
    w = apr_synth.sod(12) if which == "sod" else apr_synth.disc_planet(20000)
    cap = 4 * len(w["p"]["x"])
    o = oracle.Oracle(w, capacity=cap)
    g = sim(w, precision, capacity=cap)
    o.init()
    g.init()
    assert g.n == o.n
    tol = 1e-9 if precision == "fp64" else 1e-4
    dt = o.timestep()
    assert np.isfinite(dt) and dt > 0
    assert g.timestep() == pytest.approx(dt, rel=tol)
    o.step(0.5 * dt)
    g.step(0.5 * dt)
    assert g.n == o.n
    assert g.timestep() == pytest.approx(o.timestep(), rel=tol)


def test_init_takes_the_zones():
    """apr_init with the zones passed in (the boundary's form) gives the same state
    as apr_set_regions followed by apr_init without zones."""
    w = apr_synth.c1_lattice()
    a = sim(w, "fp64", capacity=3 * 4096)
    b = sim(w, "fp64", capacity=3 * 4096)
    b.set_regions([])
    pa = a.init()
    pb = b.init(w["regions"])
    assert pa == pb and a.n == b.n > 4096
    for f in ("x", "h", "rho", "ax", "level", "id"):
        assert np.array_equal(a.get(f), b.get(f)), f


def test_gpu_step_conserves_mass_and_momentum_fp32():
    w = with_velocities(apr_synth.lattice_box(12, 0.1, sphere_R=(0.3,), seed=4), 0.2)
    w["cfg"]["alpha_u"] = 1.0
    g = sim(w, "fp32", capacity=8 * 12 ** 3)
    g.init()
    s0 = g.stats()
    dt = 0.2 * g.timestep()
    for _ in range(5):
        _, s, _ = g.step(dt)
    assert s.mass == pytest.approx(s0.mass, rel=1e-14)
    scale = s0.mass * 0.2
    for k in range(3):
        assert abs(s.mom[k] - s0.mom[k]) < 1e-6 * scale
    assert abs((s.ekin + s.etherm) / (s0.ekin + s0.etherm) - 1) < 1e-3


@pytest.mark.slow
def test_full_size_sod_sampled():
    """The full 123,480-particle tube after the initial refinement (the bench's
    state): density and force of sampled particles against the oracle."""
    w = apr_synth.c2_sod()
    cap = 3 * len(w["p"]["x"])
    g = sim(w, "fp32", capacity=cap)
    g.init()
    o = oracle.Oracle(w, capacity=cap)
    o.init()
    assert g.n == o.n
    io, ig = o["id"], g.get("id")
    so, sg = np.argsort(io), np.argsort(ig)
    assert np.array_equal(io[so], ig[sg])
    rng = np.random.default_rng(0)
    pick = rng.choice(o.n, 300, replace=False)
    a_o, a_g = so[pick], sg[pick]
    assert rel(g.get("rho")[a_g], o["rho"][a_o]).max() < 2e-5
    scale = o["pres"][a_o] / (o["rho"][a_o] * o["h"][a_o])
    err = np.abs(g.get("ax")[a_g] - o["ax"][a_o]) / (np.abs(o["ax"][a_o]) + scale)
    assert err.max() < 2e-4


@pytest.mark.parametrize("pinned", ["pinned", "pageable", "mixed"])
def test_host_exchange_round_trip_and_step(pinned):
    """apr_download / apr_upload: the state survives a round trip through host
    buffers, and a step taken after an upload equals the device-resident one bit
    for bit (with the same step length).  Page-locked host arrays move in one
    kernel, pageable ones by copy calls, and a call may mix the two."""
    import paper_2409_11470_gb300.binding as B
    w = apr_synth.sod(8)
    cap = 4 * len(w["p"]["x"])
    a = sim(w, "fp32", capacity=cap)
    b = sim(w, "fp32", capacity=cap)
    a.init()
    b.init()
    host = b.host_buffers(pinned=pinned != "pageable")
    if pinned == "mixed":
        for f in ("x", "level", "id"):
            host[f] = host[f].clone()  # pageable copies of a few fields
            assert not host[f].is_pinned()
    n = b.download(host)
    assert n == b.n
    for f in ("x", "vx", "h", "rho", "ax", "level", "flags", "id"):
        assert np.array_equal(host[f][:n].numpy().view(b.get(f).dtype), b.get(f)), f
    for _ in range(2):
        dt = a.timestep()
        assert b.timestep() == dt
        b.upload(host, b.n)
        a.step(dt)
        b.step(dt)
        n = b.download(host)
        assert n == a.n
        for f in ("x", "vx", "u", "rho", "h", "ax", "id"):
            assert np.array_equal(a.get(f), b.get(f)), f
    small = {f: t[:3] for f, t in host.items()}
    with pytest.raises(B.AprError) as e:
        b.download(small)
    assert e.value.status == 2
    with pytest.raises(B.AprError) as e:
        b.upload(host, cap + 1)
    assert e.value.status == 1
