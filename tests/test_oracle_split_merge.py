"""Pins of the oracle's refinement rules (not GPU): Eq. 1 masses, the split of
Sec. 2.2 (Eq. 2), the pairing tree and merge of Sec. 2.3 (Eq. 3, Eq. 4), the
per-step order of Sec. 2.6, and the zone levels of Sec. 2.1 / Table 1."""
import math

import numpy as np
import pytest
from scipy import stats as sstats

import apr_synth
import oracle
from conftest import read_golden


# ----------------------------------------------------------------- levels ---

def test_eq1_mass_per_level():
    rows = [r for r in read_golden("mass_levels.txt") if r[0] != "E"]
    w = apr_synth.lattice_box(4, jitter=0.0, sphere_R=())
    o = oracle.Oracle(w)
    m0 = w["cfg"]["m0"]
    for lev, ratio in rows:
        o.a["level"][: o.n] = int(lev)
        assert o.stats().mass == pytest.approx(o.n * m0 * float(ratio), rel=1e-15)


def test_region_levels_hand_table():
    for r in read_golden("region_levels.txt"):
        shape, cx, cy, cz, radii, px, py, pz, lev = r
        region = dict(shape=0 if shape == "S" else 1, axis=0, track_sink=-1,
                      centre=[float(cx), float(cy), float(cz)],
                      R=[float(v) for v in radii.split(",")])
        w = apr_synth.lattice_box(2, jitter=0.0, sphere_R=())
        w["regions"] = [region]
        w["cfg"]["lmax"] = 8
        o = oracle.Oracle(w)
        got = o.target_levels([float(px)], [float(py)], [float(pz)])[0]
        assert got == int(lev), r


def test_levels_take_max_over_regions_and_track_sinks():
    w = apr_synth.lattice_box(2, jitter=0.0, sphere_R=())
    w["cfg"]["lmax"] = 3
    w["regions"] = [dict(shape=0, axis=0, track_sink=-1, centre=[0, 0, 0], R=[1.0]),
                    dict(shape=0, axis=0, track_sink=0, centre=[9, 9, 9], R=[1.0, 0.5])]
    w["sinks"] = [dict(x=[0.2, 0.0, 0.0], v=[0, 0, 0], m=1.0, racc=0.01)]
    o = oracle.Oracle(w)
    assert list(o.target_levels([0.0, 0.6], [0.0, 0.0], [0.0, 0.0])) == [1, 1]
    o.track_regions()
    assert list(o.target_levels([0.0, 0.8, 1.5], [0.0, 0.0, 0.0], [0.0, 0.0, 0.0])) == [2, 1, 0]


# ------------------------------------------------------------------ split ---

def test_splitmix64_published_sequence():
    gamma = 0x9E3779B97F4A7C15
    for k, hexv in read_golden("splitmix64.txt"):
        assert oracle.splitmix64(((int(k) - 1) * gamma) % 2 ** 64) == int(hexv, 16)


def test_split_random_number_uniform():
    t = np.array([oracle.split_uniform(20240917, i, 5) for i in range(20000)])
    assert t.min() >= -1.0 and t.max() < 1.0
    assert sstats.kstest((t + 1) / 2, "uniform").pvalue > 1e-3
    assert oracle.split_uniform(1, 2, 3) == oracle.split_uniform(1, 2, 3)
    assert oracle.split_uniform(1, 2, 3) != oracle.split_uniform(1, 2, 4)


def test_split_direction_tangential_and_rotated():
    rng = np.random.default_rng(3)
    sphere = dict(shape=0, axis=0, track_sink=-1, centre=[0.5, 0.5, 0.5], R=[0.3])
    slab = dict(shape=1, axis=0, track_sink=-1, centre=[0.0, 0.0, 0.0], R=[0.1])
    for _ in range(200):
        p = rng.uniform(0, 1, 3)
        t = rng.uniform(-1, 1)
        w = oracle.split_direction(sphere, p, t)
        v = (p - 0.5) / np.linalg.norm(p - 0.5)
        assert abs(np.linalg.norm(w) - 1) < 1e-14 and abs(w @ v) < 1e-14
        ws = oracle.split_direction(slab, p, t)
        assert abs(np.linalg.norm(ws) - 1) < 1e-14 and ws[0] == 0.0
    # the angle is 2 atan(t) about v, measured from the same in-plane axis
    p = np.array([0.9, 0.5, 0.5])  # v = +x, least aligned axis y, w1 = x cross y = +z
    for t in (-0.9, -0.3, 0.0, 0.4, 0.99):
        w = oracle.split_direction(sphere, p, t)
        ang = math.atan2(w[1] * -1.0, w[2])  # w2 = v x w1 = x cross z = -y
        assert abs(ang - 2 * math.atan(t)) < 1e-14


def _c1_after_density(seed=11):
    w = apr_synth.c1_lattice()
    rng = np.random.default_rng(seed)
    for f in ("vx", "vy", "vz"):
        w["p"][f] = rng.normal(0, 1, 4096)
    o = oracle.Oracle(w, capacity=3 * 4096)
    o.density()
    return o


def test_split_pass_geometry_and_conservation():
    o = _c1_after_density()
    n0 = o.n
    before = {f: o[f].copy() for f in ("x", "y", "z", "vx", "vy", "vz", "h", "dnn", "id")}
    st0 = o.stats()
    c = np.array([0.5, 0.5, 0.5])
    inside = np.sum((before["x"] - .5) ** 2 + (before["y"] - .5) ** 2 + (before["z"] - .5) ** 2
                    < 0.25 ** 2)
    ns = o.split_pass(0, 42)
    assert ns == inside and o.n == n0 + ns
    st1 = o.stats()
    assert st1.mass == pytest.approx(st0.mass, rel=1e-15)
    for k in range(3):
        assert st1.mom[k] == pytest.approx(st0.mom[k], rel=1e-12, abs=1e-15)
    parents = np.nonzero(o["flags"][:n0] & oracle.FLAG_CHANGED)[0]
    assert len(parents) == ns
    kids = n0 + np.arange(ns)
    assert np.array_equal(o["id"][kids], np.arange(n0, n0 + ns, dtype=np.uint64))
    P = np.stack([before[f][parents] for f in ("x", "y", "z")], 1)
    A = np.stack([o[f][parents] for f in ("x", "y", "z")], 1)
    B = np.stack([o[f][kids] for f in ("x", "y", "z")], 1)
    # centre of mass at the parent; separation 2 r_sep; r_sep = min(0.2 h, 0.35 d_nn)
    assert np.abs(0.5 * (A + B) - P).max() < 4e-16
    rsep = np.minimum(0.2 * before["h"][parents], 0.35 * before["dnn"][parents])
    assert np.allclose(np.linalg.norm(A - P, axis=1), rsep, rtol=1e-12)
    # tangential: both children equidistant from the zone centre
    assert np.allclose(np.linalg.norm(A - c, axis=1), np.linalg.norm(B - c, axis=1), rtol=1e-12)
    # Eq. 2: h^3 halves; level rises by one; velocities copied
    assert np.allclose((o["h"][parents] / before["h"][parents]) ** 3, 0.5, rtol=1e-15)
    assert np.array_equal(o["h"][parents], o["h"][kids])
    assert np.all(o["level"][parents] == 1) and np.all(o["level"][kids] == 1)
    assert np.array_equal(o["vx"][kids], before["vx"][parents])


def test_split_separation_capped_by_nearest_neighbour():
    w = apr_synth.lattice_box(8, jitter=0.0, sphere_R=(0.2,))
    # move one particle next to the one nearest the centre
    p = w["p"]
    d2 = (p["x"] - .5) ** 2 + (p["y"] - .5) ** 2 + (p["z"] - .5) ** 2
    a = int(np.argmin(d2))
    b = int(np.argsort(d2)[-1])
    p["x"][b], p["y"][b], p["z"][b] = p["x"][a] + 0.01, p["y"][a], p["z"][a]
    o = oracle.Oracle(w, capacity=1024)
    o.density()
    h_a, dnn_a = o["h"][a], o["dnn"][a]
    assert abs(dnn_a - 0.01) < 1e-8 and 0.35 * dnn_a < 0.2 * h_a
    x0 = np.array([o["x"][a], o["y"][a], o["z"][a]])
    o.split_pass(0, 1)
    xa = np.array([o["x"][a], o["y"][a], o["z"][a]])
    assert abs(np.linalg.norm(xa - x0) - 0.35 * dnn_a) < 1e-15


def test_split_capacity_shortfall_leaves_state():
    o = _c1_after_density()
    o.st.cap = o.n + 10
    x = o["x"].copy()
    assert o.split_pass(0, 1) == -1
    assert o.n == 4096 and np.array_equal(o["x"], x)


def test_one_level_change_per_step():
    w = apr_synth.lattice_box(10, jitter=0.05, sphere_R=(0.35, 0.25))
    o = oracle.Oracle(w, capacity=8 * 1000)
    o.density()
    cnt = o.split_merge(0)
    assert o["level"].max() == 1 and cnt.n_split[1] == 0 and cnt.n_split[0] > 0
    o.density()
    cnt = o.split_merge(1)
    assert o["level"].max() == 2 and cnt.n_split[1] > 0


# ------------------------------------------------------------------ merge ---

def _parse_points(s):
    return np.array([[int(v) for v in p.split(",")] for p in s.split(";")], np.int64)


def test_pair_tree_hand_cases():
    with open(__import__("os").path.join(__import__("conftest").GOLDEN, "pair_tree_cases.txt")) as f:
        cases = [l.split("|") for l in f if l.strip() and not l.lstrip().startswith("#")]
    assert len(cases) >= 7
    for name, pts, exp in cases:
        pairs = oracle.pair_tree(_parse_points(pts.strip()))
        got = sorted(tuple(sorted(map(int, p))) for p in pairs)
        want = sorted(tuple(sorted(int(v) for v in q.split("-"))) for q in exp.strip().split(";"))
        assert got == want, name


def test_pair_tree_partition_properties():
    rng = np.random.default_rng(5)
    for n in (2, 4, 6, 10, 64, 250, 1000):
        xi = rng.integers(0, 1 << 20, size=(n, 3))
        pairs = oracle.pair_tree(xi)
        assert pairs.shape == (n // 2, 2)
        assert np.array_equal(np.sort(pairs.ravel()), np.arange(n))
        # independent of the order the set is listed in
        perm = rng.permutation(n)
        again = oracle.pair_tree(xi, order=perm)
        assert sorted(map(tuple, np.sort(pairs, 1))) == sorted(map(tuple, np.sort(again, 1)))
        if n >= 64:  # spatially associated: about one mean spacing apart, not random
            dp = np.linalg.norm(xi[pairs[:, 0]] - xi[pairs[:, 1]], axis=1).mean()
            dr = np.linalg.norm(xi[perm[: n // 2]] - xi[perm[n // 2:]], axis=1).mean()
            spacing = (2.0 ** 60 / n) ** (1.0 / 3.0)
            assert dp < 1.5 * spacing and dp < 0.5 * dr


def test_merge_round_trip_conserves_and_places_at_com():
    o = _c1_after_density()
    o.split_pass(0, 0)
    n1 = o.n
    o.a["flags"][: o.n] &= ~np.uint8(oracle.FLAG_CHANGED)
    st0 = o.stats()
    before = {f: o[f].copy() for f in ("x", "y", "z", "vx", "vy", "vz", "u", "h", "level")}
    o.regions[0].R[0] = 1e-9  # the zone shrinks away: every leaf's centre of mass is outside
    nlev1 = int(np.sum(before["level"] == 1))
    nm, spare = o.merge_pass(1)
    assert nm == nlev1 // 2 and (spare >= 0) == (nlev1 % 2 == 1)
    dead = np.nonzero(o["flags"] & oracle.FLAG_DEAD)[0]
    surv = np.nonzero((o["flags"] & oracle.FLAG_CHANGED) & ~(o["flags"] & oracle.FLAG_DEAD))[0]
    assert len(dead) == nm and len(surv) == nm
    assert np.all(o["level"][surv] == 0)
    assert np.allclose(o["h"][surv] ** 3, 2 * before["h"][surv] ** 3, rtol=1e-15)
    # each leaf: the lower index survives at the pair's centre of mass and mean velocity
    cand = np.nonzero(before["level"] == 1)[0]
    if len(cand) % 2:
        cand = cand[:-1]
    xi = o.quantise()  # positions of the candidates are unchanged except survivors
    X = np.stack([before[f] for f in ("x", "y", "z")], 1)
    q = np.floor((X[cand] - 0.0) / o.cfg.delta).astype(np.int64)
    pairs = cand[oracle.pair_tree(q)]
    for a, b in np.sort(pairs, 1):
        assert a in surv and b in dead
        for k, f in enumerate(("x", "y", "z")):
            assert abs(o[f][a] - 0.5 * (X[a, k] + X[b, k])) < 1e-15
        assert o["vx"][a] == 0.5 * (before["vx"][a] + before["vx"][b])
    st1 = o.stats()
    assert st1.mass == pytest.approx(st0.mass, rel=1e-15)
    for k in range(3):
        assert st1.mom[k] == pytest.approx(st0.mom[k], rel=1e-12, abs=1e-14)
    removed = o.compact()
    assert removed == nm and o.n == n1 - nm
    assert np.all(np.diff(o["id"][o["level"] == 0].astype(np.int64)) != 0)


def test_merge_keeps_pairs_inside_zone_and_scales_h():
    o = _c1_after_density()
    o.split_pass(0, 0)
    o.a["flags"][: o.n] &= ~np.uint8(oracle.FLAG_CHANGED)
    h_before = o["h"].copy()
    nm, _ = o.merge_pass(1)  # zone unchanged: leaves whose centre of mass is inside stay
    surv = np.nonzero((o["flags"] & oracle.FLAG_CHANGED) & ~(o["flags"] & oracle.FLAG_DEAD))[0]
    assert nm == len(surv) and nm < 0.2 * np.sum(o["level"] == 1)
    assert np.allclose(o["h"][surv] ** 3, 2 * h_before[surv] ** 3, rtol=1e-15)
    c = 0.5
    for a in surv:
        assert (o["x"][a] - c) ** 2 + (o["y"][a] - c) ** 2 + (o["z"][a] - c) ** 2 >= 0.25 ** 2


def test_spare_mass_bound_eq4():
    bounds = {int(r[1]): float(r[2]) for r in read_golden("mass_levels.txt") if r[0] == "E"}
    for lmax in (1, 2, 3):
        w = apr_synth.lattice_box(10, jitter=0.1, sphere_R=tuple(0.45 - 0.1 * k for k in range(lmax)))
        o = oracle.Oracle(w, capacity=20000)
        for s in range(lmax + 1):
            o.density()
            o.split_merge(s)
        # remove one particle per level so each level holds an odd count, then derefine fully
        for l in range(1, lmax + 1):
            cand = np.nonzero(o["level"] == l)[0]
            if len(cand) % 2 == 0:
                o.a["flags"][cand[0]] |= oracle.FLAG_DEAD
        o.compact()
        for k in range(lmax):
            o.regions[0].R[k] = 1e-9
        spare_mass = 0.0
        cnt = o.split_merge(100)
        for l in range(1, lmax + 1):
            assert cnt.n_spare[l] <= 1
        # particles still above level 0 after one derefinement pass are either spares or
        # merged-down parents that may descend next step; the spares alone obey Eq. 4
        m0 = w["cfg"]["m0"]
        spare_mass = sum(cnt.n_spare[l] * m0 * 2.0 ** -l for l in range(1, lmax + 1))
        assert spare_mass <= bounds[lmax] * m0 < m0
