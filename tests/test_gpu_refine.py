"""GPU parity of the refinement rules (Sec. 2.1-2.6) against the oracle, from
identical inputs: split and merge results, particle order, ids and the
pairing tree are compared bit-exact."""
import numpy as np
import pytest

import apr_synth
import oracle
from gpu_util import sim, with_velocities

pytestmark = pytest.mark.gpu

FIELDS = ("x", "y", "z", "vx", "vy", "vz", "u", "h", "level", "flags", "id")


def _synthetic_dnn(w, seed=3):
    # nearest-neighbour distances as plain inputs: some caps active, some not
    rng = np.random.default_rng(seed)
    n = len(w["p"]["x"])
    d = np.where(rng.uniform(size=n) < 0.3, rng.uniform(0.1, 0.5, n) * w["p"]["h"], np.inf)
    return d


def _both(w, capacity):
    d = _synthetic_dnn(w)
    o = oracle.Oracle(w, capacity=capacity)
    o.a["dnn"][: o.n] = d
    g = sim(w, capacity=capacity)
    g.t["dnn"][: len(d)].copy_(g.torch.from_numpy(d))
    return o, g


def _same(o, g):
    assert g.n == o.n
    for f in FIELDS:
        a, b = g.get(f), o[f]
        assert np.array_equal(a, b), f


def test_split_pass_bit_exact():
    w = with_velocities(apr_synth.c1_lattice(), 0.5)
    o, g = _both(w, 3 * 4096)
    co = o.split_merge()
    cg = g.split_merge()
    assert list(cg.n_split) == list(co.n_split) and co.n_split[0] > 200
    _same(o, g)


def test_two_level_split_then_merge_bit_exact():
    w = with_velocities(apr_synth.lattice_box(14, 0.1, sphere_R=(0.4, 0.3), seed=9), 0.2)
    o, g = _both(w, 6 * 14 ** 3)
    for _ in range(3):
        co = o.split_merge()
        cg = g.split_merge()
        assert list(cg.n_split) == list(co.n_split)
        assert list(cg.n_merge) == list(co.n_merge)
        _same(o, g)
    # move the zone: particles leave it and merge level by level (Sec. 2.6 order)
    for regs in ([dict(shape=0, axis=0, track_sink=-1, centre=[0.3, 0.5, 0.5], R=[0.4, 0.3])],
                 [dict(shape=0, axis=0, track_sink=-1, centre=[0.5, 0.5, 0.5], R=[0.2, 0.1])],
                 []):
        o.w["regions"] = regs
        o.regions = oracle.make_regions(regs)
        o.nreg = len(regs)
        g.set_regions(regs)
        for _ in range(2):
            co = o.split_merge()
            cg = g.split_merge()
            assert list(cg.n_merge) == list(co.n_merge)
            assert list(cg.n_spare) == list(co.n_spare)
            assert list(cg.n_split) == list(co.n_split)
            _same(o, g)
    assert o["level"].max() <= 2


def _launches(g):
    return g.profile()["launches"]


def test_unchanging_pass_skips_its_trees_and_matches_oracle():
    """One convex zone (a slab across a non-periodic axis): a pass in which nothing
    can split or merge skips its sort, pairing trees and compaction (fewer launches)
    and still reports the oracle's counts and spares; a candidate inside its zone by
    less than the 1e-8 inset, or outside it, takes the full pass (the summary that
    decides this is read while passes stay quiet, and every eighth pass)."""
    w = with_velocities(apr_synth.lattice_box(12, 0.1, sphere_R=(), seed=4), 0.1)
    w["cfg"]["periodic"] = [0, 1, 1]
    w["cfg"]["lmax"] = 1
    slab = lambda R: [dict(shape=apr_synth.SHAPE_SLAB, axis=0, track_sink=-1,
                           centre=[0.5, 0.5, 0.5], R=[R])]
    w["regions"] = slab(0.3)
    n = len(w["p"]["x"])
    o, g = _both(w, 4 * n)
    g.profile_enable(True)

    def both_pass():
        l0 = _launches(g)
        co, cg = o.split_merge(), g.split_merge()
        for f in ("n_split", "n_merge", "n_spare"):
            assert list(getattr(cg, f)) == list(getattr(co, f)), f
        _same(o, g)
        return co, _launches(g) - l0

    co, _ = both_pass()
    assert co.n_split[0] > 100
    # nothing left to do; after a busy pass the summary is read every eighth pass
    quiet = min(both_pass()[1] for _ in range(9))
    # a level-1 particle just inside the boundary (by 5e-9 of R): the full pass
    lv = o["level"]
    d = np.abs(o["x"] - 0.5)
    j = int(np.argmax(np.where(lv == 1, d, -1.0)))
    R = float(d[j]) * (1.0 + 5e-9)
    for regs in (slab(R), slab(0.25)):          # then a zone that leaves particles outside
        o.w["regions"] = regs
        o.regions = oracle.make_regions(regs)
        o.nreg = len(regs)
        g.set_regions(regs)
        co, full = both_pass()
        assert full > quiet
    assert sum(co.n_merge) > 0


def _levelled(points, level=1, h=0.01):
    w = apr_synth.lattice_box(2, 0.0, sphere_R=())
    n = len(points)
    z = np.zeros(n)
    w["p"] = apr_synth._particles(points[:, 0], points[:, 1], points[:, 2], z, z, z, z + 1.0,
                                  z + h, level=np.full(n, level, np.uint8))
    w["cfg"]["lmax"] = 3
    return w


@pytest.mark.parametrize("case", ["uniform", "clusters", "coincident", "line", "tiny"])
def test_pairing_tree_matches_oracle(case):
    rng = np.random.default_rng(len(case))
    if case == "uniform":
        pts = rng.uniform(0, 1, (20001, 3))
    elif case == "clusters":
        c = rng.uniform(0, 1, (7, 3))
        pts = np.mod(c[rng.integers(0, 7, 5000)] + rng.normal(0, 0.01, (5000, 3)), 1.0)
    elif case == "coincident":
        pts = np.repeat(rng.uniform(0, 1, (9, 3)), 12, axis=0)
    elif case == "line":
        pts = np.stack([rng.uniform(0, 1, 999), np.full(999, 0.5), np.full(999, 0.5)], 1)
    else:
        pts = rng.uniform(0, 1, (6, 3))
    w = _levelled(pts)
    g = sim(w)
    pairs, spare = g.merge_pairs(1)
    o = oracle.Oracle(w)
    xi = o.quantise()
    cand = np.arange(len(pts))
    exp_spare = -1
    if len(cand) % 2:
        exp_spare = cand[-1]
        cand = cand[:-1]
    exp = cand[oracle.pair_tree(xi[cand])] if len(cand) else np.zeros((0, 2), int)
    assert spare == exp_spare
    got = sorted(map(tuple, np.sort(pairs, 1)))
    want = sorted(map(tuple, np.sort(exp, 1)))
    assert got == want


def test_split_capacity_shortfall_leaves_state():
    from paper_2409_11470_gb300.binding import AprError
    w = apr_synth.c1_lattice()
    g = sim(w, capacity=4096 + 10)
    x0 = g.get("x").copy()
    with pytest.raises(AprError) as e:
        g.split_merge()
    assert e.value.status == 2
    assert g.n == 4096 and np.array_equal(g.get("x"), x0)


def test_empty_and_single_particle_passes():
    for n in (0, 1):
        w = apr_synth.c1_lattice()
        w["p"] = {k: v[:n] for k, v in w["p"].items()}
        g = sim(w, capacity=64)
        g.split_merge()
        assert g.n == n


def test_derefinement_bit_exact():
    """Zones of lower resolution (level_default 1): the initial merges inside the
    zone, then splits as the zone moves away, identical to the oracle."""
    w = with_velocities(apr_synth.deref_lattice(12), 0.1)
    o, g = _both(w, 3 * 12 ** 3)
    merges = 0
    for _ in range(2):
        co = o.split_merge()
        cg = g.split_merge()
        assert list(cg.n_split) == list(co.n_split)
        assert list(cg.n_merge) == list(co.n_merge)
        _same(o, g)
        merges += co.n_merge[1]
    assert merges > 20
    regs = [dict(shape=0, axis=0, track_sink=-1, centre=[0.8, 0.5, 0.5], R=[0.25])]
    o.regions = oracle.make_regions(regs)
    o.nreg = 1
    g.set_regions(regs)
    splits = 0
    for _ in range(2):
        co = o.split_merge()
        cg = g.split_merge()
        assert list(cg.n_split) == list(co.n_split)
        assert list(cg.n_merge) == list(co.n_merge)
        _same(o, g)
        splits += co.n_split[0]
    assert splits > 0

