"""The oracle's global time-step limit (orc_timestep) on cases worked by hand
(tests/golden/timestep_cases.txt): a perfect lattice at rest (the Courant term
with v_sig = c_s), cold gas in a point mass's field (the force term, with
|a| = G M / d^2 in closed form), the same with the nearest particle fixed
(fixed particles do not limit the step), and one particle moving towards its
neighbour (the signal speed's approach term).  A wrong factor (0.3 / 0.25
swapped), a missing square root, h in place of 2h or h^2, a sum where the
reading takes a maximum, or a fixed particle counted all fail one case."""
import numpy as np
import pytest

import apr_synth
import oracle
from conftest import read_golden


def _point(s):
    return None if s == "-" else [float(v) for v in s.split(",")]


def _case(u, moving, sink, fixed):
    w = apr_synth.lattice_box(8, jitter=0.0, sphere_R=(), u0=u)
    p = w["p"]
    pos = np.stack([p["x"], p["y"], p["z"]], axis=1)

    def at(xyz):
        i = int(np.argmin(np.sum((pos - np.array(xyz)) ** 2, axis=1)))
        assert np.allclose(pos[i], xyz, atol=1e-12)
        return i

    if moving:
        p["vx"][at(moving[:3])] = moving[3]
    if sink:
        w["sinks"] = [dict(x=sink[:3], v=[0.0, 0.0, 0.0], m=sink[3], racc=1e-3)]
    if fixed:
        p["flags"][at(fixed)] |= apr_synth.FLAG_FIXED
    o = oracle.Oracle(w, capacity=len(p["x"]))
    assert o.density_force() == 0
    h = o["h"]
    assert np.ptp(h) <= 1e-12 * h.mean()  # one h on a perfect lattice
    return o, float(h.mean())


@pytest.mark.parametrize("row", read_golden("timestep_cases.txt"), ids=lambda r: r[0])
def test_timestep_worked_cases(row):
    name, u, moving, sink, fixed, quantity, expected = row
    o, h = _case(float(u), _point(moving), _point(sink), _point(fixed))
    dt = o.timestep()
    got = dt / h if quantity == "dt_over_h" else dt / np.sqrt(h)
    assert got == pytest.approx(float(expected), rel=1e-10), name
    if name == "D":
        # the viscous deceleration of the pair stays below the Courant limit
        acc = np.sqrt(o["ax"] ** 2 + o["ay"] ** 2 + o["az"] ** 2).max()
        assert 0.25 * np.sqrt(h / acc) > 1.5 * dt
