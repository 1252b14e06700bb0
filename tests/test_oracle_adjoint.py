"""Pins of the oracle's split density-error loss J and its gradient (the
adjoint row; the paper motivates the error in Sec. 2.2 and Sec. 2.5 but gives no
such function).  J = sum over children of (rho_new - rho_ref)^2 with h fixed.

Pins, chosen so that a dropped term, a wrong sign or a swapped smoothing length
fails one of them:
  * an isolated parent split into two children, worked by hand from the M4
    polynomial (children's h differs from the parent's);
  * children on top of their parent with the parent's h reproduce the reference
    density exactly (J = 0, gradient 0) on a jittered lattice;
  * J and its gradient are invariant under a periodic translation;
  * central finite differences (relative step 1e-4) agree with the gradient to
    1e-6 of its largest component;
  * the gradient of a subset equals the rows of the full gradient.
"""
import math

import numpy as np
import pytest

import apr_synth
import oracle


def _isolated(h_parent=1.0):
    cfg = apr_synth._cfg(box_lo=[-4.0] * 3, box_hi=[4.0] * 3, periodic=[0, 0, 0],
                         delta=2.0 ** -26, m0=1.0, lmax=1)
    z = np.zeros(1)
    p = apr_synth._particles(z, z, z, z, z, z, np.ones(1), np.full(1, h_parent))
    return dict(name="isolated", cfg=cfg, regions=[], sinks=[], p=p)


def test_isolated_pair_worked_by_hand():
    # parent m=1, h=1 at the origin; children m=1/2 at (+-0.5, 0, 0), h=0.8 each.
    # M4: f(q) = 1 - 1.5q^2 + 0.75q^3 (q<1), 0.25(2-q)^3 (1<=q<2); W = f/(pi h^3).
    # child 1: self at q=0 (f=1), the other child at r=1, q=1.25 (f=0.25*0.75^3);
    # the parent (reference set) at r=0.5, h=1, q=0.5 (f=0.71875).
    o = oracle.Oracle(_isolated())
    J, gd, gh = o.split_loss_grad([0], [[0.5, 0.0, 0.0]], [0.8, 0.8])
    h3, h4 = 0.8 ** 3, 0.8 ** 4
    f125, df125 = 0.25 * 0.75 ** 3, -0.75 * 0.75 ** 2
    rho_new = 0.5 * (1.0 + f125) / (math.pi * h3)
    rho_ref = 0.71875 / math.pi
    e = rho_new - rho_ref
    assert J == pytest.approx(2.0 * e * e, rel=1e-14)
    # dJ/dd = 4 e de/dd, de/dd = 0.5 * 2 * W'(2d, 0.8) - W'(d, 1), W' = f'(q)/(pi h^4)
    dfhalf = -3.0 * 0.5 + 2.25 * 0.25
    de_dd = df125 / (math.pi * h4) - dfhalf / math.pi
    assert gd[0, 0] == pytest.approx(4.0 * e * de_dd, rel=1e-13)
    assert abs(gd[0, 1]) < 1e-15 and abs(gd[0, 2]) < 1e-15
    # dJ/dh_1 = 2 e m_c [dW/dh(0) + dW/dh(r=1)], dW/dh = -(3f + q f')/(pi h^4)
    dwdh = (-3.0 - (3.0 * f125 + 1.25 * df125)) / (math.pi * h4)
    assert gh[0] == pytest.approx(2.0 * e * 0.5 * dwdh, rel=1e-13)
    assert gh[1] == pytest.approx(gh[0], rel=1e-14)


def _lattice_problem(n_side=8, jitter=0.2, seed=7, vary_h=True):
    w = apr_synth.lattice_box(n_side, jitter, seed=seed)
    if vary_h:
        rng = np.random.default_rng(seed)
        w["p"]["h"] = w["p"]["h"] * rng.uniform(0.85, 1.2, len(w["p"]["h"]))
    prob = apr_synth.adjoint_problem(w, seed=seed)
    assert len(prob["parent"]) >= 8
    return w, prob


def test_children_on_the_parent_reproduce_the_reference_density():
    w, prob = _lattice_problem(vary_h=False)  # one h for every particle
    o = oracle.Oracle(w)
    par = prob["parent"]
    hc = np.repeat(w["p"]["h"][par], 2)
    J, gd, gh = o.split_loss_grad(par, np.zeros((len(par), 3)), hc)
    assert J < 1e-26 * len(par)
    assert np.abs(gd).max() < 1e-11 and np.abs(gh).max() < 1e-11
    # moved children do leave an error
    J2, _, _ = o.split_loss_grad(par, prob["d"], prob["hc"])
    assert J2 > 1e-6


def test_periodic_translation_invariance():
    w, prob = _lattice_problem()
    J, gd, gh = oracle.Oracle(w).split_loss_grad(prob["parent"], prob["d"], prob["hc"])
    shift = (0.31, 0.17, 0.73)
    for k, key in enumerate(("x", "y", "z")):
        w["p"][key] = np.mod(w["p"][key] + shift[k], 1.0)
    J2, gd2, gh2 = oracle.Oracle(w).split_loss_grad(prob["parent"], prob["d"], prob["hc"])
    assert J2 == pytest.approx(J, rel=1e-11)
    assert np.abs(gd2 - gd).max() < 1e-9 * np.abs(gd).max()
    assert np.abs(gh2 - gh).max() < 1e-9 * np.abs(gh).max()


def test_central_differences():
    w, prob = _lattice_problem(n_side=6, seed=11)
    o = oracle.Oracle(w)
    par, d, hc = prob["parent"], prob["d"], prob["hc"]
    J, gd, gh = o.split_loss_grad(par, d, hc)
    scale = max(np.abs(gd).max(), np.abs(gh).max())
    rng = np.random.default_rng(3)
    for k in rng.choice(len(par), size=min(6, len(par)), replace=False):
        for m in range(3):
            s = 1e-4 * hc[2 * k]
            dp, dm = d.copy(), d.copy()
            dp[k, m] += s
            dm[k, m] -= s
            fd = (o.split_loss_grad(par, dp, hc)[0] - o.split_loss_grad(par, dm, hc)[0]) / (2 * s)
            assert abs(fd - gd[k, m]) <= 1e-6 * scale, (k, m, fd, gd[k, m])
        for side in range(2):
            j = 2 * k + side
            s = 1e-4 * hc[j]
            hp, hm = hc.copy(), hc.copy()
            hp[j] += s
            hm[j] -= s
            fd = (o.split_loss_grad(par, d, hp)[0] - o.split_loss_grad(par, d, hm)[0]) / (2 * s)
            assert abs(fd - gh[j]) <= 1e-6 * scale, (j, fd, gh[j])


def test_subset_gradient_is_rows_of_the_full_gradient():
    w, prob = _lattice_problem(seed=5)
    o = oracle.Oracle(w)
    par, d, hc = prob["parent"], prob["d"], prob["hc"]
    want = np.zeros(len(par), bool)
    want[::3] = True
    J, gd, gh = o.split_loss_grad(par, d, hc)
    Js, gds, ghs = o.split_loss_grad(par, d, hc, want)
    assert Js == J
    assert np.array_equal(gds[want], gd[want]) and not gds[~want].any()
    w2 = np.repeat(want, 2)
    assert np.array_equal(ghs[w2], gh[w2]) and not ghs[~w2].any()


def test_bad_parents_are_rejected():
    w, prob = _lattice_problem()
    o = oracle.Oracle(w)
    par = prob["parent"].copy()
    par[1] = par[0]
    with pytest.raises(ValueError):
        o.split_loss_grad(par, prob["d"], prob["hc"])
    par = prob["parent"].copy()
    par[0] = len(w["p"]["x"])
    with pytest.raises(ValueError):
        o.split_loss_grad(par, prob["d"], prob["hc"])
