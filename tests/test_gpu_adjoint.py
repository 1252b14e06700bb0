"""GPU parity of the split density-error loss and its adjoint against the FP64
oracle, through the C ABI.  J within 1e-4 (FP32-mixed) / 1e-10 (FP64); the
gradient with respect to offsets and children's h within 1e-3 (FP32-mixed) /
1e-9 (FP64) in relative L2 norm."""
import numpy as np
import pytest

import apr_synth
import oracle
from gpu_util import need_gpu, sim

pytestmark = pytest.mark.gpu

TOL = {"fp32": dict(J=1e-4, g=1e-3), "fp64": dict(J=1e-10, g=1e-9)}


def _l2rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def _problem(n_side=12, jitter=0.2, seed=9, vary_h=True):
    w = apr_synth.lattice_box(n_side, jitter, seed=seed)
    if vary_h:
        rng = np.random.default_rng(seed)
        w["p"]["h"] = w["p"]["h"] * rng.uniform(0.85, 1.2, len(w["p"]["h"]))
    return w, apr_synth.adjoint_problem(w, seed=seed)


def _gpu(w, prob, precision):
    n, k = len(w["p"]["x"]), len(prob["parent"])
    g = sim(w, precision, capacity=n + 2 * k)
    J, gd, gh = g.density_loss_grad(prob["parent"], prob["d"], prob["hc"])
    return g, J, gd.cpu().numpy(), gh.cpu().numpy()


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
@pytest.mark.parametrize("make", [lambda: _problem(),
                                  lambda: _problem(n_side=9, seed=4),
                                  lambda: _problem(n_side=14, jitter=0.05, seed=2, vary_h=False)])
def test_loss_and_gradient_match_oracle(make, precision):
    w, prob = make()
    Jo, gdo, gho = oracle.Oracle(w).split_loss_grad(prob["parent"], prob["d"], prob["hc"])
    _, J, gd, gh = _gpu(w, prob, precision)
    t = TOL[precision]
    assert abs(J - Jo) <= t["J"] * Jo
    assert _l2rel(gd, gdo) <= t["g"]
    assert _l2rel(gh, gho) <= t["g"]


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_isolated_split_in_an_open_box(precision):
    cfg = apr_synth._cfg(box_lo=[-4.0] * 3, box_hi=[4.0] * 3, periodic=[0, 0, 0],
                         delta=2.0 ** -26, m0=1.0, lmax=1)
    z = np.zeros(1)
    p = apr_synth._particles(z, z, z, z, z, z, np.ones(1), np.ones(1))
    w = dict(name="isolated", cfg=cfg, regions=[], sinks=[], p=p)
    prob = dict(parent=np.array([0]), d=np.array([[0.5, 0.0, 0.0]]), hc=np.array([0.8, 0.8]))
    Jo, gdo, gho = oracle.Oracle(w).split_loss_grad(prob["parent"], prob["d"], prob["hc"])
    _, J, gd, gh = _gpu(w, prob, precision)
    t = TOL[precision]
    assert abs(J - Jo) <= t["J"] * Jo
    assert np.abs(gd - gdo).max() <= t["g"] * np.abs(gdo).max()
    assert np.abs(gh - gho).max() <= t["g"] * np.abs(gho).max()


def test_children_on_the_parent_give_zero_error():
    w, prob = _problem(vary_h=False)
    par = prob["parent"]
    hc = np.repeat(w["p"]["h"][par], 2)
    n, k = len(w["p"]["x"]), len(par)
    g = sim(w, "fp64", capacity=n + 2 * k)
    J, gd, gh = g.density_loss_grad(par, np.zeros((k, 3)), hc)
    assert J < 1e-24 * k
    assert float(gd.abs().max()) < 1e-10 and float(gh.abs().max()) < 1e-10


def test_subset_of_the_oracle_gradient():
    # the oracle computes only the wanted splits' rows; the GPU computes all
    w, prob = _problem(n_side=14, seed=6)
    want = prob["want"].copy()
    want[::2] = False
    Jo, gdo, gho = oracle.Oracle(w).split_loss_grad(prob["parent"], prob["d"], prob["hc"], want)
    _, J, gd, gh = _gpu(w, prob, "fp32")
    assert abs(J - Jo) <= 1e-4 * Jo
    assert _l2rel(gd[want], gdo[want]) <= 1e-3
    assert _l2rel(gh[np.repeat(want, 2)], gho[np.repeat(want, 2)]) <= 1e-3


def test_bad_inputs_leave_the_state_unchanged():
    import paper_2409_11470_gb300.binding as B
    w, prob = _problem(n_side=9, seed=4)
    n, k = len(w["p"]["x"]), len(prob["parent"])
    g = sim(w, "fp32", capacity=n + 2 * k)
    x0 = g.get("x").copy()
    par = prob["parent"].copy()
    par[1] = par[0]
    with pytest.raises(B.AprError) as e:
        g.density_loss_grad(par, prob["d"], prob["hc"])
    assert e.value.status == 1
    hc = prob["hc"].copy()
    hc[3] = -1.0
    with pytest.raises(B.AprError) as e:
        g.density_loss_grad(prob["parent"], prob["d"], hc)
    assert e.value.status == 1
    small = sim(w, "fp32", capacity=n + 2 * k - 1)
    with pytest.raises(B.AprError) as e:
        small.density_loss_grad(prob["parent"], prob["d"], prob["hc"])
    assert e.value.status == 2
    assert g.n == n and np.array_equal(g.get("x"), x0)
    # the context still works after the errors: same J twice in a row
    J1 = g.density_loss_grad(prob["parent"], prob["d"], prob["hc"])[0]
    J2 = g.density_loss_grad(prob["parent"], prob["d"], prob["hc"])[0]
    assert J1 == J2 and J1 > 0


def test_autograd_function_and_placement_optimisation():
    import torch

    import paper_2409_11470_gb300.binding as B
    w, prob = _problem(jitter=0.05, vary_h=False)
    n, k = len(w["p"]["x"]), len(prob["parent"])
    g = sim(w, "fp32", capacity=n + 2 * k)
    dev = g.device
    d = torch.tensor(prob["d"], dtype=torch.float64, device=dev, requires_grad=True)
    hc = torch.tensor(prob["hc"], dtype=torch.float64, device=dev, requires_grad=True)
    par = torch.tensor(prob["parent"], device=dev)
    loss = B.split_density_loss(g, par, d, hc)
    loss.backward()
    J, gd, gh = g.density_loss_grad(par, d.detach(), hc.detach())
    assert float(loss.detach()) == J
    assert torch.equal(d.grad, gd) and torch.equal(hc.grad, gh)
    # the use: move the children to minimise the error the split creates
    h = float(np.mean(prob["hc"]))
    opt = torch.optim.Adam([d, hc], lr=0.02 * h)
    J0 = J
    for _ in range(30):
        opt.zero_grad()
        loss = B.split_density_loss(g, par, d, hc)
        loss.backward()
        opt.step()
    J1 = g.density_loss_grad(par, d.detach(), hc.detach())[0]
    assert J1 < 0.05 * J0


@pytest.mark.slow
def test_full_size_lattice_gradient_on_the_subset():
    """2,000,376-particle jittered lattice, first split pass of the R = 0.35 zone;
    the oracle's gradient on the 2048 splits (4096 children) nearest the centre."""
    need_gpu()
    w = apr_synth.c5_adjoint_lattice()
    prob = apr_synth.adjoint_problem(w)
    Jo, gdo, gho = oracle.Oracle(w).split_loss_grad(prob["parent"], prob["d"], prob["hc"],
                                                    prob["want"])
    _, J, gd, gh = _gpu(w, prob, "fp32")
    want = prob["want"]
    assert abs(J - Jo) <= 1e-4 * Jo
    assert _l2rel(gd[want], gdo[want]) <= 1e-3
    assert _l2rel(gh[np.repeat(want, 2)], gho[np.repeat(want, 2)]) <= 1e-3
