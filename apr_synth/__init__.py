"""Seeded synthetic workloads for the adaptive-particle-refinement (APR) SPH hot path.

This module only *places particles* and states run parameters.  It holds none of
the method's arithmetic (no kernel, no density, no split/merge rule), so both the
FP64 CPU oracle and the CUDA library can take their inputs from here without
sharing any code with each other.

Every workload is a plain ``dict``:

``cfg``        run parameters (box, quantisation unit, EOS, viscosity, APR limits)
``regions``    refinement regions (centre, nested boundaries, shape, optional sink to track)
``sinks``      point masses (position, velocity, mass, accretion radius)
``p``          particle arrays (float64 positions/velocities/u/h, uint8 level/flags, uint64 id)

The paper's own problems (the HD 142527 circumbinary disc, the planet-in-disc and
flyby runs of Section 3) need initial conditions that are not available here; the
generators below stand in for them with the same geometry, profiles and particle
counts (surface density Sigma ~ 1/R on R in [1, 10], H/R = 0.05 at R = 1,
c_s ~ R^-1/4, Keplerian rotation, a sink-tracking refinement sphere), and the
shock tube and lattices are the usual SPH test set-ups.  All randomness comes from
``numpy.random.default_rng(seed)`` with ``seed = 20240917 + index``.
"""
from __future__ import annotations

import math

import numpy as np

SEED_BASE = 20240917

# particle flag bits (shared vocabulary of the state, not arithmetic)
FLAG_CHANGED = 1   # split or merged during the current split/merge pass
FLAG_FIXED = 2     # boundary particle: never moved, split or merged
FLAG_DEAD = 4      # removed (merged away or accreted) until the next compaction
FLAG_NEW = 8       # introduced by a split or merge, not yet relaxed

SHAPE_SPHERE = 0
SHAPE_SLAB = 1
SHAPE_CYLINDER = 2

EOS_ADIABATIC = 0
EOS_LOCALLY_ISOTHERMAL = 1

KERNEL_M4 = 0
KERNEL_WENDLAND_C2 = 1


def _cfg(**kw):
    base = dict(
        box_lo=[0.0, 0.0, 0.0], box_hi=[1.0, 1.0, 1.0], periodic=[1, 1, 1],
        delta=2.0 ** -30,
        hfact=1.2, gamma=5.0 / 3.0, eos=EOS_ADIABATIC, cs0=1.0, qcs=0.0,
        alpha_av=1.0, beta_av=2.0, alpha_u=0.0,
        rsep_fac=0.2, dnn_cap=0.35,
        m0=1.0, lmax=1, seed=SEED_BASE,
        ccour=0.3, cforce=0.25, G=1.0,
        kernel=KERNEL_M4, level_default=0,
    )
    base.update(kw)
    return base


def _particles(x, y, z, vx, vy, vz, u, h, flags=None, level=None):
    n = len(x)
    # a copy per field: callers may pass one array for several fields (zero
    # velocities), and a later in-place change of one field must not reach the others
    p = dict(
        x=np.array(x, dtype=np.float64),
        y=np.array(y, dtype=np.float64),
        z=np.array(z, dtype=np.float64),
        vx=np.array(vx, dtype=np.float64),
        vy=np.array(vy, dtype=np.float64),
        vz=np.array(vz, dtype=np.float64),
        u=np.array(u, dtype=np.float64),
        h=np.array(h, dtype=np.float64),
        level=np.zeros(n, np.uint8) if level is None else np.ascontiguousarray(level, np.uint8),
        flags=np.zeros(n, np.uint8) if flags is None else np.ascontiguousarray(flags, np.uint8),
        id=np.arange(n, dtype=np.uint64),
    )
    return p


def lattice_box(n_side=16, jitter=0.05, seed=SEED_BASE, sphere_R=(0.25,), gamma=5.0 / 3.0,
                u0=1.0, rho0=1.0, hfact=1.2, name=None, kernel=KERNEL_M4):
    """Cubic lattice of ``n_side**3`` particles in the periodic unit box.

    Positions are cell centres ``(i + 1/2)/n_side`` moved by ``U(-jitter, jitter)``
    lattice spacings per axis; equal masses ``rho0/n_side**3``; ``u = u0``; ``v = 0``;
    ``h = hfact * spacing``.  A refinement sphere at the box centre with nested radii
    ``sphere_R`` (one level per radius, outermost first).
    """
    rng = np.random.default_rng(seed)
    s = 1.0 / n_side
    g = (np.arange(n_side) + 0.5) * s
    X, Y, Z = np.meshgrid(g, g, g, indexing="ij")
    pos = np.stack([X.ravel(), Y.ravel(), Z.ravel()], axis=1)
    if jitter:
        pos = pos + rng.uniform(-jitter, jitter, size=pos.shape) * s
    pos = np.mod(pos, 1.0)
    n = len(pos)
    zeros = np.zeros(n)
    p = _particles(pos[:, 0], pos[:, 1], pos[:, 2], zeros, zeros, zeros,
                   np.full(n, u0), np.full(n, hfact * s))
    cfg = _cfg(gamma=gamma, hfact=hfact, m0=rho0 * s ** 3, lmax=max(1, len(sphere_R)), seed=seed,
               kernel=kernel)
    regions = [dict(shape=SHAPE_SPHERE, axis=0, track_sink=-1, centre=[0.5, 0.5, 0.5],
                    R=list(sphere_R))] if sphere_R else []
    return dict(name=name or f"lattice{n_side}", cfg=cfg, regions=regions, sinks=[], p=p,
                rho0=rho0, spacing=s)


def c1_lattice():
    """16^3 = 4096-particle jittered lattice, periodic unit box, one refinement sphere r = 0.25."""
    return lattice_box(16, 0.05, SEED_BASE + 0, sphere_R=(0.25,), name="c1_lattice4096")


def sod(nL=28, gamma=1.4, slab=(0.15, 0.10), seed=SEED_BASE + 1, jitter=0.05, name=None):
    """Three-dimensional Sod shock tube.

    x in [-0.5, 0.5], y and z periodic with width 0.1 (to within 4e-10: a whole number
    of lattice units 2^-29).  Left state rho = 1, P = 1 on a
    lattice of spacing 0.1/nL; right state rho = 0.125, P = 0.1 on spacing 0.2/nL (equal
    particle masses).  Each particle is moved by U(-jitter, jitter) local spacings per
    axis: a perfect cubic lattice cannot rearrange sideways under the one-dimensional
    expansion and its rarefied part ends up stretched along x only, which biases the
    SPH estimates behind the rarefaction.  Particles within 4*hfact spacings of
    x = +-0.5 are FIXED.  The refinement region is a slab |x| < slab[k] for level k + 1.
    """
    assert nL % 2 == 0
    # the width 0.1 rounded to a whole number of lattice units 2^-29 (within 4e-10):
    # periodic lengths are whole numbers of units, and a power-of-two unit lets the
    # GPU quantise by a multiplication
    delta = 2.0 ** -29
    w = round(0.1 / delta) * delta
    hfact = 1.2
    sL = w / nL
    sR = 2.0 * sL
    gyz_L = (np.arange(nL) + 0.5) * sL
    gyz_R = (np.arange(nL // 2) + 0.5) * sR
    xL = (np.arange(5 * nL) + 0.5) * sL - 0.5
    xR = (np.arange(5 * nL // 2) + 0.5) * sR
    XL, YL, ZL = np.meshgrid(xL, gyz_L, gyz_L, indexing="ij")
    XR, YR, ZR = np.meshgrid(xR, gyz_R, gyz_R, indexing="ij")
    x = np.concatenate([XL.ravel(), XR.ravel()])
    y = np.concatenate([YL.ravel(), YR.ravel()])
    z = np.concatenate([ZL.ravel(), ZR.ravel()])
    nl = XL.size
    n = len(x)
    rho = np.where(np.arange(n) < nl, 1.0, 0.125)
    P = np.where(np.arange(n) < nl, 1.0, 0.1)
    u = P / ((gamma - 1.0) * rho)
    spacing = np.where(np.arange(n) < nl, sL, sR)
    h = hfact * spacing
    flags = np.zeros(n, np.uint8)
    fixed = (x < -0.5 + 4 * hfact * sL) | (x > 0.5 - 4 * hfact * sR)
    flags[fixed] = FLAG_FIXED
    if jitter:
        rng = np.random.default_rng(seed)
        x = x + rng.uniform(-jitter, jitter, n) * spacing
        y = np.mod(y + rng.uniform(-jitter, jitter, n) * spacing, w)
        z = np.mod(z + rng.uniform(-jitter, jitter, n) * spacing, w)
    zeros = np.zeros(n)
    p = _particles(x, y, z, zeros, zeros, zeros, u, h, flags=flags)
    cfg = _cfg(box_lo=[-0.6, 0.0, 0.0], box_hi=[0.6, w, w], periodic=[0, 1, 1],
               delta=delta, gamma=gamma, hfact=hfact, m0=sL ** 3,
               alpha_av=1.0, beta_av=2.0, alpha_u=1.0, lmax=len(slab), seed=seed)
    regions = [dict(shape=SHAPE_SLAB, axis=0, track_sink=-1, centre=[0.0, 0.05, 0.05],
                    R=list(slab))] if slab else []
    return dict(name=name or f"sod_nL{nL}", cfg=cfg, regions=regions, sinks=[], p=p,
                sod=dict(rhoL=1.0, PL=1.0, rhoR=0.125, PR=0.1, gamma=gamma, x0=0.0))


def c2_sod():
    """The full-size Sod tube: 140x28x28 + 70x14x14 = 123,480 particles, 2-level slab."""
    return sod(28, name="c2_sod123480")


def _disc(n, seed, Rin=1.0, Rout=10.0, mdisc=0.05, H0=0.05, q=0.25, hfact=1.2):
    rng = np.random.default_rng(seed)
    R = rng.uniform(Rin, Rout, n)          # Sigma ~ 1/R  =>  dM/dR = const
    phi = rng.uniform(0.0, 2.0 * math.pi, n)
    H = H0 * R ** (1.5 - q)                # H = c_s/Omega, c_s = H0 R^-q, Omega = R^-3/2
    z = rng.normal(0.0, 1.0, n) * H
    x = R * np.cos(phi)
    y = R * np.sin(phi)
    vphi = np.sqrt(1.0 / R)
    vx = -vphi * np.sin(phi)
    vy = vphi * np.cos(phi)
    vz = np.zeros(n)
    m = mdisc / n
    sigma0 = mdisc / (2.0 * math.pi * (Rout - Rin))
    rho = sigma0 / R / (math.sqrt(2.0 * math.pi) * H) * np.exp(-0.5 * (z / H) ** 2)
    rho = np.maximum(rho, 1e-6 * rho.max())
    h = hfact * (m / rho) ** (1.0 / 3.0)
    h = np.minimum(h, 1.0)
    u = np.zeros(n)
    p = _particles(x, y, z, vx, vy, vz, u, h)
    cfg = _cfg(box_lo=[-12.0, -12.0, -12.0], box_hi=[12.0, 12.0, 12.0], periodic=[0, 0, 0],
               delta=2.0 ** -25, gamma=1.0, eos=EOS_LOCALLY_ISOTHERMAL, cs0=H0, qcs=q,
               hfact=hfact, m0=m, alpha_av=0.1, beta_av=2.0, alpha_u=0.0, seed=seed)
    return p, cfg


def disc_planet(n=1_000_000, seed=SEED_BASE + 2, name=None):
    """Locally isothermal disc around M = 1 with a q = 1e-3 planet at R = 5 and a 3-level
    refinement sphere R = (2.0, 1.5, 1.0) that tracks the planet."""
    p, cfg = _disc(n, seed)
    cfg["lmax"] = 3
    mp = 1e-3
    vp = math.sqrt((1.0 + mp) / 5.0)
    sinks = [dict(x=[0.0, 0.0, 0.0], v=[0.0, -mp * vp, 0.0], m=1.0, racc=0.5),
             dict(x=[5.0, 0.0, 0.0], v=[0.0, vp, 0.0], m=mp, racc=0.25)]
    regions = [dict(shape=SHAPE_SPHERE, axis=0, track_sink=1, centre=[5.0, 0.0, 0.0],
                    R=[2.0, 1.5, 1.0])]
    return dict(name=name or f"c3_disc_planet{n}", cfg=cfg, regions=regions, sinks=sinks, p=p)


def c3_disc_planet():
    return disc_planet(1_000_000)


def flyby(n=8_000_000, seed=SEED_BASE + 3, name=None):
    """Disc as above (no planet) plus a unit-mass perturber on a parabolic orbit with
    periastron 20, started at true anomaly -120 degrees; a 2-level refinement sphere
    R = (7.5, 5.0) follows it."""
    p, cfg = _disc(n, seed)
    cfg["lmax"] = 2
    f = -2.0 * math.pi / 3.0
    qperi = 20.0
    ptot = 2.0 * qperi
    mtot = 2.0
    r = ptot / (1.0 + math.cos(f))
    pos = [r * math.cos(f), r * math.sin(f), 0.0]
    k = math.sqrt(mtot / ptot)
    vr, vt = k * math.sin(f), k * (1.0 + math.cos(f))
    vel = [vr * math.cos(f) - vt * math.sin(f), vr * math.sin(f) + vt * math.cos(f), 0.0]
    sinks = [dict(x=[0.0, 0.0, 0.0], v=[0.0, 0.0, 0.0], m=1.0, racc=0.5),
             dict(x=pos, v=vel, m=1.0, racc=1.0)]
    regions = [dict(shape=SHAPE_SPHERE, axis=0, track_sink=1, centre=list(pos), R=[7.5, 5.0])]
    return dict(name=name or f"c4_flyby{n}", cfg=cfg, regions=regions, sinks=sinks, p=p)


def wendland_lattice(n_side=16, jitter=0.05, seed=SEED_BASE + 5, sphere_R=(0.25,)):
    """The C1 lattice with the Wendland C2 kernel at h_fact = 1.3 (the kernel and
    h_fact of the paper's applications, Sec. 3)."""
    return lattice_box(n_side, jitter, seed, sphere_R=sphere_R, hfact=1.3,
                       kernel=KERNEL_WENDLAND_C2, name=f"wendland_lattice{n_side}")


def deref_lattice(n_side=16, jitter=0.05, seed=SEED_BASE + 6, level=1, sphere_R=(0.25,)):
    """Derefinement: a jittered lattice whose particles all start at ``level`` (mass
    m0 / 2^level with m0 = 2^level rho0 spacing^3), ``level_default = level``, and a
    zone at the box centre asking for one level less inside each radius."""
    w = lattice_box(n_side, jitter, seed, sphere_R=sphere_R, name=f"deref_lattice{n_side}")
    w["cfg"]["m0"] = w["cfg"]["m0"] * 2.0 ** level
    w["cfg"]["lmax"] = level
    w["cfg"]["level_default"] = level
    w["p"]["level"][:] = level
    return w


def sound_wave_box(n_across=64, A=0.02, seed=SEED_BASE + 7, gamma=5.0 / 3.0, cs0=1.0,
                   vx0=0.001, noise=1e-4, R=0.1, hfact=1.2, kernel=KERNEL_M4):
    """The periodic sound-wave box of the paper's appendix tests.

    A close-packed (ABAB) lattice with ``n_across`` particles along x in a box
    [0, 1) x [0, Ly) x [0, Lz) (Ly, Lz: whole numbers of rows and layers, rounded
    to whole lattice units), 64 x 74 x 12 = 56,832 particles at the default size.
    x is stretched so that the density is rho0 + A sin(2 pi x) (rho0 = 1, equal
    masses); u = u0 + A (P0/rho0) sin(2 pi x) with P0 = rho0 cs0^2 / gamma, adiabatic;
    v = (vx0, 0, 0); x and y moved by U(-noise, noise) box lengths.  The zone is a
    cylinder along z of radius R through (0.5, 0.5) with one level; the paper first
    activates it at t = 0.5 (``regions_at`` below; ``regions`` starts empty).
    """
    rng = np.random.default_rng(seed)
    a = 1.0 / n_across
    dy, dz = a * math.sqrt(3.0) / 2.0, a * math.sqrt(2.0 / 3.0)
    ny = 2 * max(1, int(round(1.0 / dy / 2.0)))
    nz = 2 * max(1, int(round(0.15 / dz / 2.0)))
    delta = 2.0 ** -29
    Ly = round(ny * dy / delta) * delta
    Lz = round(nz * dz / delta) * delta
    i, j, k = np.meshgrid(np.arange(n_across), np.arange(ny), np.arange(nz), indexing="ij")
    i, j, k = i.ravel(), j.ravel(), k.ravel()
    x0 = (i + 0.5 * (j % 2) + 0.5 * (k % 2)) * a
    y = (j + (k % 2) / 3.0) * (Ly / ny)
    z = k * (Lz / nz)
    x0 = np.mod(x0, 1.0)
    # mass coordinate -> position: x + A/(2 pi rho0) (1 - cos 2 pi x) = x0
    x = x0.copy()
    for _ in range(50):
        g = x + A / (2.0 * math.pi) * (1.0 - np.cos(2.0 * math.pi * x)) - x0
        x -= g / (1.0 + A * np.sin(2.0 * math.pi * x))
    x = np.mod(x + rng.uniform(-noise, noise, x.size), 1.0)
    y = np.mod(y + rng.uniform(-noise, noise, y.size) * 1.0, Ly)
    n = x.size
    rho = 1.0 + A * np.sin(2.0 * math.pi * x)
    m = Ly * Lz / n
    P0 = cs0 * cs0 / gamma
    u0 = P0 / (gamma - 1.0)
    u = u0 + A * P0 * np.sin(2.0 * math.pi * x)
    h = hfact * (m / rho) ** (1.0 / 3.0)
    zeros = np.zeros(n)
    p = _particles(x, y, z, np.full(n, vx0), zeros, zeros, u, h)
    cfg = _cfg(box_hi=[1.0, Ly, Lz], periodic=[1, 1, 1], delta=delta, gamma=gamma, hfact=hfact,
               m0=m, lmax=1, seed=seed, alpha_av=0.1, beta_av=0.2, kernel=kernel)
    zone = dict(shape=SHAPE_CYLINDER, axis=2, track_sink=-1, centre=[0.5, 0.5, 0.5 * Lz], R=[R])
    return dict(name=f"sound_wave_box{n}", cfg=cfg, regions=[], regions_at=(0.5, [zone]),
                sinks=[], p=p, rho0=1.0, A=A, Ly=Ly, Lz=Lz)


def wave_profile(x, y, rho, Ly, nbins=64, band=(0.4, 0.6)):
    """Mean density in x bins over the band band[0] < y/Ly < band[1] (the paper's
    cross section of the sound-wave box); returns (bin centres, means)."""
    sel = (y > band[0] * Ly) & (y < band[1] * Ly)
    idx = np.minimum((x[sel] * nbins).astype(np.int64), nbins - 1)
    cnt = np.bincount(idx, minlength=nbins)
    tot = np.bincount(idx, weights=rho[sel], minlength=nbins)
    return (np.arange(nbins) + 0.5) / nbins, tot / np.maximum(cnt, 1)


def zone_fuzz(x, y, level, h, centre=(0.5, 0.5), R=0.1):
    """How far the mixed-level transition reaches past a circular zone boundary:
    the largest distance of a level-1 particle outside R or a level-0 particle
    inside R, in units of the level-0 smoothing length (mean over level 0)."""
    r = np.hypot(x - centre[0], y - centre[1])
    out = (level >= 1) & (r >= R)
    inn = (level == 0) & (r < R)
    d = np.concatenate([r[out] - R, R - r[inn]])
    h0 = float(np.mean(h[level == 0])) if np.any(level == 0) else float(np.mean(h))
    return float(d.max() / h0) if d.size else 0.0


def c5_adjoint_lattice(n_side=126):
    """126^3 = 2,000,376-particle jittered lattice with a 2-level sphere R = (0.35, 0.25)."""
    return lattice_box(n_side, 0.05, SEED_BASE + 4, sphere_R=(0.35, 0.25),
                       name=f"c5_lattice{n_side ** 3}")


def adjoint_problem(w, radius=None, centre=(0.5, 0.5, 0.5), seed=SEED_BASE + 4, rsep=0.2,
                    subset=2048):
    """Inputs of one split's density-error loss on the particle set ``w``.

    Splits: every particle closer than ``radius`` (default: the first region's outer
    radius) to ``centre`` on the periodic unit box, in ascending index.  Offsets:
    a uniform random direction times ``rsep * h_p * U(0.5, 1.5)``.  Child smoothing
    lengths: ``h_p * U(0.75, 0.85)`` each.  ``want``: the ``subset`` splits nearest the
    centre (ties by index), the set on which gradients are compared at full size.
    Returns dict(parent, d (k x 3), hc (2k), want (k, bool)).
    """
    p = w["p"]
    if radius is None:
        radius = w["regions"][0]["R"][0]
    rng = np.random.default_rng(seed)
    sep = []
    for k, key in enumerate(("x", "y", "z")):
        dd = p[key] - centre[k]
        if w["cfg"]["periodic"][k]:
            L = w["cfg"]["box_hi"][k] - w["cfg"]["box_lo"][k]
            dd = dd - L * np.round(dd / L)
        sep.append(dd)
    r2 = sep[0] ** 2 + sep[1] ** 2 + sep[2] ** 2
    parent = np.nonzero(r2 < radius * radius)[0].astype(np.int64)
    k = len(parent)
    v = rng.normal(size=(k, 3))
    v /= np.maximum(np.linalg.norm(v, axis=1, keepdims=True), 1e-300)
    hp = p["h"][parent]
    d = v * (rsep * hp * rng.uniform(0.5, 1.5, k))[:, None]
    hc = np.repeat(hp, 2) * rng.uniform(0.75, 0.85, 2 * k)
    order = np.lexsort((parent, r2[parent]))
    want = np.zeros(k, bool)
    want[order[:subset]] = True
    return dict(parent=parent, d=np.ascontiguousarray(d), hc=np.ascontiguousarray(hc), want=want)


def copy_workload(w, capacity=None):
    """Deep copy with particle arrays grown to ``capacity`` (new slots zeroed)."""
    import copy
    out = copy.deepcopy({k: v for k, v in w.items() if k != "p"})
    n = len(w["p"]["x"])
    cap = max(capacity or n, n)
    p = {}
    for k, a in w["p"].items():
        b = np.zeros(cap, dtype=a.dtype)
        b[:n] = a
        p[k] = b
    out["p"] = p
    out["n"] = n
    return out
