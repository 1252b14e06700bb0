"""FP64 CPU oracle for the APR SPH hot path -- TEST INFRASTRUCTURE.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It is a plain, slow, obviously correct
restatement of what the paper's method computes (Nealon & Price, arXiv
2409.11470, Sections 2.1-2.6, Eq. 1-4), plus the standard grad-h SPH density,
force and energy equations the paper cites from the Phantom code.  It shares no
code with the CUDA library (``paper_2409_11470_gb300``) and neither imports the
other.

Functions and the passage each follows (all in ``apr_oracle.c``):

========================  =====================================================
``target_levels``          Sec. 2.1 rules 1-3; nested radii of Table 1
``split_pass``             Sec. 2.2, Eq. 2 (one level), Sec. 2.6 ordering
``pair_tree``              Sec. 2.3 (modified k-d tree, leaves of two)
``merge_pass``             Sec. 2.3, Eq. 3; odd particle left out (Eq. 4)
``split_merge``            Sec. 2.6 (split ascending, merge descending)
``density``                h-rho relation cited in Sec. 2.2; M4, h_fact (Table 2)
``force``                  grad-h SPH momentum/energy + artificial viscosity
                           (cited in Sec. 3 / Sec. 4), a proposed reading
``sink_gravity/accrete``   point masses with accretion (Sec. 3)
``step``                   kick-drift-kick with the per-step order of Sec. 2.6
========================  =====================================================

Every function is pinned by tests under ``tests/test_oracle_*.py`` against
values fixed by the paper or by mathematics (Table 2's neighbour number, Eq. 1
masses, Eq. 4 bound, conservation laws, a lattice, a linear pressure gradient,
the Sod closed form, hand-enumerated pairing trees).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "apr_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

MAXLEV = 8
FLAG_CHANGED, FLAG_FIXED, FLAG_DEAD, FLAG_NEW = 1, 2, 4, 8


def build(force=False):
    """Compile ``apr_oracle.c`` into ``liboracle.so`` next to it (gcc, OpenMP, no FMA)."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-ffp-contract=off", "-fPIC", "-shared",
           "-o", _LIB + ".tmp", _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(_LIB + ".tmp", _LIB)
    return _LIB


class Cfg(C.Structure):
    _fields_ = [("lo", C.c_double * 3), ("hi", C.c_double * 3), ("periodic", C.c_int * 3),
                ("delta", C.c_double), ("hfact", C.c_double), ("gamma", C.c_double),
                ("eos", C.c_int), ("cs0", C.c_double), ("qcs", C.c_double),
                ("alpha_av", C.c_double), ("beta_av", C.c_double), ("alpha_u", C.c_double),
                ("rsep_fac", C.c_double), ("dnn_cap", C.c_double), ("m0", C.c_double),
                ("lmax", C.c_int), ("seed", C.c_ulonglong), ("ccour", C.c_double),
                ("cforce", C.c_double), ("G", C.c_double), ("nthreads", C.c_int),
                ("enumerate", C.c_int), ("kernel", C.c_int), ("level_default", C.c_int)]


class Region(C.Structure):
    _fields_ = [("shape", C.c_int), ("axis", C.c_int), ("track_sink", C.c_int),
                ("nlev", C.c_int), ("centre", C.c_double * 3), ("R", C.c_double * MAXLEV)]


class Sink(C.Structure):
    _fields_ = [("x", C.c_double * 3), ("v", C.c_double * 3), ("a", C.c_double * 3),
                ("m", C.c_double), ("racc", C.c_double)]


_DP = C.POINTER(C.c_double)
_UP = C.POINTER(C.c_ubyte)
_ULP = C.POINTER(C.c_ulonglong)


class State(C.Structure):
    _fields_ = [("n", C.c_longlong), ("cap", C.c_longlong), ("next_id", C.c_longlong)] + \
        [(f, _DP) for f in ("x", "y", "z", "vx", "vy", "vz", "u", "h", "rho", "omega", "ax",
                             "ay", "az", "dudt", "vsig", "dnn", "pres", "cs")] + \
        [("level", _UP), ("flags", _UP), ("id", _ULP), ("bin", _UP)]


class Counts(C.Structure):
    _fields_ = [("n_split", C.c_longlong * MAXLEV), ("n_merge", C.c_longlong * MAXLEV),
                ("n_spare", C.c_longlong * MAXLEV), ("n_accreted", C.c_longlong),
                ("n_dead", C.c_longlong)]


class Stats(C.Structure):
    _fields_ = [("mass", C.c_double), ("mom", C.c_double * 3), ("ang", C.c_double * 3),
                ("ekin", C.c_double), ("etherm", C.c_double)]


DOUBLE_FIELDS = ("x", "y", "z", "vx", "vy", "vz", "u", "h", "rho", "omega", "ax", "ay", "az",
                 "dudt", "vsig", "dnn", "pres", "cs")


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = C.CDLL(_LIB)
            P = C.POINTER
            L.orc_threads.restype = C.c_int
            L.orc_threads.argtypes = [P(Cfg)]
            L.orc_threshold.restype = C.c_ulonglong
            L.orc_threshold.argtypes = [P(Cfg), C.c_double]
            L.orc_lattice_len.restype = C.c_longlong
            L.orc_lattice_len.argtypes = [P(Cfg), C.c_int]
            L.orc_quantise.argtypes = [P(Cfg), C.c_longlong, _DP, _DP, _DP, P(C.c_longlong)]
            L.orc_neighbours.restype = C.c_longlong
            L.orc_neighbours.argtypes = [P(Cfg), P(State), C.c_int, P(C.c_longlong), P(C.c_int),
                                         C.c_longlong]
            L.orc_density.restype = C.c_longlong
            L.orc_density.argtypes = [P(Cfg), P(State), P(C.c_longlong), C.c_longlong]
            L.orc_rho_sum.argtypes = [P(Cfg), P(State), C.c_longlong, C.c_double, _DP]
            L.orc_force.argtypes = [P(Cfg), P(State), P(C.c_longlong), C.c_longlong]
            L.orc_sink_gravity.argtypes = [P(Cfg), P(State), P(Sink), C.c_int]
            L.orc_kernel_m4.argtypes = [C.c_double, _DP]
            L.orc_kernel.argtypes = [C.c_int, C.c_double, _DP]
            L.orc_kernel.restype = None
            L.orc_target_levels.argtypes = [P(Cfg), P(Region), C.c_int, C.c_longlong, _DP, _DP,
                                            _DP, _UP]
            L.orc_track_regions.argtypes = [P(Region), C.c_int, P(Sink), C.c_int]
            L.orc_splitmix64.restype = C.c_ulonglong
            L.orc_splitmix64.argtypes = [C.c_ulonglong]
            L.orc_split_uniform.restype = C.c_double
            L.orc_split_uniform.argtypes = [C.c_ulonglong, C.c_ulonglong, C.c_ulonglong]
            L.orc_split_direction.argtypes = [P(Region), _DP, C.c_double, _DP]
            L.orc_split_pass.restype = C.c_longlong
            L.orc_split_pass.argtypes = [P(Cfg), P(State), P(Region), C.c_int, C.c_int,
                                         C.c_ulonglong]
            L.orc_pair_tree.restype = C.c_int
            L.orc_pair_tree.argtypes = [P(C.c_longlong), P(C.c_longlong), C.c_longlong]
            L.orc_merge_pass.restype = C.c_longlong
            L.orc_merge_pass.argtypes = [P(Cfg), P(State), P(Region), C.c_int, C.c_int,
                                         P(C.c_longlong)]
            L.orc_compact.restype = C.c_longlong
            L.orc_compact.argtypes = [P(State)]
            L.orc_split_merge.restype = C.c_int
            L.orc_split_merge.argtypes = [P(Cfg), P(State), P(Region), C.c_int, C.c_ulonglong,
                                          P(Counts)]
            L.orc_accrete.restype = C.c_longlong
            L.orc_accrete.argtypes = [P(Cfg), P(State), P(Sink), C.c_int]
            L.orc_stats_compute.argtypes = [P(Cfg), P(State), P(Sink), C.c_int, P(Stats)]
            L.orc_timestep.restype = C.c_double
            L.orc_timestep.argtypes = [P(Cfg), P(State)]
            L.orc_density_force.restype = C.c_longlong
            L.orc_density_force.argtypes = [P(Cfg), P(State), P(Sink), C.c_int]
            L.orc_init.restype = C.c_int
            L.orc_init.argtypes = [P(Cfg), P(State), P(Region), C.c_int, P(Sink), C.c_int,
                                   P(C.c_ulonglong)]
            L.orc_step.restype = C.c_int
            L.orc_step.argtypes = [P(Cfg), P(State), P(Region), C.c_int, P(Sink), C.c_int,
                                   C.c_double, C.c_ulonglong, P(Counts), P(Stats)]
            L.orc_interp_ref.argtypes = [P(Cfg), P(State), C.c_longlong, _DP, _DP]
            L.orc_step_bins.restype = C.c_int
            L.orc_step_bins.argtypes = [P(Cfg), P(State), P(Region), C.c_int, P(Sink), C.c_int,
                                        C.c_double, C.c_int, C.c_int, P(C.c_ulonglong),
                                        P(Counts), P(C.c_longlong), P(C.c_longlong)]
            L.orc_relax.restype = C.c_int
            L.orc_relax.argtypes = [P(Cfg), P(State), P(State), P(Sink), C.c_int, C.c_int, C.c_double,
                                    _DP]
            L.orc_split_loss_grad.restype = C.c_int
            L.orc_split_loss_grad.argtypes = [P(Cfg), P(State), C.c_longlong, P(C.c_longlong), _DP,
                                              _DP, _UP, _DP, _DP, _DP]
            _lib = L
    return _lib


def make_cfg(cfg, nthreads=0, enumerate=1):
    c = Cfg()
    for k in range(3):
        c.lo[k] = cfg["box_lo"][k]
        c.hi[k] = cfg["box_hi"][k]
        c.periodic[k] = int(cfg["periodic"][k])
    for f in ("delta", "hfact", "gamma", "cs0", "qcs", "alpha_av", "beta_av", "alpha_u",
              "rsep_fac", "dnn_cap", "m0", "ccour", "cforce", "G"):
        setattr(c, f, float(cfg[f]))
    c.eos = int(cfg["eos"])
    c.lmax = int(cfg["lmax"])
    c.seed = int(cfg["seed"])
    c.nthreads = int(nthreads)
    c.enumerate = int(enumerate)
    c.kernel = int(cfg.get("kernel", 0))
    c.level_default = int(cfg.get("level_default", 0))
    return c


def make_regions(regions):
    arr = (Region * max(1, len(regions)))()
    for j, r in enumerate(regions):
        arr[j].shape = int(r["shape"])
        arr[j].axis = int(r["axis"])
        arr[j].track_sink = int(r["track_sink"])
        arr[j].nlev = len(r["R"])
        for k in range(3):
            arr[j].centre[k] = r["centre"][k]
        for k, R in enumerate(r["R"]):
            arr[j].R[k] = R
    return arr


def make_sinks(sinks):
    arr = (Sink * max(1, len(sinks)))()
    for j, s in enumerate(sinks):
        for k in range(3):
            arr[j].x[k] = s["x"][k]
            arr[j].v[k] = s["v"][k]
        arr[j].m = s["m"]
        arr[j].racc = s["racc"]
    return arr


class Oracle:
    """Holds one particle set (numpy float64 arrays with spare capacity) and runs the
    oracle's functions on it.  ``w`` is a workload dict from ``apr_synth``."""

    def __init__(self, w, capacity=None, nthreads=0, enumerate=1):
        self.L = lib()
        self.w = w
        self.cfg = make_cfg(w["cfg"], nthreads, enumerate)
        n = len(w["p"]["x"])
        cap = max(capacity or 2 * n, n)
        self.a = {}
        for f in DOUBLE_FIELDS:
            self.a[f] = np.zeros(cap, np.float64)
        self.a["level"] = np.zeros(cap, np.uint8)
        self.a["flags"] = np.zeros(cap, np.uint8)
        self.a["id"] = np.zeros(cap, np.uint64)
        self.a["bin"] = np.zeros(cap, np.uint8)
        for f, v in w["p"].items():
            self.a[f][:n] = v
        self.a["dnn"][:n] = np.inf
        self.st = State()
        self.st.n = n
        self.st.cap = cap
        self.st.next_id = int(w["p"]["id"][:n].max()) + 1 if n else 0
        for f in DOUBLE_FIELDS:
            setattr(self.st, f, self.a[f].ctypes.data_as(_DP))
        self.st.level = self.a["level"].ctypes.data_as(_UP)
        self.st.flags = self.a["flags"].ctypes.data_as(_UP)
        self.st.id = self.a["id"].ctypes.data_as(_ULP)
        self.st.bin = self.a["bin"].ctypes.data_as(_UP)
        self.regions = make_regions(w["regions"])
        self.nreg = len(w["regions"])
        self.sinks = make_sinks(w["sinks"])
        self.nsink = len(w["sinks"])
        self.step_counter = 0

    # -- views --------------------------------------------------------------
    @property
    def n(self):
        return int(self.st.n)

    def __getitem__(self, f):
        return self.a[f][: self.n]

    def mass(self):
        return self.cfg.m0 * np.ldexp(1.0, -self["level"].astype(np.int64))

    def sinks_state(self):
        return [dict(x=list(s.x), v=list(s.v), a=list(s.a), m=s.m, racc=s.racc)
                for s in self.sinks[: self.nsink]]

    def threads(self):
        return self.L.orc_threads(C.byref(self.cfg))

    # -- pieces -------------------------------------------------------------
    def threshold(self, h):
        return self.L.orc_threshold(C.byref(self.cfg), float(h))

    def quantise(self):
        xi = np.zeros((self.n, 3), np.int64)
        self.L.orc_quantise(C.byref(self.cfg), self.n, self.st.x, self.st.y, self.st.z,
                            xi.ctypes.data_as(C.POINTER(C.c_longlong)))
        return xi

    def neighbours(self, mode=0):
        """CSR lists (offsets[n+1], idx) on the quantised lattice; mode 0 gather, 1 symmetric."""
        n = self.n
        off = np.zeros(n + 1, np.int64)
        cap = 1 << 16
        while True:
            idx = np.zeros(cap, np.int32)
            tot = self.L.orc_neighbours(C.byref(self.cfg), C.byref(self.st), mode,
                                        off.ctypes.data_as(C.POINTER(C.c_longlong)),
                                        idx.ctypes.data_as(C.POINTER(C.c_int)), cap)
            if tot >= 0:
                return off, idx[:tot]
            cap = int(off[-1]) + 1

    def density(self, sample=None):
        if sample is None:
            return self.L.orc_density(C.byref(self.cfg), C.byref(self.st), None, 0)
        s = np.ascontiguousarray(sample, np.int64)
        return self.L.orc_density(C.byref(self.cfg), C.byref(self.st),
                                  s.ctypes.data_as(C.POINTER(C.c_longlong)), len(s))

    def rho_sum(self, a, h):
        out = np.zeros(2)
        self.L.orc_rho_sum(C.byref(self.cfg), C.byref(self.st), int(a), float(h),
                           out.ctypes.data_as(_DP))
        return out

    def force(self, sample=None):
        if sample is None:
            self.L.orc_force(C.byref(self.cfg), C.byref(self.st), None, 0)
        else:
            s = np.ascontiguousarray(sample, np.int64)
            self.L.orc_force(C.byref(self.cfg), C.byref(self.st),
                             s.ctypes.data_as(C.POINTER(C.c_longlong)), len(s))

    def sink_gravity(self):
        self.L.orc_sink_gravity(C.byref(self.cfg), C.byref(self.st), self.sinks, self.nsink)

    def density_force(self):
        return self.L.orc_density_force(C.byref(self.cfg), C.byref(self.st), self.sinks,
                                        self.nsink)

    def target_levels(self, x=None, y=None, z=None):
        if x is None:
            x, y, z = self["x"], self["y"], self["z"]
        x, y, z = (np.ascontiguousarray(v, np.float64) for v in (x, y, z))
        out = np.zeros(len(x), np.uint8)
        self.L.orc_target_levels(C.byref(self.cfg), self.regions, self.nreg, len(x),
                                 x.ctypes.data_as(_DP), y.ctypes.data_as(_DP),
                                 z.ctypes.data_as(_DP), out.ctypes.data_as(_UP))
        return out

    def track_regions(self):
        self.L.orc_track_regions(self.regions, self.nreg, self.sinks, self.nsink)

    def split_pass(self, level, step):
        return self.L.orc_split_pass(C.byref(self.cfg), C.byref(self.st), self.regions,
                                     self.nreg, int(level), int(step))

    def merge_pass(self, level):
        spare = C.c_longlong(-1)
        nm = self.L.orc_merge_pass(C.byref(self.cfg), C.byref(self.st), self.regions,
                                   self.nreg, int(level), C.byref(spare))
        return nm, spare.value

    def compact(self):
        return self.L.orc_compact(C.byref(self.st))

    def split_merge(self, step=None):
        if step is None:
            step = self.step_counter
            self.step_counter += 1
        cnt = Counts()
        rc = self.L.orc_split_merge(C.byref(self.cfg), C.byref(self.st), self.regions,
                                    self.nreg, int(step), C.byref(cnt))
        if rc != 0:
            raise RuntimeError("oracle split/merge: capacity exhausted")
        return cnt

    def accrete(self):
        return self.L.orc_accrete(C.byref(self.cfg), C.byref(self.st), self.sinks, self.nsink)

    def stats(self):
        s = Stats()
        self.L.orc_stats_compute(C.byref(self.cfg), C.byref(self.st), self.sinks, self.nsink,
                                 C.byref(s))
        return s

    def timestep(self):
        return self.L.orc_timestep(C.byref(self.cfg), C.byref(self.st))

    def init(self):
        st = C.c_ulonglong(self.step_counter)
        rc = self.L.orc_init(C.byref(self.cfg), C.byref(self.st), self.regions, self.nreg,
                             self.sinks, self.nsink, C.byref(st))
        self.step_counter = st.value
        if rc < 0:
            raise RuntimeError("oracle init: capacity exhausted")
        return rc

    def copy(self):
        """An independent oracle holding a copy of the current particles (e.g. the
        reference set before a split)."""
        import copy as _copy
        w = _copy.deepcopy({k: v for k, v in self.w.items() if k != "p"})
        w["p"] = {f: self.a[f][: self.n].copy() for f in ("x", "y", "z", "vx", "vy", "vz", "u", "h",
                                                            "level", "flags", "id")}
        o = Oracle(w, capacity=self.st.cap)
        for f in DOUBLE_FIELDS:
            o.a[f][: self.n] = self.a[f][: self.n]
        o.st.next_id = self.st.next_id
        return o

    def interp_ref(self, pts):
        """This oracle's accelerations interpolated (SPH, each particle at its own h)
        to the points pts (k x 3)."""
        pts = np.ascontiguousarray(pts, np.float64).reshape(-1, 3)
        out = np.zeros_like(pts)
        self.L.orc_interp_ref(C.byref(self.cfg), C.byref(self.st), len(pts), pts.ctypes.data_as(_DP),
                              out.ctypes.data_as(_DP))
        return out

    def relax(self, ref, max_iter=50, tol=0.005):
        """Relaxing (Sec. 2.4) of the particles flagged NEW towards the reference
        oracle ``ref`` (its positions, h, density and accelerations); returns
        (shuffles done, last / first shuffle energy)."""
        ratio = C.c_double(0.0)
        it = self.L.orc_relax(C.byref(self.cfg), C.byref(self.st), C.byref(ref.st), self.sinks,
                              self.nsink, int(max_iter), float(tol), C.byref(ratio))
        return it, ratio.value

    def split_loss_grad(self, parent, d, hc, want=None):
        """Density error J of splitting ``parent[k]`` into children at x_p +- d[k] with
        smoothing lengths hc[2k], hc[2k+1], against the current particles as the
        reference set; returns (J, dJ/dd (k x 3), dJ/dhc (2k)).  ``want`` (bool per split)
        restricts the gradient to those splits (the rest are 0)."""
        par = np.ascontiguousarray(parent, np.int64)
        k = len(par)
        dd = np.ascontiguousarray(np.reshape(d, (k, 3)), np.float64)
        hh = np.ascontiguousarray(hc, np.float64)
        if hh.shape != (2 * k,):
            raise ValueError("hc needs two smoothing lengths per split")
        wnt = None if want is None else np.ascontiguousarray(want, np.uint8)
        J = C.c_double(0.0)
        gd = np.zeros((k, 3))
        gh = np.zeros(2 * k)
        rc = self.L.orc_split_loss_grad(
            C.byref(self.cfg), C.byref(self.st), k, par.ctypes.data_as(C.POINTER(C.c_longlong)),
            dd.ctypes.data_as(_DP), hh.ctypes.data_as(_DP),
            None if wnt is None else wnt.ctypes.data_as(_UP), C.byref(J), gd.ctypes.data_as(_DP),
            gh.ctypes.data_as(_DP))
        if rc != 0:
            raise ValueError("split_loss_grad: parent out of range, dead or repeated")
        return J.value, gd, gh

    def step_bins(self, dt_max, B, init_bins=False):
        """One step of length dt_max with individual time steps in bins 0..B
        (Sec. 2.5); returns (counts, force updates, saturated updates)."""
        cnt = Counts()
        st = C.c_ulonglong(self.step_counter)
        upd, sat = C.c_longlong(0), C.c_longlong(0)
        rc = self.L.orc_step_bins(C.byref(self.cfg), C.byref(self.st), self.regions, self.nreg,
                                  self.sinks, self.nsink, float(dt_max), int(B),
                                  1 if init_bins else 0, C.byref(st), C.byref(cnt), C.byref(upd),
                                  C.byref(sat))
        self.step_counter = st.value
        if rc != 0:
            raise RuntimeError("oracle step_bins: capacity exhausted")
        return cnt, upd.value, sat.value

    def step(self, dt):
        cnt, stt = Counts(), Stats()
        rc = self.L.orc_step(C.byref(self.cfg), C.byref(self.st), self.regions, self.nreg,
                             self.sinks, self.nsink, float(dt), self.step_counter,
                             C.byref(cnt), C.byref(stt))
        self.step_counter += 1
        if rc != 0:
            raise RuntimeError("oracle step: capacity exhausted")
        return cnt, stt


def kernel_m4(q):
    out = np.zeros(2)
    lib().orc_kernel_m4(float(q), out.ctypes.data_as(_DP))
    return out


def kernel_shape(kernel, q):
    """f(q), f'(q) of kernel 0 (M4) or 1 (Wendland C2)."""
    out = np.zeros(2)
    lib().orc_kernel(int(kernel), float(q), out.ctypes.data_as(_DP))
    return out


def splitmix64(z):
    return lib().orc_splitmix64(int(z))


def split_uniform(seed, pid, step):
    return lib().orc_split_uniform(int(seed), int(pid), int(step))


def split_direction(region, p, t):
    reg = make_regions([region])
    pp = np.ascontiguousarray(p, np.float64)
    w = np.zeros(3)
    lib().orc_split_direction(reg, pp.ctypes.data_as(_DP), float(t), w.ctypes.data_as(_DP))
    return w


def pair_tree(xi, order=None):
    """Pairs (k x 2 array of indices into xi) from the pairing tree on all rows of xi."""
    xi = np.ascontiguousarray(xi, np.int64)
    m = len(xi)
    s = np.ascontiguousarray(np.arange(m) if order is None else order, np.int64)
    rc = lib().orc_pair_tree(xi.ctypes.data_as(C.POINTER(C.c_longlong)),
                             s.ctypes.data_as(C.POINTER(C.c_longlong)), m)
    if rc != 0:
        raise ValueError("pair_tree needs an even count")
    return s.reshape(-1, 2)
