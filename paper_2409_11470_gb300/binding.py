"""ctypes binding of the C ABI in ``include/apr.h`` (argument marshalling only).

Every step of the hot path runs in the CUDA library ``libapr.so``; this module
only allocates device memory with PyTorch, passes raw pointers and sizes, and
turns status codes into exceptions.  It raises at import time if the library
has not been built (there is no CPU fallback).
"""
from __future__ import annotations

import ctypes as C
import os
import re

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libapr.so")
HEADER = os.path.join(os.path.dirname(HERE), "include", "apr.h")

MAXLEV, MAXREG, MAXSINK = 8, 8, 8
FLAG_CHANGED, FLAG_FIXED, FLAG_DEAD, FLAG_NEW = 1, 2, 4, 8
PREC = {"fp32": 0, "fp64": 1}
STATUS = {0: "OK", 1: "ERR_ARG", 2: "ERR_CAPACITY", 3: "ERR_NR_NOCONV", 4: "ERR_NEIGH_OVERFLOW",
          5: "ERR_CUDA", 6: "ERR_STATE", 7: "ERR_WORKSPACE"}
F64_FIELDS = ("x", "y", "z", "vx", "vy", "vz", "u", "h", "rho", "omega", "ax", "ay", "az", "dudt",
              "vsig", "dnn", "pres", "cs")


class Config(C.Structure):
    _fields_ = [("box_lo", C.c_double * 3), ("box_hi", C.c_double * 3), ("periodic", C.c_int * 3),
                ("delta", C.c_double), ("hfact", C.c_double), ("gamma", C.c_double),
                ("eos", C.c_int), ("cs0", C.c_double), ("qcs", C.c_double),
                ("alpha_av", C.c_double), ("beta_av", C.c_double), ("alpha_u", C.c_double),
                ("rsep_fac", C.c_double), ("dnn_cap", C.c_double), ("m0", C.c_double),
                ("lmax", C.c_int), ("seed", C.c_ulonglong), ("ccour", C.c_double),
                ("cforce", C.c_double), ("G", C.c_double), ("precision", C.c_int),
                ("nr_tol", C.c_double), ("nr_maxit", C.c_int), ("max_neigh", C.c_int),
                ("kernel", C.c_int), ("level_default", C.c_int),
                ("fused_density", C.c_int)]


class Region(C.Structure):
    _fields_ = [("shape", C.c_int), ("axis", C.c_int), ("track_sink", C.c_int), ("nlev", C.c_int),
                ("centre", C.c_double * 3), ("R", C.c_double * MAXLEV)]


class Sink(C.Structure):
    _fields_ = [("x", C.c_double * 3), ("v", C.c_double * 3), ("a", C.c_double * 3),
                ("m", C.c_double), ("racc", C.c_double)]


class Particles(C.Structure):
    _fields_ = [(f, C.c_void_p) for f in F64_FIELDS] + \
        [("level", C.c_void_p), ("flags", C.c_void_p), ("id", C.c_void_p), ("bin", C.c_void_p)]


class Counts(C.Structure):
    _fields_ = [("n_split", C.c_longlong * MAXLEV), ("n_merge", C.c_longlong * MAXLEV),
                ("n_spare", C.c_longlong * MAXLEV), ("n_accreted", C.c_longlong),
                ("n_dead", C.c_longlong)]


class Stats(C.Structure):
    _fields_ = [("mass", C.c_double), ("mom", C.c_double * 3), ("ang", C.c_double * 3),
                ("ekin", C.c_double), ("etherm", C.c_double)]


NPROF = 8
PROF_GROUPS = ("sort", "tree", "lists", "density", "force", "refine", "other")


class Profile(C.Structure):
    _fields_ = [("ms", C.c_double * NPROF), ("calls", C.c_longlong * NPROF),
                ("pairs", C.c_double * NPROF), ("launches", C.c_longlong),
                ("density_attempts", C.c_longlong), ("uncovered", C.c_longlong),
                ("shrunk", C.c_longlong)]


class AprError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: build the CUDA library first "
                          "(python -c 'import __graft_entry__ as g; g.build()')")
    L = C.CDLL(LIB_PATH)
    P = C.POINTER
    vp, ll, i32 = C.c_void_p, C.c_longlong, C.c_int
    sig = {
        "apr_create": [P(vp), P(Config), vp],
        "apr_destroy": [vp],
        "apr_last_error": [vp],
        "apr_workspace_size": [P(Config), ll, P(C.c_size_t)],
        "apr_bind": [vp, P(Particles), ll, ll, ll, vp, C.c_size_t],
        "apr_upload": [vp, P(Particles), ll],
        "apr_download": [vp, P(Particles), ll, P(ll)],
        "apr_set_regions": [vp, P(Region), i32],
        "apr_set_sinks": [vp, P(Sink), i32],
        "apr_get_sinks": [vp, P(Sink), i32],
        "apr_get_count": [vp, P(ll), P(ll), P(C.c_ulonglong)],
        "apr_init": [vp, P(Region), i32, P(i32)],
        "apr_split_merge": [vp, P(ll), P(Counts)],
        "apr_sph_density": [vp, P(ll)],
        "apr_sph_force": [vp],
        "apr_step": [vp, C.c_double, P(C.c_double), P(Stats), P(Counts)],
        "apr_timestep": [vp, P(C.c_double)],
        "apr_stats_compute": [vp, P(Stats)],
        "apr_reorder": [vp],
        "apr_neighbour_lists": [vp, i32, P(ll), P(i32), ll, P(ll)],
        "apr_merge_pairs": [vp, i32, P(ll), ll, P(ll), P(ll)],
        "apr_profile_enable": [vp, i32],
        "apr_profile_read": [vp, P(Profile), i32],
        "apr_density_loss_grad": [vp, ll, vp, vp, vp, P(C.c_double), vp, vp],
        "apr_relax": [vp, P(Particles), ll, i32, C.c_double, P(i32), P(C.c_double)],
        "apr_step_bins": [vp, C.c_double, i32, i32, P(Counts), P(ll), P(ll), P(Stats)],
        "apr_probe_fma_peak": [i32, i32, vp, P(C.c_double), P(C.c_double)],
    }
    for name, args in sig.items():
        f = getattr(L, name)
        f.argtypes = args
        f.restype = None if name == "apr_destroy" else (C.c_char_p if name == "apr_last_error"
                                                         else C.c_int)
    return L


lib = _load()


def probe_fma_peak(precision="fp32", iters=None, stream=None):
    """Measured rate of the FP32 (or FP64) fused multiply-add pipes of the current
    GPU (apr_probe_fma_peak): returns (TFLOP/s, ms of the timed launch)."""
    fp64 = precision == "fp64"
    it = int(iters or (1000 if fp64 else 40000))
    tf, ms = C.c_double(), C.c_double()
    st = C.c_void_p(stream.cuda_stream if stream is not None else 0)
    rc = lib.apr_probe_fma_peak(1 if fp64 else 0, it, st, C.byref(tf), C.byref(ms))
    if rc != 0:
        raise AprError(rc, "apr_probe_fma_peak failed")
    return tf.value, ms.value


def header_symbols():
    """Entry points declared in include/apr.h."""
    with open(HEADER) as f:
        src = f.read()
    return sorted(set(re.findall(r"^\s*(?:apr_status|void|const char\*)\s+(apr_\w+)\s*\(", src,
                                 re.M)))


def make_config(cfg, precision="fp32", nr_tol=0.0, nr_maxit=0, max_neigh=0):
    c = Config()
    for k in range(3):
        c.box_lo[k] = cfg["box_lo"][k]
        c.box_hi[k] = cfg["box_hi"][k]
        c.periodic[k] = int(cfg["periodic"][k])
    for f in ("delta", "hfact", "gamma", "cs0", "qcs", "alpha_av", "beta_av", "alpha_u",
              "rsep_fac", "dnn_cap", "m0", "ccour", "cforce", "G"):
        setattr(c, f, float(cfg[f]))
    c.eos = int(cfg["eos"])
    c.lmax = int(cfg["lmax"])
    c.seed = int(cfg["seed"])
    c.precision = PREC[precision]
    c.nr_tol = float(nr_tol)
    c.nr_maxit = int(nr_maxit)
    c.max_neigh = int(max_neigh)
    c.kernel = int(cfg.get("kernel", 0))
    c.level_default = int(cfg.get("level_default", 0))
    c.fused_density = int(cfg.get("fused_density", 0))
    return c


def workspace_size(cfg, capacity):
    out = C.c_size_t(0)
    st = lib.apr_workspace_size(C.byref(cfg), int(capacity), C.byref(out))
    if st != 0:
        raise AprError(st, "workspace size")
    return out.value


def _regions(regs):
    arr = (Region * max(1, len(regs)))()
    for j, r in enumerate(regs):
        arr[j].shape, arr[j].axis = int(r["shape"]), int(r["axis"])
        arr[j].track_sink, arr[j].nlev = int(r["track_sink"]), len(r["R"])
        for k in range(3):
            arr[j].centre[k] = r["centre"][k]
        for k, R in enumerate(r["R"]):
            arr[j].R[k] = R
    return arr


def _sinks(sinks):
    arr = (Sink * max(1, len(sinks)))()
    for j, s in enumerate(sinks):
        for k in range(3):
            arr[j].x[k], arr[j].v[k] = s["x"][k], s["v"][k]
        arr[j].m, arr[j].racc = s["m"], s["racc"]
    return arr


class Simulation:
    """One particle set on the GPU bound to a library context.

    ``w`` is a workload dict (``cfg``, ``regions``, ``sinks``, ``p`` with numpy
    arrays).  Particle arrays and the workspace are torch CUDA tensors owned
    here; all computation happens in ``libapr.so`` on ``stream`` (default: the
    current torch stream).
    """

    def __init__(self, w, capacity=None, precision="fp32", device="cuda", stream=None,
                 nr_tol=0.0, nr_maxit=0, max_neigh=0):
        import torch
        self.torch = torch
        n = len(w["p"]["x"])
        cap = int(capacity or max(2 * n, 64))
        self.device = torch.device(device)
        self.cfg = make_config(w["cfg"], precision, nr_tol, nr_maxit, max_neigh)
        self.precision = precision
        self.t = {}
        for f in F64_FIELDS:
            self.t[f] = torch.zeros(cap, dtype=torch.float64, device=self.device)
        self.t["level"] = torch.zeros(cap, dtype=torch.uint8, device=self.device)
        self.t["flags"] = torch.zeros(cap, dtype=torch.uint8, device=self.device)
        self.t["id"] = torch.zeros(cap, dtype=torch.int64, device=self.device)
        self.t["bin"] = torch.zeros(cap, dtype=torch.uint8, device=self.device)
        for f, v in w["p"].items():
            src = torch.from_numpy(np.ascontiguousarray(v).view(np.int64) if f == "id" else
                                   np.ascontiguousarray(v))
            self.t[f][:n].copy_(src)
        self.t["dnn"][:n] = float("inf")
        self.cap = cap
        self.ws_bytes = workspace_size(self.cfg, cap)
        self.ws = torch.empty(self.ws_bytes + 256, dtype=torch.uint8, device=self.device)
        base = self.ws.data_ptr()
        self.ws_ptr = (base + 255) & ~255
        if stream is None:
            stream = torch.cuda.current_stream(self.device)
        self.stream = stream
        self.ctx = C.c_void_p()
        self._check(lib.apr_create(C.byref(self.ctx), C.byref(self.cfg),
                                   C.c_void_p(stream.cuda_stream)), "create")
        self.parts = Particles(**{f: C.c_void_p(self.t[f].data_ptr()) for f in self.t})
        next_id = int(np.max(w["p"]["id"])) + 1 if n else 0
        self._check(lib.apr_bind(self.ctx, C.byref(self.parts), n, cap, next_id,
                                 C.c_void_p(self.ws_ptr), self.ws_bytes), "bind")
        self.set_regions(w["regions"])
        self.set_sinks(w["sinks"])

    # -- host exchange ----------------------------------------------------------
    def host_buffers(self, pinned=True):
        """Host tensors (page-locked by default) of the bound fields, capacity long,
        for upload / download."""
        return {f: self.torch.empty(self.cap, dtype=t.dtype, pin_memory=pinned)
                for f, t in self.t.items()}

    def upload(self, host, n):
        """Copy n particles from the host tensors `host` (field -> CPU tensor; missing
        fields are skipped) into the bound arrays (apr_upload)."""
        parts = Particles(**{f: C.c_void_p(host[f].data_ptr()) for f in self.t if f in host})
        self._check(lib.apr_upload(self.ctx, C.byref(parts), int(n)), "upload")

    def download(self, host):
        """Copy the current particles into the host tensors `host` (apr_download);
        returns the particle count."""
        cap = min(int(t.numel()) for t in host.values())
        parts = Particles(**{f: C.c_void_p(host[f].data_ptr()) for f in self.t if f in host})
        n = C.c_longlong(0)
        self._check(lib.apr_download(self.ctx, C.byref(parts), cap, C.byref(n)), "download")
        return n.value

    # -- plumbing ---------------------------------------------------------------
    def _check(self, st, what):
        if st != 0:
            msg = lib.apr_last_error(self.ctx).decode() if self.ctx else what
            raise AprError(st, f"{what}: {msg}")

    def close(self):
        if self.ctx:
            lib.apr_destroy(self.ctx)
            self.ctx = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_regions(self, regs):
        self._check(lib.apr_set_regions(self.ctx, _regions(regs), len(regs)), "set_regions")

    def set_sinks(self, sinks):
        self._check(lib.apr_set_sinks(self.ctx, _sinks(sinks), len(sinks)), "set_sinks")
        self.nsinks = len(sinks)

    def sinks(self):
        out = (Sink * MAXSINK)()
        self._check(lib.apr_get_sinks(self.ctx, out, self.nsinks), "get_sinks")
        return [dict(x=list(s.x), v=list(s.v), a=list(s.a), m=s.m, racc=s.racc)
                for s in out[: self.nsinks]]

    def counts(self):
        n, nid, st = C.c_longlong(), C.c_longlong(), C.c_ulonglong()
        self._check(lib.apr_get_count(self.ctx, C.byref(n), C.byref(nid), C.byref(st)), "count")
        return n.value, nid.value, st.value

    @property
    def n(self):
        return self.counts()[0]

    def get(self, f):
        """Current values of one field as a numpy array (synchronises)."""
        self.stream.synchronize()
        a = self.t[f][: self.n].cpu().numpy()
        return a.view(np.uint64) if f == "id" else a

    # -- hot path ---------------------------------------------------------------
    def init(self, regions=None):
        """Initial refinement (apr_init); ``regions`` (a list of zone dicts) replaces the
        zones set so far, None keeps them."""
        p = C.c_int(0)
        if regions is None:
            self._check(lib.apr_init(self.ctx, None, 0, C.byref(p)), "init")
        else:
            self._check(lib.apr_init(self.ctx, _regions(regions), len(regions), C.byref(p)), "init")
        return p.value

    def density(self):
        nu = C.c_longlong(0)
        self._check(lib.apr_sph_density(self.ctx, C.byref(nu)), "density")
        return nu.value

    def force(self):
        self._check(lib.apr_sph_force(self.ctx), "force")

    def split_merge(self):
        n, cnt = C.c_longlong(), Counts()
        self._check(lib.apr_split_merge(self.ctx, C.byref(n), C.byref(cnt)), "split_merge")
        return cnt

    def step(self, dt=0.0):
        used, st, cnt = C.c_double(), Stats(), Counts()
        self._check(lib.apr_step(self.ctx, float(dt), C.byref(used), C.byref(st), C.byref(cnt)),
                    "step")
        return used.value, st, cnt

    def step_bins(self, dt_max, max_bin, init_bins=False):
        """One step of dt_max with individual time steps in bins 0..max_bin
        (Sec. 2.5); returns (counts, force updates, saturated updates, stats)."""
        cnt, st = Counts(), Stats()
        upd, sat = C.c_longlong(0), C.c_longlong(0)
        self._check(lib.apr_step_bins(self.ctx, float(dt_max), int(max_bin), 1 if init_bins else 0,
                                      C.byref(cnt), C.byref(upd), C.byref(sat), C.byref(st)),
                    "step_bins")
        return cnt, upd.value, sat.value, st

    def timestep(self):
        dt = C.c_double()
        self._check(lib.apr_timestep(self.ctx, C.byref(dt)), "timestep")
        return dt.value

    def stats(self):
        st = Stats()
        self._check(lib.apr_stats_compute(self.ctx, C.byref(st)), "stats")
        return st

    def reorder(self):
        """Permute the bound arrays into the index's Morton order (apr_reorder);
        ids travel with their particles."""
        self._check(lib.apr_reorder(self.ctx), "reorder")

    def neighbour_lists(self, mode=0, cap=None):
        n = self.n
        off = np.zeros(n + 1, np.int64)
        cap = int(cap or max(1, n * 96))
        while True:
            idx = np.zeros(cap, np.int32)
            tot = C.c_longlong(0)
            st = lib.apr_neighbour_lists(self.ctx, int(mode),
                                         off.ctypes.data_as(C.POINTER(C.c_longlong)),
                                         idx.ctypes.data_as(C.POINTER(C.c_int)), cap,
                                         C.byref(tot))
            if st == 4 and tot.value > cap:
                cap = tot.value
                continue
            self._check(st, "neighbour_lists")
            return off, idx[: tot.value]

    def profile_enable(self, on=True):
        self._check(lib.apr_profile_enable(self.ctx, 1 if on else 0), "profile_enable")

    def profile(self, reset=False):
        """Per-group device ms, timed calls and pair evaluations, plus the launch count."""
        pr = Profile()
        self._check(lib.apr_profile_read(self.ctx, C.byref(pr), 1 if reset else 0), "profile")
        out = {g: dict(ms=pr.ms[k], calls=pr.calls[k], pairs=pr.pairs[k])
               for k, g in enumerate(PROF_GROUPS)}
        out["launches"] = pr.launches
        out["density_attempts"] = pr.density_attempts
        out["uncovered"] = pr.uncovered
        out["shrunk"] = pr.shrunk
        return out

    def density_loss_grad(self, parent, d, hc):
        """Density error J of splitting ``parent[k]`` into children at x_p +- d[k] with
        smoothing lengths hc[2k], hc[2k+1] (the current particles are the reference
        set), and its gradients: returns (J, dJ/dd (k x 3), dJ/dhc (2k)) with the
        gradients as float64 tensors on the device."""
        torch = self.torch
        dev = self.device
        par = torch.as_tensor(parent, dtype=torch.int64, device=dev).contiguous()
        k = par.numel()
        dd = torch.as_tensor(d, dtype=torch.float64, device=dev).reshape(k, 3).contiguous()
        hh = torch.as_tensor(hc, dtype=torch.float64, device=dev).reshape(2 * k).contiguous()
        gd = torch.empty((k, 3), dtype=torch.float64, device=dev)
        gh = torch.empty(2 * k, dtype=torch.float64, device=dev)
        J = C.c_double(0.0)
        self._check(lib.apr_density_loss_grad(self.ctx, k, C.c_void_p(par.data_ptr()),
                                              C.c_void_p(dd.data_ptr()), C.c_void_p(hh.data_ptr()),
                                              C.byref(J), C.c_void_p(gd.data_ptr()),
                                              C.c_void_p(gh.data_ptr())), "density_loss_grad")
        return J.value, gd, gh

    REF_FIELDS = ("x", "y", "z", "h", "rho", "ax", "ay", "az", "level", "flags")

    def snapshot(self):
        """Device copies of the current particles' positions, h, density,
        accelerations, levels and flags: the reference set for ``relax``."""
        n = self.n
        self.stream.synchronize()
        return {f: self.t[f][:n].clone() for f in self.REF_FIELDS}

    def relax(self, ref, max_iter=50, tol=0.005):
        """Relaxing (Sec. 2.4) of the particles flagged NEW towards the reference
        set ``ref`` (a ``snapshot`` taken before the split/merge); returns
        (shuffles done, last / first shuffle energy)."""
        nref = int(ref["x"].numel())
        parts = Particles(**{f: C.c_void_p(ref[f].data_ptr()) for f in self.REF_FIELDS})
        it, ratio = C.c_int(0), C.c_double(0.0)
        self._check(lib.apr_relax(self.ctx, C.byref(parts), nref, int(max_iter), float(tol),
                                  C.byref(it), C.byref(ratio)), "relax")
        return it.value, ratio.value

    def merge_pairs(self, level):
        n = self.n
        cap = max(1, n // 2)
        pairs = np.zeros(2 * cap, np.int64)
        npairs, spare = C.c_longlong(0), C.c_longlong(-1)
        self._check(lib.apr_merge_pairs(self.ctx, int(level),
                                        pairs.ctypes.data_as(C.POINTER(C.c_longlong)), cap,
                                        C.byref(npairs), C.byref(spare)), "merge_pairs")
        return pairs[: 2 * npairs.value].reshape(-1, 2), spare.value


def _loss_function():
    import torch

    class SplitDensityLoss(torch.autograd.Function):
        """J(d, hc) of one split pass as an autograd op.  The forward call runs the
        library's density-error forward and reverse sweeps (apr_density_loss_grad)
        and keeps both gradients; backward only scales them by the incoming
        gradient of J."""

        @staticmethod
        def forward(ctx, d, hc, sim, parent):
            J, gd, gh = sim.density_loss_grad(parent, d.detach(), hc.detach())
            ctx.save_for_backward(gd, gh)
            return torch.tensor(J, dtype=torch.float64, device=d.device)

        @staticmethod
        def backward(ctx, gJ):
            gd, gh = ctx.saved_tensors
            return gJ * gd, gJ * gh, None, None

    return SplitDensityLoss


_LOSS_FN = None


def split_density_loss(sim, parent, d, hc):
    """Differentiable J for ``torch.autograd``: gradients flow to ``d`` (k x 3) and
    ``hc`` (2k), both float64 tensors on the simulation's device."""
    global _LOSS_FN
    if _LOSS_FN is None:
        _LOSS_FN = _loss_function()
    return _LOSS_FN.apply(d, hc, sim, parent)
