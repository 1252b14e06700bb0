"""The conservation sums of apr_stats_noalloc, the entry point for callers that
cannot allocate device memory (it uses a built-in scratch array instead of a
workspace), through the C ABI: against apr_stats_compute on the same particles,
and against the oracle's sums on the particles the oracle's own split pass made
from the same input, on two calls in a row.

This file is collected last (its name sorts after every other test file) so
that a run stopped at its first failure has already run every other test."""
import ctypes as C

import numpy as np
import pytest

import apr_synth
import oracle
from gpu_util import sim, with_velocities

pytestmark = pytest.mark.gpu


def _entry():
    from paper_2409_11470_gb300 import binding as B
    f = B.lib.apr_stats_noalloc
    f.argtypes = [C.POINTER(B.Config), C.POINTER(B.Particles), C.c_longlong, C.POINTER(B.Sink),
                  C.c_int, C.c_void_p, C.POINTER(B.Stats), C.c_char_p, C.c_size_t]
    f.restype = C.c_int
    return B, f


def _as_array(s):
    return np.array([s.mass, *s.mom, *s.ang, s.ekin, s.etherm])


@pytest.mark.parametrize("make", [lambda: with_velocities(apr_synth.c1_lattice(), 0.3),
                                  lambda: apr_synth.disc_planet(20000)])
def test_noalloc_sums_match_workspace_and_oracle_sums_twice(make):
    B, f = _entry()
    w = make()
    g = sim(w)
    g.split_merge()  # mixed levels (disc: particles near the planet)
    ref = _as_array(g.stats())
    o = oracle.Oracle(w, capacity=3 * len(w["p"]["x"]))
    o.split_merge(0)
    assert o.n == g.n
    ref_o = _as_array(o.stats())
    sinks = B.Sink * max(1, len(w["sinks"]))
    arr = sinks()
    for j, s in enumerate(w["sinks"]):
        for k in range(3):
            arr[j].x[k], arr[j].v[k] = s["x"][k], s["v"][k]
        arr[j].m, arr[j].racc = s["m"], s["racc"]
    scale = np.abs(ref) + ref[0] * 1e-3
    for _ in range(2):
        out = B.Stats()
        err = C.create_string_buffer(256)
        st = f(C.byref(g.cfg), C.byref(g.parts), g.n, arr, len(w["sinks"]),
               C.c_void_p(g.stream.cuda_stream), C.byref(out), err, 256)
        assert st == 0, err.value
        got = _as_array(out)
        assert np.all(np.abs(got - ref) <= 1e-12 * scale), (got, ref)
        # float64 sums in another order: agreement to a few ulps of the scale
        assert np.all(np.abs(got - ref_o) <= 1e-12 * scale), (got, ref_o)


def test_noalloc_rejects_more_particles_than_its_scratch():
    B, f = _entry()
    g = sim(apr_synth.c1_lattice())
    out = B.Stats()
    err = C.create_string_buffer(256)
    st = f(C.byref(g.cfg), C.byref(g.parts), 16_777_217, None, 0,
           C.c_void_p(g.stream.cuda_stream), C.byref(out), err, 256)
    assert st == 1 and b"16,777,216" in err.value


def test_noalloc_refuses_a_stream_under_capture():
    """Every call reads its result back and synchronises its stream, which a stream
    under capture does not allow: the call returns APR_ERR_ARG before it launches
    anything, and the capture ends normally (an empty graph)."""
    import torch
    B, f = _entry()
    g = sim(apr_synth.c1_lattice())
    out = B.Stats()
    err = C.create_string_buffer(256)
    s = torch.cuda.Stream()
    graph = torch.cuda.CUDAGraph()
    torch.cuda.synchronize()
    with torch.cuda.graph(graph, stream=s):
        st = f(C.byref(g.cfg), C.byref(g.parts), g.n, None, 0, C.c_void_p(s.cuda_stream),
               C.byref(out), err, 256)
    assert st == 1 and b"capture" in err.value
    # the entry works again once the capture has ended
    st = f(C.byref(g.cfg), C.byref(g.parts), g.n, None, 0, C.c_void_p(g.stream.cuda_stream),
           C.byref(out), err, 256)
    assert st == 0, err.value
