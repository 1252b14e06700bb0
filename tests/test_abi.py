"""The C-ABI library loads and exports every entry point include/apr.h declares;
argument checks that need no GPU (not GPU)."""
import ctypes as C

import apr_synth
from paper_2409_11470_gb300 import binding as B


def test_library_exports_every_declared_symbol():
    declared = B.header_symbols()
    assert len(declared) >= 15
    for name in declared:
        assert hasattr(B.lib, name), name


def test_workspace_size_grows_with_capacity_and_lists():
    cfg = B.make_config(apr_synth.c1_lattice()["cfg"])
    a = B.workspace_size(cfg, 1000)
    b = B.workspace_size(cfg, 2000)
    assert 0 < a < b and a % 256 == 0
    cfg2 = B.make_config(apr_synth.c1_lattice()["cfg"], max_neigh=1024)
    assert B.workspace_size(cfg2, 1000) > a
    cfg64 = B.make_config(apr_synth.c1_lattice()["cfg"], precision="fp64")
    assert B.workspace_size(cfg64, 1000) > a


def test_create_rejects_bad_configs_before_touching_the_gpu():
    base = apr_synth.c1_lattice()["cfg"]
    bad = []
    c = dict(base, delta=0.0)
    bad.append(c)
    c = dict(base, box_hi=[1.0, 1.0, 1.0 + 1e-9])  # periodic length not whole lattice units
    bad.append(c)
    c = dict(base, lmax=9)
    bad.append(c)
    c = dict(base, delta=2.0 ** -31)  # more than 2^30 lattice units
    bad.append(c)
    cfgs = [B.make_config(cfg) for cfg in bad]
    # list capacities must be multiples of 4 (rows written 16 bytes at a time)
    cfgs += [B.make_config(base, max_neigh=6), B.make_config(base, max_neigh=-4)]
    for cfg in cfgs:
        ctx = C.c_void_p()
        st = B.lib.apr_create(C.byref(ctx), C.byref(cfg), None)
        assert st == 1 and not ctx.value


def test_null_arguments_rejected():
    assert B.lib.apr_create(None, None, None) == 1
    assert B.lib.apr_workspace_size(None, 10, None) == 1
    assert B.lib.apr_sph_density(None, None) == 1
    parts = B.Particles()
    assert B.lib.apr_upload(None, C.byref(parts), 0) == 1
    assert B.lib.apr_download(None, C.byref(parts), 0, None) == 1
