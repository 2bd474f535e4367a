"""The C-ABI library builds, loads and exports every entry point the header
declares; host-side argument checks work without a GPU (no compute calls)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_1803_01516_gb300 import build
    build.build()
    from paper_1803_01516_gb300 import gazecut
    return gazecut.lib()


def _declared():
    names = []
    inc = os.path.join(ROOT, "include")
    for f in sorted(os.listdir(inc)):
        if f.endswith(".h"):
            txt = open(os.path.join(inc, f)).read()
            names += re.findall(r"GS_API\s+[\w\s\*]+?\b(gs_\w+)\s*\(", txt)
    return names


def test_header_declares_the_pipeline():
    names = _declared()
    for n in ["gs_stereo_cost_volume", "gs_build_graph", "gs_maxflow_solve", "gs_extract_labels"]:
        assert n in names


def test_every_declared_symbol_is_exported(lib):
    for name in _declared():
        assert hasattr(lib, name), name


def test_binding_lists_every_export():
    from paper_1803_01516_gb300 import gazecut
    assert sorted(gazecut.EXPORTS) == sorted(_declared())


def test_sizes_and_param_validation(lib):
    from paper_1803_01516_gb300 import gazecut as gc
    p = gc.Params(w=384, h=288, D=16, tau=30, lam=10)
    assert gc.gs_num_nodes(p) == 354 * 288 * 15
    assert gc.gs_cost_volume_bytes(p) == 4 * 288 * 354 * 16
    assert gc.gs_graph_bytes(p) >= 36 * 354 * 288 * 15
    # the paper's cuboid: 372 x 288 sites x 24 depth numbers -> 372*288*23 nodes
    p2 = gc.Params(w=372 + 46, h=288, D=24, tau=30, lam=14)
    assert gc.gs_num_nodes(p2) + 2 == 2464130
    for bad in [gc.Params(w=30, h=4, D=16, tau=1, lam=1),         # n_g <= 0
                gc.Params(w=64, h=4, D=1, tau=1, lam=1),          # D < 2
                gc.Params(w=64, h=0, D=4, tau=1, lam=1),
                gc.Params(w=64, h=4, D=4, tau=1, lam=-1),
                gc.Params(w=64, h=4, D=4, tau=1, lam=1, dis0=5)]:  # dis0 < 2(D-1)
        assert gc.gs_graph_bytes(bad) == 0
        assert gc.gs_num_nodes(bad) == 0


def test_null_pointers_rejected_on_host(lib):
    """Invalid arguments are refused before any launch (no GPU needed)."""
    from paper_1803_01516_gb300 import gazecut as gc
    p = gc.Params(w=64, h=8, D=4, tau=30, lam=2).c()
    o = gc.SolveOpts().c()
    assert lib.gs_stereo_cost_volume(None, None, 64, ctypes.byref(p), None, None) == gc.GS_ERR_INVAL
    assert lib.gs_build_graph(None, ctypes.byref(p), None, None, None) == gc.GS_ERR_INVAL
    assert lib.gs_maxflow_solve(None, ctypes.byref(p), ctypes.byref(o), None, None, None) == gc.GS_ERR_INVAL
    assert lib.gs_extract_labels(None, ctypes.byref(p), ctypes.byref(o), None, None, None, None,
                                 None) == gc.GS_ERR_INVAL
    assert lib.gs_energy(None, None, ctypes.byref(p), None, None) == gc.GS_ERR_INVAL
    bad_o = gc.SolveOpts(sweeps_per_relabel=0).c()
    fake = ctypes.c_void_p(256)
    assert lib.gs_maxflow_solve(fake, ctypes.byref(p), ctypes.byref(bad_o), fake, fake,
                                None) == gc.GS_ERR_INVAL


def test_product_path_does_not_import_the_oracle():
    pkg = os.path.join(ROOT, "paper_1803_01516_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                txt = open(os.path.join(dirpath, f)).read()
                assert not re.search(r"^\s*(import|from)\s+oracle", txt, re.M), f
                assert "gazecut_oracle" not in txt, f


def test_delegate_params_on_host(lib):
    """Delegate problem sizes and weights of the level-1 approximation (§4.5)
    are computed on the host; bad block sizes are refused."""
    from paper_1803_01516_gb300 import gazecut as gc
    p = gc.Params(w=384, h=288, D=16, tau=30, lam=10, inhibit=1023)
    q = gc.gs_delegate_params(p, 3)
    assert (q.ng, q.h, q.D) == (118, 96, 6)
    assert (q.lam, q.inhibit, q.vertical_inhibit) == (30, 3069, 1)
    assert gc.gs_delegate_params(p, 1).c().w == p.c().w
    out = gc.GsParams()
    for b in (0, 16, -1):
        assert lib.gs_delegate_params(ctypes.byref(p.c()), b, ctypes.byref(out)) == gc.GS_ERR_INVAL
    big = gc.Params(w=64, h=4, D=8, tau=1, lam=1 << 27, inhibit=0)
    assert lib.gs_delegate_params(ctypes.byref(big.c()), 4, ctypes.byref(out)) == gc.GS_ERR_OVERFLOW
    pp = p.c()
    assert lib.gs_delegate_cost(None, ctypes.byref(pp), 2, None, None, None) == gc.GS_ERR_INVAL
    assert lib.gs_skin_bounds(None, ctypes.byref(pp), 2, None, None, None, None) == gc.GS_ERR_INVAL
    assert lib.gs_build_graph_skin(None, ctypes.byref(pp), None, None, None, None,
                                   None) == gc.GS_ERR_INVAL


def test_tuned_options_always_fit(lib):
    """Options from the autotuner's table (or the nearest bucket's) give a
    tile shape that fits the params, including depth ranges no bucket covers."""
    from paper_1803_01516_gb300 import autotune
    from paper_1803_01516_gb300 import gazecut as gc
    for w, h, D in [(384, 288, 16), (1920, 1080, 128), (640, 480, 96), (200, 100, 4)]:
        p = gc.Params(w=w, h=h, D=D, tau=30, lam=10)
        o = autotune.tuned_opts(p)
        gc.gs_tile_info(p, o)          # raises if the shape does not fit


def test_binding_refuses_host_tensors_and_bad_shapes(lib):
    """The binding checks shapes, sizes, devices and dtypes before any device
    call: a host tensor is refused (no CPU fallback), as are wrong sizes."""
    import torch
    from paper_1803_01516_gb300 import gazecut as gc
    p = gc.Params(w=64, h=8, D=4, tau=30, lam=2)
    L = torch.zeros((8, 64), dtype=torch.uint8)
    cost = torch.zeros(gc.gs_cost_volume_bytes(p) // 4, dtype=torch.int32)
    with pytest.raises(TypeError):
        gc.gs_stereo_cost_volume(L, L, p, cost)                 # host tensors
    with pytest.raises(ValueError):
        gc.gs_stereo_cost_volume(L[:, :60], L, p, cost)         # wrong image shape
    with pytest.raises(ValueError):
        gc.gs_stereo_cost_volume(L, L, p, cost[:-1])            # wrong cost size
    graph = torch.zeros(gc.gs_graph_bytes(p) - 1, dtype=torch.uint8)
    status = torch.zeros(1, dtype=torch.int32)
    with pytest.raises(ValueError):
        gc.gs_build_graph(cost, p, graph, status)               # graph too small
    with pytest.raises(ValueError):
        gc.gs_build_graph_skin(cost, p, torch.zeros((8, 3), dtype=torch.int32),
                               torch.zeros((8, 3), dtype=torch.int32),
                               torch.zeros(gc.gs_graph_bytes(p), dtype=torch.uint8), status)
    with pytest.raises(ValueError):
        gc.Batch([p] * 65, [gc.SolveOpts()] * 65)                # more than 64 pairs


def test_params_and_options_pack_like_the_header(lib):
    """ctypes mirrors of gs_params / gs_solve_opts / gs_pair_desc: sizes and
    the defaults the Python dataclasses fill in."""
    import ctypes
    from paper_1803_01516_gb300 import gazecut as gc
    assert ctypes.sizeof(gc.GsParams) == 9 * 4
    assert ctypes.sizeof(gc.GsSolveOpts) == 56      # 12 int32 + one int64, 8-byte aligned
    p = gc.Params(w=100, h=10, D=8, tau=5, lam=3)
    c = p.c()
    assert (c.dis0, c.direction, c.inhibit, c.vertical_inhibit) == (14, 0, 1023, 1)
    assert p.ng == 86
    o = gc.SolveOpts().c()
    assert (o.mode, o.engine, o.idle_limit_us, o.max_iters) == (gc.GS_MODE_EXACT,
                                                                gc.GS_ENGINE_TILED, 0, 1 << 16)


def test_solve_options_checked_alike_for_single_and_batched_solves(lib):
    """gs_maxflow_solve and gs_solve_batched refuse the same bad options on the
    host (one shared check, gs_check_solve_opts), before any device work."""
    from paper_1803_01516_gb300 import gazecut as gc
    good = gc.SolveOpts()
    assert lib.gs_check_solve_opts(ctypes.byref(good.c())) == gc.GS_OK
    bad = [gc.SolveOpts(mode=7), gc.SolveOpts(engine=3), gc.SolveOpts(sweeps_per_relabel=0),
           gc.SolveOpts(max_iters=0), gc.SolveOpts(local_iters=-1), gc.SolveOpts(relabel_passes=-2),
           gc.SolveOpts(tail_iters=-1), gc.SolveOpts(idle_limit_us=-5),
           gc.SolveOpts(cta_threads=384), gc.SolveOpts(cta_threads=128),
           gc.SolveOpts(mode=gc.GS_MODE_FIXED_SWEEPS, fixed_sweeps=-1)]
    p = gc.Params(w=64, h=8, D=4, tau=30, lam=2)
    fake = ctypes.c_void_p(256)
    for o in bad:
        oc = o.c()
        assert lib.gs_check_solve_opts(ctypes.byref(oc)) == gc.GS_ERR_INVAL, o
        assert lib.gs_maxflow_solve(fake, ctypes.byref(p.c()), ctypes.byref(oc), fake, fake,
                                    None) == gc.GS_ERR_INVAL, o
        d = gc.GsPairDesc(p.c(), oc, 256, 256, 256, 256, 256, 256, 256, 256)
        arr = (gc.GsPairDesc * 1)(d)
        assert lib.gs_solve_batched(ctypes.cast(arr, ctypes.c_void_p), 1, fake,
                                    None) == gc.GS_ERR_INVAL, o


def test_binding_refuses_a_tensor_on_another_device(lib, monkeypatch):
    """The library launches on the current device (its stream, its static
    scratch for the no-allocation solve): the binding refuses a tensor that
    lives on another device instead of passing its pointer on.  A tensor that
    only claims to be on cuda:1 (no storage, no GPU needed) stands in."""
    import torch
    from paper_1803_01516_gb300 import gazecut as gc

    class OnDevice1(torch.Tensor):
        @staticmethod
        def __new__(cls, dtype):
            return torch.Tensor._make_wrapper_subclass(cls, (16,), dtype=dtype,
                                                       device=torch.device("cuda", 1))

        @classmethod
        def __torch_dispatch__(cls, func, types, args=(), kwargs=None):
            raise RuntimeError("no compute on this stand-in")

    monkeypatch.setattr(torch.cuda, "current_device", lambda: 0)
    p = gc.Params(w=64, h=8, D=4, tau=30, lam=2)
    with pytest.raises(ValueError, match="current CUDA device"):
        gc.gs_maxflow_solve_noalloc(OnDevice1(torch.uint8), p, gc.SolveOpts(),
                                    OnDevice1(torch.int32))
    with pytest.raises(ValueError, match="current CUDA device"):
        gc.gs_energy(OnDevice1(torch.int32), OnDevice1(torch.int32), p, OnDevice1(torch.int64))
