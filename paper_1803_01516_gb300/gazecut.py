"""Python binding of the C ABI in ``include/gazecut.h`` (argument marshalling only).

Every function with a ``gs_`` name calls the C entry point of the same name in
``libgazecut.so``: it checks dtypes, devices and sizes, passes the tensors'
device pointers and the current CUDA stream, and raises on a non-zero host
status.  No step of the method runs here; torch only provides device memory
and streams.  The library must have been built (``__graft_entry__.build()``);
there is no fallback.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libgazecut.so")

GS_OK, GS_ERR_INVAL, GS_ERR_OVERFLOW, GS_ERR_TIMEOUT, GS_ERR_CUDA, GS_ERR_LABELS, \
    GS_ERR_TOO_LARGE = range(7)
STATUS_NAMES = {0: "OK", 1: "INVAL", 2: "OVERFLOW", 3: "TIMEOUT", 4: "CUDA", 5: "LABELS",
                6: "TOO_LARGE"}
GS_MODE_EXACT, GS_MODE_FIXED_SWEEPS = 0, 1
GS_ENGINE_TILED, GS_ENGINE_SIMPLE = 0, 1

EXPORTS = [
    "gs_num_sites_w", "gs_cost_volume_bytes", "gs_graph_bytes", "gs_workspace_bytes",
    "gs_num_nodes", "gs_stereo_cost_volume", "gs_build_graph", "gs_maxflow_solve",
    "gs_extract_labels", "gs_energy", "gs_solve_stats", "gs_kernel_launches",
    "gs_noalloc_scratch_bytes", "gs_maxflow_solve_noalloc", "gs_tile_info",
    "gs_stereo_cost_volume_f32", "gs_energy_backward", "gs_cost_volume_f32_backward",
    "gs_cost_add_at_labels", "gs_batch_workspace_bytes", "gs_solve_batched",
    "gs_delegate_params", "gs_delegate_cost", "gs_skin_bounds", "gs_build_graph_skin",
    "gs_build_graph_flags", "gs_check_solve_opts", "gs_stereo_cost_volume_rgb",
    "gs_level2_start", "gs_block_descent",
]
GS_BUILD_CHAIN_PREFLOW = 1


class GsParams(ctypes.Structure):
    _fields_ = [("w", ctypes.c_int32), ("h", ctypes.c_int32), ("D", ctypes.c_int32),
                ("dis0", ctypes.c_int32), ("tau", ctypes.c_int32), ("lambda_", ctypes.c_int32),
                ("inhibit", ctypes.c_int32), ("vertical_inhibit", ctypes.c_int32),
                ("direction", ctypes.c_int32)]


class GsSolveOpts(ctypes.Structure):
    _fields_ = [("mode", ctypes.c_int32), ("sweeps_per_relabel", ctypes.c_int32),
                ("fixed_sweeps", ctypes.c_int32), ("engine", ctypes.c_int32),
                ("max_iters", ctypes.c_int64), ("local_iters", ctypes.c_int32),
                ("relabel_passes", ctypes.c_int32), ("tail_iters", ctypes.c_int32),
                ("tile_w", ctypes.c_int32), ("tile_h", ctypes.c_int32),
                ("idle_limit_us", ctypes.c_int32), ("cta_threads", ctypes.c_int32)]


class GsPairDesc(ctypes.Structure):
    _fields_ = [("p", GsParams), ("o", GsSolveOpts), ("L", ctypes.c_void_p), ("R", ctypes.c_void_p),
                ("cost", ctypes.c_void_p), ("graph", ctypes.c_void_p), ("workspace", ctypes.c_void_p),
                ("labels", ctypes.c_void_p), ("flow", ctypes.c_void_p), ("status", ctypes.c_void_p)]


@dataclass
class Params:
    """Problem description (mirrors ``gs_params``)."""

    w: int
    h: int
    D: int
    tau: int
    lam: int
    inhibit: int = 1023
    vertical_inhibit: int = 1
    dis0: int | None = None      # default 2(D-1): depth covers disparities 0..2(D-1)
    direction: int = 0           # 0 auto, 1 as given, 2 label-reversed

    def c(self) -> GsParams:
        dis0 = 2 * (self.D - 1) if self.dis0 is None else self.dis0
        return GsParams(self.w, self.h, self.D, dis0, self.tau, self.lam, self.inhibit,
                        self.vertical_inhibit, self.direction)

    @property
    def ng(self) -> int:
        return self.w - (2 * (self.D - 1) if self.dis0 is None else self.dis0)


@dataclass
class SolveOpts:
    """Solver options (mirrors ``gs_solve_opts``)."""

    mode: int = GS_MODE_EXACT
    sweeps_per_relabel: int = 16
    fixed_sweeps: int = 0
    max_iters: int = 1 << 16
    engine: int = GS_ENGINE_TILED
    local_iters: int = 0          # 0: library default
    relabel_passes: int = 0       # 0: library default
    tail_iters: int = 0           # 0: library default
    tile_w: int = 0               # 0: library default
    tile_h: int = 0
    idle_limit_us: int = 0        # 0: library default (60 s)
    cta_threads: int = 0          # 0: 512 (one block per SM); 256: two blocks per SM

    def c(self) -> GsSolveOpts:
        return GsSolveOpts(self.mode, self.sweeps_per_relabel, self.fixed_sweeps, self.engine,
                           self.max_iters, self.local_iters, self.relabel_passes,
                           self.tail_iters, self.tile_w, self.tile_h, self.idle_limit_us,
                           self.cta_threads)


_lib = None


def lib():
    """Load ``libgazecut.so`` (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: run __graft_entry__.build() first "
                               "(the CUDA library has no CPU fallback)")
        L = ctypes.CDLL(LIB_PATH)
        P, I32, I64, SZ = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_size_t
        F = ctypes.c_float
        pp = ctypes.POINTER(GsParams)
        po = ctypes.POINTER(GsSolveOpts)
        sig = {
            "gs_num_sites_w": ([pp], I32),
            "gs_cost_volume_bytes": ([pp], SZ),
            "gs_graph_bytes": ([pp], SZ),
            "gs_workspace_bytes": ([pp, po], SZ),
            "gs_num_nodes": ([pp], I64),
            "gs_stereo_cost_volume": ([P, P, I32, pp, P, P], ctypes.c_int),
            "gs_build_graph": ([P, pp, P, P, P], ctypes.c_int),
            "gs_build_graph_flags": ([P, pp, I32, P, P, P], ctypes.c_int),
            "gs_maxflow_solve": ([P, pp, po, P, P, P], ctypes.c_int),
            "gs_extract_labels": ([P, pp, po, P, P, P, P, P], ctypes.c_int),
            "gs_energy": ([P, P, pp, P, P], ctypes.c_int),
            "gs_solve_stats": ([P, P, P], ctypes.c_int),
            "gs_kernel_launches": ([], I64),
            "gs_noalloc_scratch_bytes": ([], SZ),
            "gs_tile_info": ([pp, po, P], ctypes.c_int),
            "gs_stereo_cost_volume_f32": ([P, P, I32, pp, F, F, F, F, P, P], ctypes.c_int),
            "gs_energy_backward": ([P, pp, F, P, P, P], ctypes.c_int),
            "gs_cost_volume_f32_backward": ([P, P, I32, pp, F, F, F, P, P, P], ctypes.c_int),
            "gs_cost_add_at_labels": ([P, P, pp, I32, P], ctypes.c_int),
            "gs_batch_workspace_bytes": ([I32], SZ),
            "gs_solve_batched": ([P, I32, P, P], ctypes.c_int),
            "gs_delegate_params": ([pp, I32, pp], ctypes.c_int),
            "gs_delegate_cost": ([P, pp, I32, P, P, P], ctypes.c_int),
            "gs_skin_bounds": ([P, pp, I32, P, P, P, P], ctypes.c_int),
            "gs_build_graph_skin": ([P, pp, P, P, P, P, P], ctypes.c_int),
            "gs_maxflow_solve_noalloc": ([P, pp, po, P, P], ctypes.c_int),
            "gs_check_solve_opts": ([po], ctypes.c_int),
            "gs_stereo_cost_volume_rgb": ([P, P, I32, pp, P, P], ctypes.c_int),
            "gs_level2_start": ([P, pp, I32, P, P, P, P], ctypes.c_int),
            "gs_block_descent": ([P, pp, I32, P, P, P, I32, P, P], ctypes.c_int),
        }
        for name, (args, res) in sig.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = res
        _lib = L
    return _lib


def _stream(stream=None):
    s = torch.cuda.current_stream() if stream is None else stream
    return ctypes.c_void_p(s.cuda_stream)


def _dev(t: torch.Tensor, dtype, name: str):
    if not isinstance(t, torch.Tensor) or t.device.type != "cuda":
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    # the library launches on the current device, with that device's stream
    # (and, for the no-allocation solve, that device's static scratch)
    cur = torch.cuda.current_device()
    if t.device.index is not None and t.device.index != cur:
        raise ValueError(f"{name} is on {t.device} but the current CUDA device is cuda:{cur}; "
                         f"call inside torch.cuda.device({t.device.index})")
    return ctypes.c_void_p(t.data_ptr())


def _check(rc: int, what: str):
    if rc != GS_OK:
        raise RuntimeError(f"{what} failed: {STATUS_NAMES.get(rc, rc)}")


# ------------------------------------------------------------------ sizes --

def gs_cost_volume_bytes(p: Params) -> int:
    return lib().gs_cost_volume_bytes(ctypes.byref(p.c()))


def gs_graph_bytes(p: Params) -> int:
    return lib().gs_graph_bytes(ctypes.byref(p.c()))


def gs_workspace_bytes(p: Params, o: SolveOpts) -> int:
    return lib().gs_workspace_bytes(ctypes.byref(p.c()), ctypes.byref(o.c()))


def gs_num_nodes(p: Params) -> int:
    return lib().gs_num_nodes(ctypes.byref(p.c()))


# ------------------------------------------------------------------ calls --

def gs_stereo_cost_volume(L: torch.Tensor, R: torch.Tensor, p: Params, cost: torch.Tensor,
                          stream=None):
    if L.shape != (p.h, p.w) or R.shape != (p.h, p.w):
        raise ValueError("L, R must be [h, w]")
    if cost.numel() * 4 != gs_cost_volume_bytes(p):
        raise ValueError("cost has the wrong size")
    rc = lib().gs_stereo_cost_volume(_dev(L, torch.uint8, "L"), _dev(R, torch.uint8, "R"), p.w,
                                     ctypes.byref(p.c()), _dev(cost, torch.int32, "cost"),
                                     _stream(stream))
    _check(rc, "gs_stereo_cost_volume")


def gs_stereo_cost_volume_rgb(L: torch.Tensor, R: torch.Tensor, p: Params, cost: torch.Tensor,
                              stream=None):
    """Colour data term (§4.3); L, R uint8 [h, w, 3] (interleaved RGB)."""
    if L.shape != (p.h, p.w, 3) or R.shape != (p.h, p.w, 3):
        raise ValueError("L, R must be [h, w, 3]")
    if cost.numel() * 4 != gs_cost_volume_bytes(p):
        raise ValueError("cost has the wrong size")
    rc = lib().gs_stereo_cost_volume_rgb(_dev(L, torch.uint8, "L"), _dev(R, torch.uint8, "R"),
                                         3 * p.w, ctypes.byref(p.c()),
                                         _dev(cost, torch.int32, "cost"), _stream(stream))
    _check(rc, "gs_stereo_cost_volume_rgb")


def gs_build_graph(cost: torch.Tensor, p: Params, graph: torch.Tensor, status: torch.Tensor,
                   stream=None):
    if graph.numel() < gs_graph_bytes(p) or cost.numel() * 4 != gs_cost_volume_bytes(p):
        raise ValueError("graph / cost buffer has the wrong size")
    rc = lib().gs_build_graph(_dev(cost, torch.int32, "cost"), ctypes.byref(p.c()),
                              _dev(graph, torch.uint8, "graph"), _dev(status, torch.int32, "status"),
                              _stream(stream))
    _check(rc, "gs_build_graph")


def gs_build_graph_flags(cost: torch.Tensor, p: Params, flags: int, graph: torch.Tensor,
                         status: torch.Tensor, stream=None):
    if graph.numel() < gs_graph_bytes(p) or cost.numel() * 4 != gs_cost_volume_bytes(p):
        raise ValueError("graph / cost buffer has the wrong size")
    rc = lib().gs_build_graph_flags(_dev(cost, torch.int32, "cost"), ctypes.byref(p.c()),
                                    int(flags), _dev(graph, torch.uint8, "graph"),
                                    _dev(status, torch.int32, "status"), _stream(stream))
    _check(rc, "gs_build_graph_flags")


def gs_maxflow_solve(graph: torch.Tensor, p: Params, o: SolveOpts, workspace: torch.Tensor,
                     status: torch.Tensor, stream=None):
    if workspace.numel() < gs_workspace_bytes(p, o):
        raise ValueError("workspace too small")
    rc = lib().gs_maxflow_solve(_dev(graph, torch.uint8, "graph"), ctypes.byref(p.c()),
                                ctypes.byref(o.c()), _dev(workspace, torch.uint8, "workspace"),
                                _dev(status, torch.int32, "status"), _stream(stream))
    _check(rc, "gs_maxflow_solve")


def gs_extract_labels(graph: torch.Tensor, p: Params, o: SolveOpts, workspace: torch.Tensor,
                      labels: torch.Tensor, flow: torch.Tensor, status: torch.Tensor, stream=None):
    if labels.numel() != p.ng * p.h:
        raise ValueError("labels must hold h * n_g entries")
    rc = lib().gs_extract_labels(_dev(graph, torch.uint8, "graph"), ctypes.byref(p.c()),
                                 ctypes.byref(o.c()), _dev(workspace, torch.uint8, "workspace"),
                                 _dev(labels, torch.int32, "labels"), _dev(flow, torch.int64, "flow"),
                                 _dev(status, torch.int32, "status"), _stream(stream))
    _check(rc, "gs_extract_labels")


def gs_stereo_cost_volume_f32(L: torch.Tensor, R: torch.Tensor, p: Params, w1: float, w2: float,
                              tau: float, scale: float, cost: torch.Tensor, stream=None):
    if L.shape != (p.h, p.w) or R.shape != (p.h, p.w):
        raise ValueError("L, R must be [h, w]")
    if cost.numel() * 4 != gs_cost_volume_bytes(p):
        raise ValueError("cost has the wrong size")
    rc = lib().gs_stereo_cost_volume_f32(_dev(L, torch.uint8, "L"), _dev(R, torch.uint8, "R"), p.w,
                                         ctypes.byref(p.c()), w1, w2, tau, scale,
                                         _dev(cost, torch.int32, "cost"), _stream(stream))
    _check(rc, "gs_stereo_cost_volume_f32")


def gs_energy_backward(labels: torch.Tensor, p: Params, grad: float, dcost, counts: torch.Tensor,
                       stream=None):
    dc = ctypes.c_void_p(0) if dcost is None else _dev(dcost, torch.float32, "dcost")
    rc = lib().gs_energy_backward(_dev(labels, torch.int32, "labels"), ctypes.byref(p.c()), grad,
                                  dc, _dev(counts, torch.int64, "counts"), _stream(stream))
    _check(rc, "gs_energy_backward")


def gs_cost_volume_f32_backward(L: torch.Tensor, R: torch.Tensor, p: Params, w1: float, w2: float,
                                tau: float, labels: torch.Tensor, sums: torch.Tensor, stream=None):
    rc = lib().gs_cost_volume_f32_backward(_dev(L, torch.uint8, "L"), _dev(R, torch.uint8, "R"),
                                           p.w, ctypes.byref(p.c()), w1, w2, tau,
                                           _dev(labels, torch.int32, "labels"),
                                           _dev(sums, torch.int64, "sums"), _stream(stream))
    _check(rc, "gs_cost_volume_f32_backward")


def gs_cost_add_at_labels(cost: torch.Tensor, labels: torch.Tensor, p: Params, value: int,
                          stream=None):
    rc = lib().gs_cost_add_at_labels(_dev(cost, torch.int32, "cost"),
                                     _dev(labels, torch.int32, "labels"), ctypes.byref(p.c()),
                                     int(value), _stream(stream))
    _check(rc, "gs_cost_add_at_labels")


def gs_energy(cost: torch.Tensor, labels: torch.Tensor, p: Params, energy: torch.Tensor,
              stream=None):
    rc = lib().gs_energy(_dev(cost, torch.int32, "cost"), _dev(labels, torch.int32, "labels"),
                         ctypes.byref(p.c()), _dev(energy, torch.int64, "energy"), _stream(stream))
    _check(rc, "gs_energy")


def gs_solve_stats(workspace: torch.Tensor, stream=None) -> dict:
    out = (ctypes.c_int64 * 10)()
    rc = lib().gs_solve_stats(_dev(workspace, torch.uint8, "workspace"), out, _stream(stream))
    _check(rc, "gs_solve_stats")
    keys = ["relabels", "sweeps", "bfs_passes", "label_passes", "active_at_exit", "sweep_ns",
            "relabel_ns", "launches", "sweep_visits", "relabel_visits"]
    return {k: int(out[i]) for i, k in enumerate(keys)}


def gs_kernel_launches() -> int:
    return int(lib().gs_kernel_launches())


def gs_tile_info(p: Params, o: SolveOpts | None = None) -> dict:
    out = (ctypes.c_int32 * 4)()
    o = o or SolveOpts()
    _check(lib().gs_tile_info(ctypes.byref(p.c()), ctypes.byref(o.c()), out), "gs_tile_info")
    return {"tile_w": out[0], "tile_h": out[1], "tiles": out[2], "smem_bytes": out[3]}


def gs_noalloc_scratch_bytes() -> int:
    return int(lib().gs_noalloc_scratch_bytes())


def gs_maxflow_solve_noalloc(graph: torch.Tensor, p: Params, o: SolveOpts, status: torch.Tensor,
                             stream=None) -> int:
    """Solve with the library's static scratch (no workspace).  Returns the
    host status (GS_ERR_TOO_LARGE when the problem does not fit)."""
    return lib().gs_maxflow_solve_noalloc(_dev(graph, torch.uint8, "graph"), ctypes.byref(p.c()),
                                          ctypes.byref(o.c()), _dev(status, torch.int32, "status"),
                                          _stream(stream))


# ------------------------------------------------ level-1 approximation ---

def gs_delegate_params(p: Params, b: int) -> Params:
    """Params of the delegate problem for block size b (§4.5)."""
    out = GsParams()
    _check(lib().gs_delegate_params(ctypes.byref(p.c()), int(b), ctypes.byref(out)),
           "gs_delegate_params")
    return Params(w=out.w, h=out.h, D=out.D, tau=out.tau, lam=out.lambda_, inhibit=out.inhibit,
                  vertical_inhibit=out.vertical_inhibit, dis0=out.dis0, direction=out.direction)


def gs_delegate_cost(cost: torch.Tensor, p: Params, b: int, coarse: torch.Tensor,
                     status: torch.Tensor, stream=None):
    pc = gs_delegate_params(p, b)
    if cost.numel() * 4 != gs_cost_volume_bytes(p) or coarse.numel() * 4 != gs_cost_volume_bytes(pc):
        raise ValueError("cost / delegate cost buffer has the wrong size")
    rc = lib().gs_delegate_cost(_dev(cost, torch.int32, "cost"), ctypes.byref(p.c()), int(b),
                                _dev(coarse, torch.int32, "coarse"),
                                _dev(status, torch.int32, "status"), _stream(stream))
    _check(rc, "gs_delegate_cost")


def gs_skin_bounds(coarse_labels: torch.Tensor, p: Params, b: int, lo: torch.Tensor,
                   hi: torch.Tensor, status: torch.Tensor, stream=None):
    pc = gs_delegate_params(p, b)
    if coarse_labels.numel() != pc.ng * pc.h or lo.numel() != p.ng * p.h or hi.numel() != p.ng * p.h:
        raise ValueError("labels / bounds buffer has the wrong size")
    rc = lib().gs_skin_bounds(_dev(coarse_labels, torch.int32, "coarse_labels"), ctypes.byref(p.c()),
                              int(b), _dev(lo, torch.int32, "lo"), _dev(hi, torch.int32, "hi"),
                              _dev(status, torch.int32, "status"), _stream(stream))
    _check(rc, "gs_skin_bounds")


def gs_build_graph_skin(cost: torch.Tensor, p: Params, lo: torch.Tensor, hi: torch.Tensor,
                        graph: torch.Tensor, status: torch.Tensor, stream=None):
    if graph.numel() < gs_graph_bytes(p) or cost.numel() * 4 != gs_cost_volume_bytes(p):
        raise ValueError("graph / cost buffer has the wrong size")
    if lo.numel() != p.ng * p.h or hi.numel() != p.ng * p.h:
        raise ValueError("bounds must hold h * n_g entries")
    rc = lib().gs_build_graph_skin(_dev(cost, torch.int32, "cost"), ctypes.byref(p.c()),
                                   _dev(lo, torch.int32, "lo"), _dev(hi, torch.int32, "hi"),
                                   _dev(graph, torch.uint8, "graph"),
                                   _dev(status, torch.int32, "status"), _stream(stream))
    _check(rc, "gs_build_graph_skin")


# ------------------------------------------------ level-2 approximation ---

def gs_level2_start(cost: torch.Tensor, p: Params, b: int, coarse_labels: torch.Tensor,
                    labels: torch.Tensor, status: torch.Tensor, stream=None):
    pc = gs_delegate_params(p, b)
    if cost.numel() * 4 != gs_cost_volume_bytes(p) or coarse_labels.numel() != pc.ng * pc.h \
            or labels.numel() != p.ng * p.h:
        raise ValueError("cost / labels buffer has the wrong size")
    rc = lib().gs_level2_start(_dev(cost, torch.int32, "cost"), ctypes.byref(p.c()), int(b),
                               _dev(coarse_labels, torch.int32, "coarse_labels"),
                               _dev(labels, torch.int32, "labels"),
                               _dev(status, torch.int32, "status"), _stream(stream))
    _check(rc, "gs_level2_start")


def gs_block_descent(cost: torch.Tensor, p: Params, b: int, lo: torch.Tensor, hi: torch.Tensor,
                     labels: torch.Tensor, passes: int, status: torch.Tensor, stream=None):
    if cost.numel() * 4 != gs_cost_volume_bytes(p):
        raise ValueError("cost has the wrong size")
    if lo.numel() != p.ng * p.h or hi.numel() != p.ng * p.h or labels.numel() != p.ng * p.h:
        raise ValueError("bounds / labels must hold h * n_g entries")
    rc = lib().gs_block_descent(_dev(cost, torch.int32, "cost"), ctypes.byref(p.c()), int(b),
                                _dev(lo, torch.int32, "lo"), _dev(hi, torch.int32, "hi"),
                                _dev(labels, torch.int32, "labels"), int(passes),
                                _dev(status, torch.int32, "status"), _stream(stream))
    _check(rc, "gs_block_descent")


def solve_level2(cost: torch.Tensor, p: Params, b: int, passes: int = 2,
                 o: SolveOpts | None = None, bufs: "Level1Buffers | None" = None, stream=None):
    """Level-2 approximation of §4.5 from a cost volume int32 [h, n_g, D]:
    delegate cut, thin skin, start labels, `passes` two-colour passes of exact
    block cuts.  Returns (labels, coarse_labels, status) device tensors."""
    o = o or SolveOpts()
    bufs = bufs or Level1Buffers(p, b, o, device=cost.device)
    c = cost.reshape(-1)
    cb, fb = bufs.coarse, bufs.fine
    gs_delegate_cost(c, p, b, cb.cost, bufs.status, stream)
    gs_build_graph(cb.cost, bufs.pc, cb.graph, cb.status, stream)
    gs_maxflow_solve(cb.graph, bufs.pc, bufs.oc, cb.work, cb.status, stream)
    gs_extract_labels(cb.graph, bufs.pc, bufs.oc, cb.work, cb.labels, cb.flow, cb.status, stream)
    gs_skin_bounds(cb.labels, p, b, bufs.lo, bufs.hi, bufs.status, stream)
    gs_level2_start(c, p, b, cb.labels, fb.labels, bufs.status, stream)
    gs_block_descent(c, p, b, bufs.lo, bufs.hi, fb.labels, passes, bufs.status, stream)
    st = torch.where(bufs.status != 0, bufs.status, cb.status)
    return fb.labels, cb.labels, st


# ---------------------------------------------------------- whole pairs ---

class Buffers:
    """Device buffers for one problem size (cost volume, graph, workspace, outputs)."""

    def __init__(self, p: Params, o: SolveOpts, device="cuda"):
        self.p, self.o = p, o
        self.cost = torch.empty(gs_cost_volume_bytes(p) // 4, dtype=torch.int32, device=device)
        self.graph = torch.empty(gs_graph_bytes(p), dtype=torch.uint8, device=device)
        self.work = torch.empty(gs_workspace_bytes(p, o), dtype=torch.uint8, device=device)
        self.labels = torch.empty((p.h, p.ng), dtype=torch.int32, device=device)
        self.flow = torch.zeros(1, dtype=torch.int64, device=device)
        self.status = torch.zeros(1, dtype=torch.int32, device=device)


def solve_pair(L: torch.Tensor, R: torch.Tensor, p: Params, o: SolveOpts | None = None,
               buf: Buffers | None = None, stream=None):
    """All four steps on device images.  Returns (labels, flow, status) device tensors."""
    o = o or SolveOpts()
    buf = buf or Buffers(p, o, device=L.device)
    gs_stereo_cost_volume(L, R, p, buf.cost, stream)
    gs_build_graph(buf.cost, p, buf.graph, buf.status, stream)
    gs_maxflow_solve(buf.graph, p, o, buf.work, buf.status, stream)
    gs_extract_labels(buf.graph, p, o, buf.work, buf.labels, buf.flow, buf.status, stream)
    return buf.labels, buf.flow, buf.status


def solve_costs(cost: torch.Tensor, p: Params, o: SolveOpts | None = None,
                buf: Buffers | None = None, stream=None):
    """Steps 2-4 from a given cost volume int32 [h, n_g, D]."""
    o = o or SolveOpts()
    buf = buf or Buffers(p, o, device=cost.device)
    c = cost.reshape(-1)
    gs_build_graph(c, p, buf.graph, buf.status, stream)
    gs_maxflow_solve(buf.graph, p, o, buf.work, buf.status, stream)
    gs_extract_labels(buf.graph, p, o, buf.work, buf.labels, buf.flow, buf.status, stream)
    return buf.labels, buf.flow, buf.status


class Level1Buffers:
    """Device buffers of the level-1 approximation for one size and block size."""

    def __init__(self, p: Params, b: int, o: SolveOpts, oc: SolveOpts | None = None,
                 device="cuda"):
        self.p, self.b, self.o = p, b, o
        self.pc = gs_delegate_params(p, b)
        self.oc = oc or o
        self.coarse = Buffers(self.pc, self.oc, device=device)
        self.fine = Buffers(p, o, device=device)
        self.lo = torch.empty((p.h, p.ng), dtype=torch.int32, device=device)
        self.hi = torch.empty((p.h, p.ng), dtype=torch.int32, device=device)
        self.status = torch.zeros(1, dtype=torch.int32, device=device)


def solve_level1(cost: torch.Tensor, p: Params, b: int, o: SolveOpts | None = None,
                 bufs: Level1Buffers | None = None, stream=None):
    """Level-1 approximation of §4.5 from a cost volume int32 [h, n_g, D]:
    delegate cut, thin skin, exact second cut.  Returns (labels, coarse_labels,
    status) device tensors; status is the first non-OK status of the steps."""
    o = o or SolveOpts()
    bufs = bufs or Level1Buffers(p, b, o, device=cost.device)
    c = cost.reshape(-1)
    cb, fb = bufs.coarse, bufs.fine
    gs_delegate_cost(c, p, b, cb.cost, bufs.status, stream)
    gs_build_graph(cb.cost, bufs.pc, cb.graph, cb.status, stream)
    gs_maxflow_solve(cb.graph, bufs.pc, bufs.oc, cb.work, cb.status, stream)
    gs_extract_labels(cb.graph, bufs.pc, bufs.oc, cb.work, cb.labels, cb.flow, cb.status, stream)
    gs_skin_bounds(cb.labels, p, b, bufs.lo, bufs.hi, bufs.status, stream)
    gs_build_graph_skin(c, p, bufs.lo, bufs.hi, fb.graph, fb.status, stream)
    gs_maxflow_solve(fb.graph, p, o, fb.work, fb.status, stream)
    gs_extract_labels(fb.graph, p, o, fb.work, fb.labels, fb.flow, fb.status, stream)
    st = torch.where(bufs.status != 0, bufs.status, torch.where(cb.status != 0, cb.status, fb.status))
    return fb.labels, cb.labels, st


# ------------------------------------------------------------- batches ---

class Batch:
    """Device buffers for a batch of pairs of uneven sizes (one Buffers each)."""

    def __init__(self, params: list, opts: list, device="cuda"):
        if not 1 <= len(params) <= 64:
            raise ValueError("a batch holds 1 to 64 pairs")
        self.params, self.opts = params, opts
        self.bufs = [Buffers(p, o, device=device) for p, o in zip(params, opts)]
        self.ws = torch.empty(lib().gs_batch_workspace_bytes(len(params)), dtype=torch.uint8,
                              device=device)
        self._descs = None

    def descs(self, Ls, Rs):
        n = len(self.params)
        arr = (GsPairDesc * n)()
        for i, (p, o, b, L, R) in enumerate(zip(self.params, self.opts, self.bufs, Ls, Rs)):
            if L.shape != (p.h, p.w) or R.shape != (p.h, p.w):
                raise ValueError(f"pair {i}: images must be [h, w]")
            arr[i] = GsPairDesc(p.c(), o.c(), _dev(L, torch.uint8, "L").value,
                                _dev(R, torch.uint8, "R").value,
                                _dev(b.cost, torch.int32, "cost").value,
                                _dev(b.graph, torch.uint8, "graph").value,
                                _dev(b.work, torch.uint8, "workspace").value,
                                _dev(b.labels, torch.int32, "labels").value,
                                _dev(b.flow, torch.int64, "flow").value,
                                _dev(b.status, torch.int32, "status").value)
        self._descs = arr       # keep alive
        return arr


def gs_solve_batched(batch: Batch, Ls, Rs, stream=None):
    """All pairs of the batch through the whole path (two persistent launches)."""
    arr = batch.descs(Ls, Rs)
    rc = lib().gs_solve_batched(ctypes.cast(arr, ctypes.c_void_p), len(arr),
                                _dev(batch.ws, torch.uint8, "batch workspace"), _stream(stream))
    _check(rc, "gs_solve_batched")
