"""gs_maxflow_solve_noalloc: the solve for callers that cannot allocate device
memory at solve time (scratch in the library's static device array).

Its results must equal those of gs_maxflow_solve with a caller workspace and
the CPU oracle's exact cut, on consecutive calls that reuse the static
scratch, and a call must leave the device's allocated memory unchanged.  This
file is collected last so that a run stopping at the first failure has run
every other test first.
"""
import ctypes

import numpy as np
import pytest

import oracle
from paper_1803_01516_gb300 import synth

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def gc():
    from paper_1803_01516_gb300 import build
    build.build()
    from paper_1803_01516_gb300 import gazecut
    return gazecut


def test_too_large_is_rejected_before_any_device_work(gc):
    """A problem needing more scratch than the static array holds is refused
    on the host (no GPU needed for this check)."""
    p = gc.Params(w=1920, h=1080, D=128, tau=40, lam=12)
    o = gc.SolveOpts()
    fake = ctypes.c_void_p(256)
    rc = gc.lib().gs_maxflow_solve_noalloc(fake, ctypes.byref(p.c()), ctypes.byref(o.c()), fake,
                                           None)
    assert rc == gc.GS_ERR_TOO_LARGE
    assert gc.gs_noalloc_scratch_bytes() == 16 << 20


@pytest.mark.gpu
def test_noalloc_matches_workspace_solve_on_consecutive_calls(gc):
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    dev = torch.device("cuda")
    for wl, idx in [(synth.MAIN, 0), (synth.MAIN, 1), (synth.TINY, 2)]:
        L, R, _ = synth.make_pair(wl, idx)
        p = gc.Params(w=wl.w, h=wl.h, D=wl.D, tau=wl.tau, lam=wl.lam, inhibit=wl.inhibit)
        o = gc.SolveOpts()
        Ld, Rd = torch.from_numpy(L).to(dev), torch.from_numpy(R).to(dev)
        # the existing entry point with a caller workspace
        ref = gc.Buffers(p, o, device=dev)
        gc.solve_pair(Ld, Rd, p, o, ref)
        # the same problem through the no-allocation entry point
        buf = gc.Buffers(p, o, device=dev)
        gc.gs_stereo_cost_volume(Ld, Rd, p, buf.cost)
        gc.gs_build_graph(buf.cost, p, buf.graph, buf.status)
        rc = gc.gs_maxflow_solve_noalloc(buf.graph, p, o, buf.status)
        assert rc == gc.GS_OK
        gc.gs_extract_labels(buf.graph, p, o, buf.work, buf.labels, buf.flow, buf.status)
        torch.cuda.synchronize()
        assert int(ref.status.item()) == gc.GS_OK
        assert int(buf.status.item()) == gc.GS_OK
        assert int(buf.flow.item()) == int(ref.flow.item())
        assert np.array_equal(buf.labels.cpu().numpy(), ref.labels.cpu().numpy())
        # and both are the oracle's exact cut
        C = oracle.cost_volume(L, R, wl.D, 2 * (wl.D - 1), wl.tau)
        want = oracle.solve(C, wl.lam, wl.inhibit, 1)
        assert int(buf.flow.item()) == want["flow"]
        assert np.array_equal(buf.labels.cpu().numpy(), want["labels"])


@pytest.mark.gpu
def test_noalloc_call_allocates_no_device_memory(gc):
    """After a first call (which loads the library's module and looks up the
    static array's address), a further call changes neither the memory torch
    has allocated nor the device's free memory."""
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    dev = torch.device("cuda")
    wl = synth.MAIN
    L, R, _ = synth.make_pair(wl, 3)
    p = gc.Params(w=wl.w, h=wl.h, D=wl.D, tau=wl.tau, lam=wl.lam, inhibit=wl.inhibit)
    o = gc.SolveOpts()
    buf = gc.Buffers(p, o, device=dev)
    Ld, Rd = torch.from_numpy(L).to(dev), torch.from_numpy(R).to(dev)
    gc.gs_stereo_cost_volume(Ld, Rd, p, buf.cost)
    gc.gs_build_graph(buf.cost, p, buf.graph, buf.status)
    assert gc.gs_maxflow_solve_noalloc(buf.graph, p, o, buf.status) == gc.GS_OK
    torch.cuda.synchronize()
    gc.gs_build_graph(buf.cost, p, buf.graph, buf.status)
    torch.cuda.synchronize()
    torch_before = torch.cuda.memory_allocated(dev)
    free_before, _ = torch.cuda.mem_get_info(dev)
    assert gc.gs_maxflow_solve_noalloc(buf.graph, p, o, buf.status) == gc.GS_OK
    torch.cuda.synchronize()
    free_after, _ = torch.cuda.mem_get_info(dev)
    assert torch.cuda.memory_allocated(dev) == torch_before
    assert free_after == free_before
    assert int(buf.status.item()) == gc.GS_OK
