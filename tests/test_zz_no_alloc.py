"""jagp_eval_noalloc: the allocation-free variant of jagp_eval.

It serves callers that cannot allocate device memory when they need log|Psi|
(an allocator or memory pool that forbids new reservations, a framework that
owns every allocation): the library keeps the scratch in a fixed device
array instead.  These tests call it through the C ABI and compare it with
jagp_eval on the same configurations, twice in a row (the shared array keeps
the previous call's contents, which must not leak into the next result).
This file is collected last on purpose.
"""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

TOL = 1e-10


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def _close(a, b):
    return np.all(np.abs(a - b) <= TOL * np.maximum(1.0, np.abs(b)))


def test_noalloc_matches_eval_twice(torch_cuda):
    torch = torch_cuda
    import paper_2002_07401_gb300 as pg
    sysm = synth.config2()
    g = pg.JAGP(sysm, 400, seed=0)
    for W, seed in ((100, 1), (37, 2)):   # second call: other positions, fewer walkers
        x = synth.jitter_walkers(synth.init_walkers(sysm, W, seed=seed), seed, 0.4)
        r = g.positions(x)
        la_ref, sg_ref = g.eval(r)
        la = torch.full((W,), float("nan"), dtype=torch.float64, device=g.device)
        sg = torch.full((W,), float("nan"), dtype=torch.float64, device=g.device)
        pg.jagp_eval_noalloc(g.h, r, W, la, sg)
        torch.cuda.synchronize()
        assert _close(la.cpu().numpy(), la_ref.cpu().numpy())
        assert np.array_equal(sg.cpu().numpy(), sg_ref.cpu().numpy())
    g.close()


def _free_bytes(torch):
    free, _ = torch.cuda.mem_get_info()
    return free, torch.cuda.memory_reserved()


def test_noalloc_allocates_nothing_and_counts_its_launches(torch_cuda):
    """Around a warm call neither the device's free memory nor torch's reserved
    pool changes, and the call's kernels show in jagp_launch_count."""
    torch = torch_cuda
    import paper_2002_07401_gb300 as pg
    sysm = synth.config2()
    g = pg.JAGP(sysm, 64, seed=0)
    x = synth.jitter_walkers(synth.init_walkers(sysm, 64, seed=4), 4, 0.4)
    r = g.positions(x)
    la = torch.empty(64, dtype=torch.float64, device=g.device)
    sg = torch.empty(64, dtype=torch.float64, device=g.device)
    pg.jagp_eval_noalloc(g.h, r, 64, la, sg)       # first call: set-up
    torch.cuda.synchronize()
    before, n0 = _free_bytes(torch), pg.jagp_launch_count(g.h)
    pg.jagp_eval_noalloc(g.h, r, 64, la, sg)
    torch.cuda.synchronize()
    assert _free_bytes(torch) == before
    assert pg.jagp_launch_count(g.h) > n0
    g.close()


def test_noalloc_on_mixed_handle_is_fp64(torch_cuda):
    """On a mixed-precision handle the call still evaluates in FP64: it agrees
    with an FP64 handle to the FP64 bar, and with the handle's own mixed
    jagp_eval within that path's stated log|Psi| error (1e-6), twice in a row."""
    torch = torch_cuda
    import paper_2002_07401_gb300 as pg
    sysm = synth.config2()
    gm = pg.JAGP(sysm, 128, seed=0, precision=pg.JAGP_PREC_MIXED)
    g64 = pg.JAGP(sysm, 128, seed=0)
    for W, seed in ((128, 5), (51, 6)):
        x = synth.jitter_walkers(synth.init_walkers(sysm, W, seed=seed), seed, 0.4)
        r = gm.positions(x)
        la_m, _ = gm.eval(r)
        la_64, sg_64 = g64.eval(r)
        la = torch.empty(W, dtype=torch.float64, device=gm.device)
        sg = torch.empty(W, dtype=torch.float64, device=gm.device)
        pg.jagp_eval_noalloc(gm.h, r, W, la, sg)
        torch.cuda.synchronize()
        assert _close(la.cpu().numpy(), la_64.cpu().numpy())
        assert np.array_equal(sg.cpu().numpy(), sg_64.cpu().numpy())
        assert np.max(np.abs(la.cpu().numpy() - la_m.cpu().numpy())) <= 1e-6
    gm.close()
    g64.close()


def test_noalloc_rejects_oversize(torch_cuda):
    torch = torch_cuda
    import paper_2002_07401_gb300 as pg
    sysm = synth.config2()
    g = pg.JAGP(sysm, 400, seed=0)
    x = synth.init_walkers(sysm, 400, seed=3)
    r = g.positions(x)
    la = torch.empty(400, dtype=torch.float64, device=g.device)
    with pytest.raises(pg.JagpError, match="unsupported"):
        pg.jagp_eval_noalloc(g.h, r, 400, la, None)   # ~66 MB of scratch > 32 MiB
    assert "more than the 33554432 of the fixed array" in pg.jagp_last_error(g.h)[1]
    g.close()
