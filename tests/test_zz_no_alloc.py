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
    g.close()
