"""The library's walker-sharded path on one GPU: two handles owning walkers
[0, W/2) and [W/2, W) with the matching Philox walker offsets (what two
ranks run under torchrun) give bitwise the trajectory of one handle with all
W walkers; the per-sweep accumulators add up to the single run's; the
reblocked mean of the union equals the single run's."""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_two_shards_equal_one_run(torch_cuda, prec):
    torch = torch_cuda
    import paper_2002_07401_gb300 as pg
    from paper_2002_07401_gb300 import shard
    sysm = synth.config2()
    W, sweeps = 64, 3
    p = pg.JAGP_PREC_MIXED if prec == "mixed" else pg.JAGP_PREC_FP64
    x = synth.init_walkers(sysm, W, seed=21)
    g = pg.JAGP(sysm, W, seed=21, precision=p)
    r = g.positions(x)
    g.eval(r)
    eL, acc = g.sweep(r, sweeps, acc=True)
    parts, accs = [], []
    for rank in range(2):
        w0 = shard.walker_offset(W // 2, rank)
        gs = pg.JAGP(sysm, W // 2, seed=21, precision=p)
        rs = gs.positions(x[w0:w0 + W // 2])
        gs.eval(rs)
        e_s, a_s = gs.sweep(rs, sweeps, walker0=w0, acc=True)
        parts.append((rs.cpu().numpy(), e_s.cpu().numpy()))
        accs.append(a_s.cpu().numpy())
        gs.close()
    assert np.array_equal(np.concatenate([q[0] for q in parts]), r.cpu().numpy())
    assert np.array_equal(np.concatenate([q[1] for q in parts], axis=1), eL.cpu().numpy())
    a = acc.cpu().numpy()
    s = accs[0] + accs[1]
    assert np.array_equal(s[:, 2], a[:, 2])
    assert np.allclose(s[:, :2], a[:, :2], rtol=1e-13, atol=0)
    _, st = pg.jagp_reblock(eL)
    _, st0 = pg.jagp_reblock(torch.tensor(np.concatenate([q[1] for q in parts], axis=1), device="cuda"))
    assert st.cpu().numpy().tolist() == st0.cpu().numpy().tolist()
    g.close()
