"""GPU parity of the sample statistics (Sec. VMC): the per-sweep sums of e_L
and e_L^2 that vmc_sweep accumulates, and the reblocked error bar of the VMC
mean (jagp_reblock), against the oracle on the same samples."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def _rel(a, b):
    return np.max(np.abs(np.asarray(a) - np.asarray(b)) / np.maximum(1e-300, np.abs(np.asarray(b))))


@pytest.mark.parametrize("T,W", [(257, 5), (1, 3), (2, 1), (64, 4096), (1000, 1)])
def test_reblock_matches_oracle(torch_cuda, T, W):
    """Random series, including a ragged tail (T = 257), a single sweep (no
    level) and more walkers than threads of a CTA."""
    torch = torch_cuda
    import paper_2002_07401_gb300 as pg
    rng = np.random.default_rng(T * 7 + W)
    eL = np.ascontiguousarray(np.cumsum(rng.normal(size=(T, W)), axis=0) * 0.01 - 2.0)
    lev_ref, st_ref = oracle.reblock(eL)
    lev, st = pg.jagp_reblock(torch.tensor(eL, device="cuda"))
    torch.cuda.synchronize()
    lev, st = lev.cpu().numpy(), st.cpu().numpy()
    assert lev.shape == lev_ref.shape
    if len(lev_ref):
        assert np.array_equal(lev[:, :2], lev_ref[:, :2])
        assert _rel(lev[:, 2:], lev_ref[:, 2:]) < 1e-11
    assert abs(st[0] - st_ref[0]) <= 1e-13 * abs(st_ref[0])
    assert st[2:].tolist() == st_ref[2:].tolist()
    assert abs(st[1] - st_ref[1]) <= 1e-11 * max(abs(st_ref[1]), 1e-300)


def test_sweep_sums_and_reblocked_mean_match_oracle(torch_cuda):
    """The 4-electron system over 96 sweeps: the accumulated sums of e_L and
    e_L^2 per sweep, and the reblocked mean and error bar of the samples, equal
    the oracle's on its own identical trajectory."""
    torch = torch_cuda
    import paper_2002_07401_gb300 as pg
    sysm = synth.config1()
    W, sweeps = 64, 96
    x0 = synth.init_walkers(sysm, W, seed=2)
    xo = x0.copy()
    eL_ref, _, _ = oracle.Oracle(sysm).vmc(xo, sweeps, seed=2)
    g = pg.JAGP(sysm, W, seed=2)
    r = g.positions(x0)
    g.eval(r)
    eL, acc = g.sweep(r, sweeps, acc=True)
    lev, st = pg.jagp_reblock(eL)
    torch.cuda.synchronize()
    assert np.array_equal(r.cpu().numpy(), xo)
    a, e = acc.cpu().numpy(), eL.cpu().numpy()
    # the samples agree to the FP64 bar, their sums to that bar times the terms' size
    assert np.all(np.abs(e - eL_ref) <= 1e-10 * np.maximum(1.0, np.abs(eL_ref)))
    assert np.all(np.abs(a[:, 0] - eL_ref.sum(axis=1)) <= 1e-10 * np.abs(eL_ref).sum(axis=1))
    assert np.all(np.abs(a[:, 1] - (eL_ref ** 2).sum(axis=1)) <= 3e-10 * (eL_ref ** 2).sum(axis=1))
    # the reblocking of these samples: the kernel against the oracle on the same values,
    # and the VMC mean against the oracle's own chain
    lev_ref, st_ref = oracle.reblock(e)
    assert _rel(lev.cpu().numpy()[:, 2:], lev_ref[:, 2:]) < 1e-11
    assert st.cpu().numpy()[2] == st_ref[2]
    assert abs(st.cpu().numpy()[0] - oracle.reblock(eL_ref)[1][0]) < 1e-10 * abs(st_ref[0])
    g.close()
