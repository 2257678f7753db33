"""Batched uneven systems (jagp_batch_*): one CUDA graph per sweep over all
systems gives the per-system vmc_sweep results (same Philox counters), for
both precisions: bit for bit with per-system launches over streams (the same
kernels), and with grouped launches (one launch per kernel and point of the
sweep over all systems: the same formulas, compiled into another kernel) the
same trajectories and local energies equal up to rounding."""
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


def _systems():
    # the batched workload's generator, first few systems (uneven N)
    return synth.config3_systems(seed=0, n_systems=5)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("n_streams,refresh", [(0, 0), (0, 16), (-2, 16), (3, 0)])
def test_batch_equals_individual_sweeps(torch_cuda, precision, n_streams, refresh):
    """Five systems with N_up = 23..61 (both acceptance kernels, both refresh
    forms of the mixed path); refresh every 16 moves gives them two to four
    chunks per half-sweep, so the grouped launches of later chunks hold only
    some of the systems."""
    torch = torch_cuda
    import paper_2002_07401_gb300 as pg
    prec = pg.JAGP_PREC_MIXED if precision == "mixed" else pg.JAGP_PREC_FP64
    systems = _systems()
    Ws = [13, 7, 21, 5, 9]
    sweeps, sweep0 = 4, 10
    xs = [synth.init_walkers(s, W, seed=3) for s, W in zip(systems, Ws)]
    # individual
    ref_r, ref_e, ref_acc = [], [], []
    per_system_launches = 0
    for s, W, x in zip(systems, Ws, xs):
        g = pg.JAGP(s, W, seed=5, precision=prec, refresh_moves=refresh)
        r = g.positions(x)
        g.eval(r)
        n0 = pg.jagp_launch_count(g.h)
        eL, acc = g.sweep(r, sweeps, walker0=100, sweep0=sweep0, acc=True)
        per_system_launches += (pg.jagp_launch_count(g.h) - n0) // sweeps
        ref_r.append(r.cpu().numpy())
        ref_e.append(eL[-1].cpu().numpy())
        ref_acc.append(acc.cpu().numpy())
        g.close()
    # batched
    members = [pg.JAGP(s, W, seed=5, precision=prec, refresh_moves=refresh) for s, W in zip(systems, Ws)]
    pos = [m.positions(x) for m, x in zip(members, xs)]
    for m, p in zip(members, pos):
        m.eval(p)
    b = pg.Batch(members, pos, walker0=[100] * len(members), n_streams=n_streams)
    b.sweep(2, sweep0=sweep0)
    b.sweep(2, sweep0=sweep0 + 2)   # replays the captured graph
    torch.cuda.synchronize()
    graph_launches = b.launches_per_sweep()
    print(f"{precision} streams={n_streams} refresh={refresh}: {graph_launches} launches per batched sweep, "
          f"{per_system_launches} per-system launches")
    if n_streams <= 0:
        # one launch per kernel and point of the sweep (and lane), not one per system
        assert graph_launches < 0.5 * max(1, -n_streams) * per_system_launches, (graph_launches, per_system_launches)
    acc = b.acc.cpu().numpy()
    for k in range(len(systems)):
        assert np.array_equal(pos[k].cpu().numpy(), ref_r[k]), k
        e = b.eL[k].cpu().numpy()
        if n_streams > 0:
            assert np.array_equal(e, ref_e[k]), k
        else:
            assert np.allclose(e, ref_e[k], rtol=1e-11, atol=1e-11), (k, np.abs(e - ref_e[k]).max())
        assert acc[k, 2] == ref_acc[k][:, 2].sum()
        assert abs(acc[k, 0] - ref_acc[k][:, 0].sum()) <= 1e-9 * abs(ref_acc[k][:, 0]).sum()
        assert members[k].status() & (pg.WS_NONFINITE | pg.WS_SINGULAR) == 0
    b.close()


def test_batched_full_size_sampled(torch_cuda):
    """The batched workload at full size (64 systems, N = 8..128, 512 walkers
    each, refresh every 16 moves, every system autotuned, one graph of grouped
    launches, fewer than 150 per sweep): after one sweep, one sampled walker of
    each of five systems (the smallest, the largest and three others) is
    recomputed by the oracle."""
    torch = torch_cuda
    import oracle
    import paper_2002_07401_gb300 as pg
    systems = synth.config3_systems(seed=0, n_systems=64)
    W = 512
    members, pos = [], []
    for s in systems:
        m = pg.JAGP(s, W, seed=0, precision=pg.JAGP_PREC_MIXED, refresh_moves=16)
        p = m.positions(synth.init_walkers(s, W, seed=0))
        m.eval(p)
        m.autotune(p)
        members.append(m)
        pos.append(p)
    b = pg.Batch(members, pos, n_streams=0)
    b.sweep(1, sweep0=0)
    torch.cuda.synchronize()
    assert b.launches_per_sweep() < 150, b.launches_per_sweep()
    Ns = [s.N for s in systems]
    picks = sorted({int(np.argmin(Ns)), int(np.argmax(Ns)), 5, 23, 41})
    rng = np.random.default_rng(11)
    for k in picks:
        assert members[k].status() & (pg.WS_NONFINITE | pg.WS_SINGULAR) == 0, k
        w = int(rng.integers(W))
        x = np.ascontiguousarray(pos[k].cpu().numpy()[w:w + 1])
        o = oracle.Oracle(systems[k])
        la_ref, _ = o.logpsi_batch(x)
        e_ref = o.local_energy_batch(x)
        la = members[k].info()["logabs"].cpu().numpy()[w]
        e = b.eL[k].cpu().numpy()[w]
        assert abs(la - la_ref[0]) <= 1e-6, (k, la, la_ref[0])
        assert abs(e - e_ref[0]) <= 1e-5, (k, e, e_ref[0])
    b.close()
    for m in members:
        m.close()
