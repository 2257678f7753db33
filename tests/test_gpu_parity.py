"""Parity of the CUDA path (through the C ABI) with the FP64 CPU oracle.

Tolerances (FP64 path): 1e-10 relative on log|Psi| and on e_L (relative to
max(1, |value|)); positions after Metropolis sweeps are compared exactly (the
proposals are built with one correctly rounded fma on both sides and the
accept decisions are taken in FP64 on both sides); acceptance counts exactly.
"""
import math

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

TOL = 1e-10


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def _systems():
    return {
        "C1": synth.config1(),
        "C2": synth.config2(),
        "small-unpaired-slater": synth.small_random(n_atoms=3, n_up=4, n_dn=2, per_atom=20, seed=31,
                                                     slater_fraction=0.3),
        "small-nonsym": synth.small_random(n_atoms=4, n_up=5, n_dn=5, per_atom=16, seed=32, symmetric=False),
        "hydrogen": synth.hydrogen_slater(),
        "helium": synth.helium_slater(1.6875),
        "hydrogenic-J1": synth.hydrogenic_gauss_j1(2.0),
        # N_up > 32 exercises the block-wide acceptance and refresh kernels
        "mid-n40": synth.small_random(n_atoms=20, n_up=40, n_dn=37, per_atom=6, seed=33, side=7.0, Z=2.0),
    }


SYSTEMS = _systems()


def _walkers(sysm, W, seed=5):
    x = synth.init_walkers(sysm, W, seed=seed)
    return synth.jitter_walkers(x, seed + 1, 0.3)


def _close(a, b, tol=TOL):
    a, b = np.asarray(a), np.asarray(b)
    return np.abs(a - b) <= tol * np.maximum(1.0, np.abs(b))


@pytest.mark.parametrize("name", list(SYSTEMS))
def test_eval_and_local_energy_parity(torch_cuda, name):
    import paper_2002_07401_gb300 as pg
    sysm = SYSTEMS[name]
    W = 37 if sysm.L < 100 else 19          # ragged walker counts
    x = _walkers(sysm, W)
    o = oracle.Oracle(sysm)
    la_ref, sg_ref = o.logpsi_batch(x)
    e_ref = o.local_energy_batch(x)
    g = pg.JAGP(sysm, W)
    r = g.positions(x)
    la, sg = g.eval(r)
    e = g.local_energy(r).cpu().numpy()
    assert g.status() == 0
    assert np.all(_close(la.cpu().numpy(), la_ref)), np.max(np.abs(la.cpu().numpy() - la_ref))
    assert np.array_equal(sg.cpu().numpy(), sg_ref)
    assert np.all(_close(e, e_ref)), np.max(np.abs(e - e_ref) / np.maximum(1, np.abs(e_ref)))
    g.close()


def test_energy_parts_parity(torch_cuda):
    import paper_2002_07401_gb300 as pg
    sysm = SYSTEMS["small-unpaired-slater"]
    x = _walkers(sysm, 5)
    o = oracle.Oracle(sysm)
    g = pg.JAGP(sysm, 5)
    r = g.positions(x)
    g.eval(r)
    e, parts = g.local_energy(r, parts=True)
    parts = parts.cpu().numpy()
    for w in range(5):
        ref = o.local_energy(x[w], parts=True)
        # (kinetic, V_ee, V_ei, V_ii)
        assert np.all(_close(parts[w], [ref[1], ref[2], ref[3], ref[4]]))


@pytest.mark.parametrize("name,W,sweeps", [("C1", 33, 12), ("C2", 6, 3), ("small-unpaired-slater", 17, 6),
                                           ("small-nonsym", 9, 4), ("helium", 40, 10),
                                           ("mid-n40", 5, 2)])
def test_sweep_trajectory_parity(torch_cuda, name, W, sweeps):
    """Same seed, same counters: identical positions and acceptance, e_L within 1e-10."""
    import paper_2002_07401_gb300 as pg
    sysm = SYSTEMS[name]
    x0 = _walkers(sysm, W)
    xo = x0.copy()
    o = oracle.Oracle(sysm)
    eL_ref, lp_ref, nacc_ref = o.vmc(xo, sweeps, seed=7, sweep0=3, walker0=0)
    g = pg.JAGP(sysm, W, seed=7)
    r = g.positions(x0)
    g.eval(r)
    eL, acc = g.sweep(r, sweeps, walker0=0, sweep0=3, acc=True)
    info = g.info()
    # the drift bit only reports how far the Sherman-Morrison inverse moved
    # from the fresh FP64 one before the refresh replaced it
    assert g.status() & (pg.WS_NONFINITE | pg.WS_SINGULAR) == 0
    drift = info["drift"].cpu().numpy()
    assert np.all(drift < 1e-5), drift.max()
    assert np.array_equal(r.cpu().numpy(), xo)
    assert np.array_equal(info["naccept"].cpu().numpy(), nacc_ref.astype(np.float64))
    assert np.all(_close(eL.cpu().numpy(), eL_ref))
    assert np.all(_close(info["logabs"].cpu().numpy(), lp_ref, 1e-9))
    a = acc.cpu().numpy()
    assert np.allclose(a[:, 0], eL_ref.sum(1), rtol=1e-10, atol=1e-9)
    assert a[:, 2].sum() == nacc_ref.sum()
    g.close()


def test_hydrogen_zero_variance_on_gpu(torch_cuda):
    import paper_2002_07401_gb300 as pg
    sysm = SYSTEMS["hydrogen"]
    W = 256
    g = pg.JAGP(sysm, W)
    r = g.positions(_walkers(sysm, W))
    g.eval(r)
    eL, _ = g.sweep(r, 5)
    assert np.max(np.abs(eL.cpu().numpy() + 0.5)) < 1e-12


def test_full_size_c2_sampled(torch_cuda):
    """C2 at its full walker count (4096) in the launch shape the bench times:
    16 sampled walkers re-run by the oracle from the same start."""
    import paper_2002_07401_gb300 as pg
    sysm = SYSTEMS["C2"]
    W, sweeps = 4096, 2
    x0 = synth.init_walkers(sysm, W, seed=0)
    g = pg.JAGP(sysm, W, seed=0)
    r = g.positions(x0)
    g.eval(r)
    eL, _ = g.sweep(r, sweeps)
    assert g.status() == 0
    xg = r.cpu().numpy()
    eg = eL.cpu().numpy()
    o = oracle.Oracle(sysm)
    for w in np.random.default_rng(0).choice(W, size=16, replace=False):
        xs = np.ascontiguousarray(x0[w:w + 1])
        e_ref, _, _ = o.vmc(xs, sweeps, seed=0, walker0=int(w))
        assert np.array_equal(xs[0], xg[w])
        assert np.all(_close(eg[:, w], e_ref[:, 0]))


def test_determinism_and_edge_cases(torch_cuda):
    import paper_2002_07401_gb300 as pg
    sysm = SYSTEMS["C1"]
    x0 = _walkers(sysm, 3)
    outs = []
    for _ in range(2):
        g = pg.JAGP(sysm, 3, seed=1)
        r = g.positions(x0)
        g.eval(r)
        eL, acc = g.sweep(r, 4, acc=True)
        outs.append((r.cpu().numpy(), eL.cpu().numpy(), acc.cpu().numpy()))
        g.close()
    assert all(np.array_equal(a, b) for a, b in zip(outs[0], outs[1]))
    # W = 1 works; W = 0 and W > max_walkers are argument errors
    g = pg.JAGP(sysm, 3)
    r = g.positions(x0[:1])
    la, _ = g.eval(r)
    assert _close(la.cpu().numpy(), oracle.Oracle(sysm).logpsi_batch(x0[:1])[0]).all()
    with pytest.raises(pg.JagpError):
        pg.jagp_eval(g.h, r, 0, g.state)
    with pytest.raises(pg.JagpError):
        pg.jagp_eval(g.h, r, 4, g.state)
    g.close()


def test_nonfinite_position_sets_status(torch_cuda):
    """A walker poisoned on the host with NaN is flagged NONFINITE, the others
    are untouched; jagp_walker_status records which walkers carry bits."""
    import paper_2002_07401_gb300 as pg
    sysm = SYSTEMS["C1"]
    x = _walkers(sysm, 4)
    x[2, 1, 0] = np.nan
    g = pg.JAGP(sysm, 4)
    r = g.positions(x)
    la, _ = g.eval(r)
    info = g.info()
    st = info["status"].cpu().numpy()
    assert st[2] & pg.WS_NONFINITE and st[0] == st[1] == st[3] == 0
    ref, _ = oracle.Oracle(sysm).logpsi_batch(x[[0, 1, 3]])
    assert np.all(_close(la.cpu().numpy()[[0, 1, 3]], ref))
    assert g.status() & pg.WS_NONFINITE
    code, text = pg.jagp_last_error(g.h)
    assert code == 0 and "1 of 4 walkers" in text
    g.close()


def test_last_error_records_the_failing_call(torch_cuda):
    """jagp_last_error gives the failing entry point and the offending value."""
    import paper_2002_07401_gb300 as pg
    sysm = SYSTEMS["C1"]
    g = pg.JAGP(sysm, 4)
    assert pg.jagp_last_error(g.h) == (0, "no error")
    r = g.positions(_walkers(sysm, 8))
    with pytest.raises(pg.JagpError, match="W = 8 outside 1..4"):
        pg.jagp_eval(g.h, r, 8, g.state)
    code, text = pg.jagp_last_error(g.h)
    assert code == 1 and text.startswith("jagp_eval: invalid argument")
    with pytest.raises(pg.JagpError, match="vmc_sweep"):
        pg.vmc_sweep(g.h, r, g.state, 0, 1)
    assert pg.jagp_last_error(g.h)[1].startswith("vmc_sweep: invalid argument")
    g.close()


@pytest.mark.parametrize("name,W,sweeps,k", [("small-unpaired-slater", 9, 3, 1), ("C2", 4, 2, 5),
                                             ("mid-n40", 3, 2, 16)])
def test_sweep_trajectory_parity_with_refresh_every_k_moves(torch_cuda, name, W, sweeps, k):
    """Refreshing G~^-1 from the tables every k moves of a spin half-sweep
    (the option the batched workload uses with k = 16) keeps the trajectory
    move-by-move identical to the oracle's."""
    import paper_2002_07401_gb300 as pg
    sysm = SYSTEMS[name]
    x0 = _walkers(sysm, W, seed=9)
    xo = x0.copy()
    eL_ref, lp_ref, nacc_ref = oracle.Oracle(sysm).vmc(xo, sweeps, seed=5, sweep0=1, walker0=2)
    g = pg.JAGP(sysm, W, seed=5, refresh_moves=k)
    r = g.positions(x0)
    g.eval(r)
    eL, acc = g.sweep(r, sweeps, walker0=2, sweep0=1, acc=True)
    info = g.info()
    assert g.status() & (pg.WS_NONFINITE | pg.WS_SINGULAR) == 0
    assert np.array_equal(r.cpu().numpy(), xo)
    assert np.array_equal(info["naccept"].cpu().numpy(), nacc_ref.astype(np.float64))
    assert acc.cpu().numpy()[:, 2].sum() == nacc_ref.sum()
    assert np.all(_close(eL.cpu().numpy(), eL_ref))
    g.close()
