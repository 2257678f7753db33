"""GPU parity of the three/four-body Jastrow factor (Eq. threebody_jastrow):
FP64 path: log|Psi| and e_L element by element, and Metropolis trajectories
move by move (the sequential acceptance keeps the spin sums of the Jastrow
basis and their products with the couplings), against the oracle's plain
pair sums.  Mixed path: log|Psi| and e_L within its stated targets (1e-6,
1e-5 Ha) at seeded configurations and after sweeps."""
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


SYSTEMS = {
    "small-unpaired": lambda: synth.with_j3(synth.small_random(n_atoms=3, n_up=3, n_dn=2, per_atom=6, seed=131,
                                                               slater_fraction=0.3), seed=131, sd=0.2),
    "C1": lambda: synth.with_j3(synth.config1(), seed=132, sd=0.2),
    "C2": lambda: synth.with_j3(synth.config2(), seed=133, sd=0.05),
    "mid-n40": lambda: synth.with_j3(synth.small_random(n_atoms=20, n_up=40, n_dn=40, per_atom=6, seed=134,
                                                        side=9.0, Z=2.0), seed=134, sd=0.05),
}


def _close(a, b, tol=TOL):
    a, b = np.asarray(a), np.asarray(b)
    return np.all(np.abs(a - b) <= tol * np.maximum(1.0, np.abs(b)))


@pytest.mark.parametrize("name", list(SYSTEMS))
def test_j3_eval_and_local_energy(torch_cuda, name):
    import paper_2002_07401_gb300 as pg
    sysm = SYSTEMS[name]()
    W = 8
    x = synth.jitter_walkers(synth.init_walkers(sysm, W, seed=2), 3, 0.3)
    o = oracle.Oracle(sysm)
    la_ref, sg_ref = o.logpsi_batch(x)
    e_ref = o.local_energy_batch(x)
    g = pg.JAGP(sysm, W)
    r = g.positions(x)
    la, sg = g.eval(r)
    e = g.local_energy(r)
    assert _close(la.cpu().numpy(), la_ref)
    assert np.array_equal(sg.cpu().numpy(), sg_ref)
    assert _close(e.cpu().numpy(), e_ref)
    g.close()


@pytest.mark.parametrize("name,k", [("small-unpaired", 0), ("C2", 0), ("C2", 5), ("mid-n40", 16)])
def test_j3_trajectory_parity(torch_cuda, name, k):
    import paper_2002_07401_gb300 as pg
    sysm = SYSTEMS[name]()
    W, sweeps = 5, 3
    x0 = synth.jitter_walkers(synth.init_walkers(sysm, W, seed=7), 8, 0.3)
    xo = x0.copy()
    eL_ref, lp_ref, nacc_ref = oracle.Oracle(sysm).vmc(xo, sweeps, seed=9, sweep0=1, walker0=2)
    g = pg.JAGP(sysm, W, seed=9, refresh_moves=k)
    r = g.positions(x0)
    g.eval(r)
    eL, _ = g.sweep(r, sweeps, walker0=2, sweep0=1)
    assert g.status() & (pg.WS_NONFINITE | pg.WS_SINGULAR) == 0
    assert np.array_equal(r.cpu().numpy(), xo)
    info = g.info()
    assert np.array_equal(info["naccept"].cpu().numpy(), nacc_ref.astype(np.float64))
    assert _close(eL.cpu().numpy(), eL_ref)
    assert _close(info["logabs"].cpu().numpy(), lp_ref)
    g.close()


def test_j3_unsupported_paths(torch_cuda):
    torch = torch_cuda
    import paper_2002_07401_gb300 as pg
    sysm = SYSTEMS["small-unpaired"]()
    g = pg.JAGP(sysm, 4)
    r = g.positions(synth.init_walkers(sysm, 4, seed=1))
    g.eval(r)
    with pytest.raises(pg.JagpError, match="three-body"):
        g.grad(r, seed_logpsi=torch.ones(4, dtype=torch.float64, device="cuda"))
    with pytest.raises(pg.JagpError, match="three-body"):
        pg.jagp_set_guiding(g.h, 0.375, 1e-3)
    la = torch.empty(4, dtype=torch.float64, device="cuda")
    with pytest.raises(pg.JagpError, match="three-body"):
        pg.jagp_eval_noalloc(g.h, r, 4, la, None)
    work = torch.empty(pg.jagp_lrdmc_workspace_bytes(g.h, 4), dtype=torch.uint8, device="cuda")
    w = torch.ones(4, dtype=torch.float64, device="cuda")
    with pytest.raises(pg.JagpError, match="three-body"):
        pg.jagp_lrdmc_project(g.h, r, g.state, 4, work, w, 0, 0.2, 0.0, 0.1, 0.0)
    g.close()


@pytest.mark.parametrize("name", list(SYSTEMS))
def test_j3_mixed_path(torch_cuda, name):
    """The mixed path with the three-body Jastrow (its change in FP64 in the
    acceptance kernel, its value, gradient and Laplacian in FP64 in the
    double-word local energy): log|Psi| and e_L at seeded configurations,
    then after two sweeps at the walkers' final positions, against the oracle
    within 1e-6 and 1e-5 Ha."""
    import paper_2002_07401_gb300 as pg
    sysm = SYSTEMS[name]()
    W = 8
    x = synth.jitter_walkers(synth.init_walkers(sysm, W, seed=2), 3, 0.3)
    o = oracle.Oracle(sysm)
    g = pg.JAGP(sysm, W, precision=pg.JAGP_PREC_MIXED, seed=4)
    r = g.positions(x)
    la, sg = g.eval(r)
    e = g.local_energy(r).cpu().numpy()
    la_ref, sg_ref = o.logpsi_batch(x)
    e_ref = o.local_energy_batch(x)
    assert np.array_equal(sg.cpu().numpy(), sg_ref)
    assert np.abs(la.cpu().numpy() - la_ref).max() <= 1e-6
    assert np.abs(e - e_ref).max() <= 1e-5, np.abs(e - e_ref).max()
    eL, acc = g.sweep(r, 2, acc=True)
    assert g.status() & (pg.WS_NONFINITE | pg.WS_SINGULAR) == 0
    assert acc.cpu().numpy()[:, 2].sum() > 0
    xf = np.ascontiguousarray(r.cpu().numpy())
    la_ref, _ = o.logpsi_batch(xf)
    e_ref = o.local_energy_batch(xf)
    assert np.abs(g.info()["logabs"].cpu().numpy() - la_ref).max() <= 1e-6
    assert np.abs(eL.cpu().numpy()[-1] - e_ref).max() <= 1e-5
    g.close()
