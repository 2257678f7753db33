"""FP64-equivalent lambda products on the tensor cores (fp64_tensor_cores=1):
the FP64 path's parity bar against the oracle (1e-10 relative on log|Psi| and
e_L, positions after sweeps identical move by move), on systems with L <= 512
(seven 8-bit slices) and L > 512 (eight 7-bit slices)."""
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
    "C1": synth.config1,
    "C2": synth.config2,
    "small-unpaired-slater": lambda: synth.small_random(n_atoms=3, n_up=4, n_dn=2, per_atom=20, seed=31,
                                                        slater_fraction=0.3),
    "mid-n40": lambda: synth.small_random(n_atoms=20, n_up=40, n_dn=37, per_atom=6, seed=33, side=7.0, Z=2.0),
    # L = 576 > 512: the 7-bit slicing
    "n48-L576": lambda: synth.small_random(n_atoms=24, n_up=48, n_dn=48, per_atom=24, seed=34, side=8.0, Z=2.0),
}


def _walkers(sysm, W, seed=5):
    return synth.jitter_walkers(synth.init_walkers(sysm, W, seed=seed), seed + 1, 0.3)


def _close(a, b, tol=TOL):
    a, b = np.asarray(a), np.asarray(b)
    return np.abs(a - b) <= tol * np.maximum(1.0, np.abs(b))


@pytest.mark.parametrize("name", list(SYSTEMS))
def test_fp64tc_eval_and_local_energy(torch_cuda, name):
    import paper_2002_07401_gb300 as pg
    sysm = SYSTEMS[name]()
    W = 7
    x = _walkers(sysm, W)
    o = oracle.Oracle(sysm)
    la_ref, sg_ref = o.logpsi_batch(x)
    e_ref = o.local_energy_batch(x)
    g = pg.JAGP(sysm, W, fp64_tc=True)
    r = g.positions(x)
    la, sg = g.eval(r)
    e = g.local_energy(r).cpu().numpy()
    assert g.status() == 0
    assert np.all(_close(la.cpu().numpy(), la_ref)), np.max(np.abs(la.cpu().numpy() - la_ref))
    assert np.array_equal(sg.cpu().numpy(), sg_ref)
    assert np.all(_close(e, e_ref)), np.max(np.abs(e - e_ref) / np.maximum(1, np.abs(e_ref)))
    g.close()


@pytest.mark.parametrize("name,W,sweeps", [("C1", 33, 8), ("C2", 6, 3), ("small-unpaired-slater", 9, 4),
                                           ("n48-L576", 3, 1)])
def test_fp64tc_sweep_trajectory(torch_cuda, name, W, sweeps):
    import paper_2002_07401_gb300 as pg
    sysm = SYSTEMS[name]()
    x0 = _walkers(sysm, W)
    xo = x0.copy()
    eL_ref, lp_ref, nacc_ref = oracle.Oracle(sysm).vmc(xo, sweeps, seed=7, sweep0=3)
    g = pg.JAGP(sysm, W, seed=7, fp64_tc=True)
    r = g.positions(x0)
    g.eval(r)
    eL, _ = g.sweep(r, sweeps, sweep0=3)
    info = g.info()
    assert g.status() & (pg.WS_NONFINITE | pg.WS_SINGULAR) == 0
    assert np.array_equal(r.cpu().numpy(), xo)
    assert np.array_equal(info["naccept"].cpu().numpy(), nacc_ref.astype(np.float64))
    assert np.all(_close(eL.cpu().numpy(), eL_ref))
    assert np.all(_close(info["logabs"].cpu().numpy(), lp_ref, 1e-9))
    g.close()


def test_fp64tc_full_size_c2_matches_native_fp64(torch_cuda):
    """C2 at 4096 walkers: the tensor-core FP64-equivalent run follows the
    native FP64 run move by move, e_L within 1e-10."""
    import paper_2002_07401_gb300 as pg
    sysm = synth.config2()
    W = 4096
    x0 = synth.init_walkers(sysm, W, seed=0)
    out = []
    for tc in (False, True):
        g = pg.JAGP(sysm, W, seed=0, fp64_tc=tc)
        r = g.positions(x0)
        g.eval(r)
        eL, _ = g.sweep(r, 2)
        out.append((r.cpu().numpy(), eL.cpu().numpy()))
        g.close()
    assert np.array_equal(out[0][0], out[1][0])
    assert np.all(_close(out[1][1], out[0][1]))


@pytest.mark.parametrize("name,W", [("mid-n40", 4), ("C2", 4), ("n48-L576", 80)])
def test_fp64tc_adjoint_matches_native(torch_cuda, name, W):
    """jagp_grad with the tensor-core FP64-equivalent lambda products equals the
    native FP64 adjoint to 1e-9 (relative to the largest component).  With
    N_dn = N_up (C2, the L = 576 system) lambda-bar runs on the tensor cores
    as well, in segments of 2048 // N_up walkers (the 80 walkers of the L = 576
    system make one full segment and a ragged one per row set)."""
    torch = torch_cuda
    import paper_2002_07401_gb300 as pg
    sysm = SYSTEMS[name]()
    x = _walkers(sysm, W, seed=12)
    rng = np.random.default_rng(W)
    sL = torch.tensor(rng.normal(size=W), dtype=torch.float64, device="cuda")
    sE = torch.tensor(rng.normal(size=W) / W, dtype=torch.float64, device="cuda")
    outs = []
    for tc in (False, True):
        g = pg.JAGP(sysm, W, fp64_tc=tc)
        r = g.positions(x)
        g.eval(r)
        o = g.grad(r, seed_logpsi=sL, seed_eL=sE)
        outs.append({k: v.cpu().numpy() for k, v in o.items() if v is not None})
        g.close()
    for k in ("eL", "lam", "jas", "R", "r"):
        a, b = outs[1][k], outs[0][k]
        scale = max(1.0, float(np.abs(b).max()))
        assert float(np.abs(a - b).max()) <= 1e-9 * scale, (k, float(np.abs(a - b).max()) / scale)
