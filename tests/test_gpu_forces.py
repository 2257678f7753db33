"""GPU parity of the finite-variance force estimator's parts (Sec. "Atomic
forces"): the space-warp transformation applied to the adjoint's per-walker
derivatives, the guiding function's R(x) and weights, and the seeds of the
reweighted estimator, against the oracle (warped derivatives from its
analytic log|Psi| gradients and finite-difference e_L gradients)."""
import math

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


SYSTEMS = {
    "small-slater": lambda: synth.small_random(n_atoms=3, n_up=3, n_dn=2, per_atom=6, seed=111, slater_fraction=0.3),
    "small-sym": lambda: synth.small_random(n_atoms=4, n_up=2, n_dn=2, per_atom=6, seed=112),
}


@pytest.mark.parametrize("name", list(SYSTEMS))
def test_space_warp_matches_oracle(torch_cuda, name):
    """Per walker sE dEL_warp + sL dLJ_warp (oracle) against jagp_grad +
    jagp_space_warp with the same seeds, and their sum over walkers."""
    torch = torch_cuda
    import paper_2002_07401_gb300 as pg
    sysm = SYSTEMS[name]()
    W = 5
    x = synth.jitter_walkers(synth.init_walkers(sysm, W, seed=6), 7, 0.3)
    rng = np.random.default_rng(8)
    sL, sE = rng.normal(size=W), rng.uniform(0.1, 1.0, size=W)
    g = pg.JAGP(sysm, W)
    r = g.positions(x)
    g.eval(r)
    out = g.grad(r, seed_logpsi=torch.tensor(sL, device="cuda"), seed_eL=torch.tensor(sE, device="cuda"),
                 want_lambda=False)
    Rw = out["R_walker"].clone()
    dR = torch.empty_like(out["R"])
    pg.jagp_space_warp(g.h, r, W, out["r"], Rw, seed_logpsi=torch.tensor(sL, device="cuda"), dR=dR)
    o = oracle.Oracle(sysm)
    want = np.zeros((W, sysm.n_atoms, 3))
    for w in range(W):
        dE, dL = o.swct_derivs(x[w], h=1e-3)
        want[w] = sE[w] * dE + sL[w] * dL
    got = Rw.cpu().numpy()
    scale = np.abs(want).max()
    assert np.abs(got - want).max() <= 1e-7 * (1 + scale)
    assert np.abs(dR.cpu().numpy() - want.sum(axis=0)).max() <= 1e-7 * (1 + scale)
    g.close()


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_guiding_weights_match_oracle(torch_cuda, prec):
    torch = torch_cuda
    import paper_2002_07401_gb300 as pg
    sysm = synth.small_random(n_atoms=3, n_up=3, n_dn=3, per_atom=6, seed=113)
    W = 16
    x = synth.jitter_walkers(synth.init_walkers(sysm, W, seed=9), 10, 0.4)
    g = pg.JAGP(sysm, W, precision=pg.JAGP_PREC_MIXED if prec == "mixed" else pg.JAGP_PREC_FP64)
    r = g.positions(x)
    g.eval(r)
    R = torch.empty(W, dtype=torch.float64, device="cuda")
    Wt = torch.empty(W, dtype=torch.float64, device="cuda")
    o = oracle.Oracle(sysm)
    ref = np.array([o.guiding_R(x[w], 0.375) for w in range(W)])
    eps = float(np.median(ref))
    pg.jagp_guiding_weights(g.h, g.state, W, 0.375, eps, R, Wt)
    tol = 1e-10 if prec == "fp64" else 1e-5      # the mixed state keeps G~^{-1} in FP32
    assert np.max(np.abs(R.cpu().numpy() - ref) / ref) < tol
    wref = np.minimum(1.0, ref / eps) ** 2
    assert np.max(np.abs(Wt.cpu().numpy() - wref)) < 10 * tol
    g.close()


def test_force_seeds(torch_cuda):
    torch = torch_cuda
    import paper_2002_07401_gb300 as pg
    rng = np.random.default_rng(12)
    e = rng.normal(-3.0, 0.4, size=300)
    u = rng.uniform(0.2, 1.0, size=300)
    for weights in (None, u):
        sL, sE, mean = pg.jagp_force_seeds(torch.tensor(e, device="cuda"),
                                           None if weights is None else torch.tensor(weights, device="cuda"))
        uu = np.ones_like(e) if weights is None else weights
        E = np.sum(uu * e) / uu.sum()
        assert np.allclose(sE.cpu().numpy(), uu / uu.sum(), rtol=1e-13, atol=0)
        assert np.allclose(sL.cpu().numpy(), 2 * uu * (e - E) / uu.sum(), rtol=1e-11, atol=1e-15)
        assert abs(mean.cpu().numpy()[0] - E) < 1e-13 * abs(E)


GUIDED = {
    "small-unpaired": lambda: synth.small_random(n_atoms=3, n_up=3, n_dn=2, per_atom=6, seed=114,
                                                 slater_fraction=0.3),
    "C2": synth.config2,
    "mid-n40": lambda: synth.small_random(n_atoms=20, n_up=40, n_dn=40, per_atom=6, seed=115, side=9.0, Z=2.0),
}


@pytest.mark.parametrize("name", list(GUIDED))
def test_guided_sampling_trajectory_parity(torch_cuda, name):
    """Sampling the guiding function: positions move by move identical to the
    oracle's guided chain (which takes R from full inverses of every proposed
    G~), local energies to the FP64 bar; eps at the median R of the start."""
    torch = torch_cuda
    import paper_2002_07401_gb300 as pg
    sysm = GUIDED[name]()
    W, sweeps = 6, 3
    x0 = synth.jitter_walkers(synth.init_walkers(sysm, W, seed=13), 14, 0.3)
    o = oracle.Oracle(sysm)
    eps = float(np.median([o.guiding_R(x0[w]) for w in range(W)]))
    xo = x0.copy()
    eL_ref, _, nacc_ref, _ = o.vmc_guided(xo, sweeps, eps=eps, seed=15, walker0=3, sweep0=2)
    g = pg.JAGP(sysm, W, seed=15)
    pg.jagp_set_guiding(g.h, 0.375, eps)
    r = g.positions(x0)
    g.eval(r)
    eL, _ = g.sweep(r, sweeps, walker0=3, sweep0=2)
    assert g.status() & (pg.WS_NONFINITE | pg.WS_SINGULAR) == 0
    assert np.array_equal(r.cpu().numpy(), xo)
    assert np.array_equal(g.info()["naccept"].cpu().numpy(), nacc_ref.astype(np.float64))
    e = eL.cpu().numpy()
    assert np.all(np.abs(e - eL_ref) <= 1e-10 * np.maximum(1.0, np.abs(eL_ref)))
    # eps = 0 restores the plain sampler
    pg.jagp_set_guiding(g.h, 0.375, 0.0)
    g.close()


def test_guiding_rejects_unsupported_handles(torch_cuda):
    import paper_2002_07401_gb300 as pg
    gm = pg.JAGP(synth.config2(), 4, precision=pg.JAGP_PREC_MIXED)
    with pytest.raises(pg.JagpError, match="FP64 handle"):
        pg.jagp_set_guiding(gm.h, 0.375, 1e-3)
    with pytest.raises(pg.JagpError, match="theta"):
        pg.jagp_set_guiding(gm.h, -1.0, 0.0)
    gm.close()


def test_tuned_eps_gives_the_target_mean_weight(torch_cuda):
    """The automatic choice of eps (the paper: <W> near 0.8) on the C2 workload."""
    torch = torch_cuda
    import paper_2002_07401_gb300 as pg
    sysm = synth.config2()
    W = 1024
    g = pg.JAGP(sysm, W, seed=16)
    r = g.positions(synth.init_walkers(sysm, W, seed=16))
    g.eval(r)
    g.sweep(r, 10, energies=False)
    eps = pg.tune_guiding_eps(g, r, target=0.8)
    g.sweep(r, 6, sweep0=100, energies=False)
    wt = torch.empty(W, dtype=torch.float64, device="cuda")
    pg.jagp_guiding_weights(g.h, g.state, W, 0.375, eps, weights=wt)
    assert eps > 0 and abs(float(wt.mean()) - 0.8) < 0.1
    g.close()
