"""Adjoint derivatives (jagp_grad) against the FP64 oracle.

log|Psi| parts: the oracle's analytic gradients (themselves pinned by central
differences), tolerance 1e-9 relative to the largest component.  e_L parts:
the oracle's Richardson-extrapolated central differences of its own local
energy (h = 5e-4 bohr, error O(h^4)), tolerance 1e-7 relative to the largest
component.  Properties: translation invariance (sum over nuclei and electrons
of the derivative vanishes for both log|Psi| and e_L) and zero e_L derivatives
of exact eigenstates.
"""
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
    "small-unpaired-slater": lambda: synth.small_random(n_atoms=3, n_up=4, n_dn=2, per_atom=20, seed=31,
                                                        slater_fraction=0.3),
    "small-nonsym": lambda: synth.small_random(n_atoms=4, n_up=5, n_dn=5, per_atom=16, seed=32, symmetric=False),
    "C1": lambda: synth.config1(),
    "mid-n40": lambda: synth.small_random(n_atoms=20, n_up=40, n_dn=37, per_atom=6, seed=33, side=7.0, Z=2.0),
}


def _cfgs(sysm, W, seed=5):
    return synth.jitter_walkers(synth.init_walkers(sysm, W, seed=seed), seed + 1, 0.3)


def _close(a, b, rel):
    a, b = np.asarray(a), np.asarray(b)
    scale = max(1.0, float(np.abs(b).max()))
    return float(np.abs(a - b).max()) <= rel * scale, float(np.abs(a - b).max()) / scale


@pytest.mark.parametrize("name", list(SYSTEMS))
def test_logpsi_gradients_match_oracle(torch_cuda, name):
    torch = torch_cuda
    import paper_2002_07401_gb300 as pg
    sysm = SYSTEMS[name]()
    W = 5
    x = _cfgs(sysm, W)
    o = oracle.Oracle(sysm)
    seeds = np.random.default_rng(1).normal(size=W)
    g = pg.JAGP(sysm, W)
    r = g.positions(x)
    g.eval(r)
    out = g.grad(r, seed_logpsi=torch.tensor(seeds, device="cuda"))
    ref = [o.grad_logpsi(x[w]) for w in range(W)]
    lam_ref = sum(s * d["lam"] for s, d in zip(seeds, ref))
    jas_ref = sum(s * d["jas"] for s, d in zip(seeds, ref))
    R_ref = sum(s * d["R"] for s, d in zip(seeds, ref))
    r_ref = np.stack([s * d["r"] for s, d in zip(seeds, ref)])
    for got, want, what in ((out["lam"], lam_ref, "lambda"), (out["jas"], jas_ref, "jastrow"), (out["R"], R_ref, "R"),
                            (out["r"], r_ref, "r")):
        ok, err = _close(got.cpu().numpy(), want, 1e-9)
        assert ok, (what, err)
    Rw = out["R_walker"].cpu().numpy()
    for w in range(W):
        assert _close(Rw[w], seeds[w] * ref[w]["R"], 1e-9)[0]


@pytest.mark.parametrize("name", ["small-unpaired-slater", "small-nonsym", "C1"])
def test_local_energy_gradients_match_fd(torch_cuda, name):
    torch = torch_cuda
    import paper_2002_07401_gb300 as pg
    sysm = SYSTEMS[name]()
    W = 3
    x = _cfgs(sysm, W, seed=9)
    o = oracle.Oracle(sysm)
    seeds = np.array([1.0, -0.7, 0.4])
    g = pg.JAGP(sysm, W)
    r = g.positions(x)
    g.eval(r)
    out = g.grad(r, seed_eL=torch.tensor(seeds, device="cuda"))
    Rw = out["R_walker"].cpu().numpy()
    rr = out["r"].cpu().numpy()
    for w in range(W):
        dR, dr = o.elocal_grad(x[w], h=5e-4)
        ok, err = _close(Rw[w], seeds[w] * dR, 1e-7)
        assert ok, ("R", w, err)
        ok, err = _close(rr[w], seeds[w] * dr, 1e-7)
        assert ok, ("r", w, err)
    # lambda: a few entries by central differences of the oracle's e_L
    lam = out["lam"].cpu().numpy()
    rng = np.random.default_rng(2)
    for _ in range(4):
        mu, nu = rng.integers(sysm.L, size=2)
        fd = sum(seeds[w] * o.elocal_dlambda(x[w], mu, nu) for w in range(W))
        assert abs(lam[mu, nu] - fd) <= 1e-6 * max(1.0, abs(fd)), (mu, nu, lam[mu, nu], fd)


@pytest.mark.parametrize("name", list(SYSTEMS))
def test_translation_invariance_of_force_vjp(torch_cuda, name):
    torch = torch_cuda
    import paper_2002_07401_gb300 as pg
    sysm = SYSTEMS[name]()
    W = 4
    x = _cfgs(sysm, W, seed=11)
    g = pg.JAGP(sysm, W)
    r = g.positions(x)
    g.eval(r)
    eL = g.local_energy(r)
    # the force estimator's seeds: sL = 2 (e_L - <e_L>) / W, sE = 1 / W
    sL = 2.0 * (eL - eL.mean()) / W
    sE = torch.full((W,), 1.0 / W, dtype=torch.float64, device="cuda")
    out = g.grad(r, seed_logpsi=sL, seed_eL=sE, want_lambda=False)
    Rw, rr = out["R_walker"].cpu().numpy(), out["r"].cpu().numpy()
    for w in range(W):
        tot = Rw[w].sum(0) + rr[w].sum(0)
        scale = max(1.0, np.abs(Rw[w]).max(), np.abs(rr[w]).max())
        assert np.abs(tot).max() <= 1e-9 * scale, (w, tot)


def test_exact_eigenstates_have_zero_local_energy_derivatives(torch_cuda):
    torch = torch_cuda
    import paper_2002_07401_gb300 as pg
    for sysm in (synth.hydrogen_slater(), synth.hydrogenic_gauss_j1(2.0)):
        W = 8
        g = pg.JAGP(sysm, W)
        r = g.positions(_cfgs(sysm, W, seed=3))
        g.eval(r)
        out = g.grad(r, seed_eL=torch.ones(W, dtype=torch.float64, device="cuda"), want_lambda=False)
        assert np.abs(out["r"].cpu().numpy()).max() < 1e-11
        assert np.abs(out["R"].cpu().numpy()).max() < 1e-10


def test_autograd_function_force(torch_cuda):
    """The force estimator through torch.autograd: -dE/dR with E = <e_L> and the
    Pulay term from the log|Psi| dependence of the sampling distribution."""
    torch = torch_cuda
    import paper_2002_07401_gb300 as pg
    sysm = SYSTEMS["small-nonsym"]()
    W = 6
    x = _cfgs(sysm, W, seed=13)
    g = pg.JAGP(sysm, W)
    lam = torch.tensor(sysm.lam, device="cuda", requires_grad=True)
    # d e_L / d b is not formed: the Jastrow parameters stay out of this graph
    jas = torch.tensor([sysm.b_ea, sysm.b_para, sysm.b_anti], dtype=torch.float64, device="cuda")
    R = torch.tensor(sysm.R, device="cuda", requires_grad=True)
    r = g.positions(x).requires_grad_(True)
    logpsi, eL = pg.logpsi_and_local_energy(g, lam, jas, R, r)
    E = eL.mean()
    surrogate = E + 2.0 * ((eL - E).detach() * logpsi).mean()
    surrogate.backward()
    grad_R = R.grad.clone()
    # with the Jastrow parameters in the graph, an e_L gradient reaching them raises
    jas_g = jas.clone().requires_grad_(True)
    lp2, el2 = pg.logpsi_and_local_energy(g, lam, jas_g, R, r)
    with pytest.raises(pg.JagpError, match="not formed"):
        el2.sum().backward()
    lp3, _ = pg.logpsi_and_local_energy(g, lam, jas_g, R, r)
    lp3.sum().backward()            # the log|Psi| part alone is formed
    assert jas_g.grad is not None
    o = oracle.Oracle(sysm)
    el = np.array([o.local_energy(x[w]) for w in range(W)])
    want = np.zeros_like(sysm.R)
    for w in range(W):
        dR, _ = o.elocal_grad(x[w], h=5e-4)
        want += dR / W + 2.0 * (el[w] - el.mean()) / W * o.grad_logpsi(x[w], want_lam=False)["R"]
    ok, err = _close(grad_R.cpu().numpy(), want, 1e-7)
    assert ok, err


def test_large_nup_gradients_match_oracle(torch_cuda):
    """N_up = 121 (> 64): the adjoint's G~-sized steps run as per-walker GEMMs.
    log|Psi| gradients against the oracle's analytic ones, and the translation
    invariance of the e_L part."""
    torch = torch_cuda
    import paper_2002_07401_gb300 as pg
    sysm = synth.small_random(n_atoms=60, n_up=121, n_dn=119, per_atom=6, seed=51, side=14.0, Z=2.0)
    W = 2
    x = _cfgs(sysm, W)
    o = oracle.Oracle(sysm)
    seeds = np.array([0.8, -1.3])
    g = pg.JAGP(sysm, W)
    r = g.positions(x)
    g.eval(r)
    out = g.grad(r, seed_logpsi=torch.tensor(seeds, device="cuda"))
    ref = [o.grad_logpsi(x[w]) for w in range(W)]
    for key, what in (("lam", "lambda"), ("jas", "jastrow"), ("R", "R")):
        want = sum(s * d[key] for s, d in zip(seeds, ref))
        ok, err = _close(out[key].cpu().numpy(), want, 1e-9)
        assert ok, (what, err)
    ok, err = _close(out["r"].cpu().numpy(), np.stack([s * d["r"] for s, d in zip(seeds, ref)]), 1e-9)
    assert ok, ("r", err)
    sE = torch.tensor([0.5, 0.5], dtype=torch.float64, device="cuda")
    out = g.grad(r, seed_eL=sE, want_lambda=False)
    Rw, rr = out["R_walker"].cpu().numpy(), out["r"].cpu().numpy()
    for w in range(W):
        tot = Rw[w].sum(0) + rr[w].sum(0)
        scale = max(1.0, np.abs(Rw[w]).max(), np.abs(rr[w]).max())
        assert np.abs(tot).max() <= 1e-9 * scale, (w, tot)
    g.close()


def test_full_size_c4_logpsi_gradients_sampled(torch_cuda):
    """The adjoint workload at full size (64 He, N = 128, L = 1536, 2048
    walkers, after one sweep as the bench runs it): the per-walker nuclear and
    electron gradients of sum_w s_w log|Psi_w| for two sampled walkers against
    the oracle's analytic gradients, and their local energies."""
    torch = torch_cuda
    import paper_2002_07401_gb300 as pg
    sysm = synth.config4()
    W = 2048
    g = pg.JAGP(sysm, W, seed=0)
    r = g.positions(synth.init_walkers(sysm, W, seed=0))
    g.eval(r)
    eL, _ = g.sweep(r, 1)
    assert g.status() & (pg.WS_NONFINITE | pg.WS_SINGULAR) == 0
    seeds = np.random.default_rng(3).normal(size=W)
    g.eval(r)
    out = g.grad(r, seed_logpsi=torch.tensor(seeds, device="cuda"), want_lambda=False)
    Rw = out["R_walker"].cpu().numpy()
    rr = out["r"].cpu().numpy()
    x_all = r.cpu().numpy()
    o = oracle.Oracle(sysm)
    for w in np.random.default_rng(4).choice(W, size=2, replace=False):
        x = np.ascontiguousarray(x_all[w])
        ref = o.grad_logpsi(x, want_lam=False)
        ok, err = _close(Rw[w], seeds[w] * ref["R"], 1e-9)
        assert ok, ("R", w, err)
        ok, err = _close(rr[w], seeds[w] * ref["r"], 1e-9)
        assert ok, ("r", w, err)
        e_ref = o.local_energy(x)
        assert abs(eL.cpu().numpy()[0, w] - e_ref) <= 1e-10 * max(1.0, abs(e_ref)), (w, e_ref)
    g.close()


@pytest.mark.parametrize("name", ["n121", "C4"])
def test_large_local_energy_derivatives_match_fd(torch_cuda, name):
    """The e_L half of the force at N_up = 121 (the adjoint's per-walker GEMM
    branch) and at the full-size adjoint workload (64 He, N = 128, L = 1536,
    2048 walkers, after one sweep as the bench runs it): for one sampled
    walker, d e_L / d R_a at two nuclei, d e_L / d r_i at three electron
    coordinates and d e_L / d lambda at two entries against the oracle's
    Richardson-extrapolated central differences at h = 1e-4 bohr, tolerance
    1e-6 relative to the largest of them."""
    torch = torch_cuda
    import paper_2002_07401_gb300 as pg
    if name == "C4":
        sysm, W = synth.config4(), 2048
    else:
        sysm, W = synth.small_random(n_atoms=60, n_up=121, n_dn=119, per_atom=6, seed=51, side=14.0, Z=2.0), 2
    g = pg.JAGP(sysm, W, seed=0)
    r = g.positions(synth.init_walkers(sysm, W, seed=0) if name == "C4" else _cfgs(sysm, W))
    g.eval(r)
    if name == "C4":
        g.sweep(r, 1)
        g.eval(r)
    assert g.status() & (pg.WS_NONFINITE | pg.WS_SINGULAR) == 0
    rng = np.random.default_rng(7)
    w = int(rng.integers(W))
    seeds = np.zeros(W)
    seeds[w] = 1.0
    out = g.grad(r, seed_eL=torch.tensor(seeds, device="cuda"))
    x = np.ascontiguousarray(r.cpu().numpy()[w])
    atoms = rng.choice(sysm.n_atoms, size=2, replace=False)
    Rc = [(int(a), q) for a in atoms for q in range(3)]
    rc = [(int(rng.integers(sysm.N)), int(rng.integers(3))) for _ in range(3)]
    lc = [tuple(int(v) for v in rng.integers(sysm.L, size=2)) for _ in range(2)]
    fd = oracle.Oracle(sysm).elocal_fd_select(x, R=Rc, r=rc, lam=lc, h=1e-4)
    Rw, rr, lam = out["R_walker"].cpu().numpy(), out["r"].cpu().numpy(), out["lam"].cpu().numpy()
    got = np.array([Rw[w, a, q] for a, q in Rc] + [rr[w, i, q] for i, q in rc] + [lam[mu, nu] for mu, nu in lc])
    scale = max(1.0, float(np.abs(fd).max()))
    err = np.abs(got - fd) / scale
    print(name, "walker", w, "max rel err", err.max(), "components", np.abs(fd))
    assert err.max() <= 1e-6, (Rc, rc, lc, got, fd)
    g.close()
