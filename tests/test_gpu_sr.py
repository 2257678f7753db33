"""GPU parity of stochastic reconfiguration (Sec. "Stochastic
reconfiguration"; Sec. "Derivatives with respect to variational
parameters"): the per-walker log-derivatives O_k = d ln|Psi| / d alpha_k
(every entry of lambda, then b_ea, b_para, b_anti) against the oracle's
analytic ones, and the regularised SR step (matrix-free preconditioned CG on
the GPU) against the oracle's explicit S and LU solve, and at full size
against the defining residual computed on the host."""
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
    "small-sym": lambda: synth.small_random(n_atoms=2, n_up=3, n_dn=3, per_atom=6, seed=81),
    "small-nonsym-slater": lambda: synth.small_random(n_atoms=3, n_up=3, n_dn=2, per_atom=6, seed=82,
                                                     symmetric=False, slater_fraction=0.4),
    "C1": synth.config1,
}


def _rel(a, b):
    a, b = np.asarray(a), np.asarray(b)
    return np.max(np.abs(a - b) / np.maximum(1.0, np.abs(b)))


@pytest.mark.parametrize("name", list(SYSTEMS))
def test_logpsi_derivs_match_oracle(torch_cuda, name):
    """After jagp_eval and after two sweeps (the state the sweep leaves)."""
    import paper_2002_07401_gb300 as pg
    sysm = SYSTEMS[name]()
    W = 6
    x0 = synth.jitter_walkers(synth.init_walkers(sysm, W, seed=3), 4, 0.3)
    g = pg.JAGP(sysm, W, seed=3)
    r = g.positions(x0)
    g.eval(r)
    O = g.logpsi_derivs(r).cpu().numpy()
    assert _rel(O, oracle.Oracle(sysm).logpsi_derivs(x0)) < 1e-10
    g.sweep(r, 2)
    x1 = r.cpu().numpy()
    O = g.logpsi_derivs(r).cpu().numpy()
    assert _rel(O, oracle.Oracle(sysm).logpsi_derivs(x1)) < 1e-10
    g.close()


def _samples(pg, sysm, W, sweeps, seed):
    g = pg.JAGP(sysm, W, seed=seed)
    r = g.positions(synth.init_walkers(sysm, W, seed=seed))
    g.eval(r)
    eL, _ = g.sweep(r, sweeps)
    O = g.logpsi_derivs(r)
    return g, r, O, eL[-1].contiguous()


@pytest.mark.parametrize("eps", [0.1, 1e-3])
def test_sr_step_matches_oracle(torch_cuda, eps):
    """f element by element; dalpha against the oracle's LU solve (within the CG
    tolerance times the condition number of S'), and the defining residual."""
    import paper_2002_07401_gb300 as pg
    sysm = synth.small_random(n_atoms=2, n_up=2, n_dn=2, per_atom=6, seed=83)
    g, r, O, e = _samples(pg, sysm, 512, 12, 83)
    delta = 0.07
    f, da, it, res = pg.jagp_sr_step(O, e, eps=eps, delta=delta, max_iter=2000, tol=1e-13)
    On, en = O.cpu().numpy(), e.cpu().numpy()
    ref = oracle.sr(On, en, eps=eps, delta=delta)
    f, da = f.cpu().numpy(), da.cpu().numpy()
    assert res <= 1e-13 and it < 2000
    assert np.max(np.abs(f - ref["f"])) <= 1e-11 * np.max(np.abs(ref["f"]))
    S = ref["S"]
    Sp = S + eps * np.diag(np.diag(S))
    x = da / delta
    assert np.linalg.norm(Sp @ x - ref["f"]) <= 1e-11 * np.linalg.norm(ref["f"])
    cond = np.linalg.cond(Sp)
    assert np.max(np.abs(da - ref["dalpha"])) <= 1e-12 * cond * np.max(np.abs(ref["dalpha"]))
    g.close()


def test_sr_zero_variance_parameter_stays(torch_cuda):
    """A parameter whose samples do not vary (no same-spin pair: b_para) keeps
    dalpha = 0 and f = 0; the others still solve."""
    import paper_2002_07401_gb300 as pg
    sysm = synth.small_random(n_atoms=2, n_up=1, n_dn=1, per_atom=6, seed=84)
    g, r, O, e = _samples(pg, sysm, 256, 8, 84)
    P = sysm.L * sysm.L + 3
    f, da, it, res = pg.jagp_sr_step(O, e, eps=1e-2, delta=1.0, max_iter=2000, tol=1e-12)
    f, da = f.cpu().numpy(), da.cpu().numpy()
    k = sysm.L * sysm.L + 1
    assert np.all(O.cpu().numpy()[:, k] == 0.0)
    assert f[k] == 0.0 and da[k] == 0.0
    assert np.abs(da).max() > 0 and res <= 1e-12
    g.close()


def test_sr_full_size_c2(torch_cuda):
    """The C2 workload (4096 walkers, L = 320: P = 102403 parameters, 3.4 GB of
    samples): sampled walkers' O rows against the oracle, and the step against
    the defining equations evaluated on the host in FP64 (f = -2 cov(e_L, O),
    (S + eps diag S) x = f through O_c^T (O_c x) / M)."""
    torch = torch_cuda
    import paper_2002_07401_gb300 as pg
    sysm = synth.config2()
    W = 4096
    g, r, O, e = _samples(pg, sysm, W, 2, 0)
    x = r.cpu().numpy()
    o = oracle.Oracle(sysm)
    for w in (0, 1777, 4095):
        assert _rel(O[w].cpu().numpy(), o.logpsi_derivs(x[w:w + 1])[0]) < 1e-10
    eps, delta = 1e-3, 0.05
    f, da, it, res = pg.jagp_sr_step(O, e, eps=eps, delta=delta, max_iter=300, tol=1e-10)
    On, en = O.cpu().numpy(), e.cpu().numpy()
    Ob = On.mean(axis=0)
    Oc = On - Ob
    f_ref = -2.0 * (Oc.T @ (en - en.mean())) / W
    fd = f.cpu().numpy()
    assert np.max(np.abs(fd - f_ref)) <= 1e-10 * np.max(np.abs(f_ref))
    xs = da.cpu().numpy() / delta
    diag = (Oc * Oc).mean(axis=0)
    lhs = Oc.T @ (Oc @ xs) / W + eps * diag * xs
    mask = diag > 0
    assert res <= 1e-10
    assert np.linalg.norm((lhs - f_ref)[mask]) <= 2e-10 * np.linalg.norm(f_ref[mask])
    g.close()
