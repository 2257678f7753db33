"""Lattice-regularised diffusion Monte Carlo on the GPU (jagp_lrdmc_project,
jagp_lrdmc_branch, jagp_lrdmc_energy) against the oracle (Sec. "Lattice
regularized Monte Carlo").

The two sides draw the same Philox4x32-10 numbers, so generation by
generation the hop counts, the reconfiguration's parents and the positions
are compared exactly, the weights to 1e-12 and the local energies to 1e-10
(relative); the hop ratios come from the kinetic vectors M on the GPU and
from determinant recomputation in the oracle, so a decision could in
principle differ where a random number falls within rounding of a
threshold.  Then the zero-variance eigenstate, the projected hydrogen energy,
the estimator and the argument checks.
"""
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
    "C1": (lambda: synth.config1(), 0.2),
    "small-unpaired-slater": (lambda: synth.small_random(n_atoms=3, n_up=4, n_dn=2, per_atom=20, seed=31,
                                                         slater_fraction=0.3), 0.15),
    "small-nonsym": (lambda: synth.small_random(n_atoms=4, n_up=5, n_dn=5, per_atom=16, seed=32, symmetric=False),
                     0.15),
    "helium": (lambda: synth.helium_slater(27.0 / 16.0), 0.1),
}


def _rel(a, b):
    a, b = np.asarray(a, dtype=float), np.asarray(b, dtype=float)
    return float(np.max(np.abs(a - b) / np.maximum(1.0, np.abs(b)))) if a.size else 0.0


@pytest.mark.parametrize("name", list(SYSTEMS))
def test_generations_match_oracle(torch_cuda, name):
    import paper_2002_07401_gb300 as pg
    make, a = SYSTEMS[name]
    sysm = make()
    W, ngen, seed = 16, 3, 7
    x0 = synth.jitter_walkers(synth.init_walkers(sysm, W, seed=4), 5, 0.2)
    g = pg.JAGP(sysm, W, seed=seed)
    r = g.positions(x0)
    out = g.lrdmc(r, ngen, a=a, gamma=0.5, tau=0.03, e_ref=-1.0)
    xo = x0.copy()
    ref = oracle.Oracle(sysm).lrdmc(xo, ngen, seed=seed, a=a, gamma=0.5, tau=0.03, e_ref=-1.0)
    hops = out["hops"].cpu().numpy()
    print(name, "hops per generation", hops.sum(1))
    assert hops.sum() > 0
    assert np.array_equal(hops, ref["hops"])
    assert np.array_equal(out["flags"].cpu().numpy(), ref["flags"])
    assert np.array_equal(out["parent"].cpu().numpy(), ref["parent"])
    assert np.array_equal(r.cpu().numpy(), xo)
    assert _rel(out["weight"].cpu().numpy(), ref["weight"]) <= 1e-12
    assert _rel(out["eL"].cpu().numpy(), ref["eL"]) <= 1e-10
    assert _rel(out["wbar"].cpu().numpy(), ref["wbar"]) <= 1e-12
    assert _rel(out["ebar"].cpu().numpy(), ref["ebar"]) <= 1e-10
    g.close()


def test_full_size_c2_sampled(torch_cuda):
    """C2 (16 He, N = 32, L = 320) at 4096 walkers, the launch shape of the
    benchmark: one projection; two sampled walkers' hop counts, final
    positions, weights and local energies against the oracle run from the
    same start with the same walker indices."""
    import paper_2002_07401_gb300 as pg
    torch = torch_cuda
    sysm = synth.config2()
    W, seed, a, tau = 4096, 3, 0.2, 0.004
    x0 = synth.init_walkers(sysm, W, seed=0)
    g = pg.JAGP(sysm, W, seed=seed)
    r = g.positions(x0)
    work = torch.empty(pg.jagp_lrdmc_workspace_bytes(g.h, W), dtype=torch.uint8, device="cuda")
    w = torch.ones(W, dtype=torch.float64, device="cuda")
    eL = torch.empty(W, dtype=torch.float64, device="cuda")
    hops = torch.empty(W, dtype=torch.int32, device="cuda")
    flags = torch.empty(W, dtype=torch.int32, device="cuda")
    pg.jagp_lrdmc_project(g.h, r, g.state, W, work, w, 0, a, 0.5, tau, -70.0, 1 << 20, 0, eL, hops, flags)
    h = hops.cpu().numpy()
    print("hops: mean", h.mean(), "max", h.max())
    assert h.mean() > 3
    o = oracle.Oracle(sysm)
    for j in np.random.default_rng(1).choice(W, size=2, replace=False):
        xo = np.ascontiguousarray(x0[j:j + 1])
        wo = np.ones(1)
        eo, ho, fo = o.lrdmc_project(xo, wo, seed=seed, gen=0, a=a, gamma=0.5, tau=tau, e_ref=-70.0, walker0=int(j))
        assert ho[0] == h[j] and fo[0] == flags.cpu().numpy()[j], (j, ho, h[j])
        assert np.array_equal(r.cpu().numpy()[j], xo[0])
        assert _rel(w.cpu().numpy()[j], wo[0]) <= 1e-12
        assert _rel(eL.cpu().numpy()[j], eo[0]) <= 1e-10
    g.close()


def test_exact_eigenstate_zero_variance(torch_cuda):
    """psi = exp(-r) for hydrogen: ebar = -1/2 and wbar = exp(-tau (-1/2 - e_ref))
    in every generation although the walkers hop."""
    import paper_2002_07401_gb300 as pg
    sysm = synth.hydrogen_slater()
    W, tau, e_ref = 256, 0.2, -0.3
    g = pg.JAGP(sysm, W, seed=1)
    r = g.positions(np.random.default_rng(0).normal(size=(W, 1, 3)))
    out = g.lrdmc(r, 4, a=0.1, tau=tau, e_ref=e_ref)
    assert out["hops"].cpu().numpy().min() > 0
    assert np.allclose(out["ebar"].cpu().numpy(), -0.5, rtol=0, atol=1e-12)
    assert np.allclose(out["wbar"].cpu().numpy(), math.exp(-tau * (-0.5 - e_ref)), rtol=1e-12, atol=0)
    g.close()


def test_projected_hydrogen_energy(torch_cuda):
    """The nodeless trial function exp(-0.8 r) (VMC energy -0.48 Ha) projected
    with a = 0.1: within four reblocked error bars plus 2e-3 Ha (lattice and
    population bias) of the exact -1/2, and the GPU estimator equals the
    oracle's on the same series."""
    import paper_2002_07401_gb300 as pg
    sysm = synth.one_electron_slater(0.8, 1.0)
    W, ngen, eq = 1024, 300, 50
    g = pg.JAGP(sysm, W, seed=3)
    r = g.positions(np.random.default_rng(0).normal(size=(W, 1, 3)))
    out = g.lrdmc(r, ngen, a=0.1, tau=0.1, e_ref=-0.5)
    wb, eb = out["wbar"][eq:], out["ebar"][eq:]
    E = float(pg.jagp_lrdmc_energy(wb, eb, 20).cpu()[0])
    Eo = oracle.lrdmc_energy(wb.cpu().numpy(), eb.cpu().numpy(), 20)
    assert abs(E - Eo) <= 1e-13 * abs(Eo)
    _, st = oracle.reblock(eb.cpu().numpy()[:, None])
    err = max(st[1], 5e-4)
    print(f"GPU LRDMC E = {E:.5f} +- {err:.5f}")
    assert abs(E + 0.5) <= 4 * err + 2e-3
    g.close()


def test_arguments_and_unsupported_handles(torch_cuda):
    import paper_2002_07401_gb300 as pg
    torch = torch_cuda
    sysm = synth.config1()
    W = 4
    g = pg.JAGP(sysm, W)
    r = g.positions(synth.init_walkers(sysm, W, seed=0))
    work = torch.empty(pg.jagp_lrdmc_workspace_bytes(g.h, W), dtype=torch.uint8, device="cuda")
    w = torch.ones(W, dtype=torch.float64, device="cuda")
    for bad in (dict(a=0.0), dict(a=-0.1), dict(gamma=-1.0), dict(tau=-0.1), dict(max_hops=-1)):
        kw = dict(a=0.2, gamma=0.0, tau=0.1, max_hops=10)
        kw.update(bad)
        with pytest.raises(pg.JagpError, match=r"\(status 1\)"):
            pg.jagp_lrdmc_project(g.h, r, g.state, W, work, w, 0, kw["a"], kw["gamma"], kw["tau"], 0.0,
                                  kw["max_hops"])
    g.close()
    gm = pg.JAGP(sysm, W, precision=pg.JAGP_PREC_MIXED)
    with pytest.raises(pg.JagpError, match=r"FP64 handles.*\(status 6\)"):
        pg.jagp_lrdmc_project(gm.h, r, gm.state, W, work, w, 0, 0.2, 0.0, 0.1, 0.0)
    gm.close()
    # max_hops = 0: every walker stays and gets flag 1; tau = 0 changes nothing
    g = pg.JAGP(sysm, W)
    x = r.clone()
    hops = torch.empty(W, dtype=torch.int32, device="cuda")
    flags = torch.empty(W, dtype=torch.int32, device="cuda")
    pg.jagp_lrdmc_project(g.h, r, g.state, W, work, w, 0, 0.2, 0.0, 0.1, 0.0, 0, 0, None, hops, flags)
    assert np.all(hops.cpu().numpy() == 0) and np.all(flags.cpu().numpy() == 1)
    assert torch.equal(r, x)
    pg.jagp_lrdmc_project(g.h, r, g.state, W, work, w, 0, 0.2, 0.0, 0.0, 0.0, 10, 0, None, hops, flags)
    assert np.all(hops.cpu().numpy() == 0) and np.all(flags.cpu().numpy() == 0) and torch.equal(r, x)
    g.close()
