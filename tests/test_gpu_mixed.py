"""Mixed-precision path (double-word FP32 orbital tables, BF16 tensor-core
lambda products on six-slice fixed-point operands, FP64 refresh / log-det /
energies, kinetic contraction from exact fixed-point M vectors in double-word
arithmetic) against the FP64 oracle.

Stated tolerances per configuration: |log|Psi| error| <= 1e-6 and
|e_L error| <= 1e-5 Ha.  Sampling: the mixed path's accept decisions are taken
from FP32 ratios, so its trajectories are compared statistically (VMC mean
within the combined error bar), not move by move.
"""
import math

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

LOGPSI_TOL = 1e-6
EL_TOL = 1e-5
# The N_up = 40 random system is an ill-conditioned stress case outside the
# workload configurations; it is held to the same targets.
STRESS_TOL = {}


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


SYSTEMS = {
    "C1": lambda: synth.config1(),
    "C2": lambda: synth.config2(),
    "small-unpaired-slater": lambda: synth.small_random(n_atoms=3, n_up=4, n_dn=2, per_atom=20, seed=31,
                                                        slater_fraction=0.3),
    "mid-n40": lambda: synth.small_random(n_atoms=20, n_up=40, n_dn=37, per_atom=6, seed=33, side=7.0, Z=2.0),
    # the batched workload's systems: smallest, median and largest electron count
    "C3-min": lambda: _c3("min"),
    "C3-median": lambda: _c3("median"),
    "C3-max": lambda: _c3("max"),
}


def _c3(which):
    systems = synth.config3_systems()
    order = np.argsort([s.N for s in systems], kind="stable")
    return systems[int({"min": order[0], "median": order[len(order) // 2], "max": order[-1]}[which])]


def _equilibrated(sysm, W, sweeps=20, seed=5):
    """Configurations drawn from |Psi|^2 by the oracle (the inputs of the per-configuration checks)."""
    x = synth.init_walkers(sysm, W, seed=seed)
    oracle.Oracle(sysm).vmc(x, sweeps, seed=seed + 1, record_eL=False)
    return x


@pytest.mark.parametrize("name", list(SYSTEMS))
def test_mixed_per_configuration_errors(torch_cuda, name):
    import paper_2002_07401_gb300 as pg
    sysm = SYSTEMS[name]()
    W = 24
    x = _equilibrated(sysm, W, sweeps=10 if sysm.N > 40 else 20)
    o = oracle.Oracle(sysm)
    la_ref, sg_ref = o.logpsi_batch(x)
    e_ref = o.local_energy_batch(x)
    g = pg.JAGP(sysm, W, precision=pg.JAGP_PREC_MIXED)
    r = g.positions(x)
    la, sg = g.eval(r)
    e = g.local_energy(r).cpu().numpy()
    la = la.cpu().numpy()
    assert g.status() & (pg.WS_NONFINITE | pg.WS_SINGULAR) == 0
    dl = np.abs(la - la_ref).max()
    de = np.abs(e - e_ref).max()
    print(f"{name}: max |d log|psi|| = {dl:.3e}, max |d e_L| = {de:.3e} Ha")
    assert np.array_equal(sg.cpu().numpy(), sg_ref)
    lt, et = STRESS_TOL.get(name, (LOGPSI_TOL, EL_TOL))
    assert dl <= lt, dl
    assert de <= et, de


def test_mixed_refresh_every_16_moves_keeps_the_tables_consistent(torch_cuda):
    """The batched workload's setting (refresh every 16 moves) on its largest
    system: after sweeps, log|Psi| of the state and e_L agree with the oracle
    at the final positions to the mixed-path targets."""
    import paper_2002_07401_gb300 as pg
    sysm = _c3("max")
    W = 8
    x = _equilibrated(sysm, W, sweeps=4)
    g = pg.JAGP(sysm, W, precision=pg.JAGP_PREC_MIXED, seed=2, refresh_moves=16)
    r = g.positions(x)
    g.eval(r)
    eL, _ = g.sweep(r, 2)
    assert g.status() & (pg.WS_NONFINITE | pg.WS_SINGULAR) == 0
    xf = r.cpu().numpy()
    o = oracle.Oracle(sysm)
    la_ref, _ = o.logpsi_batch(xf)
    e_ref = o.local_energy_batch(xf)
    assert np.max(np.abs(g.info()["logabs"].cpu().numpy() - la_ref)) <= LOGPSI_TOL
    assert np.max(np.abs(eL.cpu().numpy()[-1] - e_ref)) <= EL_TOL
    g.close()


def test_mixed_vmc_mean_matches_oracle(torch_cuda):
    import paper_2002_07401_gb300 as pg
    sysm = synth.config1()
    W, sweeps, equil = 2048, 60, 10
    x0 = synth.init_walkers(sysm, W, seed=2)
    g = pg.JAGP(sysm, W, precision=pg.JAGP_PREC_MIXED, seed=9)
    r = g.positions(x0)
    g.eval(r)
    eL, _ = g.sweep(r, sweeps)
    assert g.status() & (pg.WS_NONFINITE | pg.WS_SINGULAR) == 0
    wm = eL.cpu().numpy()[equil:].mean(0)
    xo = x0.copy()
    eo, _, _ = oracle.Oracle(sysm).vmc(xo, sweeps, seed=9)
    wo = eo[equil:].mean(0)
    err = math.sqrt(wm.var(ddof=1) / W + wo.var(ddof=1) / W)
    assert abs(wm.mean() - wo.mean()) < 4.5 * err, (wm.mean(), wo.mean(), err)


@pytest.mark.parametrize("name", ["C2", "C3-median"])
def test_mixed_vmc_mean_paired_with_the_fp64_chain(torch_cuda, name):
    """VMC mean of the mixed chain at C2 (4096 walkers) and at the batched
    workload's median system, against the FP64 chain driven by the same random
    numbers.  The FP64 chain is the oracle's chain: the same proposals and
    uniforms, positions identical move by move (the trajectory parity tests).
    The mixed chain takes its accept decisions from FP32 ratios, so a walker
    follows the FP64 chain until a decision flips.  Three checks:
    * on the walkers that never left the FP64 trajectory the time-averaged
      e_L differ only by the evaluation error: their mean difference is
      within the per-configuration tolerance (1e-5 Ha);
    * at least 99% of the walkers never leave it over 120 sweeps, so fewer
      than about 3e-6 of the accept decisions differ (the only way the
      sampled distribution could differ);
    * over all walkers the mean difference lies within 4.5 paired error bars
      plus the per-configuration tolerance."""
    import paper_2002_07401_gb300 as pg
    sysm = SYSTEMS[name]()
    W, sweeps, equil = (4096, 120, 20) if name == "C2" else (2048, 120, 20)
    x0 = synth.init_walkers(sysm, W, seed=3)
    means, finals = {}, {}
    for prec in (pg.JAGP_PREC_MIXED, pg.JAGP_PREC_FP64):
        g = pg.JAGP(sysm, W, precision=prec, seed=11)
        r = g.positions(x0)
        g.eval(r)
        eL, _ = g.sweep(r, sweeps)
        assert g.status() & (pg.WS_NONFINITE | pg.WS_SINGULAR) == 0
        means[prec] = eL.cpu().numpy()[equil:].mean(0)
        finals[prec] = r.cpu().numpy()
        g.close()
    d = means[pg.JAGP_PREC_MIXED] - means[pg.JAGP_PREC_FP64]
    se = d.std(ddof=1) / math.sqrt(W)
    on = np.all(np.abs(finals[pg.JAGP_PREC_MIXED] - finals[pg.JAGP_PREC_FP64]) <= 1e-9, axis=(1, 2))
    spread = means[pg.JAGP_PREC_FP64].std(ddof=1) / math.sqrt(W)
    print(f"{name}: mean difference {d.mean():.3e} Ha, paired error {se:.3e} (unpaired {spread:.3e}), "
          f"walkers on the FP64 trajectory {on.mean():.4f}, their mean difference {d[on].mean():.3e}")
    assert on.mean() >= 0.99, on.mean()
    assert abs(d[on].mean()) <= EL_TOL, d[on].mean()
    assert abs(d.mean()) <= 4.5 * se + EL_TOL, (d.mean(), se)


def test_mixed_hydrogen_zero_variance(torch_cuda):
    import paper_2002_07401_gb300 as pg
    sysm = synth.hydrogen_slater()
    W = 512
    g = pg.JAGP(sysm, W, precision=pg.JAGP_PREC_MIXED)
    r = g.positions(synth.init_walkers(sysm, W, seed=4))
    g.eval(r)
    eL, _ = g.sweep(r, 4)
    assert np.max(np.abs(eL.cpu().numpy() + 0.5)) < EL_TOL


def test_fp32_orbital_value_is_rounded_once(torch_cuda):
    """One electron in one Gaussian orbital: log|Psi| = -alpha r^2 exactly, so
    the mixed path's log|Psi| exposes the FP32 orbital value's own error: at
    most half an FP32 ulp from the rounding plus a few 1e-9 from the
    exponential, for alpha r^2 up to 85 (above the FP32 denormal range)."""
    import paper_2002_07401_gb300 as pg
    alpha = 1.3
    sysm = synth.one_electron_gauss(alpha)
    W = 4096
    rng = np.random.default_rng(3)
    rad = np.sqrt(rng.uniform(0.0, 85.0 / alpha, W))
    d = rng.normal(size=(W, 3))
    x = np.ascontiguousarray((d / np.linalg.norm(d, axis=1, keepdims=True) * rad[:, None])[:, None, :])
    g = pg.JAGP(sysm, W, precision=pg.JAGP_PREC_MIXED)
    la, _ = g.eval(g.positions(x))
    exact = -alpha * (x[:, 0, :] ** 2).sum(1)
    err = np.abs(la.cpu().numpy() - exact)
    assert err.max() <= 2.0 ** -24 + 5e-9, err.max()
    g.close()


def test_full_size_c2_mixed_sampled(torch_cuda):
    """C2 at its full walker count (4096) in the mixed path, in the launch shape
    the bench times (autotuned tiles): after two sweeps, four sampled walkers'
    log|Psi| and e_L are recomputed by the oracle at their final positions."""
    import paper_2002_07401_gb300 as pg
    sysm = synth.config2()
    W, sweeps = 4096, 2
    g = pg.JAGP(sysm, W, precision=pg.JAGP_PREC_MIXED, seed=0)
    r = g.positions(synth.init_walkers(sysm, W, seed=0))
    g.autotune(r)
    eL, _ = g.sweep(r, sweeps)
    info = g.info()
    assert g.status() & (pg.WS_NONFINITE | pg.WS_SINGULAR) == 0
    pick = np.random.default_rng(7).choice(W, size=4, replace=False)
    xs = np.ascontiguousarray(r.cpu().numpy()[pick])
    o = oracle.Oracle(sysm)
    la_ref, _ = o.logpsi_batch(xs)
    e_ref = o.local_energy_batch(xs)
    assert np.max(np.abs(info["logabs"].cpu().numpy()[pick] - la_ref)) <= LOGPSI_TOL
    assert np.max(np.abs(eL.cpu().numpy()[-1, pick] - e_ref)) <= EL_TOL
    g.close()
