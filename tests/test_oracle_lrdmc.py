"""Pins of the oracle's lattice-regularised diffusion Monte Carlo (Sec.
"Lattice regularized Monte Carlo"): hop ratios and fixed-node rates against
closed forms, the zero-variance property of an exact eigenstate, the
projected energy of a nodeless trial function against the exact ground state,
the reconfiguration's selection rule and the correcting-factor estimator."""
import math

import numpy as np
import pytest

import oracle
import synth


def _slater_rates(r, zeta, a):
    """Closed form for psi = exp(-zeta |r|): rho_k = exp(-zeta (|r'| - |r|))."""
    rho = []
    for d in range(3):
        for sg in (1.0, -1.0):
            rp = np.array(r, dtype=float)
            rp[d] += sg * a
            rho.append(math.exp(-zeta * (np.linalg.norm(rp) - np.linalg.norm(r))))
    return np.array(rho)


def test_hop_ratios_and_rates_hydrogen_closed_form():
    """One electron in exp(-zeta r): the six hop ratios in the order
    (+x, -x, +y, -y, +z, -z), rates rho / (2 a^2), Gamma their sum, and
    e_L = -zeta^2/2 + (zeta - 1)/r."""
    zeta, a = 0.8, 0.13
    s = synth.one_electron_slater(zeta, 1.0)
    o = oracle.Oracle(s)
    r = np.array([0.7, -0.4, 1.1])
    rho, t, G, eL = o.lrdmc_hops(r[None, :], a, gamma=0.5)
    want = _slater_rates(r, zeta, a)
    assert np.allclose(rho, want, rtol=1e-13, atol=0)
    assert np.allclose(t, want / (2 * a * a), rtol=1e-13, atol=0)
    assert abs(G - want.sum() / (2 * a * a)) <= 1e-12 * G
    rn = np.linalg.norm(r)
    assert abs(eL - (-zeta ** 2 / 2 + (zeta - 1) / rn)) <= 1e-12


def _two_orbital_triplet(z0, z1):
    """Two up electrons, no down electron, two s Gaussians exp(-z r^2) on one
    centre as unpaired orbitals: Psi = phi0(r0) phi1(r1) - phi1(r0) phi0(r1)
    up to constant factors, with a node wherever |r0| = |r1|."""
    return synth.System("triplet2", np.zeros((1, 3)), np.array([2.0]), np.array([0, 0], np.int32),
                        np.array([0, 0], np.int32), np.array([0, 0], np.int32), np.array([z0, z1]),
                        np.zeros((2, 2)), 2, 0, unpaired=np.eye(2), use_j1=False, use_j2=False).check()


def test_fixed_node_rates_across_the_node():
    """A configuration next to the node |r0| = |r1|: the hops of electron 0
    that cross it have rho < 0 (closed form) and rate gamma |rho| / (2 a^2);
    gamma = 0 removes them; the others keep rho / (2 a^2)."""
    z0, z1, a = 0.3, 0.9, 0.2
    s = _two_orbital_triplet(z0, z1)
    o = oracle.Oracle(s)
    x = np.array([[0.95, 0.1, 0.0], [0.0, 1.0, 0.05]])

    def psi(y):
        q0, q1 = (y[0] ** 2).sum(), (y[1] ** 2).sum()
        return math.exp(-z0 * q0 - z1 * q1) - math.exp(-z1 * q0 - z0 * q1)

    want = []
    for k in range(12):
        i, d, sg = k // 6, (k % 6) // 2, k % 2
        y = x.copy()
        y[i, d] += -a if sg else a
        want.append(psi(y) / psi(x))
    want = np.array(want)
    assert (want < 0).any() and (want > 0).any()
    for gamma in (0.0, 0.7):
        rho, t, G, _ = o.lrdmc_hops(x, a, gamma=gamma)
        assert np.allclose(rho, want, rtol=1e-12, atol=1e-14)
        tw = np.where(want > 0, want, -gamma * want) / (2 * a * a)
        assert np.allclose(t, tw, rtol=1e-12, atol=1e-14)
        assert abs(G - tw.sum()) <= 1e-12 * tw.sum()


def test_exact_eigenstate_has_no_fluctuations():
    """Psi = exp(-r) is the hydrogen ground state: e_L = -1/2 everywhere, so
    every walker's weight after a projection of length tau is exp(-tau (-1/2 -
    e_ref)) whatever its path, wbar equals it and ebar = -1/2 in every
    generation (zero variance); the walkers still hop."""
    s = synth.hydrogen_slater()
    o = oracle.Oracle(s)
    x = np.ascontiguousarray(np.random.default_rng(0).normal(size=(64, 1, 3)))
    tau, e_ref = 0.2, -0.3
    out = o.lrdmc(x, 4, seed=1, a=0.1, tau=tau, e_ref=e_ref)
    assert out["hops"].min() > 0
    assert np.allclose(out["ebar"], -0.5, rtol=0, atol=1e-12)
    assert np.allclose(out["wbar"], math.exp(-tau * (-0.5 - e_ref)), rtol=1e-12, atol=0)
    assert abs(oracle.lrdmc_energy(out["wbar"], out["ebar"], 2) + 0.5) <= 1e-12


def test_projection_reaches_the_hydrogen_ground_state():
    """A nodeless trial function exp(-0.8 r) (VMC energy 0.8^2/2 - 0.8 =
    -0.48 Ha) projected with a = 0.1: the LRDMC energy of the hydrogen atom
    lies within four reblocked error bars plus the lattice and population
    bias allowance (2e-3 Ha) of the exact -1/2, well below the VMC energy."""
    s = synth.one_electron_slater(0.8, 1.0)
    o = oracle.Oracle(s)
    W, ngen, eq = 1024, 300, 50
    x = np.ascontiguousarray(np.random.default_rng(0).normal(size=(W, 1, 3)))
    out = o.lrdmc(x, ngen, seed=3, a=0.1, tau=0.1, e_ref=-0.5)
    E = oracle.lrdmc_energy(out["wbar"][eq:], out["ebar"][eq:], 20)
    _, st = oracle.reblock(out["ebar"][eq:, None])
    err = max(st[1], 5e-4)
    print(f"LRDMC E = {E:.5f} +- {err:.5f} (exact -0.5, VMC -0.48)")
    assert abs(E + 0.5) <= 4 * err + 2e-3, (E, err)
    assert E < -0.49


def test_reconfiguration_selection_rule():
    """Equal weights keep every walker; integer weights give exact copy
    counts; random weights give each walker floor or ceil of W w / sum w
    copies (systematic resampling) and W walkers in all; wbar and ebar are the
    plain and weighted means."""
    W = 8
    parent, wb, eb = oracle.lrdmc_branch(np.full(W, 0.37), np.arange(W, dtype=float), seed=5, gen=2)
    assert np.array_equal(parent, np.arange(W))
    assert abs(wb - 0.37) <= 1e-15 and abs(eb - 3.5) <= 1e-14
    w = np.array([2.0, 0.0, 1.0, 1.0, 0.0, 3.0, 1.0, 0.0])
    parent, _, _ = oracle.lrdmc_branch(w, np.zeros(W), seed=5, gen=3)
    assert np.array_equal(np.bincount(parent, minlength=W), w.astype(int))
    rng = np.random.default_rng(9)
    for gen in range(20):
        W = int(rng.integers(5, 200))
        w = rng.exponential(size=W) * (rng.random(W) < 0.8)
        w[0] += 0.1
        e = rng.normal(size=W)
        parent, wb, eb = oracle.lrdmc_branch(w, e, seed=7, gen=gen)
        cnt = np.bincount(parent, minlength=W)
        exp_cnt = W * w / w.sum()
        assert cnt.sum() == W
        assert np.all(cnt >= np.floor(exp_cnt) - 1e-9) and np.all(cnt <= np.ceil(exp_cnt) + 1e-9)
        assert np.all(np.diff(parent) >= 0)
        assert abs(wb - w.mean()) <= 1e-14 * wb and abs(eb - (w * e).sum() / w.sum()) <= 1e-12


def test_correcting_factor_estimator():
    """p = 0 gives the plain mean of ebar; p = 1 weights ebar_n by wbar_{n-1};
    p = 2 by wbar_{n-1} wbar_{n-2} (written out); p >= T is refused (NaN)."""
    wb = np.array([1.5, 0.5, 2.0, 1.0])
    eb = np.array([-1.0, -2.0, -3.0, -4.0])
    assert abs(oracle.lrdmc_energy(wb, eb, 0) - eb.mean()) <= 1e-15
    want1 = (1.5 * -2.0 + 0.5 * -3.0 + 2.0 * -4.0) / (1.5 + 0.5 + 2.0)
    assert abs(oracle.lrdmc_energy(wb, eb, 1) - want1) <= 1e-14
    want2 = (1.5 * 0.5 * -3.0 + 0.5 * 2.0 * -4.0) / (1.5 * 0.5 + 0.5 * 2.0)
    assert abs(oracle.lrdmc_energy(wb, eb, 2) - want2) <= 1e-14
    assert math.isnan(oracle.lrdmc_energy(wb, eb, 4))


def test_max_hops_stops_the_walker():
    """A walker that reaches max_hops stays for the rest of the projection:
    flag bit 1, exactly max_hops hops, and the weight of the remaining time."""
    s = synth.one_electron_slater(0.8, 1.0)
    o = oracle.Oracle(s)
    x = np.ascontiguousarray(np.random.default_rng(1).normal(size=(4, 1, 3)))
    w = np.ones(4)
    eL, hops, flags = o.lrdmc_project(x, w, seed=2, gen=0, a=0.1, tau=1.0, max_hops=3)
    assert np.all(hops == 3) and np.all(flags == 1)
