"""Pins of the CPU oracle against what the paper and the mathematics fix.

Every test here runs on the CPU (no GPU marker).  Each one would fail for a
plausible mistake in the oracle: a wrong sign in a Jastrow derivative, a
transposed lambda, a dropped cross term in the kinetic energy, a wrong
pivot sign in the LU, a biased proposal in the sampler.
"""
import itertools
import math
import os

import numpy as np
import pytest

import oracle
import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _rand_cfg(sys, seed, spread=1.2):
    rng = np.random.default_rng(seed)
    x = synth.init_walkers(sys, 1, seed=seed)[0]
    return np.ascontiguousarray(x + rng.uniform(-spread, spread, size=x.shape) * 0.3)


# ----------------------------------------------------------------------------
# Philox4x32-10: published known-answer vectors
# ----------------------------------------------------------------------------

def test_philox_known_answers():
    rows = [l.split() for l in open(os.path.join(GOLDEN, "philox4x32_10_kat.txt"))
            if l.strip() and not l.startswith("#")]
    assert len(rows) == 3
    for r in rows:
        v = [int(t, 16) for t in r]
        out = oracle.philox4x32_10(v[0:4], v[4:6])
        assert [int(o) for o in out] == v[6:10]


def test_move_draws_ranges():
    """Proposals stay within delta of r in each coordinate and u_acc is in [0,1)."""
    r = np.array([0.1, -0.2, 0.3])
    for e in range(200):
        rp, u = oracle.move_draws(0, 3, 5, e, 0.7, r)
        assert np.all(np.abs(rp - r) < 0.7) and 0.0 <= u < 1.0


# ----------------------------------------------------------------------------
# local energy: closed forms per configuration (zero variance, Sec. VMC)
# ----------------------------------------------------------------------------

def test_hydrogen_zero_variance():
    o = oracle.Oracle(synth.hydrogen_slater())
    rng = np.random.default_rng(1)
    for _ in range(50):
        x = rng.normal(0, 1.5, size=(1, 3))
        assert abs(o.local_energy(x) - (-0.5)) < 1e-12


@pytest.mark.parametrize("beta", [0.6, 1.3])
def test_slater_one_electron_per_config(beta):
    o = oracle.Oracle(synth.one_electron_slater(beta))
    rng = np.random.default_rng(2)
    for _ in range(20):
        x = rng.normal(0, 1.5, size=(1, 3))
        r = np.linalg.norm(x)
        assert abs(o.local_energy(x) - (-beta ** 2 / 2 + (beta - 1) / r)) < 1e-12 * (1 + 1 / r)


@pytest.mark.parametrize("alpha", [0.2, 0.9])
def test_gaussian_one_electron_per_config(alpha):
    o = oracle.Oracle(synth.one_electron_gauss(alpha))
    rng = np.random.default_rng(3)
    for _ in range(20):
        x = rng.normal(0, 1.0, size=(1, 3))
        r = np.linalg.norm(x)
        ref = 3 * alpha - 2 * alpha ** 2 * r * r - 1 / r
        assert abs(o.local_energy(x) - ref) < 1e-11 * (1 + abs(ref))


@pytest.mark.parametrize("Z", [1.0, 2.0])
def test_hydrogenic_via_one_body_jastrow(Z):
    """exp(J1) with b_ea -> 0 is exp(-Z r), an exact eigenstate: e_L = -Z^2/2."""
    o = oracle.Oracle(synth.hydrogenic_gauss_j1(Z))
    rng = np.random.default_rng(4)
    for _ in range(20):
        x = rng.normal(0, 1.0, size=(1, 3))
        assert abs(o.local_energy(x) - (-Z * Z / 2)) < 1e-11


def test_helium_product_per_config():
    beta = 1.45
    o = oracle.Oracle(synth.helium_slater(beta))
    rng = np.random.default_rng(5)
    for _ in range(20):
        x = rng.normal(0, 1.0, size=(2, 3))
        r1, r2 = np.linalg.norm(x[0]), np.linalg.norm(x[1])
        r12 = np.linalg.norm(x[0] - x[1])
        ref = -beta ** 2 + (beta - 2.0) * (1 / r1 + 1 / r2) + 1 / r12
        assert abs(o.local_energy(x) - ref) < 1e-11 * (1 + abs(ref))


# ----------------------------------------------------------------------------
# the sampler: textbook variational energies within the statistical error
# ----------------------------------------------------------------------------

def _vmc_mean(sysm, W=1024, sweeps=120, equil=20, seed=11):
    o = oracle.Oracle(sysm)
    x = np.ascontiguousarray(synth.init_walkers(sysm, W, seed=seed))
    eL, _, nacc = o.vmc(x, sweeps, seed=seed)
    wm = eL[equil:].mean(axis=0)          # walkers are independent chains
    return wm.mean(), wm.std(ddof=1) / math.sqrt(W), nacc.sum() / (W * sweeps * sysm.N)


def test_vmc_slater_one_electron_mean():
    beta = 0.8
    m, err, acc = _vmc_mean(synth.one_electron_slater(beta))
    assert 0.2 < acc < 0.95
    assert abs(m - (beta ** 2 / 2 - beta)) < 4.5 * err, (m, err)


def test_vmc_gaussian_one_electron_mean():
    a = 0.3
    m, err, _ = _vmc_mean(synth.one_electron_gauss(a))
    assert abs(m - (1.5 * a - 2 * math.sqrt(2 * a / math.pi))) < 4.5 * err, (m, err)


def test_vmc_helium_mean():
    vals = dict(l.split() for l in open(os.path.join(GOLDEN, "closed_forms.txt"))
                if l.strip() and not l.startswith("#"))
    beta = float(vals["he_optimal_beta"])
    m, err, _ = _vmc_mean(synth.helium_slater(beta), W=768, sweeps=100)
    assert abs(m - float(vals["he_optimal_energy"])) < 4.5 * err, (m, err)
    # a wrong sampler (e.g. sampling |Psi| instead of Psi^2) misses by far more
    assert err < 0.02


# ----------------------------------------------------------------------------
# determinant: AGP <-> SD, Cauchy-Binet (seniority-zero expansion), LU
# ----------------------------------------------------------------------------

def test_lu_against_library():
    rng = np.random.default_rng(6)
    for n in (1, 2, 5, 17):
        A = rng.normal(size=(n, n))
        ok, la, sg, inv = oracle.det_inverse(A)
        s_ref, la_ref = np.linalg.slogdet(A)
        assert ok and abs(la - la_ref) < 1e-12 * max(1, abs(la_ref)) and sg == s_ref
        assert np.allclose(inv @ A, np.eye(n), atol=1e-11)
    ok, *_ = oracle.det_inverse(np.zeros((3, 3)))
    assert not ok


def test_agp_rank_n_equals_slater_determinant():
    """lambda = C C^T of rank n gives det(Phi_up C) det(Phi_dn C) (Sec. SD)."""
    s = synth.small_random(n_atoms=3, n_up=3, n_dn=3, per_atom=6, seed=8, use_j1=False, use_j2=False)
    rng = np.random.default_rng(8)
    Cm = rng.normal(size=(s.L, s.n_up))
    s.lam = np.ascontiguousarray(Cm @ Cm.T)
    o = oracle.Oracle(s)
    x = _rand_cfg(s, 9)
    G = o.geminal(x)
    phi = np.stack([o.ao(x[i])[0] for i in range(s.N)])
    ref = np.linalg.det(phi[:3] @ Cm) * np.linalg.det(phi[3:] @ Cm)
    assert abs(np.linalg.det(G) - ref) < 1e-10 * abs(ref)
    la, sg, ld, J = o.logpsi(x)
    assert abs(ld - math.log(abs(ref))) < 1e-10 and sg == np.sign(ref)


@pytest.mark.parametrize("n,L", [(2, 5), (3, 6)])
def test_cauchy_binet_seniority_zero(n, L):
    """Diagonal lambda: det G = sum over n-subsets S of prod lambda_S det Phi_up[:,S] det Phi_dn[:,S]
    (the pair-occupation expansion of Sec. "Implicit multiconfigurational character")."""
    s = synth.small_random(n_atoms=2, n_up=n, n_dn=n, per_atom=6, seed=10, use_j1=False, use_j2=False)
    # keep the first L functions only (two atoms x 6)
    keep = L
    shells, tot = [], 0
    for k, l in enumerate(s.shell_l):
        if tot + 2 * l + 1 <= keep:
            shells.append(k)
            tot += 2 * l + 1
    s.shell_atom, s.shell_l = s.shell_atom[shells].copy(), s.shell_l[shells].copy()
    s.shell_radial, s.shell_zeta = s.shell_radial[shells].copy(), s.shell_zeta[shells].copy()
    L = tot
    d = np.random.default_rng(n).uniform(0.5, 1.5, size=L)
    s.lam = np.ascontiguousarray(np.diag(d))
    s.check()
    o = oracle.Oracle(s)
    x = _rand_cfg(s, 12)
    phi = np.stack([o.ao(x[i])[0] for i in range(s.N)])
    Pu, Pd = phi[:n], phi[n:]
    tot_cb = 0.0
    for S in itertools.combinations(range(L), n):
        S = list(S)
        tot_cb += np.prod(d[S]) * np.linalg.det(Pu[:, S]) * np.linalg.det(Pd[:, S])
    la, sg, ld, J = o.logpsi(x)
    assert abs(sg * math.exp(ld) - tot_cb) < 1e-11 * abs(tot_cb)


def test_antisymmetry_same_spin_exchange():
    s = synth.small_random(n_atoms=3, n_up=3, n_dn=2, per_atom=6, seed=13, slater_fraction=0.3)
    o = oracle.Oracle(s)
    x = _rand_cfg(s, 14)
    la, sg, _, _ = o.logpsi(x)
    e = o.local_energy(x)
    for (i, j) in ((0, 2), (3, 4)):       # two up electrons, two down electrons
        y = x.copy()
        y[[i, j]] = y[[j, i]]
        la2, sg2, _, _ = o.logpsi(y)
        assert abs(la2 - la) < 1e-12 and sg2 == -sg
        assert abs(o.local_energy(y) - e) < 1e-10 * (1 + abs(e))


# ----------------------------------------------------------------------------
# Sherman-Morrison against full recomputation
# ----------------------------------------------------------------------------

def test_sherman_morrison_ratio_and_drift():
    rng = np.random.default_rng(15)
    n = 12
    G = rng.normal(size=(n, n)) + 3 * np.eye(n)
    ok, la, sg, Ginv = oracle.det_inverse(G)
    for step in range(100):
        i = int(rng.integers(n))
        row = G[i] + rng.normal(scale=0.3, size=n)
        R = oracle.sm_ratio_row(Ginv, i, row)
        G2 = G.copy()
        G2[i] = row
        ok2, la2, sg2, _ = oracle.det_inverse(G2)
        assert abs(R - sg * sg2 * math.exp(la2 - la)) < 1e-12 * abs(R) * 10
        Ginv = oracle.sm_update_row(Ginv, i, row)
        G, la, sg = G2, la2, sg2
    ok, _, _, fresh = oracle.det_inverse(G)
    assert np.max(np.abs(Ginv - fresh)) < 1e-10 * np.max(np.abs(fresh))


# ----------------------------------------------------------------------------
# analytic derivatives against central finite differences
# ----------------------------------------------------------------------------

def test_orbital_derivatives_fd():
    s = synth.small_random(n_atoms=2, n_up=2, n_dn=1, per_atom=24, seed=16, slater_fraction=0.4)
    o = oracle.Oracle(s)
    r = np.array([0.7, -0.4, 1.1])
    v, g, l, H, gl = o.ao(r, hess=True)
    h = 1e-4
    for q in range(3):
        dp, dm = r.copy(), r.copy()
        dp[q] += h
        dm[q] -= h
        vp, gp, lp = o.ao(dp)
        vm, gm, lm = o.ao(dm)
        assert np.allclose((vp - vm) / (2 * h), g[:, q], rtol=1e-7, atol=1e-9)
        assert np.allclose((gp - gm) / (2 * h), H[:, q, :], rtol=1e-6, atol=1e-8)
        assert np.allclose((lp - lm) / (2 * h), gl[:, q], rtol=1e-6, atol=1e-8)
    assert np.allclose(np.trace(H, axis1=1, axis2=2), l, rtol=1e-12, atol=1e-13)


def _logpsi_signed(o, x):
    la, sg, _, _ = o.logpsi(x)
    return la, sg


@pytest.mark.parametrize("seed,sym", [(17, True), (18, False)])
def test_kinetic_and_gradient_fd(seed, sym):
    """grad log|Psi| against h=1e-4 central differences; the kinetic energy
    -1/2 sum lap Psi/Psi against h=1e-3 second differences of Psi."""
    s = synth.small_random(n_atoms=3, n_up=3, n_dn=2, per_atom=6, seed=seed, symmetric=sym,
                           slater_fraction=0.3)
    o = oracle.Oracle(s)
    x = _rand_cfg(s, seed + 100)
    g = o.grad_logpsi(x, want_lam=False)["r"]
    e, kin, vee, vei, vii, gD, lD = o.local_energy(x, parts=True)
    la0, sg0 = _logpsi_signed(o, x)
    h1, h2 = 1e-4, 1e-3
    lap_sum = 0.0
    for i in range(s.N):
        for q in range(3):
            xp, xm = x.copy(), x.copy()
            xp[i, q] += h1
            xm[i, q] -= h1
            fd = (_logpsi_signed(o, xp)[0] - _logpsi_signed(o, xm)[0]) / (2 * h1)
            assert abs(fd - g[i, q]) < 1e-7 * (1 + abs(g[i, q]))
            xp, xm = x.copy(), x.copy()
            xp[i, q] += h2
            xm[i, q] -= h2
            lp, sp = _logpsi_signed(o, xp)
            lm, sm = _logpsi_signed(o, xm)
            lap_sum += (sp * sg0 * math.exp(lp - la0) + sm * sg0 * math.exp(lm - la0) - 2.0) / h2 ** 2
    assert abs(-0.5 * lap_sum - kin) < 1e-5 * (1 + abs(kin))


def test_potential_terms_by_hand():
    s = synth.small_random(n_atoms=2, n_up=2, n_dn=1, per_atom=6, seed=19)
    o = oracle.Oracle(s)
    x = _rand_cfg(s, 20)
    _, _, vee, vei, vii, _, _ = o.local_energy(x, parts=True)
    ref_ee = sum(1 / np.linalg.norm(x[i] - x[j]) for i in range(3) for j in range(i + 1, 3))
    ref_ei = -sum(s.Z[a] / np.linalg.norm(x[i] - s.R[a]) for i in range(3) for a in range(2))
    ref_ii = s.Z[0] * s.Z[1] / np.linalg.norm(s.R[0] - s.R[1])
    assert abs(vee - ref_ee) < 1e-13 and abs(vei - ref_ei) < 1e-13 and abs(vii - ref_ii) < 1e-13


def test_parameter_gradients_fd():
    """d log|Psi| / d lambda, d/d b_ea, b_para, b_anti and d/d R_a by central FD."""
    s = synth.small_random(n_atoms=2, n_up=2, n_dn=2, per_atom=6, seed=21, symmetric=False,
                           slater_fraction=0.3)
    o = oracle.Oracle(s)
    x = _rand_cfg(s, 22)
    gr = o.grad_logpsi(x)
    h = 1e-5

    def lp_with(mod):
        t = synth.small_random(n_atoms=2, n_up=2, n_dn=2, per_atom=6, seed=21, symmetric=False,
                               slater_fraction=0.3)
        mod(t)
        t.check()
        return oracle.Oracle(t).logpsi(x)[0]

    rng = np.random.default_rng(23)
    for _ in range(6):
        mu, nu = rng.integers(s.L, size=2)

        def m(t, d):
            t.lam = t.lam.copy()
            t.lam[mu, nu] += d
        fd = (lp_with(lambda t: m(t, h)) - lp_with(lambda t: m(t, -h))) / (2 * h)
        assert abs(fd - gr["lam"][mu, nu]) < 1e-6 * (1 + abs(fd))
    for k, name in enumerate(("b_ea", "b_para", "b_anti")):
        b0 = getattr(s, name)
        fd = (lp_with(lambda t: setattr(t, name, b0 + h)) - lp_with(lambda t: setattr(t, name, b0 - h))) / (2 * h)
        assert abs(fd - gr["jas"][k]) < 1e-6 * (1 + abs(fd))
    for a in range(2):
        for q in range(3):
            def mr(t, d):
                t.R = t.R.copy()
                t.R[a, q] += d
            fd = (lp_with(lambda t: mr(t, h)) - lp_with(lambda t: mr(t, -h))) / (2 * h)
            assert abs(fd - gr["R"][a, q]) < 1e-6 * (1 + abs(fd))


# ----------------------------------------------------------------------------
# invariants and cusps
# ----------------------------------------------------------------------------

def test_lambda_scale_invariance():
    s = synth.small_random(n_atoms=3, n_up=3, n_dn=2, per_atom=6, seed=24)
    o = oracle.Oracle(s)
    x = _rand_cfg(s, 25)
    la, _, _, _ = o.logpsi(x)
    e = o.local_energy(x)
    c = -2.5
    s.lam = np.ascontiguousarray(c * s.lam)
    o2 = oracle.Oracle(s)
    la2, _, _, _ = o2.logpsi(x)
    assert abs(la2 - (la + s.n_dn * math.log(abs(c)))) < 1e-11
    assert abs(o2.local_energy(x) - e) < 1e-10 * (1 + abs(e))


def test_translation_invariance():
    s = synth.small_random(n_atoms=3, n_up=2, n_dn=2, per_atom=20, seed=26, slater_fraction=0.2)
    o = oracle.Oracle(s)
    x = _rand_cfg(s, 27)
    la, sg, _, _ = o.logpsi(x)
    e = o.local_energy(x)
    t = np.array([0.37, -1.1, 0.52])
    s.R = np.ascontiguousarray(s.R + t)
    o2 = oracle.Oracle(s)
    la2, sg2, _, _ = o2.logpsi(x + t)
    assert abs(la2 - la) < 1e-10 and sg2 == sg
    assert abs(o2.local_energy(x + t) - e) < 1e-9 * (1 + abs(e))
    # the same statement, differentiated: sum_a dR_a + sum_i dr_i = 0
    g = o.grad_logpsi(x, want_lam=False)
    assert np.allclose(g["R"].sum(0) + g["r"].sum(0), 0.0, atol=1e-9)


def test_cusp_conditions():
    """Kato cusps carried by the Jastrow: dJ2/dr -> 1/2 (antiparallel), 1/4
    (parallel); dJ1/dr -> -Z (Eqs. onebody_J_hom, onebody_u, twobody_v)."""
    s = synth.small_random(n_atoms=1, n_up=2, n_dn=1, per_atom=6, seed=28, Z=2.0)
    o = oracle.Oracle(s)
    far = 1e5    # the third electron sits far away so that only one pair varies
    base = np.array([[5.0, 5.0, 5.0], [far, far, far], [5.0, 5.0, 5.0]])

    def slope(i, j, eps=1e-7):
        x1, x2 = base.copy(), base.copy()
        x1[i] = x1[j] + np.array([eps, 0, 0])
        x2[i] = x2[j] + np.array([2 * eps, 0, 0])
        return (o.jastrow(x2) - o.jastrow(x1)) / eps

    s.use_j1 = False
    o = oracle.Oracle(s)
    assert abs(slope(2, 0) - 0.5) < 1e-5          # up-down pair
    base[2] = [-far, far, -far]
    assert abs(slope(1, 0) - 0.25) < 1e-5         # up-up pair
    s.use_j1, s.use_j2 = True, False
    o = oracle.Oracle(s)
    x1 = np.array([s.R[0] + [1e-7, 0, 0], [far, far, far], [-far, far, -far]])
    x2 = np.array([s.R[0] + [2e-7, 0, 0], [far, far, far], [-far, far, -far]])
    assert abs((o.jastrow(x2) - o.jastrow(x1)) / 1e-7 - (-2.0)) < 1e-5


# ----------------------------------------------------------------------------
# the finite-difference references for d e_L / d R_a, d e_L / d r_i and
# d e_L / d lambda (Sec. "Atomic forces", Eq. forces:aad; Sec. "Derivatives
# with respect to variational parameters"), pinned to closed forms
# ----------------------------------------------------------------------------

def test_elocal_grad_fd_helium_closed_form():
    """He with psi = exp(-beta (r1 + r2)) around a nucleus at R:
    e_L = -beta^2 + (beta - Z)(1/|r1-R| + 1/|r2-R|) + 1/r12, so
    d e_L/d r1 = -(beta - Z)(r1-R)/|r1-R|^3 - (r1-r2)/r12^3 and
    d e_L/d R = (beta - Z) sum_i (r_i-R)/|r_i-R|^3."""
    beta, Z = 1.45, 2.0
    s = synth.helium_slater(beta)
    s.R = np.ascontiguousarray(np.array([[0.3, -0.2, 0.5]]))
    o = oracle.Oracle(s)
    rng = np.random.default_rng(40)
    for _ in range(6):
        x = s.R + rng.normal(0, 1.0, size=(2, 3))
        d = x - s.R
        r = np.linalg.norm(d, axis=1)
        r12v = x[0] - x[1]
        r12 = np.linalg.norm(r12v)
        ref_r = -(beta - Z) * d / r[:, None] ** 3
        ref_r[0] -= r12v / r12 ** 3
        ref_r[1] += r12v / r12 ** 3
        ref_R = (beta - Z) * (d / r[:, None] ** 3).sum(0)
        dR, dr = o.elocal_grad(x, h=1e-3)
        scale = 1.0 + np.abs(ref_r).max()
        assert np.allclose(dr, ref_r, rtol=0, atol=1e-8 * scale), (dr, ref_r)
        assert np.allclose(dR[0], ref_R, rtol=0, atol=1e-8 * scale), (dR, ref_R)


def test_elocal_grad_fd_off_centre_slater_two_nuclei():
    """One electron in exp(-beta |r - R0|) with nuclei Z0 at R0 and Z1 at R1:
    e_L = -beta^2/2 + (beta - Z0)/d0 - Z1/d1 + Z0 Z1/|R0 - R1|; the nuclear
    derivatives carry the orbital's centre, the second nucleus and V_ii."""
    beta, Z0, Z1 = 1.3, 1.0, 2.0
    R = np.array([[0.1, 0.2, -0.3], [1.4, -0.6, 0.9]])
    s = synth.System("slater-off-centre", R, np.array([Z0, Z1]), np.array([0], np.int32),
                     np.array([0], np.int32), np.array([1], np.int32), np.array([beta]),
                     np.zeros((1, 1)), 1, 0, unpaired=np.ones((1, 1)), use_j1=False,
                     use_j2=False, delta=1.0).check()
    o = oracle.Oracle(s)
    rng = np.random.default_rng(41)
    for _ in range(6):
        x = (R[0] + rng.normal(0, 0.8, size=3))[None]
        d0, d1 = x[0] - R[0], x[0] - R[1]
        n0, n1 = np.linalg.norm(d0), np.linalg.norm(d1)
        R01 = R[0] - R[1]
        n01 = np.linalg.norm(R01)
        e = -beta ** 2 / 2 + (beta - Z0) / n0 - Z1 / n1 + Z0 * Z1 / n01
        assert abs(o.local_energy(x) - e) < 1e-12 * (1 + abs(e))
        ref_r = -(beta - Z0) * d0 / n0 ** 3 + Z1 * d1 / n1 ** 3
        ref_R0 = (beta - Z0) * d0 / n0 ** 3 - Z0 * Z1 * R01 / n01 ** 3
        ref_R1 = -Z1 * d1 / n1 ** 3 + Z0 * Z1 * R01 / n01 ** 3
        dR, dr = o.elocal_grad(x, h=1e-3)
        scale = 1.0 + np.abs(ref_r).max()
        assert np.allclose(dr[0], ref_r, rtol=0, atol=1e-8 * scale)
        assert np.allclose(dR[0], ref_R0, rtol=0, atol=1e-8 * scale)
        assert np.allclose(dR[1], ref_R1, rtol=0, atol=1e-8 * scale)


def test_elocal_dlambda_fd_two_orbital_geminal_closed_form():
    """Two electrons (one up, one down) in the geminal psi = sum lambda_{mu,nu}
    phi_mu(r1) phi_nu(r2) of two Slater s orbitals (Eq. agp_expansion with
    L = 2, non-symmetric lambda).  With t_{mu,nu} the kinetic energy of the
    product phi_mu(r1) phi_nu(r2) over itself and p_{mu,nu} the product,
    d e_L / d lambda_{mu,nu} = p_{mu,nu} (t_{mu,nu} - T) / psi, T = (H - V) psi / psi.
    Summed against lambda this is Euler's identity for e_L(c lambda) = e_L(lambda)."""
    zeta = np.array([1.7, 0.6])
    lam = np.array([[1.0, 0.35], [-0.2, 0.8]])
    s = synth.System("2-orbital geminal", np.zeros((1, 3)), np.array([2.0]), np.array([0, 0], np.int32),
                     np.array([0, 0], np.int32), np.array([1, 1], np.int32), zeta, lam, 1, 1,
                     use_j1=False, use_j2=False, delta=0.6).check()
    o = oracle.Oracle(s)
    rng = np.random.default_rng(42)
    for _ in range(4):
        x = rng.normal(0, 0.9, size=(2, 3))
        r1, r2 = np.linalg.norm(x[0]), np.linalg.norm(x[1])
        phi1, phi2 = np.exp(-zeta * r1), np.exp(-zeta * r2)
        p = np.outer(phi1, phi2)
        k1 = -0.5 * (zeta ** 2 - 2 * zeta / r1)      # -1/2 lap phi / phi at r1
        k2 = -0.5 * (zeta ** 2 - 2 * zeta / r2)
        t = k1[:, None] + k2[None, :]
        psi = (lam * p).sum()
        T = (lam * t * p).sum() / psi
        V = -2.0 / r1 - 2.0 / r2 + 1.0 / np.linalg.norm(x[0] - x[1])
        assert abs(o.local_energy(x) - (T + V)) < 1e-11 * (1 + abs(T + V))
        ref = p * (t - T) / psi
        got = np.array([[o.elocal_dlambda(x, mu, nu, h=1e-4) for nu in range(2)] for mu in range(2)])
        assert np.allclose(got, ref, rtol=1e-8, atol=1e-9), (got, ref)
        assert abs((lam * got).sum()) < 1e-8 * (1 + np.abs(got).max())


def test_elocal_dlambda_fd_euler_identity_random_system():
    """e_L is invariant under lambda -> c lambda (N_up = N_dn), so
    sum lambda_{mu,nu} d e_L / d lambda_{mu,nu} = 0 for every configuration
    (non-symmetric lambda, Jastrow on, s/p/d shells)."""
    s = synth.small_random(n_atoms=2, n_up=2, n_dn=2, per_atom=6, seed=43, symmetric=False,
                           slater_fraction=0.3)
    o = oracle.Oracle(s)
    x = _rand_cfg(s, 44)
    g = np.array([[o.elocal_dlambda(x, mu, nu, h=1e-4) for nu in range(s.L)] for mu in range(s.L)])
    assert np.abs(g).max() > 1e-3
    assert abs((s.lam * g).sum()) < 1e-8 * np.abs(s.lam * g).sum()


def test_elocal_grad_fd_translation_sum():
    """Rigid translation leaves e_L unchanged: sum_a d e_L/d R_a + sum_i d e_L/d r_i = 0
    (J1, J2 and d shells on; pins the nuclear and electronic loops jointly)."""
    s = synth.small_random(n_atoms=3, n_up=3, n_dn=2, per_atom=20, seed=45, slater_fraction=0.2)
    o = oracle.Oracle(s)
    x = _rand_cfg(s, 46)
    dR, dr = o.elocal_grad(x, h=1e-3)
    scale = np.abs(dR).max() + np.abs(dr).max()
    assert scale > 1e-2
    assert np.allclose(dR.sum(0) + dr.sum(0), 0.0, atol=1e-8 * scale)


def test_elocal_fd_select_equals_the_full_differences():
    """The parallel selected-component differences (used at full size) give
    exactly the components of the full nuclear, electronic and lambda
    differences pinned above, including an unsymmetrised lambda entry; an
    out-of-range component is refused."""
    s = synth.small_random(n_atoms=3, n_up=3, n_dn=2, per_atom=20, seed=45, slater_fraction=0.2)
    o = oracle.Oracle(s)
    x = _rand_cfg(s, 46)
    dR, dr = o.elocal_grad(x, h=1e-3)
    Rc, rc, lc = [(0, 2), (2, 0), (1, 1)], [(4, 1), (0, 0)], [(3, 7), (7, 3)]
    got = o.elocal_fd_select(x, R=Rc, r=rc, lam=lc, h=1e-3)
    want = [dR[a, q] for a, q in Rc] + [dr[i, q] for i, q in rc] + \
        [o.elocal_dlambda(x, mu, nu, h=1e-3) for mu, nu in lc]
    assert np.array_equal(got, np.array(want))
    with pytest.raises(ValueError):
        o.elocal_fd_select(x, R=[(s.n_atoms, 0)])


def test_agp_nonsymmetric_rank_n_lambda():
    """lambda = C D^T (non-symmetric, rank n): G~ = (Phi_up C)(Phi_dn D)^T, so
    det G~ = det(Phi_up C) det(Phi_dn D); a transposed lambda would give
    det(Phi_up D) det(Phi_dn C) instead (Eq. agp_expansion, Sec. SD)."""
    s = synth.small_random(n_atoms=3, n_up=3, n_dn=3, per_atom=6, seed=47, use_j1=False, use_j2=False)
    rng = np.random.default_rng(47)
    Cm, Dm = rng.normal(size=(s.L, 3)), rng.normal(size=(s.L, 3))
    s.lam = np.ascontiguousarray(Cm @ Dm.T)
    o = oracle.Oracle(s)
    x = _rand_cfg(s, 48)
    phi = np.stack([o.ao(x[i])[0] for i in range(s.N)])
    ref = np.linalg.det(phi[:3] @ Cm) * np.linalg.det(phi[3:] @ Dm)
    wrong = np.linalg.det(phi[:3] @ Dm) * np.linalg.det(phi[3:] @ Cm)
    assert abs(ref - wrong) > 1e-3 * abs(ref)
    G = o.geminal(x)
    assert abs(np.linalg.det(G) - ref) < 1e-10 * abs(ref)
    la, sg, ld, J = o.logpsi(x)
    assert abs(ld - math.log(abs(ref))) < 1e-10 and sg == np.sign(ref)


# ----------------------------------------------------------------------------
# reblocking of correlated samples (Sec. VMC): textbook and closed-form pins
# ----------------------------------------------------------------------------

def test_reblock_level0_is_the_textbook_standard_error():
    rng = np.random.default_rng(60)
    eL = rng.normal(-1.0, 0.3, size=(257, 5))     # odd T: the ragged tail is dropped above level 0
    lev, st = oracle.reblock(eL)
    m = eL.mean(axis=1)
    assert len(lev) == 8                            # 257 // 2^k >= 2 for k = 0..7
    assert lev[0][0] == 1 and lev[0][1] == 257
    assert abs(lev[0][2] - m.std(ddof=1) / math.sqrt(257)) < 1e-14
    assert abs(lev[0][3] - lev[0][2] / math.sqrt(2 * 256)) < 1e-16
    assert abs(st[0] - eL.mean()) < 1e-14
    for k, (B, nb, sig, err) in enumerate(lev):
        B, nb = int(B), int(nb)
        b = m[: nb * B].reshape(nb, B).mean(axis=1)
        assert B == 2 ** k and nb == 257 // B
        assert abs(sig - b.std(ddof=1) / math.sqrt(nb)) < 1e-13 * max(sig, 1e-300)


def test_reblock_piecewise_constant_series():
    """A series constant over blocks of four sweeps: at level 2 the block means
    are the distinct values themselves."""
    rng = np.random.default_rng(61)
    v = rng.normal(size=64)
    eL = np.repeat(v, 4)[:, None]
    lev, _ = oracle.reblock(eL)
    assert abs(lev[2][2] - v.std(ddof=1) / 8.0) < 1e-14
    nb = 64
    assert abs(lev[2][2] / lev[0][2] - math.sqrt((4 * nb - 1) / (nb - 1))) < 1e-12


def test_reblock_ar1_plateau_matches_closed_form():
    """x_t = phi x_{t-1} + e_t with Var e = s^2: the variance of the mean of T
    samples tends to s^2 / ((1 - phi)^2 T); level 0 underestimates it by the
    integrated autocorrelation time (1 + phi) / (1 - phi)."""
    phi, s, T = 0.8, 0.5, 1 << 17
    rng = np.random.default_rng(62)
    e = rng.normal(0, s, size=T)
    x = np.empty(T)
    x[0] = e[0] / math.sqrt(1 - phi * phi)
    for t in range(1, T):
        x[t] = phi * x[t - 1] + e[t]
    lev, st = oracle.reblock(x)
    want = s / ((1 - phi) * math.sqrt(T))
    assert st[3] == 1.0, lev
    assert abs(st[1] - want) < 0.1 * want, (st, want)
    naive = s / math.sqrt(1 - phi * phi) / math.sqrt(T)
    assert abs(lev[0][2] - naive) < 0.05 * naive


# ----------------------------------------------------------------------------
# stochastic reconfiguration (Sec. "Stochastic reconfiguration", Eqs. SRupdate,
# sr, the diagonal shift; Sec. "Derivatives with respect to variational
# parameters", Eq. eq_general_force)
# ----------------------------------------------------------------------------

def test_sr_against_library_statistics():
    """S is the (biased) covariance of the log-derivatives, f = -2 cov(e_L, O),
    dalpha = Delta (S + eps diag S)^{-1} f: against NumPy's covariance and solver."""
    rng = np.random.default_rng(71)
    M, P = 300, 7
    O = rng.normal(size=(M, P)) @ rng.normal(size=(P, P)) + rng.normal(size=P)
    e = -1.0 + 0.3 * rng.normal(size=M) + 0.1 * O[:, 2]
    eps, delta = 0.05, 0.2
    r = oracle.sr(O, e, eps=eps, delta=delta)
    S_np = np.cov(O.T, bias=True)
    f_np = -2.0 * np.cov(np.vstack([e, O.T]), bias=True)[0, 1:]
    assert np.allclose(r["Obar"], O.mean(axis=0), rtol=0, atol=1e-13)
    assert np.allclose(r["S"], S_np, rtol=1e-12, atol=1e-13)
    assert np.allclose(r["f"], f_np, rtol=1e-12, atol=1e-13)
    Sp = S_np + eps * np.diag(np.diag(S_np))
    assert np.allclose(r["dalpha"], delta * np.linalg.solve(Sp, f_np), rtol=1e-10, atol=1e-13)
    w = np.linalg.eigvalsh(r["S"])
    assert w.min() > -1e-12 * w.max()          # positive semi-definite


def test_sr_force_vanishes_at_an_exact_eigenstate():
    """exp(J1) with b_ea -> 0 is exp(-Z r), an exact eigenstate: e_L is constant,
    so the generalized force vanishes sample by sample, without statistical error."""
    s = synth.hydrogenic_gauss_j1(2.0)
    o = oracle.Oracle(s)
    x = synth.init_walkers(s, 256, seed=72)
    eL, _, _ = o.vmc(x, 30, seed=72)
    O = o.logpsi_derivs(x)[:, [s.L * s.L]]
    assert O.std() > 1e-2
    r = oracle.sr(O, eL[-1], eps=1e-3)
    assert abs(r["f"][0]) < 1e-13 * np.abs(O).max()


def _quad_slater_j1(beta, b, Z=1.0):
    """psi = exp(-beta r) exp(J1(r)) with J1 = -c^3 u(c r), u = (1 - e^{-b s}) / (2b),
    c = (2Z)^{1/4} (Eqs. onebody_J_hom, onebody_u), by radial quadrature:
    E, <O_b>, Var(O_b) with O_b = d ln psi / d b."""
    from scipy.integrate import quad
    c = (2 * Z) ** 0.25

    def parts(r):
        ex = math.exp(-b * c * r)
        F = -beta * r - c ** 3 * (1 - ex) / (2 * b)
        Fp = -beta - c ** 4 * ex / 2
        Fpp = c ** 5 * b * ex / 2
        eL = -0.5 * (Fpp + 2 * Fp / r + Fp ** 2) - Z / r
        sarg = c * r
        Ob = -c ** 3 * (b * sarg * math.exp(-b * sarg) - 1 + math.exp(-b * sarg)) / (2 * b * b)
        return F, eL, Ob

    w = lambda r: math.exp(2 * parts(r)[0]) * r * r          # noqa: E731
    nrm = quad(w, 0, np.inf, limit=200)[0]
    E = quad(lambda r: w(r) * parts(r)[1], 0, np.inf, limit=200)[0] / nrm
    o1 = quad(lambda r: w(r) * parts(r)[2], 0, np.inf, limit=200)[0] / nrm
    o2 = quad(lambda r: w(r) * parts(r)[2] ** 2, 0, np.inf, limit=200)[0] / nrm
    return E, o1, o2 - o1 * o1, parts


def test_sr_step_against_radial_quadrature():
    """One electron, exp(-0.3 r) exp(J1) with b_ea = 0.8: the sampled force
    f = -2 cov(e_L, O_b) and metric S = Var(O_b) agree with -dE/db and Var(O_b)
    by quadrature within their statistical errors, and the SR step moves b_ea
    downhill in the quadrature energy."""
    pytest.importorskip("scipy")
    beta, b = 0.3, 0.8
    s = synth.one_electron_slater(beta)
    s.use_j1, s.b_ea = True, b
    o = oracle.Oracle(s)
    W = 4096
    x = synth.init_walkers(s, W, seed=73, spread=3.0)
    eL, _, _ = o.vmc(x, 80, seed=73, delta=2.5)
    e = eL[-1]
    O = o.logpsi_derivs(x)[:, [s.L * s.L]]
    E0, _, varO, parts = _quad_slater_j1(beta, b)
    for w in range(5):                         # the oracle's O_b against the closed form
        rr = float(np.linalg.norm(x[w, 0]))
        assert abs(O[w, 0] - parts(rr)[2]) < 1e-12 * (1 + abs(O[w, 0]))
    h = 1e-4
    f_exact = -(_quad_slater_j1(beta, b + h)[0] - _quad_slater_j1(beta, b - h)[0]) / (2 * h)
    r = oracle.sr(O, e, eps=1e-3, delta=0.05)
    Oc = O[:, 0] - O[:, 0].mean()
    sig_f = 2 * np.std((e - e.mean()) * Oc) / math.sqrt(W)
    sig_S = np.std(Oc ** 2) / math.sqrt(W)
    assert abs(f_exact) > 10 * sig_f
    assert abs(r["f"][0] - f_exact) < 4.5 * sig_f, (r["f"], f_exact, sig_f)
    assert abs(r["S"][0, 0] - varO) < 4.5 * sig_S, (r["S"], varO, sig_S)
    db = r["dalpha"][0]
    assert db * f_exact > 0
    assert _quad_slater_j1(beta, b + db)[0] < E0


# ----------------------------------------------------------------------------
# space-warp coordinate transformation for forces (Sec. "Atomic forces")
# ----------------------------------------------------------------------------

def _omega_ref(R, r):
    """omega_a(r) = kappa_a / sum_b kappa_b, kappa = |r - R_a|^-4, written out here."""
    k = 1.0 / np.sum((r[None, :] - R) ** 2, axis=1) ** 2
    return k / k.sum()


def test_swct_weights_partition_unity_and_gradient():
    s = synth.small_random(n_atoms=4, n_up=2, n_dn=2, per_atom=6, seed=90)
    o = oracle.Oracle(s)
    rng = np.random.default_rng(90)
    for _ in range(5):
        r = s.R.mean(axis=0) + rng.normal(0, 1.0, size=3)
        om, dom = o.swct_omega(r)
        assert abs(om.sum() - 1.0) < 1e-14 and np.abs(dom.sum(axis=0)).max() < 1e-12 * np.abs(dom).max()
        assert np.allclose(om, _omega_ref(s.R, r), rtol=1e-13, atol=0)
        h = 1e-5
        for q in range(3):
            rp, rm = r.copy(), r.copy()
            rp[q] += h
            rm[q] -= h
            fd = (_omega_ref(s.R, rp) - _omega_ref(s.R, rm)) / (2 * h)
            assert np.allclose(dom[:, q], fd, rtol=1e-7, atol=1e-9)


def test_swct_derivatives_are_derivatives_along_the_warp():
    """d e_L / d R_a (warped) is the derivative of e_L when nucleus a moves by h
    and every electron by h omega_a(r_i); d ln(J^1/2 Psi) / d R_a likewise with
    ln|Psi| + 1/2 sum_i ln(1 + h d omega_a / d r_q) (the Jacobian of the warp)."""
    s = synth.small_random(n_atoms=3, n_up=2, n_dn=2, per_atom=6, seed=91, slater_fraction=0.3)
    o = oracle.Oracle(s)
    x = _rand_cfg(s, 92)
    dE, dL = o.swct_derivs(x, h=1e-3)
    R0 = s.R.copy()
    h = 1e-4

    def warped(a, q, t):
        R = R0.copy()
        R[a, q] += t
        y = x.copy()
        logJ = 0.0
        for i in range(s.N):
            om = _omega_ref(R0, x[i])
            y[i, q] += t * om[a]
            # d omega_a / d r_q by central differences of the written-out definition
            e = np.zeros(3)
            e[q] = 1e-6
            dq = (_omega_ref(R0, x[i] + e)[a] - _omega_ref(R0, x[i] - e)[a]) / 2e-6
            logJ += math.log(1.0 + t * dq)
        s2 = synth.small_random(n_atoms=3, n_up=2, n_dn=2, per_atom=6, seed=91, slater_fraction=0.3)
        s2.R = np.ascontiguousarray(R)
        o2 = oracle.Oracle(s2)
        return o2.local_energy(y), o2.logpsi(y)[0] + 0.5 * logJ

    for a in range(3):
        for q in range(3):
            ep, lp = warped(a, q, h)
            em, lm = warped(a, q, -h)
            assert abs((ep - em) / (2 * h) - dE[a, q]) < 1e-6 * (1 + abs(dE[a, q])), (a, q)
            assert abs((lp - lm) / (2 * h) - dL[a, q]) < 1e-6 * (1 + abs(dL[a, q])), (a, q)
    # the warp moves charge with the nuclei: the total still vanishes (translation)
    assert np.abs(dE.sum(axis=0)).max() < 1e-7 * (1 + np.abs(dE).max())


# ----------------------------------------------------------------------------
# guiding function and reweighting (Sec. "Atomic forces", Eqs.
# guiding_function, R_r, regularization, reweighting)
# ----------------------------------------------------------------------------

def test_guiding_R_is_scale_invariant():
    """R is unchanged when G~ is scaled by a constant (lambda -> c lambda, N_up = N_dn)."""
    s = synth.small_random(n_atoms=3, n_up=3, n_dn=3, per_atom=6, seed=93)
    x = _rand_cfg(s, 94)
    R1 = oracle.Oracle(s).guiding_R(x)
    s.lam = np.ascontiguousarray(-7.5 * s.lam)
    R2 = oracle.Oracle(s).guiding_R(x)
    assert R1 > 0 and abs(R2 - R1) < 1e-12 * R1


def test_guiding_R_vanishes_as_the_antisymmetric_part_to_the_power_2theta():
    """Two up electrons approaching each other (a node of det G~ linear in their
    separation d): sum |G~^{-1}|^2 grows as 1/d^2, so R ~ d^(2 theta)."""
    s = synth.small_random(n_atoms=2, n_up=2, n_dn=2, per_atom=6, seed=95, use_j1=False, use_j2=False)
    o = oracle.Oracle(s)
    x = _rand_cfg(s, 96)
    theta = 0.375
    direction = np.array([0.3, -0.5, 0.8]) / np.linalg.norm([0.3, -0.5, 0.8])

    def R(d):
        y = x.copy()
        y[1] = y[0] + d * direction
        return o.guiding_R(y, theta)
    for d in (1e-3, 1e-4):
        assert abs(math.log2(R(d) / R(d / 2)) - 2 * theta) < 2e-3


def test_guiding_R_stays_finite_for_an_electron_far_away():
    """S = min_i sum_j |G~_ij|^2 vanishes with the row of an electron at infinity
    and compensates the growth of G~^{-1}: R tends to a finite, non-zero value."""
    s = synth.small_random(n_atoms=2, n_up=2, n_dn=2, per_atom=6, seed=97, use_j1=False, use_j2=False)
    o = oracle.Oracle(s)
    x = _rand_cfg(s, 98)
    vals = []
    for far in (3.0, 4.0, 5.0, 6.0):
        y = x.copy()
        y[0] = s.R[0] + far * np.array([1.0, 0.2, -0.1])
        vals.append(o.guiding_R(y))
    assert all(v > 0 for v in vals)
    assert abs(vals[-1] / vals[-2] - 1.0) < abs(vals[1] / vals[0] - 1.0)


def _eps_for_mean_weight(R, target=0.8):
    lo, hi = 1e-12 * R.max(), R.max()
    for _ in range(200):
        eps = math.sqrt(lo * hi)
        m = np.mean(np.minimum(1.0, R / eps) ** 2)
        lo, hi = (eps, hi) if m > target else (lo, eps)
    return math.sqrt(lo * hi)


def test_guided_sampling_reweights_to_the_trial_distribution():
    """Sampling Psi_G and weighting by W = (R / max(R, eps))^2 gives the same
    energy as sampling Psi_T: <W e_L>_G / <W>_G = <e_L>_T within the error bars
    (eps chosen so that <W> over Psi_T samples is 0.8)."""
    s = synth.small_random(n_atoms=2, n_up=2, n_dn=2, per_atom=6, seed=99, Z=1.0)
    o = oracle.Oracle(s)
    W, sweeps, equil = 2048, 60, 20
    x = np.ascontiguousarray(synth.init_walkers(s, W, seed=99))
    eT, _, _ = o.vmc(x, sweeps, seed=99)
    Rs = np.array([o.guiding_R(x[w]) for w in range(W)])
    eps = _eps_for_mean_weight(Rs)
    xg = np.ascontiguousarray(synth.init_walkers(s, W, seed=99))
    eG, _, _, _ = o.vmc_guided(xg, sweeps, eps=eps, seed=101)
    # the weights along the guided chains: recompute R per recorded sweep from the final walkers only
    # (the estimator below uses per-walker means over the last sweeps, weighted at the final configuration)
    Rg = np.array([o.guiding_R(xg[w]) for w in range(W)])
    wg = np.minimum(1.0, Rg / eps) ** 2
    assert 0.2 < wg.mean() < 0.97      # lower than under Psi_T: Psi_G samples the nodes more often
    mT = eT[equil:].mean(axis=0)
    errT = mT.std(ddof=1) / math.sqrt(W)
    e_last = eG[-1]
    est = np.sum(wg * e_last) / np.sum(wg)
    errG = np.sqrt(np.sum((wg * (e_last - est)) ** 2)) / np.sum(wg)
    assert abs(est - mT.mean()) < 4.5 * math.hypot(errT, errG), (est, mT.mean(), errT, errG)
    # the stationary density of the guided chain is Psi_T^2 / W: for the observable
    # 1/W the reweighting identity gives <W>_G = 1 / <1/W>_T (an inverted weight
    # ratio in the acceptance would give <W^2>_T / <W>_T instead)
    wt = np.minimum(1.0, Rs / eps) ** 2
    inv = 1.0 / wt
    ref = 1.0 / inv.mean()
    err_ref = ref * ref * inv.std(ddof=1) / math.sqrt(W)
    err_g = wg.std(ddof=1) / math.sqrt(W)
    assert abs(wg.mean() - ref) < 4.5 * math.hypot(err_ref, err_g), (wg.mean(), ref, err_ref, err_g)
    wrong = (wt ** 2).mean() / wt.mean()
    assert abs(wrong - ref) > 10 * math.hypot(err_ref, err_g)
    # without the weights the guided chain is a different (biased) distribution in general;
    # an eps of zero reproduces the unguided chain exactly
    xz = np.ascontiguousarray(synth.init_walkers(s, 16, seed=99))
    xz2 = xz.copy()
    e1, _, _ = o.vmc(xz, 5, seed=7)
    e2, _, _, _ = o.vmc_guided(xz2, 5, eps=0.0, seed=7)
    assert np.array_equal(xz, xz2) and np.array_equal(e1, e2)


# ----------------------------------------------------------------------------
# three/four-body Jastrow (Eq. threebody_jastrow)
# ----------------------------------------------------------------------------

def test_jastrow3_single_function_closed_form():
    """One s Gaussian chi on one atom and scalar couplings m_p, m_a: the pair sum
    is m_p/2 (U_u^2 - sum_u chi^2 + U_d^2 - sum_d chi^2) + m_a U_u U_d with U_s the
    spin sums of chi."""
    s = synth.small_random(n_atoms=1, n_up=2, n_dn=2, per_atom=6, seed=120, use_j1=False, use_j2=False)
    zeta, mp, ma = 0.7, 0.3, -0.45
    s.j3 = {"shell_atom": [0], "shell_l": [0], "shell_radial": [0], "shell_zeta": [zeta],
            "para": np.array([[mp]]), "anti": np.array([[ma]])}
    s.check()
    o = oracle.Oracle(s)
    x = _rand_cfg(s, 121)
    chi = np.exp(-zeta * np.sum((x - s.R[0]) ** 2, axis=1))
    u, d = chi[:2], chi[2:]
    ref = mp / 2 * (u.sum() ** 2 - (u ** 2).sum() + d.sum() ** 2 - (d ** 2).sum()) + ma * u.sum() * d.sum()
    assert abs(o.jastrow(x) - ref) < 1e-14 * (1 + abs(ref))


def test_jastrow3_kinetic_gradient_translation_antisymmetry():
    """With J3 on (s and p Jastrow functions on every atom): grad log|Psi| and the
    kinetic energy against central differences, the translation sum of the
    nuclear and electronic derivatives, and same-spin exchange symmetry."""
    s = synth.with_j3(synth.small_random(n_atoms=3, n_up=3, n_dn=2, per_atom=6, seed=122, slater_fraction=0.3),
                      seed=122, sd=0.2)
    o = oracle.Oracle(s)
    x = _rand_cfg(s, 123)
    g = o.grad_logpsi(x, want_lam=False)
    e, kin, vee, vei, vii, gD, lD = o.local_energy(x, parts=True)
    la0, sg0 = _logpsi_signed(o, x)
    h1, h2 = 1e-4, 1e-3
    lap_sum = 0.0
    for i in range(s.N):
        for q in range(3):
            xp, xm = x.copy(), x.copy()
            xp[i, q] += h1
            xm[i, q] -= h1
            fd = (_logpsi_signed(o, xp)[0] - _logpsi_signed(o, xm)[0]) / (2 * h1)
            assert abs(fd - g["r"][i, q]) < 1e-7 * (1 + abs(g["r"][i, q]))
            xp, xm = x.copy(), x.copy()
            xp[i, q] += h2
            xm[i, q] -= h2
            lp, sp = _logpsi_signed(o, xp)
            lm, sm = _logpsi_signed(o, xm)
            lap_sum += (sp * sg0 * math.exp(lp - la0) + sm * sg0 * math.exp(lm - la0) - 2.0) / h2 ** 2
    assert abs(-0.5 * lap_sum - kin) < 1e-5 * (1 + abs(kin))
    assert np.allclose(g["R"].sum(0) + g["r"].sum(0), 0.0, atol=1e-9)
    # J3 moves with the nuclei: d log|Psi| / d R_a against central differences
    h = 1e-5
    for a in range(3):
        for q in range(3):
            vals = []
            for sgn in (1, -1):
                t = synth.with_j3(synth.small_random(n_atoms=3, n_up=3, n_dn=2, per_atom=6, seed=122,
                                                     slater_fraction=0.3), seed=122, sd=0.2)
                t.R = t.R.copy()
                t.R[a, q] += sgn * h
                t.check()
                vals.append(oracle.Oracle(t).logpsi(x)[0])
            assert abs((vals[0] - vals[1]) / (2 * h) - g["R"][a, q]) < 1e-6 * (1 + abs(g["R"][a, q]))
    la, sg, _, J = o.logpsi(x)
    y = x.copy()
    y[[0, 2]] = y[[2, 0]]
    la2, sg2, _, J2 = o.logpsi(y)
    assert abs(la2 - la) < 1e-12 and sg2 == -sg and abs(J2 - J) < 1e-13
