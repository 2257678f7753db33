"""System and walker generators (inputs only; no wave-function arithmetic).

Readings of the paper that fix these inputs:

* Basis (Sec. "Atomic basis set", Eqs. gaussian/slater): one shell is an atom,
  an angular momentum l in {0,1,2}, a radial type (0 = Gaussian, 1 = Slater) and
  one exponent zeta.  A shell carries 2l+1 real Cartesian components; the
  component order is fixed by the kernels and the oracle (s; x,y,z;
  xy,yz,zx,x^2-y^2,3z^2-r^2).  Functions are ordered atom -> l -> shell ->
  component, exponents descending within one l.
* "k Gaussians per atom" is read as the shell recipe below (counts of s, p and
  d shells); exponents are log-uniform in [0.1, 10].
* lambda (Sec. AGP, Eq. agp_expansion) is the dense L x L pairing matrix: the
  upper triangle is drawn N(0, 0.1^2) (0.1 is the standard deviation),
  mirrored, and 1 is added to the diagonal.  The banded variant keeps
  |i-j| <= w with (2w+1)/L close to 10 %.
* The same basis serves both spins (Sec. AGPn: "the most common choice").
* Walkers start with up electron i near atom i mod N_at and down electron j
  near atom (j + N_at//2) mod N_at, offset uniformly in [-1, 1]^3 bohr.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import Optional

import numpy as np

# (number of s, p, d shells) per atom for "k functions per atom"
SHELL_RECIPES = {
    1: (1, 0, 0),
    6: (3, 1, 0),
    16: (5, 2, 1),
    20: (4, 2, 2),
    24: (5, 3, 2),
}

STREAM_GEN = 2
STREAM_INIT = 0


def _rng(seed: int, stream: int, sub: int = 0) -> np.random.Generator:
    return np.random.Generator(np.random.Philox(np.random.SeedSequence([seed, stream, sub])))


@dataclass
class System:
    name: str
    R: np.ndarray            # (n_atoms, 3) float64, bohr
    Z: np.ndarray            # (n_atoms,) float64
    shell_atom: np.ndarray   # (n_shells,) int32
    shell_l: np.ndarray      # (n_shells,) int32, 0..2
    shell_radial: np.ndarray  # (n_shells,) int32, 0 Gaussian / 1 Slater
    shell_zeta: np.ndarray   # (n_shells,) float64
    lam: np.ndarray          # (L, L) float64, row-major
    n_up: int
    n_dn: int
    unpaired: Optional[np.ndarray] = None  # (n_up - n_dn, L) float64
    b_ea: float = 1.0
    b_para: float = 1.0
    b_anti: float = 1.0
    use_j1: bool = True
    use_j2: bool = True
    j2_spin_independent: bool = False
    delta: float = 0.5       # proposal half-width (bohr)
    seed: int = 0
    meta: dict = field(default_factory=dict)
    # three/four-body Jastrow (Eq. threebody_jastrow), or None: its own shells
    # (keys shell_atom, shell_l, shell_radial, shell_zeta) and the symmetric
    # coupling matrices "para" and "anti" ([LJ][LJ])
    j3: Optional[dict] = None

    @property
    def n_atoms(self) -> int:
        return int(self.R.shape[0])

    @property
    def n_shells(self) -> int:
        return int(self.shell_l.shape[0])

    @property
    def L(self) -> int:
        return int(self.lam.shape[0])

    @property
    def N(self) -> int:
        return self.n_up + self.n_dn

    @property
    def k_unpaired(self) -> int:
        return self.n_up - self.n_dn

    def check(self) -> "System":
        ncomp = {0: 1, 1: 3, 2: 5}
        L = sum(ncomp[int(l)] for l in self.shell_l)
        assert self.lam.shape == (L, L), (self.lam.shape, L)
        assert self.n_up >= self.n_dn >= 0 and self.n_up >= 1
        if self.k_unpaired:
            assert self.unpaired is not None and self.unpaired.shape == (self.k_unpaired, L)
        for a in ("R", "Z", "shell_zeta", "lam"):
            setattr(self, a, np.ascontiguousarray(getattr(self, a), dtype=np.float64))
        for a in ("shell_atom", "shell_l", "shell_radial"):
            setattr(self, a, np.ascontiguousarray(getattr(self, a), dtype=np.int32))
        if self.unpaired is not None:
            self.unpaired = np.ascontiguousarray(self.unpaired, dtype=np.float64)
        if self.j3 is not None:
            j = self.j3
            for a in ("shell_atom", "shell_l", "shell_radial"):
                j[a] = np.ascontiguousarray(j[a], dtype=np.int32)
            for a in ("shell_zeta", "para", "anti"):
                j[a] = np.ascontiguousarray(j[a], dtype=np.float64)
            LJ = _n_funcs(j["shell_l"])
            assert j["para"].shape == (LJ, LJ) and j["anti"].shape == (LJ, LJ)
            assert np.array_equal(j["para"], j["para"].T) and np.array_equal(j["anti"], j["anti"].T)
        return self


# ----------------------------------------------------------------------------
# building blocks
# ----------------------------------------------------------------------------

def place_atoms(rng: np.random.Generator, n_atoms: int, side: float, min_sep: float = 0.0) -> np.ndarray:
    """Uniform positions in [0, side]^3; sequential rejection for min_sep."""
    out = []
    tries = 0
    while len(out) < n_atoms:
        p = rng.random(3) * side
        tries += 1
        if tries > 1_000_000:
            raise RuntimeError("cannot place atoms with this minimum separation")
        if min_sep > 0 and any(np.sqrt(((p - q) ** 2).sum()) < min_sep for q in out):
            continue
        out.append(p)
    return np.array(out, dtype=np.float64)


def gaussian_shells(rng: np.random.Generator, n_atoms: int, per_atom: int,
                    zeta_lo: float = 0.1, zeta_hi: float = 10.0):
    ns, np_, nd = SHELL_RECIPES[per_atom]
    atom, ls, zeta = [], [], []
    for a in range(n_atoms):
        for l, cnt in ((0, ns), (1, np_), (2, nd)):
            z = np.exp(rng.uniform(np.log(zeta_lo), np.log(zeta_hi), size=cnt))
            for zz in sorted(z, reverse=True):
                atom.append(a)
                ls.append(l)
                zeta.append(zz)
    n = len(ls)
    return (np.array(atom, np.int32), np.array(ls, np.int32), np.zeros(n, np.int32),
            np.array(zeta, np.float64))


def random_symmetric_lambda(rng: np.random.Generator, L: int, sd: float = 0.1,
                            band: Optional[int] = None) -> np.ndarray:
    lam = np.zeros((L, L))
    iu = np.triu_indices(L)
    lam[iu] = rng.normal(0.0, sd, size=iu[0].shape[0])
    lam = lam + np.triu(lam, 1).T
    lam[np.diag_indices(L)] += 1.0
    if band is not None:
        i, j = np.indices((L, L))
        lam[np.abs(i - j) > band] = 0.0
    return lam


def _n_funcs(shell_l) -> int:
    return int(sum({0: 1, 1: 3, 2: 5}[int(l)] for l in shell_l))


# ----------------------------------------------------------------------------
# the five workload configurations
# ----------------------------------------------------------------------------

def config1(seed: int = 0) -> System:
    """4 H atoms in a 3 bohr cube, N=4 (2+2), 6 s+p Gaussians/atom (L=24),
    dense random symmetric lambda, spin-independent J2 u=r/(2(1+r)), no J1."""
    g = _rng(seed, STREAM_GEN, 1)
    R = place_atoms(g, 4, 3.0)
    sa, sl, sr, sz = gaussian_shells(g, 4, 6)
    lam = random_symmetric_lambda(g, _n_funcs(sl))
    return System("C1", R, np.ones(4), sa, sl, sr, sz, lam, 2, 2,
                  b_ea=1.0, b_para=1.0, b_anti=1.0, use_j1=False, use_j2=True,
                  j2_spin_independent=True, delta=1.6, seed=seed).check()


def config2(seed: int = 0) -> System:
    """16 He atoms in a 10 bohr cube (min separation 1.5), N=32 (16+16),
    20 s/p/d Gaussians/atom (L=320), dense lambda, J1 + spin-dependent J2."""
    g = _rng(seed, STREAM_GEN, 2)
    R = place_atoms(g, 16, 10.0, 1.5)
    sa, sl, sr, sz = gaussian_shells(g, 16, 20)
    lam = random_symmetric_lambda(g, _n_funcs(sl))
    return System("C2", R, np.full(16, 2.0), sa, sl, sr, sz, lam, 16, 16,
                  delta=1.5, seed=seed).check()


def config3_systems(seed: int = 0, n_systems: int = 64):
    """64 independent neutral systems, N uniform in {8,10,...,128}, N/2 He
    atoms each, 16 Gaussians/atom; cube side scaled to the C2 density."""
    g = _rng(seed, STREAM_GEN, 3)
    Ns = 2 * g.integers(4, 65, size=n_systems)
    out = []
    for s, N in enumerate(Ns):
        gs = _rng(seed, STREAM_GEN, 1000 + s)
        na = int(N) // 2
        side = 10.0 * (na / 16.0) ** (1.0 / 3.0)
        R = place_atoms(gs, na, side, 1.5)
        sa, sl, sr, sz = gaussian_shells(gs, na, 16)
        lam = random_symmetric_lambda(gs, _n_funcs(sl))
        out.append(System(f"C3[{s}]", R, np.full(na, 2.0), sa, sl, sr, sz, lam,
                          int(N) // 2, int(N) // 2, delta=1.5, seed=seed).check())
    return out


def config4(seed: int = 0) -> System:
    """64 He atoms in a 16 bohr cube, N=128, 24 Gaussians/atom (L=1536)."""
    g = _rng(seed, STREAM_GEN, 4)
    R = place_atoms(g, 64, 16.0, 1.5)
    sa, sl, sr, sz = gaussian_shells(g, 64, 24)
    lam = random_symmetric_lambda(g, _n_funcs(sl))
    return System("C4", R, np.full(64, 2.0), sa, sl, sr, sz, lam, 64, 64,
                  delta=1.5, seed=seed).check()


def config5(seed: int = 0) -> System:
    """256 He atoms in a 26 bohr cube, N=512, 16 Gaussians/atom (L=4096),
    banded lambda (|i-j| <= 204, ~10 % fill) stored dense."""
    g = _rng(seed, STREAM_GEN, 5)
    R = place_atoms(g, 256, 26.0, 1.5)
    sa, sl, sr, sz = gaussian_shells(g, 256, 16)
    L = _n_funcs(sl)
    lam = random_symmetric_lambda(g, L, band=204)
    return System("C5", R, np.full(256, 2.0), sa, sl, sr, sz, lam, 256, 256,
                  delta=1.5, seed=seed).check()


CONFIGS = {"C1": config1, "C2": config2, "C4": config4, "C5": config5}


# ----------------------------------------------------------------------------
# systems with closed-form answers (oracle pins) and small random systems
# ----------------------------------------------------------------------------

def one_electron_slater(beta: float, Z: float = 1.0) -> System:
    """One electron, one unpaired Slater 1s orbital exp(-beta r), no Jastrow."""
    return System(f"slater1e(b={beta})", np.zeros((1, 3)), np.array([Z]),
                  np.array([0], np.int32), np.array([0], np.int32), np.array([1], np.int32),
                  np.array([beta]), np.zeros((1, 1)), 1, 0, unpaired=np.ones((1, 1)),
                  use_j1=False, use_j2=False, delta=1.0).check()


def hydrogen_slater() -> System:
    """Exact hydrogen ground state: Slater 1s with zeta = 1."""
    return one_electron_slater(1.0, 1.0)


def one_electron_gauss(alpha: float, Z: float = 1.0) -> System:
    """One electron, one unpaired Gaussian exp(-alpha r^2), no Jastrow."""
    return System(f"gauss1e(a={alpha})", np.zeros((1, 3)), np.array([Z]),
                  np.array([0], np.int32), np.array([0], np.int32), np.array([0], np.int32),
                  np.array([alpha]), np.zeros((1, 1)), 1, 0, unpaired=np.ones((1, 1)),
                  use_j1=False, use_j2=False, delta=1.0).check()


def hydrogenic_gauss_j1(Z: float) -> System:
    """Constant orbital (Gaussian, zeta = 0) times the one-body Jastrow with
    b_ea = 0, whose limit u(r) = r/2 turns exp(J1) into exp(-Z r)."""
    return System(f"hydrogenic-J1(Z={Z})", np.zeros((1, 3)), np.array([Z]),
                  np.array([0], np.int32), np.array([0], np.int32), np.array([0], np.int32),
                  np.array([0.0]), np.zeros((1, 1)), 1, 0, unpaired=np.ones((1, 1)),
                  b_ea=0.0, use_j1=True, use_j2=False, delta=0.8 / Z).check()


def helium_slater(beta: float) -> System:
    """He with psi = exp(-beta (r1 + r2)): N_up = N_dn = 1, L = 1, lambda = [1]."""
    return System(f"He(b={beta})", np.zeros((1, 3)), np.array([2.0]),
                  np.array([0], np.int32), np.array([0], np.int32), np.array([1], np.int32),
                  np.array([beta]), np.ones((1, 1)), 1, 1, use_j1=False, use_j2=False,
                  delta=0.6).check()


def small_random(n_atoms: int = 3, n_up: int = 3, n_dn: int = 2, per_atom: int = 6,
                 seed: int = 7, side: float = 3.0, symmetric: bool = True,
                 slater_fraction: float = 0.0, Z: float = 1.0,
                 spin_independent: bool = False, use_j1: bool = True,
                 use_j2: bool = True) -> System:
    """A small random system for derivative and parity tests."""
    g = _rng(seed, STREAM_GEN, 99)
    R = place_atoms(g, n_atoms, side, 0.8)
    sa, sl, sr, sz = gaussian_shells(g, n_atoms, per_atom)
    if slater_fraction > 0:
        sr = (g.random(len(sl)) < slater_fraction).astype(np.int32)
        sz = np.where(sr == 1, 0.5 + g.random(len(sl)), sz)
    L = _n_funcs(sl)
    if symmetric:
        lam = random_symmetric_lambda(g, L)
    else:
        lam = g.normal(0.0, 0.1, size=(L, L)) + np.eye(L)
    k = n_up - n_dn
    unp = g.normal(0.0, 0.5, size=(k, L)) if k else None
    return System(f"small({n_atoms},{n_up},{n_dn})", R, np.full(n_atoms, Z), sa, sl, sr, sz,
                  lam, n_up, n_dn, unpaired=unp, b_ea=0.8, b_para=1.3, b_anti=0.7,
                  use_j1=use_j1, use_j2=use_j2, j2_spin_independent=spin_independent,
                  delta=0.5, seed=seed).check()


def with_j3(sys: System, seed: int = 0, per_atom=(1, 1), sd: float = 0.05) -> System:
    """Attach a three/four-body Jastrow to sys: per atom per_atom = (s, p)
    Gaussian shells with exponents log-uniform in [0.3, 3], and random symmetric
    coupling matrices with N(0, sd^2) entries for parallel and antiparallel pairs."""
    g = _rng(seed, STREAM_GEN, 7000 + sys.n_atoms)
    atom, ls, zeta = [], [], []
    for a in range(sys.n_atoms):
        for l, cnt in ((0, per_atom[0]), (1, per_atom[1])):
            for z in sorted(np.exp(g.uniform(np.log(0.3), np.log(3.0), size=cnt)), reverse=True):
                atom.append(a)
                ls.append(l)
                zeta.append(z)
    LJ = _n_funcs(ls)

    def sym():
        m = g.normal(0.0, sd, size=(LJ, LJ))
        return np.triu(m) + np.triu(m, 1).T
    sys.j3 = {"shell_atom": np.array(atom, np.int32), "shell_l": np.array(ls, np.int32),
              "shell_radial": np.zeros(len(ls), np.int32), "shell_zeta": np.array(zeta),
              "para": sym(), "anti": sym()}
    return sys.check()


# ----------------------------------------------------------------------------
# walkers
# ----------------------------------------------------------------------------

def init_walkers(sys: System, W: int, seed: int = 0, spread: float = 1.0) -> np.ndarray:
    """(W, N, 3) float64 starting positions: each electron near an atom plus a
    uniform offset in [-spread, spread]^3 (up electrons first)."""
    g = _rng(seed, STREAM_INIT, 0)
    na = sys.n_atoms
    centres = np.empty((sys.N, 3))
    for i in range(sys.n_up):
        centres[i] = sys.R[i % na]
    for j in range(sys.n_dn):
        centres[sys.n_up + j] = sys.R[(j + na // 2) % na]
    off = g.uniform(-spread, spread, size=(W, sys.N, 3))
    return np.ascontiguousarray(centres[None] + off)


def jitter_walkers(x: np.ndarray, seed: int, scale: float) -> np.ndarray:
    g = _rng(seed, STREAM_INIT, 1)
    return np.ascontiguousarray(x + g.uniform(-scale, scale, size=x.shape))
