"""ctypes front end of the plain FP64 CPU oracle (``jagp_oracle.c``).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the
bench's CPU-baseline leg call it; the CUDA library never does.  It shares no
code with the CUDA path.  ``build()`` compiles the C file with gcc into
``oracle/_build`` (OpenMP when available, no FP contraction).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "jagp_oracle.c")
_OUT = os.path.join(_HERE, "_build")
_LIB = os.path.join(_OUT, "libjagp_oracle.so")
_lock = threading.Lock()
_lib = None

f64p = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")


class _OrcSystem(C.Structure):
    _fields_ = [
        ("n_atoms", C.c_int), ("R", C.c_void_p), ("Z", C.c_void_p),
        ("n_shells", C.c_int), ("shell_atom", C.c_void_p), ("shell_l", C.c_void_p),
        ("shell_radial", C.c_void_p), ("shell_zeta", C.c_void_p),
        ("L", C.c_int), ("lam", C.c_void_p), ("n_up", C.c_int), ("n_dn", C.c_int),
        ("unpaired", C.c_void_p), ("b_ea", C.c_double), ("b_para", C.c_double),
        ("b_anti", C.c_double), ("use_j1", C.c_int), ("use_j2", C.c_int),
        ("j2_spin_independent", C.c_int),
        ("n_jshells", C.c_int), ("jshell_atom", C.c_void_p), ("jshell_l", C.c_void_p),
        ("jshell_radial", C.c_void_p), ("jshell_zeta", C.c_void_p), ("LJ", C.c_int),
        ("j3_para", C.c_void_p), ("j3_anti", C.c_void_p), ("use_j3", C.c_int),
    ]


def build(force: bool = False) -> str:
    """Compile the oracle (idempotent); returns the library path."""
    with _lock:
        if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
            return _LIB
        os.makedirs(_OUT, exist_ok=True)
        base = ["gcc", "-O2", "-fPIC", "-shared", "-ffp-contract=off", "-std=c11", _SRC, "-o", _LIB + ".tmp", "-lm"]
        try:
            subprocess.run(base[:1] + ["-fopenmp"] + base[1:], check=True, capture_output=True)
        except subprocess.CalledProcessError:
            subprocess.run(base, check=True, capture_output=True)
        os.replace(_LIB + ".tmp", _LIB)
        return _LIB


def lib():
    global _lib
    if _lib is None:
        path = build()
        L = C.CDLL(path)
        vp, i, d = C.c_void_p, C.c_int, C.c_double
        L.orc_philox4x32_10.argtypes = [vp, vp, vp]
        L.orc_ao_full.argtypes = [vp, vp, vp, vp, vp, vp, vp]
        L.orc_logpsi.argtypes = [vp, vp, vp]
        L.orc_logpsi.restype = i
        L.orc_local_energy_ex.argtypes = [vp, vp, vp, vp, vp]
        L.orc_local_energy_ex.restype = i
        L.orc_local_energy_batch.argtypes = [vp, vp, i, vp]
        L.orc_local_energy_batch.restype = i
        L.orc_logpsi_batch.argtypes = [vp, vp, i, vp, vp]
        L.orc_logpsi_batch.restype = i
        L.orc_det_inverse.argtypes = [i, vp, vp, vp, vp]
        L.orc_det_inverse.restype = i
        L.orc_geminal.argtypes = [vp, vp, vp]
        L.orc_jastrow.argtypes = [vp, vp]
        L.orc_jastrow.restype = d
        L.orc_jastrow_derivs.argtypes = [vp, vp, vp, vp]
        L.orc_sm_ratio_row.argtypes = [i, vp, i, vp]
        L.orc_sm_ratio_row.restype = d
        L.orc_sm_update_row.argtypes = [i, vp, i, vp]
        L.orc_move_draws.argtypes = [C.c_uint64, C.c_uint32, C.c_uint32, C.c_uint32, d, vp, vp, vp]
        L.orc_vmc.argtypes = [vp, vp, i, C.c_longlong, C.c_uint64, C.c_longlong, i, d, vp, vp, vp, i]
        L.orc_vmc.restype = i
        L.orc_grad_logpsi.argtypes = [vp, vp, vp, vp, vp, vp]
        L.orc_grad_logpsi.restype = i
        L.orc_max_threads.restype = i
        L.orc_elocal_grad_fd.argtypes = [vp, vp, d, vp, vp]
        L.orc_elocal_grad_fd.restype = i
        L.orc_elocal_dlambda_fd.argtypes = [vp, vp, i, i, d]
        L.orc_elocal_dlambda_fd.restype = d
        L.orc_elocal_fd_select.argtypes = [vp, vp, d, i, vp, vp, vp]
        L.orc_elocal_fd_select.restype = i
        L.orc_lrdmc_hops.argtypes = [vp, vp, d, d, vp, vp, vp, vp]
        L.orc_lrdmc_hops.restype = i
        L.orc_lrdmc_project.argtypes = [vp, vp, i, C.c_longlong, C.c_uint64, C.c_longlong, d, d, d, d, i, vp, vp,
                                        vp, vp, i]
        L.orc_lrdmc_project.restype = i
        L.orc_lrdmc_branch.argtypes = [i, C.c_uint64, C.c_longlong, vp, vp, vp, vp, vp]
        L.orc_lrdmc_branch.restype = None
        L.orc_lrdmc_energy.argtypes = [i, vp, vp, i]
        L.orc_lrdmc_energy.restype = d
        L.orc_reblock_levels.argtypes = [i]
        L.orc_reblock_levels.restype = i
        L.orc_reblock.argtypes = [vp, i, i, vp, vp]
        L.orc_reblock.restype = i
        L.orc_guiding_R.argtypes = [vp, vp, d]
        L.orc_guiding_R.restype = d
        L.orc_vmc_guided.argtypes = [vp, vp, i, C.c_longlong, C.c_uint64, C.c_longlong, i, d, d, d, vp, vp, vp, vp,
                                     i]
        L.orc_vmc_guided.restype = i
        L.orc_swct_omega.argtypes = [vp, vp, vp, vp]
        L.orc_swct_derivs.argtypes = [vp, vp, d, vp, vp]
        L.orc_swct_derivs.restype = i
        L.orc_sr.argtypes = [vp, vp, i, i, d, d, vp, vp, vp, vp]
        L.orc_sr.restype = i
        _lib = L
    return _lib


def _p(a):
    return None if a is None else a.ctypes.data


def philox4x32_10(ctr, key):
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    o = np.zeros(4, np.uint32)
    lib().orc_philox4x32_10(_p(c), _p(k), _p(o))
    return o


def det_inverse(A):
    A = np.ascontiguousarray(A, dtype=np.float64)
    n = A.shape[0]
    la, sg = np.zeros(1), np.zeros(1)
    inv = np.zeros((n, n))
    ok = lib().orc_det_inverse(n, _p(A), _p(la), _p(sg), _p(inv))
    return bool(ok), float(la[0]), float(sg[0]), inv


def sm_ratio_row(Ginv, i, newrow):
    Ginv = np.ascontiguousarray(Ginv, dtype=np.float64)
    newrow = np.ascontiguousarray(newrow, dtype=np.float64)
    return lib().orc_sm_ratio_row(Ginv.shape[0], _p(Ginv), int(i), _p(newrow))


def sm_update_row(Ginv, i, newrow):
    G = np.array(Ginv, dtype=np.float64, order="C")
    newrow = np.ascontiguousarray(newrow, dtype=np.float64)
    lib().orc_sm_update_row(G.shape[0], _p(G), int(i), _p(newrow))
    return G


def move_draws(seed, walker, sweep, electron, delta, r):
    r = np.ascontiguousarray(r, dtype=np.float64)
    rp = np.zeros(3)
    u = np.zeros(1)
    lib().orc_move_draws(C.c_uint64(seed), walker, sweep, electron, float(delta), _p(r), _p(rp), _p(u))
    return rp, float(u[0])


def reblock(eL):
    """Reblocking of eL [T][W] (see orc_reblock): (levels [nlev][4] = block
    size, blocks, sigma, error of sigma; stats = mean, chosen sigma, chosen
    level, plateau flag)."""
    eL = np.ascontiguousarray(eL, dtype=np.float64)
    if eL.ndim == 1:
        eL = eL[:, None]
    T, W = eL.shape
    nlev = lib().orc_reblock_levels(T)
    lev = np.zeros((max(nlev, 1), 4))
    st = np.zeros(4)
    lib().orc_reblock(_p(eL), T, W, _p(lev), _p(st))
    return lev[:nlev], st


def sr(O, e, eps=1e-3, delta=1.0, want_S=True):
    """Stochastic reconfiguration from samples (see orc_sr): O [M][P]
    log-derivatives, e [M] local energies.  Returns dict(Obar, S, f, dalpha)."""
    O = np.ascontiguousarray(O, dtype=np.float64)
    e = np.ascontiguousarray(e, dtype=np.float64)
    M, P = O.shape
    Ob, f, da = np.zeros(P), np.zeros(P), np.zeros(P)
    S = np.zeros((P, P)) if want_S else None
    ok = lib().orc_sr(_p(O), _p(e), M, P, float(eps), float(delta), _p(Ob), _p(S), _p(f), _p(da))
    if not ok:
        raise ValueError("singular regularised S matrix")
    return {"Obar": Ob, "S": S, "f": f, "dalpha": da}


def lrdmc_branch(w, eL, seed=0, gen=0):
    """Reconfiguration after an LRDMC projection (Eqs. branching-1, -2):
    (parent indices [W], wbar, ebar)."""
    w = np.ascontiguousarray(w, dtype=np.float64)
    eL = np.ascontiguousarray(eL, dtype=np.float64)
    W = int(w.shape[0])
    parent = np.zeros(W, dtype=np.int32)
    wb, eb = C.c_double(), C.c_double()
    lib().orc_lrdmc_branch(W, int(seed), int(gen), _p(w), _p(eL), _p(parent), C.addressof(wb), C.addressof(eb))
    return parent, wb.value, eb.value


def lrdmc_energy(wbar, ebar, p):
    """LRDMC energy with the correcting factor of p generations."""
    wbar = np.ascontiguousarray(wbar, dtype=np.float64)
    ebar = np.ascontiguousarray(ebar, dtype=np.float64)
    return float(lib().orc_lrdmc_energy(int(wbar.shape[0]), _p(wbar), _p(ebar), int(p)))


def max_threads() -> int:
    return int(lib().orc_max_threads())


class Oracle:
    """The oracle bound to one synthetic system (``synth.System``)."""

    def __init__(self, sys):
        self.sys = sys
        self._keep = [sys.R, sys.Z, sys.shell_atom, sys.shell_l, sys.shell_radial,
                      sys.shell_zeta, sys.lam, sys.unpaired]
        s = _OrcSystem()
        s.n_atoms = sys.n_atoms
        s.R, s.Z = _p(sys.R), _p(sys.Z)
        s.n_shells = sys.n_shells
        s.shell_atom, s.shell_l = _p(sys.shell_atom), _p(sys.shell_l)
        s.shell_radial, s.shell_zeta = _p(sys.shell_radial), _p(sys.shell_zeta)
        s.L = sys.L
        s.lam = _p(sys.lam)
        s.n_up, s.n_dn = sys.n_up, sys.n_dn
        s.unpaired = _p(sys.unpaired)
        s.b_ea, s.b_para, s.b_anti = sys.b_ea, sys.b_para, sys.b_anti
        s.use_j1, s.use_j2 = int(sys.use_j1), int(sys.use_j2)
        s.j2_spin_independent = int(sys.j2_spin_independent)
        j3 = getattr(sys, "j3", None)
        if j3 is not None:
            self._keep += [j3[k] for k in ("shell_atom", "shell_l", "shell_radial", "shell_zeta", "para", "anti")]
            s.n_jshells = int(len(j3["shell_l"]))
            s.jshell_atom, s.jshell_l = _p(j3["shell_atom"]), _p(j3["shell_l"])
            s.jshell_radial, s.jshell_zeta = _p(j3["shell_radial"]), _p(j3["shell_zeta"])
            s.LJ = int(j3["para"].shape[0])
            s.j3_para, s.j3_anti = _p(j3["para"]), _p(j3["anti"])
            s.use_j3 = 1
        self._s = s
        self._ps = C.addressof(s)
        self.N, self.L, self.nu = sys.N, sys.L, sys.n_up

    # --- single configuration --------------------------------------------
    def ao(self, r, hess=False):
        r = np.ascontiguousarray(r, dtype=np.float64)
        L = self.L
        v, g, l = np.zeros(L), np.zeros((L, 3)), np.zeros(L)
        H = np.zeros((L, 3, 3)) if hess else None
        gl = np.zeros((L, 3)) if hess else None
        lib().orc_ao_full(self._ps, _p(r), _p(v), _p(g), _p(l), _p(H), _p(gl))
        return (v, g, l, H, gl) if hess else (v, g, l)

    def geminal(self, x):
        x = np.ascontiguousarray(x, dtype=np.float64)
        phi = np.stack([self.ao(x[i])[0] for i in range(self.N)])
        G = np.zeros((self.nu, self.nu))
        lib().orc_geminal(self._ps, _p(phi), _p(G))
        return G

    def logpsi(self, x):
        """(log|Psi|, sign, log|det G~|, J)"""
        x = np.ascontiguousarray(x, dtype=np.float64)
        out = np.zeros(4)
        ok = lib().orc_logpsi(self._ps, _p(x), _p(out))
        if not ok:
            raise ValueError("singular geminal matrix")
        return tuple(float(v) for v in out)

    def jastrow(self, x):
        x = np.ascontiguousarray(x, dtype=np.float64)
        return float(lib().orc_jastrow(self._ps, _p(x)))

    def jastrow_derivs(self, x):
        x = np.ascontiguousarray(x, dtype=np.float64)
        g, l = np.zeros((self.N, 3)), np.zeros(self.N)
        lib().orc_jastrow_derivs(self._ps, _p(x), _p(g), _p(l))
        return g, l

    def local_energy(self, x, parts=False):
        """e_L (or (e_L, kinetic, V_ee, V_ei, V_ii, gradD/D, lapD/D) if parts)."""
        x = np.ascontiguousarray(x, dtype=np.float64)
        out = np.zeros(5)
        gD, lD = np.zeros((self.N, 3)), np.zeros(self.N)
        ok = lib().orc_local_energy_ex(self._ps, _p(x), _p(out), _p(gD), _p(lD))
        if not ok:
            raise ValueError("singular geminal matrix")
        return (tuple(float(v) for v in out) + (gD, lD)) if parts else float(out[0])

    def logpsi_derivs(self, x):
        """Per-configuration log-derivatives O_k = d ln|Psi| / d alpha_k for the
        parameters (every entry of lambda, row-major, then b_ea, b_para,
        b_anti): x [W][N][3] -> O [W][L*L + 3]."""
        x = np.ascontiguousarray(x, dtype=np.float64)
        W = x.shape[0]
        O = np.zeros((W, self.L * self.L + 3))
        for w in range(W):
            g = self.grad_logpsi(x[w])
            O[w, :self.L * self.L] = g["lam"].ravel()
            O[w, self.L * self.L:] = g["jas"]
        return O

    def grad_logpsi(self, x, want_lam=True):
        x = np.ascontiguousarray(x, dtype=np.float64)
        dlam = np.zeros((self.L, self.L)) if want_lam else None
        djas = np.zeros(3)
        dR = np.zeros((self.sys.n_atoms, 3))
        dr = np.zeros((self.N, 3))
        ok = lib().orc_grad_logpsi(self._ps, _p(x), _p(dlam), _p(djas), _p(dR), _p(dr))
        if not ok:
            raise ValueError("singular geminal matrix")
        return {"lam": dlam, "jas": djas, "R": dR, "r": dr}

    def elocal_grad(self, x, h=1e-3, want_R=True, want_r=True):
        """Reference d e_L / d R_a and d e_L / d r_i (Richardson-extrapolated
        central differences of the local energy, error O(h^4))."""
        x = np.ascontiguousarray(x, dtype=np.float64)
        dR = np.zeros((self.sys.n_atoms, 3)) if want_R else None
        dr = np.zeros((self.N, 3)) if want_r else None
        lib().orc_elocal_grad_fd(self._ps, _p(x), float(h), _p(dR), _p(dr))
        return dR, dr

    def elocal_fd_select(self, x, R=(), r=(), lam=(), h=1e-4):
        """Selected components of the same Richardson-extrapolated central
        differences, in parallel: R and r are lists of (atom or electron, axis),
        lam a list of (mu, nu).  Returns the values in the order R, r, lam."""
        x = np.ascontiguousarray(x, dtype=np.float64)
        kind = [0] * len(R) + [1] * len(r) + [2] * len(lam)
        index = [3 * a + q for a, q in R] + [3 * i + q for i, q in r] + [mu * self.L + nu for mu, nu in lam]
        kind = np.array(kind, dtype=np.int32)
        index = np.array(index, dtype=np.int64)
        out = np.zeros(len(kind))
        if not lib().orc_elocal_fd_select(self._ps, _p(x), float(h), len(kind), _p(kind), _p(index), _p(out)):
            raise ValueError("bad component")
        return out

    def lrdmc_hops(self, x, a, gamma=0.0):
        """Hop ratios rho [6N], rates t [6N], Gamma and e_L of one configuration
        (Sec. "Lattice regularized Monte Carlo"); hop k = 6 i + 2 d + s."""
        x = np.ascontiguousarray(x, dtype=np.float64)
        rho, t = np.zeros(6 * self.N), np.zeros(6 * self.N)
        G, e = C.c_double(), C.c_double()
        if not lib().orc_lrdmc_hops(self._ps, _p(x), float(a), float(gamma), _p(rho), _p(t), C.addressof(G),
                                    C.addressof(e)):
            raise ValueError("singular geminal matrix")
        return rho, t, G.value, e.value

    def lrdmc_project(self, x, weight, seed=0, gen=0, a=0.2, gamma=0.0, tau=0.1, e_ref=0.0, max_hops=1 << 20,
                      walker0=0, nthreads=0):
        """One continuous-time projection of length tau per walker; x [W][N][3]
        and weight [W] are updated in place.  Returns (e_L [W], hops [W], flags [W])."""
        assert x.flags.c_contiguous and x.dtype == np.float64
        assert weight.flags.c_contiguous and weight.dtype == np.float64
        W = x.shape[0]
        eL, hops, flags = np.zeros(W), np.zeros(W, dtype=np.int32), np.zeros(W, dtype=np.int32)
        ok = lib().orc_lrdmc_project(self._ps, _p(x), W, int(walker0), int(seed), int(gen), float(a), float(gamma),
                                     float(tau), float(e_ref), int(max_hops), _p(weight), _p(eL), _p(hops),
                                     _p(flags), int(nthreads))
        if not ok:
            raise ValueError("singular geminal matrix")
        return eL, hops, flags

    def lrdmc(self, x, ngen, seed=0, a=0.2, gamma=0.0, tau=0.1, e_ref=0.0, max_hops=1 << 20, gen0=0,
              branch=True, nthreads=0):
        """ngen generations (projection, then reconfiguration); x [W][N][3] in
        place.  Returns per-generation wbar, ebar [ngen], e_L, hops, parents,
        weights [ngen][W] (weights before the reconfiguration)."""
        W = x.shape[0]
        out = {k: [] for k in ("wbar", "ebar", "eL", "hops", "parent", "weight", "flags")}
        w = np.ones(W)
        for gi in range(ngen):
            g = gen0 + gi
            eL, hops, flags = self.lrdmc_project(x, w, seed, g, a, gamma, tau, e_ref, max_hops, 0, nthreads)
            out["eL"].append(eL)
            out["hops"].append(hops)
            out["flags"].append(flags)
            out["weight"].append(w.copy())
            if branch:
                parent, wb, eb = lrdmc_branch(w, eL, seed, g)
                x[:] = x[parent]
                w = np.ones(W)
            else:
                parent = np.arange(W, dtype=np.int32)
                wb, eb = w.mean(), float((w * eL).sum() / w.sum())
            out["parent"].append(parent)
            out["wbar"].append(wb)
            out["ebar"].append(eb)
        return {k: np.array(v) for k, v in out.items()}

    def guiding_R(self, x, theta=0.375):
        """R(x) = (S sum |G~^{-1}|^2)^-theta of one configuration (Eq. R_r)."""
        x = np.ascontiguousarray(x, dtype=np.float64)
        return float(lib().orc_guiding_R(self._ps, _p(x), float(theta)))

    def vmc_guided(self, x, nsweeps, theta=0.375, eps=1e-3, seed=0, sweep0=0, walker0=0, delta=None,
                   record_eL=True, nthreads=0):
        """As vmc(), sampling the guiding function Psi_G = (max(R, eps) / R) Psi_T.
        Returns (eL [nsweeps][W], logpsi [W], n_accept [W], R [W] of the final configurations)."""
        assert x.dtype == np.float64 and x.flags["C_CONTIGUOUS"]
        W = x.shape[0]
        eL = np.zeros((nsweeps, W)) if record_eL else None
        lp, R = np.zeros(W), np.zeros(W)
        nacc = np.zeros(W, dtype=np.int64)
        d = self.sys.delta if delta is None else delta
        ok = lib().orc_vmc_guided(self._ps, _p(x), W, walker0, C.c_uint64(seed), sweep0, nsweeps, float(d),
                                  float(theta), float(eps), _p(eL), _p(lp), _p(nacc), _p(R), int(nthreads))
        if not ok:
            raise ValueError("singular geminal matrix at the start of a walker")
        return eL, lp, nacc, R

    def swct_omega(self, r):
        """Space-warp weights omega_a(r) [n_atoms] and their gradients [n_atoms][3]."""
        r = np.ascontiguousarray(r, dtype=np.float64)
        na = self.sys.n_atoms
        om, dom = np.zeros(na), np.zeros((na, 3))
        lib().orc_swct_omega(self._ps, _p(r), _p(om), _p(dom))
        return om, dom

    def swct_derivs(self, x, h=1e-3):
        """(d e_L / d R_a, d ln(J^1/2 Psi) / d R_a) with the space warp, [n_atoms][3] each."""
        x = np.ascontiguousarray(x, dtype=np.float64)
        na = self.sys.n_atoms
        dE, dL = np.zeros((na, 3)), np.zeros((na, 3))
        if not lib().orc_swct_derivs(self._ps, _p(x), float(h), _p(dE), _p(dL)):
            raise ValueError("singular geminal matrix")
        return dE, dL

    def elocal_dlambda(self, x, mu, nu, h=1e-4):
        x = np.ascontiguousarray(x, dtype=np.float64)
        return float(lib().orc_elocal_dlambda_fd(self._ps, _p(x), int(mu), int(nu), float(h)))

    # --- batches ------------------------------------------------------------
    def local_energy_batch(self, x):
        x = np.ascontiguousarray(x, dtype=np.float64)
        W = x.shape[0]
        e = np.zeros(W)
        lib().orc_local_energy_batch(self._ps, _p(x), W, _p(e))
        return e

    def logpsi_batch(self, x):
        x = np.ascontiguousarray(x, dtype=np.float64)
        W = x.shape[0]
        la, sg = np.zeros(W), np.zeros(W)
        lib().orc_logpsi_batch(self._ps, _p(x), W, _p(la), _p(sg))
        return la, sg

    def vmc(self, x, nsweeps, seed=0, sweep0=0, walker0=0, delta=None, record_eL=True,
            nthreads=0):
        """Run nsweeps Metropolis sweeps in place on x [W][N][3].
        Returns (eL [nsweeps][W] or None, logpsi [W], n_accept [W])."""
        assert x.dtype == np.float64 and x.flags["C_CONTIGUOUS"]
        W = x.shape[0]
        eL = np.zeros((nsweeps, W)) if record_eL else None
        lp = np.zeros(W)
        nacc = np.zeros(W, dtype=np.int64)
        d = self.sys.delta if delta is None else delta
        ok = lib().orc_vmc(self._ps, _p(x), W, walker0, C.c_uint64(seed), sweep0, nsweeps, float(d),
                           _p(eL), _p(lp), _p(nacc), int(nthreads))
        if not ok:
            raise ValueError("singular geminal matrix at the start of a walker")
        return eL, lp, nacc
