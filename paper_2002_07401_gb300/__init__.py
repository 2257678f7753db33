"""GB300 (sm_103a) JAGP variational Monte Carlo hot path -- Python binding.

A thin ctypes layer over the C ABI in ``include/jagp.h``: the functions below
carry the same names as the C entry points and only marshal arguments (torch
tensors give device memory and streams; every step runs in libjagp's CUDA
kernels).  There is no CPU fallback: without the built library or a CUDA
device every call raises.
"""
from __future__ import annotations

import ctypes as C
import os
from typing import Optional

import numpy as np

from . import build as _build

JAGP_OK = 0
JAGP_PREC_FP64 = 0
JAGP_PREC_MIXED = 1
WS_NONFINITE, WS_SINGULAR, WS_DRIFT = 1, 2, 4


class JagpError(RuntimeError):
    pass


class _System(C.Structure):
    _fields_ = [
        ("n_atoms", C.c_int), ("R", C.c_void_p), ("Z", C.c_void_p),
        ("n_shells", C.c_int), ("shell_atom", C.c_void_p), ("shell_l", C.c_void_p),
        ("shell_radial", C.c_void_p), ("shell_zeta", C.c_void_p), ("lambda_", C.c_void_p),
        ("n_up", C.c_int), ("n_dn", C.c_int), ("unpaired", C.c_void_p),
        ("b_ea", C.c_double), ("b_para", C.c_double), ("b_anti", C.c_double),
        ("use_j1", C.c_int), ("use_j2", C.c_int), ("j2_spin_independent", C.c_int),
        ("n_jshells", C.c_int), ("jshell_atom", C.c_void_p), ("jshell_l", C.c_void_p),
        ("jshell_radial", C.c_void_p), ("jshell_zeta", C.c_void_p), ("j3_para", C.c_void_p),
        ("j3_anti", C.c_void_p), ("use_j3", C.c_int),
    ]


class _Options(C.Structure):
    _fields_ = [
        ("precision", C.c_int), ("max_walkers", C.c_int), ("delta", C.c_double),
        ("seed", C.c_uint64), ("drift_tol", C.c_double), ("refresh_moves", C.c_int),
        ("fp64_tensor_cores", C.c_int),
    ]


class _Tuning(C.Structure):
    _fields_ = [("tile_proposals", C.c_int), ("tile_refresh", C.c_int), ("umma_bn_left", C.c_int),
                ("umma_bn_right", C.c_int), ("ms", C.c_float * 4), ("umma_stages_left", C.c_int),
                ("umma_stages_right", C.c_int)]


_lib = None


def lib():
    """Load libjagp.so (building it first if the sources are newer)."""
    global _lib
    if _lib is None:
        path = _build.build()
        if not os.path.exists(path):
            raise JagpError(f"libjagp not found at {path}")
        L = C.CDLL(path)
        vp, i, d, u64 = C.c_void_p, C.c_int, C.c_double, C.c_uint64
        L.jagp_create.argtypes = [C.POINTER(vp), C.POINTER(_System), C.POINTER(_Options)]
        L.jagp_destroy.argtypes = [vp]
        L.jagp_state_bytes.argtypes = [vp, i]
        L.jagp_state_bytes.restype = C.c_size_t
        L.jagp_eval.argtypes = [vp, vp, i, vp, vp, vp, vp]
        L.vmc_sweep.argtypes = [vp, vp, vp, i, i, u64, u64, vp, vp, vp]
        L.local_energy.argtypes = [vp, vp, vp, i, vp, vp, vp]
        L.jagp_walker_info.argtypes = [vp, vp, i, vp, vp, vp, vp, vp, vp]
        L.jagp_walker_status.argtypes = [vp, vp, i, C.POINTER(C.c_int), vp]
        L.jagp_profile.argtypes = [vp, i, i]
        L.jagp_profile.restype = i
        L.jagp_profile_read.argtypes = [vp, C.POINTER(C.c_double), C.POINTER(C.c_longlong)]
        L.jagp_profile_read.restype = i
        L.jagp_launch_count.argtypes = [vp]
        L.jagp_launch_count.restype = C.c_longlong
        L.jagp_gemm_bf16x.argtypes = [vp, i, i, vp, i, i, i, i, vp, vp, vp, C.c_longlong, vp, vp, vp, vp, vp, vp]
        L.jagp_gemm_bf16x.restype = i
        L.jagp_grad_workspace_bytes.argtypes = [vp, i]
        L.jagp_grad_workspace_bytes.restype = C.c_size_t
        L.jagp_grad.argtypes = [vp, vp, vp, i, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp]
        L.jagp_grad.restype = i
        L.jagp_batch_create.argtypes = [C.POINTER(vp), i, vp, vp, vp, vp, vp, vp, vp, i]
        L.jagp_batch_create.restype = i
        L.jagp_batch_sweep.argtypes = [vp, i, u64, vp]
        L.jagp_batch_sweep.restype = i
        L.jagp_batch_launches.argtypes = [vp, C.POINTER(C.c_longlong), C.POINTER(C.c_longlong)]
        L.jagp_batch_launches.restype = i
        L.jagp_batch_destroy.argtypes = [vp]
        L.jagp_batch_destroy.restype = i
        L.jagp_autotune.argtypes = [vp, vp, i, C.POINTER(_Tuning), vp]
        L.jagp_autotune.restype = i
        L.jagp_set_tuning.argtypes = [vp, C.POINTER(_Tuning)]
        L.jagp_set_tuning.restype = i
        L.jagp_eval_noalloc.argtypes = [vp, vp, i, vp, vp, vp]
        L.jagp_eval_noalloc.restype = i
        L.jagp_last_cuda_error.argtypes = []
        L.jagp_last_cuda_error.restype = C.c_char_p
        L.jagp_logpsi_derivs_workspace_bytes.argtypes = [vp, i]
        L.jagp_logpsi_derivs_workspace_bytes.restype = C.c_size_t
        L.jagp_logpsi_derivs.argtypes = [vp, vp, vp, i, vp, vp, C.c_longlong, vp]
        L.jagp_logpsi_derivs.restype = i
        L.jagp_sr_workspace_bytes.argtypes = [i, i]
        L.jagp_sr_workspace_bytes.restype = C.c_size_t
        L.jagp_sr_step.argtypes = [vp, C.c_longlong, vp, i, i, d, d, i, d, vp, vp, vp, C.POINTER(i), C.POINTER(d),
                                   vp]
        L.jagp_sr_step.restype = i
        L.jagp_set_guiding.argtypes = [vp, d, d]
        L.jagp_set_guiding.restype = i
        L.jagp_space_warp.argtypes = [vp, vp, i, vp, vp, vp, vp, vp]
        L.jagp_space_warp.restype = i
        L.jagp_guiding_weights.argtypes = [vp, vp, i, d, d, vp, vp, vp]
        L.jagp_guiding_weights.restype = i
        L.jagp_force_seeds.argtypes = [vp, vp, i, vp, vp, vp, vp]
        L.jagp_force_seeds.restype = i
        L.jagp_reblock_levels.argtypes = [i]
        L.jagp_reblock_levels.restype = i
        L.jagp_reblock.argtypes = [vp, i, i, vp, vp, vp, vp]
        L.jagp_reblock.restype = i
        L.jagp_lrdmc_workspace_bytes.argtypes = [vp, i]
        L.jagp_lrdmc_workspace_bytes.restype = C.c_size_t
        L.jagp_lrdmc_project.argtypes = [vp, vp, vp, i, u64, u64, d, d, d, d, i, vp, vp, vp, vp, vp, vp]
        L.jagp_lrdmc_project.restype = i
        L.jagp_lrdmc_branch.argtypes = [vp, vp, i, u64, vp, vp, vp, vp, vp, vp]
        L.jagp_lrdmc_branch.restype = i
        L.jagp_lrdmc_energy.argtypes = [vp, vp, i, i, vp, vp]
        L.jagp_lrdmc_energy.restype = i
        L.jagp_last_error.argtypes = [vp, C.c_char_p, C.c_size_t]
        L.jagp_last_error.restype = i
        L.jagp_status_string.argtypes = [i]
        L.jagp_status_string.restype = C.c_char_p
        for f in ("jagp_create", "jagp_destroy", "jagp_eval", "vmc_sweep", "local_energy",
                  "jagp_walker_info", "jagp_walker_status"):
            getattr(L, f).restype = i
        _lib = L
    return _lib


def library_path() -> str:
    return _build.LIB


def _check(status: int, what: str, h=None):
    if status != JAGP_OK:
        msg = lib().jagp_status_string(status).decode()
        if h:
            msg = jagp_last_error(h)[1]
        elif status == 7:
            msg += ": " + lib().jagp_last_cuda_error().decode()
        raise JagpError(f"{what} failed: {msg} (status {status})")


def jagp_last_error(h):
    """(status, text) of the last failure recorded on handle h."""
    buf = C.create_string_buffer(512)
    st = lib().jagp_last_error(h, buf, len(buf))
    return int(st), buf.value.decode()


def _ptr(t) -> Optional[int]:
    if t is None:
        return None
    return t.data_ptr()


def _stream(stream) -> Optional[int]:
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return stream.cuda_stream


# --------------------------------------------------------------------------
# C entry points under the same names (argument marshalling only)
# --------------------------------------------------------------------------

def jagp_create(sysm, precision: int = JAGP_PREC_FP64, max_walkers: int = 1, delta: Optional[float] = None,
                seed: int = 0, drift_tol: float = 0.0, refresh_moves: int = 0, fp64_tc: bool = False) -> int:
    """sysm: a ``synth.System``-like object (numpy arrays).  Returns the handle."""
    keep = []

    def arr(a, dt):
        if a is None:
            return None
        a = np.ascontiguousarray(a, dtype=dt)
        keep.append(a)
        return a.ctypes.data

    s = _System()
    s.n_atoms = int(sysm.R.shape[0])
    s.R, s.Z = arr(sysm.R, np.float64), arr(sysm.Z, np.float64)
    s.n_shells = int(len(sysm.shell_l))
    s.shell_atom, s.shell_l = arr(sysm.shell_atom, np.int32), arr(sysm.shell_l, np.int32)
    s.shell_radial, s.shell_zeta = arr(sysm.shell_radial, np.int32), arr(sysm.shell_zeta, np.float64)
    s.lambda_ = arr(sysm.lam, np.float64)
    s.n_up, s.n_dn = int(sysm.n_up), int(sysm.n_dn)
    s.unpaired = arr(sysm.unpaired, np.float64)
    s.b_ea, s.b_para, s.b_anti = float(sysm.b_ea), float(sysm.b_para), float(sysm.b_anti)
    s.use_j1, s.use_j2 = int(sysm.use_j1), int(sysm.use_j2)
    s.j2_spin_independent = int(sysm.j2_spin_independent)
    j3 = getattr(sysm, "j3", None)
    if j3 is not None:
        s.n_jshells = int(len(j3["shell_l"]))
        s.jshell_atom, s.jshell_l = arr(j3["shell_atom"], np.int32), arr(j3["shell_l"], np.int32)
        s.jshell_radial, s.jshell_zeta = arr(j3["shell_radial"], np.int32), arr(j3["shell_zeta"], np.float64)
        s.j3_para, s.j3_anti = arr(j3["para"], np.float64), arr(j3["anti"], np.float64)
        s.use_j3 = 1
    o = _Options()
    o.precision, o.max_walkers = int(precision), int(max_walkers)
    o.delta = float(sysm.delta if delta is None else delta)
    o.seed, o.drift_tol = int(seed), float(drift_tol)
    o.refresh_moves = int(refresh_moves)
    o.fp64_tensor_cores = int(bool(fp64_tc))
    h = C.c_void_p()
    _check(lib().jagp_create(C.byref(h), C.byref(s), C.byref(o)), "jagp_create")
    return h.value


def jagp_destroy(h: int):
    _check(lib().jagp_destroy(h), "jagp_destroy")


def jagp_state_bytes(h: int, W: int) -> int:
    return int(lib().jagp_state_bytes(h, int(W)))


def jagp_eval(h, r, W, state, logabs=None, sign=None, stream=None):
    _check(lib().jagp_eval(h, _ptr(r), int(W), _ptr(state), _ptr(logabs), _ptr(sign), _stream(stream)),
           "jagp_eval", h)


NOALLOC_SCRATCH_BYTES = 32 << 20


def jagp_eval_noalloc(h, r, W, logabs=None, sign=None, stream=None):
    """log|Psi| and sign like jagp_eval, for callers that cannot allocate device
    memory: the library keeps the scratch in a fixed 32 MiB device array shared
    by all calls (serialise calls; the first call on a device must precede any
    stream capture).  Raises for W whose scratch does not fit."""
    _check(lib().jagp_eval_noalloc(h, _ptr(r), int(W), _ptr(logabs), _ptr(sign), _stream(stream)),
           "jagp_eval_noalloc", h)


def vmc_sweep(h, r, state, W, nsweeps, walker0=0, sweep0=0, eL=None, acc=None, stream=None):
    _check(lib().vmc_sweep(h, _ptr(r), _ptr(state), int(W), int(nsweeps), int(walker0), int(sweep0),
                           _ptr(eL), _ptr(acc), _stream(stream)), "vmc_sweep", h)


def local_energy(h, r, state, W, eL, parts=None, stream=None):
    _check(lib().local_energy(h, _ptr(r), _ptr(state), int(W), _ptr(eL), _ptr(parts), _stream(stream)),
           "local_energy", h)


def jagp_grad_workspace_bytes(h, W) -> int:
    return int(lib().jagp_grad_workspace_bytes(h, int(W)))


def jagp_grad(h, r, state, W, work, seed_logpsi=None, seed_eL=None, eL=None, dlambda=None, djas=None, dR=None,
              dR_walker=None, dr=None, stream=None):
    _check(lib().jagp_grad(h, _ptr(r), _ptr(state), int(W), _ptr(seed_logpsi), _ptr(seed_eL), _ptr(work), _ptr(eL),
                           _ptr(dlambda), _ptr(djas), _ptr(dR), _ptr(dR_walker), _ptr(dr), _stream(stream)),
           "jagp_grad", h)


def jagp_logpsi_derivs_workspace_bytes(h, W) -> int:
    return int(lib().jagp_logpsi_derivs_workspace_bytes(h, int(W)))


def jagp_logpsi_derivs(h, r, state, W, work, O, stream=None):
    _check(lib().jagp_logpsi_derivs(h, _ptr(r), _ptr(state), int(W), _ptr(work), _ptr(O), int(O.stride(0)),
                                    _stream(stream)), "jagp_logpsi_derivs", h)


def jagp_sr_workspace_bytes(M, P) -> int:
    return int(lib().jagp_sr_workspace_bytes(int(M), int(P)))


def jagp_sr_step(O, eL, eps=1e-3, delta=1.0, max_iter=500, tol=1e-12, P=None, work=None, stream=None):
    """One regularised SR step from samples O [M][>= P] and eL [M] (device FP64;
    see include/jagp.h).  Returns (f, dalpha, iterations, relative residual)."""
    import torch
    M = int(O.shape[0])
    P = int(O.shape[1]) if P is None else int(P)
    f64 = dict(dtype=torch.float64, device=O.device)
    if work is None:
        work = torch.empty(jagp_sr_workspace_bytes(M, P), dtype=torch.uint8, device=O.device)
    f, da = torch.empty(P, **f64), torch.empty(P, **f64)
    it, res = C.c_int(0), C.c_double(0.0)
    _check(lib().jagp_sr_step(_ptr(O), int(O.stride(0)), _ptr(eL.contiguous()), M, P, float(eps), float(delta),
                              int(max_iter), float(tol), _ptr(work), _ptr(f), _ptr(da), C.byref(it), C.byref(res),
                              _stream(stream)), "jagp_sr_step")
    return f, da, it.value, res.value


def jagp_set_guiding(h, theta=0.375, eps=0.0):
    _check(lib().jagp_set_guiding(h, float(theta), float(eps)), "jagp_set_guiding", h)


def tune_guiding_eps(g, r, target=0.8, theta=0.375, sweeps=4, rounds=8, walker0=0, sweep0=0):
    """Choose eps so that the mean reweighting factor <W> of the guided chain is
    near `target` (the paper takes 0.8): bisection in log eps over short guided
    runs of the JAGP object g on positions r (its state must be current).
    Leaves g sampling the guiding function with the chosen eps."""
    import torch
    W = r.shape[0]
    R = torch.empty(W, dtype=torch.float64, device=r.device)
    jagp_guiding_weights(g.h, g.state, W, theta, 0.0, R=R)
    Rs = R.sort().values
    lo, hi = float(Rs[0]) * 1e-3, float(Rs[-1])
    eps = float(torch.quantile(Rs, 1.0 - target))
    wt = torch.empty(W, dtype=torch.float64, device=r.device)
    for k in range(rounds):
        jagp_set_guiding(g.h, theta, eps)
        g.sweep(r, sweeps, walker0=walker0, sweep0=sweep0 + k * sweeps, energies=False)
        jagp_guiding_weights(g.h, g.state, W, theta, eps, weights=wt)
        m = float(wt.mean())
        if m > target:
            lo = eps
        else:
            hi = eps
        eps = (lo * hi) ** 0.5
    jagp_set_guiding(g.h, theta, eps)
    return eps


def jagp_space_warp(h, r, W, rbar, dR_walker, seed_logpsi=None, dR=None, stream=None):
    _check(lib().jagp_space_warp(h, _ptr(r), int(W), _ptr(rbar), _ptr(seed_logpsi), _ptr(dR_walker), _ptr(dR),
                                 _stream(stream)), "jagp_space_warp", h)


def jagp_guiding_weights(h, state, W, theta=0.375, eps=0.0, R=None, weights=None, stream=None):
    _check(lib().jagp_guiding_weights(h, _ptr(state), int(W), float(theta), float(eps), _ptr(R), _ptr(weights),
                                      _stream(stream)), "jagp_guiding_weights", h)


def jagp_force_seeds(eL, weights=None, stream=None):
    """(seed_logpsi, seed_eL, (E, mean weight)) of the (reweighted) force estimator."""
    import torch
    M = int(eL.shape[0])
    f64 = dict(dtype=torch.float64, device=eL.device)
    sL, sE, mean = torch.empty(M, **f64), torch.empty(M, **f64), torch.empty(2, **f64)
    _check(lib().jagp_force_seeds(_ptr(eL.contiguous()), _ptr(None if weights is None else weights.contiguous()), M,
                                  _ptr(sL), _ptr(sE), _ptr(mean), _stream(stream)), "jagp_force_seeds")
    return sL, sE, mean


def jagp_reblock_levels(T) -> int:
    return int(lib().jagp_reblock_levels(int(T)))


def jagp_reblock(eL, work=None, levels=None, stats=None, stream=None):
    """Reblocked error bar of the mean of eL [T][W] (device FP64; see
    include/jagp.h).  Returns (levels [nlev][4], stats [4]) device tensors."""
    import torch
    eL = eL.reshape(eL.shape[0], -1) if eL.dim() > 1 else eL.reshape(-1, 1)
    T, W = eL.shape
    f64 = dict(dtype=torch.float64, device=eL.device)
    nlev = jagp_reblock_levels(T)
    work = torch.empty(T, **f64) if work is None else work
    levels = torch.empty((max(nlev, 1), 4), **f64) if levels is None else levels
    stats = torch.empty(4, **f64) if stats is None else stats
    _check(lib().jagp_reblock(_ptr(eL.contiguous()), int(T), int(W), _ptr(work), _ptr(levels), _ptr(stats),
                              _stream(stream)), "jagp_reblock")
    return levels[:nlev], stats


def jagp_lrdmc_workspace_bytes(h, W) -> int:
    return int(lib().jagp_lrdmc_workspace_bytes(h, int(W)))


def jagp_lrdmc_project(h, r, state, W, work, weight, generation=0, a=0.2, gamma=0.0, tau=0.1, e_ref=0.0,
                       max_hops=1 << 20, walker0=0, eL=None, hops=None, flags=None, stream=None):
    """One continuous-time LRDMC projection of length tau (see include/jagp.h);
    r [W][N][3] and weight [W] (device FP64) are updated in place."""
    _check(lib().jagp_lrdmc_project(h, _ptr(r), _ptr(state), int(W), int(walker0), int(generation), float(a),
                                    float(gamma), float(tau), float(e_ref), int(max_hops), _ptr(weight), _ptr(eL),
                                    _ptr(hops), _ptr(flags), _ptr(work), _stream(stream)), "jagp_lrdmc_project", h)


def jagp_lrdmc_branch(h, r, W, work, weight, eL, generation=0, parent=None, stats=None, stream=None):
    """Reconfiguration after a projection: r replaced by the new population,
    weight reset to 1; returns (parent [W], stats [2] = (wbar, ebar)) device tensors."""
    import torch
    parent = torch.empty(W, dtype=torch.int32, device=r.device) if parent is None else parent
    stats = torch.empty(2, dtype=torch.float64, device=r.device) if stats is None else stats
    _check(lib().jagp_lrdmc_branch(h, _ptr(r), int(W), int(generation), _ptr(weight), _ptr(eL.contiguous()),
                                   _ptr(parent), _ptr(stats), _ptr(work), _stream(stream)), "jagp_lrdmc_branch", h)
    return parent, stats


def jagp_lrdmc_energy(wbar, ebar, p, stream=None):
    """LRDMC energy with the correcting factor of p generations (device tensor [1])."""
    import torch
    E = torch.empty(1, dtype=torch.float64, device=wbar.device)
    _check(lib().jagp_lrdmc_energy(_ptr(wbar.contiguous()), _ptr(ebar.contiguous()), int(wbar.shape[0]), int(p),
                                   _ptr(E), _stream(stream)), "jagp_lrdmc_energy")
    return E


def jagp_walker_info(h, state, W, logabs=None, sign=None, naccept=None, drift=None, status=None, stream=None):
    _check(lib().jagp_walker_info(h, _ptr(state), int(W), _ptr(logabs), _ptr(sign), _ptr(naccept), _ptr(drift),
                                  _ptr(status), _stream(stream)), "jagp_walker_info", h)


def jagp_walker_status(h, state, W, stream=None) -> int:
    bits = C.c_int(0)
    _check(lib().jagp_walker_status(h, _ptr(state), int(W), C.byref(bits), _stream(stream)),
           "jagp_walker_status", h)
    return bits.value


def jagp_gemm_bf16x(A, a_terms, B, b_terms, Kp, pairs, out, rows=None, count=None, err=None, stream=None,
                    row_exp=None, col_exp=None):
    """Tensor-core contraction: out[rows[m]][n] = sum over (a, b) in pairs of
    A[m, a*Kp:(a+1)*Kp] . B[n, b*Kp:(b+1)*Kp]  (A, B: bfloat16 tensors holding
    a_terms / b_terms BF16 terms of width Kp; out: float32).  With row_exp and
    col_exp (int32) the terms are fixed-point slices (see include/jagp.h)."""
    import torch
    arr_a = (C.c_int * len(pairs))(*[int(a) for a, _ in pairs])
    arr_b = (C.c_int * len(pairs))(*[int(b) for _, b in pairs])
    if err is None:
        err = torch.zeros(1, dtype=torch.int32, device=A.device)
    _check(lib().jagp_gemm_bf16x(_ptr(A), int(A.shape[0]), int(a_terms), _ptr(B), int(B.shape[0]), int(b_terms),
                                 int(Kp), len(pairs), arr_a, arr_b, _ptr(out), int(out.stride(0)), _ptr(rows),
                                 _ptr(count), _ptr(row_exp), _ptr(col_exp), _ptr(err), _stream(stream)),
           "jagp_gemm_bf16x")
    return err


KERNEL_LAMBDA_ROWS, KERNEL_GEMM_ROWS, KERNEL_METROPOLIS, KERNEL_BASIS, KERNEL_ENERGY = 1, 2, 3, 4, 5


def jagp_profile(h, kernel: int, enable: bool = True):
    _check(lib().jagp_profile(h, int(kernel), int(bool(enable))), "jagp_profile", h)


def jagp_profile_read(h):
    """(summed device milliseconds, launches) of the profiled kernel; synchronises its events."""
    ms, n = C.c_double(0.0), C.c_longlong(0)
    _check(lib().jagp_profile_read(h, C.byref(ms), C.byref(n)), "jagp_profile_read", h)
    return ms.value, n.value


def jagp_launch_count(h) -> int:
    return int(lib().jagp_launch_count(h))


# --------------------------------------------------------------------------
# convenience owner of a handle plus the walker state (device memory from torch)
# --------------------------------------------------------------------------

def jagp_autotune(h, state, W, stream=None) -> dict:
    """Tile autotuner (see include/jagp.h); returns the choices and best times."""
    t = _Tuning()
    _check(lib().jagp_autotune(h, _ptr(state), int(W), C.byref(t), _stream(stream)), "jagp_autotune", h)
    return {"tile_proposals": t.tile_proposals, "tile_refresh": t.tile_refresh, "umma_bn_left": t.umma_bn_left,
            "umma_bn_right": t.umma_bn_right, "umma_stages_left": t.umma_stages_left,
            "umma_stages_right": t.umma_stages_right, "ms": [float(v) for v in t.ms]}


def jagp_set_tuning(h, tuning: dict) -> None:
    """Pin tile choices (keys as jagp_autotune returns; see include/jagp.h)."""
    t = _Tuning()
    t.tile_proposals = int(tuning.get("tile_proposals", -1))
    t.tile_refresh = int(tuning.get("tile_refresh", -1))
    for k in ("umma_bn_left", "umma_bn_right", "umma_stages_left", "umma_stages_right"):
        setattr(t, k, int(tuning.get(k, 0)))
    _check(lib().jagp_set_tuning(h, C.byref(t)), "jagp_set_tuning", h)


class JAGP:
    """One system on the current CUDA device with state for up to W walkers."""

    def __init__(self, sysm, W: int, precision: int = JAGP_PREC_FP64, seed: int = 0,
                 delta: Optional[float] = None, drift_tol: float = 0.0, device: str = "cuda",
                 refresh_moves: int = 0, fp64_tc: bool = False):
        import torch
        if not torch.cuda.is_available():
            raise JagpError("libjagp needs a CUDA device; there is no CPU fallback")
        self.sys, self.W, self.device = sysm, int(W), torch.device(device)
        with torch.cuda.device(self.device):
            self.h = jagp_create(sysm, precision, W, delta, seed, drift_tol, refresh_moves, fp64_tc)
            nbytes = jagp_state_bytes(self.h, W)
            # 256-byte aligned: the caching allocator hands out 512-byte aligned blocks
            self.state = torch.empty(nbytes, dtype=torch.uint8, device=self.device)
        assert self.state.data_ptr() % 256 == 0
        self.N = sysm.n_up + sysm.n_dn

    def close(self):
        if getattr(self, "h", None):
            jagp_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def positions(self, x):
        import torch
        return torch.as_tensor(np.ascontiguousarray(x), dtype=torch.float64, device=self.device).contiguous()

    def autotune(self, r=None):
        """Tune the tile choices on this handle's state; re-evaluates r afterwards
        (the tuner overwrites the state's tables)."""
        out = jagp_autotune(self.h, self.state, self.W)
        if r is not None:
            self.eval(r)
        return out

    def set_tuning(self, tuning):
        jagp_set_tuning(self.h, tuning)

    def eval(self, r):
        import torch
        W = r.shape[0]
        la = torch.empty(W, dtype=torch.float64, device=self.device)
        sg = torch.empty(W, dtype=torch.float64, device=self.device)
        jagp_eval(self.h, r, W, self.state, la, sg)
        return la, sg

    def sweep(self, r, nsweeps, walker0=0, sweep0=0, energies=True, acc=False):
        import torch
        W = r.shape[0]
        eL = torch.empty((nsweeps, W), dtype=torch.float64, device=self.device) if energies else None
        ac = torch.empty((nsweeps, 4), dtype=torch.float64, device=self.device) if acc else None
        vmc_sweep(self.h, r, self.state, W, nsweeps, walker0, sweep0, eL, ac)
        return eL, ac

    def local_energy(self, r, parts=False):
        import torch
        W = r.shape[0]
        e = torch.empty(W, dtype=torch.float64, device=self.device)
        p = torch.empty((W, 4), dtype=torch.float64, device=self.device) if parts else None
        local_energy(self.h, r, self.state, W, e, p)
        return (e, p) if parts else e

    def info(self, W=None):
        import torch
        W = self.W if W is None else W
        f = lambda: torch.empty(W, dtype=torch.float64, device=self.device)  # noqa: E731
        la, sg, na, dr = f(), f(), f(), f()
        st = torch.empty(W, dtype=torch.int32, device=self.device)
        jagp_walker_info(self.h, self.state, W, la, sg, na, dr, st)
        return {"logabs": la, "sign": sg, "naccept": na, "drift": dr, "status": st}

    def status(self, W=None) -> int:
        return jagp_walker_status(self.h, self.state, self.W if W is None else W)

    def logpsi_derivs(self, r, O=None):
        """Per-walker log-derivatives O [W][L*L + 3] (lambda entries, then
        b_ea, b_para, b_anti) at the current state (jagp_logpsi_derivs)."""
        import torch
        W = r.shape[0]
        P = self.sys.L * self.sys.L + 3
        if O is None:
            O = torch.empty((W, P), dtype=torch.float64, device=self.device)
        work = torch.empty(jagp_logpsi_derivs_workspace_bytes(self.h, W), dtype=torch.uint8, device=self.device)
        jagp_logpsi_derivs(self.h, r, self.state, W, work, O)
        return O

    def lrdmc(self, r, ngen, a=0.2, gamma=0.0, tau=0.1, e_ref=0.0, max_hops=1 << 20, gen0=0, walker0=0):
        """ngen LRDMC generations (projection, then reconfiguration) on r in
        place (Sec. "Lattice regularized Monte Carlo").  Returns a dict of
        device tensors: wbar, ebar [ngen]; eL, hops, flags, parent and the
        weights before each reconfiguration, weight [ngen][W]."""
        import torch
        W = r.shape[0]
        dev = dict(device=self.device)
        work = torch.empty(jagp_lrdmc_workspace_bytes(self.h, W), dtype=torch.uint8, **dev)
        w = torch.ones(W, dtype=torch.float64, **dev)
        out = {"wbar": torch.empty(ngen, dtype=torch.float64, **dev),
               "ebar": torch.empty(ngen, dtype=torch.float64, **dev),
               "eL": torch.empty((ngen, W), dtype=torch.float64, **dev),
               "weight": torch.empty((ngen, W), dtype=torch.float64, **dev),
               "hops": torch.empty((ngen, W), dtype=torch.int32, **dev),
               "flags": torch.empty((ngen, W), dtype=torch.int32, **dev),
               "parent": torch.empty((ngen, W), dtype=torch.int32, **dev)}
        stats = torch.empty(2, dtype=torch.float64, **dev)
        for t in range(ngen):
            jagp_lrdmc_project(self.h, r, self.state, W, work, w, gen0 + t, a, gamma, tau, e_ref, max_hops, walker0,
                               out["eL"][t], out["hops"][t], out["flags"][t])
            out["weight"][t].copy_(w)
            jagp_lrdmc_branch(self.h, r, W, work, w, out["eL"][t], gen0 + t, out["parent"][t], stats)
            out["wbar"][t] = stats[0]
            out["ebar"][t] = stats[1]
        return out

    def grad(self, r, seed_logpsi=None, seed_eL=None, want_lambda=True):
        """Vector-Jacobian products of (log|Psi|, e_L) at the current state (see
        jagp_grad in include/jagp.h).  Returns a dict of device tensors."""
        import torch
        W = r.shape[0]
        work = torch.empty(jagp_grad_workspace_bytes(self.h, W), dtype=torch.uint8, device=self.device)
        f64 = dict(dtype=torch.float64, device=self.device)
        L, na = self.sys.L, self.sys.R.shape[0]
        out = {"eL": torch.empty(W, **f64), "lam": torch.empty((L, L), **f64) if want_lambda else None,
               "jas": torch.empty(3, **f64), "R": torch.empty((na, 3), **f64),
               "R_walker": torch.empty((W, na, 3), **f64), "r": torch.empty((W, self.N, 3), **f64)}
        sl = None if seed_logpsi is None else seed_logpsi.to(**f64).contiguous()
        se = None if seed_eL is None else seed_eL.to(**f64).contiguous()
        jagp_grad(self.h, r, self.state, W, work, sl, se, out["eL"], out["lam"], out["jas"], out["R"],
                  out["R_walker"], out["r"])
        return out


class Batch:
    """Independent systems swept together (jagp_batch_*): members are JAGP
    objects with their positions; every sweep is one replay of a captured CUDA
    graph, of each member's own launches over n_streams streams (bit for bit
    the per-member sweeps), or of grouped launches over all members
    (n_streams = 0, or -k for k lanes: about a hundred launches per sweep).
    eL[s] holds the last sweep's local energies, acc[s] the running (sum e_L,
    sum e_L^2, accepted moves, max drift)."""

    def __init__(self, members, positions, walker0=None, n_streams=16):
        import torch
        self.members, self.r = list(members), list(positions)
        S = len(self.members)
        dev = self.members[0].device
        self.eL = [torch.zeros(p.shape[0], dtype=torch.float64, device=dev) for p in self.r]
        self.acc = torch.zeros((S, 4), dtype=torch.float64, device=dev)
        vp = C.c_void_p
        hs = (vp * S)(*[m.h for m in self.members])
        st = (vp * S)(*[m.state.data_ptr() for m in self.members])
        rp = (vp * S)(*[p.data_ptr() for p in self.r])
        ep = (vp * S)(*[e.data_ptr() for e in self.eL])
        W = (C.c_int * S)(*[int(p.shape[0]) for p in self.r])
        w0 = (C.c_uint64 * S)(*([0] * S if walker0 is None else [int(v) for v in walker0]))
        b = vp()
        _check(lib().jagp_batch_create(C.byref(b), S, hs, st, rp, W, w0, ep, self.acc.data_ptr(), int(n_streams)),
               "jagp_batch_create")
        self.b = b.value

    def sweep(self, nsweeps, sweep0=0, stream=None):
        _check(lib().jagp_batch_sweep(self.b, int(nsweeps), int(sweep0), _stream(stream)), "jagp_batch_sweep")

    def launches_per_sweep(self) -> int:
        """Kernel launches in the graph one sweep replays (jagp_batch_launches)."""
        k, n = C.c_longlong(0), C.c_longlong(0)
        _check(lib().jagp_batch_launches(self.b, C.byref(k), C.byref(n)), "jagp_batch_launches")
        return int(k.value)

    def close(self):
        if getattr(self, "b", None):
            lib().jagp_batch_destroy(self.b)
            self.b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _autograd_function():
    import torch

    class LogPsiLocalEnergy(torch.autograd.Function):
        """(log|Psi|, e_L) of W configurations as a differentiable function of
        (lambda, Jastrow parameters, R, r); the backward pass is the library's
        adjoint (jagp_grad).  The library forms the Jastrow-parameter gradient
        of log|Psi| only (not d e_L / d b): a backward pass in which a non-zero
        e_L gradient would reach the Jastrow parameters raises instead of
        returning an incomplete gradient.  The tensors lam, jas, R must hold the
        values the JAGP object was created with."""

        @staticmethod
        def forward(ctx, g, lam, jas, R, r):
            r = r.detach().contiguous()
            la, _ = g.eval(r)
            eL = g.local_energy(r)
            ctx.g = g
            ctx.save_for_backward(r)
            return la, eL

        @staticmethod
        def backward(ctx, g_log, g_el):
            (r,) = ctx.saved_tensors
            g = ctx.g
            if ctx.needs_input_grad[2] and g_el is not None and bool((g_el != 0).any()):
                raise JagpError("d e_L / d (Jastrow parameters) is not formed by jagp_grad: detach the "
                                "Jastrow parameters or keep e_L out of the loss")
            g.eval(r)
            out = g.grad(r, seed_logpsi=g_log, seed_eL=g_el, want_lambda=ctx.needs_input_grad[1])
            return None, out["lam"], out["jas"], out["R"], out["r"]

    return LogPsiLocalEnergy


def logpsi_and_local_energy(g, lam, jas, R, r):
    """Differentiable (log|Psi|, e_L); see LogPsiLocalEnergy."""
    return _autograd_function().apply(g, lam, jas, R, r)
