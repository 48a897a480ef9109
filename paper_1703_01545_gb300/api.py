"""Python binding of the C ABI in include/afqmc.h (argument marshalling only).

The functions keep the C names.  Arrays may be numpy arrays (host) or torch
tensors (host or CUDA); every step of the method runs in the CUDA library.
``System`` and ``pair_delta_E`` are thin conveniences over the same calls.
"""
import ctypes

import numpy as np

from . import _lib

PHASELESS, FREE = 0, 1
FP64, BF16X3 = 0, 1


class AfqmcError(RuntimeError):
    pass


def _torch():
    try:
        import torch
        return torch
    except ImportError:  # pragma: no cover
        return None


def _ptr(a, kind="float64"):
    """Raw pointer of a C-contiguous numpy array or torch tensor whose elements are what the C
    side reads (``kind``: "float64", or "int32" for the alive flags), or None.  Any other
    element type is refused rather than reinterpreted."""
    if a is None:
        return None
    t = _torch()
    if t is not None and isinstance(a, t.Tensor):
        if not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        want = {"float64": t.float64, "int32": t.int32}[kind]
        if a.dtype != want:
            raise TypeError(f"tensor must be {kind}, not {a.dtype}")
        return ctypes.c_void_p(a.data_ptr())
    if isinstance(a, np.ndarray):
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        if a.dtype != np.dtype(kind):
            raise TypeError(f"array must be {kind}, not {a.dtype}")
        return ctypes.c_void_p(a.ctypes.data)
    raise TypeError(f"unsupported buffer type {type(a)}")


def _stream(stream=None):
    if stream is not None:
        return ctypes.c_void_p(int(stream))
    t = _torch()
    if t is not None and t.cuda.is_available():
        return ctypes.c_void_p(t.cuda.current_stream().cuda_stream)
    return ctypes.c_void_p(0)


def _check(code, handle=None, what=""):
    if code != 0:
        lib = _lib.load()
        msg = lib.afqmc_last_error(handle).decode() if handle else ""
        raise AfqmcError(f"{what}: {_lib.STATUS.get(code, code)} {msg}".strip())


def afqmc_default_options():
    o = _lib.AfqmcOptions()
    _lib.load().afqmc_default_options(ctypes.byref(o))
    return o


def afqmc_setup(h1, L, trial, M, X, n_up, n_dn, opt, stream=None):
    h = ctypes.c_void_p()
    code = _lib.load().afqmc_setup(ctypes.byref(h), _ptr(h1), _ptr(L), _ptr(trial), M, X, n_up,
                                   n_dn, ctypes.byref(opt), _stream(stream))
    _check(code, None, "afqmc_setup")
    return h


def afqmc_setup_multidet(h1, L, dets, coeffs, start, M, X, n_up, n_dn, opt, stream=None):
    h = ctypes.c_void_p()
    code = _lib.load().afqmc_setup_multidet(ctypes.byref(h), _ptr(h1), _ptr(L), _ptr(dets),
                                            _ptr(coeffs), len(coeffs), _ptr(start), M, X, n_up,
                                            n_dn, ctypes.byref(opt), _stream(stream))
    _check(code, None, "afqmc_setup_multidet")
    return h


def afqmc_destroy(h):
    _check(_lib.load().afqmc_destroy(h), None, "afqmc_destroy")


def afqmc_set_walkers(h, phi, w=None, stream=None):
    _check(_lib.load().afqmc_set_walkers(h, _ptr(phi), _ptr(w), _stream(stream)), h,
           "afqmc_set_walkers")


def afqmc_set_step(h, step, stream=None):
    _check(_lib.load().afqmc_set_step(h, int(step), _stream(stream)), h, "afqmc_set_step")


def afqmc_population_control(h, u, stream=None):
    u = np.ascontiguousarray(u, dtype=np.float64)
    _check(_lib.load().afqmc_population_control(h, _ptr(u), _stream(stream)), h,
           "afqmc_population_control")


def afqmc_seed_secondary(B, A, stream=None):
    _check(_lib.load().afqmc_seed_secondary(B, A, _stream(stream)), B, "afqmc_seed_secondary")


def afqmc_get_state(h, phi=None, logO=None, w=None, alive=None, stream=None):
    _check(_lib.load().afqmc_get_state(h, _ptr(phi), _ptr(logO), _ptr(w), _ptr(alive, "int32"),
                                       _stream(stream)), h, "afqmc_get_state")


def afqmc_get_info(h, stream=None):
    info = _lib.AfqmcInfo()
    _check(_lib.load().afqmc_get_info(h, ctypes.byref(info), _stream(stream)), h, "afqmc_get_info")
    return info


def afqmc_propagate(h, n_steps, fields=None, stream=None):
    _check(_lib.load().afqmc_propagate(h, int(n_steps), _ptr(fields), _stream(stream)), h,
           "afqmc_propagate")


def afqmc_orthonormalise(h, stream=None):
    _check(_lib.load().afqmc_orthonormalise(h, _stream(stream)), h, "afqmc_orthonormalise")


def afqmc_energy(h, e_local=None, e_mixed=None, w_sum=None, stream=None):
    _check(_lib.load().afqmc_energy(h, _ptr(e_local), _ptr(e_mixed), _ptr(w_sum), _stream(stream)),
           h, "afqmc_energy")


def afqmc_pair_delta_E(A, B, n_steps, energy_every, mgs_every, tau_eq, e_series=None,
                       dE_mean=None, dE_sigma=None, tau_at_min=None, stream=None,
                       raise_on_dead=True):
    """Returns the status code (0, or 3 = every walker of a system dead when
    raise_on_dead is False; the outputs are written in both cases)."""
    code = _lib.load().afqmc_pair_delta_E(A, B, int(n_steps), int(energy_every), int(mgs_every),
                                          float(tau_eq), _ptr(e_series), _ptr(dE_mean),
                                          _ptr(dE_sigma), _ptr(tau_at_min), _stream(stream))
    if code == 3 and not raise_on_dead:
        return code
    _check(code, A, "afqmc_pair_delta_E")
    return code


def afqmc_pair_graph_kernels(A):
    """Kernel launches in one measurement block of the pair graph cached on handle A."""
    n = ctypes.c_int(0)
    _check(_lib.load().afqmc_pair_graph_kernels(A, ctypes.byref(n)), A, "afqmc_pair_graph_kernels")
    return n.value


def afqmc_pair_run_form(A):
    """1: the pair graph cached on handle A runs a whole call as one graph launch (device-side
    loop over the measurement blocks); 0: one launch per block; -1: no graph cached."""
    f = ctypes.c_int(0)
    _check(_lib.load().afqmc_pair_run_form(A, ctypes.byref(f)), A, "afqmc_pair_run_form")
    return f.value


def afqmc_delta_E_stats(dE, taus, tau_eq):
    """Host statistics; returns (mean_tau, se_tau, (mean, se, tau_at_min))."""
    dE = np.ascontiguousarray(dE, dtype=np.float64)
    taus = np.ascontiguousarray(taus, dtype=np.float64)
    n, R = dE.shape
    mt, st, est = np.empty(n), np.empty(n), np.empty(3)
    code = _lib.load().afqmc_delta_E_stats(_ptr(dE), _ptr(taus), n, R, float(tau_eq), _ptr(mt),
                                           _ptr(st), _ptr(est))
    _check(code, None, "afqmc_delta_E_stats")
    return mt, st, tuple(est)


K_VHS, K_FORCE_BIAS, K_TAYLOR, K_EXCHANGE, K_OVERLAP, K_OVERLAP_UPDATE, K_MGS = 0, 1, 2, 3, 4, 5, 6
K_PAIR_LOOP = 7   # select_kernel only: pair run as one graph launch (1) or one per block (0)


def afqmc_time_kernel(h, which, reps, stream=None):
    ms = ctypes.c_double()
    _check(_lib.load().afqmc_time_kernel(h, int(which), int(reps), ctypes.byref(ms),
                                         _stream(stream)), h, "afqmc_time_kernel")
    return ms.value


def afqmc_reblock_error(series):
    s = np.ascontiguousarray(series, dtype=np.float64)
    return float(_lib.load().afqmc_reblock_error(_ptr(s), s.size))


class System:
    """One system (h1, L, trial) and its walker population on the current CUDA device."""

    def __init__(self, h1, L, trial, n_up, n_dn, dt=0.01, n_walkers=128, taylor_order=6,
                 mode=PHASELESS, n_repeats=1, seed=1, fb_cap=1.0, walker_offset=0,
                 precision=FP64, autotune=True, autotune_cache=None, independent_fields=False,
                 stream=None, dets=None, coeffs=None, start=None):
        """``dets`` [Nd, M, N] and ``coeffs`` [Nd] (with ``trial`` None) give a
        multi-determinant trial (afqmc_setup_multidet, FP64), ``start`` the walkers' first
        determinant [M, N]."""
        h1 = np.ascontiguousarray(h1, dtype=np.float64)
        L = np.ascontiguousarray(L, dtype=np.float64)
        if dets is not None:
            dets = np.ascontiguousarray(dets, dtype=np.float64)
            coeffs = np.ascontiguousarray(coeffs, dtype=np.float64)
            if start is not None:
                start = np.ascontiguousarray(start, dtype=np.float64)
            trial = dets[0]
        trial = np.ascontiguousarray(trial, dtype=np.float64)
        self.M, self.X = h1.shape[0], L.shape[0]
        self.n_up, self.n_dn, self.N = int(n_up), int(n_dn), int(n_up) + int(n_dn)
        self.n_walkers, self.n_repeats, self.dt = int(n_walkers), int(n_repeats), float(dt)
        o = afqmc_default_options()
        o.dt, o.n_walkers, o.taylor_order = float(dt), int(n_walkers), int(taylor_order)
        o.precision, o.mode, o.n_repeats = int(precision), int(mode), int(n_repeats)
        o.seed, o.fb_cap, o.walker_offset = int(seed), float(fb_cap), int(walker_offset)
        o.autotune = 1 if autotune else 0
        o.autotune_cache = autotune_cache.encode() if autotune_cache else None
        o.independent_fields = 1 if independent_fields else 0
        self.opt = o
        self.n_det = 0 if dets is None else len(coeffs)
        if dets is None:
            self.h = afqmc_setup(h1, L, trial, self.M, self.X, self.n_up, self.n_dn, o, stream)
        else:
            self.h = afqmc_setup_multidet(h1, L, dets, coeffs, start, self.M, self.X, self.n_up,
                                          self.n_dn, o, stream)

    def close(self):
        if self.h is not None:
            afqmc_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def info(self):
        return afqmc_get_info(self.h)

    def propagate(self, n_steps, fields=None):
        if isinstance(fields, np.ndarray):
            fields = np.ascontiguousarray(fields, dtype=np.float64)
        afqmc_propagate(self.h, n_steps, fields)

    def orthonormalise(self):
        afqmc_orthonormalise(self.h)

    def energy(self):
        """(E_L complex [Nw], E_mixed [R], sum w [R]) as numpy arrays."""
        el = np.empty(2 * self.n_walkers)
        em = np.empty(self.n_repeats)
        ws = np.empty(self.n_repeats)
        afqmc_energy(self.h, el, em, ws)
        return el[:self.n_walkers] + 1j * el[self.n_walkers:], em, ws

    def state(self):
        nw, M, N = self.n_walkers, self.M, self.N
        phi = np.empty(2 * nw * M * N)
        lo = np.empty(2 * nw)
        w = np.empty(2 * nw)
        al = np.empty(nw, dtype=np.int32)
        afqmc_get_state(self.h, phi, lo, w, al)
        phi = phi.reshape(2, nw, M, N)
        return dict(phi=phi[0] + 1j * phi[1], logO=lo[:nw] + 1j * lo[nw:],
                    w=w[:nw] + 1j * w[nw:], alive=al.astype(bool))

    def set_tangent(self, P):
        """Tangent mode along h1 -> h1 + lambda P (None switches it off)."""
        Pm = None if P is None else np.ascontiguousarray(P, dtype=np.float64)
        _check(_lib.load().afqmc_set_tangent(self.h, _ptr(Pm), _stream(None)), self.h,
               "afqmc_set_tangent")

    def energy_tangent(self):
        """(E_mixed [R], dE_mixed/dlambda [R], dE_L/dlambda [Nw] complex)."""
        de = np.empty(2 * self.n_walkers)
        em, dm = np.empty(self.n_repeats), np.empty(self.n_repeats)
        _check(_lib.load().afqmc_energy_tangent(self.h, _ptr(de), _ptr(em), _ptr(dm),
                                                _stream(None)), self.h, "afqmc_energy_tangent")
        return em, dm, de[:self.n_walkers] + 1j * de[self.n_walkers:]

    def tangent_state(self):
        d = np.empty(self.n_walkers)
        _check(_lib.load().afqmc_get_tangent_state(self.h, _ptr(d), _stream(None)), self.h,
               "afqmc_get_tangent_state")
        return d

    def select_kernel(self, which, variant):
        """Fix a tunable kernel's variant (K_EXCHANGE: 0 tensor cores, 2/4/8 FP32 walkers per
        CTA; K_TAYLOR: 0 L1, 1 shared memory), overriding the autotuner; K_PAIR_LOOP (either
        precision): 1 one graph launch per pair run, 0 one launch per measurement block."""
        _check(_lib.load().afqmc_select_kernel(self.h, int(which), int(variant)), self.h,
               "afqmc_select_kernel")

    def adjoint_run(self, n_steps, fields=None, mgs_every=5, energy_every=5, checkpoint=0):
        """(E, dE/dh1 [M, M]) of an n_steps FP64 run by the library's reverse mode: E is the
        mean over the measurements (every energy_every steps) of sum w Re E_L / sum w, the
        gradient takes the M^2 entries of h1 as independent.  checkpoint=0 picks about
        sqrt(n_steps) steps per checkpoint segment.  The walkers end after the run."""
        if checkpoint <= 0:
            checkpoint = max(1, int(round(np.sqrt(n_steps))))
        fp = None
        if fields is not None:
            fp = np.ascontiguousarray(fields, dtype=np.float64)
        e = np.empty(1)
        g = np.empty((self.M, self.M))
        _check(_lib.load().afqmc_adjoint_run(self.h, int(n_steps), _ptr(fp), int(mgs_every),
                                             int(energy_every), int(checkpoint), _ptr(e), _ptr(g),
                                             _stream(None)), self.h, "afqmc_adjoint_run")
        return float(e[0]), g

    def population_control(self, u):
        """Comb each repeat's walkers (Sec. II.C); u [n_repeats] uniforms in [0, 1)."""
        u = np.asarray(u, dtype=np.float64)
        if u.shape != (self.n_repeats,):
            raise ValueError(f"need one uniform per repeat ({self.n_repeats})")
        afqmc_population_control(self.h, u)

    def seed_from(self, primary):
        """Start this (secondary) system from the walkers of an equilibrated primary system
        (Sec. II.C), weights rescaled to this system's trial; the step counter follows."""
        afqmc_seed_secondary(self.h, primary.h)

    def checkpoint(self):
        """Resumable state (walkers, weights, step counter and the run's identity); best
        taken right after orthonormalise(). checkpoint.save / load write and read it."""
        from . import checkpoint
        st = self.state()
        return checkpoint.make(self, st["phi"], st["w"], self.info().step)

    def resume(self, ck):
        """Continue from a checkpoint of a run with the same Hamiltonian and options: its
        walkers and weights, and the step counter of the field stream."""
        from . import checkpoint
        checkpoint.check(ck, self)
        self.set_walkers(ck["phi"], ck["w"])
        afqmc_set_step(self.h, int(ck["step"]))

    def set_walkers(self, phi, w=None):
        phi = np.asarray(phi)
        p = np.ascontiguousarray(np.stack([phi.real, phi.imag]), dtype=np.float64)
        wp = None
        if w is not None:
            w = np.asarray(w)
            wp = np.ascontiguousarray(np.stack([w.real, w.imag]), dtype=np.float64)
        afqmc_set_walkers(self.h, p, wp)


def pair_graph_kernels(A: System):
    """Kernel launches per measurement block of the last pair run with A as its first system."""
    return afqmc_pair_graph_kernels(A.h)


def pair_run_form(A: System):
    """1 when the last pair run with A as its first system was one graph launch, 0 when it
    launched the block graph once per measurement block."""
    return afqmc_pair_run_form(A.h)


def pair_delta_E(A: System, B: System, n_steps, energy_every=5, mgs_every=5, tau_eq=0.0,
                 raise_on_dead=True):
    """Correlated pair run; returns dict(E [n_meas, 2, R], dE_mean, dE_sigma, tau_at_min,
    all_dead).  With raise_on_dead=False a run in which every walker of a system died
    returns its (NaN-bearing) results with all_dead=True instead of raising."""
    R = A.n_repeats
    n_meas = n_steps // energy_every
    es = np.empty(max(1, n_meas * 2 * R))
    m, s, t = np.empty(1), np.empty(1), np.empty(1)
    code = afqmc_pair_delta_E(A.h, B.h, n_steps, energy_every, mgs_every, tau_eq, es, m, s, t,
                              raise_on_dead=raise_on_dead)
    return dict(E=es[:n_meas * 2 * R].reshape(n_meas, 2, R), dE_mean=float(m[0]),
                dE_sigma=float(s[0]), tau_at_min=float(t[0]), all_dead=code == 3,
                taus=np.arange(1, n_meas + 1) * energy_every * A.dt)
