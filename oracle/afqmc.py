"""Correlated-sampling phaseless AFQMC, one step at a time (oracle side, FP64).

Notation follows Sec. II.A-B of the paper.  A walker is a Slater determinant
Phi [M, N] (complex; columns 0..N_up-1 spin up, N_up..N-1 spin down) with a
weight w and the log of its overlap with the trial, log O = log <psi_T|phi>.
The trial psi_T is the real M x N matrix [Psi_up | Psi_dn].

Definitions used throughout
  O_s     = Psi_s^T Phi_s,   Theta_s = Phi_s O_s^{-1}
  G_s[i,j] = <psi_T| c+_i c_j |phi> / <psi_T|phi> = (Theta_s Psi_s^T)[j, i]
  rho_g   = sum_ik L^g_ik sum_s c+_is c_ks          (so v_g = i rho_g, Sec. II.A)
  <rho_g>_T = sum_s tr(L_g Psi_s Psi_s^T)           (trial expectation, Eq. 2)
  rhobar_g  = sum_s tr(L_g G_s)                      (so vbar_g = i rhobar_g, Eq. 9)

Normal-ordering Eq. 1 with V_ijkl = sum_g L^g_ik L^g_jl and expanding Eq. 2
gives H = H_1 + H_2 with the one-body part
  H_1 = sum_ij K_ij sum_s c+_is c_js + C,
  K = h1 - 1/2 sum_g L_g L_g + sum_g <rho_g>_T L_g,   C = -1/2 sum_g <rho_g>_T^2.

One step (Eqs. 3-5, 8-9 and the hybrid weight of Sec. II.D), per live walker:
  1. xbar_g = -sqrt(dt) (vbar_g - <v_g>) = -i sqrt(dt) (rhobar_g - <rho_g>_T)   (Eq. 9)
     optionally capped: |xbar_g| > cap  ->  xbar_g * cap / |xbar_g|
  2. c_g = x_g - xbar_g;  A = i sqrt(dt) sum_g c_g L_g  (one-body matrix of Eq. 11's
     middle factor); its scalar part s = exp(-i sqrt(dt) sum_g c_g <rho_g>_T)
  3. Phi' = e^{-dt K/2} T_n(A) e^{-dt K/2} Phi,  T_n(A) = sum_{m<=n} A^m / m!
     (Eq. 3 split, Eq. 5 read with a half step on each side, Thouless theorem)
  4. R = s * O(Phi') / O(Phi)  (overlap ratio of the propagated walker)
     I = R * exp(x.xbar - xbar.xbar/2) * exp(-dt (C - E_T))   (hybrid weight, Sec. II.D;
     squares unconjugated)
  5. phaseless: dtheta = arg R,  w <- w |I| max(0, cos dtheta)  (Sec. II.A); w <= 0 kills
     the walker for good, it is no longer propagated (Sec. II.B).
     free projection: xbar = 0 and w <- w I (complex).
Every ``mgs_every`` steps each spin block is replaced by its modified
Gram-Schmidt Q factor (Sec. II.D) and log O recomputed.
Energy (Eqs. 6-7, 10): E_L = sum_s tr(h1 G_s)
      + 1/2 sum_g [ rhobar_g^2 - sum_s tr(L_g G_s L_g G_s) ],
  E = sum_k w_k Re E_L,k / sum_k w_k  (phaseless);  Re(sum w E_L / sum w) (free).

Multi-determinant trial (Sec. II.D; the truncated CASSCF expansions of Sec. III):
psi_T = sum_d c_d D_d with real M x N determinants D_d.  Every mixed quantity of the
walker is a sum over the determinants, weighted by their share of the overlap:
  O_d = <D_d|phi>,  <psi_T|phi> = sum_d c_d O_d,  w_d = c_d O_d / <psi_T|phi>
  G = sum_d w_d G_d            (G_d: the Green's function above with trial D_d)
  E_L = sum_d w_d E_L,d        (<D_d|H|phi> = O_d E_L,d; E_L,d with trial D_d)
and the force bias takes rhobar from this G.  G_d and E_L,d need O_d != 0; a walker
orthogonal to a determinant of the expansion (as a walker sitting on one determinant of an
orthonormal expansion is to all the others) would need cofactor formulas instead, so the
walkers start from a determinant outside the expansion (the paper starts them from ROHF
determinants while the trial is built on CASSCF orbitals), and a determinant with O_d = 0
contributes nothing.  The mean-field background <rho_g>_T, the one-body operator K and
the energy shift E_T are those of the first determinant D_0 (any constant background is
exact under the force-bias reweighting, and E_T cancels in every mixed estimate).
"""
import numpy as np

from .philox import gaussian_fields

PHASELESS = "phaseless"
FREE = "free"


class System:
    """Static data of one system: h1, L, trial, and the derived K, e^{-dt K/2}, C, E_T."""

    def __init__(self, h1, L, trial, n_up, n_dn, dt, fb_cap=1.0, mode=PHASELESS,
                 taylor_order=6, dets=None, coeffs=None, start=None):
        """``dets`` [Nd, M, N] and ``coeffs`` [Nd] give a multi-determinant trial (``trial``
        is then ignored: the first determinant takes its role for <rho>_T, K and E_T) and
        ``start`` the walkers' initial determinant (default: the trial)."""
        if dets is not None:
            trial = np.asarray(dets, dtype=np.float64)[0]
        self.h1 = np.asarray(h1, dtype=np.float64)
        self.L = np.asarray(L, dtype=np.float64)
        self.trial = np.asarray(trial, dtype=np.float64)
        self.M = self.h1.shape[0]
        self.X = self.L.shape[0]
        self.n_up, self.n_dn = int(n_up), int(n_dn)
        self.N = self.n_up + self.n_dn
        self.dt = float(dt)
        self.sqrt_dt = np.sqrt(self.dt)
        self.fb_cap = float(fb_cap)
        self.mode = mode
        self.taylor_order = int(taylor_order)
        self.spins = [(0, self.n_up), (self.n_up, self.N)]
        # <rho_g>_T = sum_s tr(L_g P_s)  with P_s = Psi_s Psi_s^T
        self.rho_mf = np.zeros(self.X)
        for a, b in self.spins:
            P = self.trial[:, a:b] @ self.trial[:, a:b].T
            self.rho_mf += np.einsum("gij,ji->g", self.L, P)
        # one-body part of H = H_1 + H_2 (normal ordering of Eq. 1, expansion of Eq. 2)
        self.K = (self.h1 - 0.5 * np.einsum("gik,gkj->ij", self.L, self.L)
                  + np.einsum("g,gij->ij", self.rho_mf, self.L))
        self.C = -0.5 * float(self.rho_mf @ self.rho_mf)
        lam, U = np.linalg.eigh(self.K)
        self.expK = (U * np.exp(-0.5 * self.dt * lam)) @ U.T
        # trial energy E_T = E_L(psi_T): the energy shift of exp(dt (E_T - H))
        self.dets = None
        self.E_T = float(local_energy(self, self.trial[None].astype(np.complex128))[0].real)
        self.start = self.trial if start is None else np.asarray(start, dtype=np.float64)
        if dets is not None:
            self.dets = np.asarray(dets, dtype=np.float64)
            self.coeffs = np.asarray(coeffs, dtype=np.float64)
            if self.dets.shape[1:] != (self.M, self.N) or self.coeffs.shape != self.dets.shape[:1]:
                raise ValueError("dets [Nd, M, N] and coeffs [Nd] expected")


class Walkers:
    """Walker population: Phi [Nw, M, N] complex, w complex, log O complex, alive bool."""

    def __init__(self, sys: System, n_walkers: int, phi=None, w=None):
        if phi is None:
            phi = np.broadcast_to(sys.start, (n_walkers, sys.M, sys.N))
        self.phi = np.array(phi, dtype=np.complex128)
        self.w = np.ones(n_walkers, dtype=np.complex128) if w is None else np.array(w, np.complex128)
        self.logO = overlap(sys, self.phi)
        self.alive = np.ones(n_walkers, dtype=bool) if w is None else (np.abs(self.w) > 0)

    def copy(self):
        c = object.__new__(Walkers)
        c.phi, c.w, c.logO, c.alive = self.phi.copy(), self.w.copy(), self.logO.copy(), self.alive.copy()
        return c


def det_overlap(sys: System, trial, phi):
    """log <D|phi> = sum_s log det(D_s^T Phi_s) for one determinant D = trial  (Cauchy-Binet)."""
    logO = np.zeros(phi.shape[0], dtype=np.complex128)
    for a, b in sys.spins:
        if b == a:
            continue
        O = np.einsum("ia,wib->wab", trial[:, a:b], phi[:, :, a:b])
        sign, lad = np.linalg.slogdet(O)
        logO += lad + np.log(sign.astype(np.complex128))
    return logO


def det_green(sys: System, trial, phi):
    """Green's functions G_s [Nw, M, M] of the walkers with one determinant D = trial,
    G_s[i,j] = <D| c+_i c_j |phi> / <D|phi>, for s = up, down."""
    out = []
    for a, b in sys.spins:
        if b == a:
            out.append(np.zeros((phi.shape[0], sys.M, sys.M), dtype=np.complex128))
            continue
        Psi = trial[:, a:b]
        O = np.einsum("ia,wib->wab", Psi, phi[:, :, a:b])
        Theta = phi[:, :, a:b] @ np.linalg.inv(O)
        out.append(np.swapaxes(Theta @ Psi.T, 1, 2))
    return out


def det_shares(sys: System, phi):
    """Multi-determinant trial: (log <psi_T|phi> [Nw], w [Nd, Nw]) with w_d = c_d O_d /
    <psi_T|phi>; the sum is taken relative to the largest |O_d| of each walker."""
    logO = np.array([det_overlap(sys, D, phi) for D in sys.dets])          # [Nd, Nw]
    top = np.max(logO.real, axis=0)
    t = sys.coeffs[:, None] * np.exp(logO - top[None, :])
    total = np.sum(t, axis=0)
    return top + np.log(total), t / total[None, :]


def overlap(sys: System, phi):
    """log <psi_T|phi>: one determinant, or sum_d c_d <D_d|phi> for a multi-determinant trial."""
    if sys.dets is None:
        return det_overlap(sys, sys.trial, phi)
    return det_shares(sys, phi)[0]


def green(sys: System, phi):
    """Mixed Green's functions G_s [Nw, M, M], G_s[i,j] = <psi_T|c+_i c_j|phi>/<psi_T|phi>,
    for s = up, down; for a multi-determinant trial sum_d w_d G_d (O_d = 0: no contribution)."""
    if sys.dets is None:
        return det_green(sys, sys.trial, phi)
    _, w = det_shares(sys, phi)
    out = [np.zeros((phi.shape[0], sys.M, sys.M), dtype=np.complex128) for _ in sys.spins]
    for D, wd in zip(sys.dets, w):
        use = wd != 0
        if not np.any(use):
            continue
        for si, Gs in enumerate(det_green(sys, D, phi[use])):
            out[si][use] += wd[use, None, None] * Gs
    return out


def rhobar(sys: System, G):
    """rhobar_g = sum_s tr(L_g G_s) = sum_s sum_ij L^g_ij G_s[j, i]  [Nw, X]  (vbar_g = i rhobar_g, Eq. 9)."""
    Lf = sys.L.reshape(sys.X, sys.M * sys.M)
    out = 0
    for Gs in G:
        GT = np.swapaxes(Gs, 1, 2).reshape(Gs.shape[0], sys.M * sys.M)
        out = out + GT @ Lf.T
    return out


def force_bias(sys: System, G):
    """Optimal force bias of Eq. 9, xbar_g = -i sqrt(dt) (rhobar_g - <rho_g>_T), with the cap."""
    xbar = -1j * sys.sqrt_dt * (rhobar(sys, G) - sys.rho_mf[None, :])
    if sys.fb_cap > 0:
        mag = np.abs(xbar)
        big = mag > sys.fb_cap
        xbar = np.where(big, xbar * (sys.fb_cap / np.where(big, mag, 1.0)), xbar)
    return xbar


def taylor_apply(A, phi, order):
    """T_order(A) phi = sum_{m=0}^{order} A^m phi / m!, by repeated products."""
    term = phi
    acc = phi.copy()
    for m in range(1, order + 1):
        term = (A @ term) / m
        acc = acc + term
    return acc


def step_determinant(sys: System, phi, logO, x, xbar):
    """One application of Eq. 11 with fields x and shift xbar to determinants phi.

    Returns (Phi', log O', log R, log I): R is the overlap ratio including the scalar
    part s of the shifted HS exponential, I the hybrid weight factor of Sec. II.D.
    """
    c = x - xbar
    A = 1j * sys.sqrt_dt * (c @ sys.L.reshape(sys.X, sys.M * sys.M)).reshape(-1, sys.M, sys.M)
    log_s = -1j * sys.sqrt_dt * (c @ sys.rho_mf)
    phi1 = sys.expK @ phi
    phi2 = taylor_apply(A, phi1, sys.taylor_order)
    phi3 = sys.expK @ phi2
    logO_new = overlap(sys, phi3)
    logR = log_s + logO_new - logO
    logI = logR + np.sum(x * xbar, axis=1) - 0.5 * np.sum(xbar * xbar, axis=1) \
        - sys.dt * (sys.C - sys.E_T)
    return phi3, logO_new, logR, logI


def propagate(sys: System, wk: Walkers, x):
    """Advance every live walker by one step with fields x [Nw, X] (float64)."""
    live = wk.alive
    if not np.any(live):
        return
    phi = wk.phi[live]
    xs = np.asarray(x, dtype=np.float64)[live]
    if sys.mode == PHASELESS:
        xbar = force_bias(sys, green(sys, phi))
    else:
        xbar = np.zeros_like(xs, dtype=np.complex128)
    phi3, logO_new, logR, logI = step_determinant(sys, phi, wk.logO[live], xs, xbar)
    if sys.mode == PHASELESS:
        dtheta = logR.imag
        w_new = wk.w[live].real * np.exp(logI.real) * np.maximum(0.0, np.cos(dtheta))
        w_new = w_new.astype(np.complex128)
        still = w_new.real > 0
    else:
        w_new = wk.w[live] * np.exp(logI)
        still = np.ones(w_new.shape, dtype=bool)
    idx = np.nonzero(live)[0]
    wk.phi[idx] = phi3
    wk.logO[idx] = logO_new
    wk.w[idx] = np.where(still, w_new, 0.0)
    wk.alive[idx] = still


def modified_gram_schmidt(phi_s):
    """Column-by-column MGS of phi_s [Nw, M, n]: returns Q with orthonormal columns."""
    Q = np.array(phi_s, dtype=np.complex128)
    for j in range(Q.shape[2]):
        v = Q[:, :, j]
        for i in range(j):
            r = np.sum(np.conj(Q[:, :, i]) * v, axis=1)
            v = v - r[:, None] * Q[:, :, i]
        nrm = np.sqrt(np.sum(np.abs(v) ** 2, axis=1))
        Q[:, :, j] = v / nrm[:, None]
    return Q


def orthonormalise(sys: System, wk: Walkers):
    """Replace each spin block of every live walker by its MGS Q factor; recompute log O."""
    live = wk.alive
    if not np.any(live):
        return
    idx = np.nonzero(live)[0]
    phi = wk.phi[idx]
    for a, b in sys.spins:
        if b > a:
            phi[:, :, a:b] = modified_gram_schmidt(phi[:, :, a:b])
    wk.phi[idx] = phi
    wk.logO[idx] = overlap(sys, phi)


def energy_from_green(sys: System, G):
    """E_L of walkers with single-determinant Green's functions G (Eq. 7 with Wick's theorem):
    sum_s tr(h1 G_s) + 1/2 sum_g [ (sum_s tr L_g G_s)^2 - sum_s tr(L_g G_s L_g G_s) ]."""
    e1 = sum(np.einsum("ij,wji->w", sys.h1, Gs) for Gs in G)
    rb = rhobar(sys, G)
    exch = 0.0
    for Gs in G:
        LG = sys.L[None, :, :, :] @ Gs[:, None, :, :]          # [w, g, M, M] = L_g G_s
        exch = exch + np.einsum("wgik,wgki->wg", LG, LG)
    return e1 + 0.5 * np.sum(rb * rb - exch, axis=1)


def local_energy(sys: System, phi, chunk: int = 0):
    """E_L [Nw] complex (Eq. 7 with Wick's theorem); for a multi-determinant trial
    sum_d w_d E_L,d, the two-body part taken per determinant (it is not linear in G)."""
    nw = phi.shape[0]
    if chunk <= 0:
        chunk = max(1, int(4e6 // max(1, sys.X * sys.M * sys.M)))
    out = np.empty(nw, dtype=np.complex128)
    for s0 in range(0, nw, chunk):
        p = phi[s0:s0 + chunk]
        if sys.dets is None:
            out[s0:s0 + chunk] = energy_from_green(sys, det_green(sys, sys.trial, p))
            continue
        _, w = det_shares(sys, p)
        acc = np.zeros(p.shape[0], dtype=np.complex128)
        for D, wd in zip(sys.dets, w):
            use = wd != 0
            if np.any(use):
                acc[use] += wd[use] * energy_from_green(sys, det_green(sys, D, p[use]))
        out[s0:s0 + chunk] = acc
    return out


def repeat_groups(n_walkers: int, n_repeats: int):
    """Repeat index of each global walker index k: floor(k R / Nw)."""
    return (np.arange(n_walkers) * n_repeats) // n_walkers


def mixed_energy(sys: System, w, eloc, groups, n_repeats):
    """Per-repeat mixed estimate sum w E_L / sum w (Eq. 7; Re E_L for phaseless, Eq. 10).
    The sums run over the walkers with w != 0: a dead walker contributes nothing, even when its
    local energy is not finite (a walker killed for a non-finite overlap)."""
    E = np.empty(n_repeats)
    W = np.empty(n_repeats)
    for r in range(n_repeats):
        m = (groups == r) & (w != 0)
        if sys.mode == PHASELESS:
            num = np.sum(w[m].real * eloc[m].real)
            den = np.sum(w[m].real)
            E[r] = num / den if den != 0 else np.nan
            W[r] = den
        else:
            den = np.sum(w[m])
            E[r] = (np.sum(w[m] * eloc[m]) / den).real
            W[r] = den.real
    return E, W


def run_pair(sysA: System, sysB: System, n_walkers: int, n_steps: int, seed: int,
             energy_every: int = 5, mgs_every: int = 5, n_repeats: int = 1,
             walker_index=None, fields=None, record_walkers=False, seed_B=None,
             walkers=None, t0: int = 0):
    """Correlated pair run (Sec. II.B): walker k of A and walker k of B share x_{t,k,g}.

    ``seed_B`` (optional) gives B its own key instead: the two systems then draw
    independent fields, the uncorrelated sampling that Sec. III compares against.
    ``walkers`` (optional) continues given populations, one per system, instead of starting
    from the trials, and ``t0`` is the step index of the first field drawn (the fields of
    step t0 + t; the Gram-Schmidt and measurement schedule counts from the start of the call).

    ``walker_index`` (default 0..Nw-1) gives the global pair index k of every walker
    propagated here, so a subset of a large population can be followed exactly.
    ``fields`` (optional) is an explicit [n_steps, Nw, max(X_A, X_B)] array used in
    place of the counter-based stream.  Returns dict with per-measurement per-repeat
    mixed energies for both systems and (optionally) per-walker records.
    Order within a step boundary: propagate, then MGS, then measure.
    """
    keyed = [(s, sd) for s, sd in ((sysA, seed), (sysB, seed if seed_B is None else seed_B))
             if s is not None]
    systems = [s for s, _ in keyed]
    seeds = [sd for _, sd in keyed]
    k = np.arange(n_walkers) if walker_index is None else np.asarray(walker_index)
    groups = repeat_groups(n_walkers, n_repeats)[k] if walker_index is None else \
        (k * n_repeats) // n_walkers
    wks = [Walkers(s, k.size) for s in systems] if walkers is None else \
        [w for w in walkers if w is not None]
    out = dict(steps=[], E=[[] for _ in systems], W=[[] for _ in systems],
               records=[[] for _ in systems])
    for t in range(n_steps):
        for s, wk, sd in zip(systems, wks, seeds):
            if fields is None:
                x = gaussian_fields(sd, t0 + t, k, s.X)
            else:
                x = fields[t][:, :s.X]
            propagate(s, wk, x)
        if mgs_every > 0 and (t + 1) % mgs_every == 0:
            for s, wk in zip(systems, wks):
                orthonormalise(s, wk)
        if energy_every > 0 and (t + 1) % energy_every == 0:
            out["steps"].append(t + 1)
            for i, (s, wk) in enumerate(zip(systems, wks)):
                el = local_energy(s, wk.phi)
                E, W = mixed_energy(s, wk.w, el, groups, n_repeats)
                out["E"][i].append(E)
                out["W"][i].append(W)
                if record_walkers:
                    out["records"][i].append(dict(eloc=el, w=wk.w.copy(), logO=wk.logO.copy()))
    out["E"] = [np.array(e) for e in out["E"]]
    out["W"] = [np.array(e) for e in out["W"]]
    out["walkers"] = wks
    return out
