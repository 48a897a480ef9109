"""Directional derivative of the mixed energy along a one-body perturbation (oracle side).

h1 -> h1 + lambda P (P symmetric), fields and trial held fixed.  Every quantity of a step
(Sec. II.A-B, II.D) is differentiated in the forward direction ("tangent mode"):

  K = h1 + ...            dK = P
  E = exp(-dt K/2)        dE = Frechet derivative of exp at -dt K/2 along -dt P/2
                               (upper-right block of exp([[B, dB], [0, B]]))
  Phi1 = E Phi            dPhi1 = dE Phi + E dPhi
  T_n = A T_{n-1}/n       dT_n = (dA T_{n-1} + A dT_{n-1})/n,  Phi2 = sum T_n
  Phi' = E Phi2           dPhi' = dE Phi2 + E dPhi2
  O = Psi^T Phi           dlog O = sum_s tr(O_s^{-1} Psi_s^T dPhi_s)
  G_s = (Theta Psi^T)^T   dTheta_s = (dPhi_s - Theta_s Psi_s^T dPhi_s) O_s^{-1}
  rhobar_g = tr(L_g G)    drhobar_g = sum_s tr(L_g dG_s)
  xbar = -i sqrt(dt)(rhobar - <rho>)    dxbar = -i sqrt(dt) drhobar  (through the cap)
  c = x - xbar, dc = -dxbar;  dA = i sqrt(dt) sum_g dc_g L_g
  log s = -i sqrt(dt) sum_g c_g <rho_g>   dlog s = -i sqrt(dt) sum_g dc_g <rho_g>
  log I = log s + log O' - log O + x.xbar - xbar.xbar/2 - dt (C - E_T)
          dlog I = dlog s + dlog O' - dlog O + (x - xbar).dxbar + dt dE_T
  phaseless: log w += Re log I + log cos(arg R)
             dlog w += Re dlog I - tan(arg R) Im(dlog s + dlog O' - dlog O)  (cos > 0)
  MGS: Q = Phi R^{-1}; every later quantity is invariant under Phi -> Phi M (M invertible,
       per spin), so the tangent is carried as dQ = dPhi R^{-1} with R held fixed.
  E_L = sum_s tr(h1 G_s) + 1/2 sum_g [rhobar_g^2 - sum_s tr(L_g G_s L_g G_s)]
  dE_L = sum_s [tr(P G_s) + tr(h1 dG_s)] + sum_g [rhobar_g drhobar_g - sum_s tr(L_g G_s L_g dG_s)]
  E = sum w Re E_L / sum w   dE = [sum (dw Re E_L + w Re dE_L) - E sum dw] / sum w,  dw = w dlog w
The cos cut and the force-bias cap are differentiated piecewise (a walker that crosses
either between lambda +- eps is where finite differences and the tangent part ways).
"""
import numpy as np
from scipy.linalg import expm

from . import afqmc


def frechet_exp(B, dB):
    """(exp(B), d/de exp(B + e dB) at 0) from the 2x2 block-matrix identity."""
    M = B.shape[0]
    Z = np.zeros((2 * M, 2 * M))
    Z[:M, :M] = B
    Z[M:, M:] = B
    Z[:M, M:] = dB
    F = expm(Z)
    return F[:M, :M], F[:M, M:]


class TangentSystem:
    def __init__(self, sys: afqmc.System, P):
        self.s = sys
        self.P = np.asarray(P, dtype=np.float64)
        B = -0.5 * sys.dt * sys.K
        _, self.dE = frechet_exp(B, -0.5 * sys.dt * self.P)
        # trial energy derivative: E_T = E_L(psi_T) is linear in h1 through tr(h1 P_s)
        self.dE_T = 0.0
        for a, b in sys.spins:
            Ps = sys.trial[:, a:b] @ sys.trial[:, a:b].T
            self.dE_T += float(np.sum(self.P * Ps))


class TangentWalkers:
    def __init__(self, wk: afqmc.Walkers):
        self.dphi = np.zeros_like(wk.phi)
        self.dlogw = np.zeros(wk.phi.shape[0])


def _green_and_tangent(sys, phi, dphi):
    """(G_s, dG_s, dlog O) for both spins."""
    G, dG = [], []
    dlogO = np.zeros(phi.shape[0], dtype=np.complex128)
    for a, b in sys.spins:
        if b == a:
            z = np.zeros((phi.shape[0], sys.M, sys.M), dtype=np.complex128)
            G.append(z)
            dG.append(z.copy())
            continue
        Psi = sys.trial[:, a:b]
        O = np.einsum("ia,wib->wab", Psi, phi[:, :, a:b])
        dO = np.einsum("ia,wib->wab", Psi, dphi[:, :, a:b])
        Oi = np.linalg.inv(O)
        Theta = phi[:, :, a:b] @ Oi
        dTheta = (dphi[:, :, a:b] - Theta @ dO) @ Oi
        dlogO += np.einsum("wab,wba->w", Oi, dO)
        G.append(np.swapaxes(Theta @ Psi.T, 1, 2))
        dG.append(np.swapaxes(dTheta @ Psi.T, 1, 2))
    return G, dG, dlogO


def _capped_xbar(sys, G, dG):
    raw = -1j * sys.sqrt_dt * (afqmc.rhobar(sys, G) - sys.rho_mf[None, :])
    draw = -1j * sys.sqrt_dt * afqmc.rhobar(sys, dG)
    if sys.fb_cap <= 0:
        return raw, draw
    mag = np.abs(raw)
    big = mag > sys.fb_cap
    safe = np.where(big, mag, 1.0)
    # d (cap x / |x|) = cap (dx / |x| - x Re(conj(x) dx) / |x|^3)
    dcap = sys.fb_cap * (draw / safe - raw * np.real(np.conj(raw) * draw) / safe ** 3)
    return np.where(big, raw * (sys.fb_cap / safe), raw), np.where(big, dcap, draw)


def propagate(ts: TangentSystem, wk: afqmc.Walkers, tw: TangentWalkers, x):
    """One step of the walkers and their tangents (phaseless mode)."""
    sys = ts.s
    live = wk.alive
    if not np.any(live):
        return
    idx = np.nonzero(live)[0]
    phi, dphi = wk.phi[idx], tw.dphi[idx]
    xs = np.asarray(x, dtype=np.float64)[idx]
    G, dG, dlogO_old = _green_and_tangent(sys, phi, dphi)
    xbar, dxbar = _capped_xbar(sys, G, dG)
    c, dc = xs - xbar, -dxbar
    Lf = sys.L.reshape(sys.X, sys.M * sys.M)
    A = 1j * sys.sqrt_dt * (c @ Lf).reshape(-1, sys.M, sys.M)
    dA = 1j * sys.sqrt_dt * (dc @ Lf).reshape(-1, sys.M, sys.M)
    log_s = -1j * sys.sqrt_dt * (c @ sys.rho_mf)
    dlog_s = -1j * sys.sqrt_dt * (dc @ sys.rho_mf)
    E, dE = sys.expK, ts.dE
    phi1 = E @ phi
    dphi1 = dE @ phi + E @ dphi
    T, dT = phi1, dphi1
    phi2, dphi2 = phi1.copy(), dphi1.copy()
    for n in range(1, sys.taylor_order + 1):
        T, dT = (A @ T) / n, (dA @ T + A @ dT) / n
        phi2 = phi2 + T
        dphi2 = dphi2 + dT
    phi3 = E @ phi2
    dphi3 = dE @ phi2 + E @ dphi2
    logO_new = afqmc.overlap(sys, phi3)
    _, _, dlogO_new = _green_and_tangent(sys, phi3, dphi3)
    logR = log_s + logO_new - wk.logO[idx]
    dlogR = dlog_s + dlogO_new - dlogO_old
    logI = logR + np.sum(xs * xbar, axis=1) - 0.5 * np.sum(xbar * xbar, axis=1) \
        - sys.dt * (sys.C - sys.E_T)
    dlogI = dlogR + np.sum((xs - xbar) * dxbar, axis=1) + sys.dt * ts.dE_T
    cosv = np.cos(logR.imag)
    w_new = wk.w[idx].real * np.exp(logI.real) * np.maximum(0.0, cosv)
    still = w_new > 0
    tanv = np.where(still, np.tan(logR.imag), 0.0)
    tw.dlogw[idx] = np.where(still, tw.dlogw[idx] + dlogI.real - tanv * dlogR.imag, 0.0)
    wk.phi[idx] = phi3
    tw.dphi[idx] = dphi3
    wk.logO[idx] = logO_new
    wk.w[idx] = np.where(still, w_new, 0.0).astype(np.complex128)
    wk.alive[idx] = still


def orthonormalise(sys: afqmc.System, wk: afqmc.Walkers, tw: TangentWalkers):
    """MGS of the walkers; tangents transformed by the same column operations (dPhi R^{-1})."""
    live = wk.alive
    if not np.any(live):
        return
    idx = np.nonzero(live)[0]
    phi, dphi = wk.phi[idx], tw.dphi[idx]
    for a, b in sys.spins:
        if b == a:
            continue
        Q = afqmc.modified_gram_schmidt(phi[:, :, a:b])
        R = np.conj(np.swapaxes(Q, 1, 2)) @ phi[:, :, a:b]       # upper triangular
        dphi[:, :, a:b] = dphi[:, :, a:b] @ np.linalg.inv(np.triu(R))
        phi[:, :, a:b] = Q
    wk.phi[idx] = phi
    tw.dphi[idx] = dphi
    wk.logO[idx] = afqmc.overlap(sys, phi)


def local_energy_tangent(ts: TangentSystem, phi, dphi):
    """(E_L, dE_L) per walker, complex."""
    sys = ts.s
    G, dG, _ = _green_and_tangent(sys, phi, dphi)
    e1 = sum(np.einsum("ij,wji->w", sys.h1, Gs) for Gs in G)
    de1 = sum(np.einsum("ij,wji->w", ts.P, Gs) + np.einsum("ij,wji->w", sys.h1, dGs)
              for Gs, dGs in zip(G, dG))
    rb = afqmc.rhobar(sys, G)
    drb = afqmc.rhobar(sys, dG)
    ex = 0.0
    dex = 0.0
    for Gs, dGs in zip(G, dG):
        LG = sys.L[None] @ Gs[:, None]
        LdG = sys.L[None] @ dGs[:, None]
        ex = ex + np.einsum("wgik,wgki->wg", LG, LG)
        dex = dex + 2 * np.einsum("wgik,wgki->wg", LG, LdG)
    e = e1 + 0.5 * np.sum(rb * rb - ex, axis=1)
    de = de1 + 0.5 * np.sum(2 * rb * drb - dex, axis=1)
    return e, de


def mixed_energy_tangent(w, dlogw, eloc, deloc):
    """(E, dE) of sum w Re E_L / sum w (phaseless), over the walkers with w != 0 (a dead walker
    contributes nothing, even when its local energy is not finite)."""
    w = np.asarray(w).real
    live = w != 0
    w, dlogw, eloc, deloc = w[live], np.asarray(dlogw)[live], eloc[live], deloc[live]
    dw = w * dlogw
    W = np.sum(w)
    E = np.sum(w * eloc.real) / W
    dE = (np.sum(dw * eloc.real + w * deloc.real) - E * np.sum(dw)) / W
    return E, dE


def run(sys: afqmc.System, P, n_walkers, n_steps, fields, mgs_every=5, energy_every=5):
    """Walkers + tangents through n_steps on explicit fields; returns per-measurement (E, dE)."""
    ts = TangentSystem(sys, P)
    wk = afqmc.Walkers(sys, n_walkers)
    tw = TangentWalkers(wk)
    out = []
    for t in range(n_steps):
        propagate(ts, wk, tw, fields[t][:, :sys.X])
        if mgs_every and (t + 1) % mgs_every == 0:
            orthonormalise(sys, wk, tw)
        if energy_every and (t + 1) % energy_every == 0:
            e, de = local_energy_tangent(ts, wk.phi, tw.dphi)
            out.append(mixed_energy_tangent(wk.w, tw.dlogw, e, de))
    return np.array(out), wk, tw
