"""Reverse-mode gradient dE/dh1 of the run's mixed energy (oracle side, plain FP64).

E = mean over the measurements m of E_m = sum_k w_k Re E_L,k / sum_k w_k, for one field
realisation with the trial held fixed (Sec. II.A-B, II.D).  The forward run stores every
step's walkers; the reverse pass walks the steps backwards.  Complex adjoints follow
zbar = dL/dRe z + i dL/dIm z, so for z = f(u) holomorphic ubar += zbar conj(f'(u)).

Per live walker and step (forward -> reverse):
  O = Psi^T Phi, Y = O^{-1}, Theta = Phi Y, G = Psi Theta^T
  rhobar_g = tr(L_g G);  x_r = -i sqrt(dt)(rhobar - <rho>);  xbar = cap(x_r)
  c = x - xbar;  A = i sqrt(dt) sum_g c_g L_g;  log s = -i sqrt(dt) c.<rho>
  Phi1 = E Phi;  T_n = A T_{n-1} / n;  Phi2 = sum_n T_n;  Phi' = E Phi2
  log R = log s + log det(Psi^T Phi') - log det(Psi^T Phi);  theta = Im log R
  log w' = log w + Re log R + Re(x.xbar - xbar.xbar/2) + const + log cos(theta)
reverse, given Phibar' and lwbar':
  Rbar = lwbar' (1 - i tan theta);  xbarbar = lwbar' conj(x - xbar)
  cbar = Rbar conj(-i sqrt(dt) <rho>) + ...;  Phibar' += Rbar conj(Psi O'^{-T})
  Phibar2 = E Phibar';  Ebar += Re(Phibar' Phi2^H)
  Taylor: Tbar = Phibar2; for n = order..1: Abar += Tbar T_{n-1}^H / n; Tbar = Phibar2 + A^H Tbar / n
  cbar_g += conj(i sqrt(dt)) sum_ij Abar_ij L_g,ij;  Phibar = E Tbar;  Ebar += Re(Tbar Phi^H)
  xbar adjoint through the cap, rhobarbar = conj(-i sqrt(dt)) x_rbar, Gbar += rhobarbar_g L_g,
  Thetabar = Gbar^T Psi, Phibar += Thetabar Y^H, Ybar = Phi^H Thetabar, Obar = -Y^H Ybar Y^H,
  Phibar += Psi Obar - Rbar conj(Psi O^{-T})
MGS (Q = Phi R^{-1}, R held fixed: every later quantity is invariant under Phi -> Phi M):
  Phibar = Qbar R^{-H}.
Finally E = exp(B), B = -dt K/2, K = h1 + ...: h1bar += -dt/2 L_exp(B, Ebar) (the Frechet
derivative of exp is self-adjoint at symmetric B), plus the direct one-body term of E_L.
"""
import numpy as np

from . import afqmc
from .tangent import frechet_exp


def _green_parts(sys, phi):
    """Per spin: (O, Y = O^{-1}, Theta, G) for walkers phi [Nw, M, N]."""
    out = []
    for a, b in sys.spins:
        if b == a:
            out.append(None)
            continue
        Psi = sys.trial[:, a:b]
        O = np.einsum("ia,wib->wab", Psi, phi[:, :, a:b])
        Y = np.linalg.inv(O)
        Th = phi[:, :, a:b] @ Y
        G = Psi[None] @ np.swapaxes(Th, 1, 2)
        out.append((O, Y, Th, G))
    return out


def _backprop_green(sys, phi, parts, Gbar, phibar):
    """Accumulate into phibar the adjoint of G_s(Phi) given Gbar_s (per spin)."""
    for (a, b), p, Gb in zip(sys.spins, parts, Gbar):
        if p is None or Gb is None:
            continue
        O, Y, Th, G = p
        Psi = sys.trial[:, a:b]
        Thb = np.swapaxes(Gb, 1, 2) @ Psi                    # Thetabar = Gbar^T Psi
        YH = np.conj(np.swapaxes(Y, 1, 2))
        phibar[:, :, a:b] += Thb @ YH                         # Theta = Phi Y
        Yb = np.conj(np.swapaxes(phi[:, :, a:b], 1, 2)) @ Thb
        Ob = -YH @ Yb @ YH                                   # Y = O^{-1}
        phibar[:, :, a:b] += Psi[None] @ Ob                  # O = Psi^T Phi


def _logdet_grad(sys, parts):
    """Per spin: Psi O^{-T} (d log det(Psi^T Phi) = sum_ij (Psi O^{-T})_ij dPhi_ij)."""
    out = []
    for (a, b), p in zip(sys.spins, parts):
        if p is None:
            out.append(None)
            continue
        O, Y, Th, G = p
        out.append(sys.trial[:, a:b][None] @ np.swapaxes(Y, 1, 2))
    return out


def run_with_gradient(sys: afqmc.System, n_walkers, n_steps, fields, mgs_every=5,
                      energy_every=5):
    """(E, dE/dh1 [M, M]) for one run on explicit fields (phaseless mode)."""
    M = sys.M
    wk = afqmc.Walkers(sys, n_walkers)
    tape = []      # per step: phi before, alive before, lw before, phi2, terms, x, xbar data
    meas = []      # (step index after which measured, phi, w, alive)
    mgs_R = {}     # step -> list of (a, b, R) per spin, walkers indexed by live idx
    n_meas = 0
    for t in range(n_steps):
        x = fields[t][:, :sys.X]
        live = wk.alive.copy()
        idx = np.nonzero(live)[0]
        phi = wk.phi[idx].copy()
        parts = _green_parts(sys, phi)
        Gs = [p[3] if p is not None else np.zeros((idx.size, M, M)) for p in parts]
        rb = afqmc.rhobar(sys, Gs)
        xr = -1j * sys.sqrt_dt * (rb - sys.rho_mf)
        mag = np.abs(xr)
        capped = (mag > sys.fb_cap) if sys.fb_cap > 0 else np.zeros_like(mag, bool)
        xb = np.where(capped, xr * (sys.fb_cap / np.where(capped, mag, 1.0)), xr)
        xs = x[idx]
        c = xs - xb
        Lf = sys.L.reshape(sys.X, M * M)
        A = 1j * sys.sqrt_dt * (c @ Lf).reshape(-1, M, M)
        phi1 = sys.expK @ phi
        terms = [phi1]
        for n in range(1, sys.taylor_order + 1):
            terms.append((A @ terms[-1]) / n)
        phi2 = sum(terms)
        phi3 = sys.expK @ phi2
        logO_new = afqmc.overlap(sys, phi3)
        log_s = -1j * sys.sqrt_dt * (c @ sys.rho_mf)
        logR = log_s + logO_new - wk.logO[idx]
        logI = logR + np.sum(xs * xb, axis=1) - 0.5 * np.sum(xb * xb, axis=1) \
            - sys.dt * (sys.C - sys.E_T)
        cosv = np.cos(logR.imag)
        w_new = wk.w[idx].real * np.exp(logI.real) * np.maximum(0.0, cosv)
        still = w_new > 0
        tape.append(dict(idx=idx, phi=phi, parts=parts, xr=xr, xb=xb, capped=capped, x=xs,
                         A=A, terms=terms, phi2=phi2, phi3=phi3, theta=logR.imag, still=still))
        wk.phi[idx] = phi3
        wk.logO[idx] = logO_new
        wk.w[idx] = np.where(still, w_new, 0.0)
        wk.alive[idx] = still
        if mgs_every and (t + 1) % mgs_every == 0:
            li = np.nonzero(wk.alive)[0]
            Rs = []
            ph = wk.phi[li]
            for a, b in sys.spins:
                if b > a:
                    Q = afqmc.modified_gram_schmidt(ph[:, :, a:b])
                    R = np.conj(np.swapaxes(Q, 1, 2)) @ ph[:, :, a:b]
                    Rs.append((a, b, np.triu(R)))
                    ph[:, :, a:b] = Q
            wk.phi[li] = ph
            wk.logO[li] = afqmc.overlap(sys, ph)
            mgs_R[t] = (li, Rs)
        if energy_every and (t + 1) % energy_every == 0:
            meas.append((t, wk.phi.copy(), wk.w.real.copy(), wk.alive.copy()))
            n_meas += 1
    # ---- energy and reverse pass ----
    E_total = 0.0
    phibar = np.zeros_like(wk.phi)
    lwbar = np.zeros(n_walkers)
    Ebar = np.zeros((M, M))
    h1bar = np.zeros((M, M))
    meas_at = {m[0]: m for m in meas}
    for t in reversed(range(n_steps)):
        if t in meas_at:
            _, phim, wm, am = meas_at[t]
            li = np.nonzero(am)[0]
            ph = phim[li]
            parts = _green_parts(sys, ph)
            el = afqmc.local_energy(sys, ph)
            W = wm[li].sum()
            Em = np.sum(wm[li] * el.real) / W
            E_total += Em / n_meas
            lwbar[li] += wm[li] * (el.real - Em) / W / n_meas
            ebar = wm[li] / W / n_meas
            Gs = [p[3] for p in parts if p is not None]
            rb = afqmc.rhobar(sys, [p[3] if p is not None else np.zeros((li.size, M, M)) for p in parts])
            Gbar = []
            for p in parts:
                if p is None:
                    Gbar.append(None)
                    continue
                G = p[3]
                h1bar += np.einsum("w,wji->ij", ebar, G).real
                LGL = np.einsum("gij,wjk,gkl->wil", sys.L, G, sys.L)
                F = sys.h1[None] + np.einsum("wg,gij->wij", rb, sys.L) - LGL      # dE_L/dG_ji = F_ij
                Gbar.append(ebar[:, None, None] * np.conj(np.swapaxes(F, 1, 2)))
            pb = np.zeros_like(ph)
            _backprop_green(sys, ph, parts, Gbar, pb)
            phibar[li] += pb
        if t in mgs_R:
            li, Rs = mgs_R[t]
            pb = phibar[li]
            for a, b, R in Rs:
                pb[:, :, a:b] = pb[:, :, a:b] @ np.conj(np.swapaxes(np.linalg.inv(R), 1, 2))
            phibar[li] = pb
        rec = tape[t]
        idx, still = rec["idx"], rec["still"]
        if idx.size == 0:
            continue
        pbn = np.where(still[:, None, None], phibar[idx], 0.0)      # dead after this step: no flow
        lb = np.where(still, lwbar[idx], 0.0)
        phi, parts, phi3 = rec["phi"], rec["parts"], rec["phi3"]
        th = rec["theta"]
        Rbar = lb * (1.0 - 1j * np.tan(th))
        xs, xb, xr = rec["x"], rec["xb"], rec["xr"]
        xbb = lb[:, None] * np.conj(xs - xb)                         # from x.xbar - xbar^2/2
        cbar = Rbar[:, None] * np.conj(-1j * sys.sqrt_dt * sys.rho_mf)[None, :]
        parts3 = _green_parts(sys, phi3)
        for (a, b), g in zip(sys.spins, _logdet_grad(sys, parts3)):
            if g is not None:
                pbn[:, :, a:b] += Rbar[:, None, None] * np.conj(g)
        pb2 = sys.expK @ pbn
        Ebar += np.einsum("wia,wja->ij", pbn, np.conj(rec["phi2"])).real
        terms, A = rec["terms"], rec["A"]
        AH = np.conj(np.swapaxes(A, 1, 2))
        Tb = pb2.copy()
        Abar = np.zeros_like(A)
        for n in range(sys.taylor_order, 0, -1):
            Abar += Tb @ np.conj(np.swapaxes(terms[n - 1], 1, 2)) / n
            Tb = pb2 + (AH @ Tb) / n
        cbar += np.conj(1j * sys.sqrt_dt) * np.einsum("wij,gij->wg", Abar, sys.L)
        pb_phi = sys.expK @ Tb
        Ebar += np.einsum("wia,wja->ij", Tb, np.conj(phi)).real
        xbb += -cbar
        # cap adjoint
        mag = np.abs(xr)
        safe = np.where(rec["capped"], mag, 1.0)
        xrb = np.where(rec["capped"],
                       (sys.fb_cap / safe) * (xbb - np.real(np.conj(xbb) * xr) * xr / safe ** 2),
                       xbb)
        rbb = np.conj(-1j * sys.sqrt_dt) * xrb
        Gbar = [None if p is None else np.einsum("wg,gij->wij", rbb, sys.L) for p in parts]
        _backprop_green(sys, phi, parts, Gbar, pb_phi)
        for (a, b), g in zip(sys.spins, _logdet_grad(sys, parts)):
            if g is not None:
                pb_phi[:, :, a:b] -= Rbar[:, None, None] * np.conj(g)
        phibar[idx] = pb_phi
        lwbar[idx] = lb
    B = -0.5 * sys.dt * sys.K
    _, LE = frechet_exp(B, Ebar)
    h1bar += -0.5 * sys.dt * LE
    return E_total, h1bar
