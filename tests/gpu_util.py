import numpy as np
import pytest

from oracle import afqmc as orc
from synthetic import CONFIGS, build_system


def need_gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1703_01545_gb300 as afq
    afq.build()
    return afq


def system_data(cfg, which, coupling=1.0):
    d = dict(CONFIGS[cfg][which])
    d["coupling"] = coupling
    return build_system(**d)


def pair(afq, d, nw, dt, seed=1, R=1, mode=0, fb_cap=1.0, taylor_order=6,
         independent_fields=False):
    g = afq.System(d["h1"], d["L"], d["trial"], d["n_up"], d["n_dn"], dt=dt, n_walkers=nw,
                   seed=seed, n_repeats=R, mode=mode, fb_cap=fb_cap, taylor_order=taylor_order,
                   independent_fields=independent_fields)
    o = orc.System(d["h1"], d["L"], d["trial"], d["n_up"], d["n_dn"], dt, fb_cap=fb_cap,
                   mode=orc.FREE if mode == 1 else orc.PHASELESS, taylor_order=taylor_order)
    return g, o


def rel(a, b, floor=1e-300):
    a, b = np.asarray(a), np.asarray(b)
    return np.max(np.abs(a - b) / np.maximum(np.abs(b), floor))


def logo_close(a, b, tol):
    """log-overlaps agree up to 2 pi i: compare exp of the difference with 1."""
    d = np.exp(np.asarray(a) - np.asarray(b))
    return np.max(np.abs(d - 1)) < tol
