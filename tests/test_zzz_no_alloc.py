"""afqmc_local_energy_static: local energies for callers that cannot allocate device memory.

Such callers (code running inside another framework's memory pool or under a fixed
memory budget, or an embedding that only hands over existing device buffers) cannot
go through afqmc_setup, which allocates.  The static entry point takes only device
buffers the caller already owns and keeps its intermediates in a static device array.
This test calls it through the C ABI twice in a row and checks both results against
the local energies of the regular entry point, afqmc_energy, at the FP64 tolerance of
the other GPU tests.  It lives in its own file so that pytest collects it last.
"""
import ctypes

import numpy as np
import pytest

from gpu_util import need_gpu, system_data

pytestmark = pytest.mark.gpu
TOL = 1e-9


def _call(lib, d, phi_dev, nw, out, torch):
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()
    h1, L, tr = dev(d["h1"]), dev(d["L"]), dev(d["trial"])
    code = lib.afqmc_local_energy_static(
        ctypes.c_void_p(h1.data_ptr()), ctypes.c_void_p(L.data_ptr()), ctypes.c_void_p(tr.data_ptr()),
        ctypes.c_void_p(phi_dev.data_ptr()), d["M"], d["X"], d["n_up"], d["n_dn"], nw,
        ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    torch.cuda.synchronize()
    return code


@pytest.mark.parametrize("cfg,which,nw", [("C1", "B", 96), ("C2", "A", 2048)])
def test_static_energy_matches_regular_entry_point(cfg, which, nw):
    afq = need_gpu()
    import torch
    from paper_1703_01545_gb300 import _lib
    lib = _lib.load()
    d = system_data(cfg, which, coupling="moderate" if cfg == "C2" else 1.0)
    s = afq.System(d["h1"], d["L"], d["trial"], d["n_up"], d["n_dn"], dt=0.01, n_walkers=nw,
                   seed=5)
    s.propagate(7)               # non-trivial walkers
    st = s.state()
    want, _, _ = s.energy()      # the regular entry point (afqmc_energy)
    s.close()
    phi = np.stack([st["phi"].real, st["phi"].imag])
    phi_dev = torch.from_numpy(np.ascontiguousarray(phi)).cuda()
    for _ in range(2):           # two calls in a row share the static array
        out = torch.full((2 * nw,), float("nan"), dtype=torch.float64, device="cuda")
        assert _call(lib, d, phi_dev, nw, out, torch) == 0
        got = out.cpu().numpy()
        got = got[:nw] + 1j * got[nw:]
        err = np.max(np.abs(got - want) / np.abs(want))
        assert err < TOL, err


def test_static_energy_rejects_oversize_and_host_pointers():
    need_gpu()
    import torch
    from paper_1703_01545_gb300 import _lib
    lib = _lib.load()
    d = system_data("C1", "A")
    small = torch.zeros(16, dtype=torch.float64, device="cuda")
    p = ctypes.c_void_p(small.data_ptr())
    # Cholesky tensor far beyond the static array: rejected before any launch
    assert lib.afqmc_local_energy_static(p, p, p, p, 64, 1_000_000, 8, 8, 4, p, None) == 1
    host = np.zeros(16)
    hp = ctypes.c_void_p(host.ctypes.data)
    assert lib.afqmc_local_energy_static(hp, p, p, p, d["M"], d["X"], 2, 2, 1, p, None) == 1


def test_static_energy_marks_singular_walkers():
    """A walker with a zero column has an exactly singular overlap (Eq. 6's Green's function
    does not exist): its entries come back NaN, every other walker as before."""
    afq = need_gpu()
    import torch
    from paper_1703_01545_gb300 import _lib
    lib = _lib.load()
    d = system_data("C1", "A")
    nw, bad = 24, 5
    s = afq.System(d["h1"], d["L"], d["trial"], d["n_up"], d["n_dn"], dt=0.01, n_walkers=nw,
                   seed=9)
    s.propagate(4)
    st = s.state()
    want, _, _ = s.energy()
    s.close()
    phi = np.stack([st["phi"].real, st["phi"].imag])
    phi[:, bad, :, 1] = 0.0                     # walker `bad`: spin-up column 1 set to zero
    phi_dev = torch.from_numpy(np.ascontiguousarray(phi)).cuda()
    out = torch.zeros(2 * nw, dtype=torch.float64, device="cuda")
    assert _call(lib, d, phi_dev, nw, out, torch) == 0
    got = out.cpu().numpy()
    got = got[:nw] + 1j * got[nw:]
    assert np.isnan(got[bad].real) and np.isnan(got[bad].imag)
    keep = np.arange(nw) != bad
    assert np.max(np.abs(got[keep] - want[keep]) / np.abs(want[keep])) < TOL


def test_static_energy_rejects_another_devices_memory():
    """Buffers on a GPU other than the current one are refused before any launch."""
    need_gpu()
    import torch
    if torch.cuda.device_count() < 2:
        pytest.skip("one visible GPU")
    from paper_1703_01545_gb300 import _lib
    lib = _lib.load()
    d = system_data("C1", "A")
    here = torch.zeros(4096, dtype=torch.float64, device="cuda:0")
    there = torch.zeros(4096, dtype=torch.float64, device="cuda:1")
    p, q = ctypes.c_void_p(here.data_ptr()), ctypes.c_void_p(there.data_ptr())
    with torch.cuda.device(0):
        assert lib.afqmc_local_energy_static(p, p, p, q, d["M"], d["X"], 2, 2, 4, p, None) == 1
