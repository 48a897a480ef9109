"""CPU checks of the C-ABI library: it loads, exports every declared symbol, has the
struct layout of include/afqmc.h, validates arguments before touching a device, and
its host statistics agree with the oracle's."""
import ctypes
import os
import re
import shutil
import subprocess

import numpy as np
import pytest

from oracle import stats

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "afqmc.h")


@pytest.fixture(scope="session")
def lib():
    from paper_1703_01545_gb300 import _lib
    from paper_1703_01545_gb300.build import build
    build()
    return _lib.load()


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(afqmc_[A-Za-z_0-9]+)\s*\(", text)))


def test_every_declared_symbol_is_exported_and_bound(lib):
    from paper_1703_01545_gb300 import _lib
    names = declared_functions()
    assert len(names) >= 15
    for n in names:
        assert hasattr(lib, n), n
        assert n in _lib.SIGNATURES, n


def test_struct_layout_matches_header(tmp_path):
    from paper_1703_01545_gb300 import _lib
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    src = tmp_path / "layout.c"
    src.write_text('#include <stdio.h>\n#include <stddef.h>\n#include "afqmc.h"\n'
                   'int main(void){printf("%zu %zu %zu %zu %zu %zu %zu %zu %zu %zu\\n", sizeof(afqmc_options),'
                   ' offsetof(afqmc_options, seed), offsetof(afqmc_options, walker_offset),'
                   ' offsetof(afqmc_options, autotune_cache), offsetof(afqmc_options, independent_fields),'
                   ' sizeof(afqmc_info), offsetof(afqmc_info, step), offsetof(afqmc_info, c_mf),'
                   ' offsetof(afqmc_info, n_alive), offsetof(afqmc_info, tuned_taylor_smem)); return 0;}\n')
    exe = tmp_path / "layout"
    cuda_inc = "/usr/local/cuda/include"
    r = subprocess.run([cc, "-I", os.path.join(ROOT, "include"), "-I", cuda_inc, str(src), "-o",
                        str(exe)], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    got = [int(v) for v in subprocess.run([str(exe)], capture_output=True, text=True).stdout.split()]
    O, I = _lib.AfqmcOptions, _lib.AfqmcInfo
    want = [ctypes.sizeof(O), O.seed.offset, O.walker_offset.offset, O.autotune_cache.offset,
            O.independent_fields.offset,
            ctypes.sizeof(I), I.step.offset,
            I.c_mf.offset, I.n_alive.offset, I.tuned_taylor_smem.offset]
    assert got == want


def test_default_options_and_status_strings(lib):
    from paper_1703_01545_gb300 import afqmc_default_options
    o = afqmc_default_options()
    assert (o.dt, o.n_walkers, o.taylor_order, o.mode, o.n_repeats, o.fb_cap) == (0.01, 128, 6, 0, 1, 1.0)
    assert o.independent_fields == 0
    for code in range(7):
        assert lib.afqmc_status_string(code)


def test_setup_rejects_bad_arguments_without_a_device(lib):
    from paper_1703_01545_gb300 import _lib, afqmc_default_options
    o = afqmc_default_options()
    M, X = 4, 2
    h1 = np.eye(M)
    L = np.zeros((X, M, M))
    trial = np.eye(M)[:, :2].copy()
    h = ctypes.c_void_p()

    def call(M_=M, X_=X, nu=1, nd=1, opt=o, a=h1):
        return lib.afqmc_setup(ctypes.byref(h), a.ctypes.data, L.ctypes.data, trial.ctypes.data, M_,
                               X_, nu, nd, ctypes.byref(opt), None)

    assert call(M_=0) == 1
    assert call(X_=0) == 1
    assert call(nu=0, nd=0) == 1
    assert call(nu=5) == 1
    bad = afqmc_default_options()
    bad.dt = -1.0
    assert call(opt=bad) == 1
    bad = afqmc_default_options()
    bad.n_repeats = 1000
    assert call(opt=bad) == 1
    bad = afqmc_default_options()
    bad.precision = 7
    assert call(opt=bad) == 1
    bad = afqmc_default_options()
    bad.independent_fields = 2
    assert call(opt=bad) == 1
    assert lib.afqmc_setup(None, None, None, None, 1, 1, 1, 0, None, None) == 1
    assert lib.afqmc_setup_multidet(None, None, None, None, None, 1, None, 1, 1, 1, 0, None,
                                    None) == 1
    assert lib.afqmc_destroy(None) == 0
    assert lib.afqmc_pair_delta_E(None, None, 5, 5, 5, 0.0, None, None, None, None, None) == 1
    assert lib.afqmc_pair_graph_kernels(None, None) == 1
    assert lib.afqmc_set_step(None, 5, None) == 1
    assert lib.afqmc_population_control(None, None, None) == 1
    assert lib.afqmc_seed_secondary(None, None, None) == 1


@pytest.mark.parametrize("R,tau_eq", [(11, 0.3), (4, 0.0), (1, 0.2), (5, 10.0)])
def test_host_statistics_match_oracle(lib, R, tau_eq):
    from paper_1703_01545_gb300 import afqmc_delta_E_stats
    rng = np.random.default_rng(R)
    dE = rng.standard_normal((25, R)) * 0.01 + 0.3
    taus = np.arange(1, 26) * 0.05
    mt, st, est = afqmc_delta_E_stats(dE, taus, tau_eq)
    m_o, s_o = stats.per_tau(dE)
    np.testing.assert_allclose(mt, m_o, rtol=1e-13)
    if R > 1:
        np.testing.assert_allclose(st, s_o, rtol=1e-12)
    want = stats.delta_e_estimate(dE, taus, tau_eq)
    for a, b in zip(est, want):
        assert (np.isnan(a) and np.isnan(b)) or abs(a - b) <= 1e-12 * max(1, abs(b))


def test_host_reblocking_matches_oracle(lib):
    from paper_1703_01545_gb300 import afqmc_reblock_error
    rng = np.random.default_rng(1)
    for n in (15, 16, 1000, 4097):
        x = np.cumsum(rng.standard_normal(n)) * 0.01
        assert abs(afqmc_reblock_error(x) - stats.reblock(x)) <= 1e-14 * max(1e-300, stats.reblock(x))


def test_host_statistics_edge_cases(lib):
    """Argument errors; no measurement after tau_eq (NaN estimate); one repeat (NaN error,
    the last cumulative mean); reblocking of a series too short for one 16-block level."""
    from paper_1703_01545_gb300 import afqmc_delta_E_stats, afqmc_reblock_error
    d = np.ones(4)
    est = np.empty(3)
    assert lib.afqmc_delta_E_stats(None, d.ctypes.data, 2, 2, 0.0, None, None, None) == 1
    assert lib.afqmc_delta_E_stats(d.ctypes.data, d.ctypes.data, 2, 0, 0.0, None, None, None) == 1
    assert lib.afqmc_delta_E_stats(d.ctypes.data, d.ctypes.data, -1, 2, 0.0, None, None, None) == 1
    assert lib.afqmc_delta_E_stats(d.ctypes.data, d.ctypes.data, 0, 2, 0.0, None, None,
                                   est.ctypes.data) == 0 and np.all(np.isnan(est))
    dE = np.array([[1.0, 2.0], [3.0, 5.0]])
    _, _, e = afqmc_delta_E_stats(dE, np.array([0.1, 0.2]), 0.5)       # nothing after tau_eq
    assert all(np.isnan(e))
    _, se, e = afqmc_delta_E_stats(np.array([[1.0], [3.0], [2.0]]), np.array([0.1, 0.2, 0.3]), 0.0)
    assert np.all(np.isnan(se)) and e[0] == 2.0 and np.isnan(e[1]) and e[2] == 0.3
    assert afqmc_reblock_error(np.arange(15.0)) == 0.0
    assert np.isnan(lib.afqmc_reblock_error(None, 5))
