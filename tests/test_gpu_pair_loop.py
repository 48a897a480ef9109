"""The correlated pair run as one graph launch (a device-side while loop over the
measurement blocks of both systems, Sec. II.B) against one launch of the same block graph
per measurement block.

Both forms run the same kernels in the same order on the same data, so every output must be
identical bit for bit: the per-repeat energy series of each call and the walkers, weights,
log-overlaps and alive flags after it.  Three calls per pair exercise the cached graph: the
first builds it, the second asks for fewer blocks than it was built for (the loop must stop at
the call's count, not the series' capacity), the third for more (it is rebuilt).  The
oracle parity of the default form is covered by the pair tests in test_gpu_parity.py.
"""
import numpy as np
import pytest

from gpu_util import need_gpu, system_data
from synthetic import CONFIGS

pytestmark = pytest.mark.gpu

CALLS = (30, 10, 40)   # propagation steps per call; 5 steps per measurement block


@pytest.fixture(scope="module")
def afq():
    return need_gpu()


def run(afq, form, precision, workload, nw, R):
    cfg = CONFIGS[workload]
    systems = []
    for which in ("A", "B"):
        d = system_data(workload, which, "moderate")
        systems.append(afq.System(d["h1"], d["L"], d["trial"], d["n_up"], d["n_dn"], dt=cfg["dt"],
                                  n_walkers=nw, seed=7, n_repeats=R, precision=precision,
                                  autotune=False))
    A, B = systems
    A.select_kernel(afq.K_PAIR_LOOP, form)
    series, forms = [], []
    for n in CALLS:
        res = afq.pair_delta_E(A, B, n, energy_every=5, mgs_every=5, raise_on_dead=False)
        assert res["E"].shape[0] == n // 5
        series.append(res["E"])
        forms.append(afq.pair_run_form(A))
    states = [s.state() for s in systems]
    n_kernels = afq.pair_graph_kernels(A)
    steps = A.info().step
    for s in systems:
        s.close()
    return series, states, forms, n_kernels, steps


@pytest.mark.parametrize("precision,workload,nw", [("fp64", "C1", 64), ("bf16x3", "C2", 256)])
def test_one_launch_equals_per_block_launches(afq, precision, workload, nw):
    prec = afq.FP64 if precision == "fp64" else afq.BF16X3
    loop = run(afq, 1, prec, workload, nw, 4)
    blocks = run(afq, 0, prec, workload, nw, 4)
    assert loop[2] == [1, 1, 1] and blocks[2] == [0, 0, 0]
    assert loop[3] == blocks[3] > 0
    assert loop[4] == blocks[4] == sum(CALLS)
    for a, b in zip(loop[0], blocks[0]):
        assert np.all(np.isfinite(a))
        np.testing.assert_array_equal(a, b)
    for sa, sb in zip(loop[1], blocks[1]):
        for key in ("phi", "w", "logO", "alive"):
            np.testing.assert_array_equal(sa[key], sb[key])


def test_form_selection_errors(afq):
    d = system_data("C1", "A")
    g = afq.System(d["h1"], d["L"], d["trial"], d["n_up"], d["n_dn"], dt=CONFIGS["C1"]["dt"],
                   n_walkers=8)
    assert afq.pair_run_form(g) == -1
    with pytest.raises(afq.AfqmcError, match="invalid argument"):
        g.select_kernel(afq.K_PAIR_LOOP, 2)
    g.close()
