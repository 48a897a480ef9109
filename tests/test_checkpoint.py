"""Checkpoint files on CPU: the state of a run round-trips through a file unchanged, and a
checkpoint is refused by a system whose Hamiltonian shape, walkers, seed, walker offset,
precision or mode differ (those fix which fields the resumed run draws)."""
from types import SimpleNamespace

import numpy as np
import pytest

from paper_1703_01545_gb300 import checkpoint


def fake_system(**kw):
    opt = SimpleNamespace(seed=kw.pop("seed", 7), walker_offset=kw.pop("walker_offset", 0),
                          precision=kw.pop("precision", 0), mode=kw.pop("mode", 0))
    s = dict(M=8, X=24, n_up=2, n_dn=1, n_walkers=5, n_repeats=1)
    s.update(kw)
    return SimpleNamespace(opt=opt, **s)


def state(sys_, seed=0):
    rng = np.random.default_rng(seed)
    shape = (sys_.n_walkers, sys_.M, sys_.n_up + sys_.n_dn)
    phi = rng.standard_normal(shape) + 1j * rng.standard_normal(shape)
    w = np.abs(rng.standard_normal(sys_.n_walkers)) + 0j
    w[2] = 0.0   # a dead walker stays dead through the file
    return phi, w


def test_round_trip_through_a_file(tmp_path):
    s = fake_system()
    phi, w = state(s)
    ck = checkpoint.make(s, phi, w, 2 ** 40 + 5)
    checkpoint.save(tmp_path / "ck.npz", ck)
    back = checkpoint.load(tmp_path / "ck.npz")
    assert np.array_equal(back["phi"], phi) and np.array_equal(back["w"], w)
    assert int(back["step"]) == 2 ** 40 + 5
    checkpoint.check(back, s)


@pytest.mark.parametrize("change", [dict(seed=8), dict(walker_offset=5), dict(n_walkers=6),
                                    dict(M=9), dict(X=25), dict(n_up=1, n_dn=2), dict(n_repeats=5),
                                    dict(precision=1), dict(mode=1)])
def test_a_different_run_refuses_the_checkpoint(change):
    s = fake_system()
    phi, w = state(s)
    ck = checkpoint.make(s, phi, w, 10)
    with pytest.raises(ValueError, match="does not match"):
        checkpoint.check(ck, fake_system(**change))


def test_make_checks_shapes_and_step():
    s = fake_system()
    phi, w = state(s)
    with pytest.raises(ValueError):
        checkpoint.make(s, phi[:, :, :2], w, 0)
    with pytest.raises(ValueError):
        checkpoint.make(s, phi, w[:3], 0)
    with pytest.raises(ValueError):
        checkpoint.make(s, phi, w, -1)


def test_buffers_of_the_wrong_element_type_are_refused():
    """The binding hands raw pointers to C, which reads float64 (int32 for the alive flags):
    any other element type is refused instead of being reinterpreted."""
    import torch
    from paper_1703_01545_gb300.api import _ptr
    assert _ptr(None) is None
    assert _ptr(np.zeros(3)).value and _ptr(np.zeros(3, np.int32), "int32").value
    assert _ptr(torch.zeros(3, dtype=torch.float64)).value
    for bad in (np.zeros(3, np.float32), np.zeros(3, np.int64), torch.zeros(3)):
        with pytest.raises(TypeError):
            _ptr(bad)
    with pytest.raises(TypeError):
        _ptr(np.zeros(3), "int32")
    with pytest.raises(ValueError):
        _ptr(np.zeros((3, 3))[:, 0])
