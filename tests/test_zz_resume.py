"""Resume from a checkpoint on the GPU: a run interrupted right after an orthonormalisation,
written to a file and restored into a fresh handle (walkers, weights, step counter of the
field stream) continues exactly as the uninterrupted run (FP64 path: log O and Theta are
recomputed from Phi in both)."""
import numpy as np
import pytest

from gpu_util import need_gpu, system_data

pytestmark = pytest.mark.gpu


def test_resume_continues_the_uninterrupted_run(tmp_path):
    afq = need_gpu()
    from paper_1703_01545_gb300 import checkpoint
    d = system_data("C1", "B")
    nw, seed, dt = 32, 77, 0.01

    def handle(s=seed):
        return afq.System(d["h1"], d["L"], d["trial"], d["n_up"], d["n_dn"], dt=dt,
                          n_walkers=nw, seed=s, n_repeats=2)

    ref = handle()
    ref.propagate(5)
    ref.orthonormalise()
    checkpoint.save(tmp_path / "ck.npz", ref.checkpoint())
    ref.propagate(5)
    ref.orthonormalise()
    el_ref, em_ref, _ = ref.energy()
    st_ref = ref.state()

    g = handle()
    g.resume(checkpoint.load(tmp_path / "ck.npz"))
    assert g.info().step == 5
    g.propagate(5)
    g.orthonormalise()
    el, em, _ = g.energy()
    st = g.state()
    assert np.array_equal(st["alive"], st_ref["alive"])
    np.testing.assert_allclose(st["phi"], st_ref["phi"], rtol=0, atol=1e-12 * np.abs(st_ref["phi"]).max())
    np.testing.assert_allclose(st["w"], st_ref["w"], rtol=1e-12, atol=0)
    np.testing.assert_allclose(el, el_ref, rtol=1e-12, atol=0)
    np.testing.assert_allclose(em, em_ref, rtol=1e-12, atol=0)
    # another seed draws other fields: the checkpoint is refused
    other = handle(seed + 1)
    with pytest.raises(ValueError, match="seed"):
        other.resume(checkpoint.load(tmp_path / "ck.npz"))
    for h in (ref, g, other):
        h.close()
