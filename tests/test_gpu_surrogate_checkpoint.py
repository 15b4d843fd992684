"""Surrogate checkpoint and resume on the GPU: a saved state reloaded into a
fresh network gives bit-identical outputs, and training resumed from it
reaches bit-identical parameters (the training kernels are deterministic);
a checkpoint of another scene is refused."""
import pytest

from paper_2310_07854_gb300 import binding as B
from paper_2310_07854_gb300 import surrogate as SG
from paper_2310_07854_gb300 import synth

pytestmark = pytest.mark.gpu


def test_resume_continues_bit_for_bit(tmp_path):
    import torch
    w = synth.make_workload("single_128")
    sd = B.DeviceScene(w.scene)
    s1 = SG.Surrogate(sd, synth.init_mlp_params(5))
    u, y = s1.training_set(1, n=32768)
    s1.train(u, y, epochs=1, batch=4096, seed=0)
    s1.domain.margin = 0.07
    path = str(tmp_path / "s.ckpt")
    s1.save(path, seed=0, epochs=1)
    f1 = s1.forward(u[:1000])
    s1.train(u, y, epochs=1, batch=4096, seed=5)
    p1 = s1.params()

    s2 = SG.Surrogate(sd, synth.init_mlp_params(6))
    meta = s2.load(path)
    assert meta["epochs"] == 1 and s2.domain.margin == pytest.approx(0.07)
    assert torch.equal(s2.forward(u[:1000]), f1)
    s2.train(u, y, epochs=1, batch=4096, seed=5)
    assert torch.equal(s2.params(), p1)

    other = SG.Surrogate(B.DeviceScene(synth.make_scene(99, 8)), synth.init_mlp_params(5))
    with pytest.raises(ValueError):
        other.load(path)
