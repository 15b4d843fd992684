"""Surrogate checkpoint files without a GPU: the header and raw state round
trip; a cut or foreign file is refused; the scene hash tells scenes apart."""
import numpy as np
import pytest

from paper_2310_07854_gb300 import surrogate as SG
from paper_2310_07854_gb300 import synth


def test_round_trip(tmp_path):
    state = np.random.default_rng(0).integers(0, 256, 10_000, dtype=np.uint8).tobytes()
    path = str(tmp_path / "a.ckpt")
    SG.write_checkpoint(path, state, {"scene_sha256": "x", "epochs": 3, "margin": 0.07})
    meta, back = SG.read_checkpoint(path)
    assert back == state
    assert meta == {"scene_sha256": "x", "epochs": 3, "margin": 0.07, "state_bytes": 10_000}


def test_cut_or_foreign_files_are_refused(tmp_path):
    path = tmp_path / "a.ckpt"
    SG.write_checkpoint(str(path), b"\x01" * 4096, {"k": 1})
    data = path.read_bytes()
    path.write_bytes(data[:-1])
    with pytest.raises(ValueError):
        SG.read_checkpoint(str(path))
    path.write_bytes(b"NOTACKPT" + data[8:])
    with pytest.raises(ValueError):
        SG.read_checkpoint(str(path))


def test_scene_hash():
    a, b = synth.make_scene(3, 8), synth.make_scene(3, 8)
    assert SG.scene_hash(a) == SG.scene_hash(b)
    b.pose[5, 10] = np.nextafter(b.pose[5, 10], np.float32(1))
    assert SG.scene_hash(a) != SG.scene_hash(b)
    c = synth.make_scene(3, 8)
    c.half_ext[0, 0] *= 2
    assert SG.scene_hash(a) != SG.scene_hash(c)
