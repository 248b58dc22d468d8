"""Checkpoint files: round trip, and damage detected on the host (fault injection
by truncating or flipping bytes of the file; no GPU involved)."""
import numpy as np
import pytest

import workloads as W
from paper_1511_03614_gb300 import prepare_feynman
from paper_1511_03614_gb300 import api


class _FakeInteg:
    """Stands in for an Integrator: holds grids on the host."""

    def __init__(self, prep):
        self.prep = prep
        rng = np.random.default_rng(0)
        self.grids = []
        for u in prep.units:
            g = np.sort(rng.uniform(size=(u.dim, 129)), axis=1)
            g[:, 0], g[:, -1] = 0.0, 1.0
            self.grids.append(g)

    def get_grid(self, k):
        return self.grids[k]

    def set_grid(self, k, g):
        self.grids[k] = np.array(g)


def _state(n):
    return dict(it=6, seed=3, precision="fp64", rng="philox", points=1000, gpu_ms=12.5, points_done=6000,
                sw=np.arange(n, dtype=float) + 1, swi=np.arange(n, dtype=float) * 0.5)


def test_checkpoint_round_trip(tmp_path):
    prep = prepare_feynman(W.box())
    a = _FakeInteg(prep)
    p = str(tmp_path / "ck.bin")
    api.save_checkpoint(p, a, _state(len(prep.units)))
    b = _FakeInteg(prep)
    for g in b.grids:
        g[:] = 0.5
    st = api.load_checkpoint(p, b)
    assert st["it"] == 6 and st["seed"] == 3 and st["points_done"] == 6000
    assert np.array_equal(st["sw"], np.arange(len(prep.units)) + 1.0)
    for ga, gb in zip(a.grids, b.grids):
        assert np.array_equal(ga, gb)


@pytest.mark.parametrize("damage", ["truncate", "flip", "magic"])
def test_damaged_checkpoint_is_rejected(tmp_path, damage):
    prep = prepare_feynman(W.bubble())
    a = _FakeInteg(prep)
    p = str(tmp_path / "ck.bin")
    api.save_checkpoint(p, a, _state(len(prep.units)))
    raw = bytearray(open(p, "rb").read())
    if damage == "truncate":
        raw = raw[:-40]
    elif damage == "flip":
        raw[len(raw) // 2] ^= 0x10
    else:
        raw[0:8] = b"XXXXXXXX"
    open(p, "wb").write(bytes(raw))
    with pytest.raises(ValueError):
        api.load_checkpoint(p, _FakeInteg(prep))
