"""Checkpoint files (host logic, no GPU): exact round trip of the block store,
configurations, step and seed; refusal of damaged files and of files written
for another model; an interrupted save leaves the previous checkpoint."""

import os

import numpy as np
import pytest

from paper_2503_20566_gb300 import checkpoint as ck


class FakeCtx:
    """The attributes and tensor calls of a Context, held on the host."""

    def __init__(self, complex_=False, chi=4, Q=None):
        self.N, self.Lx, self.Ly, self.D, self.chi = 2, 4, 3, 4, chi
        self.matter, self.complex, self.precision = False, complex_, "fp32"
        self.h, self.g, self.J, self.m = 1.0, 0.3, 0.0, 0.0
        self.Q = Q
        self.n_params, self.cfg_len = 37, 29
        g = np.random.default_rng(1)
        v = g.standard_normal(self.n_params).astype(np.float32).astype(np.float64)
        if complex_:
            v = v + 1j * g.standard_normal(self.n_params).astype(np.float32)
        self.params = v

    def get_tensors(self):
        return self.params.copy()

    def set_tensors(self, values):
        self.params = np.array(values, copy=True)


def _configs(n=5, cfg_len=29, seed=3):
    return np.random.default_rng(seed).integers(0, 2, size=(n, cfg_len)).astype(np.int8)


@pytest.mark.parametrize("complex_", [False, True])
def test_round_trip_is_exact(tmp_path, complex_):
    ctx = FakeCtx(complex_=complex_, Q=[1, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 1])
    cfg = _configs()
    path = str(tmp_path / "run.ck")
    ck.save(path, ctx, cfg, step=17, seed=2024, extra={"lr": 0.01})
    got = ck.load(path)
    assert got.step == 17 and got.seed == 2024 and got.extra == {"lr": 0.01}
    assert got.params.dtype == (np.complex128 if complex_ else np.float64)
    assert np.array_equal(got.params, ctx.params) and np.array_equal(got.configs, cfg)
    assert got.model == ck.model_of(ctx)
    other = FakeCtx(complex_=complex_, Q=[1, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 1])
    other.params[:] = 0
    dev = ck.restore(other, got, device="cpu")
    assert np.array_equal(other.params, ctx.params) and np.array_equal(dev.numpy(), cfg)
    assert [p for p in os.listdir(tmp_path) if ".tmp" in p] == []


def test_damaged_files_are_refused(tmp_path):
    ctx = FakeCtx()
    path = str(tmp_path / "run.ck")
    ck.save(path, ctx, _configs(), step=1, seed=7)
    blob = open(path, "rb").read()
    for name, bad in [("flipped", blob[:-3] + bytes([blob[-3] ^ 1]) + blob[-2:]),
                      ("truncated", blob[:-10]), ("magic", b"XXXXXXXX" + blob[8:]), ("empty", b"")]:
        p = str(tmp_path / name)
        open(p, "wb").write(bad)
        with pytest.raises(ck.CheckpointError):
            ck.load(p)


def test_checkpoint_of_another_model_is_refused(tmp_path):
    path = str(tmp_path / "run.ck")
    ck.save(path, FakeCtx(chi=4), _configs(), step=1, seed=7)
    got = ck.load(path)
    with pytest.raises(ck.CheckpointError, match="chi"):
        ck.restore(FakeCtx(chi=8), got, device="cpu")
    with pytest.raises(ck.CheckpointError, match="Q"):
        ck.check_model(FakeCtx(chi=4, Q=[0] * 11 + [1]), got)


def test_configs_of_the_wrong_width_are_refused(tmp_path):
    with pytest.raises(ck.CheckpointError):
        ck.save(str(tmp_path / "x.ck"), FakeCtx(), _configs(cfg_len=28), step=0, seed=0)


def test_interrupted_save_keeps_the_previous_checkpoint(tmp_path, monkeypatch):
    ctx = FakeCtx()
    path = str(tmp_path / "run.ck")
    ck.save(path, ctx, _configs(), step=3, seed=9)

    def fail(*a, **k):
        raise OSError("disk full")

    monkeypatch.setattr(ck.os, "replace", fail)
    ctx.params = ctx.params + 1.0
    with pytest.raises(OSError):
        ck.save(path, ctx, _configs(seed=4), step=4, seed=9)
    got = ck.load(path)
    assert got.step == 3 and np.array_equal(got.configs, _configs())
    assert sorted(os.listdir(tmp_path)) == ["run.ck"]


def test_header_without_a_field_is_refused(tmp_path):
    import json
    import struct

    body = b""
    hb = json.dumps({"version": ck.VERSION, "sha256": __import__("hashlib").sha256(body).hexdigest()}).encode()
    p = str(tmp_path / "h.ck")
    open(p, "wb").write(ck.MAGIC + struct.pack("<I", len(hb)) + hb + body)
    with pytest.raises(ck.CheckpointError, match="incomplete"):
        ck.load(p)
