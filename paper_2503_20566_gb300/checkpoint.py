"""Checkpoint / resume of a VMC run: the block store, the chain configurations
and the position in the Metropolis random stream.

The chains draw from a counter-based stream: a sample_batch call with seed
`seed` gives chain c its draws from (seed, c, sweep, slot) alone, so the
stream position of a run is the step index together with the rule that maps
a step to its seed.  A checkpoint stores the parameters (the block store in
the library's documented layout, as FP64 / complex128 values, exact for FP32
storage), the configurations of every chain, the step index, the base seed,
and the model the context was created with.  Restoring it into a context of
the same model and sampling step `step` with that step's seed reproduces the
chains of the original run bit for bit; the SR update that follows is
reproducible only up to rounding, because its scatter combines partial sums
with atomics.

File layout (little-endian): the 8-byte magic b"GCFVMCK1", a uint32 header
length, a UTF-8 JSON header, then the parameters (float64 or complex128,
n_params values) and the configurations (int8, n_chains x cfg_len).  The
header carries a SHA-256 of the payload; `load` refuses a file whose payload
does not match it.  `save` writes a temporary file and renames it, so an
interrupted save leaves the previous checkpoint in place.
"""

from __future__ import annotations

import hashlib
import json
import os
import struct
from dataclasses import dataclass, field

import numpy as np

MAGIC = b"GCFVMCK1"
VERSION = 1
MODEL_KEYS = ("N", "Lx", "Ly", "D", "chi", "matter", "complex", "precision", "h", "g", "J", "m", "Q")


class CheckpointError(ValueError):
    """A checkpoint file that is damaged or belongs to another model."""


@dataclass
class Checkpoint:
    model: dict
    params: np.ndarray          # (n_params,) float64 or complex128
    configs: np.ndarray         # (n_chains, cfg_len) int8
    step: int                   # index of the next step to run
    seed: int                   # base seed of the run
    extra: dict = field(default_factory=dict)


def model_of(ctx) -> dict:
    """The model a context was created with, as stored in a checkpoint."""
    return {"N": int(ctx.N), "Lx": int(ctx.Lx), "Ly": int(ctx.Ly), "D": int(ctx.D), "chi": int(ctx.chi),
            "matter": bool(ctx.matter), "complex": bool(ctx.complex), "precision": str(ctx.precision),
            "h": float(ctx.h), "g": float(ctx.g), "J": float(ctx.J), "m": float(ctx.m),
            "Q": None if ctx.Q is None else [int(q) for q in np.asarray(ctx.Q).reshape(-1)]}


def _payload(params: np.ndarray, configs: np.ndarray) -> bytes:
    return params.tobytes() + configs.tobytes()


def write(path: str, ck: Checkpoint) -> None:
    """Write a Checkpoint (atomically: temporary file, then rename)."""
    cplx = bool(ck.model["complex"])
    params = np.ascontiguousarray(ck.params, dtype="<c16" if cplx else "<f8").reshape(-1)
    configs = np.ascontiguousarray(ck.configs, dtype=np.int8)
    if configs.ndim != 2:
        raise CheckpointError("configs must be (n_chains, cfg_len)")
    body = _payload(params, configs)
    header = {"version": VERSION, "model": ck.model, "n_params": int(params.size),
              "n_chains": int(configs.shape[0]), "cfg_len": int(configs.shape[1]),
              "step": int(ck.step), "seed": int(ck.seed), "extra": ck.extra,
              "sha256": hashlib.sha256(body).hexdigest()}
    hb = json.dumps(header, sort_keys=True).encode("utf-8")
    tmp = f"{path}.tmp{os.getpid()}"
    try:
        with open(tmp, "wb") as f:
            f.write(MAGIC)
            f.write(struct.pack("<I", len(hb)))
            f.write(hb)
            f.write(body)
            f.flush()
            os.fsync(f.fileno())
        os.replace(tmp, path)
    except BaseException:
        try:
            os.remove(tmp)
        except OSError:
            pass
        raise


def load(path: str) -> Checkpoint:
    """Read and verify a checkpoint file."""
    with open(path, "rb") as f:
        blob = f.read()
    if len(blob) < 12 or blob[:8] != MAGIC:
        raise CheckpointError(f"{path}: not a checkpoint file")
    (hl,) = struct.unpack("<I", blob[8:12])
    try:
        header = json.loads(blob[12:12 + hl].decode("utf-8"))
    except (UnicodeDecodeError, json.JSONDecodeError) as err:
        raise CheckpointError(f"{path}: damaged header") from err
    if not isinstance(header, dict) or header.get("version") != VERSION:
        raise CheckpointError(f"{path}: not a version-{VERSION} checkpoint header")
    body = blob[12 + hl:]
    try:
        if hashlib.sha256(body).hexdigest() != header["sha256"]:
            raise CheckpointError(f"{path}: payload does not match its checksum")
        cplx = bool(header["model"]["complex"])
        n, nc, cl = int(header["n_params"]), int(header["n_chains"]), int(header["cfg_len"])
        step, seed = int(header["step"]), int(header["seed"])
    except (KeyError, TypeError, ValueError) as err:
        raise CheckpointError(f"{path}: incomplete header") from err
    pb = n * (16 if cplx else 8)
    if len(body) != pb + nc * cl:
        raise CheckpointError(f"{path}: payload size does not match the header")
    params = np.frombuffer(body[:pb], dtype="<c16" if cplx else "<f8").astype(
        np.complex128 if cplx else np.float64)
    configs = np.frombuffer(body[pb:], dtype=np.int8).reshape(nc, cl).copy()
    return Checkpoint(model=header["model"], params=params, configs=configs, step=step, seed=seed,
                      extra=header.get("extra") or {})


def save(path: str, ctx, configs, step: int, seed: int, extra: dict | None = None) -> None:
    """Checkpoint a run: the context's parameters, the chains' configurations
    (device or host, (n_chains, cfg_len) int8), the index of the next step and
    the base seed (with the step it fixes each sample_batch call's seed under
    the run's rule, e.g. replicas.rank_seeds)."""
    cfg = configs.detach().cpu().numpy() if hasattr(configs, "detach") else np.asarray(configs)
    if cfg.ndim != 2 or cfg.shape[1] != ctx.cfg_len:
        raise CheckpointError(f"configs must be (n_chains, {ctx.cfg_len})")
    write(path, Checkpoint(model=model_of(ctx), params=ctx.get_tensors(), configs=cfg.astype(np.int8),
                           step=step, seed=seed, extra=dict(extra or {})))


def check_model(ctx, ck: Checkpoint) -> None:
    """Raise CheckpointError unless `ck` was written for the model of `ctx`."""
    want = model_of(ctx)
    diff = [k for k in MODEL_KEYS if want.get(k) != ck.model.get(k)]
    if diff:
        raise CheckpointError("checkpoint is for another model: " +
                              ", ".join(f"{k} {ck.model.get(k)!r} != {want.get(k)!r}" for k in diff))
    if ck.params.size != ctx.n_params or ck.configs.shape[1] != ctx.cfg_len:
        raise CheckpointError("checkpoint sizes do not match the context")


def restore(ctx, ck: Checkpoint, device="cuda"):
    """Load a checkpoint's parameters into `ctx` and return its configurations
    as an int8 tensor on `device`, ready for sample_batch at step `ck.step`."""
    import torch

    check_model(ctx, ck)
    ctx.set_tensors(ck.params)
    return torch.from_numpy(ck.configs.copy()).to(device)
