"""Checkpoint files for the two optimisations of the method: the per-batch
fit of complexes (Sec. 4.1 Eq. 4-5, Adam over the Sec. 5.1 schedule) and the
learned initializer's network.

A checkpoint is one file:

    b"DISKCKPT"                      magic, 8 bytes
    u32 version (1), u32 header bytes (little endian)
    header: UTF-8 JSON {"kind", "meta", "arrays": [{"name", "dtype", "shape",
            "offset", "nbytes"}]}, offsets relative to the data section
    zero padding to a multiple of 16 bytes
    data section: the arrays' little-endian bytes, each 16-byte aligned
    u32 CRC-32 of every byte before it

Files are written to a temporary name beside the target and renamed over it,
so an interrupted save leaves the previous checkpoint intact.  `load` checks
the magic, the version, the sizes and the CRC before it returns anything.

`fit_with_checkpoints` runs a batch fit in segments through
`disk_fit_resume`, saving (theta, Adam moments, step) after every segment and
continuing from the file when one is present; the result is bit for bit the
uninterrupted fit's (same launch configuration).
"""
from __future__ import annotations

import json
import os
import struct
import threading
import zlib

import numpy as np

MAGIC = b"DISKCKPT"
VERSION = 1
_DTYPES = {"f4": np.float32, "i4": np.int32, "u1": np.uint8}


class CheckpointError(ValueError):
    """A checkpoint file that is malformed, truncated, corrupted or of
    another kind than the caller asked for."""


def _pad16(n: int) -> int:
    return (n + 15) // 16 * 16


def save(path: str, kind: str, meta: dict, arrays: dict) -> None:
    """Writes `arrays` (name -> array of float32, int32 or uint8) and the
    JSON-serialisable `meta` as a checkpoint of `kind`, atomically."""
    descs, blobs, off = [], [], 0
    for name, a in arrays.items():
        a = np.asarray(a, order="C")
        code = next((c for c, t in _DTYPES.items() if a.dtype == t), None)
        if code is None:
            raise TypeError(f"array {name!r}: dtype {a.dtype} not storable")
        raw = a.astype(a.dtype.newbyteorder("<"), copy=False).tobytes()
        descs.append({"name": name, "dtype": code, "shape": list(a.shape), "offset": off,
                      "nbytes": len(raw)})
        blobs.append(raw + b"\0" * (_pad16(len(raw)) - len(raw)))
        off += _pad16(len(raw))
    header = json.dumps({"kind": kind, "meta": meta, "arrays": descs}).encode()
    head = MAGIC + struct.pack("<II", VERSION, len(header)) + header
    head += b"\0" * (_pad16(len(head)) - len(head))
    crc = zlib.crc32(head)
    for b in blobs:
        crc = zlib.crc32(b, crc)
    tmp = f"{path}.tmp{os.getpid()}.{threading.get_ident()}"
    with open(tmp, "wb") as f:
        f.write(head)
        for b in blobs:
            f.write(b)
        f.write(struct.pack("<I", crc & 0xFFFFFFFF))
        f.flush()
        os.fsync(f.fileno())
    os.replace(tmp, path)


def load(path: str, kind: str | None = None):
    """Reads a checkpoint: returns (kind, meta, {name: array}).  Raises
    CheckpointError for a bad magic, version, size or CRC, or when `kind` is
    given and differs."""
    with open(path, "rb") as f:
        buf = f.read()
    if len(buf) < 20 or buf[:8] != MAGIC:
        raise CheckpointError(f"{path}: not a checkpoint")
    version, hlen = struct.unpack_from("<II", buf, 8)
    if version != VERSION:
        raise CheckpointError(f"{path}: version {version}, expected {VERSION}")
    if zlib.crc32(buf[:-4]) & 0xFFFFFFFF != struct.unpack_from("<I", buf, len(buf) - 4)[0]:
        raise CheckpointError(f"{path}: CRC mismatch (corrupted or truncated)")
    if 16 + hlen > len(buf) - 4:
        raise CheckpointError(f"{path}: truncated header")
    try:
        header = json.loads(buf[16:16 + hlen].decode())
    except (UnicodeDecodeError, json.JSONDecodeError) as e:
        raise CheckpointError(f"{path}: bad header ({e})") from None
    if kind is not None and header.get("kind") != kind:
        raise CheckpointError(f"{path}: a {header.get('kind')!r} checkpoint, not {kind!r}")
    base, end = _pad16(16 + hlen), len(buf) - 4
    arrays = {}
    for d in header["arrays"]:
        t = _DTYPES.get(d["dtype"])
        n = int(np.prod(d["shape"], dtype=np.int64)) * (np.dtype(t).itemsize if t else 0)
        lo = base + int(d["offset"])
        if t is None or n != d["nbytes"] or lo < base or lo + n > end:
            raise CheckpointError(f"{path}: bad array entry {d.get('name')!r}")
        arrays[d["name"]] = np.frombuffer(buf, dtype=np.dtype(t).newbyteorder("<"), count=n //
                                          np.dtype(t).itemsize, offset=lo).astype(t).reshape(
                                              d["shape"])
    return header["kind"], header["meta"], arrays


# ---- the fit ------------------------------------------------------------------

def targets_fingerprint(packed_host: np.ndarray) -> int:
    """CRC-32 of a packed target batch's float32 bytes: a resumed fit checks
    that it continues on the batch it started on."""
    return zlib.crc32(np.ascontiguousarray(packed_host, dtype="<f4").tobytes()) & 0xFFFFFFFF


def save_fit(path: str, *, sizes, L: int, T: int, step: int, total_steps: int, lr0: float,
             lr1: float, loss: int, eps: float, fingerprint: int, state, theta) -> None:
    """Fit checkpoint after `step` of `total_steps` steps: the optimiser state
    [batch, 3, L*T*3] and the complex [batch, L, T, 3] (host arrays or
    tensors)."""
    def host(x):
        return x.detach().cpu().numpy() if hasattr(x, "detach") else np.asarray(x)
    meta = {"L": int(L), "T": int(T), "step": int(step), "total_steps": int(total_steps),
            "lr0": float(lr0), "lr1": float(lr1), "loss": int(loss), "eps": float(eps),
            "fingerprint": int(fingerprint)}
    save(path, "fit", meta, {"sizes": np.asarray(sizes, dtype=np.int32),
                             "state": host(state).astype(np.float32, copy=False),
                             "theta": host(theta).astype(np.float32, copy=False)})


def load_fit(path: str):
    """(meta, sizes, state, theta) of a fit checkpoint, shapes checked."""
    _, meta, a = load(path, "fit")
    sizes, state, theta = a.get("sizes"), a.get("state"), a.get("theta")
    if sizes is None or state is None or theta is None:
        raise CheckpointError(f"{path}: missing arrays")
    b, L, T = len(sizes), meta["L"], meta["T"]
    if state.shape != (b, 3, L * T * 3) or theta.shape != (b, L, T, 3):
        raise CheckpointError(f"{path}: array shapes do not match the batch")
    if not 0 <= meta["step"] <= meta["total_steps"]:
        raise CheckpointError(f"{path}: step {meta['step']} outside the schedule")
    return meta, sizes, state, theta


def fit_with_checkpoints(path: str, packed, sizes, L: int, T: int, steps: int, every: int,
                         lr0: float = 1e-3, lr1: float = 1e-4, init: int = 1,
                         loss: int = 0, eps: float = 0.0, seed: int = 0, theta=None,
                         stop_after: int | None = None):
    """Batch fit of `steps` steps (as `disk.fit`) run `every` steps at a time
    through `disk_fit_resume`, with a checkpoint written to `path` after every
    segment.  When `path` holds a checkpoint of this batch (same sizes, L, T,
    schedule and target bytes) the fit continues from it; one of another
    batch raises CheckpointError.  `stop_after` ends the call after that many
    segments (an interrupted run).  Returns (theta, final loss, step reached)
    with device tensors."""
    import torch

    from . import disk
    if every < 1:
        raise ValueError("every >= 1 required")
    batch = len(sizes)
    fp = targets_fingerprint(packed.detach().cpu().numpy())
    dev = packed.device
    state = torch.empty((batch, 3, L * T * 3), device=dev, dtype=torch.float32)
    if os.path.exists(path):
        meta, s_sizes, s_state, s_theta = load_fit(path)
        want = {"L": L, "T": T, "total_steps": steps, "loss": loss, "fingerprint": fp}
        if list(s_sizes) != list(sizes) or any(meta[k] != v for k, v in want.items()) or \
                meta["lr0"] != np.float32(lr0) or meta["lr1"] != np.float32(lr1):
            raise CheckpointError(f"{path}: a checkpoint of another fit")
        step = meta["step"]
        state.copy_(torch.from_numpy(s_state))
        theta = torch.from_numpy(s_theta).to(dev)
    else:
        if init == disk.INIT_GIVEN and theta is None:
            raise ValueError("INIT_GIVEN needs theta")
        theta = theta.clone() if theta is not None else \
            torch.zeros((batch, L, T, 3), device=dev, dtype=torch.float32)
        step = 0
    final = None
    segments = 0
    while step < steps or final is None:
        n = min(every, steps - step)
        final, _ = disk.fit_resume(packed, sizes, state, theta, step, n, steps, lr0, lr1, init,
                                   loss, eps, seed)
        step += n
        save_fit(path, sizes=sizes, L=L, T=T, step=step, total_steps=steps,
                 lr0=float(np.float32(lr0)), lr1=float(np.float32(lr1)), loss=loss, eps=eps,
                 fingerprint=fp, state=state, theta=theta)
        segments += 1
        if stop_after is not None and segments >= stop_after:
            break
    return theta, final, step


# ---- the learned initializer's network ---------------------------------------

def save_mlp(path: str, *, shape, step: int, params, m, v) -> None:
    """Network checkpoint: shape (n_in, hidden, depth, n_out), the Adam step
    count, and the flat parameter array with its two Adam moments (host arrays
    or tensors, float32, equal lengths)."""
    def host(x):
        return x.detach().cpu().numpy() if hasattr(x, "detach") else np.asarray(x)
    arrs = {k: host(x).astype(np.float32, copy=False).reshape(-1)
            for k, x in (("params", params), ("m", m), ("v", v))}
    if len({a.size for a in arrs.values()}) != 1:
        raise ValueError("params, m and v must have the same length")
    save(path, "mlp", {"shape": [int(x) for x in shape], "step": int(step)}, arrs)


def load_mlp(path: str):
    """(shape, step, params, m, v) of a network checkpoint."""
    _, meta, a = load(path, "mlp")
    shape, step = meta.get("shape"), meta.get("step")
    if not (isinstance(shape, list) and len(shape) == 4 and all(isinstance(x, int) and x > 0
                                                                for x in shape)):
        raise CheckpointError(f"{path}: bad network shape {shape!r}")
    if not isinstance(step, int) or step < 0:
        raise CheckpointError(f"{path}: bad step {step!r}")
    p, m, v = a.get("params"), a.get("m"), a.get("v")
    if p is None or m is None or v is None or not (p.ndim == m.ndim == v.ndim == 1) or \
            not (p.size == m.size == v.size):
        raise CheckpointError(f"{path}: parameter arrays missing or of unequal length")
    return tuple(shape), step, p, m, v

