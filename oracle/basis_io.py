"""Reader and writer of the basis file format, written independently of the
library's C implementation (test infrastructure: round trips check one
against the other).

Layout: b"DISKBAS1", little-endian uint32 version=1, dims, L, T, n0, n1
(n1 = 1 for one axis), float32 node values (n0, then n1 for two axes),
float32 theta [B][L][T][3], then the uint64 FNV-1a hash of all preceding
bytes (offset basis 0xcbf29ce484222325, prime 0x100000001b3).
"""
import struct

import numpy as np

MAGIC = b"DISKBAS1"


def fnv1a64(data: bytes) -> int:
    h = 0xCBF29CE484222325
    for b in data:
        h ^= b
        h = (h * 0x100000001B3) & 0xFFFFFFFFFFFFFFFF
    return h


def write(path, node_vals, theta):
    """node_vals: list of one or two increasing sequences; theta [B][L][T][3]."""
    axes = [np.asarray(v, dtype="<f4") for v in node_vals]
    th = np.ascontiguousarray(np.asarray(theta, dtype="<f4"))
    B, L, T, _ = th.shape
    n0 = len(axes[0])
    n1 = len(axes[1]) if len(axes) == 2 else 1
    assert B == n0 * n1
    body = MAGIC + struct.pack("<6I", 1, len(axes), L, T, n0, n1)
    body += b"".join(a.tobytes() for a in axes) + th.tobytes()
    with open(path, "wb") as f:
        f.write(body + struct.pack("<Q", fnv1a64(body)))


def read(path):
    """Returns (node_vals list, theta float32 [B][L][T][3])."""
    data = open(path, "rb").read()
    if data[:8] != MAGIC:
        raise ValueError("bad magic")
    ver, dims, L, T, n0, n1 = struct.unpack("<6I", data[8:32])
    if ver != 1 or dims not in (1, 2):
        raise ValueError("bad header")
    nv = n0 + (n1 if dims == 2 else 0)
    B = n0 * n1
    need = 32 + 4 * (nv + B * L * T * 3) + 8
    if len(data) != need:
        raise ValueError("size mismatch")
    if struct.unpack("<Q", data[-8:])[0] != fnv1a64(data[:-8]):
        raise ValueError("checksum mismatch")
    vals = np.frombuffer(data, "<f4", nv, 32)
    theta = np.frombuffer(data, "<f4", B * L * T * 3, 32 + 4 * nv).reshape(B, L, T, 3)
    axes = [vals[:n0].copy()] + ([vals[n0:].copy()] if dims == 2 else [])
    return axes, theta.copy()
