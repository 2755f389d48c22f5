"""Host logic of the checkpoint files (fit state and network state): round
trips, and refusal of corrupted, truncated, mismatched or foreign files.  No
GPU: the arrays are host arrays."""
import os

import numpy as np
import pytest

from paper_2512_04556_gb300 import checkpoint as ck


def _arrays(seed=0):
    g = np.random.default_rng(seed)
    return {"a": g.standard_normal((3, 5, 7)).astype(np.float32),
            "sizes": np.array([9, 33, 129], dtype=np.int32),
            "bytes": g.integers(0, 256, 37).astype(np.uint8),
            "empty": np.zeros((0, 4), dtype=np.float32),
            "scalar": np.array(2.5, dtype=np.float32)}


def test_round_trip_is_exact(tmp_path):
    p = str(tmp_path / "x.ckpt")
    arrs = _arrays()
    arrs["special"] = np.array([np.nan, np.inf, -0.0, 1e-45], dtype=np.float32)
    ck.save(p, "demo", {"k": 3, "lr": 1e-3, "name": "x"}, arrs)
    kind, meta, got = ck.load(p)
    assert kind == "demo" and meta == {"k": 3, "lr": 1e-3, "name": "x"}
    assert set(got) == set(arrs)
    for k, a in arrs.items():
        assert got[k].dtype == a.dtype and got[k].shape == a.shape
        assert got[k].tobytes() == a.tobytes(), k
    # every array starts 16-byte aligned in the file
    with open(p, "rb") as f:
        size = len(f.read())
    assert size % 16 == 4
    assert not [n for n in os.listdir(tmp_path) if ".tmp" in n]


def test_every_flipped_byte_is_detected(tmp_path):
    p = str(tmp_path / "x.ckpt")
    ck.save(p, "demo", {"k": 1}, {"a": np.arange(40, dtype=np.float32)})
    raw = open(p, "rb").read()
    for i in range(0, len(raw), 7):
        bad = bytearray(raw)
        bad[i] ^= 0x10
        q = str(tmp_path / f"bad{i}.ckpt")
        open(q, "wb").write(bytes(bad))
        with pytest.raises(ck.CheckpointError):
            ck.load(q)


def test_truncated_and_foreign_files_are_refused(tmp_path):
    p = str(tmp_path / "x.ckpt")
    ck.save(p, "fit", {"k": 1}, {"a": np.arange(40, dtype=np.float32)})
    raw = open(p, "rb").read()
    for n in (0, 8, 19, len(raw) // 2, len(raw) - 1):
        q = str(tmp_path / f"t{n}.ckpt")
        open(q, "wb").write(raw[:n])
        with pytest.raises(ck.CheckpointError):
            ck.load(q)
    q = str(tmp_path / "other.bin")
    open(q, "wb").write(b"DISKBAS1" + raw[8:])
    with pytest.raises(ck.CheckpointError):
        ck.load(q)
    with pytest.raises(ck.CheckpointError, match="not 'mlp'"):
        ck.load(p, "mlp")


def test_failed_save_keeps_the_previous_file(tmp_path):
    p = str(tmp_path / "x.ckpt")
    ck.save(p, "demo", {}, {"a": np.ones(3, np.float32)})
    with pytest.raises(TypeError):
        ck.save(p, "demo", {}, {"a": np.ones(3, np.float64)})
    assert ck.load(p)[2]["a"].tolist() == [1.0, 1.0, 1.0]
    assert not [n for n in os.listdir(tmp_path) if ".tmp" in n]


def test_fit_checkpoint_round_trip_and_shape_checks(tmp_path):
    p = str(tmp_path / "fit.ckpt")
    g = np.random.default_rng(1)
    sizes, L, T = [9, 17, 33], 3, 5
    state = g.standard_normal((3, 3, L * T * 3)).astype(np.float32)
    theta = g.standard_normal((3, L, T, 3)).astype(np.float32)
    ck.save_fit(p, sizes=sizes, L=L, T=T, step=40, total_steps=100, lr0=1e-3, lr1=1e-4, loss=0,
                eps=0.0, fingerprint=1234, state=state, theta=theta)
    meta, s2, st2, th2 = ck.load_fit(p)
    assert list(s2) == sizes and meta["step"] == 40 and meta["total_steps"] == 100
    assert meta["fingerprint"] == 1234
    assert st2.tobytes() == state.tobytes() and th2.tobytes() == theta.tobytes()
    ck.save(p, "fit", dict(meta), {"sizes": np.array(sizes, np.int32), "state": state[:2],
                                   "theta": theta})
    with pytest.raises(ck.CheckpointError, match="shapes"):
        ck.load_fit(p)
    bad = dict(meta, step=101)
    ck.save(p, "fit", bad, {"sizes": np.array(sizes, np.int32), "state": state, "theta": theta})
    with pytest.raises(ck.CheckpointError, match="schedule"):
        ck.load_fit(p)


def test_targets_fingerprint_sees_one_bit():
    a = np.random.default_rng(2).standard_normal(1000).astype(np.float32)
    b = a.copy()
    b.view(np.uint32)[500] ^= 1
    assert ck.targets_fingerprint(a) != ck.targets_fingerprint(b)
    assert ck.targets_fingerprint(a) == ck.targets_fingerprint(a.copy())


def test_network_checkpoint_round_trip_and_checks(tmp_path):
    p = str(tmp_path / "mlp.ckpt")
    g = np.random.default_rng(3)
    params, m, v = (g.standard_normal(1000).astype(np.float32) for _ in range(3))
    ck.save_mlp(p, shape=(64, 16, 2, 12), step=7, params=params, m=m, v=v)
    shape, step, p2, m2, v2 = ck.load_mlp(p)
    assert shape == (64, 16, 2, 12) and step == 7
    assert p2.tobytes() == params.tobytes() and m2.tobytes() == m.tobytes()
    assert v2.tobytes() == v.tobytes()
    with pytest.raises(ValueError):
        ck.save_mlp(p, shape=(64, 16, 2, 12), step=7, params=params, m=m[:-1], v=v)
    ck.save(p, "mlp", {"shape": [64, 16, 2], "step": 1}, {"params": params, "m": m, "v": v})
    with pytest.raises(ck.CheckpointError, match="shape"):
        ck.load_mlp(p)
    ck.save(p, "mlp", {"shape": [64, 16, 2, 12], "step": -1}, {"params": params, "m": m, "v": v})
    with pytest.raises(ck.CheckpointError, match="step"):
        ck.load_mlp(p)


def test_concurrent_saves_leave_one_whole_file(tmp_path):
    """Threads saving the same path each write their own temporary file and
    rename it: the result is one of the saved checkpoints, whole."""
    import threading
    p = str(tmp_path / "x.ckpt")
    arrays = [np.full(5000, k, np.float32) for k in range(8)]
    ts = [threading.Thread(target=ck.save, args=(p, "demo", {"k": k}, {"a": arrays[k]}))
          for k in range(8)]
    for t in ts:
        t.start()
    for t in ts:
        t.join()
    _, meta, a = ck.load(p)
    assert a["a"].tolist() == arrays[meta["k"]].tolist()
    assert not [n for n in os.listdir(tmp_path) if ".tmp" in n]
