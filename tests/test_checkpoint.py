"""Checkpoint files (paper_1904_04825_gb300/checkpoint.py) on the host: exact
round trip of U and U_prev, header fields, and rejection of damaged files.
The module is loaded on its own, so these run without the CUDA library."""
import importlib.util
import json
import os

import numpy as np
import pytest

import synthetic as S

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _ckpt():
    spec = importlib.util.spec_from_file_location(
        "frjfnk_checkpoint", os.path.join(ROOT, "paper_1904_04825_gb300", "checkpoint.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def _state():
    xe, ye = S.stretched_mesh(5, 4, seed=2)
    X, Y = S.point_coords(xe, ye, 3)
    return (xe, ye), S.smooth_random_state(X, Y, seed=3, amp=0.1)


def test_round_trip_is_exact(tmp_path):
    ck = _ckpt()
    edges, U = _state()
    Up = U * (1 + 1e-3) - 1e-300            # values whose last bits matter
    pre = str(tmp_path / "run" / "step0042")
    h = ck.save(pre, U, t=2.1, step=42, scheme="BDF2", p=3, edges=edges, U_prev=Up, extra={"dt": 0.05})
    U2, Up2, h2 = ck.load(pre, device=None)
    assert U2.tobytes() == U.tobytes() and Up2.tobytes() == Up.tobytes()
    assert h2 == h
    assert h2["t"] == 2.1 and h2["step"] == 42 and h2["scheme"] == "BDF2" and h2["p"] == 3
    assert [np.array(e) for e in h2["edges"]][0].tobytes() == np.asarray(edges[0]).tobytes()
    assert h2["extra"] == {"dt": 0.05}


def test_single_state_and_3d_edges(tmp_path):
    ck = _ckpt()
    edges = S.uniform_mesh3d(2)
    X, Y, Z = S.point_coords3d(*edges, 1)
    V = S.TaylorGreen().state(X, Y, Z)
    pre = str(tmp_path / "tgv")
    ck.save(pre, V, t=0.0, step=0, scheme="ROW3", p=1, edges=edges)
    V2, none, h = ck.load(pre, device=None)
    assert none is None and V2.shape == V.shape and np.array_equal(V2, V)
    assert len(h["edges"]) == 3


def test_damaged_or_foreign_files_are_rejected(tmp_path):
    ck = _ckpt()
    edges, U = _state()
    pre = str(tmp_path / "c")
    ck.save(pre, U, t=1.0, step=1, scheme="ROW3", p=3, edges=edges)
    payload = str(tmp_path / json.load(open(pre + ".json"))["payload"])
    raw = bytearray(open(payload, "rb").read())
    raw[100] ^= 1
    open(payload, "wb").write(bytes(raw))
    with pytest.raises(ValueError, match="SHA-256"):
        ck.load(pre, device=None)
    h = json.load(open(pre + ".json"))
    h["format"] = "something-else"
    json.dump(h, open(pre + ".json", "w"))
    with pytest.raises(ValueError, match="header"):
        ck.load(pre, device=None)
    with pytest.raises(TypeError):
        ck.save(pre, U.astype(np.float32), t=0.0, step=0, scheme="ROW3", p=3, edges=edges)


def test_interrupted_save_leaves_the_previous_checkpoint_loadable(tmp_path, monkeypatch):
    """A save that dies after writing its payload (here: the header rename
    fails) or while writing it leaves the earlier checkpoint at the same
    prefix intact and loadable; a completed save removes the old payload."""
    ck = _ckpt()
    edges, U = _state()
    pre = str(tmp_path / "c")
    ck.save(pre, U, t=1.0, step=10, scheme="ROW3", p=3, edges=edges)
    first_payload = json.load(open(pre + ".json"))["payload"]
    real_replace = os.replace

    def dies_on_header(src, dst):
        if dst.endswith(".json"):
            raise OSError("interrupted")
        return real_replace(src, dst)
    monkeypatch.setattr(ck.os, "replace", dies_on_header)
    with pytest.raises(OSError):
        ck.save(pre, U * 2.0, t=2.0, step=20, scheme="ROW3", p=3, edges=edges)
    U1, _, h1 = ck.load(pre, device=None)
    assert h1["step"] == 10 and np.array_equal(U1, U)

    def dies_in_payload(src, dst):
        raise OSError("interrupted")
    monkeypatch.setattr(ck.os, "replace", dies_in_payload)
    with pytest.raises(OSError):
        ck.save(pre, U * 3.0, t=3.0, step=30, scheme="ROW3", p=3, edges=edges)
    U1, _, h1 = ck.load(pre, device=None)
    assert h1["step"] == 10 and np.array_equal(U1, U)

    monkeypatch.setattr(ck.os, "replace", real_replace)
    ck.save(pre, U * 4.0, t=4.0, step=40, scheme="ROW3", p=3, edges=edges)
    U4, _, h4 = ck.load(pre, device=None)
    assert h4["step"] == 40 and np.array_equal(U4, U * 4.0)
    assert not os.path.exists(str(tmp_path / first_payload))
