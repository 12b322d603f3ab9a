"""Checkpoint and resume of a time integration.

A checkpoint is two files: a payload ``<prefix>.<hash>.bin`` holds the state
U (and, for BDF2, the previous state U_prev) as raw little-endian float64
bytes in the library's layout, named after the first 16 hex digits of its
SHA-256; ``<prefix>.json`` holds the header: format tag, time, step count,
scheme, degree, mesh edges, array shapes, byte offsets, the payload's file
name and its SHA-256.  Loading checks the tag, the sizes and the hash.

Saving is safe against interruption: the new payload is written under its
own name, then the header is replaced atomically (written to a temporary
file and renamed over the old one), and only then is the previous payload
removed.  At every moment the header names a complete payload, so a save
that dies half way leaves the previous checkpoint loadable.

The steppers carry no state between steps except the previous-step guess
history (``guess = 1``), which a resumed context starts without, and BDF2's
U_prev, which the checkpoint holds.  With the default zero guess, stepping
on from a loaded checkpoint therefore reproduces the uninterrupted run bit
for bit (every reduction on the device is deterministic).
"""
from __future__ import annotations

import hashlib
import json
import os

import numpy as np

FORMAT = "frjfnk-checkpoint-1"


def _host(a) -> np.ndarray:
    """float64 C-contiguous host copy of a torch tensor or array."""
    if hasattr(a, "detach"):
        a = a.detach().cpu().numpy()
    a = np.ascontiguousarray(a)
    if a.dtype != np.float64:
        raise TypeError("checkpoint arrays must be float64")
    return a.astype("<f8", copy=False)


def save(prefix: str, U, *, t: float, step: int, scheme: str, p: int, edges, U_prev=None,
         extra: dict | None = None) -> dict:
    """Write the payload ``prefix.<hash>.bin`` and the header ``prefix.json``
    (replacing an earlier checkpoint at ``prefix`` only once the new one is
    complete); returns the header.

    ``edges``: the mesh's edge arrays (2 for quadrilaterals, 3 for
    hexahedra).  ``extra``: any JSON-serialisable fields to keep with it."""
    arrays = [("U", _host(U))]
    if U_prev is not None:
        arrays.append(("U_prev", _host(U_prev)))
    header = {"format": FORMAT, "t": float(t), "step": int(step), "scheme": str(scheme), "p": int(p),
              "edges": [np.asarray(e, dtype=np.float64).tolist() for e in edges],
              "arrays": [], "extra": extra or {}}
    h = hashlib.sha256()
    off = 0
    parts = []
    for name, a in arrays:
        b = a.tobytes()
        h.update(b)
        parts.append(b)
        header["arrays"].append({"name": name, "shape": list(a.shape), "offset": off, "nbytes": len(b)})
        off += len(b)
    header["sha256"] = h.hexdigest()
    folder = os.path.dirname(os.path.abspath(prefix))
    os.makedirs(folder, exist_ok=True)
    base = os.path.basename(prefix)
    header["payload"] = f"{base}.{header['sha256'][:16]}.bin"
    old_payload = None
    if os.path.exists(prefix + ".json"):
        try:
            old_payload = _payload_path(prefix, _read_header(prefix))
        except (OSError, ValueError):
            old_payload = None       # an unreadable old header: leave its payload alone
    new_payload = os.path.join(folder, header["payload"])
    _write_atomic(new_payload, lambda f: [f.write(b) for b in parts], binary=True)
    _write_atomic(prefix + ".json", lambda f: json.dump(header, f, indent=1), binary=False)
    if old_payload and os.path.abspath(old_payload) != os.path.abspath(new_payload) and os.path.exists(old_payload):
        os.remove(old_payload)
    return header


def _write_atomic(path: str, write, binary: bool):
    """Write through a temporary file in the same folder, flush it to disk,
    then rename it over ``path`` (a rename within a folder is atomic)."""
    tmp = path + ".tmp"
    with open(tmp, "wb" if binary else "w") as f:
        write(f)
        f.flush()
        os.fsync(f.fileno())
    os.replace(tmp, path)


def _read_header(prefix: str) -> dict:
    with open(prefix + ".json") as f:
        return json.load(f)


def _payload_path(prefix: str, header: dict) -> str:
    """The payload the header names (``<prefix>.bin`` for headers written
    before payloads were named after their hash)."""
    name = header.get("payload")
    if not name:
        return prefix + ".bin"
    if os.path.basename(name) != name:
        raise ValueError("checkpoint payload name must be a plain file name")
    return os.path.join(os.path.dirname(os.path.abspath(prefix)), name)


def load(prefix: str, device: str | None = "cuda"):
    """Read a checkpoint: returns ``(U, U_prev or None, header)``, the
    arrays as torch tensors on ``device`` (NumPy arrays if device is None).
    Raises ValueError if the header or the payload does not check out."""
    header = _read_header(prefix)
    if header.get("format") != FORMAT:
        raise ValueError(f"not a {FORMAT} header: {header.get('format')!r}")
    with open(_payload_path(prefix, header), "rb") as f:
        payload = f.read()
    if hashlib.sha256(payload).hexdigest() != header["sha256"]:
        raise ValueError("checkpoint payload does not match its SHA-256")
    out = {}
    for a in header["arrays"]:
        n = int(np.prod(a["shape"])) * 8
        if a["nbytes"] != n or a["offset"] + n > len(payload):
            raise ValueError(f"array {a['name']}: size does not match its shape")
        arr = np.frombuffer(payload, dtype="<f8", count=n // 8, offset=a["offset"]).reshape(a["shape"])
        out[a["name"]] = arr.astype(np.float64)
    if "U" not in out:
        raise ValueError("checkpoint holds no state U")
    if device is not None:
        import torch
        out = {k: torch.from_numpy(v).to(device) for k, v in out.items()}
    return out["U"], out.get("U_prev"), header
