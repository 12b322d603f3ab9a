"""Checkpoint and resume of a time integration.

A checkpoint is two files: ``<prefix>.bin`` holds the state U (and, for
BDF2, the previous state U_prev) as raw little-endian float64 bytes in the
library's layout; ``<prefix>.json`` holds the header: format tag, time, step
count, scheme, degree, mesh edges, array shapes, byte offsets and the
SHA-256 of the payload.  Loading checks the tag, the sizes and the hash.

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
    """Write ``prefix.bin`` and ``prefix.json``; returns the header.

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
    os.makedirs(os.path.dirname(os.path.abspath(prefix)), exist_ok=True)
    with open(prefix + ".bin", "wb") as f:
        for name, a in arrays:
            b = a.tobytes()
            f.write(b)
            h.update(b)
            header["arrays"].append({"name": name, "shape": list(a.shape), "offset": off, "nbytes": len(b)})
            off += len(b)
    header["sha256"] = h.hexdigest()
    with open(prefix + ".json", "w") as f:
        json.dump(header, f, indent=1)
    return header


def load(prefix: str, device: str | None = "cuda"):
    """Read a checkpoint: returns ``(U, U_prev or None, header)``, the
    arrays as torch tensors on ``device`` (NumPy arrays if device is None).
    Raises ValueError if the header or the payload does not check out."""
    with open(prefix + ".json") as f:
        header = json.load(f)
    if header.get("format") != FORMAT:
        raise ValueError(f"not a {FORMAT} header: {header.get('format')!r}")
    with open(prefix + ".bin", "rb") as f:
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
