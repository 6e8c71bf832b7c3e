"""Field checkpoints: the state of a run (B on faces, v at centres) written as raw float64 arrays
behind a JSON header, for restarting a run or handing its fields to another program.

File layout: the header is one line of UTF-8 JSON, ended by a newline and padded with spaces so
that the arrays start at a multiple of 64 bytes; then each array, C order, little-endian float64,
at the offset the header gives (each also 64-byte aligned). Header keys: "format"
("mhd-fields"), "version" (1), "grid" (nr, nt, np, r0, r1, stretch), "step", "time", "arrays"
(name, shape, dtype "<f8", offset, nbytes, in file order) and "meta" (any JSON the caller passes,
e.g. the run's parameters). Shapes are the library's field layouts: br [nr+1][nt][np],
bt [nr][nt+1][np], bp, vr, vt, vp [nr][nt][np].
"""
from __future__ import annotations

import json
import os

import numpy as np

FORMAT = "mhd-fields"
VERSION = 1
ALIGN = 64
NAMES = ("br", "bt", "bp", "vr", "vt", "vp")


def field_shapes(nr: int, nt: int, np_: int) -> dict:
    return dict(br=(nr + 1, nt, np_), bt=(nr, nt + 1, np_), bp=(nr, nt, np_), vr=(nr, nt, np_),
                vt=(nr, nt, np_), vp=(nr, nt, np_))


def _host(a) -> np.ndarray:
    if hasattr(a, "detach"):   # a torch tensor, on the device or the host
        a = a.detach().cpu().numpy()
    return np.ascontiguousarray(a, dtype="<f8")


def _pad(n: int) -> int:
    return (n + ALIGN - 1) // ALIGN * ALIGN


def save(path: str, desc, fields: dict, step: int = 0, time: float = 0.0, meta: dict | None = None) -> dict:
    """Write `fields` (br, bt, bp, vr, vt, vp: torch tensors or numpy arrays in the library's
    layouts for grid `desc`) to `path`, through a temporary file renamed into place. Returns the
    header."""
    shapes = field_shapes(desc.nr, desc.nt, desc.np)
    missing = [k for k in NAMES if k not in fields]
    if missing:
        raise ValueError(f"checkpoint: missing fields {missing}")
    host = {k: _host(fields[k]) for k in NAMES}
    for k in NAMES:
        if host[k].shape != shapes[k]:
            raise ValueError(f"checkpoint: {k} has shape {host[k].shape}, the grid needs {shapes[k]}")
    arrays = []
    header = dict(format=FORMAT, version=VERSION,
                  grid=dict(nr=desc.nr, nt=desc.nt, np=desc.np, r0=desc.r0, r1=desc.r1, stretch=desc.stretch),
                  step=int(step), time=float(time), arrays=arrays, meta=meta or {})
    # the header's own length fixes the offsets: lay out with a first guess, then settle
    start = 0
    for _ in range(4):
        arrays.clear()
        off = start
        for k in NAMES:
            arrays.append(dict(name=k, shape=list(shapes[k]), dtype="<f8", offset=off, nbytes=host[k].nbytes))
            off = _pad(off + host[k].nbytes)
        text = json.dumps(header, separators=(",", ":"))
        need = _pad(len(text.encode()) + 1)
        if need == start:
            break
        start = need
    line = text.encode()
    if len(line) + 1 > start:
        raise RuntimeError("checkpoint: header layout did not settle")
    tmp = path + ".tmp"
    with open(tmp, "wb") as fh:
        fh.write(line + b" " * (start - len(line) - 1) + b"\n")
        for a in arrays:
            fh.seek(a["offset"])
            fh.write(host[a["name"]].tobytes())
        end = max(a["offset"] + a["nbytes"] for a in arrays)
        fh.truncate(end)
    os.replace(tmp, path)
    return header


def read_header(path: str) -> dict:
    with open(path, "rb") as fh:
        line = fh.readline(1 << 20)
    try:
        header = json.loads(line.decode())
    except (UnicodeDecodeError, json.JSONDecodeError) as e:
        raise ValueError(f"checkpoint: {path} does not start with a JSON header") from e
    if header.get("format") != FORMAT or header.get("version") != VERSION:
        raise ValueError(f"checkpoint: {path} is not a version-{VERSION} {FORMAT} file")
    return header


def load(path: str, device=None) -> tuple[dict, dict]:
    """(header, fields): numpy arrays, or torch tensors on `device` when one is given."""
    header = read_header(path)
    g = header["grid"]
    shapes = field_shapes(g["nr"], g["nt"], g["np"])
    size = os.path.getsize(path)
    out = {}
    with open(path, "rb") as fh:
        for a in header["arrays"]:
            k = a["name"]
            if k not in shapes or tuple(a["shape"]) != shapes[k] or a["dtype"] != "<f8":
                raise ValueError(f"checkpoint: array {k} does not match the grid in the header")
            n = int(np.prod(a["shape"])) * 8
            if a["nbytes"] != n or a["offset"] % ALIGN or a["offset"] + n > size:
                raise ValueError(f"checkpoint: array {k} lies outside the file")
            fh.seek(a["offset"])
            out[k] = np.frombuffer(fh.read(n), dtype="<f8").reshape(a["shape"]).copy()
    if set(out) != set(NAMES):
        raise ValueError("checkpoint: the file does not hold all six fields")
    if device is not None:
        import torch
        out = {k: torch.from_numpy(v).to(device) for k, v in out.items()}
    return header, out
