"""On-disk state for long runs, and a per-step record of the statistics.

save_state / load_state: a phase field as raw little-endian values (``<name>.bin``, x
fastest, [nz][ny][nx]) beside a JSON header (``<name>.json``: shape, dtype, step, time and
whatever run parameters the caller passes), so that a long run can stop and resume.  Both
files are written to temporary names and renamed into place, data first; the header names
the byte count and the SHA-256 of the data, so a truncated file, or data and header left
from two different saves by a process that died between the two renames, is refused on
load.

RunLog: appends one JSON line per record with the step, time, mass, the mass drift against
the first record, min, max and both violation counts, as cdi.Grid.stats() reports them.
"""
from __future__ import annotations

import hashlib
import json
import os

import numpy as np

_DTYPES = {"f32": np.dtype("<f4"), "f64": np.dtype("<f8")}


def _paths(path):
    base = os.fspath(path)
    return base + ".bin", base + ".json"


def save_state(path, phi, step: int, t: float, **params) -> None:
    """Write phi (a numpy array or a torch tensor, float32 or float64, shape (nz, ny, nx))
    and its header.  ``params`` must be JSON-serialisable (eps, gamma, dt, seed, ...)."""
    if hasattr(phi, "detach"):
        phi = phi.detach().cpu().numpy()
    a = np.ascontiguousarray(phi)
    if a.ndim != 3:
        raise ValueError(f"phi must have shape (nz, ny, nx), got {a.shape}")
    key = {np.dtype(np.float32): "f32", np.dtype(np.float64): "f64"}.get(a.dtype)
    if key is None:
        raise ValueError(f"phi must be float32 or float64, got {a.dtype}")
    fbin, fjson = _paths(path)
    data = a.astype(_DTYPES[key], copy=False).tobytes()
    header = {"shape": list(a.shape), "dtype": key, "bytes": len(data),
              "sha256": hashlib.sha256(data).hexdigest(), "step": int(step), "t": float(t),
              "params": params}
    tbin, tjson = fbin + ".tmp", fjson + ".tmp"
    with open(tbin, "wb") as f:
        f.write(data)
        f.flush()
        os.fsync(f.fileno())
    with open(tjson, "w") as f:
        json.dump(header, f, indent=1)
        f.flush()
        os.fsync(f.fileno())
    os.replace(tbin, fbin)
    os.replace(tjson, fjson)


def load_state(path):
    """Read a state written by save_state: returns (phi as a numpy array, header dict).
    Raises ValueError if the data and the header disagree."""
    fbin, fjson = _paths(path)
    with open(fjson) as f:
        header = json.load(f)
    dt = _DTYPES.get(header.get("dtype"))
    if dt is None:
        raise ValueError(f"unknown dtype in header: {header.get('dtype')!r}")
    shape = tuple(int(n) for n in header["shape"])
    want = int(np.prod(shape)) * dt.itemsize
    if os.path.getsize(fbin) != want or header.get("bytes") != want:
        raise ValueError(f"{fbin}: {os.path.getsize(fbin)} bytes on disk, header expects {want}")
    raw = open(fbin, "rb").read()
    if hashlib.sha256(raw).hexdigest() != header.get("sha256"):
        raise ValueError(f"{fbin}: data does not match the header's SHA-256 (a save was interrupted)")
    phi = np.frombuffer(raw, dtype=dt).reshape(shape).astype(dt.newbyteorder("="), copy=True)
    return phi, header


class RunLog:
    """JSON-lines record of a run's statistics (one line per call of :meth:`record`)."""

    def __init__(self, path):
        self.path = os.fspath(path)
        self.mass0 = None

    def record(self, step: int, t: float, stats: dict, **extra) -> dict:
        """Append one record from a cdi statistics dict; returns the record written."""
        if self.mass0 is None:
            self.mass0 = stats["mass"]
        drift = (stats["mass"] - self.mass0) / self.mass0 if self.mass0 else 0.0
        rec = {"step": int(step), "t": float(t), "mass": stats["mass"], "mass_drift_rel": drift,
               "min": stats["min"], "max": stats["max"], "n_strict": int(stats["n_strict"]),
               "n_tol": int(stats["n_tol"])}
        rec.update(extra)
        with open(self.path, "a") as f:
            f.write(json.dumps(rec) + "\n")
        return rec
