"""Helpers for the GPU parity tests: layouts via the oracle's index maps, normwise error
metrics, and extraction of individual lines from a direction layout on the device."""
import numpy as np
import torch

import oracle

SZ = 32
TORCH = {"f64": torch.float64, "f32": torch.float32}
TOL = {"f64": 1e-12, "f32": 1e-5}


def rel_errors(got, ref):
    got = np.asarray(got, dtype=np.float64); ref = np.asarray(ref, dtype=np.float64)
    d = got - ref
    mx = float(np.max(np.abs(d)) / max(np.max(np.abs(ref)), 1e-300))
    rms = float(np.linalg.norm(d) / max(np.linalg.norm(ref), 1e-300))
    return mx, rms


def to_device_layout(cart, direction, dtype):
    lay = oracle.to_layout(cart, direction, SZ)
    return torch.from_numpy(np.ascontiguousarray(lay)).to(device="cuda", dtype=TORCH[dtype])


def from_device_layout(t, direction, shape):
    return oracle.from_layout(t.double().cpu().numpy(), direction, shape, SZ)


def line_index(direction, shape, lines, n):
    """Flat indices (len(lines), n) of whole lines in the direction layout."""
    lines = torch.as_tensor(lines, dtype=torch.int64)
    g, s = lines // SZ, lines % SZ
    j = torch.arange(n, dtype=torch.int64)
    return (s[:, None] + SZ * (j[None, :] + n * g[:, None]))


def gather_lines(t, direction, shape, lines):
    n = {"x": shape[2], "y": shape[1], "z": shape[0]}[direction]
    idx = line_index(direction, shape, lines, n).to(t.device)
    return t.reshape(-1)[idx.reshape(-1)].reshape(len(lines), n)


def sample_lines(nlines, count, seed):
    rng = np.random.default_rng(seed)
    pick = set(rng.choice(nlines, size=min(count, nlines), replace=False).tolist())
    pick.update({0, nlines - 1, min(31, nlines - 1), nlines // 2})
    return sorted(pick)


def report(case, **values):
    """Print one measured parity figure (a JSON line tagged PARITY; shown with ``pytest -s``)."""
    import json
    print("PARITY " + json.dumps(dict(case=case, **{k: (float(v) if isinstance(v, (float, np.floating)) else v)
                                                   for k, v in values.items()})))
