"""Storage of oracle end states for the long-run parity tests.

A golden file is an uncompressed ``.npz`` holding, per stored array,
``<name>.shape`` and ``<name>.data`` (zlib-compressed bytes), plus ``meta`` (a
JSON string).  The FP64 values are stored byte-plane shuffled (all first bytes,
then all second bytes, ...) so that the zlib stream sees the slowly varying
sign/exponent bytes together.  ``keep`` < 8 drops the 8 - keep low-order bytes
of every value after rounding to nearest at that boundary: 8 keep - 12
mantissa bits remain, so a stored value differs from the oracle's by at most
2^-(8 keep - 11) relative (keep = 6: 2^-37, about 7.3e-12), far below the
1e-9 relative-L1 tolerance of the tests that read it.  No arithmetic of the method lives here.
"""
from __future__ import annotations

import json
import zlib

import numpy as np


def _encode(a: np.ndarray, keep: int) -> bytes:
    bits = np.ascontiguousarray(a, dtype="<f8").view("<u8").ravel().copy()
    if keep < 8:
        drop = 8 * (8 - keep)
        half = np.uint64(1) << np.uint64(drop - 1)
        # round to nearest at the kept boundary; a carry into the exponent is
        # the correct rounding of the magnitude
        bits = (bits + half) >> np.uint64(drop) << np.uint64(drop)
    b = bits.view(np.uint8).reshape(-1, 8)[:, 8 - keep:]
    return zlib.compress(np.ascontiguousarray(b.T).tobytes(), 9)


def _decode(data: bytes, shape, keep: int) -> np.ndarray:
    n = int(np.prod(shape))
    planes = np.frombuffer(zlib.decompress(data), dtype=np.uint8).reshape(keep, n)
    b = np.zeros((n, 8), dtype=np.uint8)
    b[:, 8 - keep:] = planes.T
    return b.reshape(-1).view("<f8").reshape(shape).copy()


def save(path: str, arrays: dict, meta: dict, keep: int = 8) -> None:
    meta = dict(meta, keep=keep)
    out = {"meta": np.frombuffer(json.dumps(meta, sort_keys=True).encode(), dtype=np.uint8)}
    for name, a in arrays.items():
        out[name + ".shape"] = np.asarray(np.shape(a), dtype=np.int64)
        out[name + ".data"] = np.frombuffer(_encode(np.asarray(a), keep), dtype=np.uint8)
    np.savez(path, **out)


def load(path: str):
    """(arrays, meta) of a golden file."""
    z = np.load(path)
    meta = json.loads(bytes(z["meta"]).decode())
    keep = int(meta["keep"])
    arrays = {}
    for key in z.files:
        if key.endswith(".data"):
            name = key[:-5]
            arrays[name] = _decode(bytes(z[key]), tuple(z[name + ".shape"]), keep)
    return arrays, meta
