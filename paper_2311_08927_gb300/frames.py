"""Particle frame files: the writer side of the binary frame format that
``chad_load_frame`` reads (layout in include/chad.h).  An external CFD, or a
converter from its own output, writes one file per coupling step."""
from __future__ import annotations

import struct

import numpy as np

MAGIC = b"CHADFRM\0"
POS, VEL, ID = 1, 2, 4


def write_frame(path, pos, ids=None, vel=None, dtype=np.float64, step=0, time_s=0.0) -> None:
    """pos [3][n] (m) and optionally vel [3][n] (m/s) in `dtype` (float32 or
    float64), ids [n] (uint32: the library particle of each entry)."""
    dtype = np.dtype(dtype)
    if dtype not in (np.dtype(np.float32), np.dtype(np.float64)):
        raise ValueError("dtype must be float32 or float64")
    pos = np.asarray(pos)
    n = pos.shape[1]
    fields = POS | (VEL if vel is not None else 0) | (ID if ids is not None else 0)
    head = struct.pack("<8sIIQQdI5I", MAGIC, 1, dtype.itemsize, n, int(step), float(time_s),
                       fields, 0, 0, 0, 0, 0)
    assert len(head) == 64
    with open(path, "wb") as f:
        f.write(head)
        f.write(np.ascontiguousarray(pos, dtype=dtype.newbyteorder("<")).tobytes())
        if vel is not None:
            f.write(np.ascontiguousarray(vel, dtype=dtype.newbyteorder("<")).tobytes())
        if ids is not None:
            f.write(np.ascontiguousarray(ids, dtype="<u4").tobytes())
