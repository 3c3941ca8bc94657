"""Particle frame files read on the host through the library (no GPU): the
numpy writer and the C reader agree on the layout, FP32 frames widen exactly,
ids and header fields come through, and malformed files are refused."""
import struct

import numpy as np
import pytest

from paper_2311_08927_gb300 import build as B
from paper_2311_08927_gb300 import chad as CH
from paper_2311_08927_gb300 import frames as F


@pytest.fixture(scope="module", autouse=True)
def _lib():
    B.build()
    CH.lib()


def _pos(n, seed):
    rng = np.random.default_rng(seed)
    return rng.uniform(-0.1, 0.3, (3, n))


def test_fp64_frame_round_trip(tmp_path):
    pos = _pos(1001, 1)
    f = tmp_path / "a.frm"
    F.write_frame(f, pos, step=17, time_s=8.5)
    r = CH.chad_read_frame(f)
    assert r["n"] == 1001 and r["step"] == 17 and r["time_s"] == 8.5 and r["id"] is None
    assert np.array_equal(r["pos"], pos)


def test_fp32_frame_with_velocities_and_ids(tmp_path):
    pos = _pos(777, 2)
    ids = np.random.default_rng(3).permutation(777).astype(np.uint32)
    vel = _pos(777, 4)
    f = tmp_path / "b.frm"
    F.write_frame(f, pos, ids=ids, vel=vel, dtype=np.float32, step=3)
    r = CH.chad_read_frame(f)
    assert np.array_equal(r["pos"], pos.astype(np.float32).astype(np.float64))
    assert np.array_equal(r["id"], ids.astype(np.int64))


def test_empty_frame(tmp_path):
    f = tmp_path / "e.frm"
    F.write_frame(f, np.zeros((3, 0)))
    assert CH.chad_read_frame(f)["n"] == 0


@pytest.mark.parametrize("damage", ["magic", "version", "dtype", "no_pos", "short", "missing"])
def test_malformed_frames_are_refused(tmp_path, damage):
    f = tmp_path / "c.frm"
    F.write_frame(f, _pos(50, 5), ids=np.arange(50, dtype=np.uint32))
    raw = bytearray(f.read_bytes())
    if damage == "magic":
        raw[0:1] = b"X"
    elif damage == "version":
        raw[8:12] = struct.pack("<I", 2)
    elif damage == "dtype":
        raw[12:16] = struct.pack("<I", 2)
    elif damage == "no_pos":
        raw[40:44] = struct.pack("<I", F.ID)
    elif damage == "short":
        raw = raw[:-8]
    if damage == "missing":
        f = tmp_path / "nothing.frm"
    else:
        f.write_bytes(bytes(raw))
    with pytest.raises(CH.ChadError):
        CH.chad_read_frame(f)
