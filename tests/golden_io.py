"""Reader for the hand-worked fixtures in tests/golden/."""
import glob
import os
import struct

import numpy as np

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _parse_val(tok: str, dtype: str) -> int:
    if dtype == "u32":
        return int(tok)
    if dtype == "f32hex":
        return int(tok, 16)
    return struct.unpack("<I", struct.pack("<f", float(tok)))[0]


def load(path: str):
    lines = [l.strip() for l in open(path) if l.strip() and not l.startswith("#")]
    dtype = lines[0].split()[1]
    n = int(lines[1].split()[1])
    assert lines[2] == "W"
    W = [[_parse_val(t, dtype) for t in lines[3 + i].split()] for i in range(n)]
    assert lines[3 + n] == "M"
    M = [[_parse_val(t, dtype) for t in lines[4 + n + i].split()] for i in range(n)]
    npdt = np.uint32 if dtype == "u32" else np.float32
    Wa = np.array(W, dtype=np.uint32).view(npdt)
    Ma = np.array(M, dtype=np.uint32).view(npdt)
    return Wa, Ma


def all_fixtures():
    return sorted(glob.glob(os.path.join(GOLDEN, "*.txt")))
