"""Reader for the hand-worked fixtures in tests/golden/ (plain text)."""
import glob
import os

import numpy as np

GOLDEN_DIR = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
_DT = {"u8": (np.uint8, 0), "u16": (np.uint16, 1), "u14": (np.uint16, 2)}


def load(path):
    k = dtype = flagged = None
    detector = "extreme"
    sect = None
    rows = {"input": [], "output": []}
    with open(path) as fh:
        for line in fh:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            head = line.split()
            if head[0] == "k":
                k = int(head[1])
            elif head[0] == "dtype":
                dtype = head[1]
            elif head[0] == "detector":
                detector = head[1]
            elif head[0] in ("input", "output"):
                sect = head[0]
            elif head[0] == "flagged":
                flagged = int(head[1])
                sect = None
            else:
                rows[sect].append([int(v) for v in head])
    npdt, code = _DT[dtype]
    return {
        "name": os.path.basename(path),
        "k": k,
        "dtype": code,
        "input": np.array(rows["input"], dtype=npdt),
        "output": np.array(rows["output"], dtype=npdt),
        "flagged": flagged,
        "detector": detector,   # "extreme" (Eq. 3a/3b) or "directional" (Fig. 1)
    }


def all_fixtures(detector=None):
    """Every fixture, or those of one detector ("extreme" or "directional")."""
    fx = [load(p) for p in sorted(glob.glob(os.path.join(GOLDEN_DIR, "*.txt")))]
    return [f for f in fx if detector is None or f["detector"] == detector]
