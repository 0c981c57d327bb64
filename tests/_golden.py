"""Reader for the worked-example fixtures under tests/golden/.

Format: '#' comment lines; '@ NAME k' opens frontal slice k (1-based) of
tensor NAME; the following non-empty lines are that slice's rows.  Returns a
dict NAME -> float64 array (p, rows, cols), slice-major.
"""

import os

import numpy as np

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def load(name):
    slices = {}
    cur = None
    with open(os.path.join(GOLDEN, name)) as f:
        for raw in f:
            line = raw.strip()
            if not line or line.startswith("#"):
                continue
            if line.startswith("@"):
                _, tname, k = line.split()
                cur = []
                slices.setdefault(tname, {})[int(k)] = cur
                continue
            cur.append([float(v) for v in line.split()])
    out = {}
    for tname, by_k in slices.items():
        ks = sorted(by_k)
        assert ks == list(range(1, len(ks) + 1)), f"{name}:{tname} slices not contiguous"
        out[tname] = np.array([by_k[k] for k in ks], dtype=np.float64)
    return out
