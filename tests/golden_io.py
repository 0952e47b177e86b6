"""Reader for the hand-built text fixtures under tests/golden/."""
import os

import numpy as np

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def load(name):
    meta, blocks, cur = {}, {}, None
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            parts = line.split()
            if len(parts) == 2 and cur is None and not _num(parts[0]):
                meta[parts[0]] = parts[1]
                continue
            if len(parts) == 1 and not _num(parts[0]):
                cur = parts[0]
                blocks[cur] = []
                continue
            blocks[cur].append([float(v) for v in parts])
    out = dict(meta=meta)
    for k, rows in blocks.items():
        out[k] = np.array(rows) if len(rows) > 1 or k != "spec" else np.array(rows[0])
    return out


def _num(s):
    try:
        float(s)
        return True
    except ValueError:
        return False
