"""Reader of tests/golden/boolean_segments.txt (hand-worked per-ray Booleans,
Section 4.1 and 4.1.1)."""
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))


def cases():
    out = []
    with open(os.path.join(HERE, "golden", "boolean_segments.txt")) as fh:
        for line in fh:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            name, op, eps, a, b, res = [f.strip() for f in line.split("|")]
            out.append({"name": name, "op": op, "eps": float(eps),
                        "A": np.array([float(x) for x in a.split()], np.float32),
                        "B": np.array([float(x) for x in b.split()], np.float32),
                        "result": res.split()})
    return out


def ray(depths, first_id, seed):
    """One-ray LDNI dict with distinct unit normals and triangle ids."""
    n = depths.size
    rng = np.random.default_rng(seed)
    nrm = rng.normal(size=(n, 3)).astype(np.float32)
    nrm /= np.linalg.norm(nrm, axis=1, keepdims=True)
    return {"offsets": np.array([0, n], np.int64), "depth": depths.astype(np.float32), "nrm": nrm,
            "tri": np.arange(first_id, first_id + n, dtype=np.int32)}


def expected(case, A, B):
    """The output the case lists, built from the operand samples."""
    d, nrm, tri = [], [], []
    for tok in case["result"]:
        src, i = tok[0], int(tok[1:])
        if src == "a":
            d.append(A["depth"][i])
            nrm.append(A["nrm"][i])
            tri.append(int(A["tri"][i]))
        else:  # B's samples carry bit 31 in their id; "n" inverts the normal
            d.append(B["depth"][i])
            nrm.append((-1.0 if src == "n" else 1.0) * B["nrm"][i])
            tri.append(int(B["tri"][i]) | 0x80000000)
    n = len(d)
    return {"offsets": np.array([0, n], np.int64), "depth": np.array(d, np.float32),
            "nrm": np.array(nrm, np.float32).reshape(n, 3),
            "tri": np.array(tri, np.uint32).view(np.int32)}
