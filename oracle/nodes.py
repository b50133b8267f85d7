"""Grid-node classification oracle (TEST INFRASTRUCTURE ONLY): Section 5.1,
Step 1.  Written from the definition in plain NumPy; shares no code with the
CUDA library.

The rays of the x-, y- and z-images meet at the res^3 grid nodes
(Definition 3).  Node (i, j, k) lies at (c(i), c(j), c(k)) on the three axes,
c_a(t) = fl32(o_a + fl32((t + 1/2) * h)) with h = fl32(width / res) (the
pixel centres).  An image puts a node inside when an odd number of the
samples of its ray through the node lie strictly below the node's
coordinate along the ray (odd-to-even ranges are inside, Section 2); the
node is inside when at least two images do.
"""
from __future__ import annotations

import numpy as np


def node_coords(origin_a: float, width: float, res: int) -> np.ndarray:
    h = np.float32(width) / np.float32(res)
    t = np.arange(res, dtype=np.float32) + np.float32(0.5)
    return np.float32(origin_a) + (t * h).astype(np.float32)


def image_votes(L: dict, axis: int, origin, width: float, res: int) -> np.ndarray:
    """bool [k, j, i]: node (i, j, k) inside according to image `axis`.  L is
    an LDNI dict (offsets over rays p = jv * res + iu; in-plane axes
    (u, v) = ((a + 1) % 3, (a + 2) % 3))."""
    off = np.asarray(L["offsets"], np.int64)
    d = np.asarray(L["depth"], np.float32)
    c = node_coords(origin[axis], width, res)
    out = np.zeros((res, res, res), bool)  # [k, j, i]
    u, v = (axis + 1) % 3, (axis + 2) % 3
    for jv in range(res):
        for iu in range(res):
            p = jv * res + iu
            s = d[off[p]:off[p + 1]]
            below = np.searchsorted(s, c, side="left")  # samples strictly below each node coordinate
            inside = (below & 1).astype(bool)
            # node (x, y, z) indices: the ray's axis runs over all t, u is iu, v is jv
            sel = {axis: slice(None), u: iu, v: jv}
            out[sel[2], sel[1], sel[0]] = inside
    return out


def classify(Ls, origin, width: float, res: int) -> np.ndarray:
    """bool [k, j, i]: at least two of the three images put the node inside."""
    votes = sum(image_votes(L, a, origin, width, res).astype(np.int8) for a, L in enumerate(Ls))
    return votes >= 2
