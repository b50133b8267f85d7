"""FP64 adjoint of LDNI depths and volume (TEST INFRASTRUCTURE ONLY).

For a sample of ray (u, v) on triangle t, the depth is where the ray meets
t's plane; with lambda the barycentrics of (u, v) in t's projection and a_k
the vertex a-coordinates, d = sum_k lambda_k a_k.  Volume of one image is
h^2 sum_rays sum_k (d_{2k+1} - d_{2k}) (odd-to-even ranges inside).  The
sample set ("which triangle each ray crosses") is the one an LDNI recorded
and is held fixed.  Everything here is FP64 NumPy.
"""
import numpy as np


def frozen_set(L, res, axis, origin, width):
    """(u, v, tri, sigma) of every sample of an LDNI dict (offsets, tri)."""
    off = np.asarray(L["offsets"], dtype=np.int64)
    cnt = np.diff(off)
    p = np.repeat(np.arange(cnt.size), cnt)
    k = np.arange(p.size) - off[p]
    j, i = np.divmod(p, res)
    iu, iv = (axis + 1) % 3, (axis + 2) % 3
    h = float(width) / res
    u = float(origin[iu]) + (i + 0.5) * h
    v = float(origin[iv]) + (j + 0.5) * h
    sigma = np.where(k % 2 == 1, 1.0, -1.0)
    return u, v, np.asarray(L["tri"], dtype=np.int64)[:p.size], sigma


def depths(verts, tris, u, v, tri, axis):
    """Plane depth of each frozen sample (continuous, unsnapped)."""
    V = np.asarray(verts, dtype=np.float64)
    T = np.asarray(tris, dtype=np.int64)[tri]
    iu, iv = (axis + 1) % 3, (axis + 2) % 3
    P0, P1, P2 = V[T[:, 0]], V[T[:, 1]], V[T[:, 2]]
    u1, v1 = P1[:, iu] - P0[:, iu], P1[:, iv] - P0[:, iv]
    u2, v2 = P2[:, iu] - P0[:, iu], P2[:, iv] - P0[:, iv]
    xu, xv = u - P0[:, iu], v - P0[:, iv]
    A = u1 * v2 - v1 * u2
    l1 = (xu * v2 - xv * u2) / A
    l2 = (u1 * xv - v1 * xu) / A
    l0 = 1.0 - l1 - l2
    return l0 * P0[:, axis] + l1 * P1[:, axis] + l2 * P2[:, axis]


def volume(verts, tris, fs, axis, h):
    u, v, tri, sigma = fs
    return float(np.sum(sigma * depths(verts, tris, u, v, tri, axis)) * h * h)


def depth_vjp(verts, tris, fs, axis, w):
    """sum_s w_s d(d_s)/d(verts), as an [nv, 3] array: lambda_j n / n_a."""
    u, v, tri, _ = fs
    V = np.asarray(verts, dtype=np.float64)
    T = np.asarray(tris, dtype=np.int64)[tri]
    iu, iv = (axis + 1) % 3, (axis + 2) % 3
    P0, P1, P2 = V[T[:, 0]], V[T[:, 1]], V[T[:, 2]]
    n = np.cross(P1 - P0, P2 - P0)
    u1, v1 = P1[:, iu] - P0[:, iu], P1[:, iv] - P0[:, iv]
    u2, v2 = P2[:, iu] - P0[:, iu], P2[:, iv] - P0[:, iv]
    xu, xv = u - P0[:, iu], v - P0[:, iv]
    A = u1 * v2 - v1 * u2
    l1 = (xu * v2 - xv * u2) / A
    l2 = (u1 * xv - v1 * xu) / A
    lam = np.stack([1.0 - l1 - l2, l1, l2], 1)
    scale = (np.asarray(w, dtype=np.float64) / n[:, axis])[:, None] * n
    g = np.zeros_like(V)
    for k in range(3):
        np.add.at(g, T[:, k], lam[:, k:k + 1] * scale)
    return g


def volume_grad(verts, tris, fs, axis, h):
    return depth_vjp(verts, tris, fs, axis, fs[3] * h * h)


def mesh_volume_grad(verts, tris):
    """Gradient of the divergence-theorem volume (1/6) sum det(v0, v1, v2):
    each face adds cross(v_{k+1}, v_{k+2}) / 6 to vertex k."""
    V = np.asarray(verts, dtype=np.float64)
    T = np.asarray(tris, dtype=np.int64)
    g = np.zeros_like(V)
    for k in range(3):
        np.add.at(g, T[:, k], np.cross(V[T[:, (k + 1) % 3]], V[T[:, (k + 2) % 3]]) / 6.0)
    return g
