"""Seeded synthetic closed triangle meshes.

These generators supply the inputs for both the CUDA path and the CPU oracle.
They hold none of the LDNI arithmetic (no snapping, no crossing tests, no
depth formula): each returns ``(verts float32[V,3], tris int32[T,3])`` for a
closed, consistently outward-oriented, non-self-intersecting 2-manifold, the
input class the paper samples (Section 2, Remark 2; Section 3).

The paper's own models (octa-flower, dragon, bunny, Beethoven, gear, chair)
are not available; seeded synthetic shapes of similar structure stand in:

* ``icosphere``   geodesic sphere of frequency ``freq`` (20*freq^2 triangles)
                  with per-vertex uniform or smooth multi-octave radial noise;
* ``torus``       quad-grid torus about the z axis;
* ``flower``      star-shaped radial graph r(theta, phi) on a (theta, phi) grid;
* ``torus_knot``  tube around a (p, q) torus knot.

All geometry is built in FP64 and rounded once to FP32.  Random numbers come
from ``numpy.random.default_rng(seed)`` (PCG64).
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "icosphere", "torus", "flower", "torus_knot", "box", "octahedron",
    "tetrahedron", "signed_volume", "check_closed_oriented", "translate",
    "pr1_pair", "flower_knot_pair", "scale_sphere", "batch_meshes",
    "helix_offsets",
]

_PHI = (1.0 + 5.0 ** 0.5) / 2.0
_ICO_V = np.array([
    (-1, _PHI, 0), (1, _PHI, 0), (-1, -_PHI, 0), (1, -_PHI, 0),
    (0, -1, _PHI), (0, 1, _PHI), (0, -1, -_PHI), (0, 1, -_PHI),
    (_PHI, 0, -1), (_PHI, 0, 1), (-_PHI, 0, -1), (-_PHI, 0, 1),
], dtype=np.float64)
_ICO_F = np.array([
    (0, 11, 5), (0, 5, 1), (0, 1, 7), (0, 7, 10), (0, 10, 11),
    (1, 5, 9), (5, 11, 4), (11, 10, 2), (10, 7, 6), (7, 1, 8),
    (3, 9, 4), (3, 4, 2), (3, 2, 6), (3, 6, 8), (3, 8, 9),
    (4, 9, 5), (2, 4, 11), (6, 2, 10), (8, 6, 7), (9, 8, 1),
], dtype=np.int64)


def _orient_outward(verts: np.ndarray, tris: np.ndarray) -> np.ndarray:
    """Flip the whole winding if the enclosed signed volume is negative."""
    if signed_volume(verts, tris) < 0:
        tris = tris[:, [0, 2, 1]]
    return tris


def signed_volume(verts: np.ndarray, tris: np.ndarray) -> float:
    """Enclosed volume by the divergence theorem, (1/6) sum det(v0, v1, v2), FP64."""
    v = np.asarray(verts, dtype=np.float64)
    t = np.asarray(tris, dtype=np.int64)
    a, b, c = v[t[:, 0]], v[t[:, 1]], v[t[:, 2]]
    return float(np.einsum("ij,ij->i", a, np.cross(b, c)).sum() / 6.0)


def check_closed_oriented(tris: np.ndarray, nv: int) -> None:
    """Raise if the mesh is not a closed, consistently oriented 2-manifold.

    Every directed edge must appear exactly once and its reverse exactly once.
    """
    t = np.asarray(tris, dtype=np.int64)
    if t.size == 0:
        raise ValueError("empty mesh")
    if t.min() < 0 or t.max() >= nv:
        raise ValueError("index out of range")
    if np.any(t[:, 0] == t[:, 1]) or np.any(t[:, 1] == t[:, 2]) or np.any(t[:, 0] == t[:, 2]):
        raise ValueError("repeated vertex in a triangle")
    e = np.concatenate([t[:, [0, 1]], t[:, [1, 2]], t[:, [2, 0]]])
    key = e[:, 0] * nv + e[:, 1]
    rkey = e[:, 1] * nv + e[:, 0]
    uk, cnt = np.unique(key, return_counts=True)
    if np.any(cnt != 1):
        raise ValueError("a directed edge is used twice (inconsistent orientation or non-manifold)")
    if not np.array_equal(np.sort(key), np.sort(rkey)):
        raise ValueError("open boundary: some directed edge has no reverse")


def _finish(v64: np.ndarray, tris: np.ndarray):
    tris = _orient_outward(v64, tris)
    return np.ascontiguousarray(v64, dtype=np.float32), np.ascontiguousarray(tris, dtype=np.int32)


def _geodesic_unit(freq: int):
    """Unit geodesic sphere: icosahedron faces split into freq^2 triangles,
    points projected to the unit sphere.  Vertices are numbered in order of
    first use by the face-major, row-major triangle walk, so consecutive
    triangles and their vertices stay close in memory and in space."""
    k = int(freq)
    if k < 1:
        raise ValueError("freq >= 1")
    ii, jj = [], []
    for i in range(k + 1):
        for j in range(k + 1 - i):
            ii.append(i)
            jj.append(j)
    ii = np.array(ii, dtype=np.int64)
    jj = np.array(jj, dtype=np.int64)
    npf = ii.size
    local = -np.ones((k + 1, k + 1), dtype=np.int64)
    local[ii, jj] = np.arange(npf)
    # local triangles on one face, row by row: "up" (i,j),(i+1,j),(i,j+1) and
    # "down" (i+1,j),(i+1,j+1),(i,j+1)
    lt = []
    for i in range(k):
        for j in range(k - i):
            lt.append((local[i, j], local[i + 1, j], local[i, j + 1]))
            if i + j < k - 1:
                lt.append((local[i + 1, j], local[i + 1, j + 1], local[i, j + 1]))
    lt = np.array(lt, dtype=np.int64)
    F = _ICO_F
    nf = F.shape[0]
    wA = (k - ii - jj)[None, :].repeat(nf, 0)
    wB = ii[None, :].repeat(nf, 0)
    wC = jj[None, :].repeat(nf, 0)
    vA = F[:, 0:1].repeat(npf, 1)
    vB = F[:, 1:2].repeat(npf, 1)
    vC = F[:, 2:3].repeat(npf, 1)
    vid = np.stack([vA, vB, vC], -1).reshape(-1, 3)
    w = np.stack([wA, wB, wC], -1).reshape(-1, 3)
    vid = np.where(w > 0, vid, 15)
    order = np.argsort(vid, axis=1, kind="stable")
    vid_s = np.take_along_axis(vid, order, 1)
    w_s = np.take_along_axis(w, order, 1)
    code = vid_s * 512 + w_s
    key = (code[:, 0] * 8192 + code[:, 1]) * 8192 + code[:, 2]
    # triangle walk order decides vertex numbering
    gtri_raw = (lt[None, :, :] + (np.arange(nf) * npf)[:, None, None]).reshape(-1, 3)
    flat_use = gtri_raw.reshape(-1)
    ukey, inv = np.unique(key, return_inverse=True)
    inv = inv.reshape(-1)
    first_use = np.full(ukey.size, np.iinfo(np.int64).max, dtype=np.int64)
    np.minimum.at(first_use, inv[flat_use], np.arange(flat_use.size))
    rank = np.empty(ukey.size, dtype=np.int64)
    rank[np.argsort(first_use, kind="stable")] = np.arange(ukey.size)
    tris = rank[inv[gtri_raw]]
    # positions: one representative point per unique key
    rep = np.empty(ukey.size, dtype=np.int64)
    rep[inv] = np.arange(key.size)
    pts = (w[rep, 0:1] * _ICO_V[vA.reshape(-1)[rep]] + w[rep, 1:2] * _ICO_V[vB.reshape(-1)[rep]]
           + w[rep, 2:3] * _ICO_V[vC.reshape(-1)[rep]])
    pts /= np.linalg.norm(pts, axis=1, keepdims=True)
    unit = np.empty_like(pts)
    unit[rank] = pts
    return unit, tris


def _octave_noise(dirs: np.ndarray, rng: np.random.Generator, amplitude: float, octaves: int = 4) -> np.ndarray:
    """Smooth seeded noise on the unit sphere: sum over octaves of random plane
    waves sin(k.d + phase), |k| doubling per octave, rescaled so that max |f| =
    amplitude."""
    f = np.zeros(dirs.shape[0], dtype=np.float64)
    for o in range(octaves):
        kmag = 2.0 * (2.0 ** o)
        for _ in range(6):
            kv = rng.normal(size=3)
            kv *= kmag / np.linalg.norm(kv)
            ph = rng.uniform(0, 2 * np.pi)
            f += (0.5 ** o) * np.sin(dirs @ kv + ph)
    m = np.abs(f).max()
    return f * (amplitude / m) if m > 0 else f


def icosphere(freq: int, r: float = 0.35, noise: float = 0.0, noise_kind: str = "uniform",
              seed: int = 0, center=(0.0, 0.0, 0.0)):
    """Geodesic icosphere (20*freq^2 triangles, 10*freq^2+2 vertices).

    ``noise_kind='uniform'``: radius r + U(-noise, noise) per vertex.
    ``noise_kind='octave'``: radius r + smooth 4-octave noise with max |.| = noise.
    A radial graph over the sphere with positive radius cannot self-intersect.
    """
    unit, tris = _geodesic_unit(freq)
    rng = np.random.default_rng(seed)
    if noise > 0:
        if noise_kind == "uniform":
            rad = r + rng.uniform(-noise, noise, size=unit.shape[0])
        elif noise_kind == "octave":
            rad = r + _octave_noise(unit, rng, noise)
        else:
            raise ValueError(noise_kind)
    else:
        rad = np.full(unit.shape[0], r)
    if np.any(rad <= 0):
        raise ValueError("radius must stay positive")
    v = unit * rad[:, None] + np.asarray(center, dtype=np.float64)[None, :]
    return _finish(v, tris)


def _grid_quads(nu: int, nv: int, wrap_v: bool = True):
    """Triangles of an nu x nv periodic quad grid, vertex (i, j) -> i*nv + j."""
    i = np.arange(nu)[:, None]
    j = np.arange(nv)[None, :]
    a = i * nv + j
    b = ((i + 1) % nu) * nv + j
    c = ((i + 1) % nu) * nv + (j + 1) % nv
    d = i * nv + (j + 1) % nv
    t1 = np.stack([a, b, c], -1).reshape(-1, 3)
    t2 = np.stack([a, c, d], -1).reshape(-1, 3)
    return np.stack([t1, t2], 1).reshape(-1, 3)


def torus(R: float = 0.25, r: float = 0.1, nu: int = 64, nv: int = 32, center=(0.0, 0.0, 0.0),
          noise: float = 0.0, seed: int = 0):
    """Torus about the z axis with nu x nv quads (2*nu*nv triangles).

    ``noise`` perturbs the tube radius per vertex by U(-noise, noise) (kept
    below r so the tube stays embedded)."""
    if noise >= r:
        raise ValueError("noise must stay below the tube radius")
    u = 2 * np.pi * np.arange(nu) / nu
    w = 2 * np.pi * np.arange(nv) / nv
    U, Wv = np.meshgrid(u, w, indexing="ij")
    rr = np.full(U.shape, r)
    if noise > 0:
        rr = rr + np.random.default_rng(seed).uniform(-noise, noise, size=U.shape)
    x = (R + rr * np.cos(Wv)) * np.cos(U)
    y = (R + rr * np.cos(Wv)) * np.sin(U)
    z = rr * np.sin(Wv)
    v = np.stack([x, y, z], -1).reshape(-1, 3) + np.asarray(center, dtype=np.float64)
    return _finish(v, _grid_quads(nu, nv))


def flower(n_theta: int = 512, n_phi: int = 512, r0: float = 0.3, amp: float = 0.08, petals: int = 8):
    """Star-shaped 'flower': r(theta, phi) = r0 + amp*cos(petals*phi)*sin^2(theta).

    (n_theta-1) latitude rings of n_phi vertices plus two poles:
    2*n_phi + 2*(n_theta-2)*n_phi triangles (523,264 at 512 x 512)."""
    th = np.pi * np.arange(1, n_theta) / n_theta
    ph = 2 * np.pi * np.arange(n_phi) / n_phi
    TH, PH = np.meshgrid(th, ph, indexing="ij")
    rad = r0 + amp * np.cos(petals * PH) * np.sin(TH) ** 2
    ring = np.stack([rad * np.sin(TH) * np.cos(PH), rad * np.sin(TH) * np.sin(PH), rad * np.cos(TH)], -1)
    ring = ring.reshape(-1, 3)
    north = np.array([[0.0, 0.0, r0]])
    south = np.array([[0.0, 0.0, -r0]])
    v = np.concatenate([ring, north, south])
    nr = n_theta - 1
    iN, iS = nr * n_phi, nr * n_phi + 1
    tris = []
    j = np.arange(n_phi)
    jn = (j + 1) % n_phi
    tris.append(np.stack([np.full(n_phi, iN), j, jn], -1))
    for i in range(nr - 1):
        a = i * n_phi + j
        b = (i + 1) * n_phi + j
        c = (i + 1) * n_phi + jn
        d = i * n_phi + jn
        tris.append(np.stack([a, b, c], -1))
        tris.append(np.stack([a, c, d], -1))
    last = (nr - 1) * n_phi
    tris.append(np.stack([np.full(n_phi, iS), last + jn, last + j], -1))
    return _finish(v, np.concatenate(tris).astype(np.int64))


def torus_knot(p: int = 2, q: int = 3, R: float = 0.25, rho: float = 0.1, tube: float = 0.035,
               n_ring: int = 256, n_side: int = 32):
    """Tube of radius ``tube`` around the (p, q) torus knot
    c(t) = ((R + rho cos qt) cos pt, (R + rho cos qt) sin pt, rho sin qt).

    The cross-section frame uses m(t) = cos(qt) e_r(pt) + sin(qt) e_z, which is
    orthogonal to c'(t) for every t, so the frame is smooth and periodic."""
    t = 2 * np.pi * np.arange(n_ring) / n_ring
    er = np.stack([np.cos(p * t), np.sin(p * t), np.zeros_like(t)], -1)
    ephi = np.stack([-np.sin(p * t), np.cos(p * t), np.zeros_like(t)], -1)
    ez = np.array([0.0, 0.0, 1.0])[None, :]
    c = (R + rho * np.cos(q * t))[:, None] * er + (rho * np.sin(q * t))[:, None] * ez
    dc = (-q * rho * np.sin(q * t))[:, None] * er + (p * (R + rho * np.cos(q * t)))[:, None] * ephi \
        + (q * rho * np.cos(q * t))[:, None] * ez
    T = dc / np.linalg.norm(dc, axis=1, keepdims=True)
    N = np.cos(q * t)[:, None] * er + np.sin(q * t)[:, None] * ez
    N = N - (N * T).sum(1, keepdims=True) * T
    N /= np.linalg.norm(N, axis=1, keepdims=True)
    B = np.cross(T, N)
    s = 2 * np.pi * np.arange(n_side) / n_side
    v = c[:, None, :] + tube * (np.cos(s)[None, :, None] * N[:, None, :] + np.sin(s)[None, :, None] * B[:, None, :])
    return _finish(v.reshape(-1, 3), _grid_quads(n_ring, n_side))


def box(lo, hi):
    """Axis-aligned box [lo, hi] as 12 outward triangles."""
    lo = np.asarray(lo, dtype=np.float64)
    hi = np.asarray(hi, dtype=np.float64)
    v = np.array([[lo[0], lo[1], lo[2]], [hi[0], lo[1], lo[2]], [hi[0], hi[1], lo[2]], [lo[0], hi[1], lo[2]],
                  [lo[0], lo[1], hi[2]], [hi[0], lo[1], hi[2]], [hi[0], hi[1], hi[2]], [lo[0], hi[1], hi[2]]])
    f = np.array([[0, 3, 2], [0, 2, 1], [4, 5, 6], [4, 6, 7], [0, 1, 5], [0, 5, 4],
                  [2, 3, 7], [2, 7, 6], [1, 2, 6], [1, 6, 5], [0, 4, 7], [0, 7, 3]])
    return _finish(v, f)


def slab_stack(k: int, axis: int = 0, seed: int = 0, lo: float = -0.45, hi: float = 0.45):
    """k disjoint thin boxes stacked along ``axis`` inside [lo, hi], each with
    seeded cross-section extents, so that a ray along ``axis`` meets the two
    faces of every box over its pixel: up to 2k samples per ray, varying
    across the image."""
    rng = np.random.default_rng(seed)
    step = (hi - lo) / k
    parts = []
    for m in range(k):
        a0 = lo + m * step
        blo = np.empty(3)
        bhi = np.empty(3)
        blo[axis], bhi[axis] = a0 + 0.2 * step, a0 + 0.7 * step
        for b in range(3):
            if b == axis:
                continue
            c = rng.uniform(-0.1, 0.1)
            w = rng.uniform(0.2, 0.4)
            blo[b], bhi[b] = c - w, c + w
        parts.append(box(blo, bhi))
    verts = np.concatenate([v for v, _ in parts])
    offs = np.cumsum([0] + [len(v) for v, _ in parts[:-1]])
    tris = np.concatenate([t + o for (_, t), o in zip(parts, offs)])
    return verts, tris.astype(np.int32)


def octahedron(center, c):
    """Regular octahedron with vertices center +- c e_k."""
    ce = np.asarray(center, dtype=np.float64)
    v = np.array([[c, 0, 0], [-c, 0, 0], [0, c, 0], [0, -c, 0], [0, 0, c], [0, 0, -c]], dtype=np.float64) + ce
    f = np.array([[0, 2, 4], [2, 1, 4], [1, 3, 4], [3, 0, 4], [2, 0, 5], [1, 2, 5], [3, 1, 5], [0, 3, 5]])
    return _finish(v, f)


def tetrahedron(points):
    """Tetrahedron on four given points (outward winding fixed by volume sign)."""
    v = np.asarray(points, dtype=np.float64).reshape(4, 3)
    f = np.array([[0, 1, 2], [0, 3, 1], [1, 3, 2], [0, 2, 3]])
    return _finish(v, f)


def translate(mesh, d):
    v, t = mesh
    return (np.ascontiguousarray((v.astype(np.float64) + np.asarray(d, dtype=np.float64)).astype(np.float32)), t)


def pr1_pair(seed: int = 1):
    """Small parity case: A = level-3 icosphere (1280 tris), r 0.35, radial
    noise U(-0.03, 0.03); B = torus R 0.25 r 0.1, 64x32 quads, shifted +0.15 x."""
    A = icosphere(8, r=0.35, noise=0.03, noise_kind="uniform", seed=seed)
    B = torus(0.25, 0.1, 64, 32, center=(0.15, 0.0, 0.0))
    return A, B


def flower_knot_pair():
    """Flower (512 x 512 grid, 523,264 tris) and (2,3) torus-knot tube (16,384 tris)."""
    return flower(512, 512), torus_knot(2, 3, 0.25, 0.1, 0.035, 256, 32)


def scale_sphere(freq: int = 256, seed: int = 3, amplitude: float = 0.05):
    """Sampling-throughput mesh: geodesic icosphere (freq 256 -> 1,310,720
    tris), r 0.35, smooth 4-octave radial noise of amplitude 0.05."""
    return icosphere(freq, r=0.35, noise=amplitude, noise_kind="octave", seed=seed)


def batch_meshes(count: int = 256, seed: int = 7, tmin: int = 1000, tmax: int = 200_000,
                 resolutions=(64, 128, 256, 512)):
    """Seeded batch of noisy icospheres and tori with log-uniform triangle
    counts in [tmin, tmax] and resolutions drawn from ``resolutions``.

    Returns a list of (verts, tris, res)."""
    rng = np.random.default_rng(seed)
    out = []
    for m in range(count):
        T = float(np.exp(rng.uniform(np.log(tmin), np.log(tmax))))
        res = int(rng.choice(resolutions))
        if rng.uniform() < 0.5:
            freq = max(1, int(round((T / 20.0) ** 0.5)))
            r = rng.uniform(0.2, 0.4)
            mesh = icosphere(freq, r=r, noise=0.1 * r, noise_kind="octave", seed=int(rng.integers(1 << 30)))
        else:
            nq = max(4, int(round((T / 2.0) ** 0.5)))
            R = rng.uniform(0.2, 0.3)
            rr = rng.uniform(0.05, 0.15)
            mesh = torus(R, rr, 2 * nq, max(3, nq // 2), noise=0.2 * rr, seed=int(rng.integers(1 << 30)))
        out.append((mesh[0], mesh[1], res))
    return out


def helix_offsets(steps: int = 64, seed: int = 11, radius=None, pitch=None, turns=None):
    """Seeded helix of translation offsets inside the unit cube for a
    sweep-style union chain."""
    rng = np.random.default_rng(seed)
    radius = rng.uniform(0.1, 0.2) if radius is None else radius
    pitch = rng.uniform(0.3, 0.5) if pitch is None else pitch
    turns = rng.uniform(1.0, 2.0) if turns is None else turns
    s = np.linspace(0.0, 1.0, steps)
    ang = 2 * np.pi * turns * s
    return np.stack([radius * np.cos(ang), radius * np.sin(ang), pitch * (s - 0.5)], -1)
