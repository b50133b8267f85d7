"""CUDA adjoint of LDNI depths and volume (ldni_depth_vjp, ldni_volume_grad)
and its torch.autograd wrappers, against the FP64 oracle gradient and
central finite differences of the frozen-set volume.

The GPU and the oracle record the same crossing set (bit-exact triangle ids
per ray), so both differentiate the same function; tolerances cover FP32
barycentrics and FP32 atomic accumulation."""
import numpy as np
import pytest

import meshgen as M
import oracle
from oracle import adjoint as AD

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

O3 = (-0.5, -0.5, -0.5)


@pytest.fixture(scope="module")
def ldni():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1009_0794_gb300 as pkg
    pkg._lib.load()
    return pkg


def _rel(a, b):
    return float(np.max(np.abs(a - b)) / max(1e-30, np.max(np.abs(b))))


# The kernel's per-crossing terms are FP32 with error-free determinants (a few
# ulp each); a vertex's component adds at most some tens of them with FP32
# atomics.  64 roundings of 2^-24 of the largest component bound the error
# against the FP64 oracle at 4e-6 of the gradient's scale.
TOL_SCALE = 4e-6


def _far_from_silhouettes(v, t, a, min_na=0.2):
    """Vertices whose every incident face has |n_a| >= min_na (its normal far
    from perpendicular to the rays), where the derivative is well conditioned."""
    V = v.astype(np.float64)
    n = np.cross(V[t[:, 1]] - V[t[:, 0]], V[t[:, 2]] - V[t[:, 0]])
    n /= np.linalg.norm(n, axis=1, keepdims=True)
    bad = np.abs(n[:, a]) < min_na
    ok = np.ones(len(v), bool)
    ok[np.unique(t[bad].reshape(-1))] = False
    return ok


def _check_components(g, ref, ok, rtol):
    """Per component, relative: every component of a well-conditioned vertex
    that is at least 1e-3 of the scale."""
    scale = np.max(np.abs(ref))
    sel = ok[:, None] & (np.abs(ref) >= 1e-3 * scale)
    if not sel.any():
        return 0.0
    rel = np.abs(g[sel] - ref[sel]) / np.abs(ref[sel])
    assert rel.max() < rtol, rel.max()
    return float(rel.max())


@pytest.mark.parametrize("res", [128, 77])
def test_volume_grad_matches_oracle(ldni, res):
    A, B = M.pr1_pair()
    grid = ldni.Grid.cube(O3, 1.0, res)
    for v, t in (A, B):
        vt, tt = torch.from_numpy(v).cuda(), torch.from_numpy(t).cuda()
        for a, L in enumerate(ldni.sample(vt, tt, grid, "all")):
            g = ldni.volume_grad(vt, tt, L, 1.0).cpu().numpy()
            fs = AD.frozen_set(L.numpy(), res, a, O3, 1.0)
            ref = AD.volume_grad(v, t, fs, a, 1.0 / res)
            assert _rel(g, ref) < TOL_SCALE
            _check_components(g, ref, _far_from_silhouettes(v, t, a), 1e-4)


def test_depth_vjp_matches_oracle(ldni):
    v, t = M.icosphere(12, r=0.34, noise=0.03, noise_kind="octave", seed=6)
    grid = ldni.Grid.cube(O3, 1.0, 100)
    vt, tt = torch.from_numpy(v).cuda(), torch.from_numpy(t).cuda()
    for a, L in enumerate(ldni.sample(vt, tt, grid, "all")):
        w = torch.from_numpy(np.random.default_rng(a).normal(size=L.n).astype(np.float32)).cuda()
        g = ldni.depth_vjp(vt, tt, L, w).cpu().numpy()
        fs = AD.frozen_set(L.numpy(), 100, a, O3, 1.0)
        ref = AD.depth_vjp(v, t, fs, a, w.cpu().numpy().astype(np.float64))
        assert _rel(g, ref) < TOL_SCALE


def test_autograd_functions(ldni):
    from paper_1009_0794_gb300.autograd import LDNIDepths, LDNIVolume
    v, t = M.icosphere(10, r=0.3, noise=0.03, seed=2)
    grid = ldni.Grid.cube(O3, 1.0, 96)
    vt = torch.from_numpy(v).cuda().requires_grad_(True)
    tt = torch.from_numpy(t).cuda()
    vol = LDNIVolume.apply(vt, tt, grid, "all")
    vol.backward()
    g = vt.grad.detach().cpu().numpy()
    refs, vols = [], []
    for a in range(3):
        L = oracle.sample(v, t, O3, 1.0, 96, a, "scan")
        vols.append(oracle.volume(oracle.as_f32(L), 1.0 / 96))
        refs.append(AD.volume_grad(v, t, AD.frozen_set(L, 96, a, O3, 1.0), a, 1.0 / 96))
    assert float(vol.detach()) == pytest.approx(np.mean(vols), rel=1e-6)
    assert _rel(g, sum(refs) / 3) < 2e-4
    vt.grad = None
    d = LDNIDepths.apply(vt, tt, grid, 1)
    (d * d).sum().backward()
    L = oracle.sample(v, t, O3, 1.0, 96, 1, "scan")
    fs = AD.frozen_set(L, 96, 1, O3, 1.0)
    ref = AD.depth_vjp(v, t, fs, 1, 2.0 * d.detach().cpu().numpy().astype(np.float64))
    assert _rel(vt.grad.cpu().numpy(), ref) < 2e-4


def test_200k_sphere_against_oracle_and_central_differences(ldni):
    """The 200,000-triangle noisy icosphere at 512^2 x 3 images: the CUDA
    gradient on 1000 random vertices against the FP64 oracle gradient, and
    against central differences (h = 1e-4) of the frozen-set volume wherever
    that difference has converged (it agrees with the h/2 difference; near
    silhouettes n_a is tiny and a 1e-4 move is far outside the linear
    range)."""
    v, t = M.icosphere(100, r=0.35, noise=0.03, noise_kind="octave", seed=12)
    res = 512
    h = 1.0 / res
    grid = ldni.Grid.cube(O3, 1.0, res)
    vt, tt = torch.from_numpy(v).cuda(), torch.from_numpy(t).cuda()
    layers = ldni.sample(vt, tt, grid, "all")
    rng = np.random.default_rng(0)
    pick = rng.choice(len(v), 1000, replace=False)
    tri_of = [[] for _ in range(len(v))]
    for k, tri in enumerate(t):
        for q in tri:
            tri_of[q].append(k)
    V = v.astype(np.float64)
    worst_oracle = worst_fd = 0.0
    checked = converged = 0
    for a, L in enumerate(layers):
        g = ldni.volume_grad(vt, tt, L, 1.0).cpu().numpy()
        fs = AD.frozen_set(L.numpy(), res, a, O3, 1.0)
        ref = AD.volume_grad(v, t, fs, a, h)
        scale = np.max(np.abs(ref))
        worst_oracle = max(worst_oracle, float(np.max(np.abs(g[pick] - ref[pick])) / scale))
        u, vv, tri, sigma = fs
        order = np.argsort(tri, kind="stable")
        ts = tri[order]
        starts = np.searchsorted(ts, np.arange(len(t)))
        ends = np.searchsorted(ts, np.arange(len(t)), side="right")
        for j in pick[:200]:
            idx = np.concatenate([order[starts[k]:ends[k]] for k in tri_of[j]])
            if idx.size == 0:
                continue
            sub = (u[idx], vv[idx], tri[idx], sigma[idx])

            def fd(c, step):
                Vp, Vm = V.copy(), V.copy()
                Vp[j, c] += step
                Vm[j, c] -= step
                return (AD.volume(Vp, t, sub, a, h) - AD.volume(Vm, t, sub, a, h)) / (2 * step)

            for c in range(3):
                checked += 1
                f1, f2 = fd(c, 1e-4), fd(c, 5e-5)
                if abs(f1 - f2) > 1e-4 * scale:
                    continue
                converged += 1
                worst_fd = max(worst_fd, abs(f1 - g[j, c]) / scale)
    print(f"adjoint 200k: oracle max rel {worst_oracle:.2e}; FD max rel {worst_fd:.2e} "
          f"on {converged}/{checked} converged components")
    assert worst_oracle < TOL_SCALE
    assert converged >= 0.9 * checked
    assert worst_fd < 1e-3
