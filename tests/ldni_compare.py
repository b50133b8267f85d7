"""Parity rule between a CUDA-sampled LDNI and the FP64 oracle's.

* per-ray sample counts: bit-exact;
* per-ray multiset of triangle ids: bit-exact (a planar face crosses a ray
  at most once, so (ray, tri) identifies a sample);
* depth of each (ray, tri) sample: within tol * diag (FP32 vs FP64);
* normal components: within ntol absolute;
* order: the CUDA sequence of each ray is ascending in the oracle's depths up
  to tol * diag (equal or nearly equal depths may come in either order).
"""
import numpy as np


def ray_index(offsets):
    cnt = np.diff(np.asarray(offsets, dtype=np.int64))
    return np.repeat(np.arange(cnt.size), cnt)


def compare_ldni(got, ref, diag, tol=1e-5, ntol=1e-5):
    og = np.asarray(got["offsets"], dtype=np.int64)
    orf = np.asarray(ref["offsets"], dtype=np.int64)
    assert og.shape == orf.shape
    bad = np.nonzero(np.diff(og) != np.diff(orf))[0]
    assert bad.size == 0, f"{bad.size} rays with different counts, first {bad[:5]}"
    n = int(orf[-1])
    assert int(og[-1]) == n
    if n == 0:
        return
    r = ray_index(orf)
    tg = np.asarray(got["tri"], dtype=np.int64)[:n]
    tr = np.asarray(ref["tri"], dtype=np.int64)[:n]
    ig = np.lexsort((tg, r))
    ir = np.lexsort((tr, r))
    assert np.array_equal(tg[ig], tr[ir]), "per-ray triangle ids differ"
    dg = np.asarray(got["depth"], dtype=np.float64)[:n]
    dr = np.asarray(ref["depth"], dtype=np.float64)[:n]
    err = np.abs(dg[ig] - dr[ir])
    assert err.max() <= tol * diag, f"depth error {err.max()} > {tol * diag}"
    ng = np.asarray(got["nrm"], dtype=np.float64)[:n]
    nr = np.asarray(ref["nrm"], dtype=np.float64)[:n]
    nerr = np.abs(ng[ig] - nr[ir])
    assert nerr.max() <= ntol, f"normal error {nerr.max()}"
    # order: oracle depth of the k-th CUDA sample
    ref_depth_in_got_order = np.empty(n)
    ref_depth_in_got_order[ig] = dr[ir]
    same_ray = r[1:] == r[:-1]
    step = ref_depth_in_got_order[1:] - ref_depth_in_got_order[:-1]
    assert np.all(step[same_ray] >= -tol * diag), "CUDA order not ascending in depth"
    return {"max_depth_err": float(err.max()), "max_normal_err": float(nerr.max()), "n": n}


def bit_equal(X, Y):
    n = int(np.asarray(Y["offsets"])[-1])
    return (np.array_equal(np.asarray(X["offsets"], np.int64), np.asarray(Y["offsets"], np.int64))
            and np.array_equal(np.asarray(X["depth"])[:n], np.asarray(Y["depth"])[:n])
            and np.array_equal(np.asarray(X["nrm"])[:n], np.asarray(Y["nrm"])[:n])
            and np.array_equal(np.asarray(X["tri"])[:n], np.asarray(Y["tri"])[:n]))
