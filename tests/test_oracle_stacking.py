"""Pins of the oracle's stacking section (Sec. III.B, Fig. 1): own atan2, RING vec2pix, box
placement, cone cut.

  * atan2 in quarter turns against mpmath (40 digits): <= 4 ulp, exact on the axes;
  * vec2pix: vec2pix(pix2vec(p)) = p for every pixel (pix2vec is pinned by brute-force ring
    enumeration in test_oracle_pix2vec); a random direction lies in a pixel whose centre is
    among its 4 nearest centres and within the pixel's circumradius bound; agreement with an
    independent numpy statement of the published rules away from pixel edges; equal-area
    counts (chi-square);
  * placement: exact for permutation rotations, composition of placements, norm preserved;
  * cut: with the 12 base pixels as cones every sample is kept by exactly one shell; radius
    bounds are [r_lo, r_hi); input order is kept.
"""
import numpy as np
import pytest

import oracle

mpmath = pytest.importorskip("mpmath")


def test_atan2_quarter_vs_mpmath():
    mpmath.mp.dps = 40
    rng = np.random.default_rng(1)
    pts = list(rng.normal(size=(2000, 2)))
    pts += list(rng.normal(size=(500, 2)) * np.exp(rng.uniform(-30, 30, size=(500, 2))))
    pts += [(0.0, 1.0), (1.0, 0.0), (0.0, -1.0), (-1.0, 0.0), (1.0, 1.0), (-1.0, 1.0), (1.0, -1.0), (-1.0, -1.0),
            (np.tan(np.pi / 8), 1.0), (1.0, np.tan(np.pi / 8)), (1e-300, 1.0), (-1e-300, 1.0)]
    for y, x in pts:
        q = oracle.atan2_quarter(y, x)
        e = mpmath.atan2(mpmath.mpf(float(y)), mpmath.mpf(float(x))) / (mpmath.pi / 2)
        if e < 0:
            e += 4
        assert 0.0 <= q < 4.0
        assert abs(q - float(e)) <= 4 * np.spacing(max(abs(float(e)), 1e-300)) or abs(float(e) - 4) < 1e-15
    assert oracle.atan2_quarter(1.0, 0.0) == 1.0
    assert oracle.atan2_quarter(0.0, -1.0) == 2.0
    assert oracle.atan2_quarter(-1.0, 0.0) == 3.0
    assert oracle.atan2_quarter(0.0, 1.0) == 0.0
    assert oracle.atan2_quarter(1.0, 1.0) == 0.5


@pytest.mark.parametrize("N", [1, 2, 3, 4, 5, 8, 13, 16, 64, 256])
def test_vec2pix_roundtrip(N):
    v, _, _ = oracle.pix2vec_ring(N)
    assert np.array_equal(oracle.vec2pix_ring(N, v), np.arange(12 * N * N))
    assert np.array_equal(oracle.vec2pix_ring(N, 3.7 * v), np.arange(12 * N * N))   # scale-free


def test_vec2pix_roundtrip_nside4096_sampled():
    N = 4096
    p = np.random.default_rng(2).choice(12 * N * N, 100000, replace=False)
    v, _, _ = oracle.pix2vec_ring(N, pix=p)
    assert np.array_equal(oracle.vec2pix_ring(N, v), p)


def _unit(rng, n):
    v = rng.normal(size=(3, n))
    return v / np.linalg.norm(v, axis=0)


@pytest.mark.parametrize("N", [1, 2, 4, 16])
def test_vec2pix_nearest_centres(N):
    """A point belongs to a pixel whose centre is one of its 4 nearest centres, and lies within
    the largest centre-to-vertex angle of the grid (< 1.5 x the mean pixel size)."""
    rng = np.random.default_rng(N)
    pts = _unit(rng, 20000)
    c, _, _ = oracle.pix2vec_ring(N)
    p = oracle.vec2pix_ring(N, pts)
    d = c.T @ pts                                       # cosines to every centre
    order = np.argsort(-d, axis=0)[:4]
    assert np.all((order == p[None, :]).any(axis=0))
    ang = np.arccos(np.clip(d[p, np.arange(pts.shape[1])], -1, 1))
    assert ang.max() < 1.5 * np.sqrt(4 * np.pi / (12 * N * N)) * (1.6 if N == 1 else 1.0)


def _vec2pix_numpy(N, v):
    """Independent numpy statement of the published RING assignment; also returns the distance
    of the floored quantities to the nearest integer (to skip points on pixel edges)."""
    z = v[2] / np.linalg.norm(v, axis=0)
    za = np.abs(z)
    t = np.arctan2(v[1], v[0]) / (np.pi / 2)
    t = np.where(t < 0, t + 4, t)
    pix = np.empty(v.shape[1], dtype=np.int64)
    edge = np.empty(v.shape[1])
    eq = za <= 2 / 3
    a = N * (0.5 + t[eq] - 0.75 * z[eq])
    b = N * (0.5 + t[eq] + 0.75 * z[eq])
    jp, jm = np.floor(a).astype(np.int64), np.floor(b).astype(np.int64)
    ir = N + 1 + jp - jm
    ip = (jp + jm - N + (1 - (ir & 1)) + 1) // 2 % (4 * N)
    pix[eq] = 2 * N * (N - 1) + (ir - 1) * 4 * N + ip
    edge[eq] = np.minimum(np.abs(a - np.round(a)), np.abs(b - np.round(b)))
    po = ~eq
    tp = t[po] - np.floor(t[po])
    h = N * np.sqrt(3 * (1 - za[po]))
    u, w = tp * h, (1 - tp) * h
    jp, jm = np.floor(u).astype(np.int64), np.floor(w).astype(np.int64)
    ir = jp + jm + 1
    x = t[po] * ir
    ip = np.floor(x).astype(np.int64) % (4 * ir)
    pix[po] = np.where(z[po] > 0, 2 * ir * (ir - 1) + ip, 12 * N * N - 2 * ir * (ir + 1) + ip)
    edge[po] = np.minimum.reduce([np.abs(u - np.round(u)), np.abs(w - np.round(w)), np.abs(x - np.round(x))])
    edge = np.minimum(edge, np.abs(za - 2 / 3) * 10)
    return pix, edge


@pytest.mark.parametrize("N", [1, 2, 16, 512])
def test_vec2pix_vs_numpy_statement(N):
    pts = _unit(np.random.default_rng(10 + N), 200000)
    ref, edge = _vec2pix_numpy(N, pts)
    got = oracle.vec2pix_ring(N, pts)
    ok = edge > 1e-9
    assert ok.mean() > 0.999
    assert np.array_equal(got[ok], ref[ok])


def test_vec2pix_equal_area():
    N = 2
    pts = _unit(np.random.default_rng(5), 480000)
    cnt = np.bincount(oracle.vec2pix_ring(N, pts), minlength=12 * N * N)
    exp = pts.shape[1] / (12 * N * N)
    chi2 = np.sum((cnt - exp) ** 2 / exp)
    assert chi2 < 47 + 5 * np.sqrt(2 * 47)     # 47 degrees of freedom, 5 sigma


def _box(rng, n):
    nodes = rng.normal(size=(10, n))
    nodes[9] = rng.uniform(0.5, 2.0, n)
    return nodes


def test_box_place_exact_cases_and_composition():
    rng = np.random.default_rng(3)
    nodes = _box(rng, 50)
    box_off = [0, 20, 50]
    ident = np.r_[np.eye(3).ravel(), 0, 0, 0]
    perm = np.r_[np.array([[0, -1, 0], [1, 0, 0], [0, 0, 1]], float).ravel(), 0.5, -0.25, 2.0]
    out, off = oracle.box_place(nodes, box_off, [1, 0, 1], np.stack([ident, perm, perm]))
    assert list(off) == [0, 30, 50, 80]
    assert np.array_equal(out[:, :30], nodes[:, 20:50])
    b0 = nodes[:, :20]
    exp = b0.copy()
    for blk in range(3):
        x, y = b0[3 * blk], b0[3 * blk + 1]
        exp[3 * blk], exp[3 * blk + 1] = -y, x
    exp[0:3] += np.array([0.5, -0.25, 2.0])[:, None]
    assert np.array_equal(out[:, 30:50], exp)
    # composition: placing twice equals placing once by the product (rounding only)
    q = rng.normal(size=4)
    q /= np.linalg.norm(q)
    w_, x_, y_, z_ = q
    R = np.array([[1 - 2 * (y_ * y_ + z_ * z_), 2 * (x_ * y_ - z_ * w_), 2 * (x_ * z_ + y_ * w_)],
                  [2 * (x_ * y_ + z_ * w_), 1 - 2 * (x_ * x_ + z_ * z_), 2 * (y_ * z_ - x_ * w_)],
                  [2 * (x_ * z_ - y_ * w_), 2 * (y_ * z_ + x_ * w_), 1 - 2 * (x_ * x_ + y_ * y_)]])
    T = rng.normal(size=3)
    A = np.r_[R.ravel(), T]
    once, _ = oracle.box_place(nodes, [0, 50], [0], A[None, :])
    twice, _ = oracle.box_place(once, [0, 50], [0], A[None, :])
    AB = np.r_[(R @ R).ravel(), R @ T + T]
    direct, _ = oracle.box_place(nodes, [0, 50], [0], AB[None, :])
    np.testing.assert_allclose(twice, direct, rtol=0, atol=1e-13)
    np.testing.assert_allclose(np.linalg.norm(once[3:6], axis=0), np.linalg.norm(nodes[3:6], axis=0), rtol=1e-14)
    np.testing.assert_array_equal(once[9], nodes[9])


def test_cone_cut_partition_bounds_order():
    rng = np.random.default_rng(4)
    n = 5000
    S = _box(rng, n)
    S[0:3] = _unit(rng, n) * rng.uniform(0.1, 1.0, n)
    # 12 shells with the same samples, one per base pixel: every sample kept exactly once
    shells = np.tile(S, 12)
    off = np.arange(13) * n
    kept, koff = oracle.cone_cut(shells, off, 1, np.arange(12), np.zeros(12), np.full(12, np.inf))
    assert koff[-1] == n
    base = oracle.vec2pix_ring(1, S[0:3])
    for k in range(12):
        sel = S[:, base == k]
        assert np.array_equal(kept[:, koff[k]:koff[k + 1]], sel)        # input order kept
    # radius bounds: [r_lo, r_hi)
    T = np.zeros((10, 3))
    T[0:3, :] = np.array([[0.0, 0.0, 0.0], [0.3, 0.5, 0.7], [0.0, 0.0, 0.0]])   # radii 0.3, 0.5, 0.7 on +y
    p = oracle.vec2pix_ring(1, T[0:3, :1])[0]
    kept, koff = oracle.cone_cut(T, [0, 3], 1, [p], [0.3], [0.7])
    assert np.allclose(np.linalg.norm(kept[0:3], axis=0), [0.3, 0.5])
