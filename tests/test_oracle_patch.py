"""Pins of the oracle's patch maps (Sec. II.A: the flat-sky / small-angle limit X n -> X with
parallel photon paths; Fig. 3: full sky against flat sky on a gnomonic patch).

  * flat sky, straight segment along e1 at depth Z moving with speed v along e2: the discrete
    sum reaches the Kaiser-Stebbins closed form -4 GU gamma v [atan((L - dxi)/deta) +
    atan((L + dxi)/deta)] (angular half-length L), i.e. the step 8 pi GU gamma v for a long
    string;
  * full sky on the same patch approaches the flat-sky map at the patch centre linearly in
    the patch width;
  * samples behind the patch plane (depth <= 0) are dropped by the flat sky; linear in GU.
"""
import numpy as np
import pytest

import oracle

FRAME = np.eye(3)        # e1 = x, e2 = y, e3 = z


def _segment(Lam, Z, v, eta0=0.0, nodes=40000, xi_c=0.0):
    """Midpoint-rule nodes of a straight segment along e1 spanning angular [-Lam, Lam] + xi_c at
    depth Z, offset eta0, moving along e2 with speed v (eps = 1, d(sigma) = gamma ds)."""
    h = 2 * Lam / nodes
    xi = xi_c - Lam + (np.arange(nodes) + 0.5) * h
    g = 1 / np.sqrt(1 - v * v)
    S = np.zeros((10, nodes))
    S[0] = xi * Z
    S[1] = eta0 * Z
    S[2] = Z
    S[4] = v
    S[6] = np.sqrt(1 - v * v)
    S[9] = g * (h * Z)
    return S


def test_flat_sky_kaiser_stebbins_closed_form():
    M, width = 9, 0.09          # pixel pitch 0.01, centre pixel at xi = eta = 0
    Lam, Z, v = 0.02, 0.5, 0.6
    S = _segment(Lam, Z, v)
    th = oracle.isw_map_patch(FRAME, M, width, S, approx=oracle.FLATSKY, threads=4)
    g = 1 / np.sqrt(1 - v * v)
    pitch = width / M
    for j in range(M):
        deta = (j - 4) * pitch
        for i in range(M):
            dxi = (i - 4) * pitch
            if deta == 0:
                continue
            ref = -4 * g * v * (np.arctan((Lam - dxi) / deta) + np.arctan((Lam + dxi) / deta))
            assert th[j, i] == pytest.approx(ref, rel=1e-7, abs=1e-9)
    # long string: the step across it tends to 8 pi gamma v
    S = _segment(2.0, Z, v, nodes=400000)
    th = oracle.isw_map_patch(FRAME, 3, 0.003, S, approx=oracle.FLATSKY, threads=4)
    step = th[0, 1] - th[2, 1]
    assert step == pytest.approx(8 * np.pi * g * v, rel=2e-3)


def test_full_sky_approaches_flat_at_centre():
    rng = np.random.default_rng(1)
    diffs = []
    for width in (4e-3, 4e-4):
        S = _segment(0.3 * width, 0.5, 0.5, eta0=0.11 * width, nodes=4000, xi_c=0.05 * width)
        S[5] = 0.2                     # some line-of-sight velocity as well
        S[3] = rng.uniform(-0.1, 0.1, S.shape[1])
        full = oracle.isw_map_patch(FRAME, 5, width, S, approx=oracle.FULLSKY, threads=4)
        flat = oracle.isw_map_patch(FRAME, 5, width, S, approx=oracle.FLATSKY, threads=4)
        diffs.append(np.max(np.abs(full - flat)) / np.max(np.abs(flat)))
    assert diffs[0] < 1e-2
    assert 5 < diffs[0] / diffs[1] < 20          # first order in the patch width


def test_flat_sky_behind_plane_and_linearity():
    S = _segment(0.01, 0.5, 0.4, eta0=0.003, nodes=2000)
    B = S.copy()
    B[2] = -0.5
    a = oracle.isw_map_patch(FRAME, 7, 0.02, S, approx=oracle.FLATSKY)
    b = oracle.isw_map_patch(FRAME, 7, 0.02, np.concatenate([S, B], axis=1), approx=oracle.FLATSKY)
    assert np.array_equal(a, b)
    c = oracle.isw_map_patch(FRAME, 7, 0.02, S, approx=oracle.FLATSKY, GU=3.0)
    np.testing.assert_allclose(c, 3 * a, rtol=1e-15, atol=0)
    # full sky on a patch equals the full-sky sum at those directions
    M, width = 4, 0.02
    full = oracle.isw_map_patch(FRAME, M, width, S, approx=oracle.FULLSKY)
    h = width / M
    xi = (np.arange(M) + 0.5 - M / 2) * h
    XI, ETA = np.meshgrid(xi, xi)
    dirs = np.stack([XI.ravel(), ETA.ravel(), np.ones(M * M)])
    dirs /= np.linalg.norm(dirs, axis=0)
    ref = oracle.isw_sum_dirs(dirs, S)
    np.testing.assert_allclose(full.ravel(), ref, rtol=1e-13, atol=1e-13 * np.abs(ref).max())
