"""Pins of the oracle's angular power spectrum (Fig. 4): ring geometry, normalised Legendre
functions, the a_lm definition and C_l.

  * ring geometry (z, pixel count, first pixel, phase) equals pix2vec's (pinned elsewhere);
  * lambda_lm(z) against mpmath's associated Legendre functions at 40 digits (m < 60, l < 140),
    and in the underflow region near a pole (m = 120, l up to 2000, 1 - z = 1e-6) against the
    same recursion carried out in 60-digit arithmetic;
  * a_lm equals its definition, (4 pi / N_pix) sum_p Theta_p conj(Y_lm(n_p)), summed directly
    with scipy's spherical harmonics (an independent implementation) at every pixel;
  * exact symmetries: an azimuthally symmetric map has a_lm = 0 for m not a multiple of 4, a
    north-south odd map has a_lm = 0 for l + m even; a constant map has a_00 = sqrt(4 pi);
  * a band-limited map synthesised with scipy comes back within the equal-weight quadrature
    error (a few 1e-3 at l <= N / 2).
"""
import numpy as np
import pytest

import oracle

mpmath = pytest.importorskip("mpmath")
sp = pytest.importorskip("scipy.special")


@pytest.mark.parametrize("N", [1, 2, 3, 8, 16])
def test_ring_geometry_matches_pix2vec(N):
    v, ring, j = oracle.pix2vec_ring(N)
    for i in range(1, 4 * N):
        z, npx, p0, t0 = oracle.ring_info(N, i)
        assert ring[p0] == i and j[p0] == 1 and ring[p0 + npx - 1] == i
        assert (p0 + npx == 12 * N * N) or ring[p0 + npx] == i + 1
        phi = np.arctan2(v[1, p0], v[0, p0]) / (2 * np.pi) % 1
        assert abs(phi - t0) < 1e-14 and abs(v[2, p0] - z) < 1e-15


def _lam_mp(l, m, z):
    mpmath.mp.dps = 40
    z = mpmath.mpf(z)
    norm = mpmath.sqrt((2 * l + 1) / (4 * mpmath.pi) * mpmath.factorial(l - m) / mpmath.factorial(l + m))
    return norm * mpmath.legenp(l, m, z)       # includes the Condon-Shortley phase


def test_legendre_vs_mpmath():
    rng = np.random.default_rng(3)
    for _ in range(40):
        z = float(rng.uniform(-1, 1))
        m = int(rng.integers(0, 60))
        lmax = m + int(rng.integers(0, 80))
        col = oracle.legendre_column(z, m, lmax)
        for l in range(m, lmax + 1, max(1, (lmax - m) // 7)):
            ref = float(_lam_mp(l, m, z))
            assert col[l] == pytest.approx(ref, rel=1e-11, abs=1e-13)
    # near a pole at large m: lambda_mm underflows double range and the recursion climbs back;
    # reference: the same three-term recursion in 60-digit arithmetic (no underflow), whose
    # formula the checks above pin against legenp
    mpmath.mp.dps = 60
    z, m, lmax = 1 - 1e-6, 120, 2000
    zz = mpmath.mpf(z)
    lam = mpmath.sqrt(1 / (4 * mpmath.pi))
    for k in range(1, m + 1):
        lam *= mpmath.sqrt(mpmath.mpf(2 * k - 1) / (2 * k)) * mpmath.sqrt((1 - zz) * (1 + zz))
    lam *= (-1) ** m * mpmath.sqrt(2 * m + 1)
    ref = {m: lam}
    prev, cur = mpmath.mpf(0), lam
    for l in range(m + 1, lmax + 1):
        if l == m + 1:
            nxt = zz * mpmath.sqrt(2 * m + 3) * cur
        else:
            a_ = mpmath.sqrt(mpmath.mpf(4 * l * l - 1) / (l * l - m * m))
            b_ = mpmath.sqrt(mpmath.mpf((2 * l + 1) * (l + m - 1) * (l - m - 1)) / ((2 * l - 3) * (l * l - m * m)))
            nxt = zz * a_ * cur - b_ * prev
        prev, cur = cur, nxt
        ref[l] = cur
    col = oracle.legendre_column(z, m, lmax)
    assert abs(ref[m]) < 1e-300 and col[m] == 0.0
    seen = 0
    for l in range(m, lmax + 1, 7):
        r = float(ref[l]) if abs(ref[l]) > 1e-290 else 0.0
        if r == 0.0:
            assert abs(col[l]) < 1e-280
        else:
            seen += 1
            assert col[l] == pytest.approx(r, rel=1e-9)
    assert seen > 50


@pytest.mark.parametrize("N,lmax", [(2, 8), (4, 12), (8, 20)])
def test_alm_equals_definition(N, lmax):
    v, _, _ = oracle.pix2vec_ring(N)
    theta = np.arccos(np.clip(v[2], -1, 1))
    phi = np.arctan2(v[1], v[0])
    mp = np.random.default_rng(N).normal(size=v.shape[1])
    alm, cl = oracle.map_alm_cl(N, mp, lmax)
    omega = 4 * np.pi / mp.size
    ref_cl = np.zeros(lmax + 1)
    for l in range(lmax + 1):
        for m in range(l + 1):
            ref = omega * np.sum(mp * np.conj(sp.sph_harm_y(l, m, theta, phi)))
            assert abs(alm[m, l] - ref) <= 1e-12 * max(1.0, abs(ref))
            ref_cl[l] += abs(ref) ** 2 * (1 if m == 0 else 2)
        ref_cl[l] /= 2 * l + 1
    np.testing.assert_allclose(cl, ref_cl, rtol=1e-11, atol=1e-15)


def test_symmetries_and_constant():
    N, lmax = 16, 40
    v, _, _ = oracle.pix2vec_ring(N)
    z = v[2]
    alm, _ = oracle.map_alm_cl(N, np.cos(3 * z) + z ** 2, lmax)
    for m in range(1, lmax + 1):
        if m % 4:
            assert np.abs(alm[m, m:]).max() < 1e-13
    alm, _ = oracle.map_alm_cl(N, np.sin(2 * z) * (1 + v[0] ** 2), lmax)
    for m in range(lmax + 1):
        for l in range(m, lmax + 1):
            if (l + m) % 2 == 0:
                assert abs(alm[m, l]) < 1e-13
    alm, cl = oracle.map_alm_cl(N, np.ones(12 * N * N), 4)
    assert alm[0, 0].real == pytest.approx(np.sqrt(4 * np.pi), rel=1e-14)
    assert cl[0] == pytest.approx(4 * np.pi, rel=1e-14)


def test_band_limited_roundtrip():
    N, L = 32, 16
    v, _, _ = oracle.pix2vec_ring(N)
    theta = np.arccos(np.clip(v[2], -1, 1))
    phi = np.arctan2(v[1], v[0])
    rng = np.random.default_rng(1)
    mp = np.zeros(v.shape[1])
    truth = {}
    for l in range(L + 1):
        for m in range(l + 1):
            a = rng.normal() + (1j * rng.normal() if m else 0.0)
            truth[l, m] = a
            Y = sp.sph_harm_y(l, m, theta, phi)
            mp += (a * Y).real if m == 0 else 2 * (a * Y).real
    alm, _ = oracle.map_alm_cl(N, mp, L)
    err = max(abs(alm[m, l] - truth[l, m]) for (l, m) in truth)
    assert err < 2e-2           # equal-weight quadrature error, measured ~5e-3 here
