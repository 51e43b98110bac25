"""Pins of the oracle's trig and HEALPix RING pix2vec against facts outside the oracle.

* sin/cos: mpmath at 40 digits.
* ring indices: brute-force enumeration ring by ring with a counter.
* z: exact rational from the equal-area identity (pixel counts above and in a ring),
  compared with Python's correctly rounded Fraction -> float.
* centres at N_side = 1: the published base-pixel layout (tests/golden).
* direction: mpmath evaluation of (sin theta cos phi, sin theta sin phi, z) from exact z, phi.
* symmetries: quarter-turn rotation about z, and the half-turn about x, map pixels to
  pixels with exactly rotated vectors.
"""
import math
import os
from fractions import Fraction

import numpy as np
import pytest

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _ulp(x):
    return float(np.spacing(abs(float(x))))


def test_sincospi_frac_vs_mpmath(oracle_lib):
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.dps = 40
    rng = np.random.default_rng(7)
    cases = [(a, b) for b in range(1, 41) for a in range(-b, 2 * b + 1)]
    cases += [(int(a), int(b)) for b in rng.integers(41, 1 << 22, 60) for a in rng.integers(-3 * b, 3 * b, 20)]
    worst = 0.0
    for a, b in cases:
        s, c = oracle_lib.sincospi_frac(a, b)
        x = mpmath.mpf(a) / b
        for v, e in ((s, mpmath.sinpi(x)), (c, mpmath.cospi(x))):
            e = float(e)
            err = abs(v - e)
            # two roundings in the argument f*pi/4 plus the series: within 2 ulp of the value,
            # and exact zeros / ones at multiples of pi/2
            tol = 2.0 * _ulp(e) if e != 0.0 else 0.0
            assert err <= tol, (a, b, v, e)
            if e != 0:
                worst = max(worst, err / _ulp(e))
    assert worst <= 2.0


def test_sincos_turns_vs_mpmath(oracle_lib):
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.dps = 40
    rng = np.random.default_rng(8)
    ws = np.concatenate([rng.uniform(-3, 3, 1500), rng.uniform(-1e4, 1e4, 500), [0.0, 0.125, 0.25, 0.5, 1.0, -0.25]])
    for w in ws:
        s, c = oracle_lib.sincos_turns(float(w))
        x = 2 * mpmath.pi * mpmath.mpf(float(w))
        assert abs(s - float(mpmath.sin(x))) <= 1.0 * np.spacing(1.0)
        assert abs(c - float(mpmath.cos(x))) <= 1.0 * np.spacing(1.0)
    s, c = oracle_lib.sincos_turns(0.25)
    assert s == 1.0 and c == 0.0
    s, c = oracle_lib.sincos_turns(0.5)
    assert s == 0.0 and c == -1.0


def _brute_rings(N):
    """(ring, j) of every RING pixel, by walking rings 1..4N-1 with a counter."""
    ring, jj = [], []
    for i in range(1, 4 * N):
        if i < N:
            cnt = 4 * i
        elif i <= 3 * N:
            cnt = 4 * N
        else:
            cnt = 4 * (4 * N - i)
        ring += [i] * cnt
        jj += list(range(1, cnt + 1))
    return np.array(ring), np.array(jj)


@pytest.mark.parametrize("N", [1, 2, 3, 4, 5, 6, 7, 8, 13, 64, 1024])
def test_ring_indices_bruteforce(oracle_lib, N):
    vec, ring, jj = oracle_lib.pix2vec_ring(N)
    assert vec.shape[1] == 12 * N * N
    r_ref, j_ref = _brute_rings(N)
    assert np.array_equal(ring, r_ref)
    assert np.array_equal(jj, j_ref)


@pytest.mark.parametrize("N", [1, 2, 3, 7, 8, 13, 64, 255, 4096])
def test_z_equal_area_exact(oracle_lib, N):
    """Equal area: the centre of ring i sits where the area above it is 2*(pixels above) + (pixels in ring)
    half-pixels, i.e. 1 - z_i = (2 C_above + C_i) / N_pix exactly."""
    npix = 12 * N * N
    above = 0
    first = 0
    rings = range(1, 4 * N) if N <= 64 else list(range(1, 40)) + list(range(N - 3, N + 4)) + list(range(2 * N - 2, 2 * N + 3)) + list(range(4 * N - 40, 4 * N))
    counts = {}
    for i in range(1, 4 * N):
        counts[i] = 4 * i if i < N else (4 * N if i <= 3 * N else 4 * (4 * N - i))
    start = {}
    acc = 0
    for i in range(1, 4 * N):
        start[i] = acc
        acc += counts[i]
    assert acc == npix
    for i in rings:
        above = start[i]
        first = start[i]
        z_exact = 1 - Fraction(2 * above + counts[i], npix)
        vec, ring, _ = oracle_lib.pix2vec_ring(N, pix=[first, first + counts[i] - 1])
        assert ring[0] == i
        assert vec[2, 0] == float(z_exact), (N, i)
        assert vec[2, 1] == float(z_exact)


def test_golden_nside1(oracle_lib):
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.dps = 40
    rows = [list(map(int, l.split())) for l in open(os.path.join(GOLDEN, "healpix_nside1.txt")) if l.strip() and not l.startswith("#")]
    vec, ring, jj = oracle_lib.pix2vec_ring(1)
    for p, r, j, zn, zd, fn, fd in rows:
        assert ring[p] == r and jj[p] == j
        z = mpmath.mpf(zn) / zd
        phi = mpmath.pi * mpmath.mpf(fn) / fd
        st = mpmath.sqrt(1 - z * z)
        ref = [float(st * mpmath.cos(phi)), float(st * mpmath.sin(phi)), float(z)]
        for k in range(3):
            assert abs(vec[k, p] - ref[k]) <= 2 * np.spacing(1.0), (p, k)


def test_golden_paper_counts():
    rows = [l.split(None, 4) for l in open(os.path.join(GOLDEN, "paper_counts.txt")) if l.strip() and not l.startswith("#")]
    for name, nside, val, rtol, _cite in rows:
        N, val, rtol = int(nside), float(val), float(rtol)
        npix = 12 * N * N
        if name == "resolution_arcmin":
            got = math.degrees(math.sqrt(4 * math.pi / npix)) * 60
        else:
            got = npix
        assert abs(got - val) <= rtol * val, (name, got, val)


@pytest.mark.parametrize("N", [1, 2, 3, 8, 16, 37])
def test_direction_vs_mpmath(oracle_lib, N):
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.dps = 40
    vec, ring, jj = oracle_lib.pix2vec_ring(N)
    rng = np.random.default_rng(N)
    idx = np.arange(vec.shape[1]) if vec.shape[1] <= 800 else rng.choice(vec.shape[1], 800, replace=False)
    for p in idx:
        i, j = int(ring[p]), int(jj[p])
        if i < N or i > 3 * N:
            ic = i if i < N else 4 * N - i
            z = 1 - mpmath.mpf(ic * ic) / (3 * N * N)
            if i > 3 * N:
                z = -z
            phi = mpmath.pi * (2 * j - 1) / (4 * ic)
        else:
            z = mpmath.mpf(4 * N - 2 * i) / (3 * N)
            f = mpmath.mpf(1) if (i + N) % 2 else mpmath.mpf(1) / 2
            phi = mpmath.pi * (j - f) / (2 * N)
        st = mpmath.sqrt(1 - z * z)
        ref = (st * mpmath.cos(phi), st * mpmath.sin(phi), z)
        for k in range(3):
            assert abs(vec[k, p] - float(ref[k])) <= 3 * np.spacing(1.0), (N, p, k)


def _pixel_of(N, i, j):
    """RING index of ring i (1..4N-1), position j (1-based)."""
    if i < N:
        return 2 * i * (i - 1) + j - 1
    if i <= 3 * N:
        return 2 * N * (N - 1) + (i - N) * 4 * N + j - 1
    ic = 4 * N - i
    return 12 * N * N - 2 * ic * (ic + 1) + j - 1


@pytest.mark.parametrize("N", [1, 2, 3, 4, 8, 13, 64])
def test_symmetries_exact(oracle_lib, N):
    vec, ring, jj = oracle_lib.pix2vec_ring(N)
    npix = 12 * N * N
    for p in range(npix):
        i, j = int(ring[p]), int(jj[p])
        cnt = 4 * i if i < N else (4 * N if i <= 3 * N else 4 * (4 * N - i))
        assert _pixel_of(N, i, j) == p
        # quarter turn about z: phi -> phi + pi/2 is a shift by cnt/4 within the ring
        q = _pixel_of(N, i, (j - 1 + cnt // 4) % cnt + 1)
        assert vec[0, q] == -vec[1, p] and vec[1, q] == vec[0, p] and vec[2, q] == vec[2, p]
        # half turn about x: (x, y, z) -> (x, -y, -z): ring i -> 4N - i, phi -> -phi
        s = 1 if (i < N or i > 3 * N) else (2 if (i + N) % 2 else 1)
        jm = ((1 - j) % cnt) + 1 if s == 2 else cnt + 1 - j
        m = _pixel_of(N, 4 * N - i, jm)
        assert vec[0, m] == vec[0, p] and vec[1, m] == -vec[1, p] and vec[2, m] == -vec[2, p], (N, p, m)


def test_unit_norm(oracle_lib):
    vec, _, _ = oracle_lib.pix2vec_ring(512)
    nrm = np.sqrt((vec * vec).sum(axis=0))
    assert np.max(np.abs(nrm - 1.0)) <= 4 * np.spacing(1.0)
