"""Pins of the oracle's discrete Eq. (1)-(2) sum and of its adjoint.

* single pair term: an mpmath (40 digits) evaluation of Eq. (1)-(2) in the paper's form
  D = X n - X, including directions within 1e-9 rad of the sample;
* Kaiser-Stebbins: a straight string moving transversally at speed v makes a temperature
  step of 16 GU gamma v atan(L/(2a)) between directions at offsets -a and +a, which tends
  to 8 pi GU gamma v (flat-sky closed form of Eq. 1); line-of-sight motion makes none;
* continuum limit: for a Burden loop the node sum converges spectrally to an mpmath
  quadrature over sigma of Eq. (1) with the retarded time solved at every sigma;
* invariants: linearity in the sample set, proportionality to GU, permutation of the
  samples, exact pixel permutations under a quarter turn about z and a half turn about x,
  scale invariance (X and dsigma scaled together; exact for a factor 2), translation of the
  observer together with the samples;
* special cases: D = 0 gives a zero term, |Xdot| >= 1 samples are skipped (both counted);
* adjoint: central finite differences (h = 1e-6) of L = sum (Theta - Theta_t)^2.
"""
import numpy as np
import pytest

import oracle
import synth


def _mp_term(mpmath, nv, s, GU=1.0):
    mp = mpmath.mpf
    n = [mp(float(x)) for x in nv]
    X = [mp(float(x)) for x in s[0:3]]
    Xd = [mp(float(x)) for x in s[3:6]]
    Xp = [mp(float(x)) for x in s[6:9]]
    ds = mp(float(s[9]))
    Xn = mpmath.sqrt(sum(x * x for x in X))
    D = [Xn * n[k] - X[k] for k in range(3)]
    A = sum(n[k] * Xp[k] for k in range(3))
    B = 1 + sum(n[k] * Xd[k] for k in range(3))
    u = [Xd[k] - A * Xp[k] / B for k in range(3)]
    eps = mpmath.sqrt(sum(x * x for x in Xp) / (1 - sum(x * x for x in Xd)))
    return -4 * GU * sum(u[k] * D[k] for k in range(3)) / sum(x * x for x in D) * eps * ds


def test_pair_term_vs_mpmath(oracle_lib):
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.dps = 40
    rng = np.random.default_rng(4)
    worst = 0.0
    for k in range(600):
        X = rng.normal(size=3)
        X *= rng.uniform(0.01, 1.4) / np.linalg.norm(X)
        Xd = rng.normal(size=3)
        Xd *= rng.uniform(0, 0.9) / np.linalg.norm(Xd)
        Xp = rng.normal(size=3) * rng.uniform(0.01, 1)
        s = np.concatenate([X, Xd, Xp, [rng.uniform(1e-5, 1e-3)]])
        if k % 3 == 0:
            nv = rng.normal(size=3)
        else:                       # near pairs: direction within 1e-9 .. 1e-3 rad of the sample
            off = rng.normal(size=3)
            off -= off @ X * X / (X @ X)
            off *= 10 ** rng.uniform(-9, -3) / np.linalg.norm(off)
            nv = X / np.linalg.norm(X) + off
        nv /= np.linalg.norm(nv)
        got = oracle_lib.pair_term(nv, s)
        ref = _mp_term(mpmath, nv, s)
        # error measured against the term's scale |kappa| |u| / |D| (u.D may cancel); the
        # conditioning of B = 1 + n.Xdot is bounded by |Xdot| <= 0.9
        Xn = np.linalg.norm(X)
        Dn = np.linalg.norm(Xn * nv - X)
        B = 1 + nv @ Xd
        kappa = 4 * s[9] * np.sqrt((Xp @ Xp) / (1 - Xd @ Xd))
        scale = kappa * (np.linalg.norm(Xd) + (Xp @ Xp) / B) / Dn
        rel = abs(got - float(ref)) / scale
        worst = max(worst, rel)
    assert worst <= 2e-15, worst


def _straight_string(R, v, Lz, nn, along):
    z = np.linspace(-Lz / 2, Lz / 2, nn)
    h = z[1] - z[0]
    g = 1 / np.sqrt(1 - v * v)
    nodes = np.zeros((10, nn))
    nodes[1] = R
    nodes[2] = z
    nodes[3 + along] = v
    nodes[8] = np.sqrt(1 - v * v)
    w = np.full(nn, h)
    w[0] = w[-1] = h / 2
    nodes[9] = g * w
    return nodes, g


@pytest.mark.parametrize("a", [1e-5, 1e-4, 1e-3])
def test_kaiser_stebbins_step(oracle_lib, a):
    R, v, Lz = 0.5, 0.6, 1e-2
    nn = 4001                                   # node spacing 2.5e-6 <= a / 4
    nodes, g = _straight_string(R, v, Lz, nn, along=0)
    S, tau, st = oracle_lib.lightcone(0, nodes, t_box=1.0 - R)
    assert np.all(st == 0)
    dirs = np.array([[-a, R, 0.0], [a, R, 0.0]]).T
    dirs /= np.linalg.norm(dirs, axis=0)
    th = oracle_lib.isw_sum_dirs(dirs, S)
    step = th[0] - th[1]
    ref = 16 * g * v * np.arctan(Lz / (2 * a))
    assert abs(step - ref) <= 5e-7 * ref
    assert th[0] > 0 > th[1]                     # cold ahead of the string, hot behind (sign of Eq. 1)
    assert abs(step - 8 * np.pi * g * v) <= 0.13 * 8 * np.pi * g * v
    # motion along the line of sight gives no step
    nodes, g = _straight_string(R, v, Lz, nn, along=1)
    S, _, _ = oracle_lib.lightcone(0, nodes, t_box=1.0 - R)
    th = oracle_lib.isw_sum_dirs(dirs, S)
    assert abs(th[0] - th[1]) <= 1e-6 * ref


def test_continuum_limit_burden_loop(oracle_lib):
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.dps = 30
    mp = mpmath.mpf
    P = synth.config(0, seed=5).loop_params[:, :1].copy()
    P[12, 0], P[13, 0], P[14, 0] = 0.03, 2, 3
    c = [mp(float(x)) for x in P[0:3, 0]]
    Rm = [mp(float(x)) for x in P[3:12, 0]]
    L, m, n, psi, t0 = (mp(float(P[k, 0])) for k in range(12, 17))

    def worldsheet(sig, t):
        u, v = sig - (t - t0), sig + (t - t0)
        ka, kb = 2 * mpmath.pi * m / L, 2 * mpmath.pi * n / L
        a = [mpmath.sin(ka * u) / ka, -mpmath.cos(ka * u) / ka, 0]
        b = [mpmath.sin(kb * v) / kb, -mpmath.cos(psi) * mpmath.cos(kb * v) / kb,
             -mpmath.sin(psi) * mpmath.cos(kb * v) / kb]
        ap = [mpmath.cos(ka * u), mpmath.sin(ka * u), 0]
        bp = [mpmath.cos(kb * v), mpmath.cos(psi) * mpmath.sin(kb * v), mpmath.sin(psi) * mpmath.sin(kb * v)]
        rot = lambda q: [Rm[3 * i] * q[0] + Rm[3 * i + 1] * q[1] + Rm[3 * i + 2] * q[2] for i in range(3)]
        h = rot([(a[k] + b[k]) / 2 for k in range(3)])
        return [c[i] + h[i] for i in range(3)], rot([(bp[k] - ap[k]) / 2 for k in range(3)]), \
            rot([(ap[k] + bp[k]) / 2 for k in range(3)])

    cache = {}

    def on_cone(sig):
        if sig not in cache:
            t = 1 - mpmath.sqrt(sum(x * x for x in c))
            for _ in range(80):
                X, Xd, Xp = worldsheet(sig, t)
                rn = mpmath.sqrt(sum(x * x for x in X))
                f = rn - (1 - t)
                if abs(f) < mp(10) ** -27:
                    break
                t -= f / (1 + sum(X[k] * Xd[k] for k in range(3)) / rn)
            cache[sig] = (X, Xd, Xp)
        return cache[sig]

    def integrand(sig, nv):
        X, Xd, Xp = on_cone(sig)
        return _mp_term_exact(mpmath, nv, X, Xd, Xp)

    cdir = np.array([float(x) for x in c])
    cdir /= np.linalg.norm(cdir)
    rng = np.random.default_rng(0)
    dirs = []
    for ang in (0.2, 1.0, 2.5):
        perp = np.cross(cdir, rng.normal(size=3))
        perp /= np.linalg.norm(perp)
        dirs.append(np.cos(ang) * cdir + np.sin(ang) * perp)
    dirs = np.array(dirs).T
    ref = []
    for k in range(3):
        nv = [mp(float(x)) for x in dirs[:, k]]
        ref.append(float(mpmath.quad(lambda s: integrand(s, nv), [0, L / 4, L / 2, 3 * L / 4, L])))
    errs = {}
    for N in (64, 256, 512):
        S, _, st = oracle_lib.lightcone(1, synth.burden_nodes(P, N), P)
        assert np.all(st == 0)
        th = oracle_lib.isw_sum_dirs(dirs, S)
        errs[N] = np.max(np.abs(th - np.array(ref)))
    assert errs[64] < 1e-5
    assert errs[256] <= 1e-12 and errs[512] <= 1e-12      # spectral convergence of the node rule
    assert errs[64] > 1e3 * errs[256]


def _mp_term_exact(mpmath, n, X, Xd, Xp):
    Xn = mpmath.sqrt(sum(x * x for x in X))
    D = [Xn * n[k] - X[k] for k in range(3)]
    A = sum(n[k] * Xp[k] for k in range(3))
    B = 1 + sum(n[k] * Xd[k] for k in range(3))
    u = [Xd[k] - A * Xp[k] / B for k in range(3)]
    eps = mpmath.sqrt(sum(x * x for x in Xp) / (1 - sum(x * x for x in Xd)))
    return -4 * sum(u[k] * D[k] for k in range(3)) / sum(x * x for x in D) * eps


@pytest.fixture(scope="module")
def small_case(oracle_lib):
    w = synth.config(0, seed=21)
    S, _, st = oracle_lib.lightcone_workload(w)
    assert np.all(st == 0)
    return S[:, ::4].copy()      # 2560 samples


def test_linearity_gu_permutation(oracle_lib, small_case):
    S = small_case
    N = 8
    th, _ = oracle_lib.isw_map(N, S, threads=4)
    rms = np.sqrt(np.mean(th ** 2))
    a, _ = oracle_lib.isw_map(N, S[:, :1000], threads=4)
    b, _ = oracle_lib.isw_map(N, S[:, 1000:], threads=4)
    assert np.max(np.abs(a + b - th)) <= 1e-13 * rms
    g, _ = oracle_lib.isw_map(N, S, GU=3.5e-7, threads=4)
    assert np.max(np.abs(g - 3.5e-7 * th)) <= 1e-13 * 3.5e-7 * rms
    perm = np.random.default_rng(0).permutation(S.shape[1])
    p, _ = oracle_lib.isw_map(N, S[:, perm], threads=4)
    assert np.max(np.abs(p - th)) <= 1e-13 * rms


def _rot_samples(S, M):
    out = S.copy()
    for blk in (0, 3, 6):
        out[blk:blk + 3] = M @ S[blk:blk + 3]
    return out


def test_rotation_symmetries(oracle_lib, small_case):
    S = small_case
    N = 8
    vec, ring, jj = oracle_lib.pix2vec_ring(N)
    th, _ = oracle_lib.isw_map(N, S, threads=4)
    rms = np.sqrt(np.mean(th ** 2))
    quarter = np.array([[0.0, -1, 0], [1, 0, 0], [0, 0, 1]])
    half_x = np.array([[1.0, 0, 0], [0, -1, 0], [0, 0, -1]])
    for M in (quarter, half_x):
        thr, _ = oracle_lib.isw_map(N, _rot_samples(S, M), threads=4)
        rv = M @ vec
        # find the image pixel of every pixel by exact vector match
        key = {tuple(vec[:, p]): p for p in range(vec.shape[1])}
        img = np.array([key[tuple(rv[:, p] + 0.0)] for p in range(vec.shape[1])])
        assert np.max(np.abs(thr[img] - th)) <= 1e-13 * rms


def test_coincident_and_domain(oracle_lib):
    N = 3                                    # odd N: pixel (ring 2N, j = 2N + 1) points along -x exactly
    p = 2 * N * (N - 1) + N * 4 * N + 2 * N
    vec, ring, jj = oracle_lib.pix2vec_ring(N, pix=[p])
    assert ring[0] == 2 * N and jj[0] == 2 * N + 1 and vec[0, 0] == -1.0 and vec[2, 0] == 0.0
    S = np.zeros((10, 3))
    S[0, 0] = -0.5                           # on the line of sight of pixel p: D = 0
    S[3, 0], S[8, 0], S[9, 0] = 0.3, 0.5, 1e-3
    S[1, 1], S[3, 1], S[8, 1], S[9, 1] = 0.4, 1.0, 0.5, 1e-3   # |Xdot| = 1: skipped
    S[2, 2], S[4, 2], S[6, 2], S[9, 2] = 0.7, 0.2, 0.4, 1e-3
    th, stats = oracle_lib.isw_map(N, S, pix=[p])
    ref = oracle_lib.pair_term(vec[:, 0], S[:, 2])
    assert th[0] == ref
    assert stats[0] == 1 and stats[1] == 1


def test_adjoint_vs_finite_differences(oracle_lib):
    w = synth.config(3, seed=2)
    S, _, _ = oracle_lib.lightcone(1, w.nodes[:, :1536], w.loop_params)
    N = 16
    npix = 12 * N * N
    th, _ = oracle_lib.isw_map(N, S, threads=8)
    target = np.random.default_rng(3).normal(size=npix) * np.std(th)
    g = 2 * (th - target)
    grad = oracle_lib.isw_map_adjoint(N, S, g, ngrad=9, threads=8)
    rng = np.random.default_rng(5)
    nodes = rng.choice(S.shape[1], 32, replace=False)
    h = 1e-6
    fd = np.zeros((9, nodes.size))
    for a, s in enumerate(nodes):
        base, _ = oracle_lib.isw_map(N, S[:, s:s + 1], threads=4)
        for c in range(9):
            vals = []
            for sign in (1, -1):
                one = S[:, s:s + 1].copy()
                one[c, 0] += sign * h
                t1, _ = oracle_lib.isw_map(N, one, threads=4)
                vals.append(np.sum((th - base + t1 - target) ** 2))
            fd[c, a] = (vals[0] - vals[1]) / (2 * h)
    an = grad[:, nodes]
    for blk in (slice(0, 3), slice(3, 6), slice(6, 9)):
        scale = np.max(np.abs(an[blk]))
        assert np.max(np.abs(fd[blk] - an[blk])) <= 1e-6 * scale


def test_scale_and_observer_translation():
    """X -> lambda X with dsigma -> lambda dsigma leaves every term unchanged (the weight depends on
    dsigma / |X|, the direction on X / |X|): exactly for lambda = 2, to rounding otherwise.  Moving
    the observer and every sample by the same vector leaves the map unchanged (a use of |X| in
    place of |X - x_obs| anywhere would break it)."""
    w = synth.config(0, seed=6)
    S, _, st = oracle.lightcone(oracle.BURDEN, w.nodes[:, :1024], w.loop_params)
    assert np.all(st == 0)
    N = 8
    th, _ = oracle.isw_map(N, S)
    for lam, exact in ((2.0, True), (2.5, False)):
        T = S.copy()
        T[0:3] *= lam
        T[9] *= lam
        th2, _ = oracle.isw_map(N, T)
        if exact:
            assert np.array_equal(th2, th)
        else:
            np.testing.assert_allclose(th2, th, rtol=0, atol=1e-13 * np.abs(th).max())
    shift = np.array([0.3, -0.7, 0.45])
    T = S.copy()
    T[0:3] += shift[:, None]
    th3, _ = oracle.isw_map(N, T, x_obs=shift)
    np.testing.assert_allclose(th3, th, rtol=0, atol=1e-12 * np.abs(th).max())
