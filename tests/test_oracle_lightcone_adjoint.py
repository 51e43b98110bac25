"""Pins of the oracle's light-cone adjoint and of the dsigma row of its map adjoint.

The chain dL/d(nodes) = dL/d(samples) . d(samples)/d(nodes) differentiates the retarded-time
solve of Eq. (1) (the crossing X cap x_gamma, Sec. II.B) by the implicit-function theorem.
Pinned here by
  * linearity of the map in dsigma (the dsigma gradient times dsigma is the sample's own
    contribution to L, computed by the oracle map of that sample alone),
  * closed forms of a LINEAR node moving radially (dX/dX_b . rhat = 1/(1 + v)) and a static
    node,
  * fourth-order central finite differences of the whole oracle pipeline (light-cone solve
    followed by the map) for LINEAR nodes and BURDEN loop parameters.
"""
import numpy as np
import pytest

import oracle
import synth

THREADS = 4
N = 16


def _loss_of_samples(S, w):
    th, _ = oracle.isw_map(N, S, threads=THREADS)
    return float(np.dot(w, th))


def _linear_nodes(rng, n):
    """Straight-worldline nodes at box time 0.6: positions 0.3-0.5 from the observer,
    |Xdot| in [0.3, 0.85], X' perpendicular with eps = 1, dsigma ~ 1e-3."""
    d = rng.normal(size=(3, n))
    d /= np.linalg.norm(d, axis=0)
    X = d * rng.uniform(0.3, 0.5, n)
    t = rng.normal(size=(3, n))
    t /= np.linalg.norm(t, axis=0)
    v = rng.uniform(0.3, 0.85, n)
    e = rng.normal(size=(3, n))
    e -= t * np.sum(e * t, axis=0)
    e /= np.linalg.norm(e, axis=0)
    Xd = e * v
    Xp = t * np.sqrt(1 - v ** 2)
    ds = rng.uniform(0.5e-3, 2e-3, n)
    return np.vstack([X, Xd, Xp, ds[None, :]])


def test_map_adjoint_dsigma_row_is_linearity():
    rng = np.random.default_rng(3)
    nodes = _linear_nodes(rng, 24)
    S, _, st = oracle.lightcone(oracle.LINEAR, nodes, t_box=0.6)
    assert np.all(st == 0)
    g = rng.normal(size=12 * N * N)
    grad = oracle.isw_map_adjoint(N, S, g, ngrad=10, threads=THREADS)
    g9 = oracle.isw_map_adjoint(N, S, g, ngrad=9, threads=THREADS)
    assert np.array_equal(grad[:9], g9)
    for s in range(S.shape[1]):
        contrib = _loss_of_samples(S[:, s:s + 1], g)
        assert grad[9, s] * S[9, s] == pytest.approx(contrib, rel=1e-12, abs=1e-300)


def test_linear_radial_and_static_closed_forms():
    # radial outward motion with speed v: dX/dX_b along rhat is 1/(1 + v); transverse is 1
    v = 0.6
    rhat = np.array([0.48, -0.6, 0.64])
    e1 = np.array([0.8, 0.64, 0.0])          # perpendicular to rhat
    r0 = 0.45
    t_box = 0.2
    node = np.concatenate([r0 * rhat, v * rhat, 0.7 * e1, [1e-3]])[:, None]
    S, tau, st = oracle.lightcone(oracle.LINEAR, node, t_box=t_box)
    assert st[0] == 0
    D = (1 - t_box - r0) / (1 + v)
    assert tau[0] - t_box == pytest.approx(D, rel=1e-14)
    for gX, expect in ((rhat, rhat / (1 + v)), (e1, e1)):
        gs = np.zeros((10, 1))
        gs[0:3, 0] = gX
        gn, gP = oracle.lightcone_adjoint(oracle.LINEAR, node, None, tau, gs, t_box=t_box)
        assert gP is None
        np.testing.assert_allclose(gn[0:3, 0], expect, rtol=1e-14, atol=1e-15)
        np.testing.assert_allclose(gn[3:6, 0], D * expect, rtol=1e-14, atol=1e-15)
    # static node: the box-time gradient of X is g_X, of Xdot is g_Xdot + (tau - t_box) g_X
    node[3:6, 0] = 0.0
    S, tau, st = oracle.lightcone(oracle.LINEAR, node, t_box=t_box)
    gs = np.random.default_rng(1).normal(size=(10, 1))
    gn, _ = oracle.lightcone_adjoint(oracle.LINEAR, node, None, tau, gs, t_box=t_box)
    np.testing.assert_array_equal(gn[0:3], gs[0:3])
    np.testing.assert_allclose(gn[3:6, 0], gs[3:6, 0] + (1 - t_box - r0) * gs[0:3, 0], rtol=1e-14)
    np.testing.assert_array_equal(gn[6:10], gs[6:10])


def _fd4(f, x0, h):
    return (-f(x0 + 2 * h) + 8 * f(x0 + h) - 8 * f(x0 - h) + f(x0 - 2 * h)) / (12 * h)


def test_linear_chain_vs_finite_differences():
    rng = np.random.default_rng(5)
    nodes = _linear_nodes(rng, 16)
    t_box = 0.6
    S, tau, st = oracle.lightcone(oracle.LINEAR, nodes, t_box=t_box)
    assert np.all(st == 0)
    w = rng.normal(size=12 * N * N)
    gs = oracle.isw_map_adjoint(N, S, w, ngrad=10, threads=THREADS)
    gn, _ = oracle.lightcone_adjoint(oracle.LINEAR, nodes, None, tau, gs, t_box=t_box)
    h = 1e-6
    fd = np.zeros((10, nodes.shape[1]))
    for s in range(nodes.shape[1]):
        for c in range(10):
            def f(x, s=s, c=c):
                one = nodes[:, s:s + 1].copy()
                one[c, 0] = x
                Si, _, sti = oracle.lightcone(oracle.LINEAR, one, t_box=t_box)
                assert sti[0] == 0
                return _loss_of_samples(Si, w)
            hc = h * (1e-3 if c == 9 else 1.0)
            fd[c, s] = _fd4(f, nodes[c, s], hc)
    for sl in (slice(0, 3), slice(3, 6), slice(6, 9), slice(9, 10)):
        e = np.max(np.abs(gn[sl] - fd[sl])) / np.max(np.abs(fd[sl]))
        assert e <= 1e-6, (sl, e)


def _burden_subset(seed=2, loops=(0, 1, 2), stride=8):
    w = synth.config(0, seed=seed)
    ids = w.nodes[0].astype(int)
    sel = np.flatnonzero(np.isin(ids, loops))[::stride]
    return w, np.ascontiguousarray(w.nodes[:, sel])


def test_burden_chain_vs_finite_differences():
    w, nodes = _burden_subset()
    P = np.ascontiguousarray(w.loop_params)
    S, tau, st = oracle.lightcone(oracle.BURDEN, nodes, P, x_obs=w.x_obs, t_obs=w.t_obs)
    assert np.all(st == 0)
    rng = np.random.default_rng(9)
    wpix = rng.normal(size=12 * N * N)
    gs = oracle.isw_map_adjoint(N, S, wpix, ngrad=10, threads=THREADS)
    gn, gP = oracle.lightcone_adjoint(oracle.BURDEN, nodes, P, tau, gs, x_obs=w.x_obs)
    ids = nodes[0].astype(int)
    assert np.all(gn[[0, 2, 3, 4, 5, 6, 7, 8]] == 0)
    assert np.array_equal(gn[9], gs[9])
    assert np.all(gP[13:15] == 0) and np.all(gP[:, 3:] == 0)

    def loss_loop(l, Pl):
        m = ids == l
        Si, _, sti = oracle.lightcone(oracle.BURDEN, nodes[:, m], Pl, x_obs=w.x_obs, t_obs=w.t_obs)
        assert np.all(sti == 0)
        return _loss_of_samples(Si, wpix)

    for l in (0, 1, 2):
        fd = np.zeros(17)
        for q in [*range(13), 15, 16]:
            def f(x, q=q, l=l):
                Pl = P.copy()
                Pl[q, l] = x
                return loss_loop(l, Pl)
            # a rotation entry moved alone takes R off the rotation group and changes
            # 1 - |Xdot|^2, which is small near a cusp: that block needs a shorter step
            h = 1e-7 if 3 <= q < 12 else 1e-6 * (P[12, l] if q in (12, 16) else 1.0)
            fd[q] = _fd4(f, P[q, l], h)
        for blk in (slice(0, 3), slice(3, 12), slice(12, 13), slice(15, 16), slice(16, 17)):
            e = np.max(np.abs(gP[blk, l] - fd[blk])) / np.max(np.abs(fd[blk]))
            assert e <= 1e-6, (l, blk, e)
    # per-node sigma gradient
    for s in (0, 5, 17, 40):
        def f(x, s=s):
            one = nodes[:, s:s + 1].copy()
            one[1, 0] = x
            Si, _, _ = oracle.lightcone(oracle.BURDEN, one, P, x_obs=w.x_obs, t_obs=w.t_obs)
            return _loss_of_samples(Si, wpix)
        fd = _fd4(f, nodes[1, s], 1e-6 * P[12, ids[s]])
        assert gn[1, s] == pytest.approx(fd, rel=1e-6, abs=1e-6 * np.max(np.abs(gn[1])))
