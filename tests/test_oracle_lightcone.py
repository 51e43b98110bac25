"""Pins of the oracle's past-light-cone solve (the "X cap x_gamma" of Eq. 1).

LINEAR: exact roots from mpmath (50 digits) of |r0 + Xdot D| = T - D for the FP64
inputs, plus the closed forms of a static node and of radial motion.
BURDEN: the worldsheet satisfies the Nambu-Goto conformal-gauge constraints
(Xdot.X' = 0, Xdot^2 + X'^2 = 1), its Xdot and X' are the t- and sigma-derivatives of X
(central differences), it is periodic in sigma, its nodes average to the loop centre,
and the solved sample lies on the cone with the root bracketed by sign changes.
"""
import numpy as np
import pytest

import synth

T_OBS = 1.0


def _tol():
    return 4 * float(np.spacing(T_OBS))


def _linear_nodes(rng, n, vmax=0.95):
    X = rng.normal(size=(3, n))
    X *= rng.uniform(0.05, 0.9, n) / np.linalg.norm(X, axis=0)
    V = rng.normal(size=(3, n))
    V *= rng.uniform(0.0, vmax, n) / np.linalg.norm(V, axis=0)
    P = rng.normal(size=(3, n)) * 0.3
    nodes = np.zeros((10, n))
    nodes[0:3], nodes[3:6], nodes[6:9] = X, V, P
    nodes[9] = rng.uniform(1e-4, 1e-3, n)
    return nodes


def test_linear_static_and_radial_closed_forms(oracle_lib):
    rng = np.random.default_rng(1)
    nodes = _linear_nodes(rng, 400)
    nodes[3:6, :200] = 0.0                       # static: tau = t_obs - |X|
    r = nodes[0:3, 200:]
    v = rng.uniform(-0.9, 0.9, 200)
    nodes[3:6, 200:] = v * r / np.linalg.norm(r, axis=0)   # radial: D = (T - R) / (1 + v)
    t_box = 0.55
    out, tau, st = oracle_lib.lightcone(0, nodes, t_box=t_box)
    assert np.all(st == 0)
    R = np.linalg.norm(nodes[0:3], axis=0)
    ref_static = T_OBS - R[:200]
    assert np.max(np.abs(tau[:200] - ref_static)) <= _tol()
    D_ref = ((T_OBS - t_box) - R[200:]) / (1 + v)
    valid = R[200:] + v * D_ref > 0      # the closed form assumes the radius stays positive
    assert valid.sum() > 100
    ref_radial = t_box + D_ref
    assert np.max(np.abs(tau[200:][valid] - ref_radial[valid])) <= 2 * _tol()
    # static nodes do not move; X', Xdot, dsigma are carried unchanged
    assert np.array_equal(out[0:3, :200], nodes[0:3, :200])
    assert np.array_equal(out[3:10], nodes[3:10])


def test_linear_vs_mpmath_root(oracle_lib):
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.dps = 50
    rng = np.random.default_rng(2)
    nodes = _linear_nodes(rng, 300)
    t_box = 0.6
    out, tau, st = oracle_lib.lightcone(0, nodes, t_box=t_box)
    assert np.all(st == 0)
    for s in range(nodes.shape[1]):
        X = [mpmath.mpf(float(x)) for x in nodes[0:3, s]]
        V = [mpmath.mpf(float(x)) for x in nodes[3:6, s]]
        T = mpmath.mpf(T_OBS) - mpmath.mpf(t_box)
        # |X + V D| = T - D, past root (T - D >= 0): solve with findroot from the bisection point
        f = lambda D: mpmath.sqrt(sum((X[k] + V[k] * D) ** 2 for k in range(3))) - (T - D)
        lo, hi = -5, T
        for _ in range(200):
            mid = (lo + hi) / 2
            if f(mid) < 0:
                lo = mid
            else:
                hi = mid
        D = (lo + hi) / 2
        assert abs(float(t_box + D) - tau[s]) <= 2 * _tol(), s
        for k in range(3):
            assert abs(float(X[k] + V[k] * D) - out[k, s]) <= 4 * _tol()
    # residual on the cone
    R = np.linalg.norm(out[0:3], axis=0)
    assert np.max(np.abs(R - (T_OBS - tau))) <= 4 * _tol()


def test_linear_domain_errors(oracle_lib):
    nodes = np.zeros((10, 3))
    nodes[0, :] = 0.5
    nodes[3, 0] = 1.0          # |Xdot| = 1
    nodes[3, 1] = 1.5          # |Xdot| > 1
    nodes[0, 2] = np.nan
    out, tau, st = oracle_lib.lightcone(0, nodes, t_box=0.5)
    assert list(st) == [3, 3, 3]


@pytest.fixture(scope="module")
def loops():
    w = synth.config(0, seed=11)
    return w


def test_burden_constraints_and_derivatives(oracle_lib, loops):
    P = loops.loop_params
    rng = np.random.default_rng(3)

    def deriv(lid, sig, t, dsig, dt):
        # fourth-order central difference along (dsig, dt)
        f = lambda k: oracle_lib.burden_eval(P, lid, sig + k * dsig, t + k * dt)[0]
        return (-f(2) + 8 * f(1) - 8 * f(-1) + f(-2)) / 12.0

    for lid in range(P.shape[1]):
        L = P[12, lid]
        h = 1e-4 * L
        for _ in range(10):
            sig = rng.uniform(0, L)
            t = rng.uniform(0.3, 0.8)
            X, Xd, Xp = oracle_lib.burden_eval(P, lid, sig, t)
            assert abs(Xd @ Xp) <= 2e-15
            assert abs(Xd @ Xd + Xp @ Xp - 1.0) <= 2e-15
            assert np.max(np.abs(deriv(lid, sig, t, 0.0, h) / h - Xd)) <= 1e-8
            assert np.max(np.abs(deriv(lid, sig, t, h, 0.0) / h - Xp)) <= 1e-8
            Xc, _, _ = oracle_lib.burden_eval(P, lid, sig + L, t)
            assert np.max(np.abs(Xc - X)) <= 1e-15


def test_burden_centre_and_cone(oracle_lib, loops):
    P = loops.loop_params
    nodes = loops.nodes
    # the 512 nodes of a loop at a common time average to its centre
    for lid in range(3):
        sel = nodes[0] == lid
        Xs = np.array([oracle_lib.burden_eval(P, lid, s, 0.7)[0] for s in nodes[1, sel]])
        assert np.max(np.abs(Xs.mean(axis=0) - P[0:3, lid])) <= 1e-15
    out, tau, st = oracle_lib.lightcone(1, nodes, P)
    assert np.all(st == 0)
    R = np.linalg.norm(out[0:3], axis=0)
    assert np.max(np.abs(R - (T_OBS - tau))) <= _tol() * 1.0001
    # the sample equals the worldsheet at (sigma, tau) and the root is bracketed
    for s in range(0, nodes.shape[1], 97):
        lid, sig = int(nodes[0, s]), nodes[1, s]
        X, Xd, Xp = oracle_lib.burden_eval(P, lid, sig, tau[s])
        assert np.array_equal(X, out[0:3, s]) and np.array_equal(Xd, out[3:6, s]) and np.array_equal(Xp, out[6:9, s])
        for dt, sign in ((-1e-9, -1), (1e-9, 1)):
            Xq, _, _ = oracle_lib.burden_eval(P, lid, sig, tau[s] + dt)
            assert np.sign(np.linalg.norm(Xq) - (T_OBS - tau[s] - dt)) == sign
    assert np.array_equal(out[9], nodes[9])


def test_burden_iteration_cap(oracle_lib, loops):
    out, tau, st = oracle_lib.lightcone(1, loops.nodes[:, :64], loops.loop_params, max_iter=1)
    assert np.all((st == 4) | (st == 0)) and np.any(st == 4)
    bad = loops.nodes[:, :2].copy()
    bad[0, 0] = 10 ** 6          # loop id out of range
    _, _, st = oracle_lib.lightcone(1, bad, loops.loop_params)
    assert st[0] == 1 and st[1] == 0


def test_burden_no_two_cycles_large_workload(oracle_lib):
    """Every node of the Nside=4096 workload (2e6 samples, 1024 shells) converges: nodes 659026 and
    1117799 of seed 1 once alternated between the bracket ends under plain safeguarded Newton."""
    w = synth.config(4, seed=1)
    S, tau, st = oracle_lib.lightcone_workload(w)
    assert np.all(st == 0)
    R = np.linalg.norm(S[0:3], axis=0)
    assert np.max(np.abs(R - (T_OBS - tau))) <= _tol() * 1.0001
    for node in (659026, 1117799):
        assert w.mode[np.searchsorted(w.shell_off, node, side="right") - 1] == oracle_lib.BURDEN
