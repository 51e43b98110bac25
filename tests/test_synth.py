"""The seeded input generators keep the recipe the design states: workload sizes, Nambu-Goto
constraints of the string nodes, loop-parameter ranges, determinism, and the stacking geometry
(placements are proper rotations pointing a box axis along the base-pixel cone)."""
import numpy as np
import pytest

import oracle
import synth


@pytest.mark.parametrize("k,nside,n", [(0, 64, 10240), (1, 512, 200000), (3, 256, 50176)])
def test_config_sizes(k, nside, n):
    w = synth.config(k, seed=1)
    assert w.nside == nside and w.n == n and w.nodes.shape == (10, n)
    assert w.shell_off[0] == 0 and w.shell_off[-1] == n and np.all(np.diff(w.shell_off) >= 0)


def test_config_deterministic_and_seeded():
    a, b, c = synth.config(1, seed=4), synth.config(1, seed=4), synth.config(1, seed=5)
    assert np.array_equal(a.nodes, b.nodes) and np.array_equal(a.loop_params, b.loop_params)
    assert not np.array_equal(a.nodes, c.nodes)


def test_string_nodes_constraints():
    w = synth.config(1, seed=2)
    nodes, t_box, mode = w.shell(1)
    assert mode == synth.MODE_LINEAR and t_box == pytest.approx(0.6)
    Xd, Xp = nodes[3:6], nodes[6:9]
    v = np.linalg.norm(Xd, axis=0)
    assert np.all((v >= 0.3) & (v <= 0.85))
    np.testing.assert_allclose(np.sum(Xd * Xp, axis=0), 0, atol=1e-14)          # Xdot . X' = 0
    np.testing.assert_allclose(v ** 2 + np.sum(Xp ** 2, axis=0), 1, atol=1e-14)  # eps = 1
    # the length element |X'| dsigma is the node's share of the polyline (half of each adjacent
    # step): per string the shares add up to the polyline length; eps dsigma = gamma * share
    X = nodes[0:3]
    eps = np.sqrt(np.sum(Xp ** 2, axis=0) / (1 - v ** 2))
    np.testing.assert_allclose(eps, 1, atol=1e-14)
    share = np.linalg.norm(Xp, axis=0) * nodes[9]
    np.testing.assert_allclose(eps * nodes[9], share / np.sqrt(1 - v ** 2), rtol=1e-13)
    steps = np.linalg.norm(np.diff(X, axis=1), axis=0)
    breaks = np.flatnonzero(steps > 0.01)            # different strings start far apart
    starts = np.r_[0, breaks + 1]
    ends = np.r_[breaks + 1, X.shape[1]]
    for a, b in zip(starts, ends):
        assert np.sum(share[a:b]) == pytest.approx(np.sum(steps[a:b - 1]), rel=1e-12)


def test_loop_parameters():
    w = synth.config(0, seed=3)
    P = w.loop_params
    R = P[3:12].T.reshape(-1, 3, 3)
    np.testing.assert_allclose(R @ np.transpose(R, (0, 2, 1)), np.broadcast_to(np.eye(3), R.shape), atol=1e-13)
    np.testing.assert_allclose(np.linalg.det(R), 1, atol=1e-13)
    L, m, n, psi, t0 = P[12], P[13], P[14], P[15], P[16]
    assert np.all((L >= 0.01) & (L <= 0.1))
    assert np.all(np.isin(m, [1, 2, 3, 4, 5])) and np.all(np.isin(n, [1, 2, 3, 4, 5]))
    assert np.all((psi >= 0) & (psi < np.pi)) and np.all((t0 >= 0) & (t0 < L))
    d = np.linalg.norm(P[0:3], axis=0)
    assert np.all((d >= 0.3) & (d <= 0.5))
    ids = w.nodes[0]
    assert np.array_equal(ids, np.floor(ids)) and np.all(np.diff(ids) >= 0)   # loops contiguous
    np.testing.assert_allclose(w.nodes[9], L[ids.astype(int)] / 512, rtol=1e-15)


def test_stacking_geometry():
    w = synth.stack_config(seed=0, nside=64)
    assert w.nshell == 12 and w.nside_hz == 1 and list(w.shell_box) == [0, 0, 0, 1, 1, 1, 2, 2, 2, 3, 3, 3]
    centres, _, _ = oracle.pix2vec_ring(1)
    np.testing.assert_allclose(synth.base_pixel_centres(), centres.T, atol=1e-15)
    for k in range(12):
        R = w.place[k, :9].reshape(3, 3)
        np.testing.assert_allclose(R @ R.T, np.eye(3), atol=1e-14)
        assert np.linalg.det(R) == pytest.approx(1.0, abs=1e-14)
        axis = centres[:, k]
        np.testing.assert_allclose(R[:, k % 3], axis, atol=1e-14)               # depth axis e_(k mod 3)
        np.testing.assert_allclose(w.place[k, 9:], 0.6 * axis, atol=1e-14)
    assert np.all(w.t_box == pytest.approx(0.4)) and np.all(w.r_lo == 0.3) and np.all(w.r_hi == 0.9)
    assert w.n_placed == 3 * (w.box_off[-1])
