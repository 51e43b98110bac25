"""GPU parity of lightcone_adjoint (the adjoint of the light-cone solve) and of the
end-to-end differentiable map ISWLightconeMap, against the oracle.

Both sides are FP64; they differ only in the order of operations (and, for the per-loop sums,
of additions), so the comparison is relative to the largest magnitude of each gradient block:
<= 1e-12 for node gradients and <= 1e-11 for per-loop sums.  Error paths: a loop whose nodes
are not contiguous gets NaN rows and ISW_EINVAL; an out-of-range loop id gets zero rows and
ISW_EINVAL.
"""
import os

import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

THREADS = os.cpu_count() or 4


@pytest.fixture(scope="module")
def isw():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1204_5041_gb300 as m

    m.build()
    return m


def _d(a, dtype=torch.float64):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda", dtype)


def _blk(got, ref, blocks):
    return max(np.max(np.abs(got[b] - ref[b])) / max(np.max(np.abs(ref[b])), 1e-300) for b in blocks)


NODE_BLOCKS = (slice(0, 3), slice(3, 6), slice(6, 9), slice(9, 10))
LOOP_BLOCKS = (slice(0, 3), slice(3, 12), slice(12, 13), slice(15, 16), slice(16, 17))


@pytest.mark.parametrize("ngs", [6, 9, 10])
def test_linear_nodes_full_shell(isw, ngs):
    """The 80,192 random-walk nodes of the N_side 512 workload (LINEAR, box time 0.6)."""
    w = synth.config(1, seed=1)
    nodes, t_box, mode = w.shell(1)
    assert mode == oracle.LINEAR
    _, tau, st = oracle.lightcone(mode, nodes, None, t_box, w.x_obs, w.t_obs)
    assert np.all(st == 0)
    gs = np.random.default_rng(ngs).normal(size=(ngs, nodes.shape[1]))
    ref, _ = oracle.lightcone_adjoint(mode, nodes, None, tau, gs, t_box=t_box, x_obs=w.x_obs)
    gn, gl = isw.lightcone_adjoint(mode, _d(nodes), _d(tau), _d(gs), t_box=t_box, x_obs=w.x_obs)
    r, _ = isw.default_context().check_status()
    assert r == isw.OK and gl is None
    e = _blk(gn.cpu().numpy(), ref, NODE_BLOCKS if ngs == 10 else NODE_BLOCKS[:2 + (ngs == 9)])
    print(f"lightcone_adjoint LINEAR ngrad={ngs}: max block err {e:.3e}")
    assert e <= 1e-12


def test_burden_loops_full_shell(isw):
    """The 234 Burden loops x 512 nodes of the N_side 512 workload."""
    w = synth.config(1, seed=1)
    nodes, t_box, mode = w.shell(0)
    assert mode == oracle.BURDEN
    P = w.loop_params
    _, tau, st = oracle.lightcone(mode, nodes, P, t_box, w.x_obs, w.t_obs)
    assert np.all(st == 0)
    gs = np.random.default_rng(3).normal(size=(10, nodes.shape[1]))
    ref_n, ref_l = oracle.lightcone_adjoint(mode, nodes, P, tau, gs, x_obs=w.x_obs)
    gn, gl = isw.lightcone_adjoint(mode, _d(nodes), _d(tau), _d(gs), loop_params=_d(P), x_obs=w.x_obs)
    r, _ = isw.default_context().check_status()
    assert r == isw.OK
    gn, gl = gn.cpu().numpy(), gl.cpu().numpy()
    en = _blk(gn, ref_n, (slice(1, 2), slice(9, 10)))
    el = _blk(gl, ref_l, LOOP_BLOCKS)
    print(f"lightcone_adjoint BURDEN: node err {en:.3e}, loop err {el:.3e}")
    assert np.all(gn[[0, 2, 3, 4, 5, 6, 7, 8]] == 0) and np.all(gl[13:15] == 0)
    assert en <= 1e-12 and el <= 1e-11


def test_burden_error_paths(isw):
    w = synth.config(0, seed=2)
    P = w.loop_params
    nodes = np.ascontiguousarray(w.nodes[:, :1024])            # loops 0 and 1, 512 nodes each
    _, tau, st = oracle.lightcone(oracle.BURDEN, nodes, P, 0.0, w.x_obs, w.t_obs)
    gs = np.random.default_rng(4).normal(size=(6, nodes.shape[1]))
    ctx = isw.default_context()
    # loop 0 split into two runs by one node of loop 1
    bad = nodes.copy()
    bad[:, [100, 600]] = bad[:, [600, 100]]
    tb = tau.copy()
    tb[[100, 600]] = tb[[600, 100]]
    gn, gl = isw.lightcone_adjoint(oracle.BURDEN, _d(bad), _d(tb), _d(gs), loop_params=_d(P), x_obs=w.x_obs)
    r, _ = ctx.check_status()
    assert r == isw.EINVAL
    gl = gl.cpu().numpy()
    assert np.all(np.isnan(gl[[0, 1, 2, 15, 16], 0])) and np.all(np.isnan(gl[[0, 1, 2, 15, 16], 1]))
    assert np.all(gl[:, 2:] == 0)                               # loops without nodes
    # an out-of-range loop id: zero node rows, the rest as the oracle
    bad = nodes.copy()
    bad[0, 7] = P.shape[1] + 3
    gn, _ = isw.lightcone_adjoint(oracle.BURDEN, _d(bad), _d(tau), _d(gs), loop_params=_d(P), x_obs=w.x_obs)
    r, _ = ctx.check_status()
    assert r == isw.EINVAL
    gn = gn.cpu().numpy()
    assert np.all(gn[:9, 7] == 0)
    keep = np.arange(nodes.shape[1]) != 7
    ref_n, _ = oracle.lightcone_adjoint(oracle.BURDEN, nodes[:, keep], P, tau[keep], gs[:, keep], x_obs=w.x_obs)
    assert _blk(gn[:, keep], ref_n, (slice(1, 2),)) <= 1e-12
    # host-side argument errors
    with pytest.raises(isw.ISWError):
        isw.lightcone_adjoint(7, _d(nodes), _d(tau), _d(gs), loop_params=_d(P))


def test_map_adjoint_dsigma_row(isw):
    w = synth.config(3, seed=7)
    S, _, st = oracle.lightcone(oracle.BURDEN, w.nodes[:, :1500], w.loop_params)
    assert np.all(st == 0)
    N = 32
    g = np.random.default_rng(8).normal(size=12 * N * N)
    ref = oracle.isw_map_adjoint(N, S, g, ngrad=10, threads=THREADS)
    for prec, tol in (("f64", 1e-10), ("f32c", 1e-6)):
        got = isw.isw_map_adjoint(N, _d(S), _d(g), prec=prec, ngrad=10).cpu().numpy()
        e = _blk(got, ref, NODE_BLOCKS)
        print(f"map adjoint {prec} ngrad=10: max block err {e:.3e}")
        assert e <= tol


@pytest.mark.parametrize("prec,tol", [("f64", 1e-10), ("f32c", 1e-6)])
def test_end_to_end_autograd(isw, prec, tol):
    """ISWLightconeMap: Theta(nodes) through the light cone and the map, both modes, gradients
    of L = sum (Theta - target)^2 against the oracle's chain (oracle map adjoint with 10 rows,
    then the oracle light-cone adjoint); the oracle chain itself is pinned by finite
    differences on the CPU."""
    N = 32
    w = synth.config(1, seed=5)
    rng = np.random.default_rng(6)
    for k in (0, 1):
        nodes, t_box, mode = w.shell(k)
        nodes = np.ascontiguousarray(nodes[:, :2048])
        P = w.loop_params if mode == oracle.BURDEN else None
        S, tau, st = oracle.lightcone(mode, nodes, P, t_box, w.x_obs, w.t_obs)
        assert np.all(st == 0)
        th, _ = oracle.isw_map(N, S, threads=THREADS)
        target = rng.normal(size=th.size) * th.std()
        gs = oracle.isw_map_adjoint(N, S, 2 * (th - target), ngrad=10, threads=THREADS)
        ref_n, ref_l = oracle.lightcone_adjoint(mode, nodes, P, tau, gs, t_box=t_box, x_obs=w.x_obs)
        nd = _d(nodes).requires_grad_(True)
        Pd = _d(P).requires_grad_(True) if P is not None else None
        theta = isw.ISWLightconeMap.apply(nd, Pd, N, mode, t_box, None, w.x_obs, w.t_obs, 1.0, prec)
        loss = ((theta - _d(target)) ** 2).sum()
        loss.backward()
        r, _ = isw.default_context().check_status()
        assert r == isw.OK
        gn = nd.grad.cpu().numpy()
        if mode == oracle.LINEAR:
            e = _blk(gn, ref_n, NODE_BLOCKS)
        else:
            used = np.unique(nodes[0].astype(int))
            e = max(_blk(gn, ref_n, (slice(1, 2), slice(9, 10))),
                    _blk(Pd.grad.cpu().numpy()[:, used], ref_l[:, used], LOOP_BLOCKS))
        print(f"end-to-end {prec} mode {mode}: max block err {e:.3e}")
        assert e <= tol
