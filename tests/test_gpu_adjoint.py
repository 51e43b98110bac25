"""GPU parity of the adjoint (isw_map_adjoint, and the torch.autograd.Function ISWMap).

Loss L = sum_p (Theta_p - Theta_target_p)^2, g = dL/dTheta = 2 (Theta - Theta_target).
Gradients are compared per block (dL/dX, dL/dXdot, dL/dX') relative to the largest
magnitude of that block over the compared samples:
  FP64 GPU vs oracle analytic gradient <= 1e-10, FP32-compensated GPU vs oracle <= 1e-6,
  both GPU precisions vs oracle central finite differences (h = 1e-6, fourth-order
  stencil: the second-order one carries ~1e-5 truncation error for pixels within 1e-4 of a
  sample at Nside=256) <= 1e-6.
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


def _blockerr(got, ref):
    out = []
    for blk in range(got.shape[0] // 3):
        sl = slice(3 * blk, 3 * blk + 3)
        out.append(np.max(np.abs(got[sl] - ref[sl])) / np.max(np.abs(ref[sl])))
    return max(out)


def _fd(N, S, th, target, nodes, h=1e-6, pix=None):
    """Central finite differences of L (fourth-order stencil, step h = 1e-6) for the given
    samples and each of the 9 components, using Theta(x + k h) = Theta - t(x) + t(x + k h)
    and L(x + k h) - L(x) = sum D (2 r + D) with D = t(x + k h) - t(x)."""
    r = th - target
    fd = np.zeros((9, len(nodes)))
    for a, s in enumerate(nodes):
        base, _ = oracle.isw_map(N, S[:, s:s + 1], pix=pix, threads=THREADS)
        for c in range(9):
            dl = {}
            for k in (2, 1, -1, -2):
                one = S[:, s:s + 1].copy()
                one[c, 0] += k * h
                t1, _ = oracle.isw_map(N, one, pix=pix, threads=THREADS)
                D = t1 - base
                dl[k] = np.sum(D * (2 * r + D))
            fd[c, a] = (-dl[2] + 8 * dl[1] - 8 * dl[-1] + dl[-2]) / (12 * h)
    return fd


@pytest.fixture(scope="module")
def small():
    w = synth.config(3, seed=7)
    S, _, st = oracle.lightcone(oracle.BURDEN, w.nodes[:, :4 * 512 + 77], w.loop_params)
    assert np.all(st == 0)
    N = 32
    th, _ = oracle.isw_map(N, S, threads=THREADS)
    target = np.random.default_rng(8).normal(size=th.size) * np.std(th)
    g = 2 * (th - target)
    ref = oracle.isw_map_adjoint(N, S, g, ngrad=9, threads=THREADS)
    return N, S, th, target, g, ref


@pytest.mark.parametrize("prec,tol", [("f64", 1e-10), ("f32c", 1e-6)])
def test_adjoint_vs_oracle_small(isw, small, prec, tol):
    N, S, th, target, g, ref = small
    for ngrad in (6, 9):
        got = isw.isw_map_adjoint(N, _d(S), _d(g), prec=prec, ngrad=ngrad).cpu().numpy()
        r, counts = isw.default_context().check_status()
        assert r == isw.OK
        e = _blockerr(got, ref[:ngrad])
        print(f"adjoint {prec} ngrad={ngrad}: max block err = {e:.3e}; counts {counts}")
        assert e <= tol


def test_adjoint_mixed_sign_weights(isw, small):
    """dsigma of random sign (weights of both signs in every tile) and a negative GU, against the
    oracle's gradient; the gradient is linear in GU at fixed g."""
    N, S, th, target, g, _ = small
    S2 = S.copy()
    flip = np.random.default_rng(22).random(S.shape[1]) < 0.5
    S2[9, flip] *= -1.0
    ref = oracle.isw_map_adjoint(N, S2, g, ngrad=10, threads=THREADS)
    for prec, tol in (("f64", 1e-10), ("f32c", 1e-6)):
        got = isw.isw_map_adjoint(N, _d(S2), _d(g), prec=prec, ngrad=10).cpu().numpy()
        assert isw.default_context().check_status()[0] == isw.OK
        neg = isw.isw_map_adjoint(N, _d(S2), _d(g), prec=prec, ngrad=10, GU=-1.0).cpu().numpy()
        e, en = _blockerr(got[:9], ref[:9]), _blockerr(neg[:9], -ref[:9])
        e10 = np.max(np.abs(got[9] - ref[9])) / np.max(np.abs(ref[9]))
        print(f"adjoint mixed-sign {prec}: {e:.3e}, at -GU {en:.3e}, dsigma row {e10:.3e}")
        assert e <= tol and en <= tol and e10 <= tol


def test_adjoint_splits_and_list(isw, small):
    N, S, th, target, g, ref = small
    ctx = isw.default_context()
    try:
        for split in (1, 5):
            ctx.set_param(isw.PARAM_SPLIT, split)
            for prec, tol in (("f64", 1e-10), ("f32c", 1e-6)):
                got = isw.isw_map_adjoint(N, _d(S), _d(g), prec=prec).cpu().numpy()
                assert _blockerr(got, ref[:6]) <= tol
    finally:
        ctx.set_param(isw.PARAM_SPLIT, 0)
    # pixel list with repeats: the gradient of sum over the list
    rng = np.random.default_rng(2)
    pix = rng.integers(0, 12 * N * N, 3001)
    gl = rng.normal(size=pix.size)
    ref_l = oracle.isw_map_adjoint(N, S, gl, pix=pix, threads=THREADS)
    for prec, tol in (("f64", 1e-10), ("f32c", 1e-6)):
        got = isw.isw_map_adjoint(N, _d(S), _d(gl), pix=_d(pix, torch.int64), prec=prec).cpu().numpy()
        assert _blockerr(got, ref_l) <= tol


def test_adjoint_vs_finite_differences_small(isw, small):
    N, S, th, target, g, ref = small
    nodes = np.random.default_rng(11).choice(S.shape[1], 16, replace=False)
    fd = _fd(N, S, th, target, nodes)
    for prec in ("f64", "f32c"):
        got = isw.isw_map_adjoint(N, _d(S), _d(g), prec=prec, ngrad=9).cpu().numpy()[:, nodes]
        e = _blockerr(got, fd)
        print(f"adjoint {prec} vs FD: {e:.3e}")
        assert e <= 1e-6


def test_autograd_function(isw, small):
    N, S, th, target, g, ref = small
    Sd = _d(S).requires_grad_(True)
    tt = _d(target)
    for prec, tol in (("f64", 1e-10), ("f32c", 1e-6)):
        Sd.grad = None
        theta = isw.ISWMap.apply(Sd, N, None, None, 1.0, prec, 9)
        loss = ((theta - tt) ** 2).sum()
        loss.backward()
        grad = Sd.grad.cpu().numpy()
        assert np.all(grad[9] == 0)
        assert _blockerr(grad[:9], ref) <= tol


def test_adjoint_nside256_50k_sampled(isw):
    """The adjoint workload at full size (Nside=256, 98 loops x 512 samples): gradients of
    32 random samples against the oracle's analytic gradient and central differences."""
    w = synth.config(3, seed=1)
    S, _, st = oracle.lightcone_workload(w)
    assert np.all(st == 0)
    N = w.nside
    Sd = _d(S)
    th, _ = oracle.isw_map(N, S, threads=THREADS)          # the loss is built from the oracle's map
    target = np.random.default_rng(2).normal(size=w.npix) * float(th.std())
    g = 2 * (th - target)
    nodes = np.sort(np.random.default_rng(5).choice(S.shape[1], 32, replace=False))
    ref = oracle.isw_map_adjoint(N, np.ascontiguousarray(S[:, nodes]), g, ngrad=9, threads=THREADS)
    fd = _fd(N, S, th, target, nodes[:8])
    assert _blockerr(ref[:, :8], fd) <= 1e-6
    for prec, tol in (("f64", 1e-10), ("f32c", 1e-6)):
        got = isw.isw_map_adjoint(N, Sd, _d(g), prec=prec, ngrad=9).cpu().numpy()[:, nodes]
        r, counts = isw.default_context().check_status()
        assert r == isw.OK
        e = _blockerr(got, ref)
        efd = _blockerr(got[:, :8], fd)
        print(f"nside256 adjoint {prec}: max block err vs oracle = {e:.3e}, vs FD = {efd:.3e}; counts {counts}")
        assert e <= tol and efd <= 1e-6
