"""The GPU path with the observer away from the origin (x_obs != 0, t_obs != 1) against the
oracle: light-cone solve (bit-exact, both modes), map (FP64 <= 1e-12, FP32c <= 1e-5 of rms),
FP64 adjoint (<= 1e-10 per block) and the flat-sky patch (FP64 <= 1e-12)."""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

XO = np.array([0.11, -0.07, 0.05])
TO = 1.3


@pytest.fixture(scope="module")
def isw():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1204_5041_gb300 as m

    m.build()
    return m


def _d(a, dtype=torch.float64):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda", dtype)


@pytest.fixture(scope="module")
def case():
    w = synth.config(1, seed=3)
    # loops (BURDEN) and strings (LINEAR), a few thousand nodes of each, with the loop centres
    # and the strings moved with the observer so that the geometry stays that of the workload
    loops = np.ascontiguousarray(w.loop_params.copy())
    loops[0:3] += XO[:, None]
    bn = np.ascontiguousarray(w.shell(0)[0][:, :2048])
    ln = np.ascontiguousarray(w.shell(1)[0][:, :3000].copy())
    ln[0:3] += XO[:, None]
    sb, _, st1 = oracle.lightcone(oracle.BURDEN, bn, loops, 0.0, XO, TO)
    sl, _, st2 = oracle.lightcone(oracle.LINEAR, ln, None, 0.6 + (TO - 1.0), XO, TO)
    assert np.all(st1 == 0) and np.all(st2 == 0)
    return loops, bn, ln, sb, sl


def test_lightcone_with_observer(isw, case):
    loops, bn, ln, sb, sl = case
    gb = isw.lightcone_intersect(isw.BURDEN, _d(bn), _d(loops), x_obs=XO, t_obs=TO).cpu().numpy()
    gl = isw.lightcone_intersect(isw.LINEAR, _d(ln), t_box=0.6 + (TO - 1.0), x_obs=XO, t_obs=TO).cpu().numpy()
    assert np.array_equal(gb, sb) and np.array_equal(gl, sl)


def test_map_and_adjoint_with_observer(isw, case):
    _, _, _, sb, sl = case
    S = np.concatenate([sb, sl], axis=1)
    N = 32
    ref, _ = oracle.isw_map(N, S, x_obs=XO, threads=8)
    rms = np.sqrt(np.mean(ref ** 2))
    for prec, tol in (("f64", 1e-12), ("f32c", 1e-5)):
        got = isw.isw_map(N, _d(S), x_obs=XO, prec=prec).cpu().numpy()
        assert np.max(np.abs(got - ref)) / rms <= tol, prec
    g = np.random.default_rng(2).normal(size=ref.size)
    ref_g = oracle.isw_map_adjoint(N, S, g, x_obs=XO, ngrad=10, threads=8)
    got_g = isw.isw_map_adjoint(N, _d(S), _d(g), x_obs=XO, prec="f64", ngrad=10).cpu().numpy()
    for b in (slice(0, 3), slice(3, 6), slice(6, 9), slice(9, 10)):
        assert np.max(np.abs(got_g[b] - ref_g[b])) <= 1e-10 * np.max(np.abs(ref_g[b]))
    r, _ = isw.default_context().check_status()
    assert r == isw.OK


def test_flat_patch_with_observer(isw, case):
    _, _, _, _, sl = case
    d = sl[0:3].mean(axis=1) - XO
    e3 = d / np.linalg.norm(d)
    e1 = np.cross([0.0, 0.0, 1.0], e3)
    e1 /= np.linalg.norm(e1)
    frame = np.stack([e1, np.cross(e3, e1), e3])
    M, width = 64, 0.1
    ref = oracle.isw_map_patch(frame, M, width, sl, approx=oracle.FLATSKY, x_obs=XO, threads=8)
    got = isw.isw_map_patch(frame, M, width, _d(sl), approx=isw.FLATSKY, x_obs=XO, prec="f64").cpu().numpy()
    assert np.max(np.abs(got - ref)) <= 1e-12 * np.sqrt(np.mean(ref ** 2))
