"""Edge cases of the newer entry points, on the GPU: empty inputs, single-pixel patches, a
non-orthonormal frame, samples behind the patch plane, l_max = 0, empty boxes, mixed
LINEAR/BURDEN shells in one solve (bit-exact against the oracle) and an empty adjoint."""
import ctypes

import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def isw():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1204_5041_gb300 as m

    m.build()
    return m


def _d(a, dtype=torch.float64):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda", dtype)


def test_patch_edges(isw):
    S = np.zeros((10, 4))
    S[2] = [0.5, 0.5, -0.5, -0.2]           # two in front of the plane, two behind
    S[0] = [0.01, -0.02, 0.0, 0.1]
    S[4] = 0.3
    S[6] = np.sqrt(1 - 0.09)
    S[9] = 1e-3
    frame = np.eye(3)
    # no samples: zeros; with accumulate the output is untouched
    out = isw.isw_map_patch(frame, 5, 0.1, _d(S)[:, :0], approx=isw.FLATSKY)
    assert torch.count_nonzero(out).item() == 0
    pre = torch.full((5, 5), 2.0, dtype=torch.float64, device="cuda")
    isw.isw_map_patch(frame, 5, 0.1, _d(S)[:, :0], approx=isw.FLATSKY, accumulate=True, out=pre)
    assert torch.all(pre == 2.0)
    # single pixel, both approximations, against the oracle
    for approx in (isw.FULLSKY, isw.FLATSKY):
        got = isw.isw_map_patch(frame, 1, 0.05, _d(S), approx=approx, prec="f64").cpu().numpy()
        ref = oracle.isw_map_patch(frame, 1, 0.05, S, approx=approx)
        np.testing.assert_allclose(got, ref, rtol=1e-12, atol=1e-300)
    # only samples behind the plane: the flat sky is zero
    got = isw.isw_map_patch(frame, 4, 0.1, _d(S[:, 2:]), approx=isw.FLATSKY, prec="f32c").cpu().numpy()
    assert np.all(got == 0)
    # a frame that is not orthonormal
    with pytest.raises(isw.ISWError):
        isw.isw_map_patch(np.diag([1.0, 1.0, 1.1]), 4, 0.1, _d(S), approx=isw.FULLSKY)
    with pytest.raises(isw.ISWError):
        isw.isw_map_patch(frame, 4, -0.1, _d(S), approx=isw.FULLSKY)
    r, _ = isw.default_context().check_status()
    assert r == isw.OK


def test_cl_lmax0_and_constant(isw):
    N = 4
    m = np.random.default_rng(0).normal(size=12 * N * N)
    alm, cl = isw.isw_map_cl(N, _d(m), 0, with_alm=True)
    ref_a, ref_cl = oracle.map_alm_cl(N, m, 0)
    assert abs(alm.cpu().numpy()[0, 0] - ref_a[0, 0]) < 1e-14 and abs(cl.cpu().numpy()[0] - ref_cl[0]) < 1e-13
    cl = isw.isw_map_cl(N, _d(np.ones(12 * N * N)), 8).cpu().numpy()
    assert cl[0] == pytest.approx(4 * np.pi, rel=1e-14)


def test_box_place_empty_box_and_shell(isw):
    rng = np.random.default_rng(1)
    nodes = rng.normal(size=(10, 30))
    box_off = [0, 0, 30]                       # box 0 is empty
    place = np.tile(np.r_[np.eye(3).ravel(), 1.0, 2.0, 3.0], (3, 1))
    got, off = isw.box_place(_d(nodes), box_off, [0, 1, 0], _d(place))
    ref, roff = oracle.box_place(nodes, box_off, [0, 1, 0], place)
    assert list(off) == list(roff) == [0, 0, 30, 30]
    assert np.array_equal(got.cpu().numpy(), ref)
    with pytest.raises(isw.ISWError):
        isw.box_place(_d(nodes), box_off, [0, 2, 0], _d(place))


def test_shells_mixed_modes_bitexact(isw):
    w = synth.config(1, seed=2)                 # shell 0 BURDEN loops, shell 1 LINEAR strings
    S, _, st = oracle.lightcone_workload(w)
    assert np.all(st == 0)
    got = isw.lightcone_intersect_shells(_d(w.nodes), w.shell_off, w.t_box, w.mode, loop_params=_d(w.loop_params),
                                         x_obs=w.x_obs, t_obs=w.t_obs)
    r, _ = isw.default_context().check_status()
    assert r == isw.OK
    assert np.array_equal(got.cpu().numpy(), S)


def test_lightcone_adjoint_empty(isw):
    w = synth.config(0, seed=1)
    P = _d(w.loop_params)
    gn, gl = isw.lightcone_adjoint(isw.BURDEN, _d(np.zeros((10, 1)))[:, :0], _d(np.zeros(1))[:0],
                                   _d(np.zeros((6, 1)))[:, :0], loop_params=P)
    assert gn.shape[1] == 0 and torch.count_nonzero(gl).item() == 0
    r, _ = isw.default_context().check_status()
    assert r == isw.OK


@pytest.mark.parametrize("n", [1, 2, 1023, 1024, 1025, 3000])
def test_map_sample_counts_around_sort_blocks(isw, n):
    """The FP32 map's spatial sort works on blocks of 1024 samples: counts at and around the block
    size, and samples that all share one direction (equal sort keys: the stable order decides),
    against the oracle."""
    w = synth.config(1, seed=6)
    S, _, st = oracle.lightcone_workload(w)
    assert np.all(st == 0)
    S = np.ascontiguousarray(S[:, 119808:119808 + n])       # random-walk string samples (scattered)
    nside = 16
    ref, _ = oracle.isw_map(nside, S, threads=8)
    got = isw.isw_map(nside, _d(S), prec="f32c").cpu().numpy()
    r, _ = isw.default_context().check_status()
    assert r == isw.OK
    rms = np.sqrt(np.mean(ref ** 2))
    assert np.max(np.abs(got - ref)) / rms <= 1e-5
    # the same direction for every sample (one Morton key), different velocities
    T = S.copy()
    T[0:3] = S[0:3, :1]
    ref2, _ = oracle.isw_map(nside, T, threads=8)
    got2 = isw.isw_map(nside, _d(T), prec="f32c").cpu().numpy()
    assert isw.default_context().check_status()[0] == isw.OK
    rms2 = np.sqrt(np.mean(ref2 ** 2))
    assert np.max(np.abs(got2 - ref2)) / rms2 <= 1e-5


def test_fma_rate_calibration(isw):
    """isw_fma_rate: the FP32 and FP64 FMA-pipe throughputs the kernels are stated against are
    positive and ordered as on the hardware (GB300's FP64 unit is a small fraction of FP32)."""
    ctx = isw.default_context()
    f32 = ctx.fma_rate("f32c")
    f64 = ctx.fma_rate("f64")
    assert f32 > 1e12 and f64 > 1e10
    assert f32 > 10 * f64
    v = ctypes.c_double()
    assert isw.lib().isw_fma_rate(ctx.handle, 7, ctypes.byref(v), None) == isw.EINVAL   # unknown precision
    assert isw.lib().isw_fma_rate(ctx.handle, isw.F64, None, None) == isw.EINVAL        # no output
