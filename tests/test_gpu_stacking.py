"""GPU parity of the stacking calls (Sec. III.B, Fig. 1): hp_vec2pix_ring, box_place,
lightcone_intersect_shells, cone_cut and the stacked map, against the oracle.

Placement, light-cone solve, pixel assignment and the cut are integer decisions or exact
IEEE sequences on both sides: bit-identical.  The stacked map follows the map's bar (FP64
<= 1e-12, FP32c <= 1e-5 of the map rms) on sampled pixels of the full sky.
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


@pytest.mark.parametrize("N", [1, 2, 16, 512, 4096, 1 << 20])
def test_vec2pix_bitexact(isw, N):
    rng = np.random.default_rng(N % 1000)
    v = rng.normal(size=(3, 1000000)) * np.exp(rng.uniform(-5, 5, 1000000))
    v[:, :6] = [[1, -1, 0, 0, 0, 0], [0, 0, 1, -1, 0, 0], [0, 0, 0, 0, 1, -1]]
    ref = oracle.vec2pix_ring(N, v)
    got = isw.hp_vec2pix_ring(N, _d(v)).cpu().numpy()
    assert np.array_equal(got, ref)
    r, _ = isw.default_context().check_status()
    assert r == isw.OK


def test_vec2pix_centres_roundtrip(isw):
    for N in (64, 1024):
        p = np.arange(12 * N * N) if N == 64 else np.random.default_rng(1).choice(12 * N * N, 200000, replace=False)
        vec = isw.hp_pix2vec_ring(N, pix=_d(p, torch.int64))
        assert np.array_equal(isw.hp_vec2pix_ring(N, vec).cpu().numpy(), p)


def test_vec2pix_bad_direction(isw):
    v = np.zeros((3, 4))
    v[:, 1] = [1.0, 0.0, 0.0]
    v[0, 2] = np.nan
    got = isw.hp_vec2pix_ring(8, _d(v)).cpu().numpy()
    r, _ = isw.default_context().check_status()
    assert r == isw.EINVAL
    assert got[0] == -1 and got[2] == -1 and got[1] == oracle.vec2pix_ring(8, v[:, 1:2])[0]


@pytest.fixture(scope="module")
def stack():
    w = synth.stack_config(seed=3, nside=512)
    placed, off = oracle.box_place(w.nodes_box, w.box_off, w.shell_box, w.place)
    S = np.zeros_like(placed)
    for k in range(w.nshell):
        s, _, st = oracle.lightcone(oracle.LINEAR, placed[:, off[k]:off[k + 1]], None, w.t_box[k], w.x_obs,
                                    w.t_obs)
        assert np.all(st == 0)
        S[:, off[k]:off[k + 1]] = s
    kept, koff = oracle.cone_cut(S, off, w.nside_hz, w.cone_pix, w.r_lo, w.r_hi, w.x_obs)
    return w, placed, off, S, kept, koff


def test_place_lightcone_cut_bitexact(isw, stack):
    w, placed, off, S, kept, koff = stack
    gp, goff = isw.box_place(_d(w.nodes_box), w.box_off, w.shell_box, _d(w.place))
    assert np.array_equal(goff, off)
    assert np.array_equal(gp.cpu().numpy(), placed)
    gs = isw.lightcone_intersect_shells(gp, off, w.t_box, np.zeros(w.nshell, np.int32), x_obs=w.x_obs,
                                        t_obs=w.t_obs)
    assert np.array_equal(gs.cpu().numpy(), S)
    gk, gkoff = isw.cone_cut(gs, off, w.nside_hz, _d(w.cone_pix, torch.int64), _d(w.r_lo), _d(w.r_hi),
                             x_obs=w.x_obs)
    r, _ = isw.default_context().check_status()
    assert r == isw.OK
    assert np.array_equal(gkoff.cpu().numpy(), koff)
    assert np.array_equal(gk.cpu().numpy(), kept)
    print(f"stack: {kept.shape[1]:,} of {S.shape[1]:,} placed samples kept")


def test_cone_cut_edges(isw):
    ctx = isw.default_context()
    # empty input and empty shells
    S = np.zeros((10, 0))
    gk, goff = isw.cone_cut(_d(np.zeros((10, 1)))[:, :0], [0, 0, 0], 1, _d([0, 1], torch.int64), _d([0.0, 0.0]),
                            _d([1.0, 1.0]))
    assert gk.shape[1] == 0 and np.array_equal(goff.cpu().numpy(), [0, 0, 0])
    # one shell spanning several scan blocks, keep-all and keep-none cones
    rng = np.random.default_rng(9)
    n = 5000
    S = rng.normal(size=(10, n))
    S[0:3] /= np.linalg.norm(S[0:3], axis=0) / 0.5
    base = oracle.vec2pix_ring(1, S[0:3])
    tgt = int(np.bincount(base).argmax())
    for lo, hi, expect in ((0.0, 1.0, base == tgt), (0.6, 1.0, np.zeros(n, bool))):
        gk, goff = isw.cone_cut(_d(S), [0, n], 1, _d([tgt], torch.int64), _d([lo]), _d([hi]))
        assert np.array_equal(gk.cpu().numpy(), S[:, expect])
        assert goff.cpu().numpy()[-1] == expect.sum()
    r, _ = ctx.check_status()
    assert r == isw.OK


@pytest.mark.parametrize("prec,tol", [("f32c", 1e-5), ("f64", 1e-12)])
def test_stacked_map(isw, stack, prec, tol):
    w, placed, off, S, kept, koff = stack
    theta, gk = isw.isw_map_stacked(w.nside, _d(w.nodes_box), w.box_off, w.shell_box, _d(w.place), w.t_box,
                                    w.nside_hz, _d(w.cone_pix, torch.int64), _d(w.r_lo), _d(w.r_hi), x_obs=w.x_obs,
                                    t_obs=w.t_obs, GU=w.GU, prec=prec)
    r, counts = isw.default_context().check_status()
    assert r == isw.OK
    assert gk.shape[1] == kept.shape[1]
    rng = np.random.default_rng(0)
    pix = np.unique(np.concatenate([rng.choice(w.npix, 2000, replace=False),
                                    oracle.vec2pix_ring(w.nside, kept[0:3, rng.choice(kept.shape[1], 500)])]))
    ref, _ = oracle.isw_map(w.nside, kept, pix=pix, x_obs=w.x_obs, GU=w.GU, threads=THREADS)
    got = theta.cpu().numpy()[pix]
    e = np.max(np.abs(got - ref)) / np.sqrt(np.mean(ref ** 2))
    print(f"stacked map {prec}: max|d|/rms = {e:.3e} over {pix.size} pixels; counts {counts}")
    assert e <= tol
