"""GPU parity: the CUDA library (through its C ABI) against the oracle, element by element.

Bars: pixel directions and light-cone samples bit-exact; FP64 maps max |dTheta| <= 1e-12 of
the oracle map's rms; FP32-compensated maps max |dTheta| <= 1e-5 of the rms (both relative
to rms(Theta) = sqrt(mean Theta^2) over the evaluated pixels).
"""
import os

import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

THREADS = os.cpu_count() or 4
TOL64 = 1e-12
TOL32 = 1e-5


@pytest.fixture(scope="module")
def isw():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1204_5041_gb300 as m

    m.build()
    return m


def _d(a, dtype=torch.float64):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda", dtype)


def _err(got, ref):
    rms = np.sqrt(np.mean(ref ** 2))
    return np.max(np.abs(got - ref)) / rms


def isw_num_variants():
    import paper_1204_5041_gb300 as m

    return int(m.default_context().get_param(m.PARAM_NUM_VARIANTS))


def _status_ok(isw):
    r, counts = isw.default_context().check_status()
    return r, counts


@pytest.mark.parametrize("nside", [1, 2, 3, 4, 7, 64, 1024])
def test_pix2vec_bitexact(isw, nside):
    ref, _, _ = oracle.pix2vec_ring(nside)
    got = isw.hp_pix2vec_ring(nside).cpu().numpy()
    assert np.array_equal(got.view(np.int64), ref.view(np.int64))


def test_pix2vec_list_and_range(isw):
    N = 13
    ref, _, _ = oracle.pix2vec_ring(N)
    pix = np.random.default_rng(0).integers(0, 12 * N * N, 777)
    got = isw.hp_pix2vec_ring(N, pix=_d(pix, torch.int64)).cpu().numpy()
    assert np.array_equal(got.view(np.int64), ref[:, pix].view(np.int64))
    got = isw.hp_pix2vec_ring(N, pix0=100, npix=333).cpu().numpy()
    assert np.array_equal(got.view(np.int64), ref[:, 100:433].view(np.int64))


def test_lightcone_bitexact(isw):
    w = synth.config(1, seed=4)
    P = _d(w.loop_params)
    for k in range(w.nshell):
        nodes, t_box, mode = w.shell(k)
        ref, tau_ref, st_ref = oracle.lightcone(mode, nodes, w.loop_params, t_box)
        tau = torch.empty(nodes.shape[1], dtype=torch.float64, device="cuda")
        st = torch.empty(nodes.shape[1], dtype=torch.int32, device="cuda")
        got = isw.lightcone_intersect(mode, _d(nodes), P if mode == isw.BURDEN else None, t_box, tau=tau, status=st)
        assert np.array_equal(st.cpu().numpy(), st_ref)
        assert np.array_equal(tau.cpu().numpy().view(np.int64), tau_ref.view(np.int64))
        assert np.array_equal(got.cpu().numpy().view(np.int64), ref.view(np.int64))
    assert _status_ok(isw)[0] == isw.OK


def test_lightcone_bitexact_nside4096_workload(isw):
    """All 2e6 nodes of the 1024-shell workload, shell by shell, bit-identical to the oracle."""
    w = synth.config(4, seed=1)
    ref, _, st_ref = oracle.lightcone_workload(w)
    assert np.all(st_ref == 0)
    nodes = _d(w.nodes)
    P = _d(w.loop_params)
    out = torch.empty_like(nodes)
    for k in range(w.nshell):
        a, b = int(w.shell_off[k]), int(w.shell_off[k + 1])
        if b > a:
            isw.lightcone_intersect(int(w.mode[k]), nodes[:, a:b], P, float(w.t_box[k]), out=out[:, a:b])
    assert _status_ok(isw)[0] == isw.OK
    assert np.array_equal(out.cpu().numpy().view(np.int64), ref.view(np.int64))


def test_lightcone_status_codes(isw):
    w = synth.config(0, seed=4)
    nodes = w.nodes[:, :64].copy()
    nodes[0, 3] = 1e6                      # loop id out of range
    st = torch.empty(64, dtype=torch.int32, device="cuda")
    isw.lightcone_intersect(isw.BURDEN, _d(nodes), _d(w.loop_params), status=st)
    s = st.cpu().numpy()
    assert s[3] == isw.EINVAL and np.all(np.delete(s, 3) == 0)
    r, _ = _status_ok(isw)
    assert r == isw.EINVAL
    lin = np.zeros((10, 4))
    lin[0] = 0.5
    lin[3, 1] = 1.0                         # |Xdot| = 1
    st = torch.empty(4, dtype=torch.int32, device="cuda")
    isw.lightcone_intersect(isw.LINEAR, _d(lin), t_box=0.5, status=st)
    assert list(st.cpu().numpy()) == [0, isw.EDOMAIN, 0, 0]
    assert _status_ok(isw)[0] == isw.EDOMAIN


@pytest.fixture(scope="module")
def cfg0():
    w = synth.config(0, seed=1)
    S, _, st = oracle.lightcone_workload(w)
    assert np.all(st == 0)
    ref, stats = oracle.isw_map(w.nside, S, threads=THREADS)
    return w, S, ref


@pytest.mark.parametrize("prec,tol", [("f64", TOL64), ("f32c", TOL32)])
def test_map_full_sky_nside64(isw, cfg0, prec, tol):
    w, S, ref = cfg0
    got = isw.isw_map(w.nside, _d(S), prec=prec).cpu().numpy()
    r, counts = _status_ok(isw)
    assert r == isw.OK
    e = _err(got, ref)
    print(f"{prec}: max|d|/rms = {e:.3e}, counts {counts}")
    assert e <= tol


@pytest.mark.parametrize("prec,tol", [("f64", TOL64), ("f32c", TOL32)])
def test_map_variants_and_splits(isw, cfg0, prec, tol):
    w, S, ref = cfg0
    ctx = isw.default_context()
    nvar = isw_num_variants() if prec == "f32c" else 1
    try:
        for var in range(nvar):
            if prec == "f32c":
                ctx.set_param(isw.PARAM_VARIANT, var)
            for split in (1, 3, 16):
                ctx.set_param(isw.PARAM_SPLIT, split)
                got = isw.isw_map(w.nside, _d(S), prec=prec).cpu().numpy()
                assert _err(got, ref) <= tol, (var, split)
    finally:
        ctx.set_param(isw.PARAM_VARIANT, -1)
        ctx.set_param(isw.PARAM_SPLIT, 0)
    assert _status_ok(isw)[0] == isw.OK


def test_map_deterministic(isw, cfg0):
    w, S, _ = cfg0
    Sd = _d(S)
    for prec in ("f32c", "f64"):
        a = isw.isw_map(w.nside, Sd, prec=prec).cpu().numpy()
        b = isw.isw_map(w.nside, Sd, prec=prec).cpu().numpy()
        assert np.array_equal(a.view(np.int64), b.view(np.int64))


def test_map_mixed_sign_weights(isw, cfg0):
    """Weights c = -4 GU eps dsigma / X of both signs in every tile (dsigma of random sign) and a
    negative GU: the far-field forms carry sign(c) and sqrt(|c|/2) separately, so both signs must
    reach the oracle's map, and by the linearity of Eq. (1) in GU the map at -GU is the negated
    map."""
    w, S, _ = cfg0
    S2 = S.copy()
    flip = np.random.default_rng(21).random(S.shape[1]) < 0.5
    S2[9, flip] *= -1.0
    ref, _ = oracle.isw_map(w.nside, S2, threads=THREADS)
    Sd = _d(S2)
    for prec, tol in (("f64", TOL64), ("f32c", TOL32)):
        got = isw.isw_map(w.nside, Sd, prec=prec).cpu().numpy()
        assert _status_ok(isw)[0] == isw.OK
        neg = isw.isw_map(w.nside, Sd, prec=prec, GU=-1.0).cpu().numpy()
        e, en = _err(got, ref), _err(neg, -ref)
        print(f"mixed-sign weights {prec}: max|d|/rms = {e:.3e}, at -GU {en:.3e}")
        assert e <= tol and en <= tol


def test_map_independent_of_sample_order(isw):
    """The FP32 path writes its records in a spatial (Morton) order of the samples: a permuted
    input gives the same map up to the rounding of the different summation order, and both match
    the oracle.  Also a ragged sample count (not a multiple of the sort's 1024-element blocks)."""
    w = synth.config(1, seed=4)
    S, _, st = oracle.lightcone_workload(w)
    assert np.all(st == 0)
    S = np.ascontiguousarray(S[:, :150001])
    perm = np.random.default_rng(9).permutation(S.shape[1])
    nside = 128
    a = isw.isw_map(nside, _d(S), prec="f32c").cpu().numpy()
    b = isw.isw_map(nside, _d(np.ascontiguousarray(S[:, perm])), prec="f32c").cpu().numpy()
    assert _status_ok(isw)[0] == isw.OK
    pix = np.random.default_rng(10).choice(a.size, 2000, replace=False)
    ref, _ = oracle.isw_map(nside, S, pix=pix, threads=THREADS)
    rms = np.sqrt(np.mean(ref ** 2))
    d_ab = np.max(np.abs(a - b)) / np.sqrt(np.mean(a ** 2))
    print(f"order: max|a - b|/rms = {d_ab:.2e}, errors vs oracle {_err(a[pix], ref):.2e} / {_err(b[pix], ref):.2e}")
    assert d_ab <= 2e-6
    assert np.max(np.abs(a[pix] - ref)) / rms <= TOL32 and np.max(np.abs(b[pix] - ref)) / rms <= TOL32


def test_map_pixel_list_range_accumulate_ragged(isw):
    w = synth.config(0, seed=2)
    S, _, _ = oracle.lightcone_workload(w)
    S = np.ascontiguousarray(S[:, :1000 + 37])            # not a multiple of any segment tile
    N = 32
    rng = np.random.default_rng(9)
    pix = rng.integers(0, 12 * N * N, 1001)                # ragged pixel list, with repeats
    ref, _ = oracle.isw_map(N, S, pix=pix, threads=THREADS)
    ref_r, _ = oracle.isw_map(N, S, pix=np.arange(5, 5 + 3000), threads=THREADS)
    Sd = _d(S)
    for prec, tol in (("f64", TOL64), ("f32c", TOL32)):
        got = isw.isw_map(N, Sd, pix=_d(pix, torch.int64), prec=prec).cpu().numpy()
        assert _err(got, ref) <= tol
        got = isw.isw_map(N, Sd, pix0=5, npix=3000, prec=prec).cpu().numpy()
        assert _err(got, ref_r) <= tol
        base = torch.full((1001,), 0.25, dtype=torch.float64, device="cuda")
        got = isw.isw_map(N, Sd, pix=_d(pix, torch.int64), prec=prec, accumulate=True, out=base).cpu().numpy()
        assert _err(got - 0.25, ref) <= tol
    # samples given with a leading dimension larger than n
    big = torch.zeros((10, S.shape[1] + 13), dtype=torch.float64, device="cuda")
    big[:, : S.shape[1]] = Sd
    got = isw.isw_map(N, big[:, : S.shape[1]], pix=_d(pix, torch.int64), prec="f64").cpu().numpy()
    assert _err(got, ref) <= TOL64
    assert _status_ok(isw)[0] == isw.OK


def test_map_empty_and_degenerate(isw):
    N = 4
    # no samples: zeros (or untouched when accumulating)
    out = isw.isw_map(N, torch.zeros((10, 0), dtype=torch.float64, device="cuda"), prec="f32c")
    assert torch.all(out == 0)
    # D = 0 exactly: the sample sits on the line of sight of pixel (ring 2N, j = 2N+1) of odd N
    N = 3
    p = 2 * N * (N - 1) + N * 4 * N + 2 * N
    S = np.zeros((10, 3))
    S[0, 0] = -0.5
    S[3, 0], S[8, 0], S[9, 0] = 0.3, 0.5, 1e-3
    S[1, 1], S[3, 1], S[8, 1], S[9, 1] = 0.4, 1.0, 0.5, 1e-3     # |Xdot| = 1: skipped
    S[2, 2], S[4, 2], S[6, 2], S[9, 2] = 0.7, 0.2, 0.4, 1e-3
    ref, stats = oracle.isw_map(N, S)
    for prec in ("f64", "f32c"):
        got = isw.isw_map(N, _d(S), prec=prec).cpu().numpy()
        assert np.all(np.isfinite(got))
        r, counts = isw.default_context().check_status()
        assert r == isw.EDOMAIN and counts["skipped_samples"] == 1 and counts["zero_pairs"] == 1
        assert _err(got, ref) <= (TOL64 if prec == "f64" else TOL32)


def test_invalid_arguments(isw):
    ctx = isw.default_context()
    S = torch.zeros((10, 4), dtype=torch.float64, device="cuda")
    with pytest.raises(isw.ISWError) as e:
        isw.isw_map(0, S)
    assert e.value.code == isw.EINVAL
    host = torch.zeros((10, 4), dtype=torch.float64).pin_memory()
    r = isw.lib().isw_map(ctx.handle, 4, 0, 192, None, isw._ptr(host), 4, 4, None, 1.0, 1, 0, isw._ptr(S), None)
    assert r == isw.EINVAL and "device pointer" in ctx.last_error()
    with pytest.raises(isw.ISWError):
        isw.isw_map(4, S, pix0=100, npix=1000)
    with pytest.raises(isw.ISWError):
        isw.lightcone_intersect(isw.LINEAR, S, t_box=2.0, t_obs=1.0)


@pytest.fixture(scope="module")
def cfg1():
    w = synth.config(1, seed=1)
    S, _, st = oracle.lightcone_workload(w)
    assert np.all(st == 0)
    return w, S


def _sample_pixels(w, S, k_rand=3000, k_near=1500, seed=0):
    """Random pixels plus pixels closest to random samples (the near field of the strings)."""
    rng = np.random.default_rng(seed)
    N = w.nside
    pix = list(rng.choice(12 * N * N, k_rand, replace=False))
    vec, _, _ = oracle.pix2vec_ring(N)
    sel = rng.choice(S.shape[1], k_near, replace=False)
    X = S[0:3, sel] / np.linalg.norm(S[0:3, sel], axis=0)
    # nearest pixel centre by brute force on a coarse candidate set: dot products with all pixels
    for k in range(0, k_near, 256):
        d = vec.T @ X[:, k:k + 256]
        pix += list(np.argmax(d, axis=0))
    return np.unique(np.array(pix, dtype=np.int64))


@pytest.mark.parametrize("prec,tol", [("f32c", TOL32), ("f64", TOL64)])
def test_map_nside512_200k_sampled(isw, cfg1, prec, tol):
    """Full-size workload (Nside=512, 2e5 samples) in the full-sky launch configuration,
    checked on random pixels and on pixels closest to string samples."""
    w, S = cfg1
    pix = _sample_pixels(w, S)
    ref, _ = oracle.isw_map(w.nside, S, pix=pix, threads=THREADS)
    got_full = isw.isw_map(w.nside, _d(S), prec=prec)
    r, counts = _status_ok(isw)
    assert r == isw.OK
    got = got_full.cpu().numpy()[pix]
    e = _err(got, ref)
    print(f"nside512 {prec}: max|d|/rms = {e:.3e} over {pix.size} pixels; counts {counts}")
    assert e <= tol


def test_map_near_cusp_samples(isw):
    """Samples with |Xdot| up to 1 - 1e-8 (beamed cusps): 1 + n.Xdot cancels for n near
    -Xdot/|Xdot|; the FP32 path must still meet the bar there."""
    rng = np.random.default_rng(17)
    n = 2000
    X = rng.normal(size=(3, n))
    X *= 0.5 / np.linalg.norm(X, axis=0)
    u = rng.normal(size=(3, n))
    u /= np.linalg.norm(u, axis=0)
    v = 1.0 - 10.0 ** rng.uniform(-8, -1, n)
    p = rng.normal(size=(3, n))
    p -= (p * u).sum(0) * u
    p /= np.linalg.norm(p, axis=0)
    S = np.zeros((10, n))
    S[0:3] = X
    S[3:6] = v * u
    S[6:9] = np.sqrt(1.0 - v * v) * p
    S[9] = 1e-3
    N = 64
    ref, _ = oracle.isw_map(N, S, threads=THREADS)
    Sd = _d(S)
    for prec, tol in (("f64", TOL64), ("f32c", TOL32)):
        got = isw.isw_map(N, Sd, prec=prec).cpu().numpy()
        r, counts = isw.default_context().check_status()
        assert r == isw.OK
        e = _err(got, ref)
        print(f"near-cusp {prec}: max|d|/rms = {e:.3e}, counts {counts}")
        assert e <= tol
