"""GPU parity of isw_map_batched: many shells (light-cone solve per shell + one map over all
samples) against the oracle, against the sum of per-shell maps (linearity: the paper's final
map is the sum of maps sourced by subsets of cones, Sec. III.A), with CUDA-graph replay and
the autotuner."""
import os

import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

THREADS = os.cpu_count() or 4
TOL64, TOL32 = 1e-12, 1e-5


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
    return np.max(np.abs(got - ref)) / np.sqrt(np.mean(ref ** 2))


@pytest.fixture(scope="module")
def shells():
    w = synth.config(2, seed=3, scale=0.03)     # 64 cube shells, a few thousand samples
    w.nside = 32
    S, _, st = oracle.lightcone_workload(w)
    assert np.all(st == 0)
    ref, _ = oracle.isw_map(w.nside, S, threads=THREADS)
    return w, S, ref


def _batched(isw, w, prec, flags=0, GU=1.0, nodes=None, accumulate=False, out=None):
    return isw.isw_map_batched(w.nside, _d(w.nodes) if nodes is None else nodes, w.shell_off, w.t_box, w.mode,
                               _d(w.loop_params), GU=GU, prec=prec, flags=flags, accumulate=accumulate, out=out)


@pytest.mark.parametrize("prec,tol", [("f64", TOL64), ("f32c", TOL32)])
def test_batched_vs_oracle(isw, shells, prec, tol):
    w, S, ref = shells
    got = _batched(isw, w, prec).cpu().numpy()
    r, counts = isw.default_context().check_status()
    assert r == isw.OK
    assert _err(got, ref) <= tol


def test_batched_equals_sum_of_shell_maps(isw, shells):
    w, S, ref = shells
    Sd = _d(S)
    for prec, tol in (("f64", 1e-13), ("f32c", 2 * TOL32)):
        tot = torch.zeros(w.npix, dtype=torch.float64, device="cuda")
        for k in range(w.nshell):
            a, b = int(w.shell_off[k]), int(w.shell_off[k + 1])
            if b > a:
                isw.isw_map(w.nside, Sd[:, a:b], prec=prec, accumulate=True, out=tot)
        got = _batched(isw, w, prec).cpu().numpy()
        assert _err(got, tot.cpu().numpy()) <= tol


def test_batched_graph_replay_skip_and_accumulate(isw, shells):
    w, S, ref = shells
    nodes = _d(w.nodes)
    out = torch.empty(w.npix, dtype=torch.float64, device="cuda")
    a = _batched(isw, w, "f32c", flags=isw.GRAPH, nodes=nodes, out=out).cpu().numpy()   # eager + capture
    b = _batched(isw, w, "f32c", flags=isw.GRAPH, nodes=nodes, out=out).cpu().numpy()   # replay
    c = _batched(isw, w, "f32c", flags=isw.GRAPH, nodes=nodes, out=out).cpu().numpy()   # replay
    assert np.array_equal(a.view(np.int64), b.view(np.int64)) and np.array_equal(b.view(np.int64), c.view(np.int64))
    assert _err(a, ref) <= TOL32
    d = _batched(isw, w, "f32c", flags=isw.GRAPH, nodes=nodes, GU=2.0, out=out).cpu().numpy()   # new arguments
    assert _err(d, 2 * ref) <= TOL32
    # samples already on the cone
    e = isw.isw_map_batched(w.nside, _d(S), w.shell_off, w.t_box, w.mode, None, prec="f64",
                            flags=isw.SKIP_LIGHTCONE).cpu().numpy()
    assert _err(e, ref) <= TOL64
    base = torch.full((w.npix,), 0.5, dtype=torch.float64, device="cuda")
    f = _batched(isw, w, "f64", accumulate=True, out=base).cpu().numpy()
    assert _err(f - 0.5, ref) <= TOL64
    assert isw.default_context().check_status()[0] == isw.OK


def test_batched_autotune(isw, shells):
    w, S, ref = shells
    got = _batched(isw, w, "f32c", flags=isw.AUTOTUNE | isw.GRAPH).cpu().numpy()
    assert _err(got, ref) <= TOL32
    got = _batched(isw, w, "f32c", flags=isw.AUTOTUNE | isw.GRAPH).cpu().numpy()
    assert _err(got, ref) <= TOL32


def test_batched_nside1024_64shells_sampled(isw):
    """The batched workload at full size: Nside=1024, 64 cube shells (128 light-cone groups,
    ~1.45e6 samples), one graph-captured launch sequence with autotuned tiles, FP32
    compensated; checked on random pixels and pixels nearest to samples."""
    w = synth.config(2, seed=1)
    S, _, st = oracle.lightcone_workload(w)
    assert np.all(st == 0)
    rng = np.random.default_rng(3)
    pix = list(rng.choice(w.npix, 1500, replace=False))
    sel = rng.choice(S.shape[1], 500, replace=False)
    X = S[0:3, sel] / np.linalg.norm(S[0:3, sel], axis=0)
    vec, _, _ = oracle.pix2vec_ring(w.nside)
    for k in range(0, 500, 100):
        pix += list(np.argmax(vec.T @ X[:, k:k + 100], axis=0))
    pix = np.unique(np.array(pix, dtype=np.int64))
    ref, _ = oracle.isw_map(w.nside, S, pix=pix, threads=THREADS)
    got = _batched(isw, w, "f32c", flags=isw.AUTOTUNE | isw.GRAPH).cpu().numpy()[pix]
    r, counts = isw.default_context().check_status()
    assert r == isw.OK
    e = _err(got, ref)
    print(f"nside1024 batched f32c: max|d|/rms = {e:.3e} over {pix.size} pixels; counts {counts}")
    assert e <= TOL32
