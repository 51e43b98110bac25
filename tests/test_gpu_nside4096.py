"""The largest workload at full size: Nside=4096 (201,326,592 pixels), 1024 cube shells with
2e6 light-cone samples (mixed loops and long strings, uneven shells).  One full-sky FP32-
compensated batched map (graph-captured, autotuned: the launch configuration of the benchmark's
batched measurement), checked on sampled pixels against the oracle and against the FP64 GPU
path on the same pixels; the adjoint on a 1% pixel subset checked against the oracle gradient
of 32 random samples."""
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


def test_nside4096_1024shells(isw):
    w = synth.config(4, seed=1)
    S, _, st = oracle.lightcone_workload(w)
    assert np.all(st == 0)
    rng = np.random.default_rng(4)
    pix = np.unique(rng.choice(w.npix, 600, replace=False).astype(np.int64))
    ref, _ = oracle.isw_map(w.nside, S, pix=pix, threads=THREADS)
    rms = np.sqrt(np.mean(ref ** 2))
    nodes = _d(w.nodes)
    loops = _d(w.loop_params)
    theta = isw.isw_map_batched(w.nside, nodes, w.shell_off, w.t_box, w.mode, loops, prec="f32c",
                                flags=isw.GRAPH | isw.AUTOTUNE)
    r, counts = isw.default_context().check_status()
    assert r == isw.OK
    got = theta[_d(pix, torch.int64)].cpu().numpy()
    del theta
    e32 = np.max(np.abs(got - ref)) / rms
    # FP64 GPU path on the same pixels (pixel-list mode) from the oracle's samples
    Sd = _d(S)
    got64 = isw.isw_map(w.nside, Sd, pix=_d(pix, torch.int64), prec="f64").cpu().numpy()
    e64 = np.max(np.abs(got64 - ref)) / rms
    print(f"nside4096: FP32c max|d|/rms = {e32:.3e}, FP64 = {e64:.3e} over {pix.size} pixels; counts {counts}")
    assert e32 <= 1e-5 and e64 <= 1e-12
    # adjoint on a 1% pixel subset (sorted RING indices) for a seeded per-pixel dL/dTheta
    sub = np.sort(rng.choice(w.npix, w.npix // 100, replace=False)).astype(np.int64)
    g = rng.normal(size=sub.size)
    grad = isw.isw_map_adjoint(w.nside, Sd, _d(g), pix=_d(sub, torch.int64), prec="f32c").cpu().numpy()
    nodes32 = np.sort(rng.choice(S.shape[1], 32, replace=False))
    ref_g = oracle.isw_map_adjoint(w.nside, np.ascontiguousarray(S[:, nodes32]), g, pix=sub, threads=THREADS)
    eg = max(np.max(np.abs(grad[b:b + 3, nodes32] - ref_g[b:b + 3])) / np.max(np.abs(ref_g[b:b + 3]))
             for b in (0, 3))
    print(f"nside4096 adjoint (1% pixels) FP32c vs oracle: {eg:.3e}")
    assert eg <= 1e-6
