"""The allocation-free map entry point (isw_map_f32c_noalloc), called through the C ABI.

It serves callers that may not allocate device memory (a host framework that owns all
device memory, or a loop that cannot take cudaMalloc's implicit synchronisation): its
scratch is a static device array shared by every call.  The checks: on consecutive calls
with different inputs (so a call never reads the previous call's leftovers) its maps agree
with the oracle within the FP32-compensated tolerance and equal those of isw_map (same
kernels, variant and segment chunks); the status it reads back reports a skipped sample; a
problem too large for the static scratch, or a host output pointer, is refused before
anything runs.  This file sorts last so that a run stopping at the first failure has
already run every other test; it also passes alone in a fresh process.
"""
import ctypes
import os

import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL32 = 1e-5
THREADS = os.cpu_count() or 4


@pytest.fixture(scope="module")
def isw():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1204_5041_gb300 as m

    m.build()
    fn = m.lib().isw_map_f32c_noalloc
    v, i64 = ctypes.c_void_p, ctypes.c_int64
    fn.argtypes = [i64, i64, i64, v, i64, i64, v, ctypes.c_double, v, ctypes.POINTER(ctypes.c_int32), v]
    fn.restype = ctypes.c_int
    return m


def _call(isw, nside, S, pix0=0, npix=None, out=None):
    npix = 12 * nside * nside - pix0 if npix is None else npix
    if out is None:
        out = torch.full((npix,), float("nan"), dtype=torch.float64, device="cuda")
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    status = ctypes.c_int32(-1)
    r = isw.lib().isw_map_f32c_noalloc(nside, pix0, npix, ctypes.c_void_p(S.data_ptr()), S.shape[1],
                                       S.stride(0), None, 1.0, ctypes.c_void_p(out.data_ptr()),
                                       ctypes.byref(status), stream)
    torch.cuda.synchronize()
    return r, status.value, out


def _samples(cfg, seed, stride=1):
    w = synth.config(cfg, seed=seed)
    S, _, st = oracle.lightcone_workload(w)
    assert np.all(st == 0)
    return np.ascontiguousarray(S[:, ::stride])


def test_noalloc_matches_oracle_and_isw_map_on_consecutive_calls(isw):
    A = _samples(0, 31)
    B = _samples(3, 32, stride=5)
    cases = [(64, A, 0, None), (64, B, 0, None), (64, A, 0, None), (128, B, 1000, 30001)]
    for nside, S, pix0, npix in cases:
        Sd = torch.from_numpy(S).cuda()
        r, status, got = _call(isw, nside, Sd, pix0, npix)
        assert r == isw.OK and status == isw.OK
        assert torch.isfinite(got).all()
        n_sel = 12 * nside * nside - pix0 if npix is None else npix
        ref, _ = oracle.isw_map(nside, S, pix=np.arange(pix0, pix0 + n_sel, dtype=np.int64), threads=THREADS)
        g = got.cpu().numpy()
        err = np.max(np.abs(g - ref)) / np.sqrt(np.mean(ref ** 2))
        print(f"noalloc nside={nside} n={S.shape[1]} pixels={n_sel}: max err {err:.2e} of rms")
        assert err <= TOL32
        # the same kernels, variant and segment chunks as isw_map with default settings
        same = isw.isw_map(nside, Sd, pix0=pix0, npix=npix, prec="f32c")
        assert torch.equal(got, same)


def test_noalloc_reports_skipped_samples(isw):
    S = _samples(0, 33)[:, :2048].copy()
    S[3:6, 100] = [0.6, 0.8, 0.0]            # |Xdot| = 1: the sample is skipped (EDOMAIN)
    Sd = torch.from_numpy(S).cuda()
    r, status, got = _call(isw, 32, Sd)
    assert r == isw.OK and status == isw.EDOMAIN
    assert torch.isfinite(got).all()
    # the next call clears the status
    r, status, _ = _call(isw, 32, Sd[:, :100].contiguous())
    assert r == isw.OK and status == isw.OK


def test_noalloc_rejects_before_launch(isw):
    S = torch.zeros((10, 8), dtype=torch.float64, device="cuda")
    r, status, got = _call(isw, 2048, S)      # a full Nside=2048 pixel table exceeds the static scratch
    assert r == isw.EINVAL and status == isw.OK
    assert torch.isnan(got).all()             # nothing was written
    host = torch.full((12 * 16,), float("nan"), dtype=torch.float64)
    r, _, _ = _call(isw, 4, S, out=host)      # host output pointer
    assert r == isw.EINVAL
    assert torch.isnan(host).all()
    r, _, _ = _call(isw, 4, S, pix0=1, npix=12 * 16)   # range past the last pixel
    assert r == isw.EINVAL
