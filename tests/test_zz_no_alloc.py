"""The allocation-free map entry point (isw_map_f32c_noalloc), called through the C ABI.

It serves callers that may not allocate device memory (a host framework that owns all
device memory, or a loop that cannot take cudaMalloc's implicit synchronisation): its
scratch is a static device array shared by every call.  The checks: its maps equal those
of isw_map within the FP32-compensated tolerance on consecutive calls with different
inputs (so a call never reads the previous call's leftovers), and a problem too large for
the static scratch is refused.  This file sorts last so that a run stopping at the first
failure has already run every other test; it also passes alone in a fresh process.
"""
import ctypes

import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL32 = 1e-5


@pytest.fixture(scope="module")
def isw():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1204_5041_gb300 as m

    m.build()
    fn = m.lib().isw_map_f32c_noalloc
    v, i64 = ctypes.c_void_p, ctypes.c_int64
    fn.argtypes = [i64, i64, i64, v, i64, i64, v, ctypes.c_double, v, v]
    fn.restype = ctypes.c_int
    return m


def _call(isw, nside, S, pix0=0, npix=None):
    npix = 12 * nside * nside - pix0 if npix is None else npix
    out = torch.full((npix,), float("nan"), dtype=torch.float64, device="cuda")
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    r = isw.lib().isw_map_f32c_noalloc(nside, pix0, npix, ctypes.c_void_p(S.data_ptr()), S.shape[1],
                                       S.stride(0), None, 1.0, ctypes.c_void_p(out.data_ptr()), stream)
    torch.cuda.synchronize()
    return r, out


def _samples(cfg, seed, stride=1):
    w = synth.config(cfg, seed=seed)
    S, _, st = oracle.lightcone_workload(w)
    assert np.all(st == 0)
    return torch.from_numpy(np.ascontiguousarray(S[:, ::stride])).cuda()


def _err(got, ref):
    ref = ref.cpu().numpy()
    return np.max(np.abs(got.cpu().numpy() - ref)) / np.sqrt(np.mean(ref ** 2))


def test_noalloc_matches_isw_map_on_consecutive_calls(isw):
    A = _samples(0, 31)
    B = _samples(3, 32, stride=5)
    cases = [(64, A, 0, None), (64, B, 0, None), (64, A, 0, None), (128, B, 1000, 30001)]
    for nside, S, pix0, npix in cases:
        ref = isw.isw_map(nside, S, pix0=pix0, npix=npix, prec="f32c")
        r, got = _call(isw, nside, S, pix0, npix)
        assert r == isw.OK
        assert torch.isfinite(got).all()
        assert _err(got, ref) <= TOL32


def test_noalloc_rejects_oversized_problems(isw):
    S = torch.zeros((10, 8), dtype=torch.float64, device="cuda")
    r, got = _call(isw, 2048, S)          # a full Nside=2048 pixel table exceeds the static scratch
    assert r == isw.EINVAL
    assert torch.isnan(got).all()         # nothing was written
