"""GPU parity of isw_map_cl (Fig. 4: the angular power spectrum of the map) against the oracle:
a_lm within 1e-10 of max|a_lm| and C_l within 1e-9 relative, on a string map and a random map."""
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


@pytest.mark.parametrize("N,lmax", [(1, 3), (4, 16), (16, 47), (128, 383)])
def test_cl_vs_oracle(isw, N, lmax):
    if N == 128:
        w = synth.config(0, seed=1)
        S, _, st = oracle.lightcone_workload(w)
        assert np.all(st == 0)
        theta = isw.isw_map(N, _d(S), prec="f64").cpu().numpy()
    else:
        theta = np.random.default_rng(N).normal(size=12 * N * N)
    ref_a, ref_cl = oracle.map_alm_cl(N, theta, lmax)
    alm, cl = isw.isw_map_cl(N, _d(theta), lmax, with_alm=True)
    alm, cl = alm.cpu().numpy(), cl.cpu().numpy()
    ea = np.max(np.abs(alm - ref_a)) / np.max(np.abs(ref_a))
    ec = np.max(np.abs(cl - ref_cl) / (np.abs(ref_cl) + 1e-12 * ref_cl.max()))
    print(f"cl N={N} lmax={lmax}: alm err {ea:.3e}, cl err {ec:.3e}")
    assert ea <= 1e-10 and ec <= 1e-9


def test_cl_argument_errors(isw):
    with pytest.raises(isw.ISWError):
        isw.isw_map_cl(4, _d(np.zeros(12 * 16)), 17)          # lmax above 4 nside
