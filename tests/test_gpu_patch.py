"""GPU parity of isw_map_patch (Sec. IV, Fig. 3: full sky and the flat-sky approximation on a
gnomonic patch) against the oracle: FP64 <= 1e-12 and FP32c <= 1e-5 of the patch-map rms, on
rows of a 7.2-degree patch centred on the densest part of the N_side 512 string network."""
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


def _frame(axis):
    e3 = axis / np.linalg.norm(axis)
    h = np.array([0.0, 0.0, 1.0]) if abs(e3[2]) < 0.9 else np.array([1.0, 0.0, 0.0])
    e1 = np.cross(h, e3)
    e1 /= np.linalg.norm(e1)
    e2 = np.cross(e3, e1)
    return np.stack([e1, e2, e3])


@pytest.fixture(scope="module")
def patch_case():
    w = synth.config(1, seed=1)
    S, _, st = oracle.lightcone_workload(w)
    assert np.all(st == 0)
    # centre the patch on the string sample nearest to the mean direction of the long strings
    lin = S[:, w.shell_off[1]:]
    mean = lin[0:3].mean(axis=1)
    frame = _frame(mean)
    return S, frame


@pytest.mark.parametrize("approx", [0, 1])
@pytest.mark.parametrize("prec,tol", [("f64", 1e-12), ("f32c", 1e-5)])
def test_patch_vs_oracle(isw, patch_case, approx, prec, tol):
    S, frame = patch_case
    M, width = 512, np.deg2rad(7.2)
    got = isw.isw_map_patch(frame, M, width, _d(S), approx=approx, prec=prec).cpu().numpy()
    r, counts = isw.default_context().check_status()
    assert r == isw.OK
    rows = [(0, 4), (250, 262), (508, 512)]
    errs, rms = [], np.sqrt(np.mean(got ** 2))
    for j0, j1 in rows:
        ref = oracle.isw_map_patch(frame, M, width, S, approx=approx, rows=(j0, j1), threads=THREADS)[j0:j1]
        errs.append(np.max(np.abs(got[j0:j1] - ref)))
    e = max(errs) / rms
    print(f"patch {'flat' if approx else 'full'} {prec}: max|d|/rms = {e:.3e}; counts {counts}")
    assert e <= tol


def test_flat_sky_kaiser_stebbins_on_gpu(isw):
    """The flat-sky closed form of a straight moving segment, through the GPU path."""
    Lam, Z, v, nodes = 0.02, 0.5, 0.6, 40000
    h = 2 * Lam / nodes
    xi = -Lam + (np.arange(nodes) + 0.5) * h
    g = 1 / np.sqrt(1 - v * v)
    S = np.zeros((10, nodes))
    S[0] = xi * Z
    S[2] = Z
    S[4] = v
    S[6] = np.sqrt(1 - v * v)
    S[9] = g * h * Z
    M, width = 9, 0.09
    for prec, tol in (("f64", 1e-7), ("f32c", 2e-6)):
        th = isw.isw_map_patch(np.eye(3), M, width, _d(S), approx=1, prec=prec).cpu().numpy()
        pitch = width / M
        for j in range(M):
            deta = (j - 4) * pitch
            if deta == 0:
                continue
            for i in range(M):
                dxi = (i - 4) * pitch
                ref = -4 * g * v * (np.arctan((Lam - dxi) / deta) + np.arctan((Lam + dxi) / deta))
                assert abs(th[j, i] - ref) <= tol * abs(ref) + 1e-9
