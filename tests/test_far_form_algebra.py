"""The far-field forms that the GPU kernels evaluate, restated in numpy float64 and checked against
the oracle's pair term of Eq. (1)-(2) (no GPU).  The kernels rewrite the pair term
t = c [B (Xdot.d) - A (X'.d)] / [B (d.d)] for pixel-sample pairs at least d_far apart with
per-sample constants (e = 1 + Xdot.Xhat, f = X'.Xhat, sigma = sign c, s = sqrt(|c|/2)):
  FP32 far pass:  t = [(B2 - A2)(B2 + A2) + K] / (B hs),  K = s^2 (f^2 - e^2)/4,
  FP64 kernel:    t = [B2^2 - A2^2 - K'] / (B hs),        K' = s^2 (e^2 - f^2)/4,
  with B2 = s B - s e/2, A2 = s A - s f/2, hs = sigma (1 - n.Xhat);
and the FP32 adjoint forms Q = d.d as 2 - 2 n.Xhat.  A slip in these derivations (a sign, a
factor 2, a dropped constant) fails here on the CPU, for weights of both signs."""
import numpy as np
import pytest

import oracle


def _samples(rng, n):
    S = np.zeros((10, n))
    d = rng.normal(size=(3, n))
    S[0:3] = 0.4 * d / np.linalg.norm(d, axis=0) * rng.uniform(0.5, 1.5, n)
    v = rng.normal(size=(3, n))
    v /= np.linalg.norm(v, axis=0)
    speed = rng.uniform(0.1, 0.9, n)
    S[3:6] = v * speed
    t = rng.normal(size=(3, n))
    t -= np.sum(t * v, axis=0) * v                       # tangent orthogonal to the velocity
    t /= np.linalg.norm(t, axis=0)
    S[6:9] = t * np.sqrt(1.0 - speed ** 2)
    S[9] = rng.uniform(1e-4, 1e-3, n) * np.where(rng.random(n) < 0.5, -1.0, 1.0)
    return S


def _far_pairs(rng, S, per=6, d_far=0.25):
    """Unit directions n with |n - Xhat| >= d_far for each sample."""
    out = []
    for k in range(S.shape[1]):
        xh = S[0:3, k] / np.linalg.norm(S[0:3, k])
        got = 0
        while got < per:
            n = rng.normal(size=3)
            n /= np.linalg.norm(n)
            if np.linalg.norm(n - xh) >= d_far:
                out.append((k, n))
                got += 1
    return out


@pytest.mark.parametrize("GU", [1.0, -0.7])
def test_far_forms_match_the_pair_term(GU):
    rng = np.random.default_rng(31)
    S = _samples(rng, 40)
    pairs = _far_pairs(rng, S)
    worst32 = worst64 = worstQ = 0.0
    for k, n in pairs:
        ref = oracle.pair_term(n, S[:, k], GU=GU)
        X = np.linalg.norm(S[0:3, k])
        xh = S[0:3, k] / X
        xd, xp, dsig = S[3:6, k], S[6:9, k], S[9, k]
        eps = np.linalg.norm(xp) / np.sqrt(1.0 - xd @ xd)
        c = -4.0 * GU * eps * dsig / X
        e, f = 1.0 + xd @ xh, xp @ xh
        sg, s = np.sign(c), np.sqrt(abs(c) / 2.0)
        A, B = n @ xp, 1.0 + n @ xd
        hs = sg * (1.0 - n @ xh)
        B2, A2 = s * B - s * e / 2.0, s * A - s * f / 2.0
        t32 = ((B2 - A2) * (B2 + A2) + s * s * (f * f - e * e) / 4.0) / (B * hs)
        t64 = (B2 * B2 - A2 * A2 - s * s * (e * e - f * f) / 4.0) / (B * hs)
        d = n - xh
        Q = 2.0 - 2.0 * (n @ xh)
        tQ = c * (B * (xd @ d) - A * (xp @ d)) / (B * Q)
        scale = abs(c)
        worst32 = max(worst32, abs(t32 - ref) / scale)
        worst64 = max(worst64, abs(t64 - ref) / scale)
        worstQ = max(worstQ, abs(tQ - ref) / scale)
    assert worst32 < 1e-12 and worst64 < 1e-12 and worstQ < 1e-12, (worst32, worst64, worstQ)


def test_zero_weight_records_give_zero():
    """A zero-weight sample (s = 0, K = 0) gives exactly zero in both forms, for any finite B, hs."""
    rng = np.random.default_rng(5)
    for _ in range(100):
        B, hs = rng.uniform(0.01, 2.0), rng.uniform(0.03, 2.0)
        s = 0.0
        B2, A2 = s * B - s * 0.7, s * rng.normal() - s * 0.3
        assert ((B2 - A2) * (B2 + A2) + 0.0) / (B * hs) == 0.0
        assert (B2 * B2 - A2 * A2 - 0.0) / (B * hs) == 0.0
