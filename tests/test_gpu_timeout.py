"""The bounded device waits of the pair kernels, made to run out on purpose.

Every pair kernel waits for a stage of records to land in shared memory with a bounded
mbarrier wait; a wait that runs out stops its block, which first waits (with a separate,
longer limit) for its own bulk copies in flight, then records ISW_ETIMEOUT.  With
ISW_PARAM_WAIT_POLLS = 0 every such wait gives up at once, so each kernel takes that path on
its first stage: no fault, no hang, and the host reads ISW_ETIMEOUT.  Restoring the limit
gives a complete map again, equal to the oracle's."""
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


def _samples():
    w = synth.config(0, seed=5)
    S, _, st = oracle.lightcone(oracle.BURDEN, w.nodes[:, :2048], w.loop_params)
    assert np.all(st == 0)
    return S


def test_wait_limit_runs_out_then_recovers(isw):
    S = _samples()
    Sd = torch.from_numpy(S).cuda()
    nside = 16
    npix = 12 * nside * nside
    ctx = isw.Context(torch.cuda.current_device())   # own context: the setting stays here
    try:
        default = ctx.get_param(isw.PARAM_WAIT_POLLS)
        assert default == 2 ** 22
        ctx.set_param(isw.PARAM_WAIT_POLLS, 0)
        assert ctx.get_param(isw.PARAM_WAIT_POLLS) == 0
        g = torch.ones(npix, dtype=torch.float64, device="cuda")
        frame = np.eye(3)
        calls = {
            "map f32c": lambda: isw.isw_map(nside, Sd, prec="f32c", ctx=ctx),
            "map f64": lambda: isw.isw_map(nside, Sd, prec="f64", ctx=ctx),
            "adjoint f32c": lambda: isw.isw_map_adjoint(nside, Sd, g, prec="f32c", ctx=ctx),
            "adjoint f64": lambda: isw.isw_map_adjoint(nside, Sd, g, prec="f64", ctx=ctx),
            "flat patch f32c": lambda: isw.isw_map_patch(frame, 64, 0.2, Sd, approx=isw.FLATSKY, ctx=ctx),
            "full patch f64": lambda: isw.isw_map_patch(frame, 64, 0.2, Sd, approx=isw.FULLSKY, prec="f64",
                                                        ctx=ctx),
        }
        for name, fn in calls.items():
            fn()
            r, _ = ctx.check_status()
            assert r == isw.ETIMEOUT, (name, r, ctx.last_error())
            assert "ran out" in ctx.last_error()
        # the default limit again: complete maps, no status
        ctx.set_param(isw.PARAM_WAIT_POLLS, -1)
        assert ctx.get_param(isw.PARAM_WAIT_POLLS) == default
        th = isw.isw_map(nside, Sd, prec="f32c", ctx=ctx)
        r, _ = ctx.check_status()
        assert r == isw.OK, ctx.last_error()
        ref, _ = oracle.isw_map(nside, S, threads=THREADS)
        err = np.max(np.abs(th.cpu().numpy() - ref)) / np.sqrt(np.mean(ref ** 2))
        assert err <= 1e-5, err
    finally:
        ctx.close()


def test_wait_limit_argument_checks(isw):
    ctx = isw.Context(torch.cuda.current_device())
    try:
        for bad in (0.5, 2.0 ** 32, float("nan")):
            with pytest.raises(isw.ISWError):
                ctx.set_param(isw.PARAM_WAIT_POLLS, bad)
        ctx.set_param(isw.PARAM_WAIT_POLLS, 1000)
        assert ctx.get_param(isw.PARAM_WAIT_POLLS) == 1000
    finally:
        ctx.close()
