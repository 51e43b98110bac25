"""Oracle for the all-sky string ISW map -- TEST INFRASTRUCTURE ONLY.

A ctypes wrapper around ``isw_oracle.c``: a plain single-threaded FP64 C restatement of
the paper's method (Eq. 1-2, Sec. II.A-D) that shares no code with the CUDA library.
Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py``
may import this package.  Threads here only split independent pixels (or samples)
across calls of the single-threaded C routines; ctypes releases the GIL during a call.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "isw_oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle_isw.so")
_lib = None
_lock = threading.Lock()

OK, EINVAL, EDOMAIN, ENOCONV = 0, 1, 3, 4
LINEAR, BURDEN = 0, 1

_dp = ctypes.POINTER(ctypes.c_double)
_i64p = ctypes.POINTER(ctypes.c_int64)
_i32p = ctypes.POINTER(ctypes.c_int32)


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (IEEE evaluation order: -ffp-contract=off)."""
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-std=c11", "-Wall",
               "-shared", "-fPIC", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = ctypes.CDLL(build())
            L.or_sincospi_frac.argtypes = [ctypes.c_int64, ctypes.c_int64, _dp, _dp]
            L.or_sincospi_frac.restype = None
            L.or_sincos_turns.argtypes = [ctypes.c_double, _dp, _dp]
            L.or_sincos_turns.restype = None
            L.or_pix2vec_ring.argtypes = [ctypes.c_int64, ctypes.c_int64, ctypes.c_int64, _i64p,
                                          _dp, ctypes.c_int64, _i64p, _i64p]
            L.or_pix2vec_ring.restype = ctypes.c_int
            L.or_burden_eval.argtypes = [_dp, ctypes.c_int64, ctypes.c_int64, ctypes.c_double,
                                         ctypes.c_double, _dp]
            L.or_burden_eval.restype = None
            L.or_lightcone.argtypes = [ctypes.c_int, _dp, ctypes.c_int64, ctypes.c_int64, _dp,
                                       ctypes.c_int64, ctypes.c_int64, ctypes.c_double, _dp,
                                       ctypes.c_double, ctypes.c_double, ctypes.c_int, _dp, _dp,
                                       _i32p]
            L.or_lightcone.restype = ctypes.c_int
            L.or_pair_term.argtypes = [_dp, _dp, _dp, ctypes.c_double]
            L.or_pair_term.restype = ctypes.c_double
            L.or_isw_map.argtypes = [ctypes.c_int64, ctypes.c_int64, ctypes.c_int64, _i64p, _dp,
                                     ctypes.c_int64, ctypes.c_int64, _dp, ctypes.c_double, _dp,
                                     _i64p]
            L.or_isw_map.restype = ctypes.c_int
            L.or_isw_sum_dirs.argtypes = [ctypes.c_int64, _dp, ctypes.c_int64, _dp, ctypes.c_int64,
                                          ctypes.c_int64, _dp, ctypes.c_double, _dp]
            L.or_isw_sum_dirs.restype = ctypes.c_int
            L.or_isw_map_adjoint.argtypes = [ctypes.c_int64, ctypes.c_int64, ctypes.c_int64, _i64p,
                                             _dp, ctypes.c_int64, ctypes.c_int64, _dp,
                                             ctypes.c_double, _dp, _dp, ctypes.c_int64, ctypes.c_int]
            L.or_isw_map_adjoint.restype = ctypes.c_int
            L.or_lightcone_adjoint.argtypes = [ctypes.c_int, _dp, ctypes.c_int64, ctypes.c_int64, _dp,
                                               ctypes.c_int64, ctypes.c_int64, ctypes.c_double, _dp, _dp,
                                               _dp, ctypes.c_int64, ctypes.c_int, _dp, ctypes.c_int64, _dp,
                                               ctypes.c_int64]
            L.or_lightcone_adjoint.restype = ctypes.c_int
            L.or_atan2_quarter.argtypes = [ctypes.c_double, ctypes.c_double]
            L.or_atan2_quarter.restype = ctypes.c_double
            L.or_vec2pix_ring.argtypes = [ctypes.c_int64, _dp, ctypes.c_int64, ctypes.c_int64, _i64p]
            L.or_vec2pix_ring.restype = None
            L.or_box_place.argtypes = [_dp, ctypes.c_int64, _i64p, ctypes.c_int64, ctypes.c_int64, _i64p, _dp,
                                       _dp, ctypes.c_int64, _i64p]
            L.or_box_place.restype = ctypes.c_int
            L.or_cone_cut.argtypes = [_dp, ctypes.c_int64, _i64p, ctypes.c_int64, ctypes.c_int64, _i64p, _dp,
                                      _dp, _dp, _dp, ctypes.c_int64, _i64p]
            L.or_cone_cut.restype = ctypes.c_int64
            L.or_isw_map_patch.argtypes = [_dp, ctypes.c_int64, ctypes.c_double, ctypes.c_int64, ctypes.c_int64,
                                           _dp, ctypes.c_int64, ctypes.c_int64, _dp, ctypes.c_double, ctypes.c_int,
                                           _dp]
            L.or_isw_map_patch.restype = ctypes.c_int
            L.or_map_alm_cl.argtypes = [ctypes.c_int64, _dp, ctypes.c_int64, _dp, _dp]
            L.or_map_alm_cl.restype = ctypes.c_int
            L.or_map_alm_m.argtypes = [ctypes.c_int64, _dp, ctypes.c_int64, ctypes.c_int64, _dp, _dp]
            L.or_map_alm_m.restype = ctypes.c_int
            L.or_cl_from_alm.argtypes = [ctypes.c_int64, _dp, _dp]
            L.or_cl_from_alm.restype = None
            L.or_ring_info.argtypes = [ctypes.c_int64, ctypes.c_int64, _dp, _i64p, _i64p, _dp]
            L.or_ring_info.restype = None
            L.or_legendre_column.argtypes = [ctypes.c_double, ctypes.c_int64, ctypes.c_int64, _dp]
            L.or_legendre_column.restype = None
            _lib = L
    return _lib


def _d(a):
    return a.ctypes.data_as(_dp)


def _c64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def sincospi_frac(a: int, b: int):
    """(sin, cos) of pi*a/b with exact integer angle reduction."""
    s, c = ctypes.c_double(), ctypes.c_double()
    lib().or_sincospi_frac(int(a), int(b), ctypes.byref(s), ctypes.byref(c))
    return s.value, c.value


def sincos_turns(w: float):
    """(sin, cos) of 2*pi*w, reduction in turns."""
    s, c = ctypes.c_double(), ctypes.c_double()
    lib().or_sincos_turns(float(w), ctypes.byref(s), ctypes.byref(c))
    return s.value, c.value


def pix2vec_ring(nside: int, pix=None, pix0: int = 0, n: int | None = None):
    """RING pixel centres: returns (vec [3, n], ring [n], j [n]) (ring 1..4N-1, j 1-based)."""
    if pix is not None:
        pix = np.ascontiguousarray(pix, dtype=np.int64)
        n = pix.size
    elif n is None:
        n = 12 * nside * nside - pix0
    vec = np.empty((3, n))
    ring = np.empty(n, dtype=np.int64)
    jj = np.empty(n, dtype=np.int64)
    st = lib().or_pix2vec_ring(nside, pix0, n, pix.ctypes.data_as(_i64p) if pix is not None else None,
                               _d(vec), n, ring.ctypes.data_as(_i64p), jj.ctypes.data_as(_i64p))
    if st:
        raise ValueError(f"or_pix2vec_ring failed with status {st}")
    return vec, ring, jj


def burden_eval(loop_params, loop_id: int, sigma: float, t: float):
    """(X, Xdot, X') of Burden loop ``loop_id`` at (sigma, t)."""
    P = _c64(loop_params)
    out = np.empty(9)
    lib().or_burden_eval(_d(P), P.shape[1], loop_id, sigma, t, _d(out))
    return out[0:3], out[3:6], out[6:9]


def default_tol(t_obs: float = 1.0) -> float:
    """Light-cone residual tolerance: 4 ulp of t_obs."""
    return 4.0 * float(np.nextafter(t_obs, np.inf) - t_obs)


def lightcone(mode: int, nodes, loop_params=None, t_box: float = 0.0, x_obs=(0.0, 0.0, 0.0),
              t_obs: float = 1.0, tol: float | None = None, max_iter: int = 60):
    """Samples on the past light cone: returns (samples [10, n], tau [n], status [n])."""
    nodes = _c64(nodes)
    n = nodes.shape[1]
    P = _c64(loop_params if loop_params is not None else np.zeros((17, 0)))
    xo = _c64(x_obs)
    out = np.empty_like(nodes)
    tau = np.empty(n)
    status = np.empty(n, dtype=np.int32)
    lib().or_lightcone(int(mode), _d(nodes), n, n, _d(P) if P.size else None, P.shape[1],
                       max(P.shape[1], 1), float(t_box), _d(xo), float(t_obs),
                       default_tol(t_obs) if tol is None else float(tol), int(max_iter),
                       _d(out), _d(tau), status.ctypes.data_as(_i32p))
    return out, tau, status


def lightcone_workload(w):
    """Light-cone samples of every shell of a ``synth.Workload`` (concatenated)."""
    parts, taus, sts = [], [], []
    for k in range(w.nshell):
        nodes, t_box, mode = w.shell(k)
        s, tau, st = lightcone(mode, nodes, w.loop_params, t_box, w.x_obs, w.t_obs)
        parts.append(s)
        taus.append(tau)
        sts.append(st)
    return np.concatenate(parts, axis=1), np.concatenate(taus), np.concatenate(sts)


def pair_term(nvec, sample10, x_obs=(0.0, 0.0, 0.0), GU: float = 1.0) -> float:
    """One term of the discrete Eq. (1) for direction nvec and one 10-double sample."""
    return lib().or_pair_term(_d(_c64(nvec)), _d(_c64(sample10)), _d(_c64(x_obs)), float(GU))


def _split(n, parts):
    parts = max(1, min(parts, n))
    b = np.linspace(0, n, parts + 1).astype(np.int64)
    return [(int(b[i]), int(b[i + 1])) for i in range(parts) if b[i + 1] > b[i]]


def isw_map(nside: int, samples, pix=None, x_obs=(0.0, 0.0, 0.0), GU: float = 1.0,
            threads: int = 1):
    """Theta at RING pixels ``pix`` (all pixels when None); returns (theta, stats[2])."""
    samples = _c64(samples)
    n = samples.shape[1]
    if pix is None:
        pix = np.arange(12 * nside * nside, dtype=np.int64)
    pix = np.ascontiguousarray(pix, dtype=np.int64)
    theta = np.empty(pix.size)
    xo = _c64(x_obs)
    L = lib()
    stats_all = []
    errors = []

    def work(a, b):
        st = np.zeros(2, dtype=np.int64)
        sub = np.ascontiguousarray(pix[a:b])
        out = np.empty(b - a)
        r = L.or_isw_map(nside, 0, b - a, sub.ctypes.data_as(_i64p), _d(samples), n, n, _d(xo),
                         float(GU), _d(out), st.ctypes.data_as(_i64p))
        if r:
            errors.append(r)
        theta[a:b] = out
        stats_all.append(st)

    ranges = _split(pix.size, threads)
    ths = [threading.Thread(target=work, args=r) for r in ranges]
    for t in ths:
        t.start()
    for t in ths:
        t.join()
    if errors:
        raise ValueError(f"or_isw_map failed with status {errors[0]}")
    stats = np.array([sum(s[0] for s in stats_all), stats_all[0][1] if stats_all else 0])
    return theta, stats


def isw_sum_dirs(dirs, samples, x_obs=(0.0, 0.0, 0.0), GU: float = 1.0):
    """The discrete Eq. (1) at explicit unit directions ``dirs`` [3, k] (off the HEALPix grid)."""
    dirs = _c64(dirs)
    samples = _c64(samples)
    out = np.empty(dirs.shape[1])
    r = lib().or_isw_sum_dirs(dirs.shape[1], _d(dirs), dirs.shape[1], _d(samples), samples.shape[1],
                              samples.shape[1], _d(_c64(x_obs)), float(GU), _d(out))
    if r:
        raise ValueError(f"or_isw_sum_dirs failed with status {r}")
    return out


def isw_map_adjoint(nside: int, samples, g_pix, pix=None, x_obs=(0.0, 0.0, 0.0), GU: float = 1.0,
                    ngrad: int = 6, threads: int = 1):
    """dL/d(X, Xdot[, X'[, dsigma]]) per sample for a per-pixel dL/dTheta: returns grad
    [ngrad, n], ngrad in (6, 9, 10)."""
    samples = _c64(samples)
    n = samples.shape[1]
    if pix is None:
        pix = np.arange(12 * nside * nside, dtype=np.int64)
    pix = np.ascontiguousarray(pix, dtype=np.int64)
    g_pix = _c64(g_pix)
    assert g_pix.size == pix.size
    grad = np.zeros((ngrad, n))
    xo = _c64(x_obs)
    L = lib()
    errors = []

    def work(a, b):
        sub = np.ascontiguousarray(samples[:, a:b])
        out = np.empty((ngrad, b - a))
        r = L.or_isw_map_adjoint(nside, 0, pix.size, pix.ctypes.data_as(_i64p), _d(sub), b - a,
                                 b - a, _d(xo), float(GU), _d(g_pix), _d(out), b - a, int(ngrad))
        if r:
            errors.append(r)
        grad[:, a:b] = out

    ranges = _split(n, threads)
    ths = [threading.Thread(target=work, args=r) for r in ranges]
    for t in ths:
        t.start()
    for t in ths:
        t.join()
    if errors:
        raise ValueError(f"or_isw_map_adjoint failed with status {errors[0]}")
    return grad


def lightcone_adjoint(mode: int, nodes, loop_params, tau, grad_samples, t_box: float = 0.0,
                      x_obs=(0.0, 0.0, 0.0)):
    """Chain dL/d(samples) (rows X, Xdot[, X'[, dsigma]]) through the light-cone solve.

    Returns (grad_nodes [10, n], grad_loops [17, nloops] or None for LINEAR) and raises on a
    non-OK status.  LINEAR: gradients of the box-time nodes (X, Xdot, X', dsigma).  BURDEN:
    node rows 1 (sigma) and 9 (dsigma), and per-loop gradients of centre, rotation, L, psi, t0
    (rows m, n stay zero)."""
    nodes = _c64(nodes)
    n = nodes.shape[1]
    P = _c64(loop_params if loop_params is not None else np.zeros((17, 1)))
    nloops = P.shape[1]
    tau = _c64(tau)
    gs = _c64(grad_samples)
    assert gs.shape[1] == n and gs.shape[0] in (6, 9, 10)
    gn = np.zeros((10, n))
    gP = np.zeros((17, nloops)) if mode == BURDEN else None
    st = lib().or_lightcone_adjoint(int(mode), _d(nodes), n, n, _d(P), nloops, nloops, float(t_box),
                                    _d(_c64(x_obs)), _d(tau), _d(gs), n, gs.shape[0], _d(gn), n,
                                    _d(gP) if gP is not None else None, nloops)
    if st:
        raise ValueError(f"or_lightcone_adjoint failed with status {st}")
    return gn, gP


def atan2_quarter(y: float, x: float) -> float:
    """atan2(y, x) in quarter turns, in [0, 4) (own series)."""
    return lib().or_atan2_quarter(float(y), float(x))


def vec2pix_ring(nside: int, vec):
    """RING pixel of each direction (columns of vec [3, n], not necessarily unit)."""
    vec = _c64(vec)
    n = vec.shape[1]
    pix = np.empty(n, dtype=np.int64)
    lib().or_vec2pix_ring(int(nside), _d(vec), n, n, pix.ctypes.data_as(_i64p))
    return pix


def _i64(a):
    return np.ascontiguousarray(a, dtype=np.int64)


def box_place(nodes_box, box_off, shell_box, place):
    """Nodes of shell k = box shell_box[k] placed by place[k] (R row-major, T): returns
    (nodes [10, n_out], shell_off_out)."""
    nodes_box = _c64(nodes_box)
    box_off, shell_box = _i64(box_off), _i64(shell_box)
    place = _c64(place).reshape(-1, 12)
    nshell = shell_box.size
    n_out = int(sum(box_off[b + 1] - box_off[b] for b in shell_box))
    out = np.zeros((10, max(n_out, 1)))
    off = np.zeros(nshell + 1, dtype=np.int64)
    st = lib().or_box_place(_d(nodes_box), nodes_box.shape[1], box_off.ctypes.data_as(_i64p), box_off.size - 1,
                            nshell, shell_box.ctypes.data_as(_i64p), _d(place), _d(out), out.shape[1],
                            off.ctypes.data_as(_i64p))
    if st:
        raise ValueError(f"or_box_place failed with status {st}")
    return out[:, :n_out], off


def cone_cut(samples, shell_off, nside_hz, cone_pix, r_lo, r_hi, x_obs=(0.0, 0.0, 0.0)):
    """Samples of each shell inside its HEALPix cone and radius range, input order kept:
    returns (kept [10, m], shell_off_out)."""
    samples = _c64(samples)
    shell_off = _i64(shell_off)
    nshell = shell_off.size - 1
    cone_pix = _i64(cone_pix)
    r_lo, r_hi = _c64(r_lo), _c64(r_hi)
    out = np.zeros((10, max(samples.shape[1], 1)))
    off = np.zeros(nshell + 1, dtype=np.int64)
    m = lib().or_cone_cut(_d(samples), samples.shape[1], shell_off.ctypes.data_as(_i64p), nshell, int(nside_hz),
                          cone_pix.ctypes.data_as(_i64p), _d(r_lo), _d(r_hi), _d(_c64(x_obs)), _d(out),
                          out.shape[1], off.ctypes.data_as(_i64p))
    if m < 0:
        raise ValueError("or_cone_cut failed")
    return out[:, :m], off


FULLSKY, FLATSKY = 0, 1


def isw_map_patch(frame, M: int, width: float, samples, approx: int = FULLSKY, x_obs=(0.0, 0.0, 0.0),
                  GU: float = 1.0, rows=None, threads: int = 1):
    """Theta on an M x M gnomonic patch (frame rows e1, e2, e3; coordinate width ``width``),
    full sky (approx 0) or flat sky (approx 1): returns [M, M] (row j, column i), or only the
    rows in ``rows`` = (j0, j1) (other rows zero)."""
    frame = _c64(np.asarray(frame, dtype=np.float64).reshape(9))
    samples = _c64(samples)
    n = samples.shape[1]
    j0, j1 = (0, M) if rows is None else rows
    theta = np.zeros(M * M)
    L = lib()
    errors = []

    def work(a, b):
        r = L.or_isw_map_patch(_d(frame), M, float(width), j0 + a, j0 + b, _d(samples), n, n, _d(_c64(x_obs)),
                               float(GU), int(approx), _d(theta))
        if r:
            errors.append(r)

    ths = [threading.Thread(target=work, args=r) for r in _split(j1 - j0, threads)]
    for t in ths:
        t.start()
    for t in ths:
        t.join()
    if errors:
        raise ValueError(f"or_isw_map_patch failed with status {errors[0]}")
    return theta.reshape(M, M)


def map_alm_cl(nside: int, theta, lmax: int, threads: int = 1):
    """Spherical-harmonic analysis of a full-sky RING map: returns (alm complex [mmax+1, lmax+1],
    only l >= m filled; cl [lmax+1]).  With threads > 1 the values of m are split across threads
    (each m is an independent single-threaded call; the result is the same)."""
    theta = _c64(theta)
    assert theta.size == 12 * nside * nside
    alm = np.zeros(2 * (lmax + 1) * (lmax + 1))
    cl = np.zeros(lmax + 1)
    if threads <= 1:
        r = lib().or_map_alm_cl(int(nside), _d(theta), int(lmax), _d(alm), _d(cl))
        if r:
            raise ValueError(f"or_map_alm_cl failed with status {r}")
    else:
        a = alm.reshape(2, lmax + 1, lmax + 1)
        a[...] = map_alm_m(nside, theta, lmax, np.arange(lmax + 1), threads=threads)
        lib().or_cl_from_alm(int(lmax), _d(alm), _d(cl))
    a = alm.reshape(2, lmax + 1, lmax + 1)
    return a[0] + 1j * a[1], cl


def map_alm_m(nside: int, theta, lmax: int, ms, threads: int = 1):
    """a_lm of a full-sky RING map for the listed m only: float64 [2 (re, im), len(ms), lmax+1]."""
    theta = _c64(theta)
    assert theta.size == 12 * nside * nside
    ms = [int(m) for m in ms]
    out = np.zeros((2, len(ms), lmax + 1))
    L = lib()
    errors = []
    nxt = [0]
    lk = threading.Lock()

    def work():
        re = np.empty(lmax + 1)
        im = np.empty(lmax + 1)
        while True:
            with lk:
                k = nxt[0]
                nxt[0] += 1
            if k >= len(ms):
                return
            r = L.or_map_alm_m(int(nside), _d(theta), int(lmax), ms[k], _d(re), _d(im))
            if r:
                errors.append(r)
                return
            out[0, k] = re
            out[1, k] = im

    ths = [threading.Thread(target=work) for _ in range(max(1, min(threads, len(ms))))]
    for t in ths:
        t.start()
    for t in ths:
        t.join()
    if errors:
        raise ValueError(f"or_map_alm_m failed with status {errors[0]}")
    return out


def ring_info(nside: int, i: int):
    """(z, pixels, first pixel, phi_0 in turns) of RING ring i (1 .. 4N-1) as the analysis uses it."""
    z, t0 = ctypes.c_double(), ctypes.c_double()
    npx, p0 = ctypes.c_int64(), ctypes.c_int64()
    lib().or_ring_info(int(nside), int(i), ctypes.byref(z), ctypes.byref(npx), ctypes.byref(p0), ctypes.byref(t0))
    return z.value, npx.value, p0.value, t0.value


def legendre_column(z: float, m: int, lmax: int):
    """Normalised associated Legendre values lambda_lm(z), l = 0 .. lmax (zero for l < m)."""
    out = np.zeros(lmax + 1)
    lib().or_legendre_column(float(z), int(m), int(lmax), _d(out))
    return out
