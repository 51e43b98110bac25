"""Seeded synthetic Nambu-Goto string networks standing in for the paper's simulations.

The paper's light-cone data (a thousand Bennett-Bouchet runs, Sec. II.B-C) is not
available, so every workload here is drawn from a PCG64 stream:

* Burden loops (analytic Nambu-Goto solutions in flat space): a'(u) = (cos, sin, 0)
  at wavenumber m, b'(v) in a plane tilted by psi at wavenumber n, a random 3D
  rotation, invariant length L log-uniform in [0.01, 0.1] horizon, a random time
  offset t0.  The loop is stored as 17 parameters; its nodes carry (loop id, sigma).
* Long strings: random-walk polylines with isotropic steps, node velocities
  orthogonal to the local tangent with |Xdot| ~ U[0.3, 0.85], X' along the tangent
  with |Xdot|^2 + |X'|^2 = 1 (so eps = 1) and d(sigma) chosen so that the length
  element |X'| d(sigma) is the node's share of the polyline (half of each adjacent
  step; the end nodes get half a step); the weight eps d(sigma) is then gamma times
  that share, the string's energy element.

Units: flat conformal coordinates in horizon units; the observer sits at x_obs = 0
at conformal time t_obs = 1.

Node layout (both modes): float64 array ``[10, n]``.
  LINEAR: rows 0-2 X, 3-5 Xdot, 6-8 X' (all at the shell's box time), 9 d(sigma).
  BURDEN: row 0 loop id (exact integer), row 1 sigma, rows 2-8 zero, 9 d(sigma).
Loop parameters: float64 ``[17, nloops]``: centre (3), rotation R (9, row-major),
L, m, n, psi, t0.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

NROWS = 10
LOOP_PARAMS = 17
MODE_LINEAR = 0
MODE_BURDEN = 1

NODES_PER_LOOP = 512
STRING_STEP = 1e-3
MIN_OBSERVER_DISTANCE = 0.02


@dataclasses.dataclass
class Workload:
    """One synthetic light-cone workload: nodes grouped in shells plus sky resolution."""

    name: str
    nside: int
    nodes: np.ndarray          # float64 [10, n]
    loop_params: np.ndarray    # float64 [17, nloops]
    shell_off: np.ndarray      # int64 [nshell + 1]
    t_box: np.ndarray          # float64 [nshell]
    mode: np.ndarray           # int32 [nshell]
    x_obs: np.ndarray = dataclasses.field(default_factory=lambda: np.zeros(3))
    t_obs: float = 1.0
    GU: float = 1.0

    @property
    def n(self) -> int:
        return int(self.nodes.shape[1])

    @property
    def nshell(self) -> int:
        return int(len(self.t_box))

    @property
    def npix(self) -> int:
        return 12 * self.nside * self.nside

    def shell(self, k: int):
        """(nodes [10, m], t_box, mode) of shell k (a view into ``nodes``)."""
        a, b = int(self.shell_off[k]), int(self.shell_off[k + 1])
        return self.nodes[:, a:b], float(self.t_box[k]), int(self.mode[k])


def _unit_vectors(rng: np.random.Generator, k: int) -> np.ndarray:
    v = rng.standard_normal((k, 3))
    return v / np.linalg.norm(v, axis=1, keepdims=True)


def _random_rotations(rng: np.random.Generator, k: int) -> np.ndarray:
    """Uniform random rotations from normalised quaternions (4 iid normals)."""
    q = rng.standard_normal((k, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    w, x, y, z = q.T
    R = np.empty((k, 3, 3))
    R[:, 0, 0] = 1 - 2 * (y * y + z * z)
    R[:, 0, 1] = 2 * (x * y - z * w)
    R[:, 0, 2] = 2 * (x * z + y * w)
    R[:, 1, 0] = 2 * (x * y + z * w)
    R[:, 1, 1] = 1 - 2 * (x * x + z * z)
    R[:, 1, 2] = 2 * (y * z - x * w)
    R[:, 2, 0] = 2 * (x * z - y * w)
    R[:, 2, 1] = 2 * (y * z + x * w)
    R[:, 2, 2] = 1 - 2 * (x * x + y * y)
    return R


def burden_loop_params(rng: np.random.Generator, centres: np.ndarray) -> np.ndarray:
    """Draw Burden-loop parameters for loops centred at ``centres`` ([k, 3]).

    m, n ~ U{1..5}; psi ~ U[0, pi); rotation uniform; L log-uniform in [0.01, 0.1];
    t0 ~ U[0, L).  Returns float64 [17, k].
    """
    k = centres.shape[0]
    P = np.empty((LOOP_PARAMS, k))
    P[0:3] = centres.T
    P[3:12] = _random_rotations(rng, k).reshape(k, 9).T
    L = 10.0 ** rng.uniform(-2.0, -1.0, k)
    P[12] = L
    P[13] = rng.integers(1, 6, k)
    P[14] = rng.integers(1, 6, k)
    P[15] = rng.uniform(0.0, math.pi, k)
    P[16] = rng.uniform(0.0, 1.0, k) * L
    return P


def burden_nodes(loop_params: np.ndarray, nodes_per_loop: int = NODES_PER_LOOP,
                 first_loop: int = 0, nloops: int | None = None) -> np.ndarray:
    """BURDEN-mode nodes: uniform sigma_k = k L / N, d(sigma) = L / N (periodic trapezoid)."""
    if nloops is None:
        nloops = loop_params.shape[1] - first_loop
    ids = np.repeat(np.arange(first_loop, first_loop + nloops), nodes_per_loop)
    L = loop_params[12, ids]
    k = np.tile(np.arange(nodes_per_loop), nloops)
    nodes = np.zeros((NROWS, ids.size))
    nodes[0] = ids
    nodes[1] = k * (L / nodes_per_loop)
    nodes[9] = L / nodes_per_loop
    return nodes


def random_walk_strings(rng: np.random.Generator, counts, cube_centre, cube_side: float,
                        step: float = STRING_STEP, vmin: float = 0.3, vmax: float = 0.85,
                        min_dist: float = MIN_OBSERVER_DISTANCE) -> np.ndarray:
    """LINEAR-mode nodes of random-walk long strings (one polyline per entry of ``counts``).

    Each string starts uniformly in the cube and takes isotropic steps of length
    ``step``.  Strings that come closer than ``min_dist`` to the observer are redrawn.
    """
    out = []
    cube_centre = np.asarray(cube_centre, dtype=np.float64)
    for cnt in counts:
        cnt = int(cnt)
        if cnt < 2:
            raise ValueError("a long string needs at least 2 nodes")
        while True:
            start = cube_centre + rng.uniform(-0.5, 0.5, 3) * cube_side
            steps = _unit_vectors(rng, cnt - 1) * step
            X = np.vstack([start, start + np.cumsum(steps, axis=0)])
            if np.min(np.linalg.norm(X, axis=1)) >= min_dist:
                break
        seg = np.diff(X, axis=0)
        seglen = np.linalg.norm(seg, axis=1)
        tang = np.empty_like(X)
        tang[1:-1] = X[2:] - X[:-2]
        tang[0] = seg[0]
        tang[-1] = seg[-1]
        tang /= np.linalg.norm(tang, axis=1, keepdims=True)
        # orthonormal frame (e1, e2) perpendicular to the tangent
        helper = np.where(np.abs(tang[:, :1]) < 0.9, np.array([[1.0, 0, 0]]), np.array([[0, 1.0, 0]]))
        e1 = np.cross(tang, helper)
        e1 /= np.linalg.norm(e1, axis=1, keepdims=True)
        e2 = np.cross(tang, e1)
        az = rng.uniform(0.0, 2 * math.pi, cnt)
        v = rng.uniform(vmin, vmax, cnt)
        Xdot = v[:, None] * (np.cos(az)[:, None] * e1 + np.sin(az)[:, None] * e2)
        gam_inv = np.sqrt(1.0 - v * v)
        Xp = gam_inv[:, None] * tang
        share = np.zeros(cnt)
        share[:-1] += 0.5 * seglen
        share[1:] += 0.5 * seglen
        dsig = share / gam_inv
        nodes = np.empty((NROWS, cnt))
        nodes[0:3] = X.T
        nodes[3:6] = Xdot.T
        nodes[6:9] = Xp.T
        nodes[9] = dsig
        out.append(nodes)
    if not out:
        return np.zeros((NROWS, 0))
    return np.concatenate(out, axis=1)


def _sky_loop_centres(rng, k, dmin, dmax):
    return _unit_vectors(rng, k) * rng.uniform(dmin, dmax, k)[:, None]


def _cube_loop_centres(rng, k, centre, side, margin=0.04):
    c = centre[None, :] + rng.uniform(-0.5, 0.5, (k, 3)) * side
    bad = np.linalg.norm(c, axis=1) < margin
    while np.any(bad):
        c[bad] = centre[None, :] + rng.uniform(-0.5, 0.5, (int(bad.sum()), 3)) * side
        bad = np.linalg.norm(c, axis=1) < margin
    return c


class _Builder:
    def __init__(self):
        self.nodes, self.loops, self.t_box, self.mode = [], [], [], []
        self.nloops = 0

    def add_loops(self, P, t_box=0.0):
        k = P.shape[1]
        self.loops.append(P)
        self.nodes.append(burden_nodes(np.concatenate(self.loops, axis=1), NODES_PER_LOOP,
                                       self.nloops, k))
        self.nloops += k
        self.t_box.append(t_box)
        self.mode.append(MODE_BURDEN)

    def add_linear(self, nodes, t_box):
        self.nodes.append(nodes)
        self.t_box.append(t_box)
        self.mode.append(MODE_LINEAR)

    def build(self, name, nside):
        sizes = [a.shape[1] for a in self.nodes]
        off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
        loops = np.concatenate(self.loops, axis=1) if self.loops else np.zeros((LOOP_PARAMS, 0))
        return Workload(name=name, nside=nside,
                        nodes=np.ascontiguousarray(np.concatenate(self.nodes, axis=1)),
                        loop_params=np.ascontiguousarray(loops),
                        shell_off=off, t_box=np.asarray(self.t_box, dtype=np.float64),
                        mode=np.asarray(self.mode, dtype=np.int32))


def _shell_geometry(rng, dmin=0.05, dmax=0.95):
    d = rng.uniform(dmin, dmax)
    return _unit_vectors(rng, 1)[0] * d, d


def _add_mixed_shell(b: _Builder, rng, nseg: int, centre, side: float, t_box: float,
                     string_nodes: int = 2500):
    """A cube shell with ~60% of its nodes in Burden loops and the rest in long strings."""
    nloops = int(round(0.6 * nseg / NODES_PER_LOOP))
    nstr_nodes = max(nseg - nloops * NODES_PER_LOOP, 0)
    if nloops > 0:
        b.add_loops(burden_loop_params(rng, _cube_loop_centres(rng, nloops, centre, side)))
    if nstr_nodes >= 2:
        ns = max(1, int(round(nstr_nodes / string_nodes)))
        counts = np.full(ns, nstr_nodes // ns)
        counts[: nstr_nodes - counts.sum()] += 1
        b.add_linear(random_walk_strings(rng, counts, centre, side), t_box)


def config(index: int, seed: int = 0, scale: float = 1.0) -> Workload:
    """The five benchmark workloads (sizes as described in the module docstring).

    0: Nside=64, 20 Burden loops x 512 nodes, loops at distance 0.3-0.5, directions uniform.
    1: Nside=512, 234 loops x 512 (as 0) + 8 random-walk strings (80,192 nodes) in a cube of
       side 0.2 at distance 0.4, box time 0.6 (LINEAR).
    2: Nside=1024, 64 cube shells (side 0.1, centre distance U[0.05, 0.95], box time 1 - d),
       node counts log-uniform in [1e3, 1e5], 60% loops / 40% strings.
    3: Nside=256, 98 Burden loops x 512 as in 0 (adjoint workload).
    4: Nside=4096, 1024 shells as in 2 with counts rescaled to a total of 2e6.

    ``scale`` < 1 shrinks the node counts of workloads 2 and 4 (test sizes only).
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    b = _Builder()
    if index == 0:
        b.add_loops(burden_loop_params(rng, _sky_loop_centres(rng, 20, 0.3, 0.5)))
        return b.build("nside64_20loops_10240seg", 64)
    if index == 1:
        b.add_loops(burden_loop_params(rng, _sky_loop_centres(rng, 234, 0.3, 0.5)))
        centre = _unit_vectors(rng, 1)[0] * 0.4
        counts = np.full(8, 80192 // 8)
        b.add_linear(random_walk_strings(rng, counts, centre, 0.2), 1.0 - 0.4)
        return b.build("nside512_200k_seg", 512)
    if index == 3:
        b.add_loops(burden_loop_params(rng, _sky_loop_centres(rng, 98, 0.3, 0.5)))
        return b.build("nside256_98loops_50176seg", 256)
    if index in (2, 4):
        nshell = 64 if index == 2 else 1024
        counts = 10.0 ** rng.uniform(3.0, 5.0, nshell)
        if index == 4:
            counts *= 2e6 / counts.sum()
        counts = np.maximum((counts * scale).astype(np.int64), 2)
        for k in range(nshell):
            centre, d = _shell_geometry(rng)
            _add_mixed_shell(b, rng, int(counts[k]), centre, 0.1, 1.0 - d)
        name = ("nside1024_64shells" if index == 2 else "nside4096_1024shells_2e6seg")
        return b.build(name, 1024 if index == 2 else 4096)
    raise ValueError(f"unknown workload {index}")


CONFIG_NAMES = {0: "nside64_20loops_10240seg", 1: "nside512_200k_seg", 2: "nside1024_64shells",
                3: "nside256_98loops_50176seg", 4: "nside4096_1024shells_2e6seg"}
