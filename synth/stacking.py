"""Seeded stacking workloads: simulation boxes placed into HEALPix cones (Sec. III.B, Fig. 1).

The paper fills the comoving volume with the cones that subtend the pixels of a coarse
HEALPix grid, one simulation box per cone, each box rotated so that its depth axis points
along the cone and reused three times (three choices of depth axis).  The low-redshift stack
uses N_side^lz = 1: twelve cones around the twelve base pixels.  This module draws that setup:

* ``nbox`` boxes of random-walk long strings (LINEAR nodes in box coordinates, centred on the
  box), cube side ``box_side``;
* cone k (k = 0..11, the RING base pixels) is filled from box k // 3 with depth axis
  e_(k mod 3): the placement R_k maps e_(k mod 3) to the cone axis and T_k puts the box centre at
  distance ``d_centre`` along it; the shell's box time is t_obs - d_centre;
* the cut keeps samples of cone k between ``r_lo`` and ``r_hi``.

The cone axes are the published centres of the twelve base pixels (z = 2/3, 0, -2/3 with
phi = (2j - 1) pi/4, (j - 1) pi/2, (2j - 1) pi/4, j = 1..4), given here as a table; this module
computes no pixel assignment, light-cone solve or map sum.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

from .strings import random_walk_strings


def base_pixel_centres() -> np.ndarray:
    """[12, 3] unit vectors of the RING base pixels 0..11 (the published N_side = 1 layout)."""
    out = []
    for z, phis in ((2.0 / 3.0, [(2 * j - 1) * math.pi / 4 for j in range(1, 5)]),
                    (0.0, [(j - 1) * math.pi / 2 for j in range(1, 5)]),
                    (-2.0 / 3.0, [(2 * j - 1) * math.pi / 4 for j in range(1, 5)])):
        st = math.sqrt(1.0 - z * z)
        for phi in phis:
            out.append([st * math.cos(phi), st * math.sin(phi), z])
    return np.array(out)


def _placement(axis: np.ndarray, depth: int, d_centre: float) -> np.ndarray:
    """R (row-major) and T with R e_depth = axis, right-handed, and T = d_centre * axis."""
    helper = np.array([0.0, 0.0, 1.0]) if abs(axis[2]) < 0.9 else np.array([1.0, 0.0, 0.0])
    u = np.cross(helper, axis)
    u /= np.linalg.norm(u)
    v = np.cross(axis, u)
    cols = [None, None, None]
    cols[depth], cols[(depth + 1) % 3], cols[(depth + 2) % 3] = axis, u, v
    R = np.stack(cols, axis=1)
    return np.concatenate([R.ravel(), d_centre * axis])


@dataclasses.dataclass
class StackWorkload:
    name: str
    nside: int                 # map resolution
    nside_hz: int              # cone grid resolution
    nodes_box: np.ndarray      # [10, total box nodes], box coordinates
    box_off: np.ndarray        # [nbox + 1]
    shell_box: np.ndarray      # [nshell] box of each cone
    place: np.ndarray          # [nshell, 12]
    t_box: np.ndarray          # [nshell]
    cone_pix: np.ndarray       # [nshell]
    r_lo: np.ndarray           # [nshell]
    r_hi: np.ndarray           # [nshell]
    x_obs: np.ndarray = dataclasses.field(default_factory=lambda: np.zeros(3))
    t_obs: float = 1.0
    GU: float = 1.0

    @property
    def nshell(self) -> int:
        return int(self.shell_box.size)

    @property
    def npix(self) -> int:
        return 12 * self.nside * self.nside

    @property
    def n_placed(self) -> int:
        return int(sum(self.box_off[b + 1] - self.box_off[b] for b in self.shell_box))


def stack_config(seed: int = 0, nside: int = 512, nbox: int = 4, strings_per_box: int = 12,
                 nodes_per_string: int = 5000, box_side: float = 1.0, d_centre: float = 0.6,
                 r_lo: float = 0.3, r_hi: float = 0.9, step: float = 5e-3) -> StackWorkload:
    """Twelve cones (N_side^lz = 1) filled from ``nbox`` boxes used three times each."""
    if 3 * nbox != 12:
        raise ValueError("twelve cones, three per box: nbox must be 4")
    rng = np.random.default_rng(seed)
    boxes = [random_walk_strings(rng, [nodes_per_string] * strings_per_box, np.zeros(3), box_side, step=step,
                                 min_dist=0.0) for _ in range(nbox)]
    nodes_box = np.concatenate(boxes, axis=1)
    box_off = np.concatenate([[0], np.cumsum([b.shape[1] for b in boxes])]).astype(np.int64)
    axes = base_pixel_centres()
    shell_box = np.arange(12, dtype=np.int64) // 3
    place = np.stack([_placement(axes[k], k % 3, d_centre) for k in range(12)])
    return StackWorkload(
        name=f"stack12_nside{nside}_{nbox}boxes",
        nside=nside, nside_hz=1, nodes_box=nodes_box, box_off=box_off, shell_box=shell_box, place=place,
        t_box=np.full(12, 1.0 - d_centre), cone_pix=np.arange(12, dtype=np.int64),
        r_lo=np.full(12, r_lo), r_hi=np.full(12, r_hi))

