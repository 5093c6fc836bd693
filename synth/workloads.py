"""The five synthetic workloads (seeded), shaped like the paper's DBIE workloads.

  small_ll    Low & Lou (n=1, m=1, l=0.3, Phi=pi/4) on a 32 x 32 boundary, points
              x, y in 8..23, z in 1..8 (16 x 16 x 8 = 2,048 points).
  ll128       the same field on 128 x 128, points x, y in 32..95, z in 1..32 (131,072 points).
  ar512       sheared quadrupolar active region, 512 x 256 boundary (seed 1306), points
              (2i, 2j, k + 1), i < 256, j < 128, k < 64 (2,097,152 points).
  batch64     64 magnetograms of side U{32..256} (seed 4), 1-4 patches each, 1k-200k points each.
  ar1024      1024 x 512, 6 patches (seed 5), traced field-line samples plus a 128^3 grid.
  table1      Low & Lou (n=3, m=1, l=0.3, Phi=4 pi/5) on 192 x 192 pixels, 32 pixels per unit,
              so that the central 64 x 64 x 64 test region is the unit box [-1, 1]^2 x [0, 2]
              (the paper's Table 1 case after Schrijver et al. 2006); points: the test region's
              pixel grid at z = 1..63 (258,048; the z = 0 layer is the boundary data itself).

Coordinates are in pixels: pixel (i, j) is centred at (i, j), pixel area 1.
This module holds none of the DBIE arithmetic.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from .active_region import Magnetogram, active_region, trace_samples
from .lowlou import LowLou, box_scale, to_box


@dataclass
class Workload:
    name: str
    mag: Magnetogram
    points: np.ndarray                # float32 (n, 3)
    truth: np.ndarray | None = None   # analytic field at the points (float64), when known
    alpha: np.ndarray | None = None   # analytic force-free factor at the points (1/pixel)
    meta: dict = field(default_factory=dict)


def lowlou_magnetogram(nx: int, ll: LowLou | None = None, scale: float | None = None) -> Magnetogram:
    """nx x nx pixels centred on the source; `scale` pixels per box unit (default nx / 2: the box
    [-1, 1]^2 spans the magnetogram)."""
    ll = ll or LowLou()
    j, i = np.mgrid[0:nx, 0:nx].astype(np.float64)
    bx, by, bz = to_box(nx, nx, i, j, np.zeros_like(i), scale)
    B = ll.field(bx, by, bz)
    f32 = lambda a: np.ascontiguousarray(a, dtype=np.float32)
    return Magnetogram(nx, nx, f32(B[..., 0]), f32(B[..., 1]), f32(B[..., 2]))


def grid_points(xs, ys, zs) -> np.ndarray:
    Z, Y, X = np.meshgrid(np.asarray(zs, np.float64), np.asarray(ys, np.float64),
                          np.asarray(xs, np.float64), indexing="ij")
    return np.stack([X.ravel(), Y.ravel(), Z.ravel()], axis=1).astype(np.float32)


def _ll_workload(name, nx, lo, hi, zmax, with_truth=True):
    ll = LowLou(1, 1, 0.3, np.pi / 4)
    mag = lowlou_magnetogram(nx, ll)
    pts = grid_points(range(lo, hi + 1), range(lo, hi + 1), range(1, zmax + 1))
    truth = alpha = None
    if with_truth:
        bx, by, bz = to_box(nx, nx, pts[:, 0], pts[:, 1], pts[:, 2])
        truth = ll.field(bx, by, bz)
        alpha = ll.alpha(bx, by, bz) / box_scale(nx)
    return Workload(name, mag, pts, truth, alpha, dict(field="lowlou n=1 m=1 l=0.3 Phi=pi/4"))


def ll129_nodes(with_truth: bool = True) -> Workload:
    """The ll128 field on the 129 x 129 node grid at the same 64 px per box unit (nodes at the
    box edges, as nine-node elements need), with the ll128 points at the same box positions."""
    ll = LowLou(1, 1, 0.3, np.pi / 4)
    mag = lowlou_magnetogram(129, ll, scale=64.0)
    pts = grid_points(np.arange(32, 96) + 0.5, np.arange(32, 96) + 0.5, range(1, 33))
    truth = None
    if with_truth:
        bx, by, bz = to_box(129, 129, pts[:, 0], pts[:, 1], pts[:, 2], 64.0)
        truth = ll.field(bx, by, bz)
    return Workload("ll129_nodes", mag, pts, truth, None,
                    dict(field="lowlou n=1 m=1 l=0.3 Phi=pi/4", scale=64.0))


def small_ll() -> Workload:
    return _ll_workload("small_ll", 32, 8, 23, 8)


def ll128(with_truth: bool = True) -> Workload:
    return _ll_workload("ll128", 128, 32, 95, 32, with_truth)


def ar512(points: bool = True) -> Workload:
    mag = active_region(512, 256, 4, seed=1306)
    pts = grid_points(np.arange(256) * 2, np.arange(128) * 2, np.arange(64) + 1) if points else \
        np.zeros((0, 3), np.float32)
    return Workload("ar512", mag, pts, meta=dict(seed=1306))


def ar512_backward_subvolume(w: Workload) -> np.ndarray:
    """Indices of the 32^3 sub-grid i in [112, 144), j in [48, 80), k in [0, 32) of ar512."""
    k, j, i = np.meshgrid(np.arange(0, 32), np.arange(48, 80), np.arange(112, 144), indexing="ij")
    return (k * 128 * 256 + j * 256 + i).ravel()


def batch64(seed: int = 4, nprob: int = 64, max_points: int = 200_000):
    rng = np.random.default_rng(seed)
    out = []
    for p in range(nprob):
        n = int(rng.integers(32, 257))
        npatch = int(rng.integers(1, 5))
        mag = active_region(n, n, npatch, seed=int(rng.integers(1 << 31)), peak=(500.0, 2000.0),
                            sigma=(3.0, max(3.0, n / 8.0)))
        ne = int(rng.integers(1000, max_points + 1))
        pts = np.stack([rng.uniform(0, n - 1, ne), rng.uniform(0, n - 1, ne),
                        rng.uniform(1, 64, ne)], axis=1).astype(np.float32)
        out.append(Workload(f"batch64[{p}]", mag, pts, meta=dict(side=n, patches=npatch)))
    return out


def table1(nx: int = 192, scale: float = 32.0, nz: int = 63) -> Workload:
    """The paper's Table 1 case (Low & Lou n=3, m=1, l=0.3, Phi=4 pi/5).  nx = 193 gives the same
    field on the odd node grid that nine-node elements need (nodes at the same spacing, the
    source at the centre node); points keep their physical positions."""
    ll = LowLou(3, 1, 0.3, 4 * np.pi / 5)
    mag = lowlou_magnetogram(nx, ll, scale)
    # the central 64 x 64 pixels of the 192 grid, at the same box positions for any nx
    c192 = (192 - 1) / 2.0
    xs = np.arange(64, 128) - c192 + (nx - 1) / 2.0
    pts = grid_points(xs, xs, range(1, nz + 1))
    bx, by, bz = to_box(nx, nx, pts[:, 0], pts[:, 1], pts[:, 2], scale)
    truth = ll.field(bx, by, bz)
    # the z = 0 layer of the test region: its boundary data and the analytic field there
    bottom = grid_points(xs, xs, [0.0])
    b0x, b0y, b0z = to_box(nx, nx, bottom[:, 0], bottom[:, 1], bottom[:, 2], scale)
    return Workload("table1", mag, pts, truth, None,
                    dict(field="lowlou n=3 m=1 l=0.3 Phi=4pi/5", scale=scale,
                         bottom=bottom, bottom_truth=ll.field(b0x, b0y, b0z)))


def ar1024(nsamples: int = 4_194_304, grid: bool = True, seed: int = 5) -> Workload:
    mag = active_region(1024, 512, 6, seed=seed)
    parts = []
    if nsamples:
        parts.append(trace_samples(mag, nsamples, seed=seed + 1))
    if grid:
        parts.append(grid_points(np.arange(128) * 8, np.arange(128) * 4, np.arange(128) + 1))
    pts = np.concatenate(parts) if parts else np.zeros((0, 3), np.float32)
    return Workload("ar1024", mag, pts, meta=dict(seed=seed, samples=nsamples))
