"""Seeded synthetic inputs for reconstruction and distance-transform workloads.

The paper measures on high-resolution brain-tumour tissue images (Section 5,
experimental setup) that are not distributable; these generators stand in for
them with the same shapes, value ranges and structure:

* grayscale masks: uniform noise blurred by a separable Gaussian, rescaled to
  0..255 (smooth, tissue-like intensity landscapes); marker = mask - h clamped
  at 0, the classic regional-maxima marker (Section 2.1);
* binary images: random filled disks until a target foreground fraction is
  reached (object-like blobs for the distance transform, Section 2.2).

This module holds no arithmetic of the method itself; both the CPU oracle and
the CUDA path consume the identical bytes it returns.  Everything runs on the
host with numpy ``default_rng`` (PCG64) in float64, so the bytes are the same
on any machine that runs the same numpy/scipy.
"""
from __future__ import annotations

import math
import os
from concurrent.futures import ThreadPoolExecutor
from dataclasses import dataclass

import numpy as np

__all__ = [
    "blurred_noise_u8",
    "recon_inputs",
    "disks_binary",
    "Workload",
    "config_workload",
    "batched_workloads",
    "served_pool",
    "tissue_cells",
    "tissue_region",
    "apply_tissue",
]


def _threads() -> int:
    return max(1, min(16, os.cpu_count() or 1))


def _gauss_kernel(sigma: float) -> np.ndarray:
    r = int(math.ceil(4.0 * sigma))
    x = np.arange(-r, r + 1, dtype=np.float64)
    k = np.exp(-0.5 * (x / sigma) ** 2)
    return k / k.sum()


def _blur_axis(x: np.ndarray, sigma: float, axis: int) -> np.ndarray:
    """Separable Gaussian along one axis, radius ceil(4 sigma), reflect boundary.

    Strips perpendicular to ``axis`` are filtered independently in threads;
    each strip is a complete 1-D filtering problem, so the split does not
    change a single value.
    """
    from scipy.ndimage import correlate1d

    k = _gauss_kernel(sigma)
    out = np.empty_like(x)
    n_other = x.shape[1 - axis]
    nt = _threads() if x.size >= (1 << 20) else 1
    bounds = np.linspace(0, n_other, nt + 1).astype(int)

    def work(i):
        a, b = bounds[i], bounds[i + 1]
        if a == b:
            return
        if axis == 0:
            out[:, a:b] = correlate1d(x[:, a:b], k, axis=0, mode="reflect")
        else:
            out[a:b, :] = correlate1d(x[a:b, :], k, axis=1, mode="reflect")

    if nt == 1:
        work(0)
    else:
        with ThreadPoolExecutor(nt) as ex:
            list(ex.map(work, range(nt)))
    return out


def blurred_noise_u8(h: int, w: int, sigma: float, seed: int) -> np.ndarray:
    """Uniform U[0,1) noise, Gaussian blur (sigma), rescaled to 0..255 uint8.

    Rescale: round-half-even(255 (x - min) / (max - min)).
    """
    rng = np.random.default_rng(seed)
    x = rng.random((h, w), dtype=np.float64)
    x = _blur_axis(x, sigma, 1)
    x = _blur_axis(x, sigma, 0)
    lo, hi = float(x.min()), float(x.max())
    if hi <= lo:
        return np.zeros((h, w), dtype=np.uint8)
    y = np.rint(255.0 * (x - lo) / (hi - lo))
    return y.astype(np.uint8)


def recon_inputs(h: int, w: int, sigma: float, offset: int, seed: int):
    """(marker, mask) uint8: mask = blurred noise, marker = max(mask - offset, 0)."""
    mask = blurred_noise_u8(h, w, sigma, seed)
    marker = np.maximum(mask.astype(np.int16) - int(offset), 0).astype(np.uint8)
    return marker, mask


def disks_binary(h: int, w: int, rmin: int, rmax: int, coverage: float,
                 seed: int, max_disks: int | None = None):
    """Binary uint8 image (1 = inside some disk) and the number of disks drawn.

    Integer radius uniform in [rmin, rmax]; centre uniform over the image;
    overlaps allowed; a pixel is inside iff dx^2 + dy^2 <= r^2.  Disks are
    added until the foreground fraction reaches ``coverage`` (the coverage
    binds, the count is reported).
    """
    rng = np.random.default_rng(seed)
    img = np.zeros((h, w), dtype=np.uint8)
    target = int(math.ceil(coverage * h * w))
    covered = 0
    n = 0
    offs = {}
    while covered < target and (max_disks is None or n < max_disks):
        r = int(rng.integers(rmin, rmax + 1))
        cy = int(rng.integers(0, h))
        cx = int(rng.integers(0, w))
        n += 1
        if r not in offs:
            d = np.arange(-r, r + 1)
            offs[r] = (d[:, None] ** 2 + d[None, :] ** 2) <= r * r
        disk = offs[r]
        y0, y1 = max(cy - r, 0), min(cy + r + 1, h)
        x0, x1 = max(cx - r, 0), min(cx + r + 1, w)
        sub = img[y0:y1, x0:x1]
        dsub = disk[y0 - (cy - r):y1 - (cy - r), x0 - (cx - r):x1 - (cx - r)]
        new = dsub & (sub == 0)
        covered += int(new.sum())
        sub[new] = 1
    return img, n


@dataclass
class Workload:
    """One image job: op is 'recon' (marker, mask) or 'edt' (binary)."""
    op: str
    h: int
    w: int
    marker: np.ndarray | None = None
    mask: np.ndarray | None = None
    binary: np.ndarray | None = None
    note: str = ""

    @property
    def pixels(self) -> int:
        return self.h * self.w


def config_workload(name: str, rep: int = 0, size: int | None = None) -> Workload:
    """The named single-image workloads; ``size`` overrides the side length.

    recon512    : 512^2 uint8, sigma 4, offset 40 (8-connected)
    recon4096   : 4096^2 uint8, sigma 8, offset 60
    edt4096     : 4096^2 binary, disks r in [4, 40], 30% foreground
    recon16k    : 16384^2 uint8, sigma 16, offset 50
    edt16k      : 16384^2 binary, disks r in [4, 80], 25% foreground
    Seed = 1000 * index + rep with index 0 (512), 1 (4096), 2 (16384).
    """
    table = {
        "recon512": ("recon", 512, 4.0, 40, None, 0),
        "recon4096": ("recon", 4096, 8.0, 60, None, 1),
        "edt4096": ("edt", 4096, (4, 40), 0.30, None, 1),
        "recon16k": ("recon", 16384, 16.0, 50, None, 2),
        "edt16k": ("edt", 16384, (4, 80), 0.25, None, 2),
    }
    op, side, a, b, _, idx = table[name]
    if size is not None:
        side = size
    seed = 1000 * idx + rep
    if op == "recon":
        marker, mask = recon_inputs(side, side, a, b, seed)
        return Workload("recon", side, side, marker=marker, mask=mask,
                        note=f"{side}x{side} u8 sigma={a} offset={b} seed={seed}")
    img, n = disks_binary(side, side, a[0], a[1], b, seed)
    return Workload("edt", side, side, binary=img,
                    note=f"{side}x{side} disks r={a[0]}-{a[1]} cov={b} n={n} seed={seed}")


def batched_workloads(n: int = 512, seed: int = 3000, smin: int = 256,
                      smax: int = 2048) -> list[Workload]:
    """Mixed batch: sides log-uniform in [smin, smax] (independent h, w), half
    reconstruction (sigma ~ U[2,8], offset ~ U{20..80}) and half EDT (disks
    r in [4, 40], foreground ~ U[0.10, 0.40])."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n):
        h = int(round(math.exp(rng.uniform(math.log(smin), math.log(smax)))))
        w = int(round(math.exp(rng.uniform(math.log(smin), math.log(smax)))))
        s = int(rng.integers(0, 2**31 - 1))
        if i % 2 == 0:
            sigma = float(rng.uniform(2.0, 8.0))
            off = int(rng.integers(20, 81))
            marker, mask = recon_inputs(h, w, sigma, off, s)
            out.append(Workload("recon", h, w, marker=marker, mask=mask,
                                note=f"sigma={sigma:.2f} off={off}"))
        else:
            cov = float(rng.uniform(0.10, 0.40))
            img, nd = disks_binary(h, w, 4, 40, cov, s)
            out.append(Workload("edt", h, w, binary=img, note=f"cov={cov:.2f} n={nd}"))
    return out


def _crop(rng, img, h, w):
    H, W = img.shape
    y = int(rng.integers(0, H - h + 1))
    x = int(rng.integers(0, W - w + 1))
    return np.ascontiguousarray(img[y:y + h, x:x + w])


def batched_from_pool(n: int = 512, seed: int = 3000, smin: int = 256, smax: int = 2048,
                      pool_side: int = 2048) -> list[Workload]:
    """The batched mix, built fast from a small pool: half reconstruction
    (random crops of blurred-noise masks with sigma 2, 4, 6, 8, marker =
    mask - offset, offset ~ U{20..80}) and half EDT (random crops of disk
    images, r in [4, 40], at 10, 20, 30 and 40 % foreground).  Sides are
    log-uniform in [smin, smax], independently for h and w."""
    rng = np.random.default_rng(seed)
    masks = [blurred_noise_u8(pool_side, pool_side, s, seed + k) for k, s in enumerate((2.0, 4.0, 6.0, 8.0))]
    disks = [disks_binary(pool_side, pool_side, 4, 40, c, seed + 10 + k)[0]
             for k, c in enumerate((0.10, 0.20, 0.30, 0.40))]
    out = []
    for i in range(n):
        h = int(round(math.exp(rng.uniform(math.log(smin), math.log(smax)))))
        w = int(round(math.exp(rng.uniform(math.log(smin), math.log(smax)))))
        h, w = min(h, pool_side), min(w, pool_side)
        k = int(rng.integers(0, 4))
        if i % 2 == 0:
            mask = _crop(rng, masks[k], h, w)
            off = int(rng.integers(20, 81))
            marker = np.maximum(mask.astype(np.int16) - off, 0).astype(np.uint8)
            out.append(Workload("recon", h, w, marker=marker, mask=mask, note=f"pool{k} off={off}"))
        else:
            out.append(Workload("edt", h, w, binary=_crop(rng, disks[k], h, w), note=f"disks{k}"))
    return out


def served_pool(side: int = 8192, seed: int = 4000):
    """Source images for served jobs: one large recon pair and one binary image;
    a job of side s is a random s x s crop of them (crops of blurred noise and
    of disk fields keep the same local structure)."""
    marker, mask = recon_inputs(side, side, 8.0, 50, seed)
    img, _ = disks_binary(side, side, 4, 40, 0.25, seed + 1)
    return marker, mask, img


def tissue_cells(h: int, w: int, coverage: float, seed: int, cells: int = 256):
    """The low-resolution form of tissue_region: (keep, rows, cols) with
    keep a cells x cells boolean map, rows[y] / cols[x] the cell row /
    column of image row y / column x; the region is keep[rows][:, cols].

    A cells x cells field of U[0,1) noise is blurred (Gaussian, sigma = 4
    cells); pixel (y, x) belongs to cell (y*cells//h, x*cells//w).  Cells
    are taken in order of decreasing value (ties by index) until the pixels
    they cover reach coverage * h * w (coverage 1: everything)."""
    rows = (np.arange(h) * cells) // h
    cols = (np.arange(w) * cells) // w
    if coverage >= 1.0:
        return np.ones((cells, cells), dtype=bool), rows, cols
    rng = np.random.default_rng(seed)
    f = _blur_axis(_blur_axis(rng.random((cells, cells), dtype=np.float64), 4.0, 1), 4.0, 0)
    weight = np.outer(np.bincount(rows, minlength=cells), np.bincount(cols, minlength=cells)).ravel()
    order = np.argsort(-f.ravel(), kind="stable")
    k = int(np.searchsorted(np.cumsum(weight[order]), coverage * h * w))
    keep = np.zeros(cells * cells, dtype=bool)
    keep[order[:k + 1]] = True
    return keep.reshape(cells, cells), rows, cols


def tissue_region(h: int, w: int, coverage: float, seed: int, cells: int = 256) -> np.ndarray:
    """Boolean tissue map covering `coverage` of an h x w image in smooth,
    blob-shaped regions (the paper's images are partly background); see
    tissue_cells for the construction."""
    keep, rows, cols = tissue_cells(h, w, coverage, seed, cells)
    return keep[rows][:, cols]


def apply_tissue(marker: np.ndarray, mask: np.ndarray, region: np.ndarray):
    """(marker, mask) with everything outside the tissue region set to 0."""
    return marker * region.astype(marker.dtype), mask * region.astype(mask.dtype)



def grid_markers(h: int, w: int, spacing: int, seed: int) -> np.ndarray:
    """Watershed markers: the image is cut into spacing x spacing cells and
    each cell gets one marker pixel at a uniformly drawn position inside it
    (clipped to the image), labelled 1, 2, ... in row-major cell order;
    int32, 0 elsewhere."""
    rng = np.random.default_rng(seed)
    gy, gx = np.meshgrid(np.arange(0, h, spacing), np.arange(0, w, spacing), indexing="ij")
    py = np.minimum(gy + rng.integers(0, spacing, gy.shape), h - 1).ravel()
    px = np.minimum(gx + rng.integers(0, spacing, gx.shape), w - 1).ravel()
    m = np.zeros((h, w), np.int32)
    m[py, px] = np.arange(1, py.size + 1, dtype=np.int32)
    return m
