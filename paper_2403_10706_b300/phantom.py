"""Seeded synthetic reversed-gradient-polarity image pairs.

These stand in for the Human Connectome Project 3T/7T volumes and the simulated volumes the
paper measures on (Sec. 3.1, Table 1), which are not available here.  The module holds no
arithmetic of the correction method itself: it draws a phantom, a field map b* and the two
distorted images, and is imported by the tests (for both the CUDA path and the oracle) and by
the benchmark.

Forward model: the paper simulates its distorted pairs with push-forward matrices built from the
field map (Sec. 3.1): the intensity at x is pushed to x + b(x) (+v) and to x - b(x) (-v).  Here
that push-forward is applied per PE column as an exact mass redistribution: the mass of true
cell j, which spans the node interval [j - 1/2, j + 1/2] in cell-centred index coordinates, is
spread uniformly over the mapped interval [j - 1/2 +- b_j, j + 1/2 +- b_{j+1}] and collected by
the distorted cells.  b is stored on the e_p-staggered grid (m + 1 nodes along PE) in PE-voxel
units, as the library expects.
"""
from __future__ import annotations

import dataclasses

import numpy as np
from scipy import ndimage

# workload recipes: shapes, spacings and PE axes of the paper's 3T and 7T data (Table 1),
# as adapted by the benchmark configurations (3T 144x168x111 @1.25 mm with PE along the 168
# axis; 7T-shaped 130x130x85 @1.05 mm with PE along axis 0).
RECIPES = {
    "tiny": dict(dims=(32, 32, 16), spacing=(1.0, 1.0, 1.0), pe_dim=1, seed=1001,
                 n_ellipsoids=3, n_blobs=0, semi_axes=(3.0, 10.0), smooth=0.0,
                 n_gauss=3, sigma=(4.0, 4.0), bmax=3.0, noise=0.01),
    "3t": dict(dims=(144, 168, 111), spacing=(1.25, 1.25, 1.25), pe_dim=1, seed=1002,
               n_ellipsoids=12, n_blobs=8, semi_axes=None, smooth=1.0,
               n_gauss=20, sigma=(5.0, 15.0), bmax=8.0, noise=0.02),
    "7t": dict(dims=(130, 130, 85), spacing=(1.05, 1.05, 1.05), pe_dim=0, seed=1003,
               n_ellipsoids=12, n_blobs=8, semi_axes=None, smooth=1.0,
               n_gauss=20, sigma=(5.0, 15.0), bmax=10.0, noise=0.02),
    "small": dict(dims=(96, 96, 60), spacing=(1.5, 1.5, 1.5), pe_dim=1, seed=1004,
                  n_ellipsoids=12, n_blobs=8, semi_axes=None, smooth=1.0,
                  n_gauss=20, sigma=(5.0, 15.0), bmax=6.0, noise=0.02),
    # the size of the paper's 7T acquisitions (an extra timing row; the 7T recipe above keeps the
    # smaller shape of the parity and adjoint cases)
    "7t_paper": dict(dims=(200, 200, 132), spacing=(1.05, 1.05, 1.05), pe_dim=0, seed=1005,
                     n_ellipsoids=12, n_blobs=8, semi_axes=None, smooth=1.0,
                     n_gauss=20, sigma=(10.0, 20.0), bmax=8.0, noise=0.02),
}

# the generator redraws b* (next seed) until its largest PE difference is at most this
MAX_FIELD_SLOPE = 0.5


@dataclasses.dataclass
class Pair:
    """One synthetic acquisition pair."""
    Ip: np.ndarray          # +v image, float32, dims
    Im: np.ndarray          # -v image, float32, dims
    I_true: np.ndarray      # undistorted image, float32, dims
    b_true: np.ndarray      # field map b*, float32, field dims (PE voxel units)
    spacing: tuple
    pe_dim: int
    seed: int               # seed actually used for b* after redraws

    @property
    def dims(self):
        return tuple(self.Ip.shape)


def field_dims(dims, pe_dim):
    fd = list(dims)
    fd[pe_dim] += 1
    return tuple(fd)


def _grid(dims, pe_dim, staggered):
    """Voxel-index coordinates; along PE the staggered field sits on cell edges (k - 1/2)."""
    axes = []
    for ax, n in enumerate(dims):
        if staggered and ax == pe_dim:
            axes.append(np.arange(n + 1, dtype=np.float64) - 0.5)
        else:
            axes.append(np.arange(n, dtype=np.float64))
    return axes


def _ellipsoid_phantom(rng, dims, n_ell, n_blobs, semi_axes, smooth):
    x = np.meshgrid(*[np.arange(n, dtype=np.float64) for n in dims], indexing="ij")
    img = np.zeros(dims, dtype=np.float64)
    dims_a = np.asarray(dims, dtype=np.float64)
    if semi_axes is None:
        # a head-sized ellipsoid that holds the interior structures
        c = (dims_a - 1) / 2
        ax = 0.42 * dims_a
        inside = sum(((x[i] - c[i]) / ax[i]) ** 2 for i in range(3)) <= 1.0
        img[inside] = rng.uniform(0.3, 1.0)
    for _ in range(n_ell):
        c = dims_a * rng.uniform(0.2, 0.8, size=3)
        if semi_axes is None:
            ax = dims_a * rng.uniform(0.06, 0.2, size=3)
        else:
            ax = rng.uniform(semi_axes[0], semi_axes[1], size=3)
        inside = sum(((x[i] - c[i]) / ax[i]) ** 2 for i in range(3)) <= 1.0
        img[inside] = rng.uniform(0.3, 1.0)
    for _ in range(n_blobs):
        c = dims_a * rng.uniform(0.25, 0.75, size=3)
        s = dims_a * rng.uniform(0.03, 0.08, size=3)
        img += rng.uniform(0.3, 1.0) * 0.5 * np.exp(
            -0.5 * sum(((x[i] - c[i]) / s[i]) ** 2 for i in range(3)))
    if smooth > 0:
        img = ndimage.gaussian_filter(img, smooth, mode="nearest")
    return img


def _gaussian_field(rng, dims, pe_dim, n_gauss, sigma, bmax):
    fd = field_dims(dims, pe_dim)
    coords = _grid(dims, pe_dim, staggered=True)
    dims_a = np.asarray(dims, dtype=np.float64)
    b = np.zeros(fd, dtype=np.float64)
    for _ in range(n_gauss):
        c = dims_a * rng.uniform(0.2, 0.8, size=3)
        s = rng.uniform(sigma[0], sigma[1])
        amp = rng.choice([-1.0, 1.0]) * rng.uniform(0.5, 1.0)
        # separable evaluation of exp(-|x - c|^2 / (2 s^2))
        f = [np.exp(-0.5 * ((coords[i] - c[i]) / s) ** 2) for i in range(3)]
        b += amp * f[0][:, None, None] * f[1][None, :, None] * f[2][None, None, :]
    peak = np.abs(b).max()
    return b * (bmax / peak) if peak > 0 else b


def push_forward(I, b, pe_dim, sign):
    """Distorted image for phase-encoding direction sign*v: each true cell's mass is moved from
    [j - 1/2, j + 1/2] to [j - 1/2 + sign*b_j, j + 1/2 + sign*b_{j+1}] and collected by the
    distorted cells [i - 1/2, i + 1/2] (exact per-column mass redistribution; needs
    |b_{j+1} - b_j| < 1 so that the mapped edges stay increasing)."""
    I = np.moveaxis(np.asarray(I, dtype=np.float64), pe_dim, -1)
    bb = np.moveaxis(np.asarray(b, dtype=np.float64), pe_dim, -1)
    shape, m = I.shape, I.shape[-1]
    cols = I.reshape(-1, m)
    ncols = cols.shape[0]
    edges = np.arange(m + 1, dtype=np.float64) - 0.5
    mapped = edges[None, :] + sign * bb.reshape(ncols, m + 1)          # images of the edges
    mass = np.zeros((ncols, m + 1))
    mass[:, 1:] = np.cumsum(cols, axis=1)                               # mass left of each edge
    # cumulative mass as a function of the mapped coordinate, read at the distorted edges.  All
    # columns sit end to end on one axis (offset `span` apart) so one np.interp call serves them;
    # queries outside a column's mapped support are clamped to that column's end values.
    span = 2.0 * (m + 2.0 + np.abs(bb).max())
    offs = np.arange(ncols, dtype=np.float64)[:, None] * span
    q = edges[None, :] + offs
    M = np.interp(q.ravel(), (mapped + offs).ravel(), mass.ravel()).reshape(ncols, m + 1)
    M = np.where(q <= mapped[:, :1] + offs, mass[:, :1], M)
    M = np.where(q >= mapped[:, -1:] + offs, mass[:, -1:], M)
    out = np.diff(M, axis=1).reshape(shape)
    return np.moveaxis(out, -1, pe_dim)


def make_pair(recipe: str | dict, seed: int | None = None, bmax: float | None = None,
              noise: float | None = None) -> Pair:
    """Draw one pair from a named recipe (see RECIPES) or a recipe dict."""
    r = dict(RECIPES[recipe]) if isinstance(recipe, str) else dict(recipe)
    if seed is not None:
        r["seed"] = seed
    if bmax is not None:
        r["bmax"] = bmax
    if noise is not None:
        r["noise"] = noise
    dims, pe = tuple(r["dims"]), int(r["pe_dim"])
    rng = np.random.default_rng(r["seed"])
    I = _ellipsoid_phantom(rng, dims, r["n_ellipsoids"], r["n_blobs"], r["semi_axes"],
                           r["smooth"])
    used = r["seed"]
    for attempt in range(100):
        frng = np.random.default_rng(used)
        frng.random(7)  # decorrelate from the phantom stream of the same seed
        b = _gaussian_field(frng, dims, pe, r["n_gauss"], r["sigma"], r["bmax"])
        slope = np.abs(np.diff(b, axis=pe)).max()
        if slope <= MAX_FIELD_SLOPE:
            break
        used += 100000
    else:
        # a peak this large is too steep for the shape: keep the last draw, scaled down to the
        # largest admissible slope (its peak is then below the recipe's)
        b = b * (MAX_FIELD_SLOPE / slope)
    Ip = push_forward(I, b, pe, +1.0)
    Im = push_forward(I, b, pe, -1.0)
    nrng = np.random.default_rng(r["seed"] + 7)
    if r["noise"] > 0:
        Ip = Ip + nrng.normal(0.0, r["noise"], size=dims)
        Im = Im + nrng.normal(0.0, r["noise"], size=dims)
    c32 = lambda a: np.ascontiguousarray(a, dtype=np.float32)   # noqa: E731
    return Pair(c32(Ip), c32(Im), c32(I), c32(b), tuple(r["spacing"]), pe, used)


# precision sweep: many diffusion-volume pairs of the 3T shape that share one field map (max 8
# voxels), each with its own contrast c ~ U(0.2, 1) and N(0, 0.03) noise
SWEEP = dict(recipe="3t", n_pairs=288, contrast=(0.2, 1.0), noise=0.03, seed=3000)

_sweep_base = {}


def make_sweep_pair(i: int) -> Pair:
    """Pair i (0 <= i < 288) of the precision sweep.  The push-forward is linear in the
    intensities, so pair i is c_i times the noise-free distorted base pair plus fresh noise."""
    if not 0 <= i < SWEEP["n_pairs"]:
        raise ValueError("sweep pair index out of range")
    if "pair" not in _sweep_base:
        _sweep_base["pair"] = make_pair(SWEEP["recipe"], noise=0.0)
    base = _sweep_base["pair"]
    rng = np.random.default_rng(SWEEP["seed"] + i)
    c = rng.uniform(*SWEEP["contrast"])
    Ip = c * base.Ip.astype(np.float64) + rng.normal(0.0, SWEEP["noise"], size=base.dims)
    Im = c * base.Im.astype(np.float64) + rng.normal(0.0, SWEEP["noise"], size=base.dims)
    c32 = lambda a: np.ascontiguousarray(a, dtype=np.float32)   # noqa: E731
    return Pair(c32(Ip), c32(Im), c32(c * base.I_true), base.b_true, base.spacing, base.pe_dim,
                base.seed)


# batch of uneven pairs (diffusion directions / subjects of several protocols): the 3T, the
# 7T-shaped and the 96x96x60 shapes in a seeded shuffle, PE along axis 0 or 1, each pair with its
# own seed and field-map peak U(4, 10) voxels
BATCH = dict(n_pairs=64, counts=(("3t", 22), ("7t", 21), ("small", 21)), bmax=(4.0, 10.0),
             seed=2000)


def batch_recipes(n_pairs: int | None = None) -> list:
    """Recipe dicts of the uneven batch (the first n_pairs of the 64 when given)."""
    rng = np.random.default_rng(BATCH["seed"])
    shapes = [name for name, k in BATCH["counts"] for _ in range(k)]
    order = rng.permutation(len(shapes))
    out = []
    for i, j in enumerate(order):
        r = dict(RECIPES[shapes[j]])
        r["pe_dim"] = int(rng.integers(0, 2))
        r["bmax"] = float(rng.uniform(*BATCH["bmax"]))
        r["seed"] = BATCH["seed"] + i
        r["name"] = shapes[j]
        out.append(r)
    return out[:n_pairs] if n_pairs is not None else out


def random_field(dims, pe_dim, seed, scale=1.0, smooth=2.0, max_slope=0.6):
    """A smooth random field on the staggered grid: peak |b| = scale, shrunk further if needed so
    that its largest PE difference is at most max_slope (test input)."""
    rng = np.random.default_rng(seed)
    fd = field_dims(dims, pe_dim)
    b = rng.normal(size=fd)
    if smooth > 0:
        b = ndimage.gaussian_filter(b, smooth, mode="nearest")
    b = b / max(np.abs(b).max(), 1e-30) * scale
    slope = np.abs(np.diff(b, axis=pe_dim)).max() if fd[pe_dim] > 1 else 0.0
    if slope > max_slope:
        b *= max_slope / slope
    return b.astype(np.float32)


def random_images(dims, seed, lo=0.0, hi=1.0):
    """Independent uniform random images (test input)."""
    rng = np.random.default_rng(seed)
    return (rng.uniform(lo, hi, size=dims).astype(np.float32),
            rng.uniform(lo, hi, size=dims).astype(np.float32))
