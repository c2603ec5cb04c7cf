"""Seeded synthetic inputs shared by the CUDA path, the tests and the benchmark.

This module holds no arithmetic of the method (no operator, no regulariser, no solver):
only phantoms, masks and standard-normal noise drawn from numpy's PCG64, plus the
workload recipes (sizes and parameters) of the deblurring, inpainting and tomography
problems the solver is measured on.  The paper's own experiments (a 1D deconvolution
whose true signal exists only as a figure, and a 3D FEM fluorescence DOT model, Sec. 5)
cannot be reproduced, so these seeded images stand in for them.

Phantom recipe: background 0; shapes painted in draw order (later shapes overwrite
earlier ones); each shape's value is U[0,1]; a pixel belongs to a shape when its centre
does; shape centres are uniform in the inner 80% of the image.  Rectangle sides are
U[0.05,0.4]*n, disk radii U[0.03,0.15]*n, ellipse / ellipsoid semi-axes U[0.05,0.3]*n
with a uniform random rotation.
"""
from dataclasses import dataclass, field

import numpy as np


def _shape2(n):
    return (int(n), int(n)) if np.isscalar(n) else (int(n[0]), int(n[1]))


def _centre(rng, ny, nx):
    """Uniform centre in the inner 80% of each axis (x, y)."""
    u = rng.uniform(0.1, 0.9, size=2)
    return u[0] * nx, u[1] * ny


def phantom_rects_disks(n, n_rect, n_disk, seed):
    """2D piecewise-constant image (n or (ny, nx)) of axis-aligned rectangles then disks."""
    rng = np.random.default_rng(seed)
    ny, nx = _shape2(n)
    s = min(ny, nx)
    img = np.zeros((ny, nx))
    yy, xx = np.mgrid[0:ny, 0:nx] + 0.5
    for _ in range(n_rect):
        cx, cy = _centre(rng, ny, nx)
        wx, wy = rng.uniform(0.05, 0.4, size=2) * np.array([nx, ny])
        val = rng.uniform(0.0, 1.0)
        inside = (np.abs(xx - cx) <= 0.5 * wx) & (np.abs(yy - cy) <= 0.5 * wy)
        img[inside] = val
    for _ in range(n_disk):
        cx, cy = _centre(rng, ny, nx)
        r = rng.uniform(0.03, 0.15) * s
        val = rng.uniform(0.0, 1.0)
        img[(xx - cx) ** 2 + (yy - cy) ** 2 <= r * r] = val
    return img


def phantom_ellipses(n, count, seed):
    """2D image (n or (ny, nx)) of rotated ellipses (tomography phantom)."""
    rng = np.random.default_rng(seed)
    ny, nx = _shape2(n)
    s = min(ny, nx)
    img = np.zeros((ny, nx))
    yy, xx = np.mgrid[0:ny, 0:nx] + 0.5
    for _ in range(count):
        cx, cy = _centre(rng, ny, nx)
        a, b = rng.uniform(0.05, 0.3, size=2) * s
        phi = rng.uniform(0.0, np.pi)
        val = rng.uniform(0.0, 1.0)
        dx, dy = xx - cx, yy - cy
        xr = dx * np.cos(phi) + dy * np.sin(phi)
        yr = -dx * np.sin(phi) + dy * np.cos(phi)
        img[(xr / a) ** 2 + (yr / b) ** 2 <= 1.0] = val
    return img


def _rotation(rng):
    q, r = np.linalg.qr(rng.standard_normal((3, 3)))
    q = q * np.sign(np.diag(r))
    if np.linalg.det(q) < 0:
        q[:, 0] = -q[:, 0]
    return q


def phantom_ellipsoids(shape, count, seed):
    """3D (nz, ny, nx) volume of rotated ellipsoids."""
    rng = np.random.default_rng(seed)
    nz, ny, nx = shape
    vol = np.zeros(shape)
    zz, yy, xx = np.mgrid[0:nz, 0:ny, 0:nx] + 0.5
    for _ in range(count):
        c = np.array([rng.uniform(0.1 * nx, 0.9 * nx), rng.uniform(0.1 * ny, 0.9 * ny),
                      rng.uniform(0.1 * nz, 0.9 * nz)])
        ax = rng.uniform(0.05, 0.3, size=3) * np.array([nx, ny, nz])
        Q = _rotation(rng)
        val = rng.uniform(0.0, 1.0)
        d = np.stack([xx - c[0], yy - c[1], zz - c[2]], axis=-1)
        loc = d @ Q
        vol[((loc / ax) ** 2).sum(-1) <= 1.0] = val
    return vol


def observation_mask(shape, missing_fraction, seed):
    """uint8 mask, 1 = observed; each voxel is missing with probability missing_fraction."""
    rng = np.random.default_rng(seed)
    return (rng.random(shape) >= missing_fraction).astype(np.uint8)


def standard_noise(shape, seed):
    """Standard-normal noise field (the caller scales it to the requested level)."""
    return np.random.default_rng(seed).standard_normal(shape)


def add_noise(clean, level, z):
    """g = clean + level * ||clean|| / sqrt(m) * z: white noise at a relative RMS level."""
    clean = np.asarray(clean, dtype=np.float64)
    sig = level * np.linalg.norm(clean) / np.sqrt(clean.size)
    return clean + sig * z


@dataclass
class Workload:
    """One solver workload: problem size, forward map, regulariser and iteration counts."""
    name: str
    kind: str                 # 'blur' | 'blur_mask' | 'joseph'
    shape: tuple              # image shape (ny, nx) or (nz, ny, nx)
    precision: str            # 'fp64' | 'fp32'
    reg: str                  # 'tikhonov' | 'tv' | 'pm_log' | 'pm_exp'
    T: float
    tau: float
    n_outer: int
    n_inner: int
    levels: int
    nu: int = 2
    cycles: int = 1
    sigma: tuple = (0.0, 0.0, 0.0)   # x, y, z
    radius: tuple = (0, 0, 0)
    noise: float = 0.01
    missing: float = 0.0
    n_angles: int = 0
    n_bins: int = 0
    phantom: dict = field(default_factory=dict)

    def phantom_image(self, seed):
        p = self.phantom
        if p["type"] == "rects_disks":
            return phantom_rects_disks(self.shape, p["rects"], p["disks"], seed)
        if p["type"] == "ellipses":
            return phantom_ellipses(self.shape, p["count"], seed)
        if p["type"] == "ellipsoids":
            return phantom_ellipsoids(self.shape, p["count"], seed)
        raise ValueError(p["type"])

    def data_shape(self):
        return (self.n_angles, self.n_bins) if self.kind == "joseph" else tuple(self.shape)

    def inputs(self, seed):
        """(f_true, mask or None, unit noise) for instance `seed`."""
        f = self.phantom_image(seed)
        mask = observation_mask(self.shape, self.missing, seed + 7919) if self.kind == "blur_mask" else None
        z = standard_noise(self.data_shape(), seed + 104729)
        return f, mask, z


def _jbins(n):
    b = int(np.ceil(n * np.sqrt(2.0))) + 1
    return b if b % 2 == 1 else b + 1


WORKLOADS = {
    # 2D deblurring 64x64 in double precision
    "deblur64_fp64": Workload("deblur64_fp64", "blur", (64, 64), "fp64", "tv", 1e-2, 5e-3, 10, 30,
                              levels=3, nu=2, cycles=2, sigma=(2.0, 2.0), radius=(6, 6),
                              phantom=dict(type="rects_disks", rects=6, disks=4)),
    # 2D deblurring 1024x1024, FP32 bulk
    "deblur1024_fp32": Workload("deblur1024_fp32", "blur", (1024, 1024), "fp32", "pm_log", 5e-2, 1e-3,
                                15, 50, levels=6, nu=2, cycles=1, sigma=(4.0, 4.0), radius=(12, 12),
                                phantom=dict(type="rects_disks", rects=40, disks=25)),
    # 3D blur + inpainting 192^3, FP32 bulk, 15% of voxels missing
    "inpaint192_fp32": Workload("inpaint192_fp32", "blur_mask", (192, 192, 192), "fp32", "tv", 1e-2, 0.0,
                                10, 40, levels=5, nu=2, cycles=1, sigma=(3.0, 3.0, 5.0),
                                radius=(9, 9, 15), noise=0.005, missing=0.15,
                                phantom=dict(type="ellipsoids", count=30)),
    # 2D parallel-beam tomography 512x512, 360 angles x 725 bins, FP32 bulk
    "tomo512_fp32": Workload("tomo512_fp32", "joseph", (512, 512), "fp32", "pm_exp", 2e-2, 0.0,
                             12, 60, levels=6, nu=2, cycles=1, n_angles=360, n_bins=725,
                             phantom=dict(type="ellipses", count=10)),
}
