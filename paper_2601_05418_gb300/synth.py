"""Seeded synthetic inputs shared by the CUDA path, its tests and the oracle.

This module holds none of the compression or reconstruction arithmetic: it
only draws the objects a scan would supply (object, receive-coil maps,
sampling lines, readout grouping, noise, region of interest) and resolves the
five workload geometries.  Everything is numpy with a PCG64 generator per seed.

Workloads (all synthetic; the paper's in-vivo / ex-vivo scans are not
available, so these stand in for them with the matrix sizes, coil counts,
oversampling factors and wave parameters of Sec. 3.2 and SI Sec. 5):

* ``2d128``   128x128, 8 coils, 4x oversampling, 8 wave cycles, 16 groups,
              about 10x compression, R=3, CG 20 iterations.
* ``2d256``   256x256, 32 coils, 8x oversampling, 32 groups, 16x, R=3,
              FISTA l1-Haar 50 iterations (FP32 operator).
* ``2d256h``  the same data with the FP16 tensor-core operator and
              compression (``2d256bf``: BF16 operands).
* ``batch64`` 64 uneven 2D slices (192..320, 16..32 coils, 6..8x, 16..48
              groups), CG 30 iterations each.
* ``3d224``   224x224x160, 32 coils, corkscrew wave, 6x, 48 contiguous
              groups compressed about 20x, 3x3 CAIPI, 10 CG iterations.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional

import numpy as np

# Matrix sizes for the uneven batch: multiples of 16 inside [192, 320] whose
# prime factors are at most 7, so every readout / phase-encode length is a
# product of the radices the FFT stages implement.
BATCH_SIZES = (192, 224, 240, 256, 288, 320)


@dataclasses.dataclass
class Geometry:
    """One slice or volume: sizes, wave parameters, grouping and sampling."""

    nx: int
    ny: int
    nz: int
    nc: int
    os: int
    cycles: float
    kappa_y: float
    kappa_z: float
    w: int
    n_groups: int
    patch_group: np.ndarray  # int32 [ntx // w]
    keep: np.ndarray  # int32 [n_groups]
    line_ky: np.ndarray  # int32 [n_lines], sorted by (kz, ky)
    line_kz: np.ndarray  # int32 [n_lines]

    @property
    def ntx(self) -> int:
        return self.os * self.nx

    @property
    def n_patches(self) -> int:
        return self.ntx // self.w

    @property
    def ns(self) -> int:
        return self.nc * self.w

    @property
    def n_lines(self) -> int:
        return int(self.line_ky.shape[0])

    @property
    def shape(self):
        return (self.nz, self.ny, self.nx)


@dataclasses.dataclass
class Workload:
    name: str
    geom: Geometry
    seed: int
    sigma: float = 1e-3
    alg: str = "cg"  # "cg" | "fista"
    iters: int = 20
    lam: float = 1e-3
    haar_levels: int = 4
    precision: str = "fp32"  # "fp32" | "bf16"


# ---------------------------------------------------------------- grouping --

def grouping_periodic(ntx: int, cycles: float, n_groups: int):
    """Per-period groups: one modulation period P_s = ntx / cycles split into
    n_groups sub-intervals of w samples; the group index repeats every period
    (Sec. 2.3, Fig. 3A).  Returns (w, patch_group)."""
    ps = ntx / cycles
    if abs(ps - round(ps)) > 1e-9:
        raise ValueError(f"period {ps} is not an integer number of samples")
    ps = int(round(ps))
    if ps % n_groups:
        raise ValueError(f"{n_groups} groups do not divide the period {ps}")
    w = ps // n_groups
    n_p = ntx // w
    return w, (np.arange(n_p) % n_groups).astype(np.int32)


def grouping_contiguous(ntx: int, n_groups: int):
    """One group per contiguous readout subregion (Sec. 5 generalisation to
    groups of identical modulation): patch p is its own group."""
    if ntx % n_groups:
        raise ValueError(f"{n_groups} groups do not divide {ntx} samples")
    w = ntx // n_groups
    return w, np.arange(n_groups, dtype=np.int32)


def keep_uniform(ns: int, n_groups: int, cf: float) -> np.ndarray:
    k = max(1, int(round(ns / cf)))
    return np.full(n_groups, min(k, ns), dtype=np.int32)


# ---------------------------------------------------------------- sampling --

def lines_regular(ny: int, r: int):
    """1D regular phase-encode undersampling: ky mod R == 0."""
    ky = np.arange(0, ny, r, dtype=np.int32)
    return ky, np.zeros_like(ky)


def lines_variable_density(ny: int, accel: float, seed: int, center: int = 16, power: float = 2.0):
    """Seeded 1D variable-density random phase-encode mask, a stand-in for
    the Poisson-disc variable-density masks the paper draws with BART for
    its compressed-sensing reconstructions: the `center` lines around
    ky = N_y/2 always, the rest drawn without replacement with probability
    proportional to (1 - |ky_c| / (N_y/2))^power until round(N_y / accel)
    lines are taken.  Sorted, unique."""
    n_take = max(1, int(round(ny / accel)))
    kyc = np.arange(ny) - ny // 2
    fixed = np.flatnonzero(np.abs(kyc + 0.5) < center / 2)
    if len(fixed) >= n_take:
        ky = np.sort(fixed[np.argsort(np.abs(kyc[fixed] + 0.5), kind="stable")[:n_take]])
        return ky.astype(np.int32), np.zeros(len(ky), np.int32)
    rest = np.setdiff1d(np.arange(ny), fixed)
    wgt = np.maximum(1.0 - np.abs(kyc[rest]) / (ny / 2), 1e-6) ** power
    rng = np.random.default_rng(seed)
    pick = rng.choice(rest, size=n_take - len(fixed), replace=False, p=wgt / wgt.sum())
    ky = np.sort(np.concatenate([fixed, pick])).astype(np.int32)
    return ky, np.zeros(len(ky), np.int32)


def local_b0_fields(nx: int, ny: int, nz: int, n_fields: int, seed: int, peak: float = 6.0) -> np.ndarray:
    """Seeded synthetic fields of local B0 coils (no measured field maps
    exist here): smooth Gaussian bumps [n_fields][nz][ny][nx] centred near
    the edge of the field of view, width 0.3 FOV, in radians at unit
    amplitude (peak radians at the bump centre)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    zz, yy, xx = np.meshgrid((np.arange(nz) - nz / 2) / max(nz, 1), (np.arange(ny) - ny / 2) / ny,
                             (np.arange(nx) - nx / 2) / nx, indexing="ij")
    out = np.zeros((n_fields, nz, ny, nx))
    for k in range(n_fields):
        ang = 2 * np.pi * (k + rng.uniform(-0.2, 0.2)) / n_fields
        cy, cx = 0.45 * np.sin(ang), 0.45 * np.cos(ang)
        out[k] = peak * np.exp(-((yy - cy) ** 2 + (xx - cx) ** 2 + zz ** 2) / (2 * 0.3 ** 2))
    return out


def local_b0_amplitudes(ntx: int, cycles: float, n_fields: int, seed: int) -> np.ndarray:
    """Seeded sinusoidal drive of each local B0 coil over the readout,
    a_k(t) = sin(2 pi cycles t / N_tx + phase_k), [n_fields][ntx]."""
    rng = np.random.Generator(np.random.PCG64(seed))
    t = np.arange(ntx)
    ph = rng.uniform(0, 2 * np.pi, n_fields)
    return np.sin(2 * np.pi * cycles * t[None, :] / ntx + ph[:, None])


def lines_caipi(ny: int, nz: int, ry: int, rz: int):
    """2D CAIPI: kz mod rz == 0 and ky mod ry == (kz / rz) mod ry.
    Sorted by (kz, ky)."""
    ky_l, kz_l = [], []
    for kz in range(0, nz, rz):
        shift = (kz // rz) % ry
        for ky in range(shift, ny, ry):
            ky_l.append(ky)
            kz_l.append(kz)
    return np.asarray(ky_l, np.int32), np.asarray(kz_l, np.int32)


def lines_full(ny: int, nz: int):
    kz, ky = np.meshgrid(np.arange(nz), np.arange(ny), indexing="ij")
    return ky.ravel().astype(np.int32), kz.ravel().astype(np.int32)


# ---------------------------------------------------------------- objects --

# (cx, cy, cz, a, b, c, angle_deg, value) in field-of-view units [-0.5, 0.5).
_ELLIPSES = (
    (0.00, 0.00, 0.00, 0.42, 0.36, 0.40, 0.0, 0.80),
    (0.00, -0.02, 0.00, 0.38, 0.32, 0.36, 0.0, -0.30),
    (-0.12, 0.05, 0.04, 0.08, 0.15, 0.12, 20.0, 0.30),
    (0.14, 0.06, -0.05, 0.06, 0.12, 0.10, -15.0, 0.40),
    (0.00, -0.18, 0.10, 0.05, 0.05, 0.06, 0.0, 0.20),
    (0.05, 0.20, -0.08, 0.10, 0.04, 0.08, 10.0, -0.15),
    (-0.20, -0.10, 0.00, 0.03, 0.06, 0.05, 35.0, 0.25),
)


def _grid(nx, ny, nz):
    x = (np.arange(nx) - nx // 2) / nx
    y = (np.arange(ny) - ny // 2) / ny
    z = (np.arange(nz) - nz // 2) / max(nz, 1) if nz > 1 else np.zeros(1)
    zz, yy, xx = np.meshgrid(z, y, x, indexing="ij")
    return zz, yy, xx


def phantom(nx: int, ny: int, nz: int = 1, edge_px: float = 1.5) -> np.ndarray:
    """Smooth-edged ellipse (ellipsoid) phantom, real, maximum 1.
    Shape [nz][ny][nx], complex128."""
    zz, yy, xx = _grid(nx, ny, nz)
    img = np.zeros(zz.shape)
    for cx, cy, cz, a, b, c, ang, val in _ELLIPSES:
        th = math.radians(ang)
        dx, dy = xx - cx, yy - cy
        u = dx * math.cos(th) + dy * math.sin(th)
        v = -dx * math.sin(th) + dy * math.cos(th)
        q2 = (u / a) ** 2 + (v / b) ** 2
        if nz > 1:
            q2 = q2 + ((zz - cz) / c) ** 2
        # signed distance (in pixels of the smallest semi-axis) to the edge
        dist = (np.sqrt(q2) - 1.0) * min(a * nx, b * ny)
        img += val / (1.0 + np.exp(np.clip(dist / (edge_px / 4.0), -60, 60)))
    img = np.clip(img, 0.0, None)
    img /= img.max()
    return img.astype(np.complex128)


def coil_maps(nx: int, ny: int, nz: int, nc: int, seed: int) -> np.ndarray:
    """Gaussian-magnitude, smooth-phase receive coils on a circle (2D) or on
    rings of a cylinder (3D) of radius 0.6 FOV.  Not RSS-normalised.
    Shape [nc][nz][ny][nx], complex128."""
    rng = np.random.Generator(np.random.PCG64(seed))
    zz, yy, xx = _grid(nx, ny, nz)
    n_rings = 1 if nz == 1 else (4 if nc % 4 == 0 and nc >= 8 else 1)
    per_ring = nc // n_rings
    maps = np.empty((nc,) + zz.shape, np.complex128)
    for n in range(nc):
        ring, k = divmod(n, per_ring)
        ang = 2 * math.pi * (k + 0.5 * (ring % 2)) / per_ring
        cx, cy = 0.6 * math.cos(ang), 0.6 * math.sin(ang)
        cz = 0.0 if n_rings == 1 else (-0.3 + 0.6 * ring / (n_rings - 1))
        d2 = (xx - cx) ** 2 + (yy - cy) ** 2 + ((zz - cz) ** 2 if nz > 1 else 0)
        mag = np.exp(-d2 / (2 * 0.4 ** 2))
        ph0 = rng.uniform(-math.pi, math.pi)
        bx, by, bz = rng.uniform(-0.3, 0.3, size=3)
        amp = rng.uniform(0.25, 0.5) * math.pi
        bump = np.exp(-((xx - bx) ** 2 + (yy - by) ** 2
                        + ((zz - bz) ** 2 if nz > 1 else 0)) / (2 * 0.25 ** 2))
        maps[n] = mag * np.exp(1j * (ph0 + amp * bump))
    return maps


def roi_mask(img: np.ndarray, dilate: int = 2, thresh: float = 1e-3) -> np.ndarray:
    """Object support (|img| > thresh) dilated by `dilate` pixels (voxels).
    uint8 [nz][ny][nx]."""
    from scipy import ndimage

    sup = np.abs(img) > thresh
    if sup.shape[0] == 1:
        st = np.ones((1, 2 * dilate + 1, 2 * dilate + 1), bool)
    else:
        st = np.ones((2 * dilate + 1,) * 3, bool)
    return ndimage.binary_dilation(sup, structure=st).astype(np.uint8)


def complex_normal(shape, seed: int, sigma: float = 1.0) -> np.ndarray:
    """Circular complex Gaussian with E|n|^2 = sigma^2."""
    rng = np.random.Generator(np.random.PCG64(seed))
    s = sigma / math.sqrt(2.0)
    return rng.normal(0.0, s, shape) + 1j * rng.normal(0.0, s, shape)


def complex_normal_c64(shape, seed: int, sigma: float = 1.0) -> np.ndarray:
    """Same draw as `complex_normal`, returned as complex64."""
    return complex_normal(shape, seed, sigma).astype(np.complex64)


def random_psd(n: int, seed: int, cond: float = 4.0) -> np.ndarray:
    """Random Hermitian positive-definite matrix (a noise covariance)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    q, _ = np.linalg.qr(rng.normal(size=(n, n)) + 1j * rng.normal(size=(n, n)))
    ev = np.geomspace(1.0, cond, n)
    return (q * ev) @ q.conj().T


# ---------------------------------------------------------------- workloads --

def _geom_2d(n, nc, os, cycles, kappa, n_groups, cf, r, grouping="periodic"):
    ntx = os * n
    if grouping == "periodic":
        w, pg = grouping_periodic(ntx, cycles, n_groups)
    else:
        w, pg = grouping_contiguous(ntx, n_groups)
    ky, kz = lines_regular(n, r)
    return Geometry(nx=n, ny=n, nz=1, nc=nc, os=os, cycles=float(cycles),
                    kappa_y=float(kappa), kappa_z=0.0, w=w, n_groups=n_groups,
                    patch_group=pg, keep=keep_uniform(nc * w, n_groups, cf),
                    line_ky=ky, line_kz=kz)


def workload(name: str) -> Workload:
    if name == "2d128":
        g = _geom_2d(128, 8, 4, 8, 2.5, 16, 10.0, 3)
        return Workload(name, g, seed=1, alg="cg", iters=20)
    if name in ("2d256", "2d256bf", "2d256h"):
        g = _geom_2d(256, 32, 8, 8, 2.5, 32, 16.0, 3)
        prec = {"2d256": "fp32", "2d256bf": "bf16", "2d256h": "fp16"}[name]
        return Workload(name, g, seed=2, alg="fista", iters=50, lam=1e-3,
                        haar_levels=4, precision=prec)
    if name == "3d224":
        return Workload(name, geom_3d(224, 224, 160, 32, 6, 11, 6.0, 4.5, 48, 20.0),
                        seed=5, alg="cg", iters=10)
    if name == "3d56":  # reduced 3D case the oracle finishes in seconds
        return Workload(name, geom_3d(56, 56, 40, 8, 6, 11, 1.5, 1.125, 12, 20.0),
                        seed=5, alg="cg", iters=10)
    # the 3D volume with per-period groups: 14 cycles over 1344 samples give
    # an integer period of 96 samples, cut into 48 groups of w = 2
    if name == "3d224r1":
        return Workload(name, geom_3d(224, 224, 160, 32, 6, 14, 6.0, 4.5, 48, 20.0, grouping="periodic"),
                        seed=5, alg="cg", iters=10)
    if name == "3d56r1":  # its reduced case: 336 samples, 14 cycles -> period 24, 12 groups of w = 2
        return Workload(name, geom_3d(56, 56, 40, 8, 6, 14, 1.5, 1.125, 12, 8.0, grouping="periodic"),
                        seed=5, alg="cg", iters=10)
    raise KeyError(name)


def geom_3d(nx, ny, nz, nc, os, cycles, ky_amp, kz_amp, n_groups, cf,
            ry=3, rz=3, grouping="contiguous") -> Geometry:
    ntx = os * nx
    if grouping == "periodic":
        w, pg = grouping_periodic(ntx, cycles, n_groups)
    else:
        w, pg = grouping_contiguous(ntx, n_groups)
    ky, kz = lines_caipi(ny, nz, ry, rz)
    return Geometry(nx=nx, ny=ny, nz=nz, nc=nc, os=os, cycles=float(cycles),
                    kappa_y=float(ky_amp), kappa_z=float(kz_amp), w=w,
                    n_groups=n_groups, patch_group=pg,
                    keep=keep_uniform(nc * w, n_groups, cf),
                    line_ky=ky, line_kz=kz)


def batch_workloads(n_slices: int = 64, seed: int = 4) -> List[Workload]:
    """Uneven 2D slices: size, coils, oversampling and group count drawn per
    slice; group counts are rejection-sampled to divide the period."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    while len(out) < n_slices:
        n = int(rng.choice(BATCH_SIZES))
        nc = int(rng.choice(np.arange(16, 33, 4)))
        os = int(rng.choice((6, 7, 8)))
        ng = int(rng.choice((16, 24, 32, 48)))
        ps = os * n // 8
        if (os * n) % 8 or ps % ng:
            continue
        g = _geom_2d(n, nc, os, 8, 2.5, ng, 16.0, 3)
        out.append(Workload(f"batch{len(out)}", g, seed=seed * 1000 + len(out),
                            alg="cg", iters=30))
    return out


@dataclasses.dataclass
class Case:
    """Seeded arrays for one workload (no measured data exists)."""

    rho: np.ndarray  # [nz][ny][nx] complex128, ground-truth object
    coils: np.ndarray  # [nc][nz][ny][nx] complex128
    roi: np.ndarray  # [nz][ny][nx] uint8
    noise: np.ndarray  # [n_lines][nc][ntx] complex128, E|n|^2 = sigma^2


def make_case(wl: Workload, with_noise: bool = True) -> Case:
    g = wl.geom
    rho = phantom(g.nx, g.ny, g.nz)
    coils = coil_maps(g.nx, g.ny, g.nz, g.nc, wl.seed)
    roi = roi_mask(rho)
    shape = (g.n_lines, g.nc, g.ntx)
    noise = (complex_normal(shape, wl.seed + 7919, wl.sigma) if with_noise
             else np.zeros(shape, np.complex128))
    return Case(rho=rho, coils=coils, roi=roi, noise=noise)


def tiny_geometry(nx=8, ny=6, nz=1, nc=2, os=2, cycles=2.0, kappa_y=1.3,
                  kappa_z=0.0, n_groups=2, keep: Optional[int] = None,
                  grouping="periodic", lines="full", r=2) -> Geometry:
    """Small grids for brute-force checks."""
    ntx = os * nx
    if grouping == "periodic":
        w, pg = grouping_periodic(ntx, cycles, n_groups)
    else:
        w, pg = grouping_contiguous(ntx, n_groups)
    if lines == "full":
        ky, kz = lines_full(ny, nz)
    elif lines == "regular":
        ky, kz = lines_regular(ny, r)
        if nz > 1:
            raise ValueError("regular lines are 2D")
    else:
        ky, kz = lines_caipi(ny, nz, r, r)
    ns = nc * w
    k = ns if keep is None else keep
    return Geometry(nx=nx, ny=ny, nz=nz, nc=nc, os=os, cycles=float(cycles),
                    kappa_y=float(kappa_y), kappa_z=float(kappa_z), w=w,
                    n_groups=n_groups, patch_group=pg,
                    keep=np.full(n_groups, k, np.int32), line_ky=ky, line_kz=kz)
