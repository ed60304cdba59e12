"""Seeded synthetic RVE inputs: phase maps, notch masks, material tables, random states.

This module draws inputs only. It holds none of the solver's arithmetic, so the
CPU oracle (``oracle/``) and the CUDA library can both be fed from it.

Geometry conventions (voxel size h = 1):
  * a voxel with integer index (i, j[, k]) sits at the point x = i, y = j[, z = k];
  * arrays are indexed ``[y, x]`` in 2D and ``[z, y, x]`` in 3D (x fastest);
  * a voxel lies inside a disc / sphere of radius r centred at c when its periodic
    minimum-image distance to c is <= r;
  * Random Sequential Adsorption (Sec. 5.2, the placement method the paper cites
    for its fibre composites) keeps a gap of one voxel between inclusions.

The workloads mirror the paper's examples: the fibre cross-section of Sec. 5.1/5.2
(rigid fibres in a matrix, 121x243 voxels there), the porous solid of Sec. 5.3 (random
spherical voids, 105^3 there) and the notched homogeneous panels of Sec. 4.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Optional, Sequence

import numpy as np

SEED_BASE = 2412_17445


@dataclasses.dataclass
class RVEInput:
    """Everything needed to create one RVE.

    shape:  (ny, nx) for 2D plane strain, (nz, ny, nx) for 3D.
    phase:  uint8 phase id per voxel, same shape.
    E, nu, Gc: per-phase Young modulus, Poisson ratio, toughness (length n_phases).
    ell:    phase-field length scale in voxels.
    notch:  uint8 mask (1 = initial crack voxel, phase field held at 1), same shape.
    f:      load direction tensor (d x d, symmetric) of the bordered control E_M = f E.
    """

    shape: tuple
    phase: np.ndarray
    E: np.ndarray
    nu: np.ndarray
    Gc: np.ndarray
    ell: float
    notch: np.ndarray
    f: np.ndarray
    name: str = ""

    @property
    def dim(self) -> int:
        return len(self.shape)


def tensile_f(dim: int) -> np.ndarray:
    """f = e_y (x) e_y, the tensile control tensor of Table 1."""
    f = np.zeros((dim, dim))
    f[1, 1] = 1.0
    return f


def shear_f(dim: int) -> np.ndarray:
    """Symmetric shear control tensor of Table 1 (y-z in 3D; x-y in plane strain)."""
    f = np.zeros((dim, dim))
    if dim == 3:
        f[1, 2] = f[2, 1] = 1.0
    else:
        f[0, 1] = f[1, 0] = 1.0
    return f


def _min_image(d: np.ndarray, n: int) -> np.ndarray:
    return d - n * np.round(d / n)


def rsa_centres(shape: Sequence[int], radius: float, fraction: float, seed: int,
                gap: float = 1.0, max_attempts: int = 2_000_000) -> np.ndarray:
    """Random Sequential Adsorption of equal discs (2D) or spheres (3D).

    Centres are drawn uniformly in the periodic box and kept when their minimum-image
    distance to every kept centre is at least 2 r + gap.  The count is the one whose
    analytic area / volume fraction is closest to ``fraction``.
    Returns an array (count, d) of centres in (x, y[, z]) order.
    """
    dims = list(shape)[::-1]  # (nx, ny[, nz])
    d = len(dims)
    cell = float(np.prod(dims))
    unit = math.pi * radius ** 2 if d == 2 else 4.0 / 3.0 * math.pi * radius ** 3
    count = int(round(fraction * cell / unit))
    rng = np.random.default_rng(seed)
    box = np.asarray(dims, dtype=float)
    centres = np.empty((count, d))
    k = 0
    attempts = 0
    dmin = 2.0 * radius + gap
    dmin2 = dmin * dmin
    # periodic cell list (cells at least dmin wide): a candidate is compared with the kept
    # centres of its own and the neighbouring cells only, which are all that can lie closer
    # than dmin; the accept / reject sequence is that of the all-pairs test
    ncell = [max(1, int(L // dmin)) for L in dims]
    csize = [L / m for L, m in zip(dims, ncell)]
    cells = {}
    offs = [()]
    for a in range(d):
        span = range(-1, 2) if ncell[a] >= 3 else range(ncell[a])
        offs = [o + (t,) for o in offs for t in span]
    while k < count:
        if attempts >= max_attempts:
            raise RuntimeError(f"RSA jammed after {attempts} attempts ({k}/{count} placed)")
        batch = rng.random((256, d)) * box
        for c in batch:
            attempts += 1
            ci = [min(int(c[a] // csize[a]), ncell[a] - 1) for a in range(d)]
            near = []
            for o in offs:
                key = tuple(((ci[a] + o[a]) if ncell[a] >= 3 else o[a]) % ncell[a] for a in range(d))
                near.extend(cells.get(key, ()))
            if near:
                dd = c[None, :] - centres[near]
                dd = dd - box * np.round(dd / box)
                if np.min(np.sum(dd * dd, axis=1)) < dmin2:
                    continue
            centres[k] = c
            cells.setdefault(tuple(ci), []).append(k)
            k += 1
            if k == count:
                break
    return centres


def voxelize_balls(shape: Sequence[int], centres: np.ndarray, radius: float) -> np.ndarray:
    """uint8 mask of voxels inside any ball (periodic minimum image, voxel at integer point)."""
    dims = list(shape)[::-1]
    d = len(dims)
    inside = np.zeros(dims, dtype=bool)
    r2 = radius * radius
    for c in centres:
        # only the voxels of the ball's periodic bounding box can be inside it
        idx, sq = [], []
        for a in range(d):
            lo, hi = int(math.floor(c[a] - radius)) - 1, int(math.ceil(c[a] + radius)) + 1
            ia = np.arange(dims[a]) if hi - lo + 1 >= dims[a] else np.arange(lo, hi + 1) % dims[a]
            dd = _min_image(ia.astype(float) - c[a], dims[a])
            idx.append(ia)
            sq.append(dd * dd)
        dist2 = sq[0]
        for a in range(1, d):
            dist2 = dist2[..., None] + sq[a].reshape((1,) * a + (-1,))
        inside[np.ix_(*idx)] |= dist2 <= r2
    # back to [y, x] / [z, y, x] order
    return np.ascontiguousarray(inside.T).astype(np.uint8)


def line_notch(shape: Sequence[int], x0: int, x1: int, y: Optional[int] = None) -> np.ndarray:
    """Straight notch: voxels x in [x0, x1) on the row y (default: mid-height N_y / 2)."""
    m = np.zeros(shape, dtype=np.uint8)
    ny = shape[-2]
    yy = ny // 2 if y is None else y
    if len(shape) == 2:
        m[yy, x0:x1] = 1
    else:
        m[:, yy, x0:x1] = 1
    return m


def penny_notch(shape: Sequence[int], radius: float) -> np.ndarray:
    """Penny-shaped notch in the mid-height x-z plane: (x - N/2)^2 + (z - N/2)^2 <= r^2."""
    nz, ny, nx = shape
    m = np.zeros(shape, dtype=np.uint8)
    z, x = np.meshgrid(np.arange(nz), np.arange(nx), indexing="ij")
    disc = (x - nx // 2) ** 2 + (z - nz // 2) ** 2 <= radius * radius
    m[:, ny // 2, :] = disc.astype(np.uint8)
    return m


def homogeneous_panel(n: int = 64, notch_len: int = 16, E: float = 1.0, nu: float = 0.3,
                      Gc: float = 1e-3, ell: float = 2.0) -> RVEInput:
    """2D plane-strain n x n homogeneous panel, notch from x = 0 to notch_len at mid-height."""
    shape = (n, n)
    return RVEInput(shape=shape, phase=np.zeros(shape, np.uint8), E=np.array([E]),
                    nu=np.array([nu]), Gc=np.array([Gc]), ell=ell,
                    notch=line_notch(shape, 0, notch_len), f=tensile_f(2),
                    name=f"panel{n}")


def fibre_composite(n: int = 512, radius: float = 12.0, fraction: float = 0.4,
                    notch_len: int = 32, seed: int = SEED_BASE + 1, E_m: float = 1.0,
                    E_f: float = 10.0, nu_m: float = 0.35, nu_f: float = 0.25,
                    Gc_m: float = 1e-3, Gc_f: float = 5e-3, ell: float = 2.0,
                    ny: Optional[int] = None) -> RVEInput:
    """2D fibre cross-section: RSA discs (phase 1) in a matrix (phase 0), central notch."""
    shape = (ny or n, n)
    centres = rsa_centres(shape, radius, fraction, seed)
    phase = voxelize_balls(shape, centres, radius)
    notch = line_notch(shape, n // 2 - notch_len // 2, n // 2 + notch_len // 2)
    return RVEInput(shape=shape, phase=phase, E=np.array([E_m, E_f]), nu=np.array([nu_m, nu_f]),
                    Gc=np.array([Gc_m, Gc_f]), ell=ell, notch=notch, f=tensile_f(2),
                    name=f"composite{shape[0]}x{shape[1]}")


def porous_solid(n: int = 128, radius: float = 8.0, porosity: float = 0.15,
                 notch_radius: float = 10.0, seed: int = SEED_BASE + 2, E: float = 1.0,
                 E_pore: float = 1e-6, nu: float = 0.3, Gc: float = 1e-3,
                 ell: float = 2.0, shape: Optional[Sequence[int]] = None) -> RVEInput:
    """3D porous RVE: RSA spheres modelled as a compliant phase (1), penny notch.
    shape = (nz, ny, nx) overrides the cube of side n."""
    shape = tuple(shape) if shape is not None else (n, n, n)
    centres = rsa_centres(shape, radius, porosity, seed)
    phase = voxelize_balls(shape, centres, radius)
    notch = penny_notch(shape, notch_radius)
    # Pores carry the matrix toughness and Poisson ratio (they are a compliant solid).
    return RVEInput(shape=shape, phase=phase, E=np.array([E, E_pore]), nu=np.array([nu, nu]),
                    Gc=np.array([Gc, Gc]), ell=ell, notch=notch, f=tensile_f(3),
                    name="porous" + "x".join(map(str, shape)))


def random_rve(shape: Sequence[int], seed: int, n_phases: int = 2, notch: bool = True) -> RVEInput:
    """Small random heterogeneous RVE for parity tests (random phases, random notch row)."""
    rng = np.random.default_rng(seed)
    shape = tuple(shape)
    d = len(shape)
    phase = (rng.random(shape) < 0.3).astype(np.uint8) if n_phases > 1 else np.zeros(shape, np.uint8)
    E = np.concatenate([[1.0], 1.0 + 4.0 * rng.random(n_phases - 1)])
    nu = 0.2 + 0.15 * rng.random(n_phases)
    Gc = 1e-3 * (1.0 + rng.random(n_phases))
    nmask = np.zeros(shape, np.uint8)
    if notch:
        nx = shape[-1]
        L = max(2, nx // 4)
        nmask = line_notch(shape, nx // 2 - L // 2, nx // 2 + L // 2)
    return RVEInput(shape=shape, phase=phase, E=E, nu=nu, Gc=Gc, ell=2.0, notch=nmask,
                    f=tensile_f(d), name=f"random{'x'.join(map(str, shape))}")


def random_state(inp: RVEInput, seed: int, strain: float = 1e-2, damage: bool = True):
    """A random, non-trivial linearisation point: (eps_tilde, E, phi, H_prev).

    eps_tilde is a random symmetric fluctuation field (d x d per voxel, zero mean is NOT
    imposed: the solver only needs a point to linearise about); phi in [0, 1) with the
    notch at 1; H_prev >= 0.
    """
    rng = np.random.default_rng(seed)
    d = inp.dim
    a = rng.standard_normal(inp.shape + (d, d)) * strain
    eps = 0.5 * (a + np.swapaxes(a, -1, -2))
    E = strain * (1.0 + rng.random())
    phi = 0.6 * rng.random(inp.shape) if damage else np.zeros(inp.shape)
    phi = np.where(inp.notch > 0, 1.0, phi)
    H = 0.5 * strain * strain * rng.random(inp.shape) * (rng.random(inp.shape) < 0.5)
    return eps, E, phi, H


def random_direction(inp: RVEInput, seed: int):
    """Random Krylov-space direction (d_eps, d_phi, d_E) for operator parity tests."""
    rng = np.random.default_rng(seed)
    d = inp.dim
    a = rng.standard_normal(inp.shape + (d, d))
    deps = 0.5 * (a + np.swapaxes(a, -1, -2))
    dphi = rng.standard_normal(inp.shape)
    dE = float(rng.standard_normal())
    return deps, dphi, dE
