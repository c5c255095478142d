"""Seeded synthetic voxel geometries (inputs only; no solver arithmetic).

Every mask returned here is a C-ordered ``numpy.uint8`` array, ``[z][y][x]`` in 3D
and ``[y][x]`` in 2D, with 1 = fluid voxel and 0 = solid voxel (the binary image of
Section 2.1, eq. cube_domain / domains_partition).  The same module feeds the CUDA
path, the oracle and the benchmarks, so that both sides see identical inputs.

Generators
----------
* ``channel_2d``      plane channel: solid rows at the bottom and top of a periodic
                      box (the plane-Poiseuille workload, 32x32 with a 30-cell band).
* ``square_array_2d`` N x N cells of n_c pixels, each holding one solid square of
                      side n_c - n_avg, shifted by integer offsets in
                      [-(n_avg - n_min)/2, (n_avg - n_min)/2] (Section 4.2.1).
* ``sphere_packing``  periodic overlapping solid spheres, centres uniform in the
                      box and radii uniform in [r_min, r_max), added one by one until
                      the porosity drops to the target (stand-in for the CT images of
                      Table 1, which are not available).

Randomness comes from SplitMix64 (Steele, Lea and Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014): state += 0x9E3779B97F4A7C15, then the
published mix with shifts 30/27/31 and multipliers 0xBF58476D1CE4E5B9 and
0x94D049BB133111EB.  A double in [0, 1) is the top 53 bits times 2^-53.
"""

from __future__ import annotations

import numpy as np

_MASK64 = (1 << 64) - 1


class SplitMix64:
    """Counter-based 64-bit generator; identical sequence in any language."""

    def __init__(self, seed: int):
        self.state = int(seed) & _MASK64

    def next_u64(self) -> int:
        self.state = (self.state + 0x9E3779B97F4A7C15) & _MASK64
        z = self.state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _MASK64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _MASK64
        return z ^ (z >> 31)

    def next_double(self) -> float:
        return (self.next_u64() >> 11) * (1.0 / 9007199254740992.0)

    def next_int(self, lo: int, hi: int) -> int:
        """Uniform integer in the closed range [lo, hi]."""
        span = hi - lo + 1
        return lo + min(int(self.next_double() * span), span - 1)


def channel_2d(n: int = 32) -> np.ndarray:
    """2D n x n box, fluid everywhere except the first and last rows (y = 0, y = n-1).

    With periodic x and y this is a plane channel with ``n - 2`` fluid rows; the
    solid rows meet across the periodic y boundary, so the band is bounded by walls
    on both sides.
    """
    mask = np.ones((n, n), dtype=np.uint8)
    mask[0, :] = 0
    mask[n - 1, :] = 0
    return mask


def square_array_2d(N: int, n_c: int, n_avg: int, n_min: int, seed: int) -> np.ndarray:
    """Array of randomly shifted solid squares (Section 4.2.1, generator of Fig. 4).

    The domain is ``n = N * n_c`` pixels per side, an N x N array of cells of
    ``n_c`` pixels.  Each cell holds one solid square of side ``s = n_c - n_avg``
    whose centre sits at ``(n_c/2 + r_x, n_c/2 + r_y)`` inside the cell, with integer
    shifts drawn uniformly from ``[-(n_avg - n_min)/2, (n_avg - n_min)/2]``.  The
    paper calls that point the square's "origin"; reading it as the centre keeps
    every channel at least ``n_min`` pixels wide and reproduces Table 3.
    Shifts are drawn cell by cell in C order (row j, then column i), x before y.
    """
    s = n_c - n_avg
    if s <= 0 or s % 2 or n_c % 2:
        raise ValueError("square_array_2d needs even n_c and even n_c - n_avg > 0")
    if n_avg < n_min or (n_avg - n_min) % 2:
        raise ValueError("square_array_2d needs n_avg >= n_min with n_avg - n_min even")
    m = (n_avg - n_min) // 2
    rng = SplitMix64(seed)
    n = N * n_c
    mask = np.ones((n, n), dtype=np.uint8)
    for j in range(N):
        for i in range(N):
            rx = rng.next_int(-m, m)
            ry = rng.next_int(-m, m)
            x0 = i * n_c + n_c // 2 + rx - s // 2
            y0 = j * n_c + n_c // 2 + ry - s // 2
            mask[y0:y0 + s, x0:x0 + s] = 0
    return mask


def sphere_packing(n, r_min: float, r_max: float, porosity: float, seed: int,
                   max_spheres: int = 10_000_000) -> np.ndarray:
    """Periodic overlapping solid spheres in an ``n^3`` box (``n`` may be a 3-tuple
    ``(nx, ny, nz)``).

    Sphere k draws, in this order, its centre ``c_x, c_y, c_z`` uniform in
    ``[0, n_x) x [0, n_y) x [0, n_z)`` and its radius uniform in ``[r_min, r_max)``.
    Voxel ``(i, j, l)`` becomes solid when the periodic distance from its centre
    ``(i + 1/2, j + 1/2, l + 1/2)`` to ``c`` is at most the radius, compared as
    ``(dx*dx + dy*dy) + dz*dz <= r*r`` in double precision.  Spheres are added one at
    a time and generation stops right after the first sphere that brings the fluid
    fraction to ``porosity`` or below.
    """
    if np.isscalar(n):
        nx = ny = nz = int(n)
    else:
        nx, ny, nz = (int(v) for v in n)
    if not (0.0 < porosity < 1.0):
        raise ValueError("porosity must lie in (0, 1)")
    if 2.0 * r_max + 2.0 > min(nx, ny, nz):
        raise ValueError("sphere diameter + 2 must not exceed the box edge")
    mask = np.ones((nz, ny, nx), dtype=np.uint8)
    total = nx * ny * nz
    fluid = total
    rng = SplitMix64(seed)
    target = porosity * total
    for _ in range(max_spheres):
        cx = rng.next_double() * nx
        cy = rng.next_double() * ny
        cz = rng.next_double() * nz
        r = r_min + (r_max - r_min) * rng.next_double()
        ix = np.arange(int(np.floor(cx - r - 0.5)), int(np.ceil(cx + r - 0.5)) + 1)
        iy = np.arange(int(np.floor(cy - r - 0.5)), int(np.ceil(cy + r - 0.5)) + 1)
        iz = np.arange(int(np.floor(cz - r - 0.5)), int(np.ceil(cz + r - 0.5)) + 1)
        dx = ix + 0.5 - cx
        dy = iy + 0.5 - cy
        dz = iz + 0.5 - cz
        dxy = (dx * dx)[None, :] + (dy * dy)[:, None]            # [y][x]
        inside = (dxy[None, :, :] + (dz * dz)[:, None, None]) <= r * r
        sub = np.ix_(iz % nz, iy % ny, ix % nx)
        block = mask[sub]
        fluid -= int(np.count_nonzero(block[inside]))
        block[inside] = 0
        mask[sub] = block
        if fluid <= target:
            return mask
    raise RuntimeError("porosity target not reached within max_spheres")


def fluid_fraction(mask: np.ndarray) -> float:
    """Share of fluid voxels (the porosity of eq. porosity as a fraction)."""
    return float(np.count_nonzero(mask)) / mask.size
