"""Aggregation multigrid preconditioner for the inner solves (test infrastructure).

The paper preconditions its inner solves with BoomerAMG (Section 3.2); the CUDA path
offers Jacobi and this multigrid.  This module is the FP64 reference of the multigrid: an
unsmoothed-aggregation V-cycle on the voxel hierarchy, used as the preconditioner of the
inner CG for A and for S-hat_simple.  It is written from the definitions below, level by
level, with dense-free sparse products; the CUDA path shares none of it.

* Aggregates: level l + 1 merges the unknowns of level l whose voxel coordinates agree
  after halving (x // 2, y // 2, z // 2), and for velocity faces also the component a;
  a 2 x 2 x 2 block of voxels is one coarse unknown per component.
* P (n_l x n_(l+1)) is the piecewise-constant prolongation (P[i, agg(i)] = 1) and the
  coarse operator is the Galerkin product A_(l+1) = P^T A_l P.  With a 7-point operator
  the coarse operators stay 7-point (aggregates touch only face-adjacent aggregates).
* Coarsening continues until the grid is a single cell: the coarsest level then holds one
  unknown per velocity component (A) or one unknown (S-hat), and its matrix is diagonal
  (A couples no two components).  The coarsest system is solved exactly by the
  pseudo-inverse of that diagonal.
* A diagonal entry counts as zero when it is at most 1e-12 times the unknown's diagonal
  mass (the sum of the fine diagonal entries it aggregates): such an unknown lies in the
  nullspace (an aggregate of S-hat that is a whole isolated pore, or a component of A in
  a box without walls) and gets weight 0 in smoothing and in the coarsest solve.
* One V-cycle from x = 0: one weighted-Jacobi sweep (weight ``omega``), the coarse
  correction of the residual scaled by ``gamma`` (over-correction: a piecewise-constant
  prolongation under-estimates smooth errors), one Jacobi sweep after.  Pre- and
  post-smoothing are adjoint and the scaled coarse correction is symmetric, so the cycle
  is a symmetric operator; with omega * lambda_max(D^-1 A) <= 0.9 * 2 < 2 and
  0 < gamma < 2 it is positive definite on the range of A, as CG needs
  (``test_amg_vcycle_is_symmetric_positive_definite``).

Parameters (the same in the CUDA path): omega = 0.9; gamma = 1.3 for A and 1.7 for
S-hat, chosen by the inner iteration counts they give on sphere packings (porosity 0.15
and 0.40).
"""

from __future__ import annotations

from dataclasses import dataclass

import numpy as np
import scipy.sparse as sp

from . import mac

OMEGA = 0.9
GAMMA_A = 1.3
GAMMA_S = 1.7
ZERO_DIAG_RTOL = 1e-12


@dataclass
class Level:
    A: sp.csr_matrix
    dinv: np.ndarray              # inverse diagonal (0 where the diagonal counts as zero)
    P: sp.csr_matrix | None       # prolongation from the next level, None at the bottom


def _inverse_diagonal(A: sp.csr_matrix, mass: np.ndarray) -> np.ndarray:
    dg = A.diagonal()
    keep = dg > ZERO_DIAG_RTOL * mass
    return np.where(keep, 1.0 / np.where(keep, dg, 1.0), 0.0)


def build(A: sp.spmatrix, coords: np.ndarray, max_levels: int = 40) -> list:
    """Hierarchy for operator A whose unknown i sits at integer coordinates coords[i]
    (columns: the component first for velocity faces, then x, y, z; the component is
    never merged).  Levels are added until every unknown sits in cell (0, 0, 0)."""
    A = sp.csr_matrix(A)
    c = np.asarray(coords, dtype=np.int64)
    mass = A.diagonal().astype(np.float64)
    levels = []
    while True:
        n = A.shape[0]
        dinv = _inverse_diagonal(A, mass)
        if n == 0 or np.all(c[:, -3:] == 0) or len(levels) == max_levels - 1:
            off = A - sp.diags(A.diagonal())
            if off.count_nonzero():
                raise ValueError("the coarsest operator must be diagonal")
            levels.append(Level(A, dinv, None))
            return levels
        key = c.copy()
        key[:, -3:] //= 2                             # x, y, z halved; a component kept
        uniq, agg = np.unique(key, axis=0, return_inverse=True)
        agg = agg.ravel()
        nc = uniq.shape[0]
        P = sp.csr_matrix((np.ones(n), (np.arange(n), agg)), shape=(n, nc))
        levels.append(Level(A, dinv, P))
        A = (P.T @ A @ P).tocsr()
        mass = P.T @ mass
        c = uniq


def vcycle(levels: list, b: np.ndarray, gamma: float, omega: float = OMEGA,
           lev: int = 0) -> np.ndarray:
    """One V-cycle for A x = b from x = 0 (the preconditioner application M^-1 b)."""
    L = levels[lev]
    if L.P is None:
        return L.dinv * b                             # exact: pseudo-inverse of a diagonal
    x = omega * L.dinv * b                            # pre-smoothing from x = 0
    r = b - L.A @ x
    x = x + gamma * (L.P @ vcycle(levels, L.P.T @ r, gamma, omega, lev + 1))
    x = x + omega * L.dinv * (b - L.A @ x)            # post-smoothing (adjoint)
    return x


def face_coords(geo: mac.Geometry) -> np.ndarray:
    """(a, x, y, z) of every unknown face, in unknown order (z = 0 in 2D)."""
    out = np.zeros((geo.n_u, 4), dtype=np.int64)
    for a in range(geo.d):
        sel = geo.unknown[a]
        idx = np.nonzero(sel)
        k = geo.uidx[a][sel]
        xyz = _xyz(idx, geo.d)
        out[k, 0] = a
        out[k, 1:] = xyz
    return out


def cell_coords(geo: mac.Geometry) -> np.ndarray:
    """(x, y, z) of every fluid cell, in fluid-cell order (z = 0 in 2D)."""
    out = np.zeros((geo.n_p, 3), dtype=np.int64)
    idx = np.nonzero(geo.fluid)
    out[geo.pidx[geo.fluid]] = _xyz(idx, geo.d)
    return out


def _xyz(idx, d):
    """Array indices (C order, [z][y][x] or [y][x]) to columns x, y, z."""
    if d == 3:
        z, y, x = idx
    else:
        y, x = idx
        z = np.zeros_like(x)
    return np.stack([x, y, z], axis=1)
