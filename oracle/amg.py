"""Aggregation multigrid preconditioner for the inner solves (test infrastructure).

The paper preconditions its inner solves with BoomerAMG (Section 3.2); the CUDA path uses
Jacobi.  This module is the FP64 reference of a stronger, GPU-friendly replacement: an
unsmoothed-aggregation multigrid on the voxel hierarchy, used as the preconditioner of
the inner CG for A and for S-hat_simple.

* Aggregates: level l + 1 merges the unknowns of level l whose voxel coordinates agree
  after halving (x // 2, y // 2, z // 2), and for velocity faces also the component a;
  a 2 x 2 x 2 block of voxels is one coarse unknown per component.
* P (n_l x n_(l+1)) is the piecewise-constant prolongation (P[i, agg(i)] = 1) and the
  coarse operator is the Galerkin product A_(l+1) = P^T A_l P.  With a 7-point operator
  the coarse operators stay 7-point (aggregates touch only face-adjacent aggregates).
* Coarsening stops when a level has at most ``min_coarse`` unknowns or stops shrinking;
  the coarsest system is solved with the pseudo-inverse (S-hat_simple is singular: its
  nullspace, the constants of each fluid component, is kept by P).
* One V-cycle: ``nu`` weighted-Jacobi sweeps (weight ``omega``) from x = 0, the coarse
  correction of the residual, ``nu`` sweeps after.  Pre- and post-smoothing are adjoint,
  so the cycle is a symmetric operator; with omega = 2/3 below 2 / lambda_max(D^-1 A) it
  is positive definite on the range of A, as CG needs.

Nothing here is imported by the CUDA path; the only shared input is the voxel geometry.
"""

from __future__ import annotations

from dataclasses import dataclass

import numpy as np
import scipy.sparse as sp

from . import mac


@dataclass
class Level:
    A: sp.csr_matrix
    dinv: np.ndarray              # inverse diagonal (0 where the diagonal is 0)
    P: sp.csr_matrix | None       # prolongation to this level from the next, None at the bottom
    coarse_pinv: np.ndarray | None  # dense pseudo-inverse at the coarsest level


def _inverse_diagonal(A: sp.csr_matrix) -> np.ndarray:
    dg = A.diagonal()
    return np.where(dg > 0, 1.0 / np.where(dg > 0, dg, 1.0), 0.0)


def _pinv_sym(M: np.ndarray, rtol: float = 1e-12) -> np.ndarray:
    w, V = np.linalg.eigh(M)
    keep = np.abs(w) > rtol * max(np.abs(w).max(initial=0.0), 1e-300)
    return (V[:, keep] / w[keep]) @ V[:, keep].T


def build(A: sp.spmatrix, coords: np.ndarray, min_coarse: int = 256,
          max_levels: int = 16) -> list:
    """Hierarchy for operator A whose unknown i sits at integer coordinates coords[i]
    (columns: the component first for velocity faces, then x, y, z; the component is
    never merged)."""
    A = sp.csr_matrix(A)
    c = np.asarray(coords, dtype=np.int64)
    levels = []
    while True:
        n = A.shape[0]
        if n <= min_coarse or len(levels) == max_levels - 1:
            levels.append(Level(A, _inverse_diagonal(A), None, _pinv_sym(A.toarray())))
            return levels
        key = c.copy()
        key[:, -3:] //= 2                             # x, y, z halved; a component kept
        uniq, agg = np.unique(key, axis=0, return_inverse=True)
        agg = agg.ravel()
        nc = uniq.shape[0]
        if nc >= n:                                   # no further coarsening possible
            levels.append(Level(A, _inverse_diagonal(A), None, _pinv_sym(A.toarray())))
            return levels
        P = sp.csr_matrix((np.ones(n), (np.arange(n), agg)), shape=(n, nc))
        levels.append(Level(A, _inverse_diagonal(A), P, None))
        A = (P.T @ A @ P).tocsr()
        c = uniq


def vcycle(levels: list, b: np.ndarray, omega: float = 2.0 / 3.0, nu: int = 1,
           lev: int = 0) -> np.ndarray:
    """One V-cycle for A x = b from x = 0 (the preconditioner application M^-1 b)."""
    L = levels[lev]
    if L.P is None:
        return L.coarse_pinv @ b
    x = np.zeros_like(b)
    for _ in range(nu):                               # pre-smoothing
        x += omega * L.dinv * (b - L.A @ x)
    r = b - L.A @ x
    x += L.P @ vcycle(levels, L.P.T @ r, omega, nu, lev + 1)
    for _ in range(nu):                               # post-smoothing (adjoint order)
        x += omega * L.dinv * (b - L.A @ x)
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
