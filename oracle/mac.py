"""MAC (fully staggered) discretisation of the no-slip Stokes operator on a voxel image.

Section 2.1: the image is an n_x x n_y (x n_z) array of voxels of side h, each fully
fluid or fully solid; pressure lives at voxel centres, the velocity component u_a on
the voxel faces normal to axis a.  Eq. interior_boundary: the no-slip wall is the
fluid/solid interface, where u = 0 (eq. stokes_bc_noslip).  Section 2.2: the box is
periodic along every axis flagged periodic; along an axis that is not, the exterior is
treated as solid.

Conventions (the paper does not fix them):

* ``mask`` is C-ordered, ``[z][y][x]`` in 3D and ``[y][x]`` in 2D, 1 = fluid.
* Physical axis a = 0, 1, 2 is x, y, z; it is array axis ``d - 1 - a``.
* Face (a, c) is the lower face of cell c along axis a, shared by the cells c - e_a and
  c.  It is an *unknown* when both cells are fluid, a *wall* face (u = 0 at distance h
  from its neighbours) when exactly one is, and *solid-solid* when neither is.
* The vector Laplacian A = -Delta_h acts on the unknown faces.  For an unknown face f
  and each of its 2d neighbours of the same component (+-e_b, b = 0..d-1):
  an unknown neighbour adds h^-2 (u_f - u_nb); a wall neighbour adds h^-2 u_f (u_nb = 0);
  a solid-solid neighbour (only possible for b != a) sits behind a wall half a cell
  away and takes the ghost value -u_f, adding 2 h^-2 u_f.  Hence
  diag(A)_f = h^-2 (2d + g_f), g_f = number of solid-solid neighbours, and -h^-2 per
  unknown neighbour.
* B = -div_h:  (B u)_c = -h^-1 sum_a (u_(a, c+e_a) - u_(a, c)) over fluid cells c.
  B^T = grad_h: (B^T p)_(a, c) = h^-1 (p_c - p_(c - e_a)) over unknown faces (eq.
  coupled_matrix: the gradient is the adjoint of the negative divergence).
* Face flag byte: bit 0 = unknown, bits 1..3 = g_f; 0 for faces that are not unknown.
"""

from __future__ import annotations

from dataclasses import dataclass

import numpy as np
import scipy.sparse as sp

UNKNOWN_BIT = 1


def _arr_axis(a: int, d: int) -> int:
    return d - 1 - a


def shifted(arr: np.ndarray, a: int, s: int, periodic: bool, fill):
    """Return ``out`` with ``out[c] = arr[c + s e_a]``; outside a non-periodic box the
    value is ``fill``."""
    d = arr.ndim
    ax = _arr_axis(a, d)
    out = np.roll(arr, -s, axis=ax)
    if not periodic:
        n = arr.shape[ax]
        sl = [slice(None)] * d
        if s > 0:
            sl[ax] = slice(max(n - s, 0), n)
        else:
            sl[ax] = slice(0, min(-s, n))
        out[tuple(sl)] = fill
    return out


@dataclass
class Geometry:
    """Face classification of a voxel image (all arrays have the mask's shape)."""

    mask: np.ndarray          # uint8, 1 = fluid
    periodic: tuple           # per physical axis
    d: int
    h: float
    fluid: np.ndarray         # bool
    unknown: list             # per axis a: bool, face (a, c) is an unknown
    wall: list                # per axis a: bool, exactly one adjacent cell fluid
    solid_solid: list         # per axis a: bool, both adjacent cells solid
    ghosts: list              # per axis a: int8, solid-solid neighbours of an unknown face
    uidx: list                # per axis a: int64 unknown number or -1
    pidx: np.ndarray          # int64 fluid-cell number or -1
    n_u: int
    n_p: int


def classify(mask: np.ndarray, periodic=None) -> Geometry:
    """Sort every face into unknown / wall / solid-solid and count ghost neighbours.

    ``h = 1 / n_x``: the box has unit length (Section 2.3 takes L = 1), and every axis
    has the same voxel size, so the grid must be cubic in voxel size; boxes that are
    not cubes keep h from the x extent.
    """
    mask = np.ascontiguousarray(mask, dtype=np.uint8)
    d = mask.ndim
    if d not in (2, 3):
        raise ValueError("mask must be 2D or 3D")
    if np.any(mask > 1):
        raise ValueError("mask values must be 0 or 1")
    if min(mask.shape) < 2:
        raise ValueError("every axis needs at least 2 voxels")
    if periodic is None:
        periodic = (True,) * d
    periodic = tuple(bool(p) for p in periodic)[:d]
    n_x = mask.shape[_arr_axis(0, d)]
    h = 1.0 / n_x
    fluid = mask.astype(bool)
    unknown, wall, ss = [], [], []
    for a in range(d):
        lower = shifted(fluid, a, -1, periodic[a], False)   # fluid(c - e_a)
        unknown.append(fluid & lower)
        wall.append(fluid ^ lower)
        ss.append(~fluid & ~lower)
    ghosts = []
    for a in range(d):
        g = np.zeros(mask.shape, dtype=np.int8)
        for b in range(d):
            if b == a:
                continue
            for s in (-1, +1):
                # neighbour face (a, c + s e_b); outside a closed box both cells are solid
                g += shifted(ss[a], b, s, periodic[b], True).astype(np.int8)
        g[~unknown[a]] = 0
        ghosts.append(g)
    uidx, start = [], 0
    for a in range(d):
        idx = np.full(mask.shape, -1, dtype=np.int64)
        cnt = int(unknown[a].sum())
        idx[unknown[a]] = np.arange(start, start + cnt)
        uidx.append(idx)
        start += cnt
    pidx = np.full(mask.shape, -1, dtype=np.int64)
    n_p = int(fluid.sum())
    pidx[fluid] = np.arange(n_p)
    return Geometry(mask, periodic, d, h, fluid, unknown, wall, ss, ghosts, uidx, pidx,
                    start, n_p)


def face_flags(geo: Geometry) -> np.ndarray:
    """Flag bytes, shape ``(d,) + mask.shape``: bit 0 unknown, bits 1..3 ghost count."""
    out = np.zeros((geo.d,) + geo.mask.shape, dtype=np.uint8)
    for a in range(geo.d):
        f = geo.unknown[a].astype(np.uint8) | (geo.ghosts[a].astype(np.uint8) << 1)
        f[~geo.unknown[a]] = 0
        out[a] = f
    return out


def assemble_A(geo: Geometry) -> sp.csr_matrix:
    """Sparse no-slip vector Laplacian on the unknown faces (size n_u x n_u)."""
    d, h2inv = geo.d, 1.0 / (geo.h * geo.h)
    rows, cols, vals = [], [], []
    for a in range(d):
        sel = geo.unknown[a]
        me = geo.uidx[a][sel]
        rows.append(me)
        cols.append(me)
        vals.append((2 * d + geo.ghosts[a][sel].astype(np.float64)) * h2inv)
        for b in range(d):
            for s in (-1, +1):
                nb = shifted(geo.uidx[a], b, s, geo.periodic[b], -1)[sel]
                keep = nb >= 0
                rows.append(me[keep])
                cols.append(nb[keep])
                vals.append(np.full(int(keep.sum()), -h2inv))
    A = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                      shape=(geo.n_u, geo.n_u))
    return A.tocsr()


def diag_A(geo: Geometry) -> np.ndarray:
    """diag(A) = h^-2 (2d + g_f) on the unknown faces (the SIMPLE A-hat of eq.
    schur_uzawa_prec and the Jacobi preconditioner of the inner A solves)."""
    out = np.empty(geo.n_u)
    for a in range(geo.d):
        sel = geo.unknown[a]
        out[geo.uidx[a][sel]] = (2 * geo.d + geo.ghosts[a][sel].astype(np.float64)) / geo.h**2
    return out


def assemble_B(geo: Geometry) -> sp.csr_matrix:
    """Negative divergence, fluid cells x unknown faces.

    Unknown face (a, c) is the lower face of cell c (entry +1/h in row c) and the upper
    face of cell c - e_a (entry -1/h in that row)."""
    rows, cols, vals = [], [], []
    hinv = 1.0 / geo.h
    for a in range(geo.d):
        sel = geo.unknown[a]
        col = geo.uidx[a][sel]
        upper_cell = geo.pidx[sel]
        lower_cell = shifted(geo.pidx, a, -1, geo.periodic[a], -1)[sel]
        rows += [upper_cell, lower_cell]
        cols += [col, col]
        vals += [np.full(col.size, hinv), np.full(col.size, -hinv)]
    B = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                      shape=(geo.n_p, geo.n_u))
    return B.tocsr()


def assemble_grad(geo: Geometry) -> sp.csr_matrix:
    """Discrete pressure gradient, unknown faces x fluid cells, built from its own
    definition (B^T p)_(a,c) = (p_c - p_(c - e_a)) / h, not by transposing B."""
    rows, cols, vals = [], [], []
    hinv = 1.0 / geo.h
    for a in range(geo.d):
        sel = geo.unknown[a]
        row = geo.uidx[a][sel]
        rows += [row, row]
        cols += [geo.pidx[sel], shifted(geo.pidx, a, -1, geo.periodic[a], -1)[sel]]
        vals += [np.full(row.size, hinv), np.full(row.size, -hinv)]
    G = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                      shape=(geo.n_u, geo.n_p))
    return G.tocsr()


def force(geo: Geometry, f) -> np.ndarray:
    """Body force on the unknown faces: f_(a,c) = f[a] (Section 2.3: a unit pressure
    drop over a unit box becomes a unit volume force along the flow axis)."""
    out = np.empty(geo.n_u)
    for a in range(geo.d):
        out[geo.uidx[a][geo.unknown[a]]] = float(f[a])
    return out


def scatter_u(geo: Geometry, u: np.ndarray) -> np.ndarray:
    """Compact face vector -> dense ``(d,) + mask.shape`` array, 0 off the unknowns."""
    out = np.zeros((geo.d,) + geo.mask.shape)
    for a in range(geo.d):
        sel = geo.unknown[a]
        out[a][sel] = u[geo.uidx[a][sel]]
    return out


def gather_u(geo: Geometry, dense: np.ndarray) -> np.ndarray:
    out = np.empty(geo.n_u)
    for a in range(geo.d):
        sel = geo.unknown[a]
        out[geo.uidx[a][sel]] = dense[a][sel]
    return out


def scatter_p(geo: Geometry, p: np.ndarray) -> np.ndarray:
    out = np.zeros(geo.mask.shape)
    out[geo.fluid] = p[geo.pidx[geo.fluid]]
    return out


def gather_p(geo: Geometry, dense: np.ndarray) -> np.ndarray:
    out = np.empty(geo.n_p)
    out[geo.pidx[geo.fluid]] = dense[geo.fluid]
    return out
