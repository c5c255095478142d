"""The whole Pressure Schur Complement path in FP64 on assembled sparse matrices.

Steps (Section 1, eqs. schur_system, schur_rhs, velocity_schur; Section 2.3):

1. g = B A^-1 f                      (inner PCG on A, eps_A)
2. S p = g by Algorithm 1 with S-hat = I (Uzawa) or S-hat = B diag(A)^-1 B^T (SIMPLE,
   eq. schur_uzawa_prec), each S application running an inner PCG on A and each SIMPLE
   application an inner PCG on S-hat followed by removal of the fluid-cell mean.
3. A u = f - B^T p                   (inner PCG on A)
4. k = <u_axis> = (1/|Omega|) * integral of u_axis over the fluid, i.e. the sum of the
   axis component over the unknown faces divided by the number of voxels (eq.
   darcy_law with mu = 1, L = 1 and a unit force along the axis).

Defaults follow the readings of the paper that the tests use: Jacobi inner
preconditioners, zero initial guesses, eps_A = eps_S-hat = 1e-12.  ``inner_precond =
INNER_AMG`` replaces Jacobi in both inner solves by the aggregation multigrid of
``oracle.amg`` (the paper uses BoomerAMG there, Section 3.2).
"""

from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from . import amg, krylov, mac

UZAWA, SIMPLE = 0, 1
INNER_JACOBI, INNER_AMG = 0, 1
ZERO_RHS_RTOL = 1e-12


@dataclass
class Options:
    precond: int = SIMPLE
    stop_norm: int = krylov.STOP_UNPRECOND
    tol: float = 1e-8
    tol_inner_A: float = 1e-12
    tol_inner_S: float = 1e-12
    max_outer: int = 2000
    max_inner: int = 20000
    inner_precond: int = INNER_JACOBI


class StokesProblem:
    """Assembled operators of one geometry."""

    def __init__(self, mask, periodic=None):
        self.geo = mac.classify(mask, periodic)
        self.A = mac.assemble_A(self.geo)
        self.B = mac.assemble_B(self.geo)
        self.BT = mac.assemble_grad(self.geo)
        self.dA = mac.diag_A(self.geo)
        # S-hat_simple = B diag(A)^-1 B^T (eq. schur_uzawa_prec), a sparse product
        self.S_simple = (self.B @ (self.BT.multiply(1.0 / self.dA[:, None]))).tocsr()
        self.dS = self.S_simple.diagonal()
        self.n_comp, self.comp = fluid_components(self.geo)
        self.comp_size = np.bincount(self.comp, minlength=self.n_comp).astype(np.float64)
        self._amg = {}                          # multigrid hierarchies, built on first use

    def amg_levels(self, which: str):
        """Aggregation-multigrid hierarchy of A ("A") or S-hat_simple ("S")."""
        if which not in self._amg:
            if which == "A":
                self._amg[which] = amg.build(self.A, amg.face_coords(self.geo))
            else:
                self._amg[which] = amg.build(self.S_simple, amg.cell_coords(self.geo))
        return self._amg[which]

    # ---- single operators -------------------------------------------------------
    def solve_A(self, v, tol, max_iter, inner=INNER_JACOBI):
        if inner == INNER_AMG:
            levels = self.amg_levels("A")
            return krylov.pcg(lambda x: self.A @ x, v,
                              lambda r: amg.vcycle(levels, r, amg.GAMMA_A), tol, max_iter)
        return krylov.pcg(lambda x: self.A @ x, v, 1.0 / self.dA, tol, max_iter)

    def remove_mean(self, p):
        """Subtract from p its mean on every connected fluid component: the projection
        onto the range of S-hat_simple (and of S), whose nullspace holds the constants
        of each component (Section 3.1, Remark on the constant nullspace)."""
        if not p.size:
            return p
        mean = np.bincount(self.comp, weights=p, minlength=self.n_comp) / self.comp_size
        return p - mean[self.comp]

    def solve_simple(self, r, tol, max_iter, inner=INNER_JACOBI):
        """z = S-hat_simple^+ r.  The "special care" of Section 3.2 for the singular
        pressure operator, read as: the right-hand side is projected onto the range first
        (rounding leaves it a component along the constants that grows relative to r as
        the outer residual shrinks, and CG on an inconsistent system does not converge),
        and the returned solution is projected as well."""
        if inner == INNER_AMG:
            # The cycle's output is not projected: r stays in the range of S-hat (r = b -
            # S-hat x with b in the range), so a nullspace part of z = M^-1 r changes
            # neither r.z nor S-hat d; it enters only the stop norm ||z||, and the
            # returned solution is projected.
            levels = self.amg_levels("S")
            minv = lambda v: amg.vcycle(levels, v, amg.GAMMA_S)  # noqa: E731
        else:
            minv = np.where(self.dS > 0, 1.0 / np.where(self.dS > 0, self.dS, 1.0), 0.0)
        return krylov.pcg(lambda x: self.S_simple @ x, self.remove_mean(r), minv, tol,
                          max_iter, project=self.remove_mean)

    def apply_S(self, d, tol_A, max_inner, inner=INNER_JACOBI):
        res = self.solve_A(self.BT @ d, tol_A, max_inner, inner)
        return self.B @ res.x, res.iters

    # ---- the path ---------------------------------------------------------------
    def rhs(self, f, opts: Options):
        """g = B A^-1 f, its inner iterations, and whether g vanishes to rounding.

        g counts as zero when ||g|| <= ZERO_RHS_RTOL * || |B| |u| ||: the divergence of
        a flow that is exactly divergence-free (e.g. the x-invariant channel flow) is
        rounding noise, and Algorithm 1 started on noise has nothing to converge to.
        """
        res = self.solve_A(mac.force(self.geo, f), opts.tol_inner_A, opts.max_inner,
                           opts.inner_precond)
        g = self.B @ res.x
        scale = float(np.linalg.norm(abs(self.B) @ np.abs(res.x)))
        zero = float(np.linalg.norm(g)) <= ZERO_RHS_RTOL * scale
        return g, res.iters, zero

    def solve(self, f, opts: Options = None):
        opts = opts or Options()
        g, it_g, zero = self.rhs(f, opts)
        if zero:
            out = krylov.schur_pcg(None, np.zeros_like(g), None, opts.tol, 0, opts.stop_norm)
            out.inner_iters_A = it_g
            return out, g

        def apply_S(d):
            return self.apply_S(d, opts.tol_inner_A, opts.max_inner, opts.inner_precond)

        if opts.precond == UZAWA:
            def precond(r):
                return r.copy(), 0
        else:
            def precond(r):
                r[:] = self.remove_mean(r)      # the outer residual is projected in place
                res = self.solve_simple(r, opts.tol_inner_S, opts.max_inner,
                                        opts.inner_precond)
                return res.x, res.iters

        out = krylov.schur_pcg(apply_S, g, precond, opts.tol, opts.max_outer,
                               opts.stop_norm)
        out.inner_iters_A += it_g
        return out, g

    def recover_velocity(self, f, p, opts: Options = None):
        opts = opts or Options()
        rhs = mac.force(self.geo, f) - self.BT @ p
        return self.solve_A(rhs, opts.tol_inner_A, opts.max_inner, opts.inner_precond)

    def permeability(self, u, axis: int) -> float:
        g = self.geo
        return float(u[g.uidx[axis][g.unknown[axis]]].sum()) / g.mask.size


def solve(mask, f, opts: Options = None, periodic=None):
    """Convenience: full path, returns a dict with p, u (compact), k per axis, stats."""
    prob = StokesProblem(mask, periodic)
    opts = opts or Options()
    out, g = prob.solve(f, opts)
    rec = prob.recover_velocity(f, out.p, opts)
    k = [prob.permeability(rec.x, a) for a in range(prob.geo.d)]
    return dict(problem=prob, p=out.p, u=rec.x, g=g, k=k, schur=out, recovery=rec)


def fluid_components(geo):
    """Connected components of the fluid cells, two cells being connected when the face
    between them is an unknown (periodic axes wrap).  Returns (count, label per fluid
    cell in pidx order); labels are numbered by the smallest cell index they contain."""
    from scipy.sparse.csgraph import connected_components
    G = mac.assemble_grad(geo)              # one row per unknown face: its two cells
    adj = (abs(G).T @ abs(G)).tocsr()
    n, lab = connected_components(adj, directed=False)
    first = np.full(n, geo.n_p, dtype=np.int64)
    np.minimum.at(first, lab, np.arange(geo.n_p))
    order = np.argsort(first, kind="stable")
    rank = np.empty(n, dtype=np.int64)
    rank[order] = np.arange(n)
    return n, rank[lab]


# ---- geometry statistics (Section 4.1.1) -----------------------------------------
def porosity(mask) -> float:
    """phi = V_f / V (eq. porosity, as a fraction)."""
    m = np.asarray(mask)
    return float(np.count_nonzero(m)) / m.size


def surface_area(mask, periodic=None) -> int:
    """V_surf: solid voxels sharing a face with a fluid voxel (eq. surface_area)."""
    m = np.asarray(mask).astype(bool)
    d = m.ndim
    periodic = (True,) * d if periodic is None else tuple(periodic)
    touch = np.zeros_like(m)
    for a in range(d):
        for s in (-1, 1):
            touch |= mac.shifted(m, a, s, periodic[a], False)
    return int(np.count_nonzero(~m & touch))


def surface_to_volume(mask, periodic=None) -> float:
    """sigma_s = V_surf / V_f (eq. s-t-v-ration, as a fraction)."""
    return surface_area(mask, periodic) / float(np.count_nonzero(mask))
