"""Krylov methods of Section 3, written out step by step in FP64.

* ``pcg``         preconditioned CG (Saad, Iterative Methods, Alg. 9.1) with the
                  paper's inner stopping rule: stop at the first k with
                  ||M^-1 r_k|| / ||M^-1 r_0|| < eps  (Section 3.2, the relative
                  preconditioned residual for A and for S-hat_simple).  M is a
                  diagonal (Jacobi) matrix here; the paper uses BoomerAMG.
* ``schur_pcg``   Algorithm 1, the outer preconditioned CG on S p = g, with the sign of
                  the residual fixed (r = g - S p, p += alpha d, r -= alpha q: the
                  printed r^0 = S p^0 - g together with r += alpha q is not a descent
                  iteration) and two stopping rules: the preconditioned ||z_k||/||z_0||
                  of Algorithm 1 and the unpreconditioned ||r_k||/||r_0|| used for the
                  2D study (Section 4.2.2).

* ``lanczos_tridiagonal`` / ``lanczos_cond``  the condition-number estimate the paper
                  computes "for free" from the outer CG coefficients (Section 4.2,
                  Table 2): the Lanczos tridiagonal matrix that CG builds implicitly
                  (Saad, Iterative Methods, Section 6.7.3) and its extreme eigenvalues.

Iteration counts are the number of operator applications inside the loop.  A zero
right-hand side returns the zero vector after 0 iterations.
"""

from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

OK, NOT_CONVERGED, BREAKDOWN = 0, 1, 2
STOP_UNPRECOND, STOP_PRECOND = 0, 1


@dataclass
class CGResult:
    x: np.ndarray
    iters: int
    status: int
    rel: float                      # final ||M^-1 r|| / ||M^-1 r_0||
    alphas: list = field(default_factory=list)
    betas: list = field(default_factory=list)


def pcg(apply, b: np.ndarray, minv: np.ndarray, tol: float, max_iter: int,
        project=None) -> CGResult:
    """Preconditioned CG from x_0 = 0 (Jacobi in the paper's setting).

    ``apply(v)`` returns the operator times v; ``minv`` is the inverse diagonal (Jacobi)
    or a callable returning M^-1 r for a symmetric positive definite M (the multigrid of
    ``oracle.amg``).
    ``project`` (optional) is applied to the returned solution; the SIMPLE solve uses
    it to remove the constant pressure mode (Section 3.2: the Neumann pressure
    Laplacian has the constant in its nullspace).
    """
    prec = minv if callable(minv) else (lambda v: minv * v)
    x = np.zeros_like(b)
    r = b.copy()
    z = prec(r)
    z0 = float(np.sqrt(z @ z))
    if z0 == 0.0:
        return CGResult(x, 0, OK, 0.0)
    d = z.copy()
    rho = float(r @ z)
    res = CGResult(x, 0, NOT_CONVERGED, 1.0)
    for k in range(1, max_iter + 1):
        q = apply(d)
        dq = float(d @ q)
        if not (dq > 0.0) or not np.isfinite(dq):
            res.status = BREAKDOWN
            res.iters = k
            break
        alpha = rho / dq
        x += alpha * d
        r -= alpha * q
        z = prec(r)
        rel = float(np.sqrt(z @ z)) / z0
        res.alphas.append(alpha)
        res.iters, res.rel = k, rel
        if rel < tol:
            res.status = OK
            break
        rho_new = float(r @ z)
        beta = rho_new / rho
        res.betas.append(beta)
        d = z + beta * d
        rho = rho_new
    if project is not None:
        x = project(x)
    res.x = x
    return res


@dataclass
class SchurResult:
    p: np.ndarray
    outer_iters: int
    status: int
    rel_res: float            # ||r_k|| / ||r_0||
    rel_res_precond: float    # ||z_k|| / ||z_0|| (nan when the last z was not formed)
    inner_iters_A: int
    inner_iters_S: int
    history: list             # ||r_k|| / ||r_0|| for k = 0, 1, ...
    alphas: list
    betas: list


def schur_pcg(apply_S, g: np.ndarray, precond, tol: float, max_outer: int,
              stop_norm: int = STOP_UNPRECOND) -> SchurResult:
    """Algorithm 1 (sign fixed) from p_0 = 0.

    ``apply_S(d)`` returns (S d, inner iterations spent); ``precond(r)`` returns
    (S-hat^-1 r, inner iterations spent).  Under the unpreconditioned rule the test
    follows the residual update and a converged step skips the last S-hat solve; under
    the preconditioned rule it follows the S-hat solve, as in Algorithm 1.
    """
    p = np.zeros_like(g)
    r = g.copy()
    r0 = float(np.sqrt(r @ r))
    it_A = 0
    it_S = 0
    out = SchurResult(p, 0, OK, 0.0, float("nan"), 0, 0, [1.0], [], [])
    if r0 == 0.0:
        out.history = [0.0]
        out.rel_res_precond = 0.0
        return out
    z, n_s = precond(r)
    it_S += n_s
    z0 = float(np.sqrt(z @ z))
    if z0 == 0.0:
        out.rel_res = 1.0
        out.rel_res_precond = 0.0
        out.inner_iters_S = it_S
        return out
    d = z.copy()
    rho = float(r @ z)
    out.status = NOT_CONVERGED
    rel = 1.0
    relz = 1.0
    for k in range(1, max_outer + 1):
        q, n_a = apply_S(d)
        it_A += n_a
        dq = float(d @ q)
        out.outer_iters = k
        if not (dq > 0.0) or not np.isfinite(dq):
            out.status = BREAKDOWN
            break
        alpha = rho / dq
        p += alpha * d
        r -= alpha * q
        rel = float(np.sqrt(r @ r)) / r0
        out.history.append(rel)
        out.alphas.append(alpha)
        if stop_norm == STOP_UNPRECOND and rel < tol:
            out.status = OK
            relz = float("nan")
            break
        z, n_s = precond(r)
        it_S += n_s
        relz = float(np.sqrt(z @ z)) / z0
        if stop_norm == STOP_PRECOND and relz < tol:
            out.status = OK
            break
        rho_new = float(r @ z)
        beta = rho_new / rho
        out.betas.append(beta)
        d = z + beta * d
        rho = rho_new
    out.p = p
    out.rel_res = rel
    out.rel_res_precond = relz
    out.inner_iters_A = it_A
    out.inner_iters_S = it_S
    return out


def lanczos_tridiagonal(alphas, betas) -> np.ndarray:
    """The m x m symmetric tridiagonal T_m of the Lanczos process that m steps of
    (preconditioned) CG carry out implicitly, from the step lengths alpha_j and the
    direction coefficients beta_j = rho_(j+1) / rho_j (Saad, Section 6.7.3):
    T[j, j] = 1/alpha_j + beta_(j-1)/alpha_(j-1) (no second term for j = 0) and
    T[j, j+1] = T[j+1, j] = sqrt(beta_j) / alpha_j.  Its eigenvalues (Ritz values)
    approximate those of M^-1 S from the extremes inwards."""
    a = np.asarray(alphas, dtype=np.float64)
    b = np.asarray(betas, dtype=np.float64)
    m = len(a)
    if m == 0:
        return np.zeros((0, 0))
    T = np.zeros((m, m))
    for j in range(m):
        T[j, j] = 1.0 / a[j]
        if j > 0:
            T[j, j] += b[j - 1] / a[j - 1]
        if j + 1 < m:
            off = np.sqrt(b[j]) / a[j]
            T[j, j + 1] = off
            T[j + 1, j] = off
    return T


def lanczos_cond(alphas, betas):
    """(lambda_min, lambda_max, lambda_max / lambda_min) of the Lanczos tridiagonal; a CG
    run that stopped before forming beta of its last step uses the first len(betas) + 1
    step lengths."""
    m = min(len(alphas), len(betas) + 1)
    w = np.linalg.eigvalsh(lanczos_tridiagonal(alphas[:m], betas[:m - 1]))
    return float(w[0]), float(w[-1]), float(w[-1] / w[0])
