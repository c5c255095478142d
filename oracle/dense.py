"""Dense Schur complements for tiny grids (spectra, condition numbers, exact solutions).

S = B A^+ B^T (eq. schur_rhs); A^+ is the inverse when A is nonsingular and the
eigen-pseudo-inverse otherwise (the empty periodic box, where constant velocities are
in the kernel of A).  S and S-hat_simple are singular (constant pressure per connected
fluid component, the Remark after Algorithm 1), so condition numbers are effective:
largest over smallest nonzero eigenvalue.  The minimum-norm solution of S p = g is
formed by projection on the eigenvectors with nonzero eigenvalue.
"""

from __future__ import annotations

import numpy as np
import scipy.linalg as sla

from .stokes import StokesProblem


def pinv_sym(M: np.ndarray, rtol: float = 1e-10) -> np.ndarray:
    w, V = np.linalg.eigh(M)
    keep = np.abs(w) > rtol * np.max(np.abs(w))
    return (V[:, keep] / w[keep]) @ V[:, keep].T


def schur_dense(prob: StokesProblem) -> np.ndarray:
    A = prob.A.toarray()
    B = prob.B.toarray()
    w = np.linalg.eigvalsh(A)
    if w[0] > 1e-10 * w[-1]:
        X = np.linalg.solve(A, B.T)
    else:
        X = pinv_sym(A) @ B.T
    S = B @ X
    return 0.5 * (S + S.T)


def simple_dense(prob: StokesProblem) -> np.ndarray:
    return prob.S_simple.toarray()


def spectrum(prob: StokesProblem) -> np.ndarray:
    return np.linalg.eigvalsh(schur_dense(prob))


def effective_cond(w: np.ndarray, rtol: float = 1e-9) -> float:
    w = np.sort(np.abs(w))
    nz = w[w > rtol * w[-1]]
    return float(nz[-1] / nz[0])


def preconditioned_spectrum(prob: StokesProblem) -> np.ndarray:
    """Nonzero eigenvalues of S-hat_simple^+ S: the generalised problem S v = lam S-hat v
    restricted to the complement of the common nullspace."""
    S = schur_dense(prob)
    P = simple_dense(prob)
    wp, V = np.linalg.eigh(P)
    keep = wp > 1e-10 * wp[-1]
    Vr = V[:, keep]
    Sr = Vr.T @ S @ Vr
    Pr = Vr.T @ P @ Vr
    return sla.eigh(Sr, Pr, eigvals_only=True)


def min_norm_solution(S: np.ndarray, g: np.ndarray, rtol: float = 1e-10) -> np.ndarray:
    w, V = np.linalg.eigh(S)
    keep = w > rtol * w[-1]
    c = V[:, keep].T @ g
    return V[:, keep] @ (c / w[keep])
