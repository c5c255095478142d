"""Helpers for the GPU parity tests: move oracle vectors to and from the library's
dense device layouts (face space [d][stride], cell space [n_cells])."""

import numpy as np
import torch

from oracle import mac


def face_dense_to_device(geo_gpu, dense):
    """numpy [d, *shape] -> flat float64 CUDA tensor [d * stride]."""
    d, s, n = geo_gpu.ndim, geo_gpu.face_stride, geo_gpu.n_cells
    out = torch.zeros(d * s, dtype=torch.float64, device="cuda")
    out.view(d, s)[:, :n] = torch.from_numpy(np.ascontiguousarray(dense).reshape(d, n)).cuda()
    return out


def face_device_to_dense(geo_gpu, t):
    return geo_gpu.faces_to_grid(t).cpu().numpy()


def cell_dense_to_device(dense):
    return torch.from_numpy(np.ascontiguousarray(dense, dtype=np.float64).ravel()).cuda()


def face_compact_to_device(geo_gpu, geo, u):
    return face_dense_to_device(geo_gpu, mac.scatter_u(geo, u))


def face_device_to_compact(geo_gpu, geo, t):
    return mac.gather_u(geo, face_device_to_dense(geo_gpu, t))


def cell_device_to_compact(geo, t):
    return mac.gather_p(geo, t.cpu().numpy().reshape(geo.mask.shape))


def cell_compact_to_device(geo, p):
    return cell_dense_to_device(mac.scatter_p(geo, p))


def component_mean_free(geo, p):
    """Remove the mean of p on every connected fluid component (connectivity through
    unknown faces): the nullspace of S and of B^T."""
    import scipy.sparse as sp
    from scipy.sparse.csgraph import connected_components
    G = mac.assemble_grad(geo)
    adj = (abs(G).T @ abs(G)).tocsr()
    n, lab = connected_components(adj, directed=False)
    out = p.copy()
    for k in range(n):
        sel = lab == k
        out[sel] -= out[sel].mean()
    return out


def check_velocity(prob, geo, force, u, u_ref, rtol=1e-9):
    """Velocity parity: relative L2 within rtol of ||u_ref||.  Where the force is
    balanced by pressure (u_ref ~ 0, e.g. the force across a channel) the relative error
    is undefined, and the scale is the unconstrained flow ||A^-1 f|| instead."""
    n_ref = np.linalg.norm(u_ref)
    u_f = prob.solve_A(mac.force(geo, force), 1e-12, 20000).x
    scale = n_ref if n_ref > 1e-6 * np.linalg.norm(u_f) else np.linalg.norm(u_f)
    assert np.linalg.norm(u - u_ref) <= rtol * scale


def smallest_schur_eigenvalue(mask, periodic, force, tol):
    """Smallest non-zero eigenvalue of S seen by g, as the Lanczos estimate from the
    oracle's CG-Uzawa run (Section 4.2's estimate from the CG coefficients): the Ritz
    value lo >= the smallest eigenvalue of S with a component in g, the only ones that
    CG's error can contain."""
    from oracle import krylov, stokes
    out = stokes.solve(mask, force, stokes.Options(precond=stokes.UZAWA, tol=tol), periodic)
    lo, _, _ = krylov.lanczos_cond(out["schur"].alphas, out["schur"].betas)
    return lo


def check_pressure(geo, p, p_ref, g, tol, lam_min):
    """Element-wise pressure parity modulo the nullspace (one constant per connected
    fluid component).  Both iterates stop with ||g - S p|| <= tol ||g||, so
    ||S (p - p_ref)|| <= 2 tol ||g||, and with e the component-mean-free part of
    p - p_ref, ||e||_inf <= ||e||_2 <= 2 tol ||g|| / lambda_min(S) (lambda_max(S) = 1,
    so 1 / lambda_min is cond(S)).  A factor 2 covers the inexact inner solves and a
    Ritz value slightly above the true lambda_min."""
    e = component_mean_free(geo, p - p_ref)
    bound = 4.0 * tol * np.linalg.norm(g) / lam_min
    assert np.max(np.abs(e)) <= bound, (np.max(np.abs(e)), bound)
