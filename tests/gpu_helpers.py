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
