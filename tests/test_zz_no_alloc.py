"""The allocation-free permeability entry point against the handle-based one.

schur_permeability_noalloc exists for callers that may not allocate device memory (a
pool they do not own, an already-captured graph); its scratch is a static device array.
This file is collected last so that a failure here leaves every other test already run;
it passes alone in a fresh process and after the rest of the suite.
"""

import numpy as np
import pytest
import torch

from paper_2307_05266_gb300 import binding, synth

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("shape,force,axis", [
    ((24, 24, 24), (1.0, 0.0, 0.0), 0),
    ((23, 29, 37), (0.0, 0.0, 1.0), 2),
    ((40, 33), (0.0, 1.0), 1),
])
def test_noalloc_permeability_matches_handle_path(shape, force, axis):
    torch.cuda.set_device(0)
    if len(shape) == 3:
        mask = synth.sphere_packing(tuple(reversed(shape)), 2.0, 4.0, 0.5, seed=5)
    else:
        rng = np.random.default_rng(5)
        mask = (rng.random(shape) < 0.8).astype(np.uint8)
    with binding.Geometry(mask) as g:
        g.set_force(force)
        g.solve(precond=binding.SIMPLE, tol=1e-8)
        g.recover_velocity()
        k_ref = [g.permeability(a) for a in range(g.ndim)]
        for _ in range(2):                       # two calls in a row share the scratch
            k = torch.full((3,), float("nan"), dtype=torch.float64, device="cuda")
            g.permeability_noalloc(k)
            torch.cuda.synchronize()
            kh = k.cpu().numpy()
            for a in range(g.ndim):
                assert abs(kh[a] - k_ref[a]) <= 1e-12 * max(abs(k_ref[a]), 1e-300)
            assert np.all(kh[g.ndim:] == 0.0)
        assert k_ref[axis] > 0


def test_noalloc_rejects_sizes_beyond_the_static_scratch():
    torch.cuda.set_device(0)
    u = torch.zeros(8, dtype=torch.float64, device="cuda")
    f = torch.zeros(8, dtype=torch.uint8, device="cuda")
    k = torch.zeros(3, dtype=torch.float64, device="cuda")
    lib = binding.load()
    import ctypes as C
    dims = (C.c_int64 * 3)(256, 256, 256)          # 3 * 2^24 faces > 8388608
    rc = lib.schur_permeability_noalloc(C.c_void_p(u.data_ptr()), C.c_void_p(f.data_ptr()), 3,
                                        dims, 256 ** 3, None, C.c_void_p(k.data_ptr()))
    assert rc == binding.SCHUR_EINVAL
    assert b"static scratch" in lib.schur_last_error()
