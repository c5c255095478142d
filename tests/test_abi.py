"""CPU checks of the C ABI: the library builds, loads and exports every declared symbol,
and the ctypes structures match the C header layout.  No GPU call is made."""

import ctypes
import os
import re
import subprocess
import tempfile

import numpy as np
import pytest

from paper_2307_05266_gb300 import _build, binding

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "schur.h")


@pytest.fixture(scope="module")
def lib():
    _build.build()
    return binding.load(build_if_missing=False)


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(schur_[a-z_A-Z0-9]+)\s*\(", text)))


def test_header_declares_binding_names():
    assert declared_functions() == sorted(binding.EXPORTED)


def test_library_exports_every_declared_symbol(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_struct_layouts_match_header():
    src = r'''
#include <stdio.h>
#include <stddef.h>
#include "schur.h"
int main(void) {
  printf("%zu %zu %zu %zu %zu %zu\n", sizeof(schur_opts), sizeof(schur_stats),
         sizeof(schur_geom_info), offsetof(schur_opts, tol), offsetof(schur_stats, g_norm),
         offsetof(schur_geom_info, device_bytes));
  return 0;
}
'''
    with tempfile.TemporaryDirectory() as td:
        c = os.path.join(td, "l.c")
        exe = os.path.join(td, "l")
        open(c, "w").write(src)
        subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), c, "-o", exe])
        vals = [int(v) for v in subprocess.check_output([exe]).split()]
    got = [ctypes.sizeof(binding.Opts), ctypes.sizeof(binding.Stats),
           ctypes.sizeof(binding.GeomInfo), binding.Opts.tol.offset,
           binding.Stats.g_norm.offset, binding.GeomInfo.device_bytes.offset]
    assert vals == got


def test_defaults(lib):
    o = binding.default_opts()
    assert o.precond == binding.SIMPLE and o.stop_norm == binding.STOP_UNPRECOND
    assert o.tol == 1e-8 and o.tol_inner_A == 1e-12 and o.max_inner == 20000


def test_null_arguments_rejected_without_gpu(lib):
    out = ctypes.c_void_p()
    dims = (ctypes.c_int64 * 3)(4, 4, 4)
    per = (ctypes.c_int * 3)(1, 1, 1)
    assert lib.schur_create_geometry(None, 3, dims, per, None, ctypes.byref(out)) == binding.SCHUR_EINVAL
    m = (ctypes.c_uint8 * 64)()
    assert lib.schur_create_geometry(m, 4, dims, per, None, ctypes.byref(out)) == binding.SCHUR_EINVAL
    dims1 = (ctypes.c_int64 * 3)(1, 4, 4)
    assert lib.schur_create_geometry(m, 3, dims1, per, None, ctypes.byref(out)) == binding.SCHUR_EINVAL
    assert b"extent" in lib.schur_last_error()
    assert lib.schur_solve(None, None, None) == binding.SCHUR_EINVAL
    assert lib.schur_set_launch(None, 8, 1, 1) == binding.SCHUR_EINVAL
    lib.schur_destroy(None)


def test_footprint_bound_grows_with_size_and_precision(lib):
    fp = [binding.footprint_bytes((n, n, n)) for n in (16, 32, 64)]
    assert fp[0] < fp[1] < fp[2]
    assert binding.footprint_bytes((32, 32, 32), binding.MIXED) > fp[1]
    # an upper bound on what a 64^3 geometry can allocate: per cell at least the dense
    # FP64 outer vectors and the velocity (5 + 3 doubles) and the mask
    assert fp[2] >= 64 ** 3 * (8 * 8 + 1)


def test_server_rejects_job_larger_than_budget_without_gpu(lib):
    """Host-side admission check (no device work happens before progress())."""
    srv = binding.Server(1 << 20, max_active=2)
    with pytest.raises(binding.SchurError) as e:
        srv.submit(np.ones((64, 64, 64), np.uint8))
    assert e.value.code == binding.SCHUR_ENOMEM
    srv.close()


def test_lanczos_extremes_host_computation_matches_numpy(lib):
    """The library's Sturm-bisection eigen-solve of the CG Lanczos tridiagonal (host code,
    no GPU) against the oracle's dense eigvalsh on the same coefficients, from CG runs on
    SPD matrices and from Algorithm 1 on a small Stokes problem."""
    from oracle import krylov, stokes
    from paper_2307_05266_gb300 import synth
    rng = np.random.default_rng(3)
    for n, span in ((12, 1e2), (40, 1e5)):
        Q = np.linalg.qr(rng.standard_normal((n, n)))[0]
        A = (Q * np.geomspace(1.0, span, n)) @ Q.T
        res = krylov.pcg(lambda x: A @ x, rng.standard_normal(n), 1.0 / np.diag(A), 1e-14, 300)
        m = min(len(res.alphas), len(res.betas) + 1)
        lo, hi = binding.lanczos_extremes(res.alphas[:m], res.betas[:m - 1])
        ref = krylov.lanczos_cond(res.alphas, res.betas)
        assert lo == pytest.approx(ref[0], rel=1e-9) and hi == pytest.approx(ref[1], rel=1e-9)
    m_ = synth.square_array_2d(2, 10, 4, 2, seed=1)
    r = stokes.solve(m_, (1.0, 0.0), stokes.Options(precond=stokes.SIMPLE, tol=1e-10))
    a, b = r["schur"].alphas, r["schur"].betas
    lo, hi = binding.lanczos_extremes(a, b[:len(a) - 1])
    ref = krylov.lanczos_cond(a, b)
    assert hi / lo == pytest.approx(ref[2], rel=1e-9)
    assert binding.lanczos_extremes([2.0], [])[0] == pytest.approx(0.5)   # 1 x 1: 1/alpha
    with pytest.raises(binding.SchurError):
        binding.lanczos_extremes([1.0, -1.0], [0.5])
