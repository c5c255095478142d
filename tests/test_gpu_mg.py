"""Multigrid inner preconditioner (SCHUR_INNER_MG) against the oracle's multigrid path.

The oracle (oracle/amg.py with Options.inner_precond = INNER_AMG) states the V-cycle the
CUDA path implements: 2 x 2 x 2 aggregates, Galerkin coarse operators down to a single
cell solved exactly, omega = 0.9, over-correction gamma = 1.3 (A) / 1.7 (S-hat).  The
bars are those of the Jacobi path: outer iterations within 2, inner iterations within 2
per inner solve, u within 1e-9 of ||u_ref||, p modulo per-component constants within
4 tol ||g|| / lambda_min(S), k within 1e-8 (FP64) and 1e-6 (mixed precision).
"""

import numpy as np
import pytest
import torch

from oracle import krylov, mac, stokes
from paper_2307_05266_gb300 import binding, synth

from gpu_helpers import (cell_device_to_compact, check_pressure, check_velocity,
                         face_device_to_compact, smallest_schur_eigenvalue)

pytestmark = pytest.mark.gpu


def _rand_mask(shape, phi, seed):
    rng = np.random.default_rng(seed)
    return (rng.random(shape) < phi).astype(np.uint8)


# (mask, periodic, force, outer tol)
CASES = {
    "squares2d": (synth.square_array_2d(2, 10, 4, 2, seed=1), None, (1.0, 0.0), 1e-9),
    "rand2d_closed_y": (_rand_mask((21, 34), 0.75, 3), (True, False), (1.0, 0.0), 1e-9),
    "spheres24": (synth.sphere_packing(24, 4.0, 8.0, 0.4, seed=0), None, (1.0, 0.0, 0.0), 1e-8),
    "rand3d_ragged": (_rand_mask((13, 19, 37), 0.8, 5), (True, False, True), (0.0, 0.0, 1.0), 1e-9),
    "spheres_ragged": (synth.sphere_packing((37, 29, 23), 2.0, 4.0, 0.4, seed=3), None,
                       (0.0, 1.0, 0.0), 1e-8),
    "tight32": (synth.sphere_packing(32, 2.0, 4.0, 0.15, seed=5), None, (1.0, 0.0, 0.0), 1e-8),
}


@pytest.fixture(scope="module")
def cuda():
    assert torch.cuda.is_available()
    torch.cuda.set_device(0)
    binding.load()
    return True


def _inner_solves(outer, precond):
    """Inner A solves of a solve: g, one per outer iteration; S-hat solves: one per
    iteration and the start (SIMPLE)."""
    return outer + 1, (outer + 1 if precond == stokes.SIMPLE else 0)


@pytest.mark.parametrize("precond", [binding.UZAWA, binding.SIMPLE])
@pytest.mark.parametrize("name", list(CASES))
def test_mg_solve_matches_oracle(cuda, name, precond):
    mask, per, force, tol = CASES[name]
    ref = stokes.solve(mask, force, stokes.Options(precond=precond, tol=tol,
                                                   inner_precond=stokes.INNER_AMG), per)
    rs = ref["schur"]
    prob = ref["problem"]
    geo = prob.geo
    with binding.Geometry(mask, per) as g:
        g.set_force(force)
        st = g.solve(precond=precond, tol=tol, inner_precond=binding.INNER_MG)
        rec = g.recover_velocity()
        assert st.status == binding.SCHUR_OK and rs.status == krylov.OK
        assert abs(st.outer_iters - rs.outer_iters) <= 2
        nA, nS = _inner_solves(max(st.outer_iters, rs.outer_iters), precond)
        assert abs(st.inner_iters_A - rs.inner_iters_A) <= 2 * nA
        assert abs(st.inner_iters_S - rs.inner_iters_S) <= 2 * nS
        assert abs(rec.inner_iters_A - ref["recovery"].iters) <= 2
        u = face_device_to_compact(g, geo, g.field(binding.FIELD_U))
        p = cell_device_to_compact(geo, g.field(binding.FIELD_P))
        check_velocity(prob, geo, force, u, ref["u"])
        if np.linalg.norm(ref["g"]) > 0 and st.outer_iters > 0:
            check_pressure(geo, p, ref["p"], ref["g"], tol,
                           smallest_schur_eigenvalue(mask, per, force, tol))
        for a in range(geo.d):
            k = g.permeability(a)
            assert abs(k - ref["k"][a]) <= 1e-8 * abs(ref["k"][a]) + 1e-9 * geo.h ** 2


@pytest.mark.parametrize("precond", [binding.UZAWA, binding.SIMPLE])
def test_mg_needs_fewer_inner_iterations_than_jacobi(cuda, precond):
    """The point of the multigrid: the same k with several times fewer inner iterations."""
    mask, per, force, tol = CASES["spheres24"]
    with binding.Geometry(mask, per) as g:
        g.set_force(force)
        sj = g.solve(precond=precond, tol=tol)
        g.recover_velocity()
        kj = g.permeability(0)
        sm = g.solve(precond=precond, tol=tol, inner_precond=binding.INNER_MG)
        g.recover_velocity()
        km = g.permeability(0)
    assert abs(km - kj) <= 1e-8 * abs(kj)
    assert 2 * sm.inner_iters_A < sj.inner_iters_A
    if precond == binding.SIMPLE:
        assert 3 * sm.inner_iters_S < sj.inner_iters_S


@pytest.mark.parametrize("precond", [binding.UZAWA, binding.SIMPLE])
@pytest.mark.parametrize("name", ["spheres24", "rand3d_ragged", "tight32", "squares2d"])
def test_mg_mixed_precision_against_fp64_oracle(cuda, name, precond):
    """FP32 multigrid inner solves inside the FP64 flexible outer CG and defect correction:
    k within 1e-6 of the FP64 oracle."""
    mask, per, force, tol = CASES[name]
    ref = stokes.solve(mask, force, stokes.Options(precond=precond, tol=tol), per)
    geo = ref["problem"].geo
    with binding.Geometry(mask, per) as g:
        g.set_force(force)
        st = g.solve(precond=precond, precision=binding.MIXED, tol=tol,
                     inner_precond=binding.INNER_MG)
        assert st.status == binding.SCHUR_OK and st.rel_res < tol
        assert st.inner_iters_A_f32 > 0
        g.recover_velocity()
        for a in range(geo.d):
            assert abs(g.permeability(a) - ref["k"][a]) <= 1e-6 * abs(ref["k"][a]) + 1e-9 * geo.h ** 2


def test_mg_and_jacobi_graphs_alternate_on_one_handle(cuda):
    """Switching the inner preconditioner rebuilds the recorded graphs; results repeat
    bitwise for equal options."""
    mask, per, force, tol = CASES["spheres_ragged"]
    out = []
    with binding.Geometry(mask, per) as g:
        g.set_force(force)
        for ip in (binding.INNER_MG, binding.INNER_JACOBI, binding.INNER_MG):
            st = g.solve(precond=binding.SIMPLE, tol=tol, inner_precond=ip)
            g.recover_velocity()
            out.append((st.outer_iters, st.inner_iters_S, g.permeability(1)))
    assert out[0] == out[2]
    assert abs(out[1][2] - out[0][2]) <= 1e-8 * abs(out[0][2])
    assert out[1][1] > out[0][1]


def test_mg_edge_cases(cuda):
    # one fluid voxel (a single-entry hierarchy) and an all-solid box
    m = np.zeros((4, 4, 4), np.uint8)
    m[0, 0, 0] = 1
    with binding.Geometry(m) as g:
        st = g.solve(precond=binding.SIMPLE, inner_precond=binding.INNER_MG)
        g.recover_velocity()
        assert g.permeability(0) == 0.0
    with binding.Geometry(np.zeros((6, 5, 4), np.uint8)) as g:
        st = g.solve(inner_precond=binding.INNER_MG)
        assert st.zero_rhs == 1
    # the x-invariant channel: g = 0, u from one multigrid A solve = the closed form
    with binding.Geometry(synth.channel_2d(32)) as g:
        st = g.solve(precond=binding.UZAWA, tol=1e-10, inner_precond=binding.INNER_MG)
        assert st.outer_iters == 0 and st.zero_rhs == 1
        g.recover_velocity()
        assert abs(g.permeability(0) - 2255 / 32768) <= 1e-12 * 2255 / 32768


def test_mg_field_parity_64(cuda):
    """64^3 packing (radii U[3, 6), porosity 0.40, seed 11; 272,467 unknown faces, 97 fluid
    components; flow along y): the fine levels of both hierarchies take several grid-stride
    steps per thread, the coarse levels run on the grid and in the shared-memory tail.
    FP64 SIMPLE with multigrid inner solves against the oracle's multigrid path: outer
    iterations within 2, inner within 2 per inner solve, u within 1e-9 of ||u_ref||, k within
    1e-8."""
    mask = synth.sphere_packing(64, 3.0, 6.0, 0.40, 11)
    f = (0.0, 1.0, 0.0)
    tol = 1e-9
    ref = stokes.solve(mask, f, stokes.Options(precond=stokes.SIMPLE, tol=tol,
                                               inner_precond=stokes.INNER_AMG))
    rs, prob = ref["schur"], ref["problem"]
    geo = prob.geo
    with binding.Geometry(mask) as g:
        g.set_force(f)
        st = g.solve(precond=binding.SIMPLE, tol=tol, inner_precond=binding.INNER_MG)
        rec = g.recover_velocity()
        levels_A, tail_A = g.mg_levels(False)
        assert levels_A[0] == geo.n_u and tail_A > 1 and len(levels_A) >= 6
        assert st.status == binding.SCHUR_OK
        assert abs(st.outer_iters - rs.outer_iters) <= 2
        nA, nS = _inner_solves(max(st.outer_iters, rs.outer_iters), stokes.SIMPLE)
        assert abs(st.inner_iters_A - rs.inner_iters_A) <= 2 * nA
        assert abs(st.inner_iters_S - rs.inner_iters_S) <= 2 * nS
        assert abs(rec.inner_iters_A - ref["recovery"].iters) <= 2
        u = face_device_to_compact(g, geo, g.field(binding.FIELD_U))
        check_velocity(prob, geo, f, u, ref["u"])
        for a in range(3):
            assert abs(g.permeability(a) - ref["k"][a]) <= 1e-8 * abs(ref["k"][1])
