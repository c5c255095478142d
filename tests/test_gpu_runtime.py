"""Asynchronous, batched and served execution: each result equals the same job run alone.

Kernels use a fixed grid per geometry and deterministic reductions, so a job gives the
same bits whether it runs alone, inside one batch graph with other geometries, or
interleaved with other requests in the server (the stated tolerance is 1e-6 in k for
the mixed-precision path; bitwise equality is checked where the launch shape is equal).
"""

import time

import numpy as np
import pytest
import torch

from oracle import stokes
from paper_2307_05266_gb300 import binding, synth

pytestmark = pytest.mark.gpu

# members of the batch and jobs of the server that are also checked against the oracle
ORACLE_MEMBERS = (0, 2, 5)
_ORACLE_K = {}


def _oracle_k(i, mask, axis, precond, tol=1e-8):
    """The FP64 oracle's permeability of mask i along `axis` (cached per test module)."""
    key = (i, axis, precond, tol)
    if key not in _ORACLE_K:
        f = [0.0, 0.0, 0.0]
        f[axis] = 1.0
        ref = stokes.solve(mask, tuple(f), stokes.Options(precond=precond, tol=tol))
        _ORACLE_K[key] = ref["k"][axis]
    return _ORACLE_K[key]


def _check_oracle_k(i, mask, axis, precond, k, precision):
    """Batched and served results against the oracle: k within 1e-8 (FP64) or 1e-6
    (mixed precision) of the oracle's k on the same mask and axis."""
    k_ref = _oracle_k(i, mask, axis, precond)
    rtol = 1e-8 if precision == binding.FP64 else 1e-6
    assert abs(k - k_ref) <= rtol * abs(k_ref), (i, k, k_ref)


def _masks():
    specs = [(24, 2.0, 4.0, 0.45, 1), (32, 3.0, 6.0, 0.35, 2), (20, 2.0, 3.0, 0.5, 3),
             (28, 2.0, 5.0, 0.3, 4), (36, 3.0, 7.0, 0.4, 5), ((32, 24, 20), 2.0, 4.0, 0.45, 6)]
    return [synth.sphere_packing(n, a, b, phi, s) for n, a, b, phi, s in specs]


def _alone(mask, axis, launch=None, **opts):
    f = [0.0, 0.0, 0.0]
    f[axis] = 1.0
    with binding.Geometry(mask) as g:
        if launch is not None:
            g.set_launch(*launch)
        g.set_force(f)
        st = g.solve(**opts)
        rs = g.recover_velocity()
        return st.outer_iters, st.inner_iters_A + st.inner_iters_A_f32, g.permeability(axis)


def test_async_equals_sync():
    torch.cuda.set_device(0)
    mask = _masks()[0]
    ref = _alone(mask, 0, precond=binding.SIMPLE)
    with binding.Geometry(mask) as g:
        g.solve_async(precond=binding.SIMPLE)
        while not g.query():
            time.sleep(0.001)
        st, rs = g.finish()
        assert (st.outer_iters, st.inner_iters_A) == ref[:2]
        assert g.permeability(0) == ref[2]
        assert rs.inner_iters_A > 0


@pytest.mark.parametrize("precision", [binding.FP64, binding.MIXED])
def test_batch_equals_individual(precision):
    torch.cuda.set_device(0)
    masks = _masks()
    # a batch member runs with launch shape (blocks_per_sm, 16 entries per thread)
    refs = [_alone(m, 0, launch=(8, 16, 1), precond=binding.SIMPLE, precision=precision,
                   tol=1e-8) for m in masks]
    geoms = [binding.Geometry(m) for m in masks]
    b = binding.Batch(geoms, blocks_per_sm=8, precond=binding.SIMPLE, precision=precision,
                      tol=1e-8)
    for _ in range(2):                      # the batch graph can be relaunched
        ss, rs, ks = b.run()
        for i, ref in enumerate(refs):
            assert ss[i].outer_iters == ref[0]
            assert ks[i][0] == ref[2]
    for i in ORACLE_MEMBERS:
        _check_oracle_k(i, masks[i], 0, stokes.SIMPLE, ks[i][0], precision)
    b.close()
    for g in geoms:
        g.close()


def test_batch_autotune_keeps_results():
    torch.cuda.set_device(0)
    masks = _masks()
    refs = [_alone(m, 0, precond=binding.UZAWA, precision=binding.MIXED, tol=1e-8) for m in masks]
    geoms = [binding.Geometry(m) for m in masks]
    best, ms = binding.Batch.autotune(geoms, precond=binding.UZAWA, precision=binding.MIXED,
                                      tol=1e-8)
    assert len(best) == 3 and best[2] in (0, 1) and ms > 0
    b = binding.Batch(geoms, blocks_per_sm=0, precond=binding.UZAWA,
                      precision=binding.MIXED, tol=1e-8)
    ss, rs, ks = b.run()
    for i, ref in enumerate(refs):
        assert abs(ks[i][0] - ref[2]) <= 1e-6 * abs(ref[2])
    for i in ORACLE_MEMBERS:
        _check_oracle_k(i, masks[i], 0, stokes.UZAWA, ks[i][0], binding.MIXED)
    b.close()
    for g in geoms:
        g.close()


def _serve(masks, axes, budget, max_active, **opts):
    srv = binding.Server(budget, max_active=max_active, **opts)
    ids = [srv.submit(m, axis=a) for m, a in zip(masks, axes)]
    res = {}
    t0 = time.time()
    while len(res) < len(ids):
        srv.progress()
        for r in srv.take():
            res[r["id"]] = r
        assert time.time() - t0 < 300
        time.sleep(0.0005)
    info = srv.info()
    srv.close()
    return [res[i] for i in ids], info


def test_server_results_alone_equal_in_mix():
    """Continuous batching: every job's permeability is the same when it runs alone
    (one job at a time) and when it overlaps with the others."""
    torch.cuda.set_device(0)
    masks = _masks()
    axes = [0, 1, 2, 0, 1, 2]
    opts = dict(precond=binding.SIMPLE, precision=binding.MIXED, tol=1e-8)
    alone, _ = _serve(masks, axes, 1 << 36, 1, **opts)
    mixed, info = _serve(masks, axes, 1 << 36, 6, **opts)
    assert info["peak_active"] > 1
    for a, m in zip(alone, mixed):
        assert a["status"] == binding.SCHUR_OK and m["status"] == binding.SCHUR_OK
        assert a["k"] == m["k"] and a["outer_iters"] == m["outer_iters"]
    for mask, ax, r in zip(masks, axes, mixed):
        ref = _alone(mask, ax, **opts)
        assert abs(r["k"] - ref[2]) <= 1e-6 * abs(ref[2])
    for i in ORACLE_MEMBERS:
        _check_oracle_k(i, masks[i], axes[i], stokes.SIMPLE, mixed[i]["k"], binding.MIXED)


def test_server_admission_respects_budget():
    torch.cuda.set_device(0)
    masks = _masks()
    need = max(binding.footprint_bytes(m.shape, binding.MIXED) for m in masks)
    budget = int(2.5 * need)                # at most two of the largest at a time
    res, info = _serve(masks, [0] * len(masks), budget, 16, precision=binding.MIXED)
    assert info["peak_bytes"] <= budget
    assert all(r["status"] == binding.SCHUR_OK for r in res)
    # waiting jobs start only after earlier ones free memory
    assert all(r["t_start"] >= r["t_submit"] for r in res)


def test_launch_shape_changes_only_rounding():
    """The launch shape (grid cap, entries per thread) changes the order of the floating-
    point reductions only: results agree to rounding, and an equal shape repeats the bits."""
    torch.cuda.set_device(0)
    mask = _masks()[1]
    out = []
    with binding.Geometry(mask) as g:
        g.set_force((1.0, 0.0, 0.0))
        for shape in ((8, 1, 1), (2, 16, 1), (1, 64, 1), (8, 1, 0), (8, 1, 1)):
            g.set_launch(*shape)
            st = g.solve(precond=binding.SIMPLE, tol=1e-8)
            g.recover_velocity()
            out.append((st.outer_iters, g.permeability(0)))
        with pytest.raises(RuntimeError):
            g.set_launch(0, 1)
    assert out[4] == out[0]
    for it, k in out[1:4]:
        assert abs(it - out[0][0]) <= 1
        assert abs(k - out[0][1]) <= 1e-10 * abs(out[0][1])


def test_server_auto_preconditioner_by_porosity():
    """SCHUR_PRECOND_AUTO: SIMPLE for tight jobs (fluid fraction below 0.25), Uzawa otherwise;
    each result matches the same job solved alone with that preconditioner."""
    torch.cuda.set_device(0)
    masks = [synth.sphere_packing(24, 2.0, 3.0, 0.15, 8), synth.sphere_packing(24, 2.0, 4.0, 0.45, 9)]
    res, _ = _serve(masks, [0, 0], 1 << 36, 4, precond=binding.PRECOND_AUTO,
                    precision=binding.MIXED, tol=1e-8)
    want = [binding.SIMPLE if m.mean() < binding.AUTO_SIMPLE_BELOW else binding.UZAWA for m in masks]
    assert want == [binding.SIMPLE, binding.UZAWA]
    for m, r, pc in zip(masks, res, want):
        assert r["status"] == binding.SCHUR_OK and r["precond"] == pc
        ref = _alone(m, 0, precond=pc, precision=binding.MIXED, tol=1e-8)
        assert abs(r["k"] - ref[2]) <= 1e-6 * abs(ref[2])


def test_batch_auto_preconditioner_matches_individual():
    torch.cuda.set_device(0)
    masks = [synth.sphere_packing(24, 2.0, 3.0, 0.15, 8), synth.sphere_packing(24, 2.0, 4.0, 0.45, 9)]
    want = [binding.SIMPLE, binding.UZAWA]
    refs = [_alone(m, 0, launch=(8, 16, 1), precond=pc, precision=binding.MIXED, tol=1e-8)
            for m, pc in zip(masks, want)]
    geoms = [binding.Geometry(m) for m in masks]
    b = binding.Batch(geoms, blocks_per_sm=8, precond=binding.PRECOND_AUTO,
                      precision=binding.MIXED, tol=1e-8)
    ss, rs, ks = b.run()
    for s_, ref, k in zip(ss, refs, ks):
        assert s_.outer_iters == ref[0] and k[0] == ref[2]
    b.close()
    for g in geoms:
        g.close()


def test_batch_and_server_with_multigrid_inner_solves():
    """Multigrid inner solves in the batch graph (persistent loop kernels in parallel
    branches) and in the server: each result equals the same job solved alone with the same
    launch shape, and three of them are checked against the oracle's multigrid path."""
    torch.cuda.set_device(0)
    masks = _masks()
    opts = dict(precond=binding.SIMPLE, precision=binding.MIXED, tol=1e-8,
                inner_precond=binding.INNER_MG)
    refs = [_alone(m, 0, launch=(2, 16, 1), **opts) for m in masks]
    geoms = [binding.Geometry(m) for m in masks]
    b = binding.Batch(geoms, blocks_per_sm=2, **opts)
    ss, rs, ks = b.run()
    for i, ref in enumerate(refs):
        assert ss[i].status == binding.SCHUR_OK
        assert ss[i].outer_iters == ref[0] and ks[i][0] == ref[2]
    b.close()
    for g in geoms:
        g.close()
    axes = [0, 1, 2, 0, 1, 2]
    res, info = _serve(masks, axes, 1 << 36, 6, **opts)
    for i in ORACLE_MEMBERS:
        f = [0.0, 0.0, 0.0]
        f[axes[i]] = 1.0
        ref = stokes.solve(masks[i], tuple(f), stokes.Options(precond=stokes.SIMPLE, tol=1e-8,
                                                              inner_precond=stokes.INNER_AMG))
        k_ref = ref["k"][axes[i]]
        assert res[i]["status"] == binding.SCHUR_OK
        assert abs(res[i]["k"] - k_ref) <= 1e-6 * abs(k_ref)
        assert abs(ks[i][0] - _oracle_k(i, masks[i], 0, stokes.SIMPLE)) <= 1e-6 * abs(ks[i][0])
