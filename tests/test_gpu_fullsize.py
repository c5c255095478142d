"""Full-size parity: the CUDA path against oracle runs stored by oracle/record_reference.py
(64^3 and 128^3 periodic sphere packings, radii U[4,8), porosity 0.40, f = e_x, tol 1e-8,
inner 1e-12).  Permeability within 1e-8 relative, outer and inner iteration counts
within 2, plus properties of the GPU solution checked with the oracle's own operators
(divergence-free velocity, momentum residual)."""

import json
import os

import numpy as np
import pytest
import torch

from oracle import mac, stokes
from paper_2307_05266_gb300 import binding, synth

from gpu_helpers import (cell_device_to_compact, check_pressure, check_velocity,
                         face_device_to_compact)

pytestmark = pytest.mark.gpu
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
PRECONDS = {"uzawa": binding.UZAWA, "simple": binding.SIMPLE}


def _golden(workload, pc):
    with open(os.path.join(GOLDEN, f"oracle_{workload}_{pc}.json")) as f:
        return json.load(f)


@pytest.mark.parametrize("workload,n", [("spheres64", 64), ("spheres128", 128)])
@pytest.mark.parametrize("pc", ["uzawa", "simple"])
def test_fullsize_against_recorded_oracle(workload, n, pc):
    ref = _golden(workload, pc)
    torch.cuda.set_device(0)
    mask = synth.sphere_packing(n, 4.0, 8.0, 0.40, 0)
    with binding.Geometry(mask) as g:
        info = g.geometry_info()
        assert sum(info.n_unknown[a] for a in range(3)) == ref["n_unknown"]
        assert info.n_fluid == ref["n_fluid"]
        g.set_force((1.0, 0.0, 0.0))
        st = g.solve(precond=PRECONDS[pc], tol=1e-8)
        rec = g.recover_velocity()
        k = [g.permeability(a) for a in range(3)]
        assert abs(st.outer_iters - ref["outer_iters"]) <= 2
        assert abs(st.inner_iters_A - ref["inner_iters_A"]) <= 2 * max(1, ref["outer_iters"])
        assert abs(rec.inner_iters_A - ref["recovery_iters"]) <= 2
        assert abs(k[0] - ref["k"][0]) <= 1e-8 * abs(ref["k"][0])
        if n == 64:
            # properties of the GPU solution with the oracle's assembled operators
            prob = stokes.StokesProblem(mask)
            geo = prob.geo
            u = face_device_to_compact(g, geo, g.field(binding.FIELD_U))
            p = cell_device_to_compact(geo, g.field(binding.FIELD_P))
            div = prob.B @ u
            assert np.linalg.norm(div) <= 1e-7 * np.linalg.norm(abs(prob.B) @ np.abs(u))
            res = prob.A @ u - (mac.force(geo, (1.0, 0.0, 0.0)) - prob.BT @ p)
            assert np.linalg.norm(res) <= 1e-9 * np.linalg.norm(prob.A @ u)


@pytest.mark.parametrize("workload,n", [("spheres64", 64), ("spheres128", 128)])
@pytest.mark.parametrize("pc", ["uzawa", "simple"])
def test_fullsize_mixed_precision(workload, n, pc):
    """Mixed precision at full size: permeability within 1e-6 of the FP64 oracle record."""
    ref = _golden(workload, pc)
    torch.cuda.set_device(0)
    mask = synth.sphere_packing(n, 4.0, 8.0, 0.40, 0)
    with binding.Geometry(mask) as g:
        g.set_force((1.0, 0.0, 0.0))
        st = g.solve(precond=PRECONDS[pc], precision=binding.MIXED, tol=1e-8)
        assert st.status == binding.SCHUR_OK and st.rel_res < 1e-8
        g.recover_velocity()
        assert abs(g.permeability(0) - ref["k"][0]) <= 1e-6 * abs(ref["k"][0])


def test_tight256_properties_at_full_size():
    """The tight 256^3 workload (porosity 0.15, radii U[2, 4)) at full size, where a whole
    oracle solve does not fit a test: face flags bit-exact against the oracle's
    classification; the FP64 SIMPLE solution's velocity divergence-free and k equal to the
    box average of u_x (Section 2.3); mixed precision within 1e-6 of the FP64 k."""
    torch.cuda.set_device(0)
    mask = synth.sphere_packing(256, 2.0, 4.0, 0.15, 0)
    ref_flags = mac.face_flags(mac.classify(mask))
    with binding.Geometry(mask) as g:
        info = g.geometry_info()
        stride = info.face_stride
        flags = g.field(binding.FIELD_FLAGS).cpu().numpy().reshape(3, stride)[:, :mask.size]
        assert np.array_equal(flags.reshape(ref_flags.shape), ref_flags)
        g.set_force((1.0, 0.0, 0.0))
        st = g.solve(precond=binding.SIMPLE, tol=1e-8)
        assert st.status == binding.SCHUR_OK
        g.recover_velocity()
        k64 = g.permeability(0)
        u = g.field(binding.FIELD_U).clone()
        div = torch.zeros(mask.size, dtype=torch.float64, device="cuda")
        g.apply_B(u, div)
        ux = u[:stride][:mask.size]
        assert k64 == pytest.approx(float(ux.sum()) / mask.size, rel=1e-12)
        # B u = g - S p = the outer residual (plus inner-solve error): ||r|| <= tol ||g||
        assert float(div.norm()) <= 1e-7 * st.g_norm
        g.solve(precond=binding.SIMPLE, precision=binding.MIXED, tol=1e-8)
        g.recover_velocity()
        assert abs(g.permeability(0) - k64) <= 1e-6 * abs(k64)


# 48^3 periodic packing, radii U[3, 6), porosity 0.40, seed 7: 115,112 unknown faces and
# 44,169 fluid cells in one component of 44,115 cells plus 45 small ones, so the persistent
# loops take several grid-stride steps per thread and both per-component reductions (the
# grid-wide one for big components, the warp-per-component one for small ones) run.
FIELD_TOL = 1e-9


@pytest.fixture(scope="module")
def field48():
    mask = synth.sphere_packing(48, 3.0, 6.0, 0.40, 7)
    f = (1.0, 0.0, 0.0)
    refs = {pc: stokes.solve(mask, f, stokes.Options(precond=pc, tol=FIELD_TOL))
            for pc in (stokes.UZAWA, stokes.SIMPLE)}
    from oracle import krylov
    lam_min, _, _ = krylov.lanczos_cond(refs[stokes.UZAWA]["schur"].alphas,
                                        refs[stokes.UZAWA]["schur"].betas)
    return mask, f, refs, lam_min


@pytest.mark.parametrize("pc", [binding.UZAWA, binding.SIMPLE])
def test_field_parity_48(field48, pc):
    """u, p (modulo per-component constants) and k of the FP64 CUDA path against the
    oracle on the same 48^3 mask, element by element."""
    mask, f, refs, lam_min = field48
    ref = refs[pc]
    prob = ref["problem"]
    geo = prob.geo
    assert prob.n_comp > 1 and np.bincount(prob.comp).max() >= 2048
    torch.cuda.set_device(0)
    with binding.Geometry(mask) as g:
        g.set_force(f)
        st = g.solve(precond=pc, tol=FIELD_TOL)
        rec = g.recover_velocity()
        assert st.status == binding.SCHUR_OK
        assert abs(st.outer_iters - ref["schur"].outer_iters) <= 2
        assert abs(rec.inner_iters_A - ref["recovery"].iters) <= 2
        u = face_device_to_compact(g, geo, g.field(binding.FIELD_U))
        p = cell_device_to_compact(geo, g.field(binding.FIELD_P))
        check_velocity(prob, geo, f, u, ref["u"])
        check_pressure(geo, p, ref["p"], ref["g"], FIELD_TOL, lam_min)
        for a in range(3):
            assert abs(g.permeability(a) - ref["k"][a]) <= 1e-8 * abs(ref["k"][0])
