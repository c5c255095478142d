"""Pins of the FP64 oracle against facts that do not come from the oracle itself.

Each test names what fixes the expected value: a closed form, an invariant of the
discretisation, a number the paper prints, or a brute-force / library computation on
a tiny grid.  ``test_planted_*`` plant plausible mistakes in a copy of the oracle and
check that a pin catches each of them.
"""

import os

import numpy as np
import pytest
import scipy.sparse.linalg as spla

from oracle import dense, krylov, mac, stokes
from paper_2307_05266_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _random_mask(shape, phi, seed):
    rng = np.random.default_rng(seed)
    return (rng.random(shape) < phi).astype(np.uint8)


SMALL_GEOMETRIES = [
    ((6, 7), 0.75, 1, None),
    ((5, 6, 4), 0.8, 2, None),
    ((7, 5), 0.8, 3, (True, False)),
    ((4, 5, 6), 0.85, 4, (False, True, True)),
    ((6, 6, 5), 0.7, 5, (True, True, False)),
]


def _load_table(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append([float(v) for v in line.split()])
    return rows


# ---- operator invariants --------------------------------------------------------
@pytest.mark.parametrize("shape,phi,seed,periodic", SMALL_GEOMETRIES)
def test_gradient_is_transpose_of_divergence(shape, phi, seed, periodic):
    """eq. coupled_matrix: the discrete gradient is the adjoint of -div.  B and B^T are
    assembled from their own definitions, so a sign or index slip in either breaks
    the identity."""
    geo = mac.classify(_random_mask(shape, phi, seed), periodic)
    B = mac.assemble_B(geo)
    G = mac.assemble_grad(geo)
    assert abs(G - B.T).max() == 0.0
    assert B.nnz == 2 * geo.n_u


@pytest.mark.parametrize("shape,phi,seed,periodic", SMALL_GEOMETRIES)
def test_A_symmetric_positive_definite(shape, phi, seed, periodic):
    """A = -Delta_h with no-slip walls is symmetric, and positive definite once every
    face component meets a wall."""
    geo = mac.classify(_random_mask(shape, phi, seed), periodic)
    A = mac.assemble_A(geo)
    assert abs(A - A.T).max() == 0.0
    w = np.linalg.eigvalsh(A.toarray())
    assert w[0] > 0.0


def test_flags_by_hand():
    """Flag bytes of a 4x4 periodic box with one solid voxel at (x=1, y=2), worked out by
    hand: bit 0 = both cells fluid, bits 1..3 = solid-solid tangential neighbours."""
    m = np.ones((4, 4), np.uint8)
    m[2, 1] = 0
    flags = mac.face_flags(mac.classify(m))
    fx, fy = flags[0], flags[1]
    # x-faces touching the solid voxel are walls: lower face of (1,2) and of (2,2)
    assert fx[2, 1] == 0 and fx[2, 2] == 0
    # no two solid voxels are adjacent, so no face is solid-solid and no ghost appears
    assert np.all((fx >> 1) == 0) and np.all((fy >> 1) == 0)
    assert fx.sum() == 14 and fy.sum() == 14


def test_flags_ghosts_by_hand():
    """A solid row y = 0 in a 4x4 periodic box: the x-faces of row 1 have the solid-solid
    x-face of row 0 as their -y neighbour (one ghost), row 3 has it as +y neighbour."""
    m = np.ones((4, 4), np.uint8)
    m[0, :] = 0
    flags = mac.face_flags(mac.classify(m))
    fx, fy = flags[0], flags[1]
    assert np.all(fx[0] == 0)
    assert np.all(fx[1] == 1 | (1 << 1)) and np.all(fx[3] == 1 | (1 << 1))
    assert np.all(fx[2] == 1)
    # y-faces: lower face of row 1 and of row 0 are walls, rows 2 and 3 are unknowns
    assert np.all(fy[0] == 0) and np.all(fy[1] == 0)
    assert np.all(fy[2] == 1) and np.all(fy[3] == 1)


DIAG_GEOMETRIES = SMALL_GEOMETRIES + [
    ((9, 11), 0.6, 6, (True, True)),
    ((8, 10), 0.55, 7, (False, False)),
    ((7, 6, 9), 0.6, 8, None),
    ((6, 8, 7), 0.55, 9, (False, False, False)),
    ((5, 9, 8), 0.65, 10, (False, True, False)),
]


@pytest.mark.parametrize("shape,phi,seed,periodic", DIAG_GEOMETRIES)
def test_diag_A_is_the_assembled_diagonal(shape, phi, seed, periodic):
    """diag_A (the SIMPLE A-hat and the inner Jacobi weights) writes the diagonal
    h^-2 (2d + g_f) out separately from assemble_A; the two must agree exactly on walled
    and periodic, 2D and 3D geometries with ghosts, up to the rounding of h^-2 (the two
    divide by h^2 in a different order; h = 1/n_x is not a power of two here).
    assemble_A's diagonal is itself pinned by the Poiseuille closed form and by the
    hand-worked case below."""
    geo = mac.classify(_random_mask(shape, phi, seed), periodic)
    assert sum(int((g > 0).sum()) for g in geo.ghosts) > 0        # ghosts are exercised
    np.testing.assert_allclose(mac.diag_A(geo), mac.assemble_A(geo).diagonal(), rtol=1e-15,
                               atol=0)


def test_diag_A_ghost_by_hand():
    """Solid row y = 0 in a 4x4 periodic box (h = 1/4): the x-faces of rows 1 and 3 have
    the solid-solid x-face of row 0 as a tangential neighbour, a wall half a cell away
    whose ghost value -u_f adds one to the diagonal: (2d + 1) / h^2 = 5 * 16 = 80.
    Row 2 has no ghost (4 * 16 = 64); the y-faces of rows 2 and 3 have their normal
    neighbours (the wall faces of rows 1 and 0) at distance h: no ghost, 64."""
    m = np.ones((4, 4), np.uint8)
    m[0, :] = 0
    geo = mac.classify(m)
    dA = mac.diag_A(geo)
    dx = dA[geo.uidx[0][geo.unknown[0]]].reshape(3, 4)        # rows 1, 2, 3
    np.testing.assert_array_equal(dx, [[80.0] * 4, [64.0] * 4, [80.0] * 4])
    dy = dA[geo.uidx[1][geo.unknown[1]]]
    np.testing.assert_array_equal(dy, np.full(8, 64.0))
    np.testing.assert_array_equal(mac.assemble_A(geo).diagonal(), dA)


def test_planted_double_ghost_in_diag_A(monkeypatch):
    """A slip in diag_A alone (2d + 2g instead of 2d + g) leaves assemble_A, and with it
    every solve of A, unchanged; the two diagonal pins above catch it."""
    def two_ghosts(geo):
        out = np.empty(geo.n_u)
        for a in range(geo.d):
            sel = geo.unknown[a]
            out[geo.uidx[a][sel]] = (2 * geo.d + 2.0 * geo.ghosts[a][sel]) / geo.h**2
        return out

    monkeypatch.setattr(mac, "diag_A", two_ghosts)
    geo = mac.classify(_random_mask((6, 6, 5), 0.7, 5), (True, True, False))
    assert not np.allclose(mac.diag_A(geo), mac.assemble_A(geo).diagonal(), rtol=1e-15,
                           atol=0)
    m = np.ones((4, 4), np.uint8)
    m[0, :] = 0
    g2 = mac.classify(m)
    assert mac.diag_A(g2)[g2.uidx[0][1, 0]] != 80.0


def test_simple_operator_empty_box_symbol():
    """With no walls diag(A) = 2d/h^2, so S-hat_simple = B B^T h^2 / (2d): the
    dimensionless periodic Laplacian over 2d, eigenvalues sum_b 4 sin^2(pi k_b / n_b)/(2d)."""
    shape = (5, 6, 4)                      # [z][y][x]
    prob = stokes.StokesProblem(np.ones(shape, np.uint8))
    w = np.sort(np.linalg.eigvalsh(prob.S_simple.toarray()))
    ks = [np.arange(n) for n in shape]
    sym = sum(4 * np.sin(np.pi * k / n) ** 2 for k, n in
              zip(np.meshgrid(*ks, indexing="ij"), shape))
    np.testing.assert_allclose(w, np.sort((sym / 6.0).ravel()), atol=1e-12)


# ---- spectra (Section 1, Section 4.2.4) ----------------------------------------
@pytest.mark.parametrize("shape", [(6, 6), (5, 7), (4, 4, 4), (3, 4, 5)])
def test_empty_periodic_box_spectrum_is_unit(shape):
    """Without no-slip walls S is the identity on mean-free pressures (the paper's
    conjecture that the non-unit eigenvalues come from the no-slip walls, in the limit
    with no walls): spectrum {0, 1, ..., 1}."""
    w = dense.spectrum(stokes.StokesProblem(np.ones(shape, np.uint8)))
    assert abs(w[0]) < 1e-12
    np.testing.assert_allclose(w[1:], 1.0, atol=1e-12)


@pytest.mark.parametrize("shape,phi,seed,periodic", SMALL_GEOMETRIES)
def test_lambda_max_is_one(shape, phi, seed, periodic):
    """lambda_max(S) = 1 (Section 4.2.2, eq. lambda_cg_rate)."""
    w = dense.spectrum(stokes.StokesProblem(_random_mask(shape, phi, seed), periodic))
    assert abs(w.max() - 1.0) < 1e-12
    assert w.min() > -1e-12


@pytest.mark.parametrize("N,n_c,n_avg", [(1, 10, 4), (2, 8, 4), (2, 10, 4), (2, 10, 6),
                                         (3, 8, 4)])
@pytest.mark.parametrize("seed", [0, 1, 2])
def test_non_unit_eigenvalue_count_law(N, n_c, n_avg, seed):
    """eq. spectrum_relation: N_ev = V_surf + 3 N^2 - 1 on square arrays (Section 4.2.4)."""
    m = synth.square_array_2d(N, n_c, n_avg, 2, seed)
    w = dense.spectrum(stokes.StokesProblem(m))
    n_ev = int(np.sum(np.abs(w - 1.0) > 1e-8))
    assert n_ev == stokes.surface_area(m) + 3 * N * N - 1


def test_condition_trend_with_surface_to_volume():
    """Table 4 / Section 4.2.3: cond(S) grows and cond(S-hat^-1 S) falls as the
    channels narrow (sigma_s grows)."""
    cs, cp, sig = [], [], []
    for n_avg in (4, 6, 8, 10):
        m = synth.square_array_2d(3, 14, n_avg, 2, seed=7)
        prob = stokes.StokesProblem(m)
        cs.append(dense.effective_cond(dense.spectrum(prob)))
        cp.append(dense.effective_cond(dense.preconditioned_spectrum(prob)))
        sig.append(stokes.surface_to_volume(m))
    assert all(np.diff(sig) < 0)
    assert all(np.diff(cs) < 0), cs
    assert all(np.diff(cp) > 0), cp
    assert cs[0] > cp[0] and cs[-1] < cp[-1]


# ---- closed-form solutions ------------------------------------------------------
@pytest.mark.parametrize("precond", [stokes.UZAWA, stokes.SIMPLE])
def test_plane_poiseuille_permeability(precond):
    """Discrete plane Poiseuille flow: k = phi (H^2/12 + h^2/6) (golden file)."""
    for n, m, num, den, _ in _load_table("poiseuille_2d.txt"):
        n, m = int(n), int(m)
        mask = synth.channel_2d(n)
        assert int(mask.sum()) == m * n
        r = stokes.solve(mask, (1.0, 0.0), stokes.Options(precond=precond, tol=1e-10))
        assert r["schur"].outer_iters == 0          # g vanishes: x-invariant flow
        assert abs(r["k"][0] - num / den) <= 1e-12 * (num / den)
        assert abs(r["k"][1]) <= 1e-15


def test_poiseuille_3d_slab():
    """The same closed form for a 3D slab (walls normal to z, flow along x or y)."""
    n = 8
    mask = np.ones((n, n, n), np.uint8)
    mask[0] = 0
    mask[n - 1] = 0
    h, H, phi = 1.0 / n, (n - 2) / n, (n - 2) / n
    k_exact = phi * (H * H / 12 + h * h / 6)
    for f, a in (((1.0, 0, 0), 0), ((0, 1.0, 0), 1)):
        r = stokes.solve(mask, f, stokes.Options(precond=stokes.SIMPLE))
        assert abs(r["k"][a] - k_exact) <= 1e-12 * k_exact


def test_poiseuille_approaches_continuum():
    """As h -> 0 the discrete channel permeability tends to phi H^2 / 12."""
    errs = []
    for n in (8, 16, 32):
        r = stokes.solve(synth.channel_2d(n), (1.0, 0.0), stokes.Options())
        H = (n - 2) / n
        errs.append(abs(r["k"][0] - (n - 2) / n * H * H / 12))
    assert errs[1] < errs[0] / 3 and errs[2] < errs[1] / 3


@pytest.mark.parametrize("precond", [stokes.UZAWA, stokes.SIMPLE])
def test_channel_cross_force_hydrostatic(precond):
    """Force across the band: the exact solution is u = 0 with B^T p = f (pressure
    linear in y inside the band), so the whole Schur path runs with ||g|| != 0."""
    mask = synth.channel_2d(16)
    r = stokes.solve(mask, (0.0, 1.0), stokes.Options(precond=precond, tol=1e-8))
    prob = r["problem"]
    assert r["schur"].status == krylov.OK and r["schur"].outer_iters >= 1
    assert np.abs(r["u"]).max() < 1e-9
    f = mac.force(prob.geo, (0.0, 1.0))
    # the outer tolerance bounds the residual; the error may be cond(S) times larger
    np.testing.assert_allclose(prob.BT @ r["p"], f, atol=1e-5)


# ---- brute force on tiny grids ---------------------------------------------------
@pytest.mark.parametrize("shape,phi,seed,periodic", SMALL_GEOMETRIES)
@pytest.mark.parametrize("precond", [stokes.UZAWA, stokes.SIMPLE])
def test_cg_solution_equals_dense_min_norm(shape, phi, seed, periodic, precond):
    """Algorithm 1 with tight inner solves reaches the minimum-norm solution of the
    dense S p = g; velocity and permeability follow from eq. velocity_schur."""
    mask = _random_mask(shape, phi, seed)
    d = len(shape)
    f = (1.0,) + (0.0,) * (d - 1)
    r = stokes.solve(mask, f, stokes.Options(precond=precond, tol=1e-11, max_outer=500),
                     periodic)
    prob = r["problem"]
    S = dense.schur_dense(prob)
    A = prob.A.toarray()
    u_f = np.linalg.solve(A, mac.force(prob.geo, f))
    g = prob.B @ u_f
    p_ref = dense.min_norm_solution(S, g)
    u_ref = np.linalg.solve(A, mac.force(prob.geo, f) - prob.BT @ p_ref)
    # p is unique up to the nullspace of B^T: compare gradients, velocities, k
    np.testing.assert_allclose(prob.BT @ r["p"], prob.BT @ p_ref, atol=1e-8)
    np.testing.assert_allclose(r["u"], u_ref, atol=1e-10 * max(1.0, np.abs(u_ref).max()))
    ux = u_ref[prob.geo.uidx[0][prob.geo.unknown[0]]]
    k_ref = ux.sum() / mask.size
    # h^2 |f| is the velocity scale of a one-voxel pore; k is ~0 when x is blocked
    assert abs(r["k"][0] - k_ref) <= 1e-9 * (abs(k_ref) + prob.geo.h ** 2)


def test_inner_pcg_matches_sparse_direct():
    """Jacobi PCG on A reaches the sparse direct solution."""
    m = synth.sphere_packing(16, 2, 4, 0.5, seed=3)
    prob = stokes.StokesProblem(m)
    b = mac.force(prob.geo, (0.3, -1.0, 0.5))
    res = prob.solve_A(b, 1e-13, 5000)
    x = spla.spsolve(prob.A.tocsc(), b)
    assert res.status == krylov.OK
    np.testing.assert_allclose(res.x, x, rtol=0, atol=1e-10 * np.abs(x).max())


def test_pcg_finite_termination():
    """CG on an SPD matrix with k distinct eigenvalues converges in k steps."""
    rng = np.random.default_rng(0)
    Q, _ = np.linalg.qr(rng.standard_normal((40, 40)))
    lam = np.repeat([1.0, 2.0, 5.0, 9.0, 30.0], 8)
    M = (Q * lam) @ Q.T
    res = krylov.pcg(lambda v: M @ v, rng.standard_normal(40), np.ones(40), 1e-10, 100)
    assert res.status == krylov.OK and res.iters == 5


def test_recovered_velocity_divergence_free():
    """A u = f - B^T p with S p = g makes B u = 0 up to the solver tolerances."""
    m = synth.sphere_packing(16, 3, 5, 0.45, seed=1)
    r = stokes.solve(m, (0.0, 0.0, 1.0), stokes.Options(precond=stokes.SIMPLE, tol=1e-10))
    prob = r["problem"]
    div = prob.B @ r["u"]
    assert np.linalg.norm(div) <= 1e-8 * np.linalg.norm(abs(prob.B) @ np.abs(r["u"]))


def test_both_preconditioners_agree():
    m = synth.sphere_packing(16, 3, 5, 0.4, seed=4)
    ks = [stokes.solve(m, (1.0, 0, 0), stokes.Options(precond=p, tol=1e-10))["k"][0]
          for p in (stokes.UZAWA, stokes.SIMPLE)]
    assert abs(ks[0] - ks[1]) <= 1e-8 * abs(ks[0])


# ---- geometry statistics against Table 3 ----------------------------------------
def test_table3_square_array_statistics():
    """Table 3: V^f, porosity and sigma_s of the N=7, n_c=50, n_min=2 square arrays, to
    the paper's print rounding (its last digit may be off by one)."""
    for n_avg, vf_k, phi_pct, sig_pct in _load_table("table3_square_arrays.txt"):
        for seed in (0, 1):
            m = synth.square_array_2d(7, 50, int(n_avg), 2, seed)
            assert m.shape == (350, 350)
            assert abs(m.sum() / 1000.0 - vf_k) <= 0.1 + 1e-9
            assert abs(100 * stokes.porosity(m) - phi_pct) <= 0.1 + 1e-9
            assert abs(100 * stokes.surface_to_volume(m) - sig_pct) <= 0.1 + 1e-9


# ---- planted mistakes: each must fail a pin ------------------------------------
def _poiseuille_k():
    r = stokes.solve(synth.channel_2d(16), (1.0, 0.0), stokes.Options())
    return r["k"][0]


def test_planted_dropped_ghost_term(monkeypatch):
    """Dropping the ghost contribution (diag 2d instead of 2d + g) misses Poiseuille."""
    orig = mac.classify

    def no_ghosts(mask, periodic=None):
        geo = orig(mask, periodic)
        geo.ghosts = [np.zeros_like(g) for g in geo.ghosts]
        return geo

    monkeypatch.setattr(mac, "classify", no_ghosts)
    k = _poiseuille_k()
    assert abs(k - 231 / 4096) > 1e-3 * 231 / 4096


def test_planted_gradient_sign(monkeypatch):
    """A gradient with the wrong sign breaks B^T = transpose(B)."""
    orig = mac.assemble_grad
    monkeypatch.setattr(mac, "assemble_grad", lambda geo: -orig(geo))
    geo = mac.classify(_random_mask((6, 7), 0.75, 1))
    assert abs(mac.assemble_grad(geo) - mac.assemble_B(geo).T).max() > 0


def test_planted_alg1_printed_sign():
    """Algorithm 1 as printed (r = S p - g, p += alpha d, r += alpha q) does not solve
    S p = g; the sign-fixed loop does (checked on a dense SPD system)."""
    rng = np.random.default_rng(1)
    Q, _ = np.linalg.qr(rng.standard_normal((20, 20)))
    S = (Q * np.linspace(0.1, 1.0, 20)) @ Q.T
    g = rng.standard_normal(20)
    good = krylov.schur_pcg(lambda d: (S @ d, 0), g, lambda r: (r.copy(), 0), 1e-12, 200)
    assert np.linalg.norm(S @ good.p - g) < 1e-10 * np.linalg.norm(g)
    # printed variant
    p = np.zeros(20)
    r = S @ p - g
    z = r.copy()
    d = z.copy()
    for _ in range(40):
        q = S @ d
        alpha = (r @ z) / (d @ q)
        p = p + alpha * d
        r_new = r + alpha * q
        beta = (r_new @ r_new) / (r @ r)
        d = r_new + beta * d
        r = z = r_new
    assert np.linalg.norm(S @ p - g) > 1e-3 * np.linalg.norm(g)


# ---- nullspace handling of the SIMPLE solve (Section 3.2, "special care") ------
def _bfs_components(mask, periodic):
    """Brute force: flood fill over fluid cells through faces whose two cells are fluid."""
    d = mask.ndim
    shape = mask.shape
    lab = -np.ones(shape, dtype=np.int64)
    n = 0
    for start in zip(*np.nonzero(mask)):
        if lab[start] >= 0:
            continue
        stack = [start]
        lab[start] = n
        while stack:
            c = stack.pop()
            for ax in range(d):
                for s in (-1, 1):
                    nb = list(c)
                    nb[ax] += s
                    a = d - 1 - ax
                    if not (0 <= nb[ax] < shape[ax]):
                        if not periodic[a]:
                            continue
                        nb[ax] %= shape[ax]
                    nb = tuple(nb)
                    if mask[nb] and lab[nb] < 0:
                        lab[nb] = n
                        stack.append(nb)
        n += 1
    return n, lab


@pytest.mark.parametrize("shape,phi,seed,periodic", SMALL_GEOMETRIES)
def test_fluid_components_match_flood_fill(shape, phi, seed, periodic):
    mask = _random_mask(shape, phi, seed)
    per = periodic or (True,) * len(shape)
    geo = mac.classify(mask, per)
    n, comp = stokes.fluid_components(geo)
    n_ref, lab = _bfs_components(mask, per)
    assert n == n_ref
    # same partition: labels agree up to renaming
    ref = lab[mask.astype(bool)]
    pairs = set(zip(comp.tolist(), ref.tolist()))
    assert len(pairs) == n


def test_simple_solve_projects_onto_range():
    """z = S-hat^+ r: with r carrying a constant per component (rounding in the outer
    residual), the projected solve still converges, S-hat z equals the projected r and z
    has zero mean on every component."""
    mask = synth.sphere_packing(16, 2.0, 4.0, 0.3, seed=1)
    prob = stokes.StokesProblem(mask)
    assert prob.n_comp > 1
    rng = np.random.default_rng(0)
    r = prob.remove_mean(rng.standard_normal(prob.geo.n_p))
    r_noisy = r + 1e-3 * np.ones_like(r)
    res = prob.solve_simple(r_noisy, 1e-12, 20000)
    assert res.status == krylov.OK
    np.testing.assert_allclose(prob.S_simple @ res.x, r, atol=1e-9 * np.abs(r).max())
    means = np.bincount(prob.comp, weights=res.x) / prob.comp_size
    assert np.abs(means).max() < 1e-12 * max(1.0, np.abs(res.x).max())


# ---- Lanczos condition estimate from CG coefficients (Section 4.2) ----------------
def test_lanczos_tridiagonal_recovers_spectrum_of_preconditioned_matrix():
    """CG run to completion on an SPD matrix with Jacobi M: the Ritz values of the
    implicit Lanczos tridiagonal reach the extreme eigenvalues of M^-1 A (linear algebra,
    independent of the Stokes code)."""
    rng = np.random.default_rng(0)
    n = 30
    Q = np.linalg.qr(rng.standard_normal((n, n)))[0]
    A = (Q * np.geomspace(1.0, 1e3, n)) @ Q.T
    minv = 1.0 / np.diag(A)
    res = krylov.pcg(lambda x: A @ x, rng.standard_normal(n), minv, 1e-15, 200)
    lmin, lmax, cond = krylov.lanczos_cond(res.alphas, res.betas)
    s = np.sqrt(minv)
    w = np.linalg.eigvalsh((s[:, None] * A) * s[None, :])
    assert lmin == pytest.approx(w[0], rel=1e-10)
    assert lmax == pytest.approx(w[-1], rel=1e-10)
    assert cond == pytest.approx(w[-1] / w[0], rel=1e-10)


@pytest.mark.parametrize("n_avg", [4, 8])
def test_lanczos_cond_of_outer_cg_matches_dense(n_avg):
    """The estimate from Algorithm 1's coefficients: cond(S) of CG-Uzawa equals the dense
    effective condition number; the CG-SIMPLE estimate of cond(S-hat^-1 S) lies within a
    few per cent below it (Ritz values lie inside the spectrum)."""
    m = synth.square_array_2d(3, 14, n_avg, 2, seed=7)
    prob = stokes.StokesProblem(m)
    r = stokes.solve(m, (1.0, 0.0), stokes.Options(precond=stokes.UZAWA, tol=1e-10))
    est = krylov.lanczos_cond(r["schur"].alphas, r["schur"].betas)
    assert est[1] == pytest.approx(1.0, rel=1e-9)             # lambda_max(S) = 1
    assert est[2] == pytest.approx(dense.effective_cond(dense.spectrum(prob)), rel=1e-5)
    r = stokes.solve(m, (1.0, 0.0), stokes.Options(precond=stokes.SIMPLE, tol=1e-10))
    est = krylov.lanczos_cond(r["schur"].alphas, r["schur"].betas)
    ref = dense.effective_cond(dense.preconditioned_spectrum(prob))
    assert 0.95 * ref <= est[2] <= ref * (1 + 1e-9)


# ---- stopping rules (Section 3.2, Algorithm 1, Section 4.2.2) ----------------------
def test_inner_stop_is_the_preconditioned_residual():
    """Jacobi PCG stops at the first k with ||M^-1 r_k|| / ||M^-1 r_0|| < eps, r_k the
    recursive residual: recomputed from the returned x (true residual), the ratio agrees
    to rounding, and the unpreconditioned ratio is a different number."""
    m = synth.sphere_packing(14, 2.0, 3.0, 0.5, seed=5)
    prob = stokes.StokesProblem(m)
    b = mac.force(prob.geo, (1.0, 0.0, 0.0))
    minv = 1.0 / prob.dA
    tol = 1e-6
    res = prob.solve_A(b, tol, 20000)
    z0 = np.linalg.norm(minv * b)
    r = b - prob.A @ res.x
    rel_pre = np.linalg.norm(minv * r) / z0
    assert res.status == krylov.OK and rel_pre < tol * 1.01
    assert res.rel == pytest.approx(rel_pre, rel=1e-4)
    prev = prob.solve_A(b, tol, res.iters - 1)            # one iteration earlier: not yet
    assert np.linalg.norm(minv * (b - prob.A @ prev.x)) / z0 >= tol * 0.99
    rel_unpre = np.linalg.norm(r) / np.linalg.norm(b)
    assert abs(rel_unpre - rel_pre) > 1e-3 * rel_pre


@pytest.mark.parametrize("precond", [stokes.UZAWA, stokes.SIMPLE])
def test_outer_preconditioned_stop_rule(precond):
    """Algorithm 1's rule ||z_k|| / ||z_0|| < eps with z = S-hat^-1 r: recomputed from the
    final pressure (r = g - S p, z = S-hat^+ r) it holds at the stop and not one
    iteration earlier; for Uzawa z = r, so both norms coincide."""
    m = synth.square_array_2d(2, 10, 4, 2, seed=1)
    prob = stokes.StokesProblem(m)
    f = (1.0, 0.0)
    tol = 1e-5
    opts = stokes.Options(precond=precond, stop_norm=krylov.STOP_PRECOND, tol=tol)
    out, g = prob.solve(f, opts)
    assert out.status == krylov.OK and out.outer_iters > 1
    assert out.rel_res_precond < tol

    def zrel(p):
        r = g - prob.apply_S(p, 1e-13, 20000)[0]
        if precond == stokes.UZAWA:
            return np.linalg.norm(r) / np.linalg.norm(g)
        r0 = prob.remove_mean(g.copy())
        z0 = prob.solve_simple(r0, 1e-13, 20000).x
        z = prob.solve_simple(prob.remove_mean(r), 1e-13, 20000).x
        return np.linalg.norm(z) / np.linalg.norm(z0)

    assert zrel(out.p) == pytest.approx(out.rel_res_precond, rel=1e-3)
    early = stokes.Options(precond=precond, stop_norm=krylov.STOP_PRECOND, tol=tol,
                           max_outer=out.outer_iters - 1)
    out_e, _ = prob.solve(f, early)
    assert out_e.status == krylov.NOT_CONVERGED and zrel(out_e.p) >= tol * 0.99
    if precond == stokes.UZAWA:
        assert out.rel_res_precond == pytest.approx(out.rel_res, rel=1e-12)


# ---- aggregation multigrid inner preconditioner (oracle.amg) -------------------------
def test_amg_vcycle_is_symmetric_positive_definite():
    """The V-cycle with adjoint Jacobi pre/post-smoothing and the scaled coarse correction
    is a symmetric positive definite operator, for A and for S-hat (the property CG needs
    of a preconditioner)."""
    from oracle import amg
    m = synth.sphere_packing(8, 1.5, 2.5, 0.6, seed=2)
    prob = stokes.StokesProblem(m)
    for op, coords, gamma, n_last in ((prob.A, amg.face_coords(prob.geo), amg.GAMMA_A, 3),
                                      (prob.S_simple, amg.cell_coords(prob.geo), amg.GAMMA_S, 1)):
        levels = amg.build(op, coords)
        assert len(levels) == 4                      # 8^3 -> 4^3 -> 2^3 -> 1^3
        assert levels[-1].A.shape[0] == n_last       # one unknown per component
        n = op.shape[0]
        M = np.column_stack([amg.vcycle(levels, e, gamma) for e in np.eye(n)])
        assert np.abs(M - M.T).max() <= 1e-12 * np.abs(M).max()
        assert np.linalg.eigvalsh(0.5 * (M + M.T)).min() > 0


def test_amg_coarse_operator_of_the_empty_box():
    """Galerkin coarsening by 2 x 2 x 2 aggregates of the 7-point operator: on the empty
    periodic 8^3 box S-hat_simple is the 7-point Laplacian / 6, and the coarse operator
    is 4/6 times the 7-point Laplacian of the 4^3 box (each aggregate sums 8 x 6 - 24
    internal couplings = 24 on the diagonal, and 4 fine couplings cross each face)."""
    from oracle import amg
    prob = stokes.StokesProblem(np.ones((8, 8, 8), np.uint8))
    levels = amg.build(prob.S_simple, amg.cell_coords(prob.geo))
    Ac = levels[1].A.toarray()
    n = 4
    lap1 = 2 * np.eye(n) - np.roll(np.eye(n), 1, axis=0) - np.roll(np.eye(n), -1, axis=0)
    eye = np.eye(n)
    lap3 = (np.kron(np.kron(lap1, eye), eye) + np.kron(np.kron(eye, lap1), eye)
            + np.kron(np.kron(eye, eye), lap1))
    # coarse unknowns are ordered by (x, y, z) keys; the 3D Laplacian is symmetric in the
    # axes, so any consistent lexicographic order gives the same matrix
    np.testing.assert_allclose(Ac, (4.0 / 6.0) * lap3, atol=1e-12)


@pytest.mark.parametrize("phi", [0.4, 0.15])
def test_amg_pcg_reaches_the_jacobi_solution_in_fewer_iterations(phi):
    """Multigrid-preconditioned inner CG reaches the same A and S-hat solutions as the
    Jacobi-preconditioned one, in at least 2 (A; its condition number is bounded by the
    pore size) and 3 (S-hat) times fewer iterations."""
    m = synth.sphere_packing(24, 2.0, 4.0, phi, seed=3)
    prob = stokes.StokesProblem(m)
    b = mac.force(prob.geo, (1.0, 0.0, 0.0))
    rj = prob.solve_A(b, 1e-11, 20000)
    ra = prob.solve_A(b, 1e-11, 20000, stokes.INNER_AMG)
    assert ra.status == krylov.OK and 2 * ra.iters <= rj.iters
    np.testing.assert_allclose(ra.x, rj.x, atol=1e-9 * np.abs(rj.x).max())
    g = prob.B @ rj.x
    sj = prob.solve_simple(g, 1e-11, 20000)
    sa = prob.solve_simple(g, 1e-11, 20000, stokes.INNER_AMG)
    assert sa.status == krylov.OK and 3 * sa.iters <= sj.iters
    np.testing.assert_allclose(sa.x, sj.x, atol=1e-8 * np.abs(sj.x).max())


@pytest.mark.parametrize("precond", [stokes.UZAWA, stokes.SIMPLE])
def test_full_solve_with_amg_inner_solves(precond):
    """The whole path with multigrid inner solves gives the permeability of the Jacobi
    path (both converged to 1e-9 outer, 1e-12 inner)."""
    m = synth.sphere_packing(16, 2.0, 4.0, 0.35, seed=4)
    f = (1.0, 0.0, 0.0)
    rj = stokes.solve(m, f, stokes.Options(precond=precond, tol=1e-9))
    ra = stokes.solve(m, f, stokes.Options(precond=precond, tol=1e-9,
                                          inner_precond=stokes.INNER_AMG))
    assert ra["schur"].status == krylov.OK
    assert abs(ra["k"][0] - rj["k"][0]) <= 1e-8 * abs(rj["k"][0])
    assert ra["schur"].inner_iters_A < rj["schur"].inner_iters_A


def test_amg_isolated_pore_is_a_nullspace_unknown():
    """A fluid voxel with solid on every side is a pore of its own: its S-hat row is zero
    (diagonal mass 0) and its weight in smoothing and in the coarsest solve is 0; an
    aggregate that is a whole pore of two voxels has coarse diagonal 0 (its couplings stay
    inside the aggregate) and weight 0, although its diagonal mass is positive."""
    from oracle import amg
    m = np.ones((8, 8, 8), np.uint8)
    m[0:6, 0:6, 0:6] = 0
    m[1, 1, 1] = 1                              # isolated voxel
    m[2, 2, 2] = m[2, 2, 3] = 1                 # two-voxel pore inside aggregate (1, 1, 1)
    prob = stokes.StokesProblem(m)
    levels = amg.build(prob.S_simple, amg.cell_coords(prob.geo))
    c = prob.geo.pidx
    assert levels[0].dinv[c[1, 1, 1]] == 0.0 and levels[0].dinv[c[2, 2, 2]] > 0
    lone = levels[0].P[c[1, 1, 1]].indices[0]
    pair = levels[0].P[c[2, 2, 2]].indices[0]
    assert levels[0].P[c[2, 2, 3]].indices[0] == pair and pair != lone
    assert abs(levels[1].A[pair, pair]) <= 1e-15 and levels[1].dinv[pair] == 0.0
    assert levels[1].dinv[lone] == 0.0
    z = amg.vcycle(levels, np.ones(prob.geo.n_p), amg.GAMMA_S)
    assert z[c[1, 1, 1]] == 0.0
