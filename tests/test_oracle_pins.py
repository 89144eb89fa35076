"""Pins of the CPU oracle against facts fixed by the paper and by mathematics.

Each test ties one oracle function to something other than itself: closed
forms, the exact lattice Green's function, complex symmetry of the row-scaled
operator, dense brute-force solves, the boundary-value-problem form of the
transmission operators, the paper's printed index formulas, the m=1 special
case, the naive O(m^2) superposition and a brute-force minimal-residual
Krylov solution.  A plausible slip in the oracle (dropped term, wrong sign,
wrong half-point or layer index, transposed ordering, wrong trace side) fails
at least one of them.
"""
import math
import os

import numpy as np
import pytest
import scipy.sparse as sp

import workloads as W
from oracle import fgmres, operator, partition, pml, subproblems, sweeping

GOLD = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------- PML profile

def test_pml_profile_integral_and_edges():
    """sigma integrates to C/3 over each PML (quadratic profile of Section 2),
    vanishes on [eta, 1-eta] and reaches C/eta at the Dirichlet nodes."""
    n, gamma, C = 255, 16, 20.0
    g = pml.global_profile(n, gamma, C)
    h, eta = 1.0 / (n + 1), gamma / (n + 1)
    x = np.linspace(0.0, eta, 200001)
    integral = np.trapezoid(g.sigma(x), x)
    assert abs(integral - C / 3) < 1e-6 * C
    assert np.allclose(g.sigma(np.array([0.0, 1.0])), C / eta)
    inner = np.linspace(eta, 1 - eta, 101)
    assert np.all(g.sigma(inner) == 0.0)
    # s = (1 + i sigma/omega)^-1 has |s| <= 1 and Im s <= 0 where sigma > 0 (absorbing)
    s = g.s(np.linspace(0, 1, 1001), 10.0)
    assert np.all(np.abs(s) <= 1 + 1e-15) and np.all(s.imag <= 0)


# ------------------------------------------------------------- operator A

@pytest.mark.parametrize("dim,n", [(1, 40), (2, 12), (3, 6)])
def test_operator_sine_eigenpairs_without_pml(dim, n):
    """C = 0 (no PML), constant c: A sin-mode = lambda sin-mode with
    lambda = -(4/h^2) sum_j sin^2(pi k_j h/2) + omega^2/c^2 (Dirichlet Laplacian)."""
    omega, cval = 7.3, 1.3
    h = 1.0 / (n + 1)
    A = operator.helmholtz_matrix(dim, n, omega, np.full((n,) * dim, cval), 3, 0.0)
    rng = np.random.default_rng(0)
    for _ in range(3):
        ks = rng.integers(1, n + 1, size=dim)
        xs = W.grid_nodes(n, dim)
        mode = np.ones((n,) * dim)
        lam = omega**2 / cval**2
        for ax in range(dim):
            mode = mode * np.sin(math.pi * ks[ax] * xs[ax])
            lam -= 4.0 / h**2 * math.sin(math.pi * ks[ax] * h / 2) ** 2
        y = (A @ mode.reshape(-1)).reshape(mode.shape)
        assert np.allclose(y, lam * mode, rtol=1e-12, atol=1e-9 * abs(lam))


def test_operator_1d_matches_lattice_greens_function():
    """1D, constant c, PML on both ends: the solution of A u = delta_{i0}/h in the
    physical region equals the free-space outgoing lattice Green's function
    u_j = h e^{i theta |j-j0|} / (2 i sin theta), 2 cos theta = 2 - (omega h)^2,
    up to the PML's reflection.  An amplifying (sign-flipped) PML or a wrong
    scale fails this."""
    n, gamma, C = 511, 24, 20.0
    omega = 2 * math.pi * 16  # 32 points per wavelength
    h = 1.0 / (n + 1)
    A = operator.helmholtz_matrix(1, n, omega, np.ones(n), gamma, C)
    j0 = 200
    f = np.zeros(n, dtype=complex)
    f[j0 - 1] = 1.0 / h
    u = sp.linalg.spsolve(A.tocsc(), f)
    theta = math.acos(1 - (omega * h) ** 2 / 2)
    j = np.arange(1, n + 1)
    exact = h * np.exp(1j * theta * np.abs(j - j0)) / (2j * math.sin(theta))
    phys = (j >= gamma) & (j <= n + 1 - gamma)
    err = np.max(np.abs(u[phys] - exact[phys])) / np.max(np.abs(exact))
    assert err < 2e-3, err


@pytest.mark.parametrize("dim,n", [(1, 30), (2, 14), (3, 7)])
def test_row_scaled_operator_is_complex_symmetric(dim, n):
    """Section 3.1, practical remark 4: dividing row (i1,..) by s_{i1} s_{i2}..
    makes A complex symmetric (not Hermitian).  A misplaced half-point or a
    mismatched coefficient breaks the symmetry."""
    omega, gamma, C = 9.0, 3, 20.0
    c = W.lens_velocity(n, dim) if dim > 1 else np.linspace(0.9, 1.2, n)
    A = operator.helmholtz_matrix(dim, n, omega, c, gamma, C).toarray()
    g = pml.global_profile(n, gamma, C)
    s = g.s(np.arange(1, n + 1) / (n + 1), omega)
    d = np.ones((n,) * dim, dtype=complex)
    for ax in range(dim):
        shape = [1] * dim
        shape[dim - 1 - ax] = n
        d = d * s.reshape(shape)
    S = A / d.reshape(-1)[:, None]
    assert np.allclose(S, S.T, rtol=0, atol=1e-12 * np.abs(S).max())
    assert not np.allclose(S, S.conj().T, atol=1e-6 * np.abs(S).max())


# ----------------------------------------------------------- partition

def test_partition_matches_printed_index_formulas():
    rows = [ln.split() for ln in open(os.path.join(GOLD, "partition_gamma3_b2_m4.txt"))
            if ln.strip() and not ln.startswith("#")]
    part = partition.make_partition(12, 3, 2)
    assert part.m == 4
    for kind, p, lo, hi in rows:
        L = part.layers[int(p) - 1]
        got = {"X": (L.x_lo, L.x_hi), "M": (L.m_lo, L.m_hi), "R": (L.r_lo, L.r_hi),
               "L": (L.l_lo, L.l_hi)}[kind]
        assert got == (int(lo), int(hi)), (kind, p, got)


def test_partition_with_arbitrary_widths_matches_hand_evaluated_ranges():
    """Section 3.1, practical remark 3: layers of arbitrary widths (here 3, 1,
    4, 2 with a thinner auxiliary PML), ranges evaluated by hand
    (tests/golden/partition_widths_3142.txt)."""
    rows = [ln.split() for ln in open(os.path.join(GOLD, "partition_widths_3142.txt"))
            if ln.strip() and not ln.startswith("#")]
    part = partition.make_partition(14, 3, 1, gamma_a=2, widths=[3, 1, 4, 2])
    assert part.m == 4
    for kind, p, lo, hi in rows:
        L = part.layers[int(p) - 1]
        got = {"X": (L.x_lo, L.x_hi), "M": (L.m_lo, L.m_hi), "R": (L.r_lo, L.r_hi),
               "L": (L.l_lo, L.l_hi)}[kind]
        assert got == (int(lo), int(hi)), (kind, p, got)
    # equal widths with the remainder on the last layer reproduce the printed formulas
    u = partition.make_partition(40, 5, 4)
    w = partition.make_partition(40, 5, 4, widths=partition.uniform_widths(40, 5, 4))
    assert u.layers == w.layers
    with pytest.raises(ValueError):
        partition.make_partition(14, 3, 1, widths=[3, 1, 4, 1])  # does not sum to P


def _aux_fixture():
    """tests/golden/aux_pml_gamma4_ga2_b3.txt: padded grids and sigma*h/C of
    every subproblem at n=18, gamma=4, gamma_a=2, b=3, evaluated by hand from
    the printed piecewise profiles (Sections 2.1.1-2.1.3) with the thinner
    auxiliary width of Section 3.1, practical remark 2."""
    from fractions import Fraction
    grids, sig = {}, {}
    for ln in open(os.path.join(GOLD, "aux_pml_gamma4_ga2_b3.txt")):
        t = ln.split()
        if not t or t[0].startswith("#"):
            continue
        if t[0] == "G":
            grids[(t[1], int(t[2]))] = (int(t[3]), int(t[4]))
        else:
            sig.setdefault((t[1], int(t[2])), []).append((float(t[3]), float(Fraction(t[4]))))
    return grids, sig


def test_auxiliary_pml_profiles_match_printed_definitions():
    """sigma_q^M, sigma_p^R, sigma_p^L with a thinner auxiliary PML (gamma_a = 2
    against gamma = 4): the padded grids span beta + gamma_a - 1 and
    alpha - gamma_a + 1, the auxiliary sides grow as (C/eta_a)(d/eta_a)^2 with
    eta_a = gamma_a h, and the first layer's left side and the last layer's
    right side keep the boundary width.  Every node and half node of every
    subproblem, including the half nodes just outside its grid."""
    grids, sig = _aux_fixture()
    n, gamma, b, ga, C = 18, 4, 3, 2, 20.0
    part = partition.make_partition(n, gamma, b, ga)
    assert part.m == 4 and len(grids) == 10 and len(sig) == 10
    h = part.h
    for (kind, p), (lo, hi) in grids.items():
        L = part.layers[p - 1]
        got = {"M": (L.m_lo, L.m_hi), "R": (L.r_lo, L.r_hi), "L": (L.l_lo, L.l_hi)}[kind]
        assert got == (lo, hi), (kind, p, got)
        pts = sig[(kind, p)]
        assert [x for x, _ in pts] == [lo - 0.5 + 0.5 * j for j in range(2 * (hi - lo) + 3)]
        prof = partition.sweep_profile(part, p, kind, C)
        for x, v in pts:
            got_s = float(prof.sigma(np.array([x * h]))[0])
            assert abs(got_s - v * C / h) <= 1e-12 * C / h, (kind, p, x, got_s, v * C / h)


def test_auxiliary_subproblem_assembly_uses_printed_profiles():
    """1D H_p^kind assembled by the oracle equals the second difference of
    Eq. (2) built directly from the fixture's sigma values at nodes and half
    nodes (s = (1 + i sigma/omega)^-1), plus omega^2/c^2 on the diagonal."""
    grids, sig = _aux_fixture()
    n, gamma, b, ga, C, omega = 18, 4, 3, 2, 20.0, 11.0
    part = partition.make_partition(n, gamma, b, ga)
    h = part.h
    c = np.linspace(0.9, 1.1, n)
    for (kind, p), (lo, hi) in grids.items():
        s = {x: 1.0 / (1.0 + 1j * (v * C / h) / omega) for x, v in sig[(kind, p)]}
        w = hi - lo + 1
        H = np.zeros((w, w), dtype=complex)
        for j in range(w):
            i = lo + j
            up = s[i] * s[i + 0.5] / h**2
            dn = s[i] * s[i - 0.5] / h**2
            H[j, j] = -(up + dn) + omega**2 / c[i - 1] ** 2
            if j + 1 < w:
                H[j, j + 1] = up
            if j > 0:
                H[j, j - 1] = dn
        Ho = subproblems.subproblem_matrix(1, n, omega, c, gamma, C, part, p, kind).toarray()
        assert np.allclose(Ho, H, rtol=1e-13, atol=0), (kind, p)


def test_partition_experiment_layer_widths_and_remainder():
    """Section 3.2: gamma=9, b=8 gives a leftmost layer of b+gamma-1 = 16 nodes.
    Ragged case: the last layer absorbs the remainder and layers tile [1, n]."""
    part = partition.make_partition(40, 9, 8)
    L1 = part.layers[0]
    assert L1.x_hi - L1.x_lo + 1 == 16
    for n, gamma, b in [(127, 12, 4), (511, 16, 4), (1023, 20, 4), (95, 8, 4), (41, 5, 3)]:
        part = partition.make_partition(n, gamma, b)
        cover = []
        for L in part.layers:
            cover.extend(range(L.x_lo, L.x_hi + 1))
        assert cover == list(range(1, n + 1))
        P = n + 2 - 2 * gamma
        assert part.m == P // b
        last = part.layers[-1]
        assert last.phys_hi - last.phys_lo + 1 == b + P - part.m * b


# --------------------------------------------------------- subproblems

def _small(dim, n, omega, gamma, b, vel="lens"):
    P = W.small_problem(dim, n, omega, gamma, b, vel)
    part = partition.make_partition(n, gamma, b)
    return P, part


@pytest.mark.parametrize("dim,n,gamma,b", [(1, 25, 4, 3), (2, 17, 4, 3), (3, 9, 3, 2)])
def test_banded_lu_solve_matches_dense_solve(dim, n, gamma, b):
    """Every subproblem: the banded LU (quasi-1D ordering, partial pivoting)
    solves H v = g like a dense solve of H in the paper's natural ordering."""
    omega = 2 * math.pi * 2.5
    P, part = _small(dim, n, omega, gamma, b, "lens" if dim > 1 else "const")
    rng = np.random.default_rng(1)
    for p in range(1, part.m + 1):
        for kind in ("M", "R", "L"):
            if (kind == "R" and p == 1) or (kind == "L" and p == part.m):
                continue
            F = subproblems.factor_subproblem(dim, n, omega, P.c, gamma, P.C, part, p, kind)
            Hn = subproblems.subproblem_matrix(dim, n, omega, P.c, gamma, P.C, part, p, kind)
            g = rng.standard_normal((F.w, F.T)) + 1j * rng.standard_normal((F.w, F.T))
            v = F.solve(g)
            vd = np.linalg.solve(Hn.toarray(), g.reshape(-1)).reshape(g.shape)
            assert np.allclose(v, vd, rtol=0, atol=1e-11 * np.abs(vd).max())


def test_subproblems_without_pml_are_principal_submatrices():
    """C = 0: H_q^M, H_p^R, H_p^L are the Dirichlet truncations of A to their
    padded grids (same stencil, no auxiliary absorption)."""
    n, gamma, b, omega = 15, 3, 2, 5.0
    c = W.lens_velocity(n, 2)
    part = partition.make_partition(n, gamma, b)
    A = operator.helmholtz_matrix(2, n, omega, c, gamma, 0.0).toarray()
    for p in range(1, part.m + 1):
        L = part.layers[p - 1]
        for kind, (lo, hi) in (("M", (L.m_lo, L.m_hi)), ("R", (L.r_lo, L.r_hi)),
                               ("L", (L.l_lo, L.l_hi))):
            H = subproblems.subproblem_matrix(2, n, omega, c, gamma, 0.0, part, p, kind).toarray()
            idx = np.arange((lo - 1) * n, hi * n)
            assert np.allclose(H, A[np.ix_(idx, idx)], atol=1e-9)


@pytest.mark.parametrize("dim,n,gamma,b,gamma_a", [(1, 40, 4, 5, None), (2, 17, 4, 3, 2), (3, 9, 2, 2, None)])
def test_subproblem_rows_away_from_the_auxiliary_pml_equal_rows_of_A(dim, n, gamma, b, gamma_a):
    """C > 0: a row of H_p^M, H_p^R or H_p^L whose stencil stays inside the
    layer's PML-free columns (alpha_p .. beta_p) is the row of A, restricted to
    the subproblem's grid; so are the rows in the boundary PML of the first
    and last layers, which keep it unchanged (Section 3.1).  An auxiliary PML
    placed one column off, or the boundary PML of the end layers replaced by
    the auxiliary one, changes one of these rows."""
    omega, C = 9.0, 20.0
    c = W.lens_velocity(n, dim)
    part = partition.make_partition(n, gamma, b, gamma_a)
    A = operator.helmholtz_matrix(dim, n, omega, c, gamma, C).toarray()
    T = n ** (dim - 1)
    checked = 0
    for p in range(1, part.m + 1):
        L = part.layers[p - 1]
        first = 1 if p == 1 else L.phys_lo + 1
        last = n if p == part.m else L.phys_hi - 1
        for kind, (lo, hi) in (("M", (L.m_lo, L.m_hi)), ("R", (L.r_lo, L.r_hi)), ("L", (L.l_lo, L.l_hi))):
            if (kind == "R" and p == 1) or (kind == "L" and p == part.m):
                continue
            H = subproblems.subproblem_matrix(dim, n, omega, c, gamma, C, part, p, kind, order="natural").toarray()
            cols = np.arange((lo - 1) * T, hi * T)
            rows_g = np.arange((first - 1) * T, last * T)
            rows_l = rows_g - (lo - 1) * T
            outside = np.setdiff1d(np.arange(n ** dim), cols)
            assert np.all(A[np.ix_(rows_g, outside)] == 0)
            assert np.allclose(H[rows_l], A[np.ix_(rows_g, cols)], rtol=1e-13, atol=1e-9)
            checked += len(rows_l)
    assert checked > 0


def _bvp_solution(dim, n, omega, c, gamma, C, part, p, kind, w):
    """Independent form of G~_p^R w / G~_p^L w: the boundary value problem of
    Section 3.1 with v = w held on the boundary column (x2 = alpha_p - 1 for R,
    beta_p + 1 for L), assembled on the grid extended by that column, and
    solved densely."""
    L = part.layers[p - 1]
    lo, hi = (L.r_lo, L.r_hi) if kind == "R" else (L.l_lo, L.l_hi)
    elo, ehi = (lo - 1, hi) if kind == "R" else (lo, hi + 1)
    prof = partition.sweep_profile(part, p, kind, C)
    # sweep-axis operator on the extended range, with the subproblem's profile
    Ds = operator.second_difference(elo, ehi, n, prof, omega).toarray()
    Dt = operator.transverse_operator(dim, n, gamma, C, omega).toarray()
    T = n ** (dim - 1)
    we = ehi - elo + 1
    cc = np.asarray(c).reshape(n, T)[elo - 1:ehi]
    K = np.kron(Ds, np.eye(T)) + np.kron(np.eye(we), Dt) + np.diag((omega**2 / cc**2).reshape(-1))
    bcol = 0 if kind == "R" else we - 1
    rows = np.arange(we * T).reshape(we, T)
    K[rows[bcol]] = 0.0
    K[rows[bcol], rows[bcol]] = 1.0
    rhs = np.zeros(we * T, dtype=complex)
    rhs[rows[bcol]] = w
    v = np.linalg.solve(K, rhs).reshape(we, T)
    inner = v[1:] if kind == "R" else v[:-1]
    return inner[L.x_lo - lo: L.x_hi - lo + 1]


@pytest.mark.parametrize("dim", [1, 2, 3])
def test_transmission_operators_solve_the_boundary_value_problem(dim):
    """G~_p^R w (g = (-1/h^2)[w, 0, ...]) and G~_p^L w (g on the last column)
    equal the restriction to X_p of the Helmholtz solution on D_p^R / D_p^L
    with v = w on the left / right boundary and zero elsewhere (Section 3.1).
    A wrong sign, scale or side of g fails this."""
    n, gamma, b, omega, C = {1: (30, 4, 3, 12.0, 20.0), 2: (13, 3, 2, 9.0, 20.0), 3: (9, 2, 2, 6.0, 20.0)}[dim]
    c = np.linspace(0.9, 1.1, n) if dim == 1 else W.lens_velocity(n, dim)
    part = partition.make_partition(n, gamma, b)
    assert part.m >= 3
    rng = np.random.default_rng(3)
    T = n ** (dim - 1)
    for p in range(2, part.m):
        w = rng.standard_normal(T) + 1j * rng.standard_normal(T)
        for kind, G in (("R", subproblems.G_R), ("L", subproblems.G_L)):
            F = subproblems.factor_subproblem(dim, n, omega, c, gamma, C, part, p, kind)
            z = G(F, w, part.h)
            zb = _bvp_solution(dim, n, omega, c, gamma, C, part, p, kind, w)
            assert np.allclose(z, zb, rtol=0, atol=1e-10 * np.abs(zb).max()), (kind, p)


# ------------------------------------------------------ preconditioner

@pytest.mark.parametrize("dim,n,gamma,b", [(1, 40, 4, 3), (2, 23, 4, 3), (3, 11, 3, 2)])
def test_accumulated_sweep_equals_naive_superposition(dim, n, gamma, b):
    """Section 2.2: accumulating boundary values gives exactly (by linearity)
    the O(m^2) superposition u~_p = sum_q u~_{p,q} of Section 2.1."""
    omega = 2 * math.pi * 2.0
    P = W.small_problem(dim, n, omega, gamma, b, "lens" if dim > 1 else "const", nrhs=2)
    pc = sweeping.Preconditioner(dim, n, omega, P.c, gamma, b, P.C)
    assert pc.m >= 3
    z1 = pc.apply(P.f)
    z2 = pc.apply_naive(P.f)
    assert np.linalg.norm(z1 - z2) <= 1e-12 * np.linalg.norm(z1)


@pytest.mark.parametrize("dim,n,gamma,widths", [(1, 40, 4, [2, 7, 1, 5, 3, 6, 3, 7]), (2, 23, 4, [2, 5, 1, 4, 5]),
                                                 (3, 11, 3, [1, 3, 3])])
def test_accumulated_sweep_with_arbitrary_widths_equals_naive_superposition(dim, n, gamma, widths):
    """The same identity with layers of arbitrary widths (Section 3.1, practical
    remark 3), including one-column layers, and with the subproblems of such
    layers solving their boundary value problems."""
    omega = 2 * math.pi * 2.0
    assert sum(widths) == n + 2 - 2 * gamma
    P = W.small_problem(dim, n, omega, gamma, 1, "lens" if dim > 1 else "const", nrhs=2)
    pc = sweeping.Preconditioner(dim, n, omega, P.c, gamma, 1, P.C, widths=widths)
    assert pc.m == len(widths)
    z1 = pc.apply(P.f)
    z2 = pc.apply_naive(P.f)
    assert np.linalg.norm(z1 - z2) <= 1e-12 * np.linalg.norm(z1)
    part = pc.part
    rng = np.random.default_rng(3)
    T = n ** (dim - 1)
    for p, kind in ((2, "R"), (part.m - 1, "L")):
        F = pc.FR[p] if kind == "R" else pc.FL[p]
        w = rng.standard_normal(T) + 1j * rng.standard_normal(T)
        got = (subproblems.G_R if kind == "R" else subproblems.G_L)(F, w, part.h)
        ref = _bvp_solution(dim, n, omega, P.c, gamma, P.C, part, p, kind, w)
        assert np.allclose(got, ref, rtol=1e-10, atol=1e-12 * np.abs(ref).max())


@pytest.mark.parametrize("dim,n", [(1, 20), (2, 11), (3, 7)])
def test_single_layer_preconditioner_is_exact_inverse(dim, n):
    """m = 1: X_1 is the whole grid with the boundary PML on both sides, so
    H_1^M = A and the preconditioner is A^-1; FGMRES converges in 1 iteration."""
    gamma, omega = 4, 6.0
    b = n + 2 - 2 * gamma  # all physical nodes in one layer
    c = W.lens_velocity(n, dim) if dim > 1 else np.ones(n)
    pc = sweeping.Preconditioner(dim, n, omega, c, gamma, b)
    assert pc.m == 1
    A = operator.helmholtz_matrix(dim, n, omega, c, gamma, 20.0)
    rng = np.random.default_rng(5)
    f = rng.standard_normal((n,) * dim) + 1j * rng.standard_normal((n,) * dim)
    z = pc.apply(f)
    ref = np.linalg.solve(A.toarray(), f.reshape(-1)).reshape(f.shape)
    assert np.allclose(z, ref, atol=1e-11 * np.abs(ref).max())
    u, its, res = fgmres.solve(pc, A, f[..., None], tol=1e-10)
    assert its[0] == 1 and res[0] < 1e-10


def test_preconditioner_approximates_the_green_operator():
    """The sweeping preconditioner approximates A^-1 (Section 2: each piece is
    an outgoing wave through absorbing layers): for constant c its error is far
    below 1, while a wrong trace side or sweep direction gives O(1) error."""
    n, gamma, b = 63, 8, 4
    omega = (n + 1) * math.pi / 8
    P = W.small_problem(2, n, omega, gamma, b, "const", nrhs=1)
    pc = sweeping.Preconditioner(2, n, omega, P.c, gamma, b, P.C)
    A = operator.helmholtz_matrix(2, n, omega, P.c, gamma, P.C)
    f = P.f[..., 0]
    u = sp.linalg.spsolve(A.tocsc(), f.reshape(-1)).reshape(f.shape)
    z = pc.apply(f)
    assert np.linalg.norm(z - u) / np.linalg.norm(u) < 0.05


# --------------------------------------------------------------- FGMRES

def test_givens_rotation_is_unitary_and_annihilates():
    """The complex Givens rotation of the FGMRES least-squares update: the
    2 x 2 matrix [[c, s], [-conj(s), c]] is unitary, maps (a, b) to (r, 0) with
    |r| = |(a, b)|, and keeps the phase of a (r = e^{i arg a} |(a, b)|), also
    when a or b is zero."""
    rng = np.random.default_rng(11)
    pairs = [(complex(*rng.standard_normal(2)), complex(*rng.standard_normal(2))) for _ in range(20)]
    pairs += [(1.5 - 2j, 0j), (0j, -0.3 + 0.4j), (0j, 0j), (1e-300 + 0j, 1.0 + 0j)]
    for a, b in pairs:
        c, s = fgmres.givens(a, b)
        G = np.array([[c, s], [-np.conj(s), c]])
        assert abs(np.imag(c)) == 0.0
        assert np.allclose(G @ G.conj().T, np.eye(2), atol=1e-14)
        r, zero = G @ np.array([a, b])
        rho = math.hypot(abs(a), abs(b))
        assert abs(zero) <= 1e-14 * max(rho, 1e-300)
        assert math.isclose(abs(r), rho, rel_tol=1e-14, abs_tol=1e-300)
        if a != 0 and rho > 0:
            assert abs(r - rho * a / abs(a)) <= 1e-14 * rho


@pytest.mark.parametrize("dim,n", [(2, 9), (3, 5)])
def test_matrix_free_apply_handles_single_and_batched_fields(dim, n):
    """apply_A on a sine eigenmode (C = 0, constant c) returns lambda times
    the mode, for one grid function and for a batch with a trailing
    right-hand-side axis whose columns are different modes."""
    omega, cval = 5.1, 0.9
    h = 1.0 / (n + 1)
    c = np.full((n,) * dim, cval)
    xs = W.grid_nodes(n, dim)
    modes, lams = [], []
    for ks in ([1] * dim, [2] + [1] * (dim - 1), [n] * dim):
        mode = np.ones((n,) * dim)
        lam = omega**2 / cval**2
        for ax in range(dim):
            mode = mode * np.sin(math.pi * ks[ax] * xs[ax])
            lam -= 4.0 / h**2 * math.sin(math.pi * ks[ax] * h / 2) ** 2
        modes.append(mode)
        lams.append(lam)
    y0 = operator.apply_A(dim, n, omega, c, 3, 0.0, modes[0])
    assert y0.shape == modes[0].shape
    assert np.allclose(y0, lams[0] * modes[0], rtol=1e-12, atol=1e-9 * abs(lams[0]))
    batch = np.stack(modes, axis=-1).astype(np.complex128)
    yb = operator.apply_A(dim, n, omega, c, 3, 0.0, batch)
    assert yb.shape == batch.shape
    for r, lam in enumerate(lams):
        assert np.allclose(yb[..., r], lam * modes[r], rtol=1e-12, atol=1e-9 * abs(lam))


def test_fgmres_identity_preconditioner_is_minimal_residual():
    """With M = I, FGMRES after k steps returns the minimal-residual vector of
    the Krylov space span{f, Af, ..., A^{k-1} f}; compare with a brute-force
    least-squares solve over an explicit (orthonormalised) Krylov basis."""
    rng = np.random.default_rng(11)
    N = 40
    A = rng.standard_normal((N, N)) + 1j * rng.standard_normal((N, N)) + 6 * np.eye(N)
    f = rng.standard_normal(N) + 1j * rng.standard_normal(N)
    for k in (1, 3, 7):
        x, its, _ = fgmres.fgmres(lambda v: A @ v, lambda v: v, f, fixed_iters=k)
        K = np.stack([np.linalg.matrix_power(A, j) @ f for j in range(k)], axis=1)
        Q, _ = np.linalg.qr(K)
        y, *_ = np.linalg.lstsq(A @ Q, f, rcond=None)
        xb = Q @ y
        assert its == k
        assert np.allclose(x, xb, atol=1e-10 * np.abs(xb).max())


def test_fgmres_restart_and_convergence_against_dense_solve():
    rng = np.random.default_rng(12)
    N = 60
    A = rng.standard_normal((N, N)) + 1j * rng.standard_normal((N, N)) + 12 * np.eye(N)
    f = rng.standard_normal(N) + 1j * rng.standard_normal(N)
    x, its, hist = fgmres.fgmres(lambda v: A @ v, lambda v: v, f, tol=1e-10, restart=5, maxit=400)
    ref = np.linalg.solve(A, f)
    assert np.linalg.norm(A @ x - f) / np.linalg.norm(f) <= 1e-10 * 1.01
    assert np.allclose(x, ref, atol=1e-8 * np.abs(ref).max())
    assert its > 5  # needed at least one restart


def test_preconditioned_solve_matches_direct_solve():
    n, gamma, b = 31, 5, 3
    omega = (n + 1) * math.pi / 8
    P = W.small_problem(2, n, omega, gamma, b, "layered", nrhs=2)
    pc = sweeping.Preconditioner(2, n, omega, P.c, gamma, b, P.C)
    A = operator.helmholtz_matrix(2, n, omega, P.c, gamma, P.C)
    u, its, res = fgmres.solve(pc, A, P.f, tol=1e-10)
    for r in range(2):
        ref = sp.linalg.spsolve(A.tocsc(), P.f[..., r].reshape(-1)).reshape(P.f.shape[:-1])
        assert res[r] <= 1e-10 * 1.01
        assert np.linalg.norm(u[..., r] - ref) / np.linalg.norm(ref) < 1e-7
        assert its[r] <= 12


def test_iteration_counts_small_and_nearly_frequency_independent():
    """Soft check at the workloads' setting (16 points per wavelength, tolerance
    1e-6): iteration counts stay small and grow at most slowly with omega."""
    counts = []
    for n in (63, 127, 255):
        gamma = {63: 8, 127: 12, 255: 14}[n]
        omega = (n + 1) * math.pi / 8
        P = W.small_problem(2, n, omega, gamma, 4, "const", nrhs=1)
        pc = sweeping.Preconditioner(2, n, omega, P.c, gamma, 4, P.C)
        A = operator.helmholtz_matrix(2, n, omega, P.c, gamma, P.C)
        _, its, res = fgmres.solve(pc, A, P.f, tol=1e-6)
        counts.append(int(its[0]))
        assert res[0] <= 1e-6
    assert max(counts) <= 10 and max(counts) - min(counts) <= 3, counts


def _paper_iteration_tables():
    """tests/golden/iteration_counts_tables.txt: the GMRES iteration counts of
    Tables 1-3 (2D) as {n: [counts over the three velocities and two forces]}."""
    out = {}
    for ln in open(os.path.join(GOLD, "iteration_counts_tables.txt")):
        t = ln.split()
        if not t or t[0].startswith("#") or t[0] != "2":
            continue
        out.setdefault(int(t[3]), []).extend([int(t[4]), int(t[5])])
    return out


def test_iteration_counts_within_the_papers_tables():
    """Soft check against Tables 1-3 at the paper's own setting (Section 3.2:
    8 points per wavelength, so omega/(2 pi) = (n+1)/8; boundary and auxiliary
    PML gamma = 9; b = 8; relative residual 1e-3; restart 40).  The paper's
    velocity fields are not published, so the oracle runs its synthetic lens
    with a Gaussian point source and is held to the tables' envelope: at each
    n no more iterations than the largest count the tables print for that n,
    and from n to 2n + 1 no faster growth than the tables' largest growth
    between the same two sizes."""
    tab = _paper_iteration_tables()
    sizes = (127, 255, 511)
    counts = {}
    for n in sizes:
        omega = 2 * math.pi * (n + 1) / 8
        P = W.small_problem(2, n, omega, 9, 8, "lens", nrhs=1)
        pc = sweeping.Preconditioner(2, n, omega, P.c, 9, 8, P.C)
        A = operator.helmholtz_matrix(2, n, omega, P.c, 9, P.C)
        _, its, res = fgmres.solve(pc, A, P.f, tol=1e-3, restart=40)
        assert res[0] <= 1e-3
        counts[n] = int(its[0])
        assert 1 <= counts[n] <= max(tab[n]), (n, counts[n], tab[n])
    for a, b in zip(sizes, sizes[1:]):
        growth = max(tb - ta for ta, tb in zip(tab[a], tab[b]))
        assert counts[b] - counts[a] <= max(growth, 1), (counts, growth)


# ---- nested dissection of the 3D slab subproblems (Section 4)

@pytest.mark.parametrize("name,n,gamma,b,gamma_a", [("ragged", 13, 3, 4, None), ("thin_aux", 15, 4, 3, 2)])
def test_nested_dissection_solve_equals_sparse_direct_solve(name, n, gamma, b, gamma_a):
    """Section 4 solves each slab subproblem by nested dissection after grouping
    the unknowns along x3; the result is H^-1 g, so it must equal a sparse
    direct solve (scipy's LU) of the same slab matrix for every H_q^M, H_p^R,
    H_p^L of a 3D partition."""
    import scipy.sparse.linalg as spl
    from oracle import nested_dissection as nd
    P = W.small_problem(3, n, 3 * math.pi, gamma, b, "bump", nrhs=1, pml_aux=gamma_a)
    part = partition.make_partition(P.n, P.pml, P.b, gamma_a)
    rng = np.random.default_rng(11)
    for p in range(1, part.m + 1):
        for kind in "MRL":
            if (kind == "R" and p == 1) or (kind == "L" and p == part.m):
                continue
            H = subproblems.subproblem_matrix(3, P.n, P.omega, P.c, P.pml, P.C, part, p, kind, order="natural")
            w = H.shape[0] // (P.n * P.n)
            g = rng.standard_normal((H.shape[0], 2)) + 1j * rng.standard_normal((H.shape[0], 2))
            x = nd.solve(nd.factor(H, P.n, w), g)
            xr = spl.spsolve(H.tocsc(), g)
            assert np.abs(x - xr).max() <= 1e-11 * np.abs(xr).max(), (p, kind)


@pytest.mark.parametrize("n", [3, 5, 9, 13, 20])
def test_nested_dissection_tree_is_a_dissection(n):
    """Brute force on small grids: every column is owned by exactly one node;
    a node's two children lie on either side of its separator line, so no
    4-neighbour pair of columns joins the two children's regions; and every
    leaf region holds at most 8 columns."""
    from oracle import nested_dissection as nd
    nodes = nd.separator_tree(n, 8)
    owned = [c for t in nodes for c in t.own]
    assert sorted(owned) == list(range(n * n))
    for t in nodes:
        x0, x1, y0, y1 = t.region
        if not t.children:
            assert (x1 - x0) * (y1 - y0) <= 8 and len(t.own) == (x1 - x0) * (y1 - y0)
            continue
        a, b = (nodes[c].region for c in t.children)
        ra = {(x, y) for y in range(a[2], a[3]) for x in range(a[0], a[1])}
        rb = {(x, y) for y in range(b[2], b[3]) for x in range(b[0], b[1])}
        sep = {(c % n, c // n) for c in t.own}
        assert ra | rb | sep == {(x, y) for y in range(y0, y1) for x in range(x0, x1)}
        assert not (ra & rb) and not (ra & sep) and not (rb & sep)
        for (x, y) in ra:
            for q in ((x + 1, y), (x - 1, y), (x, y + 1), (x, y - 1)):
                assert q not in rb
