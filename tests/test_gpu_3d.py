"""3D slab path (Section 4) on the GPU against the oracle.

Small grids: the 7-point matvec, every H_q^M, H_p^R, H_p^L slab solve, the
preconditioner apply and FGMRES, element by element against the oracle's
banded-LU reference (same tolerances as the 2D parity tests: the complex128
path differs from the oracle only in the order of rounding; the complex64 path
rounds factors and applies to FP32).  The 95^3 workload is too large for the
oracle's banded LU, so it is checked by properties that hold at any size: the
residual of slab solves against the assembled slab operator, and the FP64 true
residual of the FGMRES solution.  Both slab solvers run every case: block
elimination over the x2 planes ("block") and nested dissection of the slab's
column grid ("nd", Section 4); both are exact, so they share the oracle and the
tolerances.
"""
import math

import numpy as np
import pytest

import workloads as W
from parity_metrics import emax, rel
from oracle import fgmres, operator, partition, subproblems, sweeping

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

SMALL3 = {
    # name: (n, omega, gamma, b, velocity, nrhs, gamma_aux)
    "ragged_bump": (15, 3 * math.pi, 3, 3, "bump", 2, None),     # m = 3, last layer 5 planes
    "five_layers_lens": (19, 4 * math.pi, 3, 3, "lens", 1, None),  # m = 5
    "one_layer": (11, 2 * math.pi, 3, 7, "const", 1, None),       # m = 1: H^M is A itself
    "two_layers": (13, 3 * math.pi, 3, 4, "bump", 1, None),       # m = 2
    "five_rhs": (13, 3 * math.pi, 3, 3, "lens", 5, None),         # right-hand sides 4 + 1
    "thin_aux": (17, 4 * math.pi, 4, 3, "bump", 2, 2),            # auxiliary PML of 2 points
    "wide_blocks": (25, 4 * math.pi, 3, 10, "bump", 2, None),     # blocks of 350 / 300: two outer blocks
}


@pytest.fixture(scope="module", autouse=True)
def gpu():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1504_04058_gb300 import build
    build.build()
    yield


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.complex128)).to("cuda")


def host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()




def small3(name):
    n, om, g, b, vel, R, ga = SMALL3[name]
    return W.small_problem(3, n, om, g, b, vel, nrhs=R, pml_aux=ga)


SOLVERS = ["block", "nd"]


def handle3(P, precision="c128", max_rhs=None, restart=40, solver="block"):
    import paper_1504_04058_gb300 as asp
    prm = asp.make_params(P.n, P.omega, P.pml, P.b, pml_aux=P.pml_aux or 0, C=P.C, precision=precision,
                          max_rhs=max_rhs or P.nrhs, restart=restart, dim=3, slab_solver=solver)
    h = asp.asp_setup(P.c, prm)
    h.factor()
    return h


def oracle_pc3(P):
    return sweeping.Preconditioner(3, P.n, P.omega, P.c, P.pml, P.b, P.C, gamma_a=P.pml_aux)


@pytest.mark.parametrize("name", ["ragged_bump", "five_rhs"])
def test_matvec3d_matches_oracle(name):
    P = small3(name)
    h = handle3(P)
    rng = np.random.default_rng(0)
    x = rng.standard_normal(P.f.shape) + 1j * rng.standard_normal(P.f.shape)
    y = host(h.matvec(dev(x)))
    A = operator.helmholtz_matrix(3, P.n, P.omega, P.c, P.pml, P.C)
    yo = (A @ x.reshape(P.n ** 3, -1)).reshape(x.shape)
    assert emax(y, yo) <= 1e-13, (emax(y, yo), rel(y, yo))


@pytest.mark.parametrize("solver", SOLVERS)
@pytest.mark.parametrize("precision,tol", [("c128", 1e-11), ("c64", 2e-4)])
@pytest.mark.parametrize("name", ["ragged_bump", "two_layers", "thin_aux", "wide_blocks"])
def test_slab_solves_match_oracle(name, precision, tol, solver):
    """Every slab: GPU slab solve (block inverses or nested dissection) vs the
    oracle's banded LU."""
    import paper_1504_04058_gb300 as asp
    P = small3(name)
    h = handle3(P, precision, max_rhs=3, solver=solver)
    part = partition.make_partition(P.n, P.pml, P.b, P.pml_aux)
    rng = np.random.default_rng(1)
    worst = 0.0
    for p in range(1, part.m + 1):
        for kind, code in (("M", asp.KIND_M), ("R", asp.KIND_R), ("L", asp.KIND_L)):
            if (kind == "R" and p == 1) or (kind == "L" and p == part.m):
                continue
            F = subproblems.factor_subproblem(3, P.n, P.omega, P.c, P.pml, P.C, part, p, kind)
            assert h.subproblem_width(code, p) == F.w
            shape = (F.w, P.n, P.n, 3)
            g = rng.standard_normal(shape) + 1j * rng.standard_normal(shape)
            v = host(h.subproblem_solve(code, p, dev(g)))
            vo = F.solve(g.reshape(F.w, P.n * P.n, 3)).reshape(shape)
            worst = max(worst, emax(v, vo))
    assert worst <= tol, worst


@pytest.mark.parametrize("solver", SOLVERS)
@pytest.mark.parametrize("precision,tol", [("c128", 1e-10), ("c64", 2e-4)])
@pytest.mark.parametrize("name", list(SMALL3))
def test_apply3d_matches_oracle(name, precision, tol, solver):
    P = small3(name)
    h = handle3(P, precision, solver=solver)
    z = host(h.apply_preconditioner(dev(P.f)))
    zo = oracle_pc3(P).apply(P.f)
    assert emax(z, zo) <= tol, (emax(z, zo), rel(z, zo))


def test_apply3d_right_hand_sides_independent():
    P = small3("five_rhs")
    h = handle3(P, "c128")
    z_all = host(h.apply_preconditioner(dev(P.f)))
    for r in (0, 3, 4):
        z1 = host(h.apply_preconditioner(dev(P.f[..., r:r + 1])))
        assert emax(z1[..., 0], z_all[..., r], single=True) <= 1e-12, rel(z1[..., 0], z_all[..., r])


@pytest.mark.parametrize("solver", SOLVERS)
def test_fgmres3d_fp64_parity_and_iteration_counts(solver):
    P = W.small_problem(3, 19, 4 * math.pi, 3, 3, "bump", nrhs=2)
    pc = oracle_pc3(P)
    A = operator.helmholtz_matrix(3, P.n, P.omega, P.c, P.pml, P.C)
    uo, itso, _ = fgmres.solve(pc, A, P.f, tol=P.tol, restart=P.restart)
    k = int(itso.max())
    uk, _, _ = fgmres.solve(pc, A, P.f, tol=P.tol, restart=P.restart, fixed_iters=k)
    h = handle3(P, "c128", solver=solver)
    ug, _ = h.gmres_solve(dev(P.f), tol=0.0, maxit=k)
    assert emax(host(ug), uk) <= 1e-9, (emax(host(ug), uk), rel(host(ug), uk))
    ug, info = h.gmres_solve(dev(P.f), tol=P.tol, maxit=200)
    u = host(ug)
    for r in range(P.nrhs):
        assert abs(info[r]["iterations"] - int(itso[r])) <= 1, (info[r], itso[r])
        fr = P.f[..., r].reshape(-1)
        assert np.linalg.norm(fr - A @ u[..., r].reshape(-1)) / np.linalg.norm(fr) <= P.tol


def test_fgmres3d_c64_reaches_fp64_tolerance():
    P = W.small_problem(3, 19, 4 * math.pi, 3, 3, "lens", nrhs=2)
    A = operator.helmholtz_matrix(3, P.n, P.omega, P.c, P.pml, P.C)
    h = handle3(P, "c64")
    ug, info = h.gmres_solve(dev(P.f), tol=P.tol, maxit=200)
    u = host(ug)
    for r in range(P.nrhs):
        assert info[r]["converged"]
        fr = P.f[..., r].reshape(-1)
        assert np.linalg.norm(fr - A @ u[..., r].reshape(-1)) / np.linalg.norm(fr) <= P.tol


@pytest.mark.parametrize("solver", SOLVERS)
def test_3d_n95_workload_properties(solver):
    """The 95^3 workload (complex64 factors): slab solves leave a small residual
    against the assembled slab operator, and FGMRES reaches the FP64 true
    residual 1e-6."""
    import paper_1504_04058_gb300 as asp
    P = W.problem_3d_n95_bump()
    h = handle3(P, "c64", max_rhs=1, solver=solver)
    part = partition.make_partition(P.n, P.pml, P.b, None)
    rng = np.random.default_rng(3)
    for kind, code, p in (("M", asp.KIND_M, 1), ("M", asp.KIND_M, part.m // 2), ("R", asp.KIND_R, part.m),
                          ("L", asp.KIND_L, 1)):
        w = h.subproblem_width(code, p)
        g = rng.standard_normal((w, P.n, P.n, 1)) + 1j * rng.standard_normal((w, P.n, P.n, 1))
        v = host(h.subproblem_solve(code, p, dev(g)))
        Hs = subproblems.subproblem_matrix(3, P.n, P.omega, P.c, P.pml, P.C, part, p, kind, order="natural")
        res = np.linalg.norm(Hs @ v.reshape(-1) - g.reshape(-1)) / np.linalg.norm(g)
        assert res <= 1e-3, (kind, p, res)
    ug, info = h.gmres_solve(dev(P.f), tol=P.tol, maxit=200)
    u = host(ug)
    A = operator.helmholtz_matrix(3, P.n, P.omega, P.c, P.pml, P.C)
    fr = P.f[..., 0].reshape(-1)
    assert info[0]["converged"]
    assert np.linalg.norm(fr - A @ u[..., 0].reshape(-1)) / np.linalg.norm(fr) <= P.tol


def test_apply3d_wave_packet_sources():
    P = W.small_problem(3, 19, 4 * math.pi, 3, 3, "bump", nrhs=2, source="packet")
    h = handle3(P, "c128")
    z = host(h.apply_preconditioner(dev(P.f)))
    zo = oracle_pc3(P).apply(P.f)
    assert emax(z, zo) <= 1e-10, (emax(z, zo), rel(z, zo))


@pytest.mark.parametrize("name", ["ragged_bump", "wide_blocks", "five_rhs"])
def test_nested_dissection_equals_block_elimination(name):
    """Both slab solvers are exact, so their complex128 applies agree to rounding."""
    P = small3(name)
    zb = host(handle3(P, "c128", solver="block").apply_preconditioner(dev(P.f)))
    zn = host(handle3(P, "c128", solver="nd").apply_preconditioner(dev(P.f)))
    assert emax(zn, zb) <= 1e-11, (emax(zn, zb), rel(zn, zb))


def test_nested_dissection_refactor_and_reuse():
    """A second factorization on the same handle (the work area and pivot tables
    reused) gives the same apply, and two applies in a row agree."""
    P = small3("wide_blocks")
    h = handle3(P, "c128", solver="nd")
    z1 = host(h.apply_preconditioner(dev(P.f)))
    h.factor()
    z2 = host(h.apply_preconditioner(dev(P.f)))
    z3 = host(h.apply_preconditioner(dev(P.f)))
    assert emax(z2, z1) <= 1e-14 and emax(z3, z2) == 0.0


def test_nested_dissection_tensor_core_fronts():
    """One layer of n = 39 (H^M is A itself, w = 39): the top fronts have 1521
    and 2262 unknowns, so their complex64 updates run on the tensor cores.  The
    solution's residual against the oracle's assembled A, and its difference
    from the block-elimination solve, stay at complex64 accuracy."""
    P = W.small_problem(3, 39, 6 * math.pi, 3, 33, "bump", nrhs=2)
    A = operator.helmholtz_matrix(3, P.n, P.omega, P.c, P.pml, P.C)
    zn = host(handle3(P, "c64", solver="nd").apply_preconditioner(dev(P.f)))
    zb = host(handle3(P, "c64", solver="block").apply_preconditioner(dev(P.f)))
    for r in range(P.nrhs):
        fr = P.f[..., r].reshape(-1)
        res = np.linalg.norm(A @ zn[..., r].reshape(-1) - fr) / np.linalg.norm(fr)
        assert res <= 1e-4, (r, res)
    assert emax(zn, zb) <= 2e-4, (emax(zn, zb), rel(zn, zb))
