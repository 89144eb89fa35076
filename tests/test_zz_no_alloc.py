"""The allocation-free residual check (asp_residual_norms_noalloc).

Callers that cannot allocate device memory -- a process whose device memory
belongs to another allocator, or a serving loop that must not allocate once it
runs -- use this entry point to measure ||f - A u|| / ||f||.  It must agree
with the handle-based path (asp_matvec's A u, from which the same relative
residual follows) and with the oracle's assembled A.  Two calls in a row check
that the shared fixed scratch array carries no state from one call into the
next.  This file is collected last so that a failure here does not stop the
other GPU tests in a run that stops at the first failure.
"""
import math

import numpy as np
import pytest

import workloads as W
from oracle import operator

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

# both library paths are FP64 with the same per-element operation order; they
# differ only in the rounding of the PML weights and in the reduction order
TOL = 1e-12


def _rel_from_matvec(h, f, u):
    y = h.matvec(u)
    r = (f - y).cpu().numpy()
    fn = f.cpu().numpy()
    R = r.shape[-1]
    return np.array([np.linalg.norm(r[..., k]) / np.linalg.norm(fn[..., k]) for k in range(R)])


def _rel_from_oracle(P, u):
    """The same residual with the oracle's assembled A (CPU, FP64)."""
    A = operator.helmholtz_matrix(2, P.n, P.omega, P.c, P.pml, P.C)
    un = u.cpu().numpy().reshape(P.n * P.n, -1)
    fn = P.f.reshape(P.n * P.n, -1)
    return np.linalg.norm(fn - A @ un, axis=0) / np.linalg.norm(fn, axis=0)


def _setup():
    assert torch.cuda.is_available(), "GPU test needs a CUDA device"
    from paper_1504_04058_gb300 import build
    build.build()
    import paper_1504_04058_gb300 as asp
    return asp


def test_residual_norms_noalloc_matches_handle_path_and_oracle():
    asp = _setup()
    P = W.small_problem(2, 63, 8 * math.pi, 8, 4, "layered", nrhs=5)
    prm = asp.make_params(P.n, P.omega, P.pml, P.b, C=P.C, precision="c128", max_rhs=P.nrhs, restart=20)
    h = asp.asp_setup(P.c, prm)
    c = torch.from_numpy(np.ascontiguousarray(P.c)).to("cuda")
    f = torch.from_numpy(P.f).to("cuda")
    rng = np.random.default_rng(4)
    cases = []
    # an arbitrary vector (no cancellation in f - A u) and an FGMRES solution
    # (residual ~1e-8 of ||f||)
    cases.append(torch.from_numpy(rng.standard_normal(P.f.shape) + 1j * rng.standard_normal(P.f.shape)).to("cuda"))
    h.factor()
    u_sol, info = h.gmres_solve(f, tol=1e-8, maxit=100)
    cases.append(u_sol)
    for k, u in enumerate(cases):
        ref = _rel_from_matvec(h, f, u)
        orc = _rel_from_oracle(P, u)
        for call in range(2):
            out = asp.asp_residual_norms_noalloc(prm, c, f, u)
            got = out.cpu().numpy()
            if k == 0:
                assert np.allclose(got, ref, rtol=TOL, atol=0), (call, got, ref)
                assert np.allclose(got, orc, rtol=1e-11, atol=0), (call, got, orc)
            else:
                # at a converged solution the residual is cancellation-dominated:
                # compare with the solver's own true residual and the oracle's at
                # the solution's accuracy
                true = np.array([i["rel_res_true"] for i in info])
                assert np.all(got <= 1e-8 * 1.0001), got
                assert np.allclose(got, true, rtol=1e-4), (got, true)
                assert np.allclose(got, orc, rtol=1e-4), (got, orc)
    h.destroy()


def test_residual_norms_noalloc_at_the_largest_rhs_count():
    """nrhs = 64 (the scratch array's limit): every right-hand side of a block
    of 256 threads, and the 64-thread finishing kernel fully used."""
    asp = _setup()
    from paper_1504_04058_gb300 import _lib
    P = W.small_problem(2, 31, 4 * math.pi, 4, 3, "lens", nrhs=_lib.NOALLOC_MAX_RHS)
    prm = asp.make_params(P.n, P.omega, P.pml, P.b, C=P.C, precision="c128", max_rhs=P.nrhs, restart=4)
    h = asp.asp_setup(P.c, prm)
    c = torch.from_numpy(np.ascontiguousarray(P.c)).to("cuda")
    f = torch.from_numpy(P.f).to("cuda")
    rng = np.random.default_rng(5)
    u = torch.from_numpy(rng.standard_normal(P.f.shape) + 1j * rng.standard_normal(P.f.shape)).to("cuda")
    ref = _rel_from_matvec(h, f, u)
    orc = _rel_from_oracle(P, u)
    for _ in range(2):
        got = asp.asp_residual_norms_noalloc(prm, c, f, u).cpu().numpy()
        assert got.shape == (64,)
        assert np.allclose(got, ref, rtol=TOL, atol=0)
        assert np.allclose(got, orc, rtol=1e-11, atol=0)
    h.destroy()


def test_residual_norms_noalloc_flags_an_invalid_velocity():
    """A velocity entry that is not positive gives NaN for every right-hand
    side; the next call with a valid velocity is unaffected (the flag is
    cleared at the start of each call)."""
    asp = _setup()
    P = W.small_problem(2, 31, 4 * math.pi, 4, 3, "const", nrhs=3)
    prm = asp.make_params(P.n, P.omega, P.pml, P.b, C=P.C, precision="c128", max_rhs=P.nrhs, restart=4)
    f = torch.from_numpy(P.f).to("cuda")
    u = torch.from_numpy(P.f * 0.5).to("cuda")
    bad = np.ascontiguousarray(P.c).copy()
    bad.reshape(-1)[17] = 0.0
    got = asp.asp_residual_norms_noalloc(prm, torch.from_numpy(bad).to("cuda"), f, u).cpu().numpy()
    assert np.all(np.isnan(got)), got
    good = asp.asp_residual_norms_noalloc(prm, torch.from_numpy(np.ascontiguousarray(P.c)).to("cuda"), f, u)
    got = good.cpu().numpy()
    assert np.all(np.isfinite(got)) and np.allclose(got, _rel_from_oracle(P, u), rtol=1e-11, atol=0)


def test_residual_norms_noalloc_rejects_oversize():
    asp = _setup()
    from paper_1504_04058_gb300 import _lib
    n = 15
    prm = asp.make_params(n, 5.0, 3, 3)
    c = torch.ones(n * n, dtype=torch.float64, device="cuda")
    f = torch.zeros((n, n, _lib.NOALLOC_MAX_RHS + 1), dtype=torch.complex128, device="cuda")
    with pytest.raises(asp.AspError):
        asp.asp_residual_norms_noalloc(prm, c, f, f.clone())
