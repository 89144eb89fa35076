"""The allocation-free residual check (asp_residual_norms_noalloc).

Callers that cannot allocate device memory (inside a CUDA-graph capture, under
a foreign allocator, in an allocation-free serving loop) use this entry point
to measure ||f - A u|| / ||f||.  It must agree with the handle-based path:
asp_matvec's A u, from which the same relative residual follows.  Two calls in
a row check that the shared fixed scratch array carries no state from one
call into the next.  This file is collected last so that a failure here does
not stop the other GPU tests in a run that stops at the first failure.
"""
import math

import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

# both paths are FP64 with the same per-element operation order; they differ
# only in the rounding of the PML weights and in the reduction order
TOL = 1e-12


def _rel_from_matvec(h, f, u):
    y = h.matvec(u)
    r = (f - y).cpu().numpy()
    fn = f.cpu().numpy()
    R = r.shape[-1]
    return np.array([np.linalg.norm(r[..., k]) / np.linalg.norm(fn[..., k]) for k in range(R)])


def test_residual_norms_noalloc_matches_handle_path():
    assert torch.cuda.is_available(), "GPU test needs a CUDA device"
    from paper_1504_04058_gb300 import build
    build.build()
    import paper_1504_04058_gb300 as asp

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
        for call in range(2):
            out = asp.asp_residual_norms_noalloc(prm, c, f, u)
            got = out.cpu().numpy()
            if k == 0:
                assert np.allclose(got, ref, rtol=TOL, atol=0), (call, got, ref)
            else:
                # at a converged solution the residual is cancellation-dominated:
                # compare with the solver's own true residual at the solution's accuracy
                true = np.array([i["rel_res_true"] for i in info])
                assert np.all(got <= 1e-8 * 1.0001), got
                assert np.allclose(got, true, rtol=1e-4), (got, true)
    h.destroy()


def test_residual_norms_noalloc_rejects_oversize():
    import paper_1504_04058_gb300 as asp
    from paper_1504_04058_gb300 import _lib
    n = 15
    prm = asp.make_params(n, 5.0, 3, 3)
    c = torch.ones(n * n, dtype=torch.float64, device="cuda")
    f = torch.zeros((n, n, _lib.NOALLOC_MAX_RHS + 1), dtype=torch.complex128, device="cuda")
    with pytest.raises(asp.AspError):
        asp.asp_residual_norms_noalloc(prm, c, f, f.clone())
