"""Device-side failure detection without a GPU fault.

Every device-side wait of the library (mbarrier phases, grid barriers) is
bounded; when one runs out the kernel records ASP_ERR_TIMEOUT in the error word,
returns, and the host reports it.  asp_selftest_bounded_wait runs that path on
purpose: one CTA waits, with the library's wait helper and a short limit, on an
mbarrier that nothing arrives on.  The test checks the reported status and that
the context still runs work afterwards.

Allocation failure is injected on the host: asp_testhook_fail_device_alloc
makes the k-th device allocation of a setup report out-of-memory without
calling the allocator, for every k the setup reaches.  Each setup must return
ASP_ERR_OOM, free what it had allocated, and leave the library usable.
"""
import math

import numpy as np
import pytest

import workloads as W
from oracle import operator

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def test_bounded_wait_reports_timeout_and_context_survives():
    import paper_1504_04058_gb300 as asp
    from paper_1504_04058_gb300 import _lib, build
    build.build()
    assert asp.asp_selftest_bounded_wait(4096) == _lib.ASP_ERR_TIMEOUT
    assert asp.asp_selftest_bounded_wait(1) == _lib.ASP_ERR_TIMEOUT
    # the context still runs the library's work: a matvec against the oracle
    P = W.small_problem(2, 31, 4 * math.pi, 4, 3, "lens", nrhs=2)
    prm = asp.make_params(P.n, P.omega, P.pml, P.b, C=P.C, precision="c128", max_rhs=P.nrhs)
    h = asp.asp_setup(P.c, prm)
    rng = np.random.default_rng(5)
    x = rng.standard_normal(P.f.shape) + 1j * rng.standard_normal(P.f.shape)
    y = h.matvec(torch.from_numpy(x).to("cuda"))
    torch.cuda.synchronize()
    A = operator.helmholtz_matrix(2, P.n, P.omega, P.c, P.pml, P.C)
    yo = (A @ x.reshape(P.n ** 2, -1)).reshape(x.shape)
    assert np.linalg.norm(y.cpu().numpy() - yo) <= 1e-13 * np.linalg.norm(yo)
    h.destroy()


def _oom_sweep(asp, _lib, c, prm, widths=None, cap=400):
    """Fail each device allocation of one setup in turn; returns how many the
    setup makes.  Checks the status and that no device memory is left behind."""
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    k = 0
    try:
        while k < cap:
            asp.asp_testhook_fail_device_alloc(k)
            try:
                h = asp.asp_setup(c, prm, widths)
            except _lib.AspError as e:
                assert e.code == _lib.ASP_ERR_OOM, str(e)
                k += 1
                continue
            # k is past the last allocation: the hook never fired
            asp.asp_testhook_fail_device_alloc(-1)
            h.factor()
            torch.cuda.synchronize()
            h.destroy()
            break
    finally:
        asp.asp_testhook_fail_device_alloc(-1)
    assert 0 < k < cap
    torch.cuda.synchronize()
    leaked = free0 - torch.cuda.mem_get_info()[0]
    assert leaked <= 8 << 20, f"{leaked} bytes not returned after {k} failed setups"
    return k


@pytest.mark.parametrize("case", ["2d_c64", "2d_c128", "3d_block", "3d_nd"])
def test_setup_allocation_failure_reports_oom_and_frees_everything(case):
    import paper_1504_04058_gb300 as asp
    from paper_1504_04058_gb300 import _lib, build
    build.build()
    if case.startswith("2d"):
        P = W.small_problem(2, 63, 8 * math.pi, 4, 4, "lens", nrhs=2)
        prm = asp.make_params(P.n, P.omega, P.pml, P.b, C=P.C, precision=case[3:], max_rhs=P.nrhs)
    else:
        P = W.small_problem(3, 19, 4 * math.pi, 3, 3, "lens", nrhs=1)
        prm = asp.make_params(P.n, P.omega, P.pml, P.b, C=P.C, precision="c64", max_rhs=P.nrhs, dim=3,
                              slab_solver=case[3:])
    nalloc = _oom_sweep(asp, _lib, P.c, prm)
    assert nalloc >= 20
    # the library still sets up, factors and applies after the failures
    h = asp.asp_setup(P.c, prm)
    h.factor()
    r = torch.from_numpy(np.ascontiguousarray(P.f)).to("cuda")
    z = h.apply_preconditioner(r)
    torch.cuda.synchronize()
    assert torch.isfinite(torch.view_as_real(z)).all()
    h.destroy()


def test_setup_beyond_the_device_is_refused_before_any_allocation():
    import paper_1504_04058_gb300 as asp
    from paper_1504_04058_gb300 import _lib, build
    build.build()
    n = 1023
    prm = asp.make_params(n, n * math.pi / 8, 20, 4, precision="c64", max_rhs=256, restart=64)
    torch.cuda.synchronize()
    free0, total = torch.cuda.mem_get_info()
    assert asp.asp_footprint_bytes(prm) > total
    c = np.ones((n, n))
    with pytest.raises(_lib.AspError) as ei:
        asp.asp_setup(c, prm)
    assert ei.value.code == _lib.ASP_ERR_OOM
    assert "exceeds the free device memory" in str(ei.value)
    torch.cuda.synchronize()
    assert abs(torch.cuda.mem_get_info()[0] - free0) <= 8 << 20
