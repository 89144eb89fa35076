"""Device-side failure detection without a GPU fault.

Every device-side wait of the library (mbarrier phases, grid barriers) is
bounded; when one runs out the kernel records ASP_ERR_TIMEOUT in the error word,
returns, and the host reports it.  asp_selftest_bounded_wait runs that path on
purpose: one CTA waits, with the library's wait helper and a short limit, on an
mbarrier that nothing arrives on.  The test checks the reported status and that
the context still runs work afterwards.
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
