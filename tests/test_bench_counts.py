"""The algorithmic work counts behind the benchmark's roofline figures, checked
against a direct count of the block steps the method performs.

The layer subproblems are block tridiagonal along the layer (n blocks of w
unknowns).  A solve with one right-hand side is a forward pass over the n
blocks and a backward pass over n - 1 of them, one w x w complex product per
block (8 real flops per complex multiply-add).  A transfer map (Section 3.1,
"Putting together": the boundary trace of G~_p^R or G~_p^L as a function of the
incoming trace) takes n unit right-hand sides; the one in block r is zero before
block r, so its forward pass starts there.  The sweep chain applies each map to
the traces once per right-hand side.  The benchmark states these counts in
closed form (banded-LU form for the layer solves, n*w*(2w+1) band entries per
subproblem); here they are recounted step by step on small cases.
"""
import math
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def bench():
    sys.path.insert(0, ROOT)
    import bench as B
    return B


CASES = [(63, 5, 4), (127, 12, 4), (255, 20, 4), (200, 8, 7)]


def block_solve_macs(n, w, first_block=0):
    """Complex multiply-adds of one block-tridiagonal solve whose right-hand
    side is zero before `first_block`."""
    return ((n - first_block) + (n - 1)) * w * w


@pytest.mark.parametrize("n,gamma,b", CASES)
def test_transfer_map_flops_match_a_count_of_block_steps(bench, n, gamma, b):
    m, wM, wR, wL, wT = bench._layer_widths(n, gamma, b)
    counted = 0
    for w in wT:
        for _kind in ("R", "L"):
            counted += 8 * sum(block_solve_macs(n, w, r) for r in range(n))
    closed = bench.algorithmic(n, gamma, b, 1, 8)["tmap"]["flops"]
    # the closed form 1.5 n^2 w^2 drops the O(n) terms of the step count
    assert abs(closed - counted) / counted <= 1.0 / n, (closed, counted)


@pytest.mark.parametrize("n,gamma,b", CASES)
def test_tensor_core_map_flops_match_a_count_of_chain_steps(bench, n, gamma, b):
    """Maps from the diagonal blocks of the inverse: a column with data in
    block r runs r chain steps (blocks r-1 .. 0), once for the upper triangle
    (data in the boundary column) and once for the lower (data in the traced
    column), one w x w complex product per step; the diagonal-block recursion
    takes two w x w x w complex products per block below the last."""
    m, wM, wR, wL, wT = bench._layer_widths(n, gamma, b)
    counted = 0
    counted_diag = 0
    for w in wT:
        for _kind in ("R", "L"):
            for _family in ("upper", "lower"):
                counted += 8 * sum(r * w * w for r in range(n))
            counted_diag += 8 * 2 * (n - 1) * w ** 3
    alg = bench.algorithmic(n, gamma, b, 1, 8, tc=True)
    assert alg["tmap"]["flops"] == counted
    assert alg["tdiag"]["flops"] == counted_diag


@pytest.mark.parametrize("n,gamma,b", CASES)
@pytest.mark.parametrize("nrhs", [1, 32])
def test_layer_solve_flops_match_a_count_of_block_steps(bench, n, gamma, b, nrhs):
    """M-solves and fills: one full solve per subproblem and right-hand side.
    The banded-LU form counts w(2w+1) multiply-adds per unknown, the block
    form 2w^2 per block row, so they agree to O(1/w + 1/n)."""
    m, wM, wR, wL, wT = bench._layer_widths(n, gamma, b)
    alg = bench.algorithmic(n, gamma, b, nrhs, 8)
    for phase, widths in (("embed", wM), ("fill", wR + wL)):
        counted = 8 * nrhs * sum(block_solve_macs(n, w) for w in widths)
        tol = 1.0 / min(widths) + 1.0 / n
        assert abs(alg[phase]["flops"] - counted) / counted <= tol, (phase, alg[phase]["flops"], counted)


@pytest.mark.parametrize("n,gamma,b", CASES)
def test_chain_flops_and_bytes_match_the_map_count(bench, n, gamma, b):
    """The chain applies 2(m-2) dense n x n maps (p = 2 .. m-1, both sweeps)
    to every right-hand side and reads each map once."""
    m, wM, wR, wL, wT = bench._layer_widths(n, gamma, b)
    assert len(wT) == m - 2
    nrhs, esz = 32, 8
    alg = bench.algorithmic(n, gamma, b, nrhs, esz)
    maps = 2 * (m - 2)
    assert alg["chain"]["flops"] == 8 * nrhs * maps * n * n
    assert alg["chain"]["bytes"] == maps * n * n * esz


def test_layer_widths_follow_the_partition(bench):
    """Layer count and widths: P = n + 2 - 2*gamma physical columns, m =
    floor(P/b) layers, the last absorbing the remainder; M-layers are padded by
    gamma_a - 1 columns on both sides, R/L layers on one."""
    n, gamma, b = 1023, 20, 4
    m, wM, wR, wL, wT = bench._layer_widths(n, gamma, b)
    P = n + 2 - 2 * gamma
    assert m == P // b == 246
    r = P - m * b
    assert wM[:-1] == [2 * gamma + b - 2] * (m - 1) and wM[-1] == 2 * gamma + b - 2 + r
    assert wR[:-1] == [gamma + b - 1] * (m - 2) and wR[-1] == gamma + b - 1 + r
    assert wL == [gamma + b - 1] * (m - 1)
    # the benchmark's transfer-map launch at n = 1023: 3.24e12 flops
    flops = bench.algorithmic(n, gamma, b, 32, 8)["tmap"]["flops"]
    assert math.isclose(flops, 2 * 8 * 1.5 * n * n * (m - 2) * (gamma + b - 1) ** 2)
