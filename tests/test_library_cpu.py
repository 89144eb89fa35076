"""CPU-side checks of the C-ABI library: it builds for sm_103a, loads, exports
every entry point include/asp.h declares, and rejects invalid parameters on the
host (no GPU compute is called here)."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_1504_04058_gb300 import build
    build.build()
    from paper_1504_04058_gb300 import _lib
    return _lib.load()


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "asp.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(asp_[a-z_0-9]+)\s*\(", src)))


def test_header_declarations_match_binding():
    from paper_1504_04058_gb300 import _lib
    assert declared_symbols() == sorted(_lib.EXPORTS)


def test_library_exports_every_declared_symbol(lib):
    from paper_1504_04058_gb300 import _lib
    out = subprocess.run(["nm", "-D", "--defined-only", _lib.LIB_PATH], capture_output=True, text=True,
                         check=True).stdout
    exported = set(re.findall(r"\bT (asp_\w+)", out))
    for name in declared_symbols():
        assert name in exported, name
        assert hasattr(lib, name)


def test_error_strings(lib):
    assert lib.asp_error_string(0) == b"ASP_OK"
    assert lib.asp_error_string(-4) == b"ASP_ERR_SMALL_PIVOT"
    assert lib.asp_error_string(12345) == b"ASP_ERR_UNKNOWN"


def test_invalid_parameters_rejected_on_host(lib):
    from paper_1504_04058_gb300 import _lib, make_params
    bad = [
        make_params(127, 50.0, 1, 4),             # gamma < 2
        make_params(127, -1.0, 12, 4),            # omega <= 0
        make_params(20, 50.0, 12, 4),             # n too small for the PML
        make_params(127, 50.0, 12, 0),            # b < 1
        make_params(127, 50.0, 12, 4, max_rhs=0),
        make_params(127, 50.0, 12, 4, restart=0),
    ]
    for p in bad:
        assert lib.asp_footprint_bytes(ctypes.byref(p)) == 0
        out = ctypes.c_void_p()
        import numpy as np
        c = np.ones(p.n ** 2)
        code = lib.asp_setup(ctypes.byref(p), c.ctypes.data_as(ctypes.c_void_p), 0, ctypes.byref(out))
        assert code == _lib.ASP_ERR_INVALID
        assert out.value is None
        assert lib.asp_last_error_detail()


def test_dimension_checks(lib):
    """dim must be 2 or 3; a 3D slab block larger than the kernels take is
    reported as unsupported before any device work."""
    import numpy as np
    from paper_1504_04058_gb300 import _lib, make_params
    out = ctypes.c_void_p()
    p = make_params(31, 50.0, 4, 4, dim=4)
    c = np.ones(31 ** 3)
    assert lib.asp_setup(ctypes.byref(p), c.ctypes.data_as(ctypes.c_void_p), 0,
                         ctypes.byref(out)) == _lib.ASP_ERR_INVALID
    p = make_params(255, 50.0, 12, 4, dim=3)  # blocks of 255 * 26 unknowns
    c = np.ones(255 ** 3)
    assert lib.asp_setup(ctypes.byref(p), c.ctypes.data_as(ctypes.c_void_p), 0,
                         ctypes.byref(out)) == _lib.ASP_ERR_UNSUPPORTED
    assert lib.asp_footprint_bytes(ctypes.byref(p)) == 0


def test_2d_grid_beyond_the_sweep_chain_is_unsupported(lib):
    """The sweep chain holds at most 16 map rows per CTA on half of the SMs,
    so on 152 SMs (the count assumed without a device) a 2D grid of more
    than 1216 points per side is refused by setup, not by the first apply."""
    import numpy as np
    from paper_1504_04058_gb300 import _lib, make_params
    ok = make_params(1216, 128 * 3.141592653589793, 20, 4, precision="c64", max_rhs=1, restart=4)
    big = make_params(1217, 128 * 3.141592653589793, 20, 4, precision="c64", max_rhs=1, restart=4)
    assert lib.asp_footprint_bytes(ctypes.byref(ok)) > 0
    assert lib.asp_footprint_bytes(ctypes.byref(big)) == 0
    out = ctypes.c_void_p()
    c = np.ones(1217 ** 2)
    assert lib.asp_setup(ctypes.byref(big), c.ctypes.data_as(ctypes.c_void_p), 0,
                         ctypes.byref(out)) == _lib.ASP_ERR_UNSUPPORTED
    assert b"sweep chain" in lib.asp_last_error_detail()
    assert not out.value


def test_3d_footprint_counts_every_slab_factor(lib):
    """3D factors: n dense blocks of (n w) x (n w) per slab (rows padded to a
    multiple of 4), for every M, R and L slab."""
    from paper_1504_04058_gb300 import make_params
    n, gamma, b = 95, 8, 4
    p = make_params(n, 48 * 3.141592653589793, gamma, b, precision="c64", max_rhs=1, dim=3)
    m = (n + 2 - 2 * gamma) // b
    alpha = [gamma + (q - 1) * b for q in range(1, m + 1)]
    beta = [gamma + q * b - 1 if q < m else n + 1 - gamma for q in range(1, m + 1)]
    mlo = [1 if q == 1 else alpha[q - 1] - gamma + 1 for q in range(1, m + 1)]
    mhi = [n if q == m else beta[q - 1] + gamma - 1 for q in range(1, m + 1)]
    widths = [mhi[q] - mlo[q] + 1 for q in range(m)]
    widths += [mhi[q] - alpha[q] + 1 for q in range(1, m)]
    widths += [beta[q] - mlo[q] + 1 for q in range(m - 1)]
    factor_bytes = sum(n * (n * w) * ((n * w + 3) // 4 * 4) * 8 for w in widths)
    fp = lib.asp_footprint_bytes(ctypes.byref(p))
    assert factor_bytes < fp < 1.2 * factor_bytes
    assert 70e9 < factor_bytes < 80e9


def test_nonpositive_velocity_rejected(lib):
    import numpy as np
    from paper_1504_04058_gb300 import _lib, make_params
    p = make_params(31, 20.0, 4, 3)
    c = np.ones(31 * 31)
    c[100] = 0.0
    out = ctypes.c_void_p()
    code = lib.asp_setup(ctypes.byref(p), c.ctypes.data_as(ctypes.c_void_p), 0, ctypes.byref(out))
    assert code == _lib.ASP_ERR_INVALID


def test_non_finite_inputs_rejected(lib):
    """NaN or infinite velocity entries, omega or C are invalid (the checks
    are written so that NaN fails them), reported before any device work."""
    import numpy as np
    from paper_1504_04058_gb300 import _lib, make_params
    out = ctypes.c_void_p()
    for bad in (np.nan, np.inf):
        p = make_params(31, 20.0, 4, 3)
        c = np.ones(31 * 31)
        c[7] = bad
        assert lib.asp_setup(ctypes.byref(p), c.ctypes.data_as(ctypes.c_void_p), 0,
                             ctypes.byref(out)) == _lib.ASP_ERR_INVALID
        assert b"velocity" in lib.asp_last_error_detail()
        for field in ("omega", "C"):
            p = make_params(31, 20.0, 4, 3)
            setattr(p, field, bad)
            assert lib.asp_footprint_bytes(ctypes.byref(p)) == 0
            c = np.ones(31 * 31)
            assert lib.asp_setup(ctypes.byref(p), c.ctypes.data_as(ctypes.c_void_p), 0,
                                 ctypes.byref(out)) == _lib.ASP_ERR_INVALID
            assert field.encode() in lib.asp_last_error_detail()
    assert not out.value


def test_footprint_matches_layer_sizes(lib):
    """The footprint grows with n and includes the factor bytes of every layer
    subproblem: sum over 3m-2 subproblems of n*w*w_pad elements."""
    from paper_1504_04058_gb300 import make_params
    p1 = make_params(127, 16 * 3.14159, 12, 4, precision="c64", max_rhs=1, restart=8)
    p2 = make_params(255, 32 * 3.14159, 12, 4, precision="c64", max_rhs=1, restart=8)
    f1 = lib.asp_footprint_bytes(ctypes.byref(p1))
    f2 = lib.asp_footprint_bytes(ctypes.byref(p2))
    assert 0 < f1 < f2
    n, g, b = 127, 12, 4
    m = (n + 2 - 2 * g) // b
    r = n + 2 - 2 * g - m * b
    fac = 0
    for q in range(1, m + 1):  # X_q^M: 2*gamma+b-2 columns, the last layer + remainder
        w = 2 * g + b - 2 + (r if q == m else 0)
        fac += n * w * (w + (w % 2))
    for q in range(2, m + 1):  # X_q^R: gamma+b-1 columns
        w = g + b - 1 + (r if q == m else 0)
        fac += n * w * (w + (w % 2))
    for q in range(1, m):      # X_q^L
        w = g + b - 1
        fac += n * w * (w + (w % 2))
    assert f1 > fac * 8


def test_selftest_bounded_wait_rejects_bad_limits():
    """The argument check of the bounded-wait self-test runs before any CUDA call."""
    from paper_1504_04058_gb300 import _lib
    lib = _lib.load()
    assert lib.asp_selftest_bounded_wait(0, None) == _lib.ASP_ERR_INVALID
    assert lib.asp_selftest_bounded_wait(-3, None) == _lib.ASP_ERR_INVALID
    assert lib.asp_selftest_bounded_wait((1 << 26) + 1, None) == _lib.ASP_ERR_INVALID


# ------------------------------------------------ layers of arbitrary widths

def _widths_for(c, n, gamma, b_min, b_max, dim=2, pml_aux=0):
    import paper_1504_04058_gb300 as asp
    prm = asp.make_params(n, 10.0, gamma, b_min, pml_aux=pml_aux, dim=dim)
    return asp.layer_widths_from_velocity(prm, c, b_min, b_max)


def test_layer_widths_for_a_smooth_velocity_are_uniform(lib):
    """No heavy jump: every layer has b_min columns and the last takes the
    remainder, which is the uniform partition."""
    import numpy as np
    n, gamma = 127, 12
    w = _widths_for(np.ones((n, n)), n, gamma, 4, 8)
    P = n + 2 - 2 * gamma
    m = P // 4
    assert sum(w) == P
    assert w == [4] * (m - 1) + [4 + P - 4 * m]


def test_layer_widths_grow_where_the_velocity_jumps(lib):
    """Section 3.1, practical remark 3: wider layers where the velocity varies
    heavily.  With sharp jumps between constant bands, no layer boundary
    falls between two columns with a jump unless the layer already has b_max
    columns; a layer grows beyond b_min only to carry its boundary past a
    jump."""
    import numpy as np
    n, gamma, b_min, b_max = 200, 8, 3, 7
    prof = np.ones(n)
    jumps = [40, 41, 97, 150, 151, 152]  # column j (1-based) jumps to j+1
    for j in jumps:
        prof[j:] *= 1.15
    c = np.broadcast_to(prof[:, None], (n, n)).copy()  # c[i2-1, i1-1]: varies along x2
    w = _widths_for(c, n, gamma, b_min, b_max)
    P = n + 2 - 2 * gamma
    assert sum(w) == P and min(w) >= 1
    ends, a = [], gamma
    for x in w:
        ends.append(a + x - 1)
        a += x
    for e, x in zip(ends[:-1], w[:-1]):
        assert e not in jumps or x == b_max, (e, x)
    # where a boundary would have fallen on a jump the layer grew past it
    assert any(x > b_min for x in w[:-1])
    assert all(x in (b_min, b_max) or any(e - x < j < e for j in jumps) for e, x in zip(ends[:-1], w[:-1]))


def test_layer_widths_rejected_on_host(lib):
    """Widths that do not sum to P, zero widths and an oversized padded width
    are refused before any device work."""
    import numpy as np
    import paper_1504_04058_gb300 as asp
    from paper_1504_04058_gb300 import _lib
    n, gamma = 31, 4
    prm = asp.make_params(n, 10.0, gamma, 3, max_rhs=1, restart=4)
    P = n + 2 - 2 * gamma
    for bad in ([3] * (P // 3), [0] + [3] * (P // 3), [P + 1]):
        with pytest.raises(asp.AspError) as ei:
            asp.asp_setup(np.ones((n, n)), prm, widths=bad)
        assert ei.value.code == _lib.ASP_ERR_INVALID
        assert asp.asp_footprint_bytes(prm, widths=bad) == 0
    with pytest.raises(asp.AspError):
        asp.layer_widths_from_velocity(prm, np.ones((n, n)), 0, 4)


def test_footprint_with_explicit_widths(lib):
    """Uniform widths passed explicitly give asp_footprint_bytes' value; wider
    layers (fewer, larger subproblems) give a different one."""
    import paper_1504_04058_gb300 as asp
    n, gamma, b = 127, 12, 4
    prm = asp.make_params(n, 40.0, gamma, b, precision="c64", max_rhs=2, restart=8)
    P = n + 2 - 2 * gamma
    m = P // b
    uniform = [b] * (m - 1) + [b + P - m * b]
    f0 = asp.asp_footprint_bytes(prm)
    assert f0 > 0 and asp.asp_footprint_bytes(prm, widths=uniform) == f0
    wider = [8] * (P // 8 - 1) + [8 + P - 8 * (P // 8)]
    f1 = asp.asp_footprint_bytes(prm, widths=wider)
    assert f1 > 0 and f1 != f0


def _nd_stats(lib, n, w):
    st = (ctypes.c_longlong * 8)()
    assert lib.asp_nd_plan_check(n, w, st, 8) == 0
    return list(st)


@pytest.mark.parametrize("n,w", [(3, 1), (5, 2), (8, 1), (10, 3), (15, 4), (31, 5), (47, 9), (95, 18)])
def test_nested_dissection_plan_assembles_every_coupling_once(lib, n, w):
    """Every directed stencil coupling of an n x n x w slab is assembled at
    exactly one front (Section 4's nested dissection of the column grid): the
    count equals the 7-point operator's nonzeros, none twice, none missing."""
    nodes, depth, front, factor, assembled, nnz, dup, miss = _nd_stats(lib, n, w)
    assert nnz == n * n * w + 2 * ((n - 1) * n * w + n * (n - 1) * w + n * n * (w - 1))
    assert assembled == nnz and dup == 0 and miss == 0


def test_nested_dissection_plan_shape_at_95(lib):
    """n = 95: a leaf is a region of at most 8 columns, so the 95 x 95 grid is cut
    10 times along every branch (2047 nodes).  The largest front is a child of
    the root: its separator (47 columns) plus the root separator beside it
    (95 columns), 18 planes each."""
    nodes, depth, front, factor, *_ = _nd_stats(lib, 95, 18)
    assert (nodes, depth) == (2047, 10)
    assert front == (47 + 95) * 18
    # the root stores X (1710 x 1710, rows padded to 4) and nothing else
    assert factor > 1710 * 1712


def test_nested_dissection_parameters(lib):
    from paper_1504_04058_gb300 import make_params
    nd2 = make_params(63, 20.0, 6, 4, slab_solver="nd")        # 2D: rejected
    assert lib.asp_footprint_bytes(ctypes.byref(nd2)) == 0
    blk = make_params(95, 48 * 3.141592653589793, 8, 4, precision="c64", dim=3)
    nd3 = make_params(95, 48 * 3.141592653589793, 8, 4, precision="c64", dim=3, slab_solver="nd")
    fb, fn = lib.asp_footprint_bytes(ctypes.byref(blk)), lib.asp_footprint_bytes(ctypes.byref(nd3))
    assert fb > 0 and fn > 0
    assert fn < fb  # fewer factor entries than the dense block inverses
    bad = make_params(95, 48 * 3.141592653589793, 8, 4, precision="c64", dim=3)
    bad.slab_solver = 7
    assert lib.asp_footprint_bytes(ctypes.byref(bad)) == 0


@pytest.mark.parametrize("n,w", [(13, 4), (31, 5), (95, 18)])
def test_nested_dissection_plan_matches_the_oracle_tree(lib, n, w):
    """The library's host plan and the oracle's separator tree are written
    independently from the same rule; they must agree on the number of nodes,
    the depth and the largest front."""
    from oracle import nested_dissection as nd
    nodes = nd.separator_tree(n, 8)

    def bcols(t):
        x0, x1, y0, y1 = t.region
        out = 0
        out += (x1 - x0) if y0 > 0 else 0
        out += (x1 - x0) if y1 < n else 0
        out += (y1 - y0) if x0 > 0 else 0
        out += (y1 - y0) if x1 < n else 0
        return out

    front = max((len(t.own) + bcols(t)) * w for t in nodes)
    depth = max(t.depth for t in nodes)
    st = _nd_stats(lib, n, w)
    assert (st[0], st[1], st[2]) == (len(nodes), depth, front)
