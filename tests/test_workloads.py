"""The seeded input generators (no method arithmetic): the Gaussian wave
packet of Section 3.2 / 4.2 has a unit envelope peak at its centre and its
spectrum peaks at the wave number omega/c in its direction."""
import math

import numpy as np

import workloads as W


def test_wave_packet_envelope_and_direction():
    n, omega = 255, 32 * math.pi
    centre = (0.5, 0.5)
    d = np.array([1.0, 1.0]) / math.sqrt(2)
    f = W.wave_packet(n, 2, centre, d, omega)
    assert f.dtype == np.complex128 and f.shape == (n, n)
    assert np.abs(f).max() <= 1.0 + 1e-12
    h = 1.0 / (n + 1)
    i2, i1 = np.unravel_index(np.abs(f).argmax(), f.shape)  # x1 varies along the last axis
    assert abs((i1 + 1) * h - centre[0]) <= h and abs((i2 + 1) * h - centre[1]) <= h
    # spectral peak at k d (grid period (n+1) h = 1 with zero padding to n+1)
    F = np.abs(np.fft.fft2(f, s=(n + 1, n + 1)))
    k = np.array(np.unravel_index(F.argmax(), F.shape), dtype=float)
    k[k > (n + 1) / 2] -= n + 1
    kw = omega / (2 * math.pi)  # cycles per unit length
    expect = kw * np.array([abs(d[1]), abs(d[0])])  # numpy axes (x2, x1)
    assert np.allclose(np.abs(k), expect, atol=1.0), (k, expect)


def test_point_and_packet_problems_are_seeded():
    a = W.small_problem(2, 31, 4 * math.pi, 4, 3, "lens", nrhs=2, source="packet", seed=5)
    b = W.small_problem(2, 31, 4 * math.pi, 4, 3, "lens", nrhs=2, source="packet", seed=5)
    c = W.small_problem(2, 31, 4 * math.pi, 4, 3, "lens", nrhs=2, source="point", seed=5)
    assert np.array_equal(a.f, b.f)
    assert np.iscomplexobj(a.f) and np.abs(a.f.imag).max() > 0.1
    assert np.abs(c.f.imag).max() == 0.0
