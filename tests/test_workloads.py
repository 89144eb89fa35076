"""The seeded input generators (no method arithmetic) against their stated
recipes: the Gaussian wave packet of Section 3.2 / 4.2 (unit envelope peak at
its centre, spectrum peaked at the wave number omega/c in its direction), the
layered, lens and bump velocities and the Gaussian point source."""
import math

import numpy as np
import pytest

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


def test_layered_velocity_follows_its_recipe():
    """16 equal bands along the sweep axis (numpy axis 0), band values drawn by
    numpy's PCG64 generator with the given seed from U[0.8, 1.2], smoothed
    along that axis only by a Gaussian of standard deviation 3h truncated at
    3 standard deviations: far from a band edge the field equals its band's
    draw, near one it moves monotonically between the two draws, and it is
    constant along x1 (and x2 in 3D)."""
    n, seed, layers = 255, 1504, 16
    c = W.layered_velocity(n, seed)
    assert c.shape == (n, n)
    assert np.all(c == c[:, :1])
    vals = np.random.default_rng(seed).uniform(0.8, 1.2, size=layers)
    prof = c[:, 0]
    assert prof.min() >= 0.8 and prof.max() <= 1.2
    band = np.minimum((np.arange(n) * layers) // n, layers - 1)
    edges = np.nonzero(np.diff(band))[0]  # last node of each band but the last
    reach = 9  # 3 standard deviations of 3h, in nodes
    for i in range(n):
        if np.all(np.abs(edges + 0.5 - i) > reach):
            assert prof[i] == pytest.approx(vals[band[i]], rel=1e-14)
    starts = np.concatenate([[0], edges + 1])
    ends = np.concatenate([edges, [n - 1]])
    for k, e in enumerate(edges):
        # nodes whose 3-sigma reach covers only the two bands meeting at e
        seg = prof[starts[k] + reach:ends[k + 1] - reach + 1]
        assert len(seg) > 2
        steps = np.diff(seg)
        assert np.all(steps * np.sign(vals[band[e + 1]] - vals[band[e]]) >= -1e-15)
    c3 = W.layered_velocity(31, seed, dim=3)
    assert np.all(c3 == c3[:, :1, :1])


def test_lens_and_bump_extremes():
    """Lens: 4/3 (1 - 0.5 exp(-32 r^2)) reaches its minimum 2/3 at the centre;
    bump: 1 + 0.3 exp(-32 r^2) reaches 1.3 there (odd n puts a node on it)."""
    n = 63
    lens, bump = W.lens_velocity(n, 2), W.bump_velocity(n, 3)
    mid = n // 2
    assert lens[mid, mid] == pytest.approx(2.0 / 3.0, rel=1e-14) and lens.min() == lens[mid, mid]
    assert lens.max() < 4.0 / 3.0
    assert bump[mid, mid, mid] == pytest.approx(1.3, rel=1e-14) and bump.max() == bump[mid, mid, mid]
    assert bump.min() > 1.0


def test_gaussian_source_width_and_centre():
    """The sampled Gaussian of width s = 2h has its peak 1 at a node placed on
    its centre, is symmetric about it, and its second moment along each axis
    is s^2 (Riemann sum over the nodes)."""
    n = 127
    h = 1.0 / (n + 1)
    s = 2 * h
    f = W.gaussian_source(n, 2, (0.5, 0.5), s)
    mid = n // 2
    assert f[mid, mid] == 1.0
    assert np.allclose(f, f[::-1, :]) and np.allclose(f, f[:, ::-1]) and np.allclose(f, f.T)
    x = (np.arange(n) + 1) * h - 0.5
    w = f.sum(axis=0)
    assert (w * x * x).sum() / w.sum() == pytest.approx(s * s, rel=1e-12)
