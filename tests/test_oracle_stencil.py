"""Pins for the oracle's iterated stencils (Sec. 2.2 jacobi_1d, Sec. 4.3 jacobi_2d).

Pins used: closed forms on constant / linear / quadratic fields, eigenmodes of
the 5-point and 7-point averaging operators, sum conservation under periodic
boundaries, a pure shift (catches an offset sign error that symmetric
stencils hide), brute force against an explicit dense operator matrix raised
to the power T, the paper's own slice-assignment form of the jacobi
programs, and the transpose identity for the adjoint.
"""
import math

import numpy as np
import pytest

import oracle

FIVE = [(0, 0), (0, -1), (0, 1), (1, 0), (-1, 0)]          # c, w, e, s, n (paper order)
SEVEN = [(0, 0, 0), (0, 0, -1), (0, 0, 1), (0, -1, 0), (0, 1, 0), (-1, 0, 0), (1, 0, 0)]
W5 = [0.2] * 5
W7 = [0.4] + [0.1] * 6


def test_constant_field_periodic():
    c = 0.75
    u = np.full((9, 7), c)
    out = oracle.stencil(u, FIVE, W5, "periodic", 3)
    assert np.allclose(out, c, rtol=0, atol=4e-16)
    u3 = np.full((5, 6, 7), -1.25)
    out3 = oracle.stencil(u3, SEVEN, W7, "periodic", 4)
    assert np.allclose(out3, -1.25, rtol=0, atol=1e-15)


def test_constant_field_zero_boundary_one_step():
    # a border cell loses exactly the weights of its out-of-range neighbours
    u = np.ones((6, 8))
    out = oracle.stencil(u, FIVE, W5, "zero", 1)
    assert abs(out[3, 3] - 1.0) < 1e-15
    assert abs(out[0, 3] - 0.8) < 1e-15        # north neighbour missing
    assert abs(out[0, 0] - 0.6) < 1e-15        # corner: two missing
    assert abs(out[5, 7] - 0.6) < 1e-15


def test_linear_field_reproduced_in_interior():
    y, x = np.meshgrid(np.arange(12.0), np.arange(10.0), indexing="ij")
    u = 0.5 * x - 0.25 * y + 3.0
    out = oracle.stencil(u, FIVE, W5, "zero", 2)
    assert np.max(np.abs(out[2:-2, 2:-2] - u[2:-2, 2:-2])) < 1e-14
    z, y3, x3 = np.meshgrid(np.arange(7.0), np.arange(8.0), np.arange(9.0), indexing="ij")
    u3 = x3 - 2 * y3 + 0.5 * z
    out3 = oracle.stencil(u3, SEVEN, W7, "fixed_ring", 2)
    assert np.max(np.abs(out3[2:-2, 2:-2, 2:-2] - u3[2:-2, 2:-2, 2:-2])) < 1e-14


def test_quadratic_field_gains_constant_per_step():
    # 2-D: 0.2 * ((x-1)^2 + (x+1)^2 + 3 x^2) = x^2 + 0.4 per step
    y, x = np.meshgrid(np.arange(16.0), np.arange(16.0), indexing="ij")
    out = oracle.stencil(x * x, FIVE, W5, "zero", 3)
    assert np.max(np.abs(out[4:-4, 4:-4] - (x * x + 1.2)[4:-4, 4:-4])) < 1e-12
    # 3-D: 0.4 x^2 + 0.1 ((x-1)^2 + (x+1)^2 + 4 x^2) = x^2 + 0.2 per step
    z, y3, x3 = np.meshgrid(np.arange(9.0), np.arange(9.0), np.arange(12.0), indexing="ij")
    out3 = oracle.stencil(x3 * x3, SEVEN, W7, "zero", 2)
    assert np.max(np.abs(out3[3:-3, 3:-3, 3:-3] - (x3 * x3 + 0.4)[3:-3, 3:-3, 3:-3])) < 1e-12


def test_periodic_fourier_mode_3d():
    n = (8, 10, 12)
    k = (1, 2, 3)
    z, y, x = np.meshgrid(*[np.arange(m) for m in n], indexing="ij")
    phase = 2 * np.pi * (k[0] * z / n[0] + k[1] * y / n[1] + k[2] * x / n[2])
    u = np.cos(phase)
    lam = 0.4 + 0.2 * sum(math.cos(2 * math.pi * k[i] / n[i]) for i in range(3))
    T = 10
    out = oracle.stencil(u, SEVEN, W7, "periodic", T)
    assert np.max(np.abs(out - lam ** T * u)) < 1e-14


def test_zero_boundary_sine_mode_2d():
    N, p, q, T = 20, 2, 3, 10
    i, j = np.meshgrid(np.arange(N), np.arange(N), indexing="ij")
    u = np.sin(np.pi * p * (i + 1) / (N + 1)) * np.sin(np.pi * q * (j + 1) / (N + 1))
    lam = 0.2 * (1 + 2 * math.cos(math.pi * p / (N + 1)) + 2 * math.cos(math.pi * q / (N + 1)))
    out = oracle.stencil(u, FIVE, W5, "zero", T)
    assert np.max(np.abs(out - lam ** T * u)) < 1e-14


def test_sum_conservation_periodic():
    rng = np.random.default_rng(1)
    u = rng.uniform(-1, 1, (6, 7, 9))
    out = oracle.stencil(u, SEVEN, W7, "periodic", 5)
    assert abs(math.fsum(out.ravel()) - math.fsum(u.ravel())) < 1e-13


def test_pure_shift_is_roll():
    """out[p] = in[p + o]: a shift by +1 along x equals np.roll(u, -1) exactly."""
    rng = np.random.default_rng(2)
    u = rng.normal(size=(5, 11))
    out = oracle.stencil(u, [(0, 1)], [1.0], "periodic", 1)
    assert np.array_equal(out, np.roll(u, -1, axis=1))
    out = oracle.stencil(u, [(2, 0)], [1.0], "periodic", 3)
    assert np.array_equal(out, np.roll(u, -6, axis=0))
    z = oracle.stencil(u, [(0, 1)], [1.0], "zero", 1)
    assert np.array_equal(z[:, :-1], u[:, 1:]) and np.all(z[:, -1] == 0.0)


def _dense_operator(shape, offsets, weights, bc):
    """Explicit matrix A with (A u)[p] = one stencil step, built cell by cell."""
    n = int(np.prod(shape))
    A = np.zeros((n, n))
    idx = np.arange(n).reshape(shape)
    ndim = len(shape)
    ring = [max(abs(o[a]) for o in offsets) for a in range(ndim)]
    for p in np.ndindex(*shape):
        r = idx[p]
        if bc == "fixed_ring" and any(p[a] < ring[a] or p[a] >= shape[a] - ring[a]
                                      for a in range(ndim)):
            A[r, r] = 1.0
            continue
        for o, w in zip(offsets, weights):
            q = [p[a] + o[a] for a in range(ndim)]
            if bc == "periodic":
                q = [q[a] % shape[a] for a in range(ndim)]
            elif any(q[a] < 0 or q[a] >= shape[a] for a in range(ndim)):
                continue
            A[r, idx[tuple(q)]] += w
    return A


@pytest.mark.parametrize("bc", ["zero", "periodic", "fixed_ring"])
@pytest.mark.parametrize("shape", [(7,), (4, 5), (3, 4, 5), (2, 2), (1, 3)])
def test_brute_force_dense_power(bc, shape):
    rng = np.random.default_rng(len(shape) * 10 + len(bc))
    ndim = len(shape)
    npts = 4
    offs = [tuple(int(v) for v in rng.integers(-2, 3, ndim)) for _ in range(npts)]
    w = rng.normal(size=npts)
    u = rng.normal(size=shape)
    T = 3
    A = _dense_operator(shape, offs, w, bc)
    ref = (np.linalg.matrix_power(A, T) @ u.ravel()).reshape(shape)
    out = oracle.stencil(u, offs, w, bc, T)
    assert np.max(np.abs(out - ref)) < 1e-12 * max(1.0, np.max(np.abs(ref)))
    # the adjoint is the transpose
    g = rng.normal(size=shape)
    gin = oracle.stencil_vjp(g, offs, w, bc, T)
    refT = (np.linalg.matrix_power(A.T, T) @ g.ravel()).reshape(shape)
    assert np.max(np.abs(gin - refT)) < 1e-12 * max(1.0, np.max(np.abs(refT)))


def test_paper_jacobi_2d_slice_form():
    """The paper's jacobi_2d updates only the interior, from five shifted views;
    with both buffers starting equal, each half-step is one fixed-ring step."""
    rng = np.random.default_rng(7)
    A0 = rng.uniform(0, 1, (13, 11))
    A = A0.copy()
    for _ in range(4):
        B = A.copy()
        B[1:-1, 1:-1] = 0.2 * (A[1:-1, 1:-1] + A[1:-1, :-2] + A[1:-1, 2:] + A[2:, 1:-1]
                               + A[:-2, 1:-1])
        A = B
    out = oracle.stencil(A0, FIVE, W5, "fixed_ring", 4)
    assert np.max(np.abs(out - A)) < 1e-15


def test_paper_jacobi_1d_slice_form():
    rng = np.random.default_rng(8)
    A0 = rng.uniform(0, 1, 40)
    A = A0.copy()
    for _ in range(6):
        B = A.copy()
        B[1:-1] = 0.33333 * (A[:-2] + A[1:-1] + A[2:])
        A = B
    out = oracle.stencil(A0, [(-1,), (0,), (1,)], [0.33333] * 3, "fixed_ring", 6)
    assert np.max(np.abs(out - A)) < 1e-15


@pytest.mark.parametrize("bc", ["zero", "periodic", "fixed_ring"])
def test_cone_point_matches_full_grid(bc):
    rng = np.random.default_rng(9)
    u = rng.uniform(-1, 1, (6, 9, 10))
    T = 4
    full = oracle.stencil(u, SEVEN, W7, bc, T)
    for _ in range(12):
        p = tuple(int(rng.integers(0, s)) for s in u.shape)
        v = oracle.stencil_point(u, SEVEN, W7, bc, T, p)
        assert abs(v - full[p]) < 1e-15, p
    u2 = rng.uniform(0, 1, (5, 7))
    full2 = oracle.stencil(u2, FIVE, W5, bc, 6)
    for p in [(0, 0), (4, 6), (2, 3), (0, 6)]:
        assert abs(oracle.stencil_point(u2, FIVE, W5, bc, 6, p) - full2[p]) < 1e-15


def test_zero_steps_is_identity():
    u = np.arange(12.0).reshape(3, 4)
    assert np.array_equal(oracle.stencil(u, FIVE, W5, "zero", 0), u)
