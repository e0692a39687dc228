"""Pins for the oracle's reductions (Sec. 2.3, write-conflict resolution) and its
reverse / tangent passes.

Reductions: known sequences with exact sums, the max of a permutation,
NaN propagation, integer wrap against Python ints, and the exactly rounded
sum against Python's independent ``math.fsum`` on adversarial inputs.
Adjoint: central finite differences of the forward program (independent of
every derivative formula), and the dot-product test tying the reverse pass
to the forward tangent pass.
"""
import math

import numpy as np
import pytest

import oracle


def test_sum_of_first_n_integers_is_exact():
    for n in (1, 2, 1000, 1 << 20):
        y = np.arange(1, n + 1, dtype=np.float64)
        assert oracle.sum_seq(y) == n * (n + 1) / 2
        assert oracle.fsum(y) == n * (n + 1) / 2


def test_alternating_signs():
    y = np.tile([1.0, -1.0], 5001)
    assert oracle.sum_seq(y) == 0.0 and oracle.fsum(y) == 0.0
    y = np.append(y, 1.0)
    assert oracle.sum_seq(y) == 1.0
    assert oracle.sum_abs(y) == y.size


def test_max_of_permutation():
    rng = np.random.default_rng(4)
    y = rng.permutation(1000).astype(np.float64) - 300.0
    v, arg = oracle.reduce_ext("max", y)
    assert v == 699.0 and y[arg] == 699.0
    v, arg = oracle.reduce_ext("min", y)
    assert v == -300.0 and y[arg] == -300.0
    v, arg = oracle.reduce_ext("maxabs", y)
    assert v == 699.0
    y[17] = -5000.0
    v, arg = oracle.reduce_ext("maxabs", y)
    assert v == 5000.0 and arg == 17


def test_first_index_wins_ties_and_nan_propagates():
    y = np.array([1.0, 3.0, 3.0, -3.0])
    assert oracle.reduce_ext("max", y) == (3.0, 1)
    assert oracle.reduce_ext("maxabs", y) == (3.0, 1)
    y = np.array([1.0, np.nan, 5.0])
    v, arg = oracle.reduce_ext("max", y)
    assert math.isnan(v) and arg == 1
    with pytest.raises(ValueError):
        oracle.reduce_ext("max", np.array([]))


@pytest.mark.parametrize("case", [
    [1e100, 1.0, -1e100, 1e-100, 1e50, -1.0, -1e50],
    [1.0, 1e-16, 1e-16],
    [2.0 ** 53, 1.0, 1.0],
    [0.1] * 10,
    [1e308, -1e308, 1e-308, 3.0, -3.0],
    # half-way cases: the two leading terms tie (and would round to even),
    # the lower-order term decides the direction
    [1e16, 1.0, 1e-16],
    [1e16, 1.0, -1e-16],
    [2.0 ** 53, 1.0, 2.0 ** -60],
    [-(2.0 ** 53), -1.0, -(2.0 ** -60)],
])
def test_fsum_matches_python_fsum(case):
    y = np.array(case, dtype=np.float64)
    assert oracle.fsum(y) == math.fsum(case)


def test_fsum_half_way_rounding():
    """The exact sum 1e16 + 1 + 1e-16 lies just above the midpoint of two
    doubles (1e16 and 1e16 + 2): it rounds up, although 1e16 + 1 alone ties
    to the even neighbour 1e16."""
    assert oracle.fsum(np.array([1e16, 1.0, 1e-16])) == 1e16 + 2.0
    assert oracle.fsum(np.array([1e16, 1.0, -1e-16])) == 1e16
    rng = np.random.default_rng(13)
    for _ in range(200):
        big = float(2.0 ** int(rng.integers(53, 60)))
        ulp = big / 2.0 ** 52
        tiny = float(rng.choice([-1.0, 1.0])) * ulp * 2.0 ** -int(rng.integers(5, 40))
        case = [big, ulp / 2.0 * float(rng.choice([-1.0, 1.0])), tiny]
        assert oracle.fsum(np.array(case)) == math.fsum(case), case


def test_fsum_random_cancellation_matches_python_fsum():
    rng = np.random.default_rng(12)
    for trial in range(20):
        n = int(rng.integers(1, 5000))
        y = rng.normal(size=n) * 10.0 ** rng.integers(-20, 20, n)
        y = np.concatenate([y, -y[: n // 2]])
        rng.shuffle(y)
        assert oracle.fsum(y) == math.fsum(y.tolist())


def test_fsum_within_backward_bound_of_seq():
    rng = np.random.default_rng(13)
    y = rng.normal(size=100000)
    s, f, a = oracle.sum_seq(y), oracle.fsum(y), oracle.sum_abs(y)
    assert abs(s - f) <= y.size * 2.0 ** -53 * a


@pytest.mark.parametrize("bits", [32, 64])
def test_integer_reductions(bits):
    rng = np.random.default_rng(bits + 1)
    lo, hi = -(1 << (bits - 1)), (1 << (bits - 1))
    y = rng.integers(lo, hi, 777, dtype=np.int64)
    s = sum(int(v) for v in y) & ((1 << bits) - 1)
    s = s - (1 << bits) if s >= (1 << (bits - 1)) else s
    assert oracle.reduce_i("sum", bits, y) == s
    assert oracle.reduce_i("max", bits, y) == int(y.max())
    assert oracle.reduce_i("min", bits, y) == int(y.min())
    assert oracle.reduce_i("maxabs", bits, y) == max(abs(int(v)) for v in y)
    assert oracle.reduce_i("sum", bits, np.array([], dtype=np.int64)) == 0


# ---------------------------------------------------------------------------
# programs, adjoint and tangent
# ---------------------------------------------------------------------------

SEVEN = [(0, 0, 0), (0, 0, -1), (0, 0, 1), (0, -1, 0), (0, 1, 0), (-1, 0, 0), (1, 0, 0)]
W7 = [0.4] + [0.1] * 6


def _tanh_stencil_program(shape, T, bc="periodic"):
    """u_{t+1} = tanh(S u_t), loss = sum(u_T^2)."""
    p = oracle.Program()
    u = p.input("f64", shape)
    for _ in range(T):
        u = p.map("tanh", [p.stencil(u, SEVEN, W7, bc, 1)])
    loss = p.reduce(p.map("square", [u]), "sum")
    p.output(loss)
    return p


def _all_ops_program(n):
    p = oracle.Program()
    x = p.input("f64", (n,))
    a = p.input("f64", (n,))
    v = p.map("mul", [a, x])
    v = p.map("add", [v, p.map("sin", [x])])
    v = p.map("sub", [v, p.map("cos", [a])])
    v = p.map("div", [v, p.map("add_s", [p.map("exp", [x])], 1.0)])
    v = p.map("max", [v, p.map("neg", [a])])
    v = p.map("min", [v, p.map("mul_s", [x], 3.0)])
    v = p.map("sqrt", [p.map("add_s", [p.map("square", [v])], 0.5)])
    v = p.map("tanh", [p.map("rsub_s", [p.map("sub_s", [v], 0.25)], 2.0)])
    v = p.map("abs", [p.map("add", [v, p.map("neg", [x])])])
    s = p.reduce(v, "sum")
    m = p.reduce(p.map("mul", [v, a]), "maxabs")
    p.output(s)
    p.output(m)
    p.output(v)
    return p


def _forward_scalar(prog, inputs, out_grads):
    """<outputs, out_grads> as a scalar function of the inputs."""
    vals = oracle.run(prog, inputs)
    return sum(float(np.sum(np.asarray(vals[h]) * np.asarray(g)))
               for h, g in zip(prog.outputs, out_grads))


def test_adjoint_matches_central_differences_per_coordinate():
    shape, T = (4, 4, 5), 3
    prog = _tanh_stencil_program(shape, T)
    rng = np.random.default_rng(21)
    u0 = rng.uniform(-1, 1, shape)
    (g,) = oracle.adjoint(prog, [u0], [1.0])
    eps = 1e-6
    for idx in np.ndindex(*shape):
        up, dn = u0.copy(), u0.copy()
        up[idx] += eps
        dn[idx] -= eps
        fd = (_forward_scalar(prog, [up], [1.0]) - _forward_scalar(prog, [dn], [1.0])) / (2 * eps)
        assert abs(fd - g[idx]) < 1e-8 * max(1.0, abs(fd)), idx


@pytest.mark.parametrize("bc", ["zero", "fixed_ring"])
def test_adjoint_other_boundaries_central_differences(bc):
    shape, T = (3, 4, 5), 2
    prog = _tanh_stencil_program(shape, T, bc)
    rng = np.random.default_rng(22)
    u0 = rng.uniform(-1, 1, shape)
    (g,) = oracle.adjoint(prog, [u0], [1.0])
    d = rng.normal(size=shape)
    eps = 1e-6
    fd = (_forward_scalar(prog, [u0 + eps * d], [1.0])
          - _forward_scalar(prog, [u0 - eps * d], [1.0])) / (2 * eps)
    assert abs(fd - float(np.sum(g * d))) < 1e-8 * max(1.0, abs(fd))


def test_all_map_ops_adjoint_central_differences():
    n = 64
    prog = _all_ops_program(n)
    rng = np.random.default_rng(23)
    x = rng.normal(size=n)
    a = rng.normal(size=n)
    outg = [1.3, -0.7, rng.normal(size=n)]
    gx, ga = oracle.adjoint(prog, [x, a], outg)
    eps = 1e-7
    for arr, g, which in ((x, gx, 0), (a, ga, 1)):
        for i in range(n):
            up = [x.copy(), a.copy()]
            dn = [x.copy(), a.copy()]
            up[which][i] += eps
            dn[which][i] -= eps
            fd = (_forward_scalar(prog, up, outg) - _forward_scalar(prog, dn, outg)) / (2 * eps)
            assert abs(fd - g[i]) < 1e-6 * max(1.0, abs(fd)), (which, i)


def test_dot_product_reverse_vs_tangent():
    n = 200
    prog = _all_ops_program(n)
    rng = np.random.default_rng(24)
    x, a = rng.normal(size=n), rng.normal(size=n)
    v = [rng.normal(size=n), rng.normal(size=n)]
    w = [0.9, 0.4, rng.normal(size=n)]
    jv = oracle.jvp(prog, [x, a], v)
    jtw = oracle.adjoint(prog, [x, a], w)
    lhs = sum(float(np.sum(np.asarray(t) * np.asarray(ww))) for t, ww in zip(jv, w))
    rhs = sum(float(np.sum(t * vv)) for t, vv in zip(jtw, v))
    assert abs(lhs - rhs) < 1e-12 * max(1.0, abs(lhs))
    # stencil program
    prog = _tanh_stencil_program((5, 6, 7), 4)
    u0 = rng.uniform(-1, 1, (5, 6, 7))
    d = rng.normal(size=u0.shape)
    (jv,) = oracle.jvp(prog, [u0], [d])
    (g,) = oracle.adjoint(prog, [u0], [1.0])
    assert abs(float(jv) - float(np.sum(g * d))) < 1e-12 * max(1.0, abs(float(jv)))


def test_linear_stencil_loss_gradient_closed_form():
    """loss = sum((S^T u0)^2) has gradient 2 (S^T)^T S^T u0, and for the periodic
    7-point stencil (symmetric) a Fourier mode is an eigenvector: grad = 2 lam^(2T) u0."""
    n = (6, 8, 10)
    z, y, x = np.meshgrid(*[np.arange(m) for m in n], indexing="ij")
    u0 = np.cos(2 * np.pi * (z / 6 + 2 * y / 8 + 3 * x / 10))
    lam = 0.4 + 0.2 * (math.cos(2 * math.pi / 6) + math.cos(4 * math.pi / 8)
                       + math.cos(6 * math.pi / 10))
    T = 5
    p = oracle.Program()
    u = p.input("f64", n)
    s = p.stencil(u, SEVEN, W7, "periodic", T)
    p.output(p.reduce(p.map("square", [s]), "sum"))
    (g,) = oracle.adjoint(p, [u0], [1.0])
    assert np.max(np.abs(g - 2 * lam ** (2 * T) * u0)) < 1e-13


def test_scalar_operand_broadcast_values():
    """A 0-axis operand broadcasts like NumPy (hand-derived values; the
    non-commutative ops catch a swapped operand)."""
    p = oracle.Program()
    x = p.input("f64", (3,))
    s = p.input("f64", ())
    outs = [p.map("sub", [x, s]), p.map("sub", [s, x]), p.map("div", [s, x]),
            p.map("mul", [x, s]), p.map("max", [s, x])]
    for o in outs:
        p.output(o)
    vals = oracle.run(p, [np.array([1.0, 2.0, 4.0]), np.array(2.0)])
    got = [vals[o].tolist() for o in outs]
    assert got == [[-1.0, 0.0, 2.0], [1.0, 0.0, -2.0], [2.0, 1.0, 0.5], [2.0, 4.0, 8.0],
                   [2.0, 2.0, 4.0]]


def test_broadcast_adjoint_central_differences():
    """y = (x - mean(x)) / max|x|, loss = sum(y^2): gradient through 0-axis
    operands checked against central differences."""
    n = 40
    p = oracle.Program()
    x = p.input("f64", (n,))
    mean = p.map("mul_s", [p.reduce(x, "sum")], 1.0 / n)
    y = p.map("mul", [p.map("sub", [x, mean]), p.map("add_s", [p.reduce(x, "sum")], 3.0)])
    p.output(p.reduce(p.map("square", [y]), "sum"))
    rng = np.random.default_rng(29)
    x0 = rng.normal(size=n)
    (g,) = oracle.adjoint(p, [x0], [1.0])
    eps = 1e-6
    for i in range(n):
        up, dn = x0.copy(), x0.copy()
        up[i] += eps
        dn[i] -= eps
        fd = (float(oracle.run(p, [up])[-1]) - float(oracle.run(p, [dn])[-1])) / (2 * eps)
        assert abs(fd - g[i]) < 1e-6 * max(1.0, abs(fd)), i
    d = rng.normal(size=n)
    (jv,) = oracle.jvp(p, [x0], [d])
    assert abs(float(jv) - float(np.sum(g * d))) < 1e-10 * max(1.0, abs(float(jv)))


@pytest.mark.parametrize("op", ["max", "min"])
def test_max_min_adjoint_at_ties_follows_the_selected_operand(op):
    """At a tie max/min is not differentiable; the adjoint goes to the operand
    the forward pass returned.  Signed zeros make that operand visible (the
    forward result of a +0/-0 tie carries b's sign), and the reverse pass must
    agree with the tangent pass there: <J v, w> = <v, J^T w> holds only if
    both take the same operand at every tie."""
    a = np.array([0.0, -0.0, 1.5, 2.0, -3.0])
    b = np.array([-0.0, 0.0, 1.5, 2.0, -3.0])
    y = oracle.map_f(op, a, b)
    assert np.array_equal(np.signbit(y), np.signbit(b))
    g = np.array([1.0, 2.0, 3.0, 4.0, 5.0])
    ga, gb = oracle.map_vjp(op, a, b, 0.0, y, g)
    assert np.array_equal(ga, np.zeros(5)) and np.array_equal(gb, g)
    rng = np.random.default_rng(31)
    da, db = rng.normal(size=5), rng.normal(size=5)
    dy = oracle.map_jvp(op, a, b, 0.0, y, da, db)
    assert np.array_equal(dy, db)
    assert float(np.dot(dy, g)) == pytest.approx(float(np.dot(da, ga) + np.dot(db, gb)), rel=1e-15)
