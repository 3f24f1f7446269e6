"""Pins of the oracle's building blocks against mathematics that does not
go through its code: exactness of the FD stencils on polynomials, the WENO3
linear limit and ENO property, and the cumulant formulas (Sec. II.C, Eq. 22)
against the general set-partition formula for joint cumulants."""
import itertools
import math

import numpy as np
import pytest


def poly_line(coeffs, x0):
    """phi at x0-2..x0+2 and its exact first and second derivative at x0."""
    p = np.polynomial.Polynomial(coeffs)
    v = np.array([p(x0 + j) for j in range(-2, 3)], dtype=np.float64)
    return v, p.deriv(1)(x0), p.deriv(2)(x0)


@pytest.mark.parametrize("deg", [0, 1, 2, 3, 4])
def test_d1_exact_to_degree_4(oracle_mod, deg):
    rng = np.random.default_rng(deg)
    for _ in range(5):
        c = rng.normal(size=deg + 1)
        x0 = rng.uniform(-3, 3)
        v, d1, _ = poly_line(c, x0)
        assert abs(oracle_mod.d1(v) - d1) <= 1e-11 * max(1.0, abs(d1))


@pytest.mark.parametrize("deg", [0, 1, 2, 3, 4, 5])
def test_d2_exact_to_degree_5(oracle_mod, deg):
    rng = np.random.default_rng(10 + deg)
    for _ in range(5):
        c = rng.normal(size=deg + 1)
        x0 = rng.uniform(-3, 3)
        v, _, d2 = poly_line(c, x0)
        assert abs(oracle_mod.d2(v) - d2) <= 1e-10 * max(1.0, abs(d2))


def test_fourth_order_not_fifth(oracle_mod):
    """d1 is 4th order: x^5 is not differentiated exactly (error 4!*... != 0)."""
    v, d1, _ = poly_line([0, 0, 0, 0, 0, 1.0], 0.0)
    assert abs(oracle_mod.d1(v) - d1) > 1.0


def test_c2_exact_on_quadratics(oracle_mod):
    v, d1, _ = poly_line([0.3, -1.2, 2.5], 0.7)
    assert abs(oracle_mod.c2(v) - d1) < 1e-12


@pytest.mark.parametrize("u", [0.3, -0.3])
def test_weno3_linear_limit_is_third_order_upwind(oracle_mod, u):
    """With eps >> smoothness indicators the weights are the linear ones and
    the scheme is the 3rd-order upwind-biased difference: exact on cubics."""
    rng = np.random.default_rng(1)
    for _ in range(10):
        c = rng.normal(size=4)
        x0 = rng.uniform(-2, 2)
        v, d1, _ = poly_line(c, x0)
        assert abs(oracle_mod.weno3(v, u, 1e30) - d1) <= 1e-9 * max(1.0, abs(d1))
    # and not exact on quartics (it is not a central 4th-order scheme)
    v, d1, _ = poly_line([0, 0, 0, 0, 1.0], 0.0)
    assert abs(oracle_mod.weno3(v, u, 1e30) - d1) > 0.1


def test_weno3_upwind_side(oracle_mod):
    """The linear scheme for u > 0 uses points i-2..i+1, for u < 0 i-1..i+2."""
    e = np.zeros(5)
    e[4] = 1.0  # perturb phi_{i+2}
    assert oracle_mod.weno3(e, 1.0, 1e30) == 0.0
    assert oracle_mod.weno3(e, -1.0, 1e30) != 0.0
    e = np.zeros(5)
    e[0] = 1.0  # perturb phi_{i-2}
    assert oracle_mod.weno3(e, -1.0, 1e30) == 0.0
    assert oracle_mod.weno3(e, 1.0, 1e30) != 0.0


def test_weno3_eno_property_at_a_step(oracle_mod):
    """At a jump the nonlinear weights select the smooth sub-stencil, so the
    face values stay within the data range and the derivative upstream of
    the jump is ~0."""
    v = np.array([0.0, 0.0, 0.0, 1.0, 1.0])
    # u > 0: face i+1/2 is reconstructed from {i-1, i, i+1}: the jump is in
    # the downwind sub-stencil, whose weight is ~eps^2
    assert abs(oracle_mod.weno3(v, 1.0, 1e-6)) < 1e-10
    # the linear scheme would give 1/3 there
    assert abs(oracle_mod.weno3(v, 1.0, 1e30) - 1.0 / 3.0) < 1e-12


# ---------------------------------------------------------------------------
# cumulants
# ---------------------------------------------------------------------------

def set_partitions(items):
    if len(items) == 1:
        yield [items]
        return
    first, rest = items[0], items[1:]
    for part in set_partitions(rest):
        for k in range(len(part)):
            yield part[:k] + [[first] + part[k]] + part[k + 1:]
        yield [[first]] + part


def joint_cumulant(axes, c, f):
    """kappa(X_a1, ..., X_an) of the discrete distribution f on velocities c
    by the partition formula sum_pi (|pi|-1)! (-1)^(|pi|-1) prod_B E[prod X]."""
    total = 0.0
    for part in set_partitions(list(range(len(axes)))):
        prod = 1.0
        for block in part:
            prod *= float(np.sum(f * np.prod([c[:, axes[j]] for j in block], axis=0)))
        k = len(part)
        total += math.factorial(k - 1) * (-1) ** (k - 1) * prod
    return total


def lattice(dim):
    rng3 = [-1, 0, 1]
    if dim == 2:
        return np.array([[cx, cy, 0] for cy in rng3 for cx in rng3], dtype=np.float64)
    return np.array([[cx, cy, cz] for cz in rng3 for cy in rng3 for cx in rng3], dtype=np.float64)


def exps(j):
    return j % 3, (j // 3) % 3, j // 9


@pytest.mark.parametrize("dim", [2, 3])
def test_cumulants_match_partition_formula(oracle_mod, dim):
    """For a normalised distribution, the central moments about its mean fed
    to Eq. 22 (typos fixed) must give the joint cumulants of every order."""
    c = lattice(dim)
    rng = np.random.default_rng(dim)
    cfg = __import__("paper_2304_05657_gb300.inputs", fromlist=["x"]).base_config(dim=dim, nx=2, ny=2, nz=2)
    sim = oracle_mod.Sim(cfg, np.zeros(cfg["nx"] * cfg["ny"] * (cfg["nz"] if dim == 3 else 1), np.uint8))
    for trial in range(3):
        f = rng.uniform(0.2, 1.0, size=len(c))
        f /= f.sum()
        u = (f[:, None] * c).sum(axis=0)
        Pi = sim.central_moments(f, u)
        K = oracle_mod.cumulants(dim, Pi)
        for j in range(len(c)):
            p, q, r = exps(j)
            if p + q + r < 2:
                continue
            axes = [0] * p + [1] * q + [2] * r
            kap = joint_cumulant(axes, c, f)
            assert abs(K[j] - kap) <= 1e-13, (dim, (p, q, r), K[j], kap)


def test_product_distribution_has_no_mixed_cumulants(oracle_mod):
    """Independent axes: every mixed cumulant of order >= 4 vanishes."""
    c = lattice(3)
    a = np.array([0.2, 0.5, 0.3])
    b = np.array([0.1, 0.6, 0.3])
    d = np.array([0.25, 0.25, 0.5])
    f = np.array([a[int(cx) + 1] * b[int(cy) + 1] * d[int(cz) + 1] for cx, cy, cz in c])
    u = (f[:, None] * c).sum(axis=0)
    cfg = __import__("paper_2304_05657_gb300.inputs", fromlist=["x"]).base_config(dim=3, nx=2, ny=2, nz=2)
    sim = oracle_mod.Sim(cfg, np.zeros(8, np.uint8))
    K = oracle_mod.cumulants(3, sim.central_moments(f, u))
    for j in range(27):
        p, q, r = exps(j)
        if p + q + r >= 4:
            assert abs(K[j]) < 1e-15, (p, q, r, K[j])


@pytest.mark.parametrize("dim", [2, 3])
def test_cumulant_round_trip(oracle_mod, dim):
    rng = np.random.default_rng(7)
    Q = 9 if dim == 2 else 27
    for _ in range(20):
        Pi = rng.normal(size=Q)
        back = oracle_mod.cumulants_inverse(dim, oracle_mod.cumulants(dim, Pi))
        assert np.allclose(back, Pi, rtol=0, atol=1e-13)


@pytest.mark.parametrize("dim", [2, 3])
def test_central_moments_via_binomial_shift_and_inverse(oracle_mod, dim):
    """Central moments equal the binomially shifted raw moments, and the
    inverse transform recovers the populations."""
    c = lattice(dim)
    Q = len(c)
    rng = np.random.default_rng(11)
    cfg = __import__("paper_2304_05657_gb300.inputs", fromlist=["x"]).base_config(dim=dim, nx=2, ny=2, nz=2)
    sim = oracle_mod.Sim(cfg, np.zeros(4 if dim == 2 else 8, np.uint8))
    f = rng.normal(size=Q)
    u = rng.uniform(-0.2, 0.2, size=3)
    if dim == 2:
        u[2] = 0.0
    Pi = sim.central_moments(f, u)

    def raw(a, b, e):
        return float(np.sum(f * c[:, 0] ** a * c[:, 1] ** b * c[:, 2] ** e))

    for j in range(Q):
        p, q, r = exps(j)
        s = 0.0
        for a, b, e in itertools.product(range(p + 1), range(q + 1), range(r + 1)):
            s += (math.comb(p, a) * math.comb(q, b) * math.comb(r, e) * (-u[0]) ** (p - a) * (-u[1]) ** (q - b)
                  * (-u[2]) ** (r - e) * raw(a, b, e))
        assert abs(Pi[j] - s) < 1e-13
    assert np.allclose(sim.central_moments_inverse(Pi, u), f, rtol=0, atol=1e-13)
