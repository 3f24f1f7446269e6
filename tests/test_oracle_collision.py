"""Pins of the oracle's source term and cumulant collision (Sec. II.B-C):
moments of Xi derived from Eq. 9, conservation of the collision, the BGK
special case (all rates 1, uniform density), and that each class of moments
relaxes at its own rate."""
import numpy as np
import pytest

from paper_2304_05657_gb300 import inputs

CS2 = 1.0 / 3.0


def lattice(dim):
    r = [-1, 0, 1]
    if dim == 2:
        return np.array([[cx, cy, 0] for cy in r for cx in r], dtype=np.float64)
    return np.array([[cx, cy, cz] for cz in r for cy in r for cx in r], dtype=np.float64)


def weights(c):
    w1 = {-1: 1 / 6, 0: 2 / 3, 1: 1 / 6}
    dim = 3 if np.any(c[:, 2] != 0) else 2
    return np.array([w1[int(a)] * w1[int(b)] * (w1[int(e)] if dim == 3 else 1.0) for a, b, e in c])


def sim_for(oracle_mod, dim, **over):
    cfg = inputs.base_config(dim=dim, nx=3, ny=3, nz=3, bc=["periodic"] * 6, **over)
    n = 9 if dim == 2 else 27
    return oracle_mod.Sim(cfg, np.zeros(n, np.uint8))


def random_cell(rng, dim):
    Q = 9 if dim == 2 else 27
    g = rng.uniform(-2e-3, 2e-3, size=Q)
    rho = rng.uniform(0.3, 1.2)
    u = lattice(dim).T @ g / (rho * CS2)  # Eq. 13b
    gr = rng.uniform(-0.02, 0.02, size=3)
    if dim == 2:
        gr[2] = 0.0
    lam = rng.uniform(-0.01, 0.01)
    return g, rho, u, gr, lam


@pytest.mark.parametrize("dim", [2, 3])
def test_source_moments(oracle_mod, dim):
    """From Eq. 9: sum_i Xi_i = cs^2 (u.grad rho + rho Lambda) and
    sum_i c_i Xi_i = 0 (the source does not act on momentum)."""
    sim = sim_for(oracle_mod, dim)
    c = lattice(dim)
    rng = np.random.default_rng(dim)
    for _ in range(10):
        g, rho, u, gr, lam = random_cell(rng, dim)
        _, xi, _ = sim.collide_cell(g, rho, u, gr, lam)
        assert abs(xi.sum() - CS2 * (u @ gr + rho * lam)) < 1e-16
        assert np.abs(c.T @ xi).max() < 1e-16


@pytest.mark.parametrize("dim", [2, 3])
def test_collision_conservation(oracle_mod, dim):
    """Orders 0 and 1 are carried through the collision: the zeroth moment
    changes by exactly the source, the first moment not at all."""
    sim = sim_for(oracle_mod, dim, omega_bulk=1.3, omega_hi=0.7)
    c = lattice(dim)
    rng = np.random.default_rng(10 + dim)
    for _ in range(10):
        g, rho, u, gr, lam = random_cell(rng, dim)
        gs, xi, ph = sim.collide_cell(g, rho, u, gr, lam)
        assert abs(gs.sum() - g.sum() - xi.sum()) < 1e-15
        assert np.abs(c.T @ gs - c.T @ g).max() < 1e-15
        assert abs(ph - (g.sum() + 0.5 * rho * CS2 * lam)) < 1e-16  # Eq. 13a


@pytest.mark.parametrize("dim", [2, 3])
def test_rest_state_is_a_fixed_point(oracle_mod, dim):
    """No velocity, no gradient, no source: the populations stay zero."""
    sim = sim_for(oracle_mod, dim)
    Q = 9 if dim == 2 else 27
    gs, xi, ph = sim.collide_cell(np.zeros(Q), 0.8, [0, 0, 0], [0, 0, 0], 0.0)
    # g^eq = w (P_h - rho cs^2) + cs^2 f^eq cancels only to rounding
    assert np.abs(gs).max() < 1e-16 and not xi.any() and ph == 0.0


@pytest.mark.parametrize("dim", [2, 3])
def test_all_rates_one_is_bgk(oracle_mod, dim):
    """With every relaxation rate 1 and a uniform density the cumulant
    collision must return the textbook BGK result for omega = 1:
    g* = g^eq + Xi/2, g^eq_i = w_i (P_h - rho cs^2) + cs^2 f^eq_i (Eq. 10, 12)."""
    nu = (1.0 - 0.5) * CS2  # omega_s = 1
    sim = sim_for(oracle_mod, dim, nu=nu, omega_bulk=1.0, omega_hi=1.0)
    assert abs(sim.omega_s - 1.0) < 1e-15
    c = lattice(dim)
    w = weights(c)
    rng = np.random.default_rng(20 + dim)
    for _ in range(10):
        g, rho, u, _, lam = random_cell(rng, dim)
        gs, xi, ph = sim.collide_cell(g, rho, u, [0, 0, 0], lam)
        cu = c @ u
        feq = w * rho * (1 + cu / CS2 + cu ** 2 / (2 * CS2 ** 2) - (u @ u) / (2 * CS2))
        P_h = g.sum() + 0.5 * rho * CS2 * lam
        geq = w * (P_h - rho * CS2) + CS2 * feq
        xi_ref = w * rho * CS2 * lam
        assert np.allclose(xi, xi_ref, rtol=0, atol=1e-17)
        assert np.allclose(gs, geq + 0.5 * xi_ref, rtol=0, atol=2e-15)


def moment_indices(dim):
    Q = 9 if dim == 2 else 27
    return {(j % 3, (j // 3) % 3, j // 9): j for j in range(Q)}


@pytest.mark.parametrize("dim", [2, 3])
def test_each_moment_class_relaxes_at_its_rate(oracle_mod, dim):
    """Perturb the pre-conditioned populations away from equilibrium along
    one central moment and check its post-collision deviation is
    (1 - omega) times the perturbation, with omega = omega_s for shear
    (xy and xx-yy), omega_bulk for the trace, omega_hi for orders >= 3."""
    wb, wh = 1.25, 0.6
    sim = sim_for(oracle_mod, dim, omega_bulk=wb, omega_hi=wh)
    ws = sim.omega_s
    c = lattice(dim)
    w = weights(c)
    idx = moment_indices(dim)
    Q = len(c)
    rng = np.random.default_rng(30 + dim)
    rho = 0.9
    u = np.array([0.03, -0.02, 0.01 if dim == 3 else 0.0])
    P_h = 2e-3
    cu = c @ u
    feq = w * rho * (1 + cu / CS2 + cu ** 2 / (2 * CS2 ** 2) - (u @ u) / (2 * CS2))
    geq = w * (P_h - rho * CS2) + CS2 * feq
    base_Pi = sim.central_moments(geq / (rho * CS2), u)
    eps = 1e-7
    cases = [({(1, 1, 0): 1.0}, ws), ({(2, 0, 0): 1.0, (0, 2, 0): -1.0}, ws),
             ({(2, 1, 0): 1.0}, wh), ({(2, 2, 0): 1.0}, wh)]
    if dim == 2:
        cases.append(({(2, 0, 0): 1.0, (0, 2, 0): 1.0}, wb))
    else:
        cases += [({(2, 0, 0): 1.0, (0, 2, 0): 1.0, (0, 0, 2): 1.0}, wb), ({(0, 1, 1): 1.0}, ws),
                  ({(1, 1, 1): 1.0}, wh), ({(2, 1, 1): 1.0}, wh), ({(1, 2, 2): 1.0}, wh), ({(2, 2, 2): 1.0}, wh)]
    for pert, omega in cases:
        dPi = np.zeros(Q)
        for key, val in pert.items():
            dPi[idx[key]] = val * eps
        # g with zero source (Lambda = 0, grad rho = 0): f' = g / (rho cs^2)
        g = rho * CS2 * sim.central_moments_inverse(base_Pi + dPi, u)
        # keep P_h: the perturbation leaves orders 0-1 untouched
        gs, _, _ = sim.collide_cell(g, rho, u, [0, 0, 0], 0.0)
        Pis = sim.central_moments(gs / (rho * CS2), u)
        dev = Pis - base_Pi
        for key, val in pert.items():
            got = dev[idx[key]] / (val * eps)
            assert abs(got - (1.0 - omega)) < 1e-5, (dim, pert, key, got, 1.0 - omega)
