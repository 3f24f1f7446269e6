"""Pins of the FP64 CPU discrete adjoint (``oracle/adjoint.py``).

Its forward step is a second, vectorised restatement of the 2-D coupled
step; it must equal the C oracle's step to rounding on every boundary type
(inlet plug and Poiseuille, Eq. 32 and constant-pressure outlets, adiabatic
and isothermal walls and solids, periodic faces).  Its gradient of the
flame position with respect to theta = (ln A, Ta, T_wall, u_in) must equal
central differences of the C oracle's flame position (relative steps 1e-4,
absolute in ln A), and must not depend on the checkpoint interval."""
import numpy as np
import pytest

from paper_2304_05657_gb300 import grad, inputs

torch = pytest.importorskip("torch")


def cases():
    cfg, solid, T, Y = inputs.channel(nx=30, ny=10, walls="isothermal", T_wall=350.0, ignite=(8, 18))
    g, T, Y = inputs.perturbed_state(cfg, solid, T, Y, seed=3)
    out = [("isothermal channel", cfg, solid, T, Y, g)]
    cfg2 = dict(cfg, poiseuille_inlet=True,
                bc=["inlet", "outlet", "wall_adiabatic", "wall_adiabatic", "periodic", "periodic"])
    out.append(("Poiseuille inlet, Eq. 32 outlet", cfg2, solid, T, Y, g))
    cfg3 = dict(cfg, bc=["periodic"] * 6, T_solid=350.0)
    s3 = solid.copy()
    s3[3:6, 10:14] = 1
    s3[7, 20] = 1
    g3, T3, Y3 = inputs.perturbed_state(cfg3, s3, T, Y, seed=4)
    out.append(("periodic with isothermal solids", cfg3, s3, T3, Y3, g3))
    cfg4 = dict(cfg, bc=["wall_isothermal", "outlet_pressure", "wall_isothermal", "inlet", "periodic", "periodic"])
    s4 = s3.copy()
    s4[0, 29] = 1
    g4, T4, Y4 = inputs.perturbed_state(cfg4, s4, T, Y, seed=5)
    out.append(("inlet on +y, walls on -x and -y, solids", cfg4, s4, T4, Y4, g4))
    cfg5 = dict(cfg, solid_isothermal=False,
                bc=["inlet", "outlet_pressure", "wall_adiabatic", "wall_adiabatic", "periodic", "periodic"])
    out.append(("adiabatic solids", cfg5, s3, T3, Y3, g3))
    return out


@pytest.mark.parametrize("case", cases(), ids=lambda c: c[0])
def test_forward_step_equals_the_c_oracle(oracle_mod, case):
    from oracle import adjoint

    _, cfg, solid, T, Y, g = case
    o = oracle_mod.Sim(cfg, solid)
    o.set_state(T, Y, g)
    o.step(5)
    To, Yo, go = o.get_state()
    ga, Ta, Ya = adjoint.forward(cfg, solid, T, Y, g, 5)
    assert np.abs(Ta - To).max() <= 1e-13 * np.abs(To).max()
    assert np.abs(Ya - Yo).max() <= 1e-13
    assert np.abs(ga - go).max() <= 1e-13 * np.abs(go).max()


def flame_case():
    cfg, solid, T, Y = inputs.channel(nx=24, ny=10, walls="isothermal", T_wall=350.0, u_in=0.01)
    T, Y = inputs.ignition_fields(cfg, solid, 8, 16)
    return cfg, solid, T, Y


def central_fd_oracle(oracle_mod, cfg, solid, T, Y, steps):
    def J(theta):
        o = oracle_mod.Sim(grad.apply_theta(cfg, theta), solid)
        o.set_state(T, Y)
        o.step(steps)
        return o.diagnostics()["x_f"] * cfg["dx"]

    th = grad.theta_of(cfg)
    fd = np.zeros(4)
    for k in range(4):
        h = 1e-4 if k == 0 else 1e-4 * abs(th[k])
        tp, tm = th.copy(), th.copy()
        tp[k] += h
        tm[k] -= h
        fd[k] = (J(tp) - J(tm)) / (2 * h)
    return J(th), fd


def test_adjoint_equals_central_differences_of_the_c_oracle(oracle_mod):
    """Measured agreement: 2e-9 (ln A), 2e-7 (Ta), 3e-6 (T_wall), 3e-10
    (u_in); the bar 1e-5 covers the O(h^2) truncation of the differences."""
    from oracle import adjoint

    cfg, solid, T, Y = flame_case()
    steps = 60
    J, g = adjoint.adjoint_gradient(cfg, solid, T, Y, steps)
    Jo, fd = central_fd_oracle(oracle_mod, cfg, solid, T, Y, steps)
    assert abs(J - Jo) <= 1e-13 * abs(Jo)
    assert np.all(np.abs(g - fd) <= 1e-5 * np.abs(fd)), (g, fd)
    Jc, gc = adjoint.adjoint_gradient(cfg, solid, T, Y, steps, checkpoint_every=7)
    assert Jc == J and np.allclose(gc, g, rtol=1e-13, atol=0)


def test_adjoint_with_solids_and_the_eq32_outlet(oracle_mod):
    """Isothermal in-domain solids (the T_wall parameter moves them with the
    walls), Poiseuille inlet and the Eq. 32 outlet."""
    from oracle import adjoint

    cfg, solid, T, Y = inputs.channel(nx=26, ny=12, walls="isothermal", T_wall=330.0, u_in=0.012,
                                      poiseuille_inlet=True, T_solid=330.0)
    cfg["bc"] = ["inlet", "outlet", "wall_isothermal", "wall_isothermal", "periodic", "periodic"]
    solid[4:7, 5:8] = 1
    T, Y = inputs.ignition_fields(cfg, solid, 10, 18)
    steps = 30
    J, g = adjoint.adjoint_gradient(cfg, solid, T, Y, steps)
    Jo, fd = central_fd_oracle(oracle_mod, cfg, solid, T, Y, steps)
    assert abs(J - Jo) <= 1e-13 * abs(Jo)
    assert np.all(np.abs(g - fd) <= 1e-5 * np.abs(fd)), (g, fd)


def test_quench_distance_objective_closed_form():
    """Only the cells of one row react (the others are cold): the soft
    minimum of the wall distance is that row's distance to the nearest cold
    wall, half-way between cells: row y of an isothermal channel of height
    H is min(y + 1/2, H - y - 1/2) from the walls."""
    from oracle import adjoint

    nx, ny = 20, 11
    cfg = inputs.base_config(dim=2, nx=nx, ny=ny, bc=["inlet", "outlet_pressure", "wall_isothermal",
                                                      "wall_isothermal", "periodic", "periodic"])
    solid = np.zeros((ny, nx), np.uint8)
    st = adjoint.Step(cfg, solid)
    for row in (0, 3, 5, 8):
        T = np.full(nx * ny, 300.0)
        T.reshape(ny, nx)[row, :] = 1800.0
        Y = np.tile(np.asarray(cfg["Y_in"])[:, None], (1, nx * ny))
        J = float(st.quench_distance(torch.as_tensor(T), torch.as_tensor(Y), st.theta0()))
        d = min(row + 0.5, ny - row - 0.5)
        # the cold rows' rate exp(-Ta/300) / exp(-Ta/1800) ~ 1e-18 contributes nothing measurable
        assert abs(J - d) <= 1e-9 * d, (row, J, d)
    # a solid block: distance to the nearest solid cell along the axes
    solid[5, 10] = 1
    st2 = adjoint.Step(dict(cfg, bc=["periodic"] * 6), solid)
    c = 5 * nx + 7
    assert st2.geo.wall_distance[list(st2.geo.fluid).index(c)] == 2.5


def test_quench_adjoint_equals_central_differences_of_the_c_oracle(oracle_mod):
    """The quenching-distance objective of the C oracle's final state
    (evaluated by the objective pinned above), differentiated by central
    differences, against the reverse accumulation: 1e-4 (measured 3e-5)."""
    from oracle import adjoint

    cfg, solid, T, Y = inputs.channel(nx=40, ny=12, walls="isothermal", T_wall=350.0, u_in=0.004)
    T, Y = inputs.ignition_fields(cfg, solid, 10, 30, burnt=False)
    steps = 40
    J, g = adjoint.adjoint_gradient(cfg, solid, T, Y, steps, objective="quench_distance")

    def Jq(theta):
        c = grad.apply_theta(cfg, theta)
        o = oracle_mod.Sim(c, solid)
        o.set_state(T, Y)
        o.step(steps)
        To, Yo, _ = o.get_state()
        st = adjoint.Step(c, solid)
        return float(st.quench_distance(torch.as_tensor(To), torch.as_tensor(Yo), st.theta0()))

    th = grad.theta_of(cfg)
    assert abs(J - Jq(th)) <= 1e-12 * abs(J)
    for k in range(4):
        h = 1e-4 if k == 0 else 1e-4 * abs(th[k])
        tp, tm = th.copy(), th.copy()
        tp[k] += h
        tm[k] -= h
        fd = (Jq(tp) - Jq(tm)) / (2 * h)
        assert abs(g[k] - fd) <= 1e-4 * abs(fd), (k, g[k], fd)
