"""Forward-mode (tangent-linear) gradients of flame observables with respect
to theta = (ln A, Ta, T_wall, u_in), checked against central finite
differences with relative step 1e-4 (absolute 1e-4 in ln A) computed with
the FP64 GPU step and with the FP64 CPU oracle: <= 1e-4 relative per
component."""
import math

import numpy as np
import pytest

from paper_2304_05657_gb300 import grad, inputs, lbfd

pytestmark = pytest.mark.gpu

STEPS = 150
H = 1e-4


def case():
    cfg, solid, T, Y = inputs.channel(nx=64, ny=20, walls="isothermal", T_wall=350.0, u_in=0.01)
    T, Y = inputs.ignition_fields(cfg, solid, 20, 40)
    return cfg, solid, T, Y


def J_gpu(cfg, solid, T, Y, theta, objective):
    c = grad.apply_theta(cfg, theta)
    c["precision"] = "fp64"
    s = lbfd.Solver(c, solid)
    s.variant = 0
    s.init_fields(T, Y)
    s.step(STEPS)
    d = s.diagnostics()
    s.close()
    return d["x_f"] * cfg["dx"] if objective == lbfd.OBJ_FLAME_POSITION else d["heat_release"]


def J_oracle(oracle_mod, cfg, solid, T, Y, theta, objective):
    c = grad.apply_theta(cfg, theta)
    o = oracle_mod.Sim(c, solid)
    o.set_state(T, Y)
    o.step(STEPS)
    d = o.diagnostics()
    return d["x_f"] * cfg["dx"] if objective == lbfd.OBJ_FLAME_POSITION else d["heat_release"]


def central_fd(fun, theta):
    g = np.zeros(4)
    for k in range(4):
        h = H if k == 0 else H * abs(theta[k])
        tp, tm = theta.copy(), theta.copy()
        tp[k] += h
        tm[k] -= h
        g[k] = (fun(tp) - fun(tm)) / (2 * h)
    return g


@pytest.mark.parametrize("objective", [lbfd.OBJ_FLAME_POSITION, lbfd.OBJ_HEAT_RELEASE])
def test_tangent_gradient_matches_central_differences(lbfd_lib, oracle_mod, objective):
    cfg, solid, T, Y = case()
    theta = grad.theta_of(cfg)
    J, g = grad.run_tangent(cfg, solid, T, Y, STEPS, objective)
    assert abs(J - J_gpu(cfg, solid, T, Y, theta, objective)) <= 1e-12 * abs(J)
    fd_gpu = central_fd(lambda t: J_gpu(cfg, solid, T, Y, t, objective), theta)
    fd_cpu = central_fd(lambda t: J_oracle(oracle_mod, cfg, solid, T, Y, t, objective), theta)
    for k, name in enumerate(lbfd.THETA):
        assert abs(g[k] - fd_gpu[k]) <= 1e-4 * abs(fd_gpu[k]), (name, g[k], fd_gpu[k])
        assert abs(g[k] - fd_cpu[k]) <= 1e-4 * abs(fd_cpu[k]), (name, g[k], fd_cpu[k])
    assert np.all(np.abs(g) > 0)  # every parameter acts on the objective


@pytest.mark.parametrize("objective", [lbfd.OBJ_FLAME_POSITION, lbfd.OBJ_HEAT_RELEASE])
def test_mixed_tangent_gradient_matches_fp64_tangent(lbfd_lib, objective):
    """FP32 forward pass with FP64 Arrhenius above 1000 K and FP64
    accumulation of the objective: J within 1e-5 and every component of
    dJ/dtheta within 2e-3 of the FP64 tangent (FP32 rounding carried over
    150 steps through the state and its derivatives)."""
    cfg, solid, T, Y = case()
    J, g = grad.run_tangent(cfg, solid, T, Y, STEPS, objective)
    Jm, gm = grad.run_tangent(cfg, solid, T, Y, STEPS, objective, precision="tangent_mixed")
    assert abs(Jm - J) <= 1e-5 * abs(J), (Jm, J)
    for k, name in enumerate(lbfd.THETA):
        assert abs(gm[k] - g[k]) <= 2e-3 * abs(g[k]), (name, gm[k], g[k])


def test_adjoint_gradient_matches_tangent(lbfd_lib):
    """The discrete adjoint (reverse mode with checkpointed recomputation)
    and the tangent (forward mode) are both the exact derivative of the same
    discrete map, so they agree to rounding: 1e-9 relative per component;
    J equals the FP64 run's.  Checkpoint intervals 1, 7 and all steps give
    the same gradient (1e-12; atomic accumulation order aside)."""
    cfg, solid, T, Y = case()
    J, g = grad.run_tangent(cfg, solid, T, Y, STEPS)
    theta = grad.theta_of(cfg)
    ref = None
    for K in (STEPS, 7, 1):
        Ja, ga = grad.run_tangent(cfg, solid, T, Y, STEPS, precision="adjoint", checkpoint_every=K)
        assert abs(Ja - J) <= 1e-12 * abs(J), (K, Ja, J)
        for k, name in enumerate(lbfd.THETA):
            assert abs(ga[k] - g[k]) <= 1e-9 * abs(g[k]), (K, name, ga[k], g[k])
        if ref is None:
            ref = ga
        else:
            assert np.allclose(ga, ref, rtol=1e-12, atol=0), (K, ga, ref)
    assert np.all(np.isfinite(theta))


def test_tangent_values_match_fp64_kernel(lbfd_lib):
    """The value part of the tangent state is the FP64 step."""
    cfg, solid, T, Y = case()
    a = lbfd.Solver(dict(cfg, precision="tangent"), solid)
    b = lbfd.Solver(dict(cfg, precision="fp64"), solid)
    b.variant = 0
    for s in (a, b):
        s.init_fields(T, Y)
        s.step(60)
    for f in [lbfd.FIELD_T] + [lbfd.FIELD_Y0 + k for k in range(5)] + [lbfd.FIELD_G0 + i for i in range(9)]:
        x, y = a.read_field(f), b.read_field(f)
        assert np.linalg.norm(x - y) <= 1e-12 * max(np.linalg.norm(y), 1e-30), f
    # a state field's tangent is consistent with the gradient reduction
    dYF = a.read_tangent(lbfd.FIELD_Y0, 1)
    fluid = solid.ravel() == 0
    J, g = a.gradient(lbfd.OBJ_FLAME_POSITION)
    section = (solid[:, 0] == 0).sum()
    scale = cfg["dx"] / (cfg["Y_in"][0] * section)
    assert abs(dYF[fluid].sum() * scale - g[1]) <= 1e-12 * abs(g[1])


def test_autograd_function_backward(lbfd_lib):
    torch = pytest.importorskip("torch")
    cfg, solid, T, Y = case()
    theta = torch.tensor(grad.theta_of(cfg), dtype=torch.float64, requires_grad=True)
    J = grad.FlameObjective.apply(theta, cfg, solid, T, Y, 40, lbfd.OBJ_FLAME_POSITION)
    (2.0 * J).backward()
    J2, g = grad.run_tangent(cfg, solid, T, Y, 40)
    assert abs(J.item() - J2) <= 1e-14 * abs(J2)
    assert np.allclose(theta.grad.numpy(), 2.0 * g, rtol=1e-14, atol=0)
    assert math.isfinite(J.item())


def test_adjoint_matches_the_cpu_adjoint_and_central_differences(lbfd_lib):
    """The GPU discrete adjoint (reverse-mode tape of the CUDA step) against
    the FP64 CPU adjoint of the oracle (reverse accumulation through an
    independent restatement of the step): both are the transpose of the
    derivative of the same discrete map, so they agree to rounding, 1e-8
    relative per component; and directly against central differences of
    the FP64 GPU step, 1e-4."""
    from oracle import adjoint

    cfg, solid, T, Y = case()
    Jg, gg = grad.run_tangent(cfg, solid, T, Y, STEPS, precision="adjoint", checkpoint_every=50)
    Jc, gc = adjoint.adjoint_gradient(cfg, solid, T, Y, STEPS, checkpoint_every=50)
    assert abs(Jg - Jc) <= 1e-12 * abs(Jc), (Jg, Jc)
    for k, name in enumerate(lbfd.THETA):
        assert abs(gg[k] - gc[k]) <= 1e-8 * abs(gc[k]), (name, gg[k], gc[k])
    theta = grad.theta_of(cfg)
    fd = central_fd(lambda t: J_gpu(cfg, solid, T, Y, t, lbfd.OBJ_FLAME_POSITION), theta)
    for k, name in enumerate(lbfd.THETA):
        assert abs(gg[k] - fd[k]) <= 1e-4 * abs(fd[k]), (name, gg[k], fd[k])


def quench_case():
    cfg, solid, T, Y = inputs.channel(nx=40, ny=12, walls="isothermal", T_wall=350.0, u_in=0.004)
    T, Y = inputs.ignition_fields(cfg, solid, 10, 30, burnt=False)
    return cfg, solid, T, Y


def test_quench_distance_tangent_adjoint_cpu_and_fd(lbfd_lib):
    """The quenching-distance objective: the FP64 tangent, the GPU adjoint and
    the CPU adjoint agree (1e-8 relative per component; J to 1e-12), and all
    match central differences of the FP64 GPU step (1e-4)."""
    from oracle import adjoint

    cfg, solid, T, Y = quench_case()
    steps = 40
    Jt, gt = grad.run_tangent(cfg, solid, T, Y, steps, lbfd.OBJ_QUENCH_DISTANCE)
    Ja, ga = grad.run_tangent(cfg, solid, T, Y, steps, lbfd.OBJ_QUENCH_DISTANCE, precision="adjoint",
                              checkpoint_every=9)
    Jc, gc = adjoint.adjoint_gradient(cfg, solid, T, Y, steps, objective="quench_distance")
    assert abs(Jt - Jc) <= 1e-12 * Jc and abs(Ja - Jc) <= 1e-12 * Jc, (Jt, Ja, Jc)
    for k, name in enumerate(lbfd.THETA):
        assert abs(ga[k] - gc[k]) <= 1e-8 * abs(gc[k]), (name, ga[k], gc[k])
        assert abs(gt[k] - gc[k]) <= 1e-8 * abs(gc[k]), (name, gt[k], gc[k])

    def J_gpu_q(theta):
        c = grad.apply_theta(cfg, theta)
        c["precision"] = "tangent"
        s = lbfd.Solver(c, solid)
        s.init_fields(T, Y)
        s.step(steps)
        J, _ = s.gradient(lbfd.OBJ_QUENCH_DISTANCE)
        s.close()
        return J

    fd = central_fd(J_gpu_q, grad.theta_of(cfg))
    for k, name in enumerate(lbfd.THETA):
        assert abs(ga[k] - fd[k]) <= 1e-4 * abs(fd[k]), (name, ga[k], fd[k])


@pytest.mark.parametrize("objective", [lbfd.OBJ_FLAME_POSITION, lbfd.OBJ_QUENCH_DISTANCE])
def test_mixed_forward_adjoint_matches_fp64_adjoint(lbfd_lib, objective):
    """FP32 forward pass (the mixed kernels, FP64 Arrhenius above 1000 K),
    adjoint and gradient in FP64 at that trajectory: within 2e-3 of the FP64
    adjoint per component (FP32 rounding of the trajectory, as for the mixed
    tangent form), J within 1e-5."""
    cfg, solid, T, Y = case() if objective == lbfd.OBJ_FLAME_POSITION else quench_case()
    J, g = grad.run_tangent(cfg, solid, T, Y, STEPS, objective, precision="adjoint", checkpoint_every=40)
    Jm, gm = grad.run_tangent(cfg, solid, T, Y, STEPS, objective, precision="adjoint_mixed", checkpoint_every=40)
    assert abs(Jm - J) <= 1e-5 * abs(J), (Jm, J)
    for k, name in enumerate(lbfd.THETA):
        assert abs(gm[k] - g[k]) <= 2e-3 * abs(g[k]), (name, gm[k], g[k])


def test_adjoint_record_backward_and_autograd(lbfd_lib):
    """The forward/backward split: backward with seed s gives s dJ/dtheta;
    backward without a record is EINVAL; FlameObjective with the adjoint
    keeps only checkpoints in forward and sweeps in backward."""
    torch = pytest.importorskip("torch")
    cfg, solid, T, Y = case()
    steps = 60
    J1, g1 = grad.run_tangent(cfg, solid, T, Y, steps, precision="adjoint", checkpoint_every=25)
    s = grad.adjoint_solver(cfg, solid, T, Y, None, 25)
    J2 = s.adjoint_record(steps)
    g2 = s.adjoint_backward(-3.0)
    assert J2 == J1 and np.allclose(g2, -3.0 * g1, rtol=1e-12, atol=0)
    with pytest.raises(lbfd.LbfdError) as err:
        s.adjoint_backward(1.0)  # the record was consumed
    assert err.value.status == lbfd.EINVAL
    s.close()
    for prec in ("adjoint", "adjoint_mixed"):
        theta = torch.tensor(grad.theta_of(cfg), dtype=torch.float64, requires_grad=True)
        J = grad.FlameObjective.apply(theta, cfg, solid, T, Y, steps, lbfd.OBJ_FLAME_POSITION, prec, 25)
        (2.0 * J).backward()
        tol = 1e-12 if prec == "adjoint" else 2e-3
        assert abs(J.item() - J1) <= (1e-14 if prec == "adjoint" else 1e-5) * abs(J1)
        assert np.allclose(theta.grad.numpy(), 2.0 * g1, rtol=tol, atol=0), (prec, theta.grad, g1)
