"""Domain decomposition along x with halo exchange, on CPU ranks (gloo).

Two ranks each advance one x-slab of the oracle and exchange two columns of
T, Y_k and the populations with the neighbour after every step (the FD
stencils reach two cells, the pull one).  The gathered result must equal
the undecomposed run bit for bit: the halo width of the multi-GPU design is
sufficient and the slab update reads nothing beyond it."""
import os
import socket

import numpy as np
import pytest

HALO = 2
STEPS = 12


def _case():
    from paper_2304_05657_gb300 import inputs

    cfg, solid, T, Y = inputs.channel(nx=40, ny=11, walls="isothermal", ignite=(12, 26))
    solid = solid.copy()
    solid[4:7, 18:21] = 1  # an obstacle across the cut
    T, Y = inputs.ignition_fields(cfg, solid, 12, 26)
    g, T, Y = inputs.perturbed_state(cfg, solid, T, Y, seed=21)
    return cfg, solid, T, Y, g


def _worker(rank, world, port, out_path):
    import torch
    import torch.distributed as dist

    import oracle

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    cfg, solid, T, Y, g = _case()
    nx, ny = cfg["nx"], cfg["ny"]
    cut = nx // 2
    x0, x1 = (0, cut) if rank == 0 else (cut, nx)
    sim = oracle.Sim(cfg, solid)
    sim.set_state(T, Y, g)
    for _ in range(STEPS):
        sim.step_slab(x0, x1)
        T2, Y2, g2 = sim.get_state()
        state = np.concatenate([T2[None], Y2, g2]).reshape(-1, ny, nx)
        if rank == 0:
            send = np.ascontiguousarray(state[:, :, cut - HALO:cut])
            recv = np.empty_like(send)
            dist.send(torch.from_numpy(send), dst=1)
            dist.recv(t := torch.from_numpy(recv), src=1)
            state[:, :, cut:cut + HALO] = t.numpy()
        else:
            send = np.ascontiguousarray(state[:, :, cut:cut + HALO])
            recv = np.empty_like(send)
            dist.recv(t := torch.from_numpy(recv), src=0)
            dist.send(torch.from_numpy(send), dst=0)
            state[:, :, cut - HALO:cut] = t.numpy()
        flat = state.reshape(state.shape[0], -1)
        sim.set_state(flat[0], flat[1:6], flat[6:])
    T2, Y2, g2 = sim.get_state()
    state = np.concatenate([T2[None], Y2, g2]).reshape(-1, ny, nx)
    mine = torch.from_numpy(np.ascontiguousarray(state[:, :, x0:x1]))
    if rank == 0:
        other = torch.empty((state.shape[0], ny, nx - cut), dtype=torch.float64)
        dist.recv(other, src=1)
        full = np.concatenate([mine.numpy(), other.numpy()], axis=2)
        np.save(out_path, full)
    else:
        dist.send(mine, dst=0)
    dist.destroy_process_group()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_two_rank_slab_decomposition_is_bitwise_exact(tmp_path, oracle_mod):
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp

    out = str(tmp_path / "full.npy")
    mp.start_processes(_worker, args=(2, _free_port(), out), nprocs=2, join=True, start_method="spawn")
    got = np.load(out)
    cfg, solid, T, Y, g = _case()
    sim = oracle_mod.Sim(cfg, solid)
    sim.set_state(T, Y, g)
    sim.step(STEPS)
    T2, Y2, g2 = sim.get_state()
    ref = np.concatenate([T2[None], Y2, g2]).reshape(-1, cfg["ny"], cfg["nx"])
    assert np.array_equal(got, ref)
