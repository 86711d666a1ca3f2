"""Spatial domain decomposition of the step, checked on CPU ranks: the box is split into z slabs,
one per gloo rank, each slab carries H ghost planes on either side, and after every step the ranks
exchange their outermost owned planes of f and phi. One step reads phi within 5 cells and f within
1 cell (the near-contact window of radius 3 on normals that need radius 1, then one streaming hop;
the phi update reads u one cell away), so H = 6 keeps every owned plane exact. The split run must
equal the unsplit oracle run bit for bit: this is the halo exchange a multi-GPU domain
decomposition would perform, with the oracle standing in for each GPU's step."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")

H = 6
STEPS = 8


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _case():
    from paper_2603_17481_gb300 import workloads as W
    cfg = W.base_config(3, 24, 20, 32, 19, rho_g=0.1, g=(0.0, 0.0, -1e-5))
    # two droplets facing each other across the slab border at z = 16, plus random velocity
    phi, u = W.droplet_fields(cfg, [(11.5, 9.5, 10.2), (12.0, 10.0, 21.9)], [4.5, 4.5],
                              [(0, 0, 0.01), (0, 0, -0.01)])
    u = u + W.noise(u.shape, 3, 2e-3)
    return cfg, W.to_q30_grid(phi), u


def _rank_main(rank, world, port, out, H=H):
    import torch.distributed as dist

    import oracle as O
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    cfg, phi, u = _case()
    nx, ny, nz, Q = cfg["nx"], cfg["ny"], cfg["nz"], cfg["Q"]
    P = O.make_params(cfg)
    f = O.init(P, phi, u)  # also fixes the global mean density used by the buoyancy force
    rho_bar = P.rho_bar
    nzl = nz // world
    z0 = rank * nzl
    zs = [(z0 - H + k) % nz for k in range(nzl + 2 * H)]  # owned planes with H ghosts each side
    plane = nx * ny
    f_ext = f.reshape(Q, nz, plane)[:, zs, :].copy()
    ph_ext = phi.reshape(nz, plane)[zs, :].copy()
    Pe = O.make_params(dict(cfg, nz=nzl + 2 * H))
    Pe.rho_bar = rho_bar
    up, down = (rank + 1) % world, (rank - 1) % world
    for _ in range(STEPS):
        f_new, ph_new, _ = O.step(Pe, f_ext, ph_ext, 1)
        f_ext = f_new.reshape(Q, nzl + 2 * H, plane)
        ph_ext = ph_new.reshape(nzl + 2 * H, plane)
        # halo exchange: the lowest H owned planes go down, the highest H go up
        send_lo = torch.from_numpy(np.concatenate([f_ext[:, H:2 * H].ravel(), ph_ext[H:2 * H].ravel()]))
        send_hi = torch.from_numpy(np.concatenate([f_ext[:, nzl:nzl + H].ravel(), ph_ext[nzl:nzl + H].ravel()]))
        recv_lo, recv_hi = torch.empty_like(send_lo), torch.empty_like(send_hi)
        reqs = [dist.isend(send_lo, down), dist.isend(send_hi, up),
                dist.irecv(recv_hi, up), dist.irecv(recv_lo, down)]
        for r in reqs:
            r.wait()
        nf = Q * H * plane
        f_ext[:, :H] = recv_lo[:nf].numpy().reshape(Q, H, plane)
        ph_ext[:H] = recv_lo[nf:].numpy().reshape(H, plane)
        f_ext[:, nzl + H:] = recv_hi[:nf].numpy().reshape(Q, H, plane)
        ph_ext[nzl + H:] = recv_hi[nf:].numpy().reshape(H, plane)
    out[rank] = (f_ext[:, H:H + nzl].copy(), ph_ext[H:H + nzl].copy())
    dist.destroy_process_group()


def _split_run(cfg, h):
    import torch.multiprocessing as mp
    port = _free_port()
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.spawn(_rank_main, args=(2, port, out, h), nprocs=2, join=True)
    f_split = np.concatenate([out[r][0] for r in (0, 1)], axis=1).reshape(cfg["Q"], -1)
    ph_split = np.concatenate([out[r][1] for r in (0, 1)], axis=0).reshape(-1)
    return f_split, ph_split


def test_two_slab_ranks_equal_the_unsplit_step(orc):
    import oracle as O
    cfg, phi, u = _case()
    P = O.make_params(cfg)
    f = O.init(P, phi, u)
    f_ref, ph_ref, _ = O.step(P, f, phi, STEPS)
    _, frep_ref, _ = O.nci(P, phi)
    assert np.any(frep_ref != 0.0)  # the repulsion acts across the slab border
    f_split, ph_split = _split_run(cfg, H)
    assert f_split.shape == f_ref.shape and ph_split.shape == ph_ref.shape
    assert np.array_equal(ph_split, ph_ref)
    assert np.array_equal(f_split, f_ref)
    # control: ghosts narrower than the step's reach corrupt the owned planes
    f_bad, ph_bad = _split_run(cfg, 2)
    assert not np.array_equal(ph_bad, ph_ref)
