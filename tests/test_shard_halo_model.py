"""CPU model of the panel-sharded ghost fill of the multi-GPU design (no GPU): two gloo ranks,
each owning three panels, exchange exactly the cells that the design says a rank needs --
the edge bands of depth 2H = k - 1 of every panel that shares an edge with one of its own --
and fill their own panels' ghost rings from their own cells plus what they received,
with the oracle's literal ghost iteration (section 3.3.1: ten sweeps of neighbour-panel
stencils that include the neighbours' ghosts).  The rings equal the single-process fill
bitwise; the FP64 mass, summed per rank in a fixed order and combined in rank order, equals
the single-process mass to round-off.  This checks the exchange lists, not a transport:
the design's transport is NCCL point-to-point on GPUs, which no run here has two of.
"""
import os
import socket
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
OWNED = ([0, 1, 4], [2, 3, 5])  # panels of rank 0 and rank 1


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _band(N, depth):
    i = np.arange(N)
    d1 = np.minimum(i, N - 1 - i)
    return np.minimum(d1[:, None], d1[None, :]) < depth  # [j][i]


def _needed(nbr, own, other):
    """Panels of `other` whose edge bands a rank owning `own` needs: the neighbours of its
    own panels that `other` owns (ascending)."""
    return sorted({int(r) for p in own for r in nbr[p] if int(r) in other})


def _rank(rank, world, port, k, N, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    from oracle import oracle as O
    from synth import noise_field, perturb_h
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        o = O.Oracle(N, k)
        H, me = (k - 1) // 2, (k + 1) // 2
        q = np.ascontiguousarray(perturb_h(o.rossby_haurwitz(), noise_field((6, N, N), 3)))
        nbr = o.edge_tables()["B"].reshape(6, 4, N, me)[:, :, 0, 0]
        band = _band(N, 2 * H)
        own, other = OWNED[rank], OWNED[1 - rank]
        # what the peer needs from me, and what I need from the peer (same band per panel)
        send_panels = _needed(nbr, other, own)
        recv_panels = _needed(nbr, own, other)
        send = torch.from_numpy(np.concatenate([q[:, p][:, band].ravel() for p in send_panels]))
        recv = torch.empty(len(recv_panels) * 3 * int(band.sum()), dtype=torch.float64)
        if rank == 0:
            dist.send(send, 1)
            dist.recv(recv, 1)
        else:
            dist.recv(recv, 0)
            dist.send(send, 0)
        local = np.zeros_like(q)
        local[:, own] = q[:, own]
        chunks = recv.numpy().reshape(len(recv_panels), 3, -1)
        for t, p in enumerate(recv_panels):
            local[:, p][:, band] = chunks[t]
        ext, _ = o.fill_ghosts(local)
        full, _ = o.fill_ghosts(q)
        ring = np.ones((N + 2 * H, N + 2 * H), bool)
        ring[H:-H, H:-H] = False
        same = all(np.array_equal(ext[:, p][:, ring], full[:, p][:, ring]) for p in own)
        # the mass diagnostic: per-rank FP64 partial in a fixed order, combined in rank order
        part = torch.tensor([float(np.sum(q[0, own])) * (np.pi / (2 * N)) ** 2], dtype=torch.float64)
        parts = [torch.zeros(1, dtype=torch.float64) for _ in range(world)]
        dist.all_gather(parts, part)
        mass = float(sum(float(x) for x in parts))
        out[rank] = (same, abs(mass - o.mass(q)) / abs(o.mass(q)), send.numel() * 8, send_panels, recv_panels)
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("k,N", [(3, 12), (5, 16)])
def test_two_ranks_fill_their_ghost_rings_from_the_exchanged_edge_bands(k, N):
    world, port = 2, _free_port()
    out = mp.get_context("spawn").Manager().dict()
    mp.spawn(_rank, args=(world, port, k, N, out), nprocs=world, join=True)
    H = (k - 1) // 2
    for r in range(world):
        same, mass_err, nbytes, send_panels, recv_panels = out[r]
        assert same, r
        assert mass_err < 1e-14, (r, mass_err)
        # every panel of the peer borders one of this rank's three panels here
        assert len(send_panels) == 3 and len(recv_panels) == 3
        assert nbytes == 3 * 3 * 8 * (N * N - (N - 4 * H) ** 2)
