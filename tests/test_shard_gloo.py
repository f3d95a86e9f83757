"""Spatial sharding of one network over two to four ranks (gloo, CPU): the
partitioner, the halo index maps and the exchange of the row sums, and the
all-reduce of the Conv counts, against the single-process FP64 oracle.

Each rank runs the column-patch ADMM on its own patches only, its local
arithmetic taken from the oracle (the column blocks' projector and offsets,
the row clamp of the Phi-step), and learns every other contribution it reads
through `shard.exchange`.  The iterates of its patches must equal the
oracle's over the whole network (fixed K), and the stopped run must end at
the oracle's iteration count on every rank.
"""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

from oracle import dlmpc_oracle as O
from paper_2103_14990_gb300 import instances as I
from paper_2103_14990_gb300 import shard


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _problem(kind):
    """Input bounds of 0.1 bind on 13-14 rows at the stopped solution (96 and
    166 oracle iterations)."""
    if kind == "chain":
        return I.make_instance(12, 4, 1, seed=13, boxes=True, x0_dist="uniform", u_bound=0.1)
    return I.make_instance(16, 4, 1, graph="grid", seed=14, boxes=True, x0_dist="uniform", u_bound=0.1)


def _sharded_admm(p, plan, K, stop, group=None):
    """The ADMM of Alg. 2 on this rank's patches; returns ({j: Psi_j}, iters)."""
    import torch
    pat = shard.patches(p)
    nx, rs = p.nx, p.r_sub
    x = p.x0
    s_of = {m: float(sum(x[k] @ x[k] for k in pat[m])) for m in plan.members}
    blocks = {j: O.column_block(p, j) for j in plan.own}
    lay = O.Layout(p)
    Psi = {j: np.zeros((nx, rs * len(pat[j]))) for j in plan.own}
    Lam = {j: np.zeros((nx, rs * len(pat[j]))) for j in plan.own}
    G = torch.zeros(len(plan.slots) * rs, dtype=torch.float64)
    it = 0
    for it in range(1, K + 1):
        Gv = G.view(-1, rs).numpy()
        w = {m: sum(Gv[plan.slot_of[(m, s)]] for s in pat[m]) for m in plan.members}
        nc = 0
        for j in plan.own:
            # Phi-step of every row of every member (row clamp, oracle's formula)
            Phi = Psi[j] - Lam[j]
            for pos, m in enumerate(pat[j]):
                for r in range(rs):
                    g = O.global_row(p, m, r)
                    sm = s_of[m]
                    if sm == 0.0:
                        continue
                    wr = w[m][r]
                    z = min(max(p.rho * wr / (p.rho + 2.0 * lay.qw[g] * sm), lay.lo[g]), lay.hi[g])
                    Phi[:, pos * rs + r] += (z - wr) / sm * x[j]
            # Psi-step (the oracle's projector and min-norm offsets), Lambda-step
            new = np.stack([blocks[j].P @ (Phi[c] + Lam[j][c]) + blocks[j].q[c] for c in range(nx)])
            Lam[j] = Lam[j] + Phi - new
            r_j = np.linalg.norm(Phi - new)
            s_j = p.rho * np.linalg.norm(new - Psi[j])
            Psi[j] = new
            nc += int(not (r_j <= p.eps_p and s_j <= p.eps_d))
        # own contributions, then the halo exchange
        Gv = G.view(-1, rs).numpy()
        for j in plan.own:
            V = Psi[j] - Lam[j]
            for pos, m in enumerate(pat[j]):
                Gv[plan.slot_of[(m, j)]] = x[j] @ V[:, pos * rs:(pos + 1) * rs]
        shard.exchange(G, plan, group)
        total = shard.not_converged_total(nc, group=group)
        if stop and total == 0:
            break
    return Psi, it


def _worker(rank, world, port, kind, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    p = _problem(kind)
    owner = shard.partition(p, world)
    plan = shard.halo_plans(p, owner)[rank]
    psi_k, _ = _sharded_admm(p, plan, 15, stop=False)
    psi_s, its = _sharded_admm(p, plan, 2000, stop=True)
    out[rank] = ({j: v.tolist() for j, v in psi_k.items()}, {j: v.tolist() for j, v in psi_s.items()}, its)
    dist.destroy_process_group()


@pytest.mark.parametrize("kind,world", [("chain", 2), ("grid", 2), ("chain", 3), ("grid", 4)])
def test_sharded_admm_matches_the_oracle(kind, world):
    ctx = mp.get_context("spawn")
    with ctx.Manager() as m:
        out = m.dict()
        mp.start_processes(_worker, args=(world, _free_port(), kind, out), nprocs=world, start_method="spawn")
        res = dict(out)
    p = _problem(kind)
    o = O.Oracle(p)
    ref_k = O.column_major_state(o.lay, O.admm(o.lay, o.blocks, p.x0, fixed_iters=15).Psi)
    stopped = O.admm(o.lay, o.blocks, p.x0, max_iter=2000)
    ref_s = O.column_major_state(o.lay, stopped.Psi)
    seen = set()
    for r in range(world):
        psi_k, psi_s, its = res[r]
        assert its == stopped.iters
        for j, v in psi_k.items():
            assert np.allclose(np.array(v), ref_k[j], rtol=0, atol=1e-12)
            seen.add(j)
        for j, v in psi_s.items():
            assert np.allclose(np.array(v), ref_s[j], rtol=0, atol=1e-12)
    assert seen == set(range(p.n_sub))


def test_halo_maps_cover_exactly_the_remote_contributions():
    """Every slot a rank reads is either written by itself or received from
    its owner, once; send and receive lists pair up slot for slot."""
    p = I.make_instance(30, 4, 2, graph="grid", seed=3, boxes=False)
    for ranks in (2, 3, 5):
        owner = shard.partition(p, ranks)
        sizes = np.bincount(owner, minlength=ranks)
        assert sizes.max() - sizes.min() <= 1
        plans = shard.halo_plans(p, owner)
        for pl in plans:
            got = set()
            for q, idx in pl.recv.items():
                assert len(idx) == len(plans[q].send[pl.rank])
                for k in idx:
                    m, s = pl.slots[k]
                    assert owner[s] == q and k not in got
                    got.add(k)
            for k, (m, s) in enumerate(pl.slots):
                assert (owner[s] == pl.rank) != (k in got)
            for q, idx in pl.send.items():
                for k, kq in zip(idx, plans[q].recv[pl.rank]):
                    assert pl.slots[k] == plans[q].slots[kq]


def test_partition_keeps_spatial_blocks():
    p = I.make_instance(64, 4, 1, graph="grid", seed=3, boxes=False)
    owner = shard.partition(p, 4)
    # row bands of the 8 x 8 grid: rank r owns rows 2r, 2r + 1
    assert all(owner[v] == (v // 8) // 2 for v in range(64))
