"""Spatial sharding of one DLMPC network over several ranks (Sec. V: the
fully distributed setting), data plane only.

In the column-patch form every column patch j, after its Psi- and
Lambda-steps, writes one row sum per row of each member m of Patch(j):
G[m][j][r] = sum over j's columns c of (Psi - Lambda)[row (m, r), c] x_c.
The Phi-step of a row of m needs w_r = sum over s in Patch(m) of G[m][s][r],
and a patch recomputes the Phi rows of all its members.  With the patches
split over ranks, a rank therefore needs, for every member m of its own
patches, the contributions G[m][s] of every s in Patch(m): those of patches
owned elsewhere (up to 2d hops away) come in by one exchange per iteration,
and the Conv decision takes one all-reduce of the not-converged counts.

This module holds the partitioner, the halo index maps and the exchange
(torch.distributed point-to-point into local buffers: gloo on CPU, NCCL on
GPUs; no peer-memory loads), nothing of the ADMM arithmetic.  One slot is
the r_sub row sums G[m][s] of one (member m, patch s) pair.
"""
from __future__ import annotations

import collections
import dataclasses
from typing import Dict, List, Tuple

import numpy as np


def _hops(prob, src: int, max_hops: int) -> Dict[int, int]:
    dist = {src: 0}
    queue = collections.deque([src])
    while queue:
        v = queue.popleft()
        if dist[v] == max_hops:
            continue
        for w in prob.adj_idx[prob.adj_ptr[v]:prob.adj_ptr[v + 1]]:
            w = int(w)
            if w not in dist:
                dist[w] = dist[v] + 1
                queue.append(w)
    return dist


def patches(prob) -> List[List[int]]:
    """Patch(j) = subsystems within d hops of j, ascending, for every j."""
    return [sorted(_hops(prob, j, prob.d)) for j in range(prob.n_sub)]


def partition(prob, ranks: int) -> np.ndarray:
    """owner[j] of every subsystem (and of its column patch): contiguous
    spatial blocks -- ranges of a chain, bands of rows of a grid (row-major
    numbering), else ranges of a breadth-first order -- with sizes differing
    by at most one subsystem."""
    n = prob.n_sub
    if ranks < 1 or ranks > n:
        raise ValueError("ranks must be in 1..n_sub")
    if prob.graph in ("chain", "grid"):
        order = np.arange(n)                      # row-major grid numbering keeps bands contiguous
    else:
        order = np.array(list(_hops(prob, 0, n)), dtype=np.int64)
    owner = np.empty(n, np.int32)
    bounds = np.linspace(0, n, ranks + 1).round().astype(int)
    for r in range(ranks):
        owner[order[bounds[r]:bounds[r + 1]]] = r
    return owner


@dataclasses.dataclass
class HaloPlan:
    """The slots one rank holds and exchanges.

    own      patches (= subsystems) this rank owns, ascending
    members  every member of an own patch (the rows this rank recomputes)
    slots    (m, s) pairs of the local exchange buffer: m in members, s in
             Patch(m); slot k occupies floats [k r_sub, (k + 1) r_sub)
    send     per peer rank: local slot indices this rank writes (s own) and
             the peer needs (m is a member of one of the peer's patches)
    recv     per peer rank: local slot indices filled from that peer's send,
             in the same (m, s) order as the peer's send list"""
    rank: int
    own: List[int]
    members: List[int]
    slots: List[Tuple[int, int]]
    slot_of: Dict[Tuple[int, int], int]
    send: Dict[int, List[int]]
    recv: Dict[int, List[int]]
    r_sub: int


def halo_plans(prob, owner: np.ndarray) -> List[HaloPlan]:
    """Halo index maps of every rank (built identically on all ranks)."""
    pat = patches(prob)
    ranks = int(owner.max()) + 1
    r_sub = prob.r_sub
    plans = []
    needed_by = []                                   # per rank: set of members it recomputes
    for r in range(ranks):
        own = [j for j in range(prob.n_sub) if owner[j] == r]
        mem = sorted({m for j in own for m in pat[j]})
        needed_by.append(set(mem))
        slots = [(m, s) for m in mem for s in pat[m]]
        plans.append(HaloPlan(r, own, mem, slots, {sl: k for k, sl in enumerate(slots)}, {}, {}, r_sub))
    for r, pl in enumerate(plans):
        for q in range(ranks):
            if q == r:
                continue
            # slots written here (s owned by r) that rank q needs, in a fixed order
            pairs = [(m, s) for (m, s) in plans[q].slots if owner[s] == r]
            if pairs:
                pl.send[q] = [pl.slot_of[(m, s)] for (m, s) in pairs]
                plans[q].recv[r] = [plans[q].slot_of[(m, s)] for (m, s) in pairs]
    return plans


def exchange(buf, plan: HaloPlan, group=None):
    """One halo exchange of the local slot buffer `buf` (a torch tensor of
    len(plan.slots) * r_sub floats): every peer's contributions to the slots
    this rank reads are received in place.  Point-to-point sends of packed
    slots (isend/irecv), so gloo and NCCL both serve it."""
    import torch
    import torch.distributed as dist
    rs = plan.r_sub
    view = buf.view(-1, rs)
    reqs, inbox = [], {}
    for q, idx in sorted(plan.recv.items()):
        inbox[q] = torch.empty((len(idx), rs), dtype=buf.dtype, device=buf.device)
        reqs.append(dist.irecv(inbox[q], src=q, group=group))
    for q, idx in sorted(plan.send.items()):
        out = view[torch.as_tensor(idx, device=buf.device)].contiguous()
        reqs.append(dist.isend(out, dst=q, group=group))
    for rq in reqs:
        rq.wait()
    for q, idx in plan.recv.items():
        view[torch.as_tensor(idx, device=buf.device)] = inbox[q]
    return buf


def not_converged_total(count: int, device="cpu", group=None) -> int:
    """Conv over all ranks: the sum of the ranks' not-converged patch counts
    (the network has converged when it is zero)."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([int(count)], dtype=torch.int64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
    return int(t.item())
