"""Learned warm start: training data from the solver, training and evaluation.

Every arithmetic step runs in the library's CUDA kernels through the C ABI:
the batched solver produces the ADMM solutions (many closed loops of the same
plant in one persistent launch per MPC step), the feature/target kernels turn
them into (patch state -> Phi rows, Lambda rows) pairs, and the network's BF16
forward/backward/AdamW kernels train on them.  PyTorch only holds the device
buffers, shuffles batches and normalises targets.

Training pairs come from the converged MPC steps of closed loops started at
random x(0) ~ U[-0.9, 0.9]: the states a running controller visits.  Steps
whose boxes cannot be met (they stop at max_iter) are left out.
"""
from __future__ import annotations

import dataclasses
from typing import List, Optional

import numpy as np

from . import instances as I


@dataclasses.dataclass
class Pairs:
    feats: object     # torch [n, d_in] (device)
    targets: object   # torch [n, d_out] (device)
    steps_used: int
    steps_skipped: int


def replicate(problem, x0s):
    """One context instance per initial state (same plant)."""
    probs = []
    for x0 in x0s:
        p = dataclasses.replace(problem)
        p.x0 = np.asarray(x0, np.float64)
        probs.append(p)
    return probs


def closed_loop_pairs(problem, x0s, steps: int, skip_first: int = 0, plant: bool = True) -> Pairs:
    """Runs len(x0s) closed loops of `steps` MPC steps in one batched context
    and keeps the pairs of converged steps.  Every step starts cold, so each
    target is the solution ADMM reaches from zero for that state (Phi at the
    optimum is not unique; a history-dependent start would make the targets
    depend on the path).  plant=True adds each member's plant blocks to the
    network input."""
    import torch
    import paper_2103_14990_gb300 as pkg
    B = len(x0s)
    s = pkg.Solver(replicate(problem, x0s))
    s.set_option(pkg.OPT_EXPORT_PHI, 1)
    s.set_option(pkg.OPT_LEARN_PLANT, 1 if plant else 0)
    n = problem.n_sub
    x = torch.tensor(np.concatenate(x0s).astype(np.float32), device="cuda")
    xn = torch.empty_like(x)
    u = torch.empty(B * n, problem.nu, device="cuda")
    feats, targets = [], []
    used = skipped = 0
    for tau in range(steps):
        f = s.learned_features(x)
        rc, st = s.step(x, u, xn, warm=pkg.WARM_COLD)
        if tau >= skip_first:
            tg = s.learned_targets()
            for b, sb in enumerate(st):
                if sb["status"] == pkg.DLMPC_OK:
                    feats.append(f[b * n:(b + 1) * n].clone())
                    targets.append(tg[b * n:(b + 1) * n].clone())
                    used += 1
                else:
                    skipped += 1
        x, xn = xn, x
    s.close()
    return Pairs(torch.cat(feats), torch.cat(targets), used, skipped)


def train(pairs: Pairs, hidden: int = 256, epochs: int = 20, batch: int = 2048, lr: float = 1e-3,
          weight_decay: float = 1e-5, seed: int = 0, log: Optional[list] = None):
    """Trains the network on normalised targets; returns the MLP with its
    output de-normalisation set."""
    import torch
    import paper_2103_14990_gb300 as pkg
    X, Y = pairs.feats, pairs.targets
    mean = Y.mean(0)
    std = Y.std(0).clamp_min(1e-4)
    Yn = ((Y - mean) / std).contiguous()
    mlp = pkg.MLP(X.shape[1], hidden, Y.shape[1], seed=seed)
    mlp.set_params(mlp.get_params(), scale=std.cpu().numpy(), shift=mean.cpu().numpy())
    g = torch.Generator(device="cpu").manual_seed(seed)
    n = X.shape[0]
    for ep in range(epochs):
        perm = torch.randperm(n, generator=g).to(X.device)
        last = None
        for i in range(0, n - batch + 1, batch):
            idx = perm[i:i + batch]
            xb, yb = X[idx].contiguous(), Yn[idx].contiguous()
            last = mlp.train_step(xb, yb, lr, weight_decay, want_loss=(i + 2 * batch > n))
        if log is not None:
            log.append(last)
    return mlp


def prediction_error(mlp, pairs: Pairs) -> float:
    """Relative Frobenius error of the de-normalised network output on pairs."""
    import torch
    y = mlp.forward(pairs.feats.contiguous())
    return float(torch.linalg.norm(y - pairs.targets) / torch.linalg.norm(pairs.targets))


def compare_starts(problem, mlp, states, max_iter: Optional[int] = None, eps: Optional[float] = None,
                   plant: bool = True):
    """ADMM iterations to Conv from each state: cold start vs learned start.
    Returns (cold_iters, learned_iters, cold_status, learned_status, u_cold, u_learned)."""
    import torch
    import paper_2103_14990_gb300 as pkg
    B = len(states)
    probs = replicate(problem, states)
    for p in probs:
        if max_iter is not None:
            p.max_iter = max_iter
        if eps is not None:
            p.eps_p = p.eps_d = eps
    s = pkg.Solver(probs)
    s.set_option(pkg.OPT_LEARN_PLANT, 1 if plant else 0)
    s.attach_mlp(mlp)
    n = problem.n_sub
    x = torch.tensor(np.concatenate(states).astype(np.float32), device="cuda")
    u = torch.empty(B * n, problem.nu, device="cuda")
    _, st_c = s.step(x, u, None, warm=pkg.WARM_COLD)
    u_c = u.cpu().numpy().copy()
    _, st_l = s.step(x, u, None, warm=pkg.WARM_LEARNED)
    u_l = u.cpu().numpy().copy()
    s.close()
    return (np.array([a["iters"] for a in st_c]), np.array([a["iters"] for a in st_l]),
            np.array([a["status"] for a in st_c]), np.array([a["status"] for a in st_l]), u_c, u_l)


def heldout_states(problem, seed: int, trajectories: int, steps: int):
    """States visited by closed loops from held-out x(0) draws, with the status
    of their MPC step (cold start): returns (states [m, n_sub, nx], status [m])."""
    import torch
    import paper_2103_14990_gb300 as pkg
    x0s = I.random_x0(problem.n_sub, trajectories, seed)
    s = pkg.Solver(replicate(problem, x0s))
    n = problem.n_sub
    x = torch.tensor(np.concatenate(x0s).astype(np.float32), device="cuda")
    xn = torch.empty_like(x)
    u = torch.empty(trajectories * n, problem.nu, device="cuda")
    states, status = [], []
    for tau in range(steps):
        xs = x.cpu().numpy().reshape(trajectories, n, problem.nx).copy()
        rc, st = s.step(x, u, xn, warm=pkg.WARM_COLD if tau == 0 else pkg.WARM_PREVIOUS)
        for b in range(trajectories):
            states.append(xs[b])
            status.append(st[b]["status"])
        x, xn = xn, x
    s.close()
    return np.array(states), np.array(status)


def heldout_trajectories(problem, seed: int, trajectories: int, steps: int):
    """Closed loops from held-out x(0) draws (previous-step warm starts, one
    batched context): the visited states [trajectories, steps, n_sub, nx]
    and the status of each step [trajectories, steps]."""
    states, status = heldout_states(problem, seed, trajectories, steps)
    n, nx = problem.n_sub, problem.nx
    # heldout_states lists the states step-major: step tau, then trajectory b
    st = states.reshape(steps, trajectories, n, nx).transpose(1, 0, 2, 3)
    ss = status.reshape(steps, trajectories).T
    return st, ss


def evaluate_starts(problem, mlp, trajectories, status, plant: bool = True):
    """Every visited state of every held-out trajectory solved on one
    single-instance context, in trajectory order, three ways to the same
    eps: cold (zeros), learned (the network's start), previous (the solution
    of the trajectory's previous state, the way a running controller starts).
    Only steps whose cold solve converged are kept.  Returns per-start arrays
    of iterations, statuses and whole-step milliseconds (CUDA events)."""
    import torch
    import paper_2103_14990_gb300 as pkg
    s = pkg.Solver([problem])
    s.set_option(pkg.OPT_LEARN_PLANT, 1 if plant else 0)
    s.set_option(pkg.OPT_TIMING, 1)
    s.attach_mlp(mlp)
    u = torch.empty(problem.n_sub, problem.nu, device="cuda")
    out = {k: {"iters": [], "status": [], "ms": []} for k in ("cold", "learned", "previous")}
    for tr, stt in zip(trajectories, status):
        xs = [torch.tensor(x.astype(np.float32), device="cuda") for x in tr]
        keep = []
        for k, x in enumerate(xs):
            _, st = s.step(x, u, None, warm=pkg.WARM_COLD)
            if st[0]["status"] == pkg.DLMPC_OK and stt[k] == pkg.DLMPC_OK:
                keep.append(k)
                out["cold"]["iters"].append(st[0]["iters"])
                out["cold"]["status"].append(st[0]["status"])
                out["cold"]["ms"].append(s.timing()[1])
        for k in keep:
            _, st = s.step(xs[k], u, None, warm=pkg.WARM_LEARNED)
            out["learned"]["iters"].append(st[0]["iters"])
            out["learned"]["status"].append(st[0]["status"])
            out["learned"]["ms"].append(s.timing()[1])
        # the previous-step start: walk the trajectory in order, each step
        # warm-started from the one before (all steps run, kept ones counted)
        for k, x in enumerate(xs):
            _, st = s.step(x, u, None, warm=pkg.WARM_COLD if k == 0 else pkg.WARM_PREVIOUS)
            if k in keep:
                out["previous"]["iters"].append(st[0]["iters"])
                out["previous"]["status"].append(st[0]["status"])
                out["previous"]["ms"].append(s.timing()[1])
    s.close()
    return {k: {f: np.array(v) for f, v in d.items()} for k, d in out.items()}
