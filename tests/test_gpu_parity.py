"""CUDA path against the FP64 oracle on the same seeded inputs.

Parity modes:
  fixed-K  both sides run exactly K ADMM iterations from the same start;
           ||X_gpu - X_oracle||_F / ||X_oracle||_F <= 1e-4 for Phi, Psi,
           Lambda (column-owned layout) and u(0).
  stopped  Conv on; iteration counts within a few of the oracle's, and at
           the oracle's count from the same start u, Psi (also per column
           patch) and Lambda within 1e-4 relative (absolute floor 1e-7);
           the stopped u itself within 1e-4 where the counts agree.
Every call goes through the C ABI (libdlmpc.so) via the ctypes binding.
"""
import dataclasses

import numpy as np
import pytest

from oracle import dlmpc_oracle as O
from paper_2103_14990_gb300 import instances as I
from parity_helpers import REL, max_patch_rel, rel, stopped_closed_loop

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    import torch
    assert torch.cuda.is_available()
    return torch


def gpu_solver(probs, torch):
    import paper_2103_14990_gb300 as pkg
    return pkg.Solver(probs)


def run_fixed(solver, torch, x0, K, warm=0, export=True):
    """K iterations from `warm`; with export=False the step runs on the
    compact iterate after its first iteration and phi comes back as None."""
    import paper_2103_14990_gb300 as pkg
    solver.set_option(pkg.OPT_FIXED_ITERS, K)
    solver.set_option(pkg.OPT_EXPORT_PHI, 1 if export else 0)
    x = torch.tensor(np.asarray(x0, np.float32).reshape(-1, solver.nx), device="cuda")
    u = torch.zeros(solver.n_sub, solver.nu, device="cuda")
    xn = torch.zeros_like(x)
    rc, st = solver.step(x, u, xn, warm=warm)
    phi, psi, lam = solver.get_state(phi=export)
    torch.cuda.synchronize()
    solver.set_option(pkg.OPT_FIXED_ITERS, 0)
    solver.set_option(pkg.OPT_EXPORT_PHI, 0)
    return (rc, st, phi.cpu().numpy() if export else None, psi.cpu().numpy(), lam.cpu().numpy(),
            u.cpu().numpy(), xn.cpu().numpy())


def _rho07():
    p = I.make_instance(16, 6, 2, seed=7, boxes=True, x0_dist="uniform", rho=0.7, u_bound=0.05, mpc_steps=6)
    p.x0 = 0.5 * p.x0
    return p


SMALL = {
    "chain10": lambda: I.chain10(),
    "chain16_T10_d3_box": lambda: I.make_instance(16, 10, 3, seed=1, boxes=True, x0_dist="uniform"),
    "grid5x5_T6_d2_box": lambda: I.make_instance(25, 6, 2, graph="grid", seed=2, boxes=True),
    "grid3x4_T4_d1": lambda: I.make_instance(12, 4, 1, graph="grid", seed=4, boxes=False, x0_dist="normal"),
    "chain1_T2": lambda: I.make_instance(1, 2, 1, seed=5, boxes=True),
    "chain7_T5_d6_nolocality": lambda: I.make_instance(7, 5, 6, seed=6, boxes=False, x0_dist="normal"),
    "chain16_T6_d2_rho07_box": _rho07,
}


@pytest.mark.parametrize("name", list(SMALL))
def test_operator_matches_oracle_projector(name, torch):
    p = SMALL[name]()
    s = gpu_solver([p], torch)
    for j in range(p.n_sub):
        N, q = s.operator(j)
        blk = O.column_block(p, j)
        assert N.shape[1] == blk.P.shape[0] - blk.rank          # same nullity
        assert np.max(np.abs(N @ N.T - blk.P)) < 2e-6            # N N^T = I - Z^+ Z
        assert np.max(np.abs(q - blk.q)) < 2e-6                  # Z^+ e_c
    s.close()


@pytest.mark.parametrize("name", list(SMALL))
@pytest.mark.parametrize("K", [1, 7, 60])
def test_fixed_iterations_parity(name, K, torch):
    p = SMALL[name]()
    o = O.Oracle(p)
    ref = O.admm(o.lay, o.blocks, p.x0, fixed_iters=K)
    s = gpu_solver([p], torch)
    rc, st, phi, psi, lam, u, xn = run_fixed(s, torch, p.x0, K)
    assert st[0]["iters"] == K
    assert rel(psi, ref.Psi) <= REL
    assert rel(lam, ref.Lam) <= REL or np.linalg.norm(ref.Lam) < 1e-6
    assert rel(phi, ref.Phi) <= REL
    u_ref = o.control(ref)
    assert rel(u, u_ref) <= REL or np.max(np.abs(u - u_ref)) < 1e-7
    xn_ref = o.dynamics(p.x0, u)  # dynamics of the GPU's own u, FP64
    assert np.max(np.abs(xn.reshape(-1) - xn_ref.reshape(-1))) < 1e-6
    s.close()


@pytest.mark.parametrize("name", list(SMALL))
@pytest.mark.parametrize("K", [1, 2, 3, 60])
def test_fixed_iterations_parity_compact(name, K, torch):
    """Iterations after the first on the compact iterate (Psi = q + N t,
    Lambda = x_c lhat), expanded at the end of the step: Psi, Lambda and u
    against the oracle, and against the full form of the same step."""
    import paper_2103_14990_gb300 as pkg
    p = SMALL[name]()
    o = O.Oracle(p)
    ref = O.admm(o.lay, o.blocks, p.x0, fixed_iters=K)
    s = gpu_solver([p], torch)
    rc, st, _, psi, lam, u, xn = run_fixed(s, torch, p.x0, K, export=False)
    assert st[0]["iters"] == K
    assert rel(psi, ref.Psi) <= REL
    assert rel(lam, ref.Lam) <= REL or np.linalg.norm(ref.Lam) < 1e-6
    u_ref = o.control(ref)
    assert rel(u, u_ref) <= REL or np.max(np.abs(u - u_ref)) < 1e-7
    s.set_option(pkg.OPT_COMPACT, 0)
    rc, st_f, _, psi_f, lam_f, u_f, _ = run_fixed(s, torch, p.x0, K, export=False)
    assert rel(psi, psi_f) <= 2e-5
    assert rel(u, u_f) <= 2e-5 or np.max(np.abs(u - u_f)) < 1e-7
    # residuals of the last iteration agree between the two forms
    # (absolute floor: FP32 rounding of Lambda and Psi themselves)
    scale = 1e-6 * max(np.linalg.norm(lam_f), np.linalg.norm(psi_f))
    assert abs(st[0]["r_max"] - st_f[0]["r_max"]) <= 1e-3 * st_f[0]["r_max"] + scale
    assert abs(st[0]["s_max"] - st_f[0]["s_max"]) <= 1e-3 * st_f[0]["s_max"] + scale
    # warm continuation from the expanded state
    s.set_option(pkg.OPT_COMPACT, 1)
    rc, st2, _, psi2, lam2, u2, _ = run_fixed(s, torch, p.x0, K, warm=pkg.WARM_PREVIOUS, export=False)
    ref2 = O.admm(o.lay, o.blocks, p.x0, Psi0=psi.astype(np.float64), Lam0=lam.astype(np.float64), fixed_iters=K)
    assert rel(psi2, ref2.Psi) <= REL
    assert rel(lam2, ref2.Lam) <= REL or np.linalg.norm(ref2.Lam) < 1e-6
    s.close()


@pytest.mark.parametrize("warm", ["cold", "previous"])
def test_stopped_closed_loop_chain10(warm, torch):
    """20 closed-loop MPC steps of the N=10 chain (cold and previous-step
    warm starts), stopped-run parity at 1e-4 (see stopped_closed_loop)."""
    p = I.chain10()
    stopped_closed_loop(p, torch, warm, p.mpc_steps, check_next=True)


def test_stopped_closed_loop_rho_not_one(torch):
    """The same with rho = 0.7 and active input bounds (30-50 rows at a bound
    per step): the Phi-step and the dual residual carry rho."""
    p = _rho07()
    stopped_closed_loop(p, torch, "previous", p.mpc_steps)


def test_batch_equals_single_instances(torch):
    """Instances solved together in one persistent launch give bit-identical
    results to the same instances solved alone."""
    probs = [SMALL["chain10"](), SMALL["grid5x5_T6_d2_box"](), SMALL["chain16_T10_d3_box"]()]
    sb = gpu_solver(probs, torch)
    x0 = np.concatenate([p.x0 for p in probs])
    rc, st, phi, psi, lam, u, xn = run_fixed(sb, torch, x0, 25)
    off = 0
    uoff = 0
    for p in probs:
        s1 = gpu_solver([p], torch)
        r1 = run_fixed(s1, torch, p.x0, 25)
        n = s1.info()["state_floats"]
        assert np.array_equal(psi[off:off + n], r1[3])
        assert np.array_equal(lam[off:off + n], r1[4])
        assert np.array_equal(u[uoff:uoff + p.n_sub], r1[5])
        off += n
        uoff += p.n_sub
        s1.close()
    sb.close()


def test_batch_stopping_per_instance(torch):
    """Each instance of a batch stops at its own convergence iteration."""
    import paper_2103_14990_gb300 as pkg
    probs = [SMALL["chain10"](), SMALL["grid3x4_T4_d1"]()]
    sb = gpu_solver(probs, torch)
    x = torch.tensor(np.concatenate([p.x0 for p in probs]).astype(np.float32), device="cuda")
    u = torch.zeros(sum(p.n_sub for p in probs), 1, device="cuda")
    rc, st = sb.step(x, u, None, warm=pkg.WARM_COLD)
    for p, s in zip(probs, st):
        o = O.Oracle(p)
        ref = O.admm(o.lay, o.blocks, p.x0)
        assert s["status"] == 0
        assert abs(s["iters"] - ref.iters) <= max(3, 0.02 * ref.iters)
    sb.close()


def test_host_buffer_step_matches_device_step(torch):
    import paper_2103_14990_gb300 as pkg
    p = SMALL["chain16_T10_d3_box"]()
    s = gpu_solver([p], torch)
    rc, u_h, xn_h, st_h = s.step_host(p.x0, warm=pkg.WARM_COLD)
    x = torch.tensor(p.x0.astype(np.float32), device="cuda")
    u = torch.zeros(p.n_sub, 1, device="cuda")
    xn = torch.zeros_like(x)
    rc2, st = s.step(x, u, xn, warm=pkg.WARM_COLD)
    assert np.array_equal(u.cpu().numpy().reshape(-1), u_h)
    assert np.array_equal(xn.cpu().numpy().reshape(-1), xn_h)
    assert st[0]["iters"] == st_h[0]["iters"]
    s.close()


def test_max_iter_status(torch):
    import paper_2103_14990_gb300 as pkg
    p = SMALL["chain10"]()
    p.max_iter = 3
    s = gpu_solver([p], torch)
    x = torch.tensor(p.x0.astype(np.float32), device="cuda")
    u = torch.zeros(p.n_sub, 1, device="cuda")
    rc, st = s.step(x, u, None, warm=pkg.WARM_COLD)
    assert rc == pkg.DLMPC_MAX_ITER and st[0]["status"] == pkg.DLMPC_MAX_ITER and st[0]["iters"] == 3
    s.close()


# threads per CTA span the three register tiers: <= 768, 769..896 (128 x 7), > 896 (64 x 15)
SHAPES = [(128, 4, 2, 2), (128, 4, 1, 0), (64, 4, 3, 1), (256, 2, 2, 0), (128, 1, 1, 2), (64, 2, 4, 0),
          (64, 15, 1, 1), (96, 5, 1, 2), (96, 3, 2, 0), (128, 7, 1, 2)]


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("name", ["chain16_T10_d3_box", "grid5x5_T6_d2_box", "chain1_T2"])
def test_sweep_shapes_and_streaming(name, shape, torch):
    """Every launch shape (threads per group, groups per CTA, Phi-step wave)
    and residency level (0: N, Psi, Lambda, q all streamed from global memory)
    gives the same iterates as the oracle."""
    import paper_2103_14990_gb300 as pkg
    gt, ng, wave, res = shape
    p = SMALL[name]()
    o = O.Oracle(p)
    K = 23
    ref = O.admm(o.lay, o.blocks, p.x0, fixed_iters=K)
    s = gpu_solver([p], torch)
    s.set_option(pkg.OPT_SWEEP_SHAPE, gt * 10000 + ng * 100 + wave)
    s.set_option(pkg.OPT_RESIDENCY, res)
    info = s.info()
    assert info["group_threads"] == gt and info["groups_per_cta"] == ng and info["wave"] == wave
    if res == 0:
        assert info["resident_n_items"] == 0 and info["resident_state_items"] == 0
    rc, st, phi, psi, lam, u, xn = run_fixed(s, torch, p.x0, K)
    assert rel(psi, ref.Psi) <= REL
    assert rel(phi, ref.Phi) <= REL
    assert rel(u, o.control(ref)) <= REL or np.max(np.abs(u - o.control(ref))) < 1e-7
    # warm continuation from the state left behind (resident state written back)
    rc, st2, phi2, psi2, lam2, u2, xn2 = run_fixed(s, torch, p.x0, K, warm=pkg.WARM_PREVIOUS)
    ref2 = O.admm(o.lay, o.blocks, p.x0, Psi0=ref.Psi, Lam0=ref.Lam, fixed_iters=K)
    assert rel(psi2, ref2.Psi) <= REL
    # the compact iterate (resident or in global memory) on the same shape
    rc, st3, _, psi3, lam3, u3, _ = run_fixed(s, torch, p.x0, K, export=False)
    assert rel(psi3, ref.Psi) <= REL
    assert rel(lam3, ref.Lam) <= REL
    assert rel(u3, o.control(ref)) <= REL or np.max(np.abs(u3 - o.control(ref))) < 1e-7
    s.close()


def test_row_records_cached_and_derived_agree_bit_for_bit(torch):
    """A plan whose groups hold one wave of patches caches every row's record
    in shared memory once per launch; a plan whose groups cycle through several
    waves derives each record where it is used.  With the same threads per
    group both give the same iterates bit for bit (fixed iterations and
    closed-loop steps stopped by Conv), and the derived form matches the
    oracle."""
    import paper_2103_14990_gb300 as pkg
    p = I.make_instance(400, 6, 2, seed=31, boxes=True, x0_dist="uniform")
    runs = []
    for shape, grid in ((1280301, 134), (1280101, 152)):  # 402 groups for 400 patches / about 3 per group
        s = gpu_solver([p], torch)
        s.set_option(pkg.OPT_SWEEP_SHAPE, shape)
        assert s.info()["grid_ctas"] == grid
        fixed = run_fixed(s, torch, p.x0, 30, export=False)
        xa = torch.tensor(p.x0.astype(np.float32), device="cuda")
        xb = torch.zeros_like(xa)
        u = torch.zeros(p.n_sub, p.nu, device="cuda")
        loop = []
        for tau in range(3):
            rc, st = s.step(xa, u, xb, warm=pkg.WARM_COLD if tau == 0 else pkg.WARM_CONVERGED)
            loop.append((u.cpu().numpy().copy(), st[0]["iters"], st[0]["status"]))
            xa, xb = xb, xa
        runs.append((fixed, loop))
        s.close()
    (fa, la), (fb, lb) = runs
    for k in (3, 4, 5, 6):
        assert np.array_equal(fa[k], fb[k])
    for (ua, ia, sa), (ub, ib, sb) in zip(la, lb):
        assert ia == ib and sa == sb and np.array_equal(ua, ub)
    o = O.Oracle(p)
    ref = O.admm(o.lay, o.blocks, p.x0, fixed_iters=30)
    assert rel(fb[3], ref.Psi) <= REL
    assert max_patch_rel(o.lay, fb[3], ref.Psi) <= REL


def test_graph_replay_is_bit_identical(torch):
    """Steps replayed from captured CUDA graphs (one graph per buffer set of a
    ping-pong closed loop) equal directly launched steps bit for bit."""
    import paper_2103_14990_gb300 as pkg
    p = SMALL["chain16_T10_d3_box"]()
    outs = []
    for graph in (0, 1):
        s = gpu_solver([p], torch)
        s.set_option(pkg.OPT_GRAPH, graph)
        xa = torch.tensor(p.x0.astype(np.float32), device="cuda")
        xb = torch.zeros_like(xa)
        u = torch.zeros(p.n_sub, 1, device="cuda")
        us, its = [], []
        for tau in range(6):
            rc, st = s.step(xa, u, xb, warm=pkg.WARM_COLD if tau == 0 else pkg.WARM_PREVIOUS)
            us.append(u.cpu().numpy().copy())
            its.append(st[0]["iters"])
            xa, xb = xb, xa
        outs.append((np.array(us), its))
        s.close()
    assert outs[0][1] == outs[1][1]
    assert np.array_equal(outs[0][0], outs[1][0])


def test_sweep_shape_rejects_sixteen_groups(torch):
    """Groups synchronise on named barriers 1..15: a 16th group is refused."""
    import paper_2103_14990_gb300 as pkg
    s = gpu_solver([SMALL["grid5x5_T6_d2_box"]()], torch)
    with pytest.raises(pkg.DlmpcError):
        s.set_option(pkg.OPT_SWEEP_SHAPE, 64 * 10000 + 16 * 100 + 1)
    s.close()


def test_autotune_keeps_state_and_parity(torch):
    import paper_2103_14990_gb300 as pkg
    p = SMALL["grid5x5_T6_d2_box"]()
    s = gpu_solver([p], torch)
    x = torch.tensor(p.x0.astype(np.float32), device="cuda")
    _, psi0, lam0 = s.get_state()
    psi0, lam0 = psi0.clone(), lam0.clone()
    table = s.autotune(x, iters=5)
    assert len(table) >= 2 and all(e["ms"] > 0 for e in table)
    _, psi1, lam1 = s.get_state()
    assert torch.equal(psi0, psi1) and torch.equal(lam0, lam1)
    best = table[0]
    info = s.info()
    assert (info["group_threads"], info["wave"]) == (best["group_threads"], best["wave"])
    o = O.Oracle(p)
    ref = O.admm(o.lay, o.blocks, p.x0, fixed_iters=30)
    rc, st, phi, psi, lam, u, xn = run_fixed(s, torch, p.x0, 30)
    assert rel(psi, ref.Psi) <= REL and rel(phi, ref.Phi) <= REL
    s.close()


@pytest.mark.parametrize("variant", [0, 1, 2])
@pytest.mark.parametrize("name", ["chain16_T10_d3_box", "grid5x5_T6_d2_box"])
def test_paper_variants_match_oracle(name, variant, torch):
    """The paper's naive and combined GPU mappings and the persistent sweep
    compute the same iterates as the oracle."""
    p = SMALL[name]()
    o = O.Oracle(p)
    K = 12
    ref = O.admm(o.lay, o.blocks, p.x0, fixed_iters=K)
    s = gpu_solver([p], torch)
    x = torch.tensor(p.x0.astype(np.float32), device="cuda")
    ms = s.run_variant(variant, x, K)
    assert ms > 0
    phi, psi, lam = [a.cpu().numpy() for a in s.get_state(phi=True)]
    assert rel(psi, ref.Psi) <= REL and rel(lam, ref.Lam) <= REL and rel(phi, ref.Phi) <= REL
    s.close()


# --------------------------------------------------------------------------
# Full cost blocks Q_i, R_i (slot box-QP Phi-step)
# --------------------------------------------------------------------------

BLOCK = {
    "chain16_T10_d3_box_blk": lambda: I.with_block_costs(SMALL["chain16_T10_d3_box"](), seed=31),
    "grid5x5_T6_d2_box_blk": lambda: I.with_block_costs(SMALL["grid5x5_T6_d2_box"](), seed=32),
    "chain10_blk": lambda: I.with_block_costs(I.chain10(), seed=33),
}


@pytest.mark.parametrize("name", list(BLOCK))
@pytest.mark.parametrize("K", [1, 7, 60])
def test_block_cost_fixed_iterations_parity(name, K, torch):
    """Phi, Psi, Lambda and u after K iterations against the oracle's block
    Phi-step (full form with Phi export, and the compact iterate)."""
    p = BLOCK[name]()
    o = O.Oracle(p)
    ref = O.admm(o.lay, o.blocks, p.x0, fixed_iters=K)
    s = gpu_solver([p], torch)
    rc, st, phi, psi, lam, u, xn = run_fixed(s, torch, p.x0, K)
    assert rel(psi, ref.Psi) <= REL and rel(phi, ref.Phi) <= REL
    assert rel(lam, ref.Lam) <= REL or np.linalg.norm(ref.Lam) < 1e-6
    u_ref = o.control(ref)
    assert rel(u, u_ref) <= REL or np.max(np.abs(u - u_ref)) < 1e-7
    rc, st, _, psi2, lam2, u2, _ = run_fixed(s, torch, p.x0, K, export=False)
    assert rel(psi2, ref.Psi) <= REL
    assert rel(u2, u_ref) <= REL or np.max(np.abs(u2 - u_ref)) < 1e-7
    s.close()


def test_block_cost_register_tiers_and_row_records_agree(torch):
    """The block Phi-step in every register tier (CTAs of 1024, 896 and 512
    threads at 128 threads per group), and with row records cached (one wave
    per group) or derived (several waves per group), gives the same iterates
    bit for bit; the 512-thread plan also against the oracle."""
    import paper_2103_14990_gb300 as pkg
    p = BLOCK["chain16_T10_d3_box_blk"]()
    res = []
    for shape in (1280801, 1280701, 1280401):
        s = gpu_solver([p], torch)
        s.set_option(pkg.OPT_SWEEP_SHAPE, shape)
        assert s.info()["threads_per_cta"] == (shape // 10000) * ((shape // 100) % 100)
        res.append(run_fixed(s, torch, p.x0, 25, export=False))
        s.close()
    for r in res[1:]:
        assert np.array_equal(r[3], res[0][3]) and np.array_equal(r[4], res[0][4]) and np.array_equal(r[5], res[0][5])
    o = O.Oracle(p)
    ref = O.admm(o.lay, o.blocks, p.x0, fixed_iters=25)
    assert rel(res[2][3], ref.Psi) <= REL
    q = I.with_block_costs(I.make_instance(400, 6, 2, seed=35, boxes=True, x0_dist="uniform"), seed=36)
    out = []
    for shape, grid in ((1280301, 134), (1280101, 152)):  # one patch per group / about 3 per group
        s = gpu_solver([q], torch)
        s.set_option(pkg.OPT_SWEEP_SHAPE, shape)
        assert s.info()["grid_ctas"] == grid
        out.append(run_fixed(s, torch, q.x0, 20, export=False))
        s.close()
    assert np.array_equal(out[0][3], out[1][3]) and np.array_equal(out[0][5], out[1][5])


def test_block_cost_stopped_closed_loop(torch):
    p = BLOCK["chain10_blk"]()
    stopped_closed_loop(p, torch, "previous", p.mpc_steps)


@pytest.mark.parametrize("name", ["chain16_T10_d3_box", "grid5x5_T6_d2_box"])
def test_block_phi_on_diagonal_costs_matches_row_phi(name, torch):
    """The slot box-QP with diagonal blocks is the per-row closed form."""
    import paper_2103_14990_gb300 as pkg
    p = SMALL[name]()
    s = gpu_solver([p], torch)
    _, _, phi_a, psi_a, _, u_a, _ = run_fixed(s, torch, p.x0, 30)
    s.set_option(pkg.OPT_BLOCK_PHI, 1)
    _, _, phi_b, psi_b, _, u_b, _ = run_fixed(s, torch, p.x0, 30)
    assert rel(phi_b, phi_a) <= 1e-5 and rel(psi_b, psi_a) <= 1e-5
    assert rel(u_b, u_a) <= 1e-5 or np.max(np.abs(u_a - u_b)) < 1e-7
    s.close()


def test_failed_replan_keeps_the_previous_plan(torch):
    """A residency or shape the kernel cannot take is refused and the
    previous plan stays in force (the step still matches the oracle)."""
    import paper_2103_14990_gb300 as pkg
    p = SMALL["chain16_T10_d3_box"]()
    s = gpu_solver([p], torch)
    s.set_option(pkg.OPT_SWEEP_SHAPE, 1280402)
    before = s.info()
    with pytest.raises(pkg.DlmpcError):
        s.set_option(pkg.OPT_SWEEP_SHAPE, 961102)          # 11 x 96 threads exceed a CTA
    with pytest.raises(pkg.DlmpcError):
        s.set_option(pkg.OPT_SWEEP_SHAPE, 1280409)         # wave 9 is out of range
    after = s.info()
    for key in ("group_threads", "groups_per_cta", "wave", "resident_n_items", "smem_bytes"):
        assert after[key] == before[key], key
    o = O.Oracle(p)
    ref = O.admm(o.lay, o.blocks, p.x0, fixed_iters=9)
    _, _, phi, psi, _, _, _ = run_fixed(s, torch, p.x0, 9)
    assert rel(psi, ref.Psi) <= REL
    s.close()


def test_block_cost_validation(torch):
    import paper_2103_14990_gb300 as pkg
    p = BLOCK["chain10_blk"]()
    bad = p.Q_blk.copy()
    bad[3] = np.array([[1.0, 2.0], [2.0, 1.0]])          # indefinite
    import dataclasses
    with pytest.raises(pkg.DlmpcError):
        pkg.Solver([dataclasses.replace(p, Q_blk=bad)])
    s = gpu_solver([p], torch)
    x = torch.tensor(p.x0.astype(np.float32), device="cuda")
    with pytest.raises(pkg.DlmpcError):
        s.run_variant(0, x, 2)                            # the paper variants take diagonal weights
    s.close()


def test_steps_are_deterministic(torch):
    """No atomics sit in value paths: the same step twice gives the same bits
    (state, u, x(t+1), statistics)."""
    import paper_2103_14990_gb300 as pkg
    p = SMALL["grid5x5_T6_d2_box"]()
    outs = []
    for _ in range(2):
        s = gpu_solver([p], torch)
        x = torch.tensor(p.x0.astype(np.float32), device="cuda")
        u = torch.zeros(p.n_sub, 1, device="cuda")
        xn = torch.zeros_like(x)
        rc, st = s.step(x, u, xn, warm=pkg.WARM_COLD)
        rc2, st2 = s.step(xn.clone(), u, xn, warm=pkg.WARM_PREVIOUS)
        _, psi, lam = s.get_state()
        outs.append((psi.cpu().numpy(), lam.cpu().numpy(), u.cpu().numpy(), xn.cpu().numpy(), st, st2))
        s.close()
    a, b = outs
    for i in range(4):
        assert np.array_equal(a[i], b[i])
    assert a[4] == b[4] and a[5] == b[5]


def test_operator_checkpoint_round_trip(torch):
    """Operators exported after precompute and imported into a fresh context
    (no factorisation) give the same iterates bit for bit; a blob of another
    problem structure is refused."""
    import paper_2103_14990_gb300 as pkg
    p = SMALL["grid5x5_T6_d2_box"]()
    a = gpu_solver([p], torch)
    blob = a.export_operators()
    b = pkg.Solver([p], precompute=False)
    b.import_operators(blob)
    ra = run_fixed(a, torch, p.x0, 25)
    rb = run_fixed(b, torch, p.x0, 25)
    for x, y in zip(ra[2:], rb[2:]):
        assert np.array_equal(x, y)
    other = pkg.Solver([SMALL["chain16_T10_d3_box"]()], precompute=False)
    with pytest.raises(pkg.DlmpcError):
        other.import_operators(blob)
    with pytest.raises(pkg.DlmpcError):
        b2 = pkg.Solver([p], precompute=False)
        b2.import_operators(blob[:-8])
    for s in (a, b, other):
        s.close()


# --------------------------------------------------------------------------
# Coupled per-slot constraints (Gx x_t <= gx, Gu u_t <= gu beside the boxes):
# the explicit slot-QP solution, rebuilt from x(tau) in the sweep's prologue
# at every MPC step, against the oracle's active-set enumeration
# --------------------------------------------------------------------------

def binding_rows(p, z):
    """Coupled rows active (to 1e-6) at the slot values z of the oracle."""
    nb = 0
    for i in range(p.n_sub):
        for t in range(1, p.T):
            rr = [O.global_row(p, i, t * p.nx + a) for a in range(p.nx)]
            if p.Gx is not None:
                nb += int(np.sum(p.Gx[i] @ z[rr] - p.gx[i] > -1e-6))
        for t in range(p.T - 1):
            rr = [O.global_row(p, i, p.nx * p.T + t * p.nu + b) for b in range(p.nu)]
            if p.Gu is not None:
                nb += int(np.sum(p.Gu[i] @ z[rr] - p.gu[i] > -1e-6))
    return nb


COUPLED = {
    "chain16_T10_d3_box_cpl": lambda: I.with_coupled_constraints(
        I.make_instance(16, 10, 3, seed=1, boxes=True, x0_dist="uniform"), seed=51, n_cx=2, n_cu=1),
    "grid5x5_T6_d2_box_cpl": lambda: I.with_coupled_constraints(
        I.make_instance(25, 6, 2, graph="grid", seed=2, boxes=True), seed=52, n_cx=2),
    "chain10_nobox_cpl4": lambda: I.with_coupled_constraints(I.chain10(), seed=53, n_cx=4, n_cu=2,
                                                             g_range=(0.2, 0.6)),
}


@pytest.mark.parametrize("name", list(COUPLED))
@pytest.mark.parametrize("K", [1, 7, 60])
def test_coupled_fixed_iterations_parity(name, K, torch):
    """Phi, Psi, Lambda and u after K iterations (full form with Phi export,
    and the compact iterate) against the oracle's slot QP with coupled rows."""
    p = COUPLED[name]()
    o = O.Oracle(p)
    ref = O.admm(o.lay, o.blocks, p.x0, fixed_iters=K)
    if K == 60:
        assert binding_rows(p, ref.z) > 0, "the coupled rows must bind"
    s = gpu_solver([p], torch)
    rc, st, phi, psi, lam, u, xn = run_fixed(s, torch, p.x0, K)
    assert rel(psi, ref.Psi) <= REL and rel(phi, ref.Phi) <= REL
    assert rel(lam, ref.Lam) <= REL or np.linalg.norm(ref.Lam) < 1e-6
    u_ref = o.control(ref)
    assert rel(u, u_ref) <= REL or np.max(np.abs(u - u_ref)) < 1e-7
    rc, st, _, psi2, lam2, u2, _ = run_fixed(s, torch, p.x0, K, export=False)
    assert rel(psi2, ref.Psi) <= REL
    assert rel(lam2, ref.Lam) <= REL or np.linalg.norm(ref.Lam) < 1e-6
    assert rel(u2, u_ref) <= REL or np.max(np.abs(u2 - u_ref)) < 1e-7
    s.close()


def test_coupled_stopped_closed_loop(torch):
    """Conv on, warm start from the previous step, on a feasible instance
    whose coupled rows bind at the first step (stopped-run parity at 1e-4)."""
    base = I.make_instance(4, 4, 1, seed=3, boxes=True, x0_dist="uniform", x_bound=1.0, u_bound=0.5, mpc_steps=4)
    base.x0 = 0.3 * base.x0
    p = dataclasses.replace(I.with_coupled_constraints(base, seed=8, n_cx=2, g_range=(0.1, 0.3)), max_iter=3000)
    o = O.Oracle(p)
    first = O.admm(o.lay, o.blocks, p.x0)
    assert binding_rows(p, first.z) > 0
    stopped_closed_loop(p, torch, "previous", p.mpc_steps, iter_tol=0.05)


def test_slack_coupled_rows_match_the_box_slot_qp(torch):
    """Coupled rows that can never bind (g = 100) leave the slot QP a box-QP:
    the explicit solution gives what the box solver gives."""
    base = I.with_block_costs(I.make_instance(16, 10, 3, seed=1, boxes=True, x0_dist="uniform"), seed=31)
    cpl = I.with_coupled_constraints(base, seed=54, n_cx=2, n_cu=1)
    cpl = dataclasses.replace(cpl, gx=np.full_like(cpl.gx, 100.0), gu=np.full_like(cpl.gu, 100.0))
    outs = []
    for p in (base, cpl):
        s = gpu_solver([p], torch)
        outs.append(run_fixed(s, torch, p.x0, 40))
        s.close()
    (_, _, phi_a, psi_a, _, u_a, _), (_, _, phi_b, psi_b, _, u_b, _) = outs
    assert rel(phi_b, phi_a) <= 1e-5 and rel(psi_b, psi_a) <= 1e-5
    assert rel(u_b, u_a) <= 1e-5 or np.max(np.abs(u_a - u_b)) < 1e-7


def test_coupled_in_a_batch_with_a_plain_instance(torch):
    """Two instances in one context, one with coupled rows and one without:
    each against its own oracle run (the plain one through the slot QP of its
    boxes)."""
    a = COUPLED["grid5x5_T6_d2_box_cpl"]()
    b = I.make_instance(16, 10, 3, seed=1, boxes=True, x0_dist="uniform")
    K = 25
    s = gpu_solver([a, b], torch)
    x0 = np.concatenate([a.x0, b.x0])
    rc, st, phi, psi, lam, u, xn = run_fixed(s, torch, x0, K)
    off_s = 0
    off_u = 0
    for p in (a, b):
        o = O.Oracle(p)
        ref = O.admm(o.lay, o.blocks, p.x0, fixed_iters=K)
        n = ref.Psi.size
        assert rel(psi[off_s:off_s + n], ref.Psi) <= REL
        u_ref = o.control(ref)
        uu = u[off_u:off_u + p.n_sub]
        assert rel(uu, u_ref) <= REL or np.max(np.abs(uu - u_ref)) < 1e-7
        off_s += n
        off_u += p.n_sub
    s.close()


# --------------------------------------------------------------------------
# Simulated lost messages (the distributed setting of Sec. V): the receiver
# keeps the last row sums it got; SplitMix64 draws on both sides
# --------------------------------------------------------------------------

STALE_CASES = {
    "chain16_T10_d3_box": lambda: SMALL["chain16_T10_d3_box"](),
    "grid5x5_T6_d2_box": lambda: SMALL["grid5x5_T6_d2_box"](),
    "chain16_T10_d3_box_blk": lambda: BLOCK["chain16_T10_d3_box_blk"](),
}


@pytest.mark.parametrize("name", list(STALE_CASES))
@pytest.mark.parametrize("K,prob", [(1, 0.3), (7, 0.3), (40, 0.3), (25, 1.0)])
def test_stale_messages_fixed_iterations_parity(name, K, prob, torch):
    import paper_2103_14990_gb300 as pkg
    p = STALE_CASES[name]()
    o = O.Oracle(p)
    ref = O.admm(o.lay, o.blocks, p.x0, fixed_iters=K, stale=(prob, 1234))
    s = gpu_solver([p], torch)
    s.set_option(pkg.OPT_STALE_PROB, prob)
    s.set_option(pkg.OPT_STALE_SEED, 1234)
    rc, st, phi, psi, lam, u, xn = run_fixed(s, torch, p.x0, K)
    assert rel(psi, ref.Psi) <= REL and rel(phi, ref.Phi) <= REL
    assert rel(lam, ref.Lam) <= REL or np.linalg.norm(ref.Lam) < 1e-6
    u_ref = o.control(ref)
    assert rel(u, u_ref) <= REL or np.max(np.abs(u - u_ref)) < 1e-7
    rc, st, _, psi2, lam2, u2, _ = run_fixed(s, torch, p.x0, K, export=False)
    assert rel(psi2, ref.Psi) <= REL
    assert rel(lam2, ref.Lam) <= REL or np.linalg.norm(ref.Lam) < 1e-6
    s.close()


def test_stale_messages_change_the_iterates_and_p0_is_exact(torch):
    import paper_2103_14990_gb300 as pkg
    p = SMALL["grid5x5_T6_d2_box"]()
    s = gpu_solver([p], torch)
    _, _, phi_a, psi_a, _, u_a, _ = run_fixed(s, torch, p.x0, 20)
    s.set_option(pkg.OPT_STALE_SEED, 5)
    s.set_option(pkg.OPT_STALE_PROB, 0.0)
    _, _, phi_b, psi_b, _, u_b, _ = run_fixed(s, torch, p.x0, 20)
    assert np.array_equal(psi_a, psi_b) and np.array_equal(phi_a, phi_b)
    s.set_option(pkg.OPT_STALE_PROB, 0.25)
    _, _, phi_c, psi_c, _, u_c, _ = run_fixed(s, torch, p.x0, 20)
    assert np.max(np.abs(psi_c - psi_a)) > 1e-5
    # graph replay with losses: the same bits as the direct launch
    s.set_option(pkg.OPT_GRAPH, 1)
    _, _, phi_d, psi_d, _, u_d, _ = run_fixed(s, torch, p.x0, 20)
    _, _, phi_e, psi_e, _, u_e, _ = run_fixed(s, torch, p.x0, 20)
    s.set_option(pkg.OPT_GRAPH, 0)
    assert np.array_equal(psi_c, psi_d) and np.array_equal(psi_d, psi_e)
    with pytest.raises(pkg.DlmpcError):
        s.set_option(pkg.OPT_STALE_PROB, 1.5)
    with pytest.raises(pkg.DlmpcError):
        s.run_variant(0, torch.tensor(p.x0.astype(np.float32), device="cuda"), 2)
    s.close()


# --------------------------------------------------------------------------
# Other state and input sizes: the kernels' NX = 1..4 instantiations and the
# slot solvers of sizes 1..4
# --------------------------------------------------------------------------

GENERAL = {
    "nx1_nu1_chain": lambda: I.make_general(8, 5, 1, 1, 1, seed=3),
    "nx3_nu2_chain": lambda: I.make_general(8, 5, 2, 3, 2, seed=3),
    "nx4_nu1_grid": lambda: I.make_general(9, 4, 1, 4, 1, graph="grid", seed=3),
    "nx4_nu4_chain": lambda: I.make_general(6, 4, 1, 4, 4, seed=3),
    "nx3_nu1_grid": lambda: I.make_general(12, 5, 2, 3, 1, graph="grid", seed=3),
}


@pytest.mark.parametrize("name", list(GENERAL))
@pytest.mark.parametrize("K", [1, 7, 40])
def test_general_shapes_fixed_iterations_parity(name, K, torch):
    p = GENERAL[name]()
    o = O.Oracle(p)
    ref = O.admm(o.lay, o.blocks, p.x0, fixed_iters=K)
    s = gpu_solver([p], torch)
    rc, st, phi, psi, lam, u, xn = run_fixed(s, torch, p.x0, K)
    assert rel(psi, ref.Psi) <= REL and rel(phi, ref.Phi) <= REL
    assert rel(lam, ref.Lam) <= REL or np.linalg.norm(ref.Lam) < 1e-6
    u_ref = o.control(ref)
    assert rel(u, u_ref) <= REL or np.max(np.abs(u - u_ref)) < 1e-7
    rc, st, _, psi2, lam2, u2, _ = run_fixed(s, torch, p.x0, K, export=False)
    assert rel(psi2, ref.Psi) <= REL
    assert rel(u2, u_ref) <= REL or np.max(np.abs(u2 - u_ref)) < 1e-7
    s.close()


@pytest.mark.parametrize("name", ["nx3_nu2_chain", "nx4_nu4_chain", "nx1_nu1_chain"])
def test_general_shapes_block_and_coupled_parity(name, torch):
    """Full cost blocks (slot box-QP of sizes nx and nu) and coupled rows
    (explicit solution of sizes nx and nu) on other state and input sizes."""
    base = GENERAL[name]()
    for p in (I.with_block_costs(base, seed=41),
              I.with_coupled_constraints(base, seed=42, n_cx=2, n_cu=1, g_range=(0.2, 0.6))):
        o = O.Oracle(p)
        ref = O.admm(o.lay, o.blocks, p.x0, fixed_iters=30)
        s = gpu_solver([p], torch)
        rc, st, phi, psi, lam, u, xn = run_fixed(s, torch, p.x0, 30)
        assert rel(psi, ref.Psi) <= REL and rel(phi, ref.Phi) <= REL
        u_ref = o.control(ref)
        assert rel(u, u_ref) <= REL or np.max(np.abs(u - u_ref)) < 1e-7
        rc, st, _, psi2, _, u2, _ = run_fixed(s, torch, p.x0, 30, export=False)
        assert rel(psi2, ref.Psi) <= REL
        s.close()


def test_general_shape_stopped_closed_loop(torch):
    """Conv on, warm start from the previous step, u(tau) and x(tau+1) on a
    plant with three states and two inputs (stopped-run parity at 1e-4)."""
    p = GENERAL["nx3_nu2_chain"]()
    stopped_closed_loop(p, torch, "previous", 5, check_next=True)


def test_solve_batch_equals_step_on_concatenated_buffers(torch):
    """dlmpc_solve_batch (one device buffer per instance) gives the bits of
    dlmpc_step on the concatenated buffers, state and statistics included."""
    import paper_2103_14990_gb300 as pkg
    probs = [SMALL["chain16_T10_d3_box"](), SMALL["grid5x5_T6_d2_box"](), I.chain10()]
    outs = []
    for mode in ("step", "batch"):
        s = gpu_solver(probs, torch)
        s.set_option(pkg.OPT_FIXED_ITERS, 17)
        xs = [torch.tensor(p.x0.astype(np.float32), device="cuda") for p in probs]
        us = [torch.zeros(p.n_sub, p.nu, device="cuda") for p in probs]
        xns = [torch.zeros(p.n_sub, p.nx, device="cuda") for p in probs]
        if mode == "step":
            x = torch.cat(xs)
            u = torch.zeros(x.shape[0], probs[0].nu, device="cuda")
            xn = torch.zeros_like(x)
            rc, st = s.step(x, u, xn, warm=pkg.WARM_COLD)
            u_list, xn_list = list(torch.split(u, [p.n_sub for p in probs])), \
                list(torch.split(xn, [p.n_sub for p in probs]))
        else:
            rc, st = s.solve_batch(xs, us, xns, warm=pkg.WARM_COLD)
            u_list, xn_list = us, xns
        _, psi, lam = s.get_state()
        torch.cuda.synchronize()
        outs.append((psi.cpu().numpy(), lam.cpu().numpy(), [a.cpu().numpy() for a in u_list],
                     [a.cpu().numpy() for a in xn_list], [(d["iters"], d["status"]) for d in st]))
        s.close()
    a, b = outs
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
    assert all(np.array_equal(x, y) for x, y in zip(a[2], b[2]))
    assert all(np.array_equal(x, y) for x, y in zip(a[3], b[3]))
    assert a[4] == b[4]


def test_set_state_continues_from_the_given_iterate(torch):
    """Psi and Lambda written with dlmpc_set_state are the start of the next
    warm step: K more iterations equal the oracle's K iterations from that
    state."""
    import paper_2103_14990_gb300 as pkg
    p = SMALL["grid5x5_T6_d2_box"]()
    o = O.Oracle(p)
    mid = O.admm(o.lay, o.blocks, p.x0, fixed_iters=9)
    ref = O.admm(o.lay, o.blocks, p.x0, Psi0=mid.Psi, Lam0=mid.Lam, fixed_iters=11)
    s = gpu_solver([p], torch)
    s.set_state(torch.tensor(mid.Psi.astype(np.float32), device="cuda"),
                torch.tensor(mid.Lam.astype(np.float32), device="cuda"))
    rc, st, phi, psi, lam, u, xn = run_fixed(s, torch, p.x0, 11, warm=pkg.WARM_PREVIOUS)
    assert rel(psi, ref.Psi) <= REL and rel(phi, ref.Phi) <= REL and rel(lam, ref.Lam) <= REL
    s.close()


def test_contexts_with_different_plans_interleave(torch):
    """The sweep kernel's dynamic shared-memory limit is a property of the
    kernel function, shared by all contexts: a context planned after another
    (with a smaller arena) must not break the first one's launches."""
    import paper_2103_14990_gb300 as pkg
    big = I.chain1024()
    s1 = gpu_solver([big], torch)
    a = run_fixed(s1, torch, big.x0, 5, export=False)
    small = I.chain10()
    s2 = gpu_solver([small], torch)
    assert s2.info()["smem_bytes"] < s1.info()["smem_bytes"]
    run_fixed(s2, torch, small.x0, 5, export=False)
    b = run_fixed(s1, torch, big.x0, 5, export=False)
    assert np.array_equal(a[3], b[3]) and np.array_equal(a[5], b[5])
    run_fixed(s2, torch, small.x0, 5, export=False)
    s1.close()
    s2.close()


def test_warm_start_from_converged_steps_only(torch):
    """DLMPC_WARM_CONVERGED decides per instance on the device: a closed loop
    run with it gives the bits of the same loop whose host picks, step by
    step, the previous state after a converged step and zeros after a step
    stopped at max_iter; and the loop matches the oracle's "converged"
    policy (stopped-run parity at 1e-4, capped steps included)."""
    import paper_2103_14990_gb300 as pkg
    p = I.chain10()
    cap = 252                                     # steps 0-2 stop at the cap, the others converge
    o = O.Oracle(p)
    _, _, its, stats = o.run_mpc(p.mpc_steps, warm="converged", max_iter=cap)
    assert 0 < sum(s.status == O.STATUS_CONVERGED for s in stats) < p.mpc_steps
    runs = []
    for mode in ("device", "host"):
        s = gpu_solver([p], torch)
        s.set_option(pkg.OPT_MAX_ITER, cap)
        x = torch.tensor(p.x0.astype(np.float32), device="cuda")
        xn = torch.zeros_like(x)
        u = torch.zeros(p.n_sub, 1, device="cuda")
        rec, last = [], None
        for tau in range(p.mpc_steps):
            if mode == "device":
                warm = pkg.WARM_CONVERGED
            else:
                warm = pkg.WARM_PREVIOUS if (last is not None and last == 0) else pkg.WARM_COLD
            rc, st = s.step(x, u, xn, warm=warm)
            last = st[0]["status"]
            rec.append((st[0]["iters"], last, u.cpu().numpy().copy()))
            x, xn = xn, x
        runs.append(rec)
        s.close()
    for a, b in zip(*runs):
        assert a[0] == b[0] and a[1] == b[1] and np.array_equal(a[2], b[2])
    out = stopped_closed_loop(p, torch, "converged", p.mpc_steps, max_iter=cap)
    assert out["iters_oracle"] == list(its)
