"""C ABI checks that need no GPU: every symbol declared in include/dlmpc.h is
exported by the built library, and the host-side setup (locality structure,
argument validation, infeasible locality) behaves as documented."""
import ctypes
import os
import re

import numpy as np
import pytest

import paper_2103_14990_gb300 as pkg
from oracle import dlmpc_oracle as O
from paper_2103_14990_gb300 import instances as I

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "dlmpc.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(dlmpc_[a-z_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def clib():
    if not os.path.exists(pkg.LIB_PATH):
        from paper_2103_14990_gb300 import build
        build.build()
    return pkg.load_library()


def test_every_declared_symbol_is_exported(clib):
    names = declared_symbols()
    assert len(names) >= 13
    assert sorted(pkg.EXPORTED) == names
    for n in names:
        assert hasattr(clib, n), n


class _Marshal:
    def __init__(self):
        self._keep = []


def _setup(clib, probs):
    arr = (pkg.Problem_C * len(probs))()
    m = _Marshal()
    for k, p in enumerate(probs):
        arr[k] = pkg.Solver._marshal(m, p)
    ctx = ctypes.c_void_p()
    rc = clib.dlmpc_setup(arr, len(probs), None, ctypes.byref(ctx))
    return rc, ctx, m


@pytest.mark.parametrize("prob", [I.chain10(), I.make_instance(30, 5, 2, graph="grid", seed=1),
                                  I.make_instance(20, 6, 3, seed=2)])
def test_patches_match_oracle_bfs(clib, prob):
    rc, ctx, _ = _setup(clib, [prob])
    assert rc == 0
    try:
        buf = np.zeros(64, np.int32)
        for j in range(prob.n_sub):
            n = clib.dlmpc_get_patch(ctx, j, buf.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), 64)
            assert list(buf[:n]) == O.patch_members(prob, j)
    finally:
        clib.dlmpc_destroy(ctx)


def test_batch_patches_use_global_indices(clib):
    probs = [I.chain10(), I.make_instance(12, 4, 1, graph="grid", seed=3)]
    rc, ctx, _ = _setup(clib, probs)
    assert rc == 0
    buf = np.zeros(64, np.int32)
    n = clib.dlmpc_get_patch(ctx, 10 + 5, buf.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), 64)
    assert list(buf[:n]) == [10 + m for m in O.patch_members(probs[1], 5)]
    clib.dlmpc_destroy(ctx)


def test_setup_rejects_bad_arguments(clib):
    p = I.chain10()
    p.rho = -1.0
    rc, ctx, _ = _setup(clib, [p])
    assert rc == pkg.DLMPC_ERR_ARG and b"rho" in clib.dlmpc_last_error(None)
    p = I.chain10()
    p.T = 1
    rc, ctx, _ = _setup(clib, [p])
    assert rc == pkg.DLMPC_ERR_ARG
    p = I.make_instance(6, 4, 1, boxes=True)
    p.u_lo = np.full((6, 1), 0.5)       # 0 outside [u_lo, u_hi]
    rc, ctx, _ = _setup(clib, [p])
    assert rc == pkg.DLMPC_ERR_ARG
    q = I.chain10()
    q2 = I.make_instance(5, 4, 1)
    q2.nx = 3
    rc, ctx, _ = _setup(clib, [q, q2])
    assert rc == pkg.DLMPC_ERR_ARG


def test_zero_locality_is_infeasible_on_both_sides(clib):
    """d = 0 on the coupled chain: a neighbour's slot-1 state would need A_ij e_c = 0."""
    p = I.make_instance(5, 4, 0, seed=0, boxes=False)
    rc, ctx, _ = _setup(clib, [p])
    assert rc == pkg.DLMPC_ERR_INFEASIBLE_LOCALITY
    assert O.column_block(p, 2).feas > 1e-3


def test_missing_library_fails_loudly(tmp_path):
    with pytest.raises(RuntimeError):
        pkg._LIB_saved = pkg._LIB
        try:
            pkg._LIB = None
            pkg.load_library(str(tmp_path / "nope.so"))
        finally:
            pkg._LIB = pkg._LIB_saved


def _with_coupled(n_cx=2, n_cu=1):
    return I.with_coupled_constraints(I.make_instance(8, 4, 1, seed=4, boxes=True), seed=9, n_cx=n_cx, n_cu=n_cu)


def test_setup_validates_coupled_rows(clib):
    rc, ctx, _ = _setup(clib, [_with_coupled()])
    assert rc == 0
    clib.dlmpc_destroy(ctx)
    rc, ctx, _ = _setup(clib, [_with_coupled(n_cx=pkg.DLMPC_MAX_COUPLED, n_cu=pkg.DLMPC_MAX_COUPLED)])
    assert rc == 0
    clib.dlmpc_destroy(ctx)
    p = _with_coupled(n_cx=pkg.DLMPC_MAX_COUPLED + 1)
    rc, ctx, _ = _setup(clib, [p])
    assert rc == pkg.DLMPC_ERR_ARG
    p = _with_coupled()
    p.Gx[3, 1] = 0.0                                   # zero normal
    rc, ctx, _ = _setup(clib, [p])
    assert rc == pkg.DLMPC_ERR_ARG and b"normal" in clib.dlmpc_last_error(None)
    p = _with_coupled()
    p.gu[2, 0] = -0.1                                  # 0 would violate the row
    rc, ctx, _ = _setup(clib, [p])
    assert rc == pkg.DLMPC_ERR_ARG
    p = _with_coupled()
    p.gx[1, 0] = np.nan
    rc, ctx, _ = _setup(clib, [p])
    assert rc == pkg.DLMPC_ERR_ARG


def _header_defines():
    import re
    out = {}
    for line in open(os.path.join(ROOT, "include", "dlmpc.h")):
        m = re.match(r"#define (DLMPC_\w+)\s+\(?(-?\d+)\)?", line)
        if m:
            out[m.group(1)] = int(m.group(2))
    return out


def test_binding_constants_match_header():
    d = _header_defines()
    assert len(d) >= 20
    checked = 0
    for name, v in d.items():
        short = name[len("DLMPC_"):]
        for cand in (name, short):
            if hasattr(pkg, cand):
                assert getattr(pkg, cand) == v, name
                checked += 1
                break
    assert checked >= 20


def test_struct_layout_matches_header(tmp_path):
    """sizeof and field offsets of the ABI structs as the C compiler lays them
    out, against the binding's ctypes structures."""
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    fields = [f for f, _ in pkg.Problem_C._fields_]
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "dlmpc.h"', "int main(void) {",
             '  printf("%zu\\n", sizeof(dlmpc_problem));']
    lines += ['  printf("%%zu\\n", offsetof(dlmpc_problem, %s));' % f for f in fields]
    lines += ['  printf("%zu\\n", sizeof(dlmpc_stats));', "  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    vals = [int(v) for v in subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split()]
    assert vals[0] == ctypes.sizeof(pkg.Problem_C)
    for f, off in zip(fields, vals[1:1 + len(fields)]):
        assert getattr(pkg.Problem_C, f).offset == off, f
    assert vals[-1] == ctypes.sizeof(pkg.Stats_C)


def test_update_plant_needs_a_precomputed_context(clib):
    """The plant update replaces operators: before dlmpc_precompute there are
    none, and the call is refused without touching the device."""
    p = I.make_instance(8, 4, 1, seed=4, boxes=True)
    rc, ctx, _ = _setup(clib, [p])
    assert rc == 0
    sub = np.array([3], np.int32)
    ad = np.ascontiguousarray(p.A_diag[3:4])
    ao = np.ascontiguousarray(p.A_off[p.adj_ptr[3]:p.adj_ptr[4]])
    bb = np.ascontiguousarray(p.B[3:4])
    dp = ctypes.POINTER(ctypes.c_double)
    rc = clib.dlmpc_update_plant(ctx, 1, sub.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                                 ad.ctypes.data_as(dp), ao.ctypes.data_as(dp), bb.ctypes.data_as(dp))
    assert rc == pkg.DLMPC_ERR_ARG and b"precompute" in clib.dlmpc_last_error(ctx)
    clib.dlmpc_destroy(ctx)
