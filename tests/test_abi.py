"""C-ABI checks that need no GPU: the library loads, exports every entry point
declared in include/maze.h, the ctypes structures match the C layout, and
configuration errors are reported before any device work."""
import ctypes
import os
import re
import subprocess
import tempfile

import numpy as np
import pytest

from paper_2505_20418_gb300 import maze as M
from paper_2505_20418_gb300 import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "maze.h")


@pytest.fixture(scope="module")
def lib():
    if not os.path.exists(M.LIB_PATH):
        import __graft_entry__ as g
        g.build()
    return M.load()


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(maze_[a-z_]+)\s*\(", src)))


def test_header_declares_binding_exports():
    assert declared_functions() == sorted(M.EXPORTS)


def test_library_exports_every_declared_symbol(lib):
    out = subprocess.run(["nm", "-D", "--defined-only", M.LIB_PATH], capture_output=True, text=True).stdout
    syms = set(re.findall(r"\sT\s(maze_\w+)", out))
    for name in declared_functions():
        assert name in syms, name
        assert hasattr(lib, name)


def test_struct_layout_matches_c():
    """Compile a probe against the header with gcc and compare sizes/offsets."""
    fields_cfg = [f for f, _ in M.MazeConfig._fields_]
    fields_st = [f for f, _ in M.MazeStats._fields_]
    fields_b = [f for f, _ in M.MazeBatchConfig._fields_]
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "maze.h"', "int main(void){"]
    lines.append('printf("%zu %zu %zu\\n", sizeof(maze_config), sizeof(maze_stats), sizeof(maze_batch_config));')
    for f in fields_cfg:
        lines.append(f'printf("%zu\\n", offsetof(maze_config, {f}));')
    for f in fields_st:
        lines.append(f'printf("%zu\\n", offsetof(maze_stats, {f}));')
    for f in fields_b:
        lines.append(f'printf("%zu\\n", offsetof(maze_batch_config, {f}));')
    lines.append("return 0;}")
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "probe.c")
        exe = os.path.join(d, "probe")
        open(c, "w").write("\n".join(lines))
        subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), c, "-o", exe], check=True)
        vals = subprocess.run([exe], capture_output=True, text=True, check=True).stdout.split()
    vals = [int(v) for v in vals]
    assert vals[0] == ctypes.sizeof(M.MazeConfig)
    assert vals[1] == ctypes.sizeof(M.MazeStats)
    assert vals[2] == ctypes.sizeof(M.MazeBatchConfig)
    offs = vals[3:]
    py = ([getattr(M.MazeConfig, f).offset for f in fields_cfg] + [getattr(M.MazeStats, f).offset for f in fields_st]
          + [getattr(M.MazeBatchConfig, f).offset for f in fields_b])
    assert offs == py


def _cfg(**over):
    w = synth.workload("nacl64")
    pos, vel, types = synth.make_state(w)
    kw = dict(r_cut=w.rc, dt=w.dt, tol=w.tol)
    types = over.pop("types", types)
    N = over.pop("N", w.N)
    kw.update(over)
    return M.make_config(pos, vel, types, w.L, N, synth.tosi_fumi_nacl(), **kw)


@pytest.mark.parametrize("over, msg", [
    (dict(order=3), "order_P"),
    (dict(r_cut=7.0), "r_cut"),
    (dict(dt=0.0), "dt"),
    (dict(tol=-1.0), "tol"),
    (dict(max_iter=0), "max_iter"),
    (dict(solver=7), "solver"),
    (dict(solver=1, mg_pre=0), "mg_pre"),
    (dict(precision=9), "precision"),
    (dict(scheme=3), "scheme"),
    (dict(force_estimator=2), "force_estimator"),
    (dict(langevin_gamma=-1.0), "langevin_gamma"),
    (dict(langevin_T=float("nan")), "langevin_T"),
    (dict(solver=1, N=36), "coarsest edge"),    # 36 -> 18 -> 9: a 9^3 coarsest level
    (dict(solver=1, N=250), "coarsest edge"),   # 250 -> 125
])
def test_invalid_config_rejected(lib, over, msg):
    cfg, keep = _cfg(**over)
    h = ctypes.c_void_p()
    st = lib.maze_create(ctypes.byref(cfg), ctypes.byref(h))
    assert st == M.MAZE_ERR_INVALID and h.value is None
    assert msg in M.maze_last_error()


def test_non_neutral_and_bad_grid_rejected(lib):
    w = synth.workload("nacl64")
    pos, vel, types = synth.make_state(w)
    bad = types.copy()
    bad[0] = 1 - bad[0]
    cfg, keep = M.make_config(pos, vel, bad, w.L, w.N, synth.tosi_fumi_nacl(), r_cut=w.rc)
    h = ctypes.c_void_p()
    assert lib.maze_create(ctypes.byref(cfg), ctypes.byref(h)) == M.MAZE_ERR_INVALID
    assert "neutral" in M.maze_last_error()
    for N in (7, 6, 2048):
        cfg, keep = M.make_config(pos, vel, types, w.L, N, synth.tosi_fumi_nacl(), r_cut=w.rc)
        assert lib.maze_create(ctypes.byref(cfg), ctypes.byref(h)) == M.MAZE_ERR_INVALID
    cfg, keep = M.make_config(pos[:1], vel[:1], types[:1], w.L, w.N, synth.tosi_fumi_nacl(), r_cut=w.rc)
    assert lib.maze_create(ctypes.byref(cfg), ctypes.byref(h)) == M.MAZE_ERR_INVALID
    assert lib.maze_create(None, ctypes.byref(h)) == M.MAZE_ERR_INVALID
    pos2 = pos.copy()
    pos2[3, 1] = np.nan
    cfg, keep = M.make_config(pos2, vel, types, w.L, w.N, synth.tosi_fumi_nacl(), r_cut=w.rc)
    assert lib.maze_create(ctypes.byref(cfg), ctypes.byref(h)) == M.MAZE_ERR_INVALID


def test_null_context_calls_are_errors(lib):
    assert lib.maze_batch_step(None, 1) == M.MAZE_ERR_INVALID
    assert lib.maze_batch_remove(None, 0) == M.MAZE_ERR_INVALID
    lib.maze_batch_destroy(None)  # NULL-safe
    assert lib.maze_spread(None) == M.MAZE_ERR_INVALID
    assert lib.maze_step(None, 1) == M.MAZE_ERR_INVALID
    assert lib.maze_gather(None) == M.MAZE_ERR_INVALID
    assert lib.maze_step_io(None, None, None, 1, None, None, None) == M.MAZE_ERR_INVALID
    lib.maze_destroy(None)  # NULL-safe
    assert M.maze_version().startswith("maze-gb300")
