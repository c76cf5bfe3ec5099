"""Batched simulations (maze_batch_*): many boxes advanced by one persistent
kernel launch per step.

A box in a batch runs the same device bodies as the single-box mixed path and
every reduction on the way is exact or independent of how the work is split,
so the batch must reproduce, bit for bit, the positions, velocities, forces
and potential of each box advanced alone (energies to rounding). The single
box path itself is held to the FP64 oracle in test_gpu_mixed.py; one box is
also checked against the oracle directly here.
"""
import numpy as np
import pytest

import oracle as O
from paper_2505_20418_gb300 import maze as M
from paper_2505_20418_gb300 import synth
from tests.test_gpu_parity import force_err

pytestmark = pytest.mark.gpu

MIXED_BAR = 1e-5
TF = synth.tosi_fumi_nacl()
GiB = 1 << 30


def box(n_ions, seed, **kw):
    if n_ions == 64:
        w = synth.workload("nacl64")
        w.seed = seed
    else:
        w = synth.replica(n_ions, seed)
    pos, vel, types = synth.make_state(w)
    args = dict(r_cut=w.rc, dt=w.dt, tol=w.tol, order=w.order)
    args.update(kw)
    return (pos, vel, types, w.L, w.N), args


def alone(spec, args, steps):
    (pos, vel, types, L, N) = spec
    sim = M.MazeSim(pos, vel, types, L, N, TF, solver=M.MAZE_SOLVER_MG, precision=M.MAZE_MIXED, **args)
    st = M.maze_step(sim.h, steps)
    return sim, st


def add(b, spec, args):
    (pos, vel, types, L, N) = spec
    return b.add(pos, vel, types, L, N, TF, **args)


SPECS = [(216, 11, {}), (512, 12, {}), (1000, 13, {}), (64, 14, {}), (216, 15, {"order": 2}),
         (1728, 16, {})]
FIELDS = (M.MAZE_POS, M.MAZE_VEL, M.MAZE_FORCE, M.MAZE_PHI, M.MAZE_PHI_PREV, M.MAZE_Y)


def same(b, i, sim):
    for what in FIELDS:
        a, c = b.get(i, what), sim.get(what)
        assert np.array_equal(a, c), (i, what, float(np.abs(a - c).max()))
    s1, s2 = b.stats(i), sim.stats()
    assert s1["step"] == s2["step"] and s1["total_iters"] == s2["total_iters"]
    # energies are sums over ions grouped differently by the two launch forms;
    # both round the exact fixed-point sums at about 2^-37 of the largest
    # block partial
    for k in ("ke", "v_tf", "v_disc", "v_work"):
        assert abs(s1[k] - s2[k]) <= 1e-10 * max(1.0, abs(s2[k])), (k, s1[k], s2[k])


@pytest.mark.parametrize("cta", [1, 4, 16])
def test_batch_equals_each_box_alone(cta):
    steps = 12
    b = M.MazeBatch(2 * GiB, 16, cluster_ctas=cta)
    specs = [box(n, s, **kw) for n, s, kw in SPECS]
    ids = [add(b, sp, a) for sp, a in specs]
    b.step(steps)
    assert b.info()["count"] == len(SPECS)
    for i, (sp, a) in zip(ids, specs):
        sim, st = alone(sp, a, steps)
        assert st == M.MAZE_OK
        same(b, i, sim)
        sim.close()
    b.close()


def test_batch_box_against_oracle():
    spec, args = box(512, 21)
    pos, vel, types, L, N = spec
    w = synth.replica(512, 21)
    b = M.MazeBatch(GiB, 4)
    i = add(b, spec, args)
    p = O.Params(L=L, N=N, dt=w.dt, tol=w.tol, rc=w.rc, P=w.order, solver="mg")
    st = O.init(pos, vel, types, p, TF)
    for _ in range(3):
        st = O.step(st, p, TF)
    b.step(3)
    assert force_err(b.get(i, M.MAZE_FORCE), st.F) < MIXED_BAR
    s = b.stats(i)
    assert s["status"] == 0 and s["resid"] < p.tol and s["step"] == 3
    b.close()


def test_add_remove_reuse_and_admission():
    spec_a, args_a = box(216, 31)
    spec_b, args_b = box(1000, 32)
    spec_c, args_c = box(512, 33)
    pos, vel, types, L, N = spec_b
    need = M.MazeBatch.box_bytes(pos, vel, types, L, N, TF, **args_b)
    assert need > 0
    # an arena with room for two 1000-ion boxes only
    b = M.MazeBatch(2 * need + (1 << 20), 8)
    i0 = add(b, spec_b, args_b)
    i1 = add(b, spec_b, args_b)
    assert b.try_add(*spec_b, TF, **args_b) is None          # admission refused: no room
    b.step(3)
    b.remove(i0)
    i2 = add(b, spec_a, args_a)                               # reuses the freed slot
    assert i2 == i0
    i3 = b.try_add(*spec_c, TF, **args_c)
    b.step(4)
    # the box that stayed advanced 7 steps, the new ones 4, each as if alone
    sim, _ = alone(spec_b, args_b, 7)
    same(b, i1, sim)
    sim.close()
    sim, _ = alone(spec_a, args_a, 4)
    same(b, i2, sim)
    sim.close()
    if i3 is not None:
        sim, _ = alone(spec_c, args_c, 4)
        same(b, i3, sim)
        sim.close()
    b.close()


def test_slots_full():
    spec, args = box(216, 41)
    b = M.MazeBatch(GiB, 2)
    add(b, spec, args)
    add(b, spec, args)
    with pytest.raises(M.MazeError) as e:
        add(b, spec, args)
    assert e.value.status == M.MAZE_ERR_OOM
    b.close()


def test_failing_box_does_not_stop_the_others():
    good, ga = box(512, 51)
    bad, ba = box(216, 52, max_iter=1)
    b = M.MazeBatch(GiB, 4)
    ig = add(b, good, ga)
    ib = add(b, bad, ba)
    st = b.step_status(5)
    assert st == M.MAZE_ERR_NOT_CONVERGED
    assert f"simulation {ib}" in M.maze_last_error()
    sim, st1 = alone(good, ga, 5)
    assert st1 == M.MAZE_OK
    same(b, ig, sim)
    sim.close()
    sim, st2 = alone(bad, ba, 5)
    assert st2 == M.MAZE_ERR_NOT_CONVERGED
    same(b, ib, sim)
    assert b.stats(ib)["status"] == M.MAZE_ERR_NOT_CONVERGED and b.stats(ib)["step"] == 1
    sim.close()
    b.close()


def test_tune_keeps_state():
    specs = [box(n, s) for n, s in ((216, 61), (1000, 62), (512, 63))]
    b = M.MazeBatch(GiB, 4)
    ids = [add(b, sp, a) for sp, a in specs]
    b.step(2)
    before = [b.get(i, M.MAZE_POS) for i in ids]
    cta, ms = b.tune(2)
    assert cta in (1, 2, 4, 8, 16) and ms > 0
    assert b.info()["cluster_ctas"] == cta
    for i, x in zip(ids, before):
        assert np.array_equal(b.get(i, M.MAZE_POS), x)
    b.step(3)
    for i, (sp, a) in zip(ids, specs):
        sim, _ = alone(sp, a, 5)
        same(b, i, sim)
        sim.close()
    b.close()


def test_batch_rejects_what_it_cannot_run():
    spec, args = box(216, 71)
    b = M.MazeBatch(GiB, 2)
    pos, vel, types, L, N = spec
    with pytest.raises(M.MazeError) as e:
        b.add(pos, vel, types, L, N, TF, precision=M.MAZE_FP64, **args)
    assert e.value.status == M.MAZE_ERR_INVALID
    b.close()


def test_autotune_per_size_class_keeps_results():
    """maze_batch_autotune: a row per grid size; the state is restored after
    its trials; a class that kept the configured V-cycle schedule advances bit
    for bit as its boxes alone (cluster size and tail change no result), a
    class given another schedule still meets the tolerance and the oracle's
    forces within the mixed-precision bar."""
    specs = [box(n, s) for n, s in ((216, 81), (216, 82), (512, 83), (512, 84), (1000, 85), (1000, 86))]
    b = M.MazeBatch(GiB, 8)
    ids = [add(b, sp, a) for sp, a in specs]
    b.step(2)
    before = [b.get(i, M.MAZE_POS) for i in ids]
    table = b.autotune(2)
    assert sorted(t["grid_N"] for t in table) == [16, 24, 32]
    for t in table:
        assert t["boxes"] == 2 and t["cluster_ctas"] in (1, 2, 4, 8, 16) and t["tail_n"] in (0, 8, 16)
        assert (t["mg_pre"], t["mg_post"]) in ((2, 2), (1, 2), (2, 1), (1, 1), (3, 3))
        assert 0 < t["ms_after"] <= t["ms_before"]
    for i, x in zip(ids, before):
        assert np.array_equal(b.get(i, M.MAZE_POS), x)
    b.step(3)
    by_n = {t["grid_N"]: t for t in table}
    for i, (sp, a) in zip(ids, specs):
        t = by_n[sp[4]]
        s = b.stats(i)
        assert s["status"] == 0 and s["step"] == 5 and s["resid"] < a["tol"]
        if (t["mg_pre"], t["mg_post"]) == (2, 2):
            sim, _ = alone(sp, a, 5)
            same(b, i, sim)
            sim.close()
        else:
            pos, vel, types, L, N = sp
            p = O.Params(L=L, N=N, dt=a["dt"], tol=a["tol"], rc=a["r_cut"], P=a["order"], solver="mg")
            st = O.init(pos, vel, types, p, TF)
            for _ in range(5):
                st = O.step(st, p, TF)
            assert force_err(b.get(i, M.MAZE_FORCE), st.F) < MIXED_BAR
    # the one-size tuner puts every box back on one cluster size and the
    # configured schedule
    cta, _ = b.tune(2)
    b.step(1)
    for i in ids:
        assert b.stats(i)["step"] == 6
    b.close()
