"""Host copies of a standalone context (maze_set / maze_get / maze_get_stats
and the one-call exchange maze_step_io).

maze_set uploads positions and velocities from a pinned stage without
synchronising, maze_step queues the copies of the positions and velocities
the caller read after the previous step together with its record read, and
maze_get_stats serves a record that no call has changed since it was read.
These tests interleave the calls in the orders a caller may use and check
every value against a second context driven with step_async and explicit
reads, which takes none of those shortcuts' state."""
import numpy as np
import pytest

from paper_2505_20418_gb300 import maze as M
from paper_2505_20418_gb300 import synth

pytestmark = pytest.mark.gpu


def make(w):
    pos, vel, types = synth.make_state(w)
    return M.MazeSim(pos, vel, types, w.L, w.N, synth.tosi_fumi_nacl(), r_cut=w.rc, dt=w.dt, tol=w.tol,
                     order=w.order, solver=M.MAZE_SOLVER_MG, precision=M.MAZE_MIXED)


def test_interleaved_gets_sets_and_steps_match_a_plain_context():
    w = synth.workload("nacl1000")
    a, b = make(w), make(w)
    rng = np.random.default_rng(3)
    for k in range(6):
        if k == 3:
            # a caller's edit between steps: new positions and velocities
            x = a.get(M.MAZE_POS) + rng.normal(scale=1e-3, size=(w.n_ions, 3))
            v = a.get(M.MAZE_VEL) * 0.999
            for s in (a, b):
                s.set(M.MAZE_POS, x)
                s.set(M.MAZE_VEL, v)
        assert M.maze_step(a.h, 1) == M.MAZE_OK
        b.step_async(1)
        sb = b.stats()
        sa = a.stats()
        assert sa["step"] == sb["step"] and sa["ke"] == sb["ke"]
        # reads in varying orders, the forces through the velocities' stage
        order = [M.MAZE_POS, M.MAZE_VEL, M.MAZE_FORCE, M.MAZE_VEL] if k % 2 else \
            [M.MAZE_FORCE, M.MAZE_VEL, M.MAZE_POS, M.MAZE_POS]
        for what in order:
            assert np.array_equal(a.get(what), b.get(what)), (k, what)
    a.close()
    b.close()


def test_set_then_get_without_a_step_returns_the_new_values():
    w = synth.workload("nacl1000")
    a = make(w)
    assert M.maze_step(a.h, 1) == M.MAZE_OK
    a.get(M.MAZE_POS)
    a.get(M.MAZE_VEL)
    assert M.maze_step(a.h, 1) == M.MAZE_OK     # queues both copies
    v = a.get(M.MAZE_VEL) + 0.25
    a.set(M.MAZE_VEL, v)
    assert np.array_equal(a.get(M.MAZE_VEL), v)
    x = np.mod(a.get(M.MAZE_POS) + 0.5, w.L)
    a.set(M.MAZE_POS, x)
    assert np.allclose(a.get(M.MAZE_POS), x, atol=0, rtol=0)
    a.close()


def test_step_io_equals_set_step_get_stats():
    """maze_step_io against maze_set, maze_step, maze_get and maze_get_stats
    on a twin context, bit for bit, with and without inputs and outputs."""
    w = synth.workload("nacl1000")
    a, b = make(w), make(w)
    n = w.n_ions
    rng = np.random.default_rng(11)
    x, v = a.get(M.MAZE_POS), a.get(M.MAZE_VEL)
    cases = [(True, True, 1, True, True), (False, False, 2, True, False), (True, False, 1, False, True),
             (False, True, 0, True, True), (False, False, 1, False, False), (True, True, 3, True, True)]
    for pin, vin, nsteps, pout, vout in cases:
        x = np.mod(x + rng.normal(scale=1e-3, size=(n, 3)), w.L)
        v = v * 0.9995
        st = M.MazeStats()
        po = np.full((n, 3), np.nan) if pout else None
        vo = np.full((n, 3), np.nan) if vout else None
        a.step_io(nsteps, pos=x if pin else None, vel=v if vin else None, out_pos=po, out_vel=vo, stats=st)
        if pin:
            b.set(M.MAZE_POS, x)
        if vin:
            b.set(M.MAZE_VEL, v)
        assert M.maze_step(b.h, nsteps) == M.MAZE_OK
        sb = b.stats()
        sa = st.as_dict()
        assert sa == sb, (pin, vin, nsteps)
        if pout:
            assert np.array_equal(po, b.get(M.MAZE_POS))
        if vout:
            assert np.array_equal(vo, b.get(M.MAZE_VEL))
        # and the context's own reads agree afterwards
        assert np.array_equal(a.get(M.MAZE_FORCE), b.get(M.MAZE_FORCE))
        x, v = b.get(M.MAZE_POS), b.get(M.MAZE_VEL)
    a.close()
    b.close()


def test_step_io_rejects_non_finite_input_before_running():
    w = synth.workload("nacl1000")
    a = make(w)
    a.step(1)
    before = a.stats()["step"]
    x = a.get(M.MAZE_POS)
    v = a.get(M.MAZE_VEL)
    v[7, 2] = np.inf
    po = np.zeros_like(x)
    st = M.maze_step_io(a.h, w.n_ions, x + 0.1, v, 1, po, None)
    assert st == M.MAZE_ERR_INVALID
    assert a.stats()["step"] == before
    assert np.array_equal(a.get(M.MAZE_POS), x)     # the valid positions were not uploaded either
    assert not po.any()
    with pytest.raises(ValueError):
        a.step_io(1, out_pos=np.zeros((w.n_ions, 2)))
    a.close()


def test_step_io_large_box_host_threads():
    """64000 ions: the host transposes and checks run on several threads;
    the results equal the single-call sequence bit for bit."""
    w = synth.workload("nacl64000")
    a, b = make(w), make(w)
    n = w.n_ions
    x = np.mod(a.get(M.MAZE_POS) + 1e-3, w.L)
    v = a.get(M.MAZE_VEL) * 0.999
    po, vo = np.empty((n, 3)), np.empty((n, 3))
    st = M.MazeStats()
    a.step_io(1, pos=x, vel=v, out_pos=po, out_vel=vo, stats=st)
    b.set(M.MAZE_POS, x)
    b.set(M.MAZE_VEL, v)
    assert M.maze_step(b.h, 1) == M.MAZE_OK
    assert st.as_dict() == b.stats()
    assert np.array_equal(po, b.get(M.MAZE_POS))
    assert np.array_equal(vo, b.get(M.MAZE_VEL))
    v[n - 1, 0] = np.nan     # in the last thread's range
    assert M.maze_step_io(a.h, n, None, v, 1, None, None) == M.MAZE_ERR_INVALID
    a.close()
    b.close()


def test_step_io_exchange_graph_over_rotations_and_mixed_calls():
    """Full one-step exchanges (the single-graph form) for seven steps in a
    row, every rotation of the potentials twice, then interleaved with
    plain steps, sets and gets: bit for bit the six-call sequence."""
    w = synth.workload("nacl1000")
    a, b = make(w), make(w)
    n = w.n_ions
    x, v = a.get(M.MAZE_POS), a.get(M.MAZE_VEL)
    st = M.MazeStats()

    def twin(x, v, nsteps=1):
        b.set(M.MAZE_POS, x)
        b.set(M.MAZE_VEL, v)
        assert M.maze_step(b.h, nsteps) == M.MAZE_OK
        return b.get(M.MAZE_POS), b.get(M.MAZE_VEL), b.stats()

    for k in range(7):
        po, vo = np.empty((n, 3)), np.empty((n, 3))
        a.step_io(1, pos=x, vel=v, out_pos=po, out_vel=vo, stats=st)
        bx, bv, bs = twin(x, v)
        assert np.array_equal(po, bx) and np.array_equal(vo, bv) and st.as_dict() == bs, k
        x, v = po, vo * 0.9999
    # interleaved with the other calls
    a.step(2)
    b.step(2)
    assert np.array_equal(a.get(M.MAZE_POS), b.get(M.MAZE_POS))
    x, v = a.get(M.MAZE_POS), a.get(M.MAZE_VEL)
    a.set(M.MAZE_VEL, v * 1.0001)
    b.set(M.MAZE_VEL, v * 1.0001)
    po, vo = np.empty((n, 3)), np.empty((n, 3))
    a.step_io(1, pos=x, vel=v, out_pos=po, out_vel=vo, stats=st)
    bx, bv, bs = twin(x, v)
    assert np.array_equal(po, bx) and np.array_equal(vo, bv) and st.as_dict() == bs
    assert np.array_equal(a.get(M.MAZE_FORCE), b.get(M.MAZE_FORCE))
    assert np.array_equal(a.get(M.MAZE_VEL), vo)
    a.close()
    b.close()


def test_exchange_buffers_equal_step_io():
    """MazeSim.exchange on pinned buffers against step_io on plain arrays."""
    w = synth.workload("nacl1000")
    a, b = make(w), make(w)
    io = a.exchange_buffers()
    x, v = b.get(M.MAZE_POS), b.get(M.MAZE_VEL)
    st = M.MazeStats()
    for _ in range(4):
        a.exchange(io)
        b.step_io(1, pos=x, vel=v, out_pos=x, out_vel=v, stats=st)
        assert np.array_equal(io.pos, x) and np.array_equal(io.vel, v)
        assert io.stats.as_dict() == st.as_dict()
    a.close()
    b.close()


def test_full_exchange_rejects_non_finite_input_before_running():
    """The one-graph exchange checks its inputs in its staging pass: a NaN
    returns MAZE_ERR_INVALID with nothing uploaded or run."""
    w = synth.workload("nacl1000")
    a = make(w)
    io = a.exchange_buffers()
    a.exchange(io)                          # the exchange graph is built and used
    before = a.stats()["step"]
    x0, v0 = io.pos.copy(), io.vel.copy()
    io.vel[w.n_ions - 1, 1] = np.nan
    with pytest.raises(M.MazeError):
        a.exchange(io)
    assert a.stats()["step"] == before
    assert np.array_equal(a.get(M.MAZE_POS), x0) and np.array_equal(a.get(M.MAZE_VEL), v0)
    io.vel[w.n_ions - 1, 1] = v0[w.n_ions - 1, 1]
    a.exchange(io)                          # and the context carries on
    assert a.stats()["step"] == before + 1
    a.close()


@pytest.mark.parametrize("wl,precision", [("nacl64", M.MAZE_MIXED), ("nacl1000", M.MAZE_FP64),
                                          ("nacl64000", M.MAZE_MIXED)])
def test_exchange_other_step_forms(wl, precision):
    """The exchange graph over the other step forms: a box without cells
    (S1-S6 in one cluster launch), the FP64 path (separate launches, the
    cooperative solve) and a box solved on the whole grid; bit for bit the
    separate calls."""
    w = synth.workload(wl)
    pos, vel, types = synth.make_state(w)
    kw = dict(r_cut=w.rc, dt=w.dt, tol=w.tol, order=w.order, solver=M.MAZE_SOLVER_MG, precision=precision)
    a = M.MazeSim(pos, vel, types, w.L, w.N, synth.tosi_fumi_nacl(), **kw)
    b = M.MazeSim(pos, vel, types, w.L, w.N, synth.tosi_fumi_nacl(), **kw)
    io = a.exchange_buffers()
    for _ in range(4):
        x, v = io.pos.copy(), io.vel.copy()
        a.exchange(io)
        b.set(M.MAZE_POS, x)
        b.set(M.MAZE_VEL, v)
        assert M.maze_step(b.h, 1) == M.MAZE_OK
        assert np.array_equal(io.pos, b.get(M.MAZE_POS)) and np.array_equal(io.vel, b.get(M.MAZE_VEL))
        assert io.stats.as_dict() == b.stats()
    a.close()
    b.close()
