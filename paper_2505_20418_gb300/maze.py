"""Thin ctypes binding of libmaze (include/maze.h).

Argument marshalling only: every step of the MaZe path runs in the CUDA
kernels of libmaze.so. The module-level functions carry the C names; the
:class:`MazeSim` class wraps one context. Loading fails loudly when the
library has not been built (``python -m paper_2505_20418_gb300.build``).
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libmaze.so")

MAZE_OK, MAZE_ERR_INVALID, MAZE_ERR_OOM, MAZE_ERR_NOT_CONVERGED = 0, 1, 2, 3
MAZE_ERR_NONFINITE, MAZE_ERR_TIMEOUT, MAZE_ERR_CUDA = 4, 5, 6
MAZE_SOLVER_CG, MAZE_SOLVER_MG = 0, 1
MAZE_FP64, MAZE_MIXED, MAZE_FP64_FIXMG = 0, 1, 2
MAZE_SCHEME_MAZE, MAZE_SCHEME_MG_STATIC, MAZE_SCHEME_MG_TIMEPROP = 0, 1, 2
MAZE_FORCE_CD, MAZE_FORCE_GRADW = 0, 1
MAZE_POS, MAZE_VEL, MAZE_FORCE, MAZE_FORCE_EL = 0, 1, 2, 3
MAZE_PHI, MAZE_PHI_PREV, MAZE_Y, MAZE_CHARGE, MAZE_SIGMA = 4, 5, 6, 7, 8

# every entry point declared in include/maze.h
EXPORTS = ("maze_create", "maze_spread", "maze_solve", "maze_gather", "maze_step",
           "maze_step_async", "maze_get", "maze_set", "maze_get_stats", "maze_step_io", "maze_get_state",
           "maze_set_state", "maze_destroy", "maze_last_error", "maze_version",
           "maze_set_timing", "maze_get_timing", "maze_solve_shake_noalloc",
           "maze_batch_create", "maze_batch_box_bytes", "maze_batch_free_bytes", "maze_batch_add",
           "maze_batch_remove", "maze_batch_info", "maze_batch_step", "maze_batch_step_async",
           "maze_batch_get", "maze_batch_set", "maze_batch_get_stats", "maze_batch_get_all_stats",
           "maze_batch_tune",
           "maze_batch_destroy", "maze_wait_probe", "maze_batch_step_ready_async", "maze_batch_sync",
           "maze_batch_refresh", "maze_batch_autotune", "maze_convert_probe", "maze_exp_probe",
           "maze_df_probe")

_D = ctypes.c_double
_I = ctypes.c_int32


class MazeConfig(ctypes.Structure):
    _fields_ = [
        ("n_ions", _I), ("grid_N", _I), ("box_L", _D),
        ("pos", ctypes.POINTER(_D)), ("vel", ctypes.POINTER(_D)), ("type", ctypes.POINTER(_I)),
        ("charge", _D * 2), ("mass", _D * 2),
        ("tf_A", _D * 3), ("tf_B", _D), ("tf_s", _D * 3), ("tf_C", _D * 3), ("tf_D", _D * 3),
        ("r_cut", _D), ("dt", _D), ("tol", _D),
        ("max_iter", _I), ("solver", _I), ("mg_pre", _I), ("mg_post", _I),
        ("order_P", _I), ("precision", _I), ("scheme", _I), ("force_estimator", _I),
        ("langevin_gamma", _D), ("langevin_T", _D), ("seed", ctypes.c_uint64),
        ("cuda_stream", ctypes.c_void_p),
    ]


class MazeStats(ctypes.Structure):
    _fields_ = [
        ("step", ctypes.c_int64), ("iters", _I), ("status", _I), ("resid", _D),
        ("ke", _D), ("v_tf", _D), ("v_work", _D), ("v_disc", _D), ("e_tot", _D),
        ("momentum", _D * 3), ("total_iters", ctypes.c_int64),
    ]

    def as_dict(self):
        d = {k: getattr(self, k) for k, _ in self._fields_}
        d["momentum"] = list(self.momentum)
        return d


class MazeTuneEntry(ctypes.Structure):
    _fields_ = [("grid_N", _I), ("boxes", _I), ("cluster_ctas", _I), ("mg_pre", _I), ("mg_post", _I),
                ("tail_n", _I), ("ms_before", _D), ("ms_after", _D)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class MazeBatchConfig(ctypes.Structure):
    _fields_ = [("arena_bytes", ctypes.c_size_t), ("max_sims", _I), ("cluster_ctas", _I),
                ("cuda_stream", ctypes.c_void_p)]


class MazeError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"maze status {status}: {msg}")
        self.status = status


_lib = None


def load(path: str = LIB_PATH):
    """Load libmaze.so (cached). Raises if it is missing: there is no fallback."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"libmaze.so not built at {path}; run __graft_entry__.build()")
    lib = ctypes.CDLL(path)
    P = ctypes.c_void_p
    lib.maze_create.argtypes = [ctypes.POINTER(MazeConfig), ctypes.POINTER(P)]
    lib.maze_spread.argtypes = [P]
    lib.maze_solve.argtypes = [P, ctypes.POINTER(_I), ctypes.POINTER(_D)]
    lib.maze_gather.argtypes = [P]
    lib.maze_step.argtypes = [P, _I]
    lib.maze_step_async.argtypes = [P, _I]
    lib.maze_get.argtypes = [P, _I, ctypes.POINTER(_D)]
    lib.maze_set.argtypes = [P, _I, ctypes.POINTER(_D)]
    lib.maze_get_stats.argtypes = [P, ctypes.POINTER(MazeStats)]
    lib.maze_step_io.argtypes = [P, P, P, _I, P, P, ctypes.POINTER(MazeStats)]
    lib.maze_get_state.argtypes = [P, P, ctypes.POINTER(ctypes.c_size_t)]
    lib.maze_set_state.argtypes = [P, P, ctypes.c_size_t]
    lib.maze_set_timing.argtypes = [P, _I]
    lib.maze_get_timing.argtypes = [P, ctypes.POINTER(_D)]
    lib.maze_solve_shake_noalloc.argtypes = [_I, P, P, _D, _I, P, ctypes.POINTER(_I), ctypes.POINTER(_D)]
    lib.maze_destroy.argtypes = [P]
    lib.maze_destroy.restype = None
    SZ = ctypes.POINTER(ctypes.c_size_t)
    lib.maze_batch_create.argtypes = [ctypes.POINTER(MazeBatchConfig), ctypes.POINTER(P)]
    lib.maze_batch_box_bytes.argtypes = [ctypes.POINTER(MazeConfig), SZ]
    lib.maze_batch_free_bytes.argtypes = [P, SZ, SZ]
    lib.maze_batch_add.argtypes = [P, ctypes.POINTER(MazeConfig), ctypes.POINTER(_I)]
    lib.maze_batch_remove.argtypes = [P, _I]
    lib.maze_batch_info.argtypes = [P, ctypes.POINTER(_I), ctypes.POINTER(_I), ctypes.POINTER(_I)]
    lib.maze_batch_step.argtypes = [P, _I]
    lib.maze_batch_step_async.argtypes = [P, _I]
    lib.maze_batch_get.argtypes = [P, _I, _I, ctypes.POINTER(_D)]
    lib.maze_batch_set.argtypes = [P, _I, _I, ctypes.POINTER(_D)]
    lib.maze_batch_get_stats.argtypes = [P, _I, ctypes.POINTER(MazeStats)]
    lib.maze_batch_get_all_stats.argtypes = [P, ctypes.POINTER(MazeStats), _I]
    lib.maze_batch_tune.argtypes = [P, _I, ctypes.POINTER(_I), ctypes.POINTER(_D)]
    lib.maze_batch_destroy.argtypes = [P]
    lib.maze_batch_destroy.restype = None
    lib.maze_wait_probe.argtypes = [_I, P, ctypes.POINTER(_I)]
    lib.maze_convert_probe.argtypes = [P, _I, P, P, P, P, P, P, P, P]
    lib.maze_exp_probe.argtypes = [P, _I, P, P]
    lib.maze_df_probe.argtypes = [ctypes.POINTER(MazeConfig), _I, P, P, _I, P, P]
    lib.maze_batch_step_ready_async.argtypes = [P, _I]
    lib.maze_batch_sync.argtypes = [P]
    lib.maze_batch_refresh.argtypes = [P, ctypes.POINTER(_I), _I, ctypes.POINTER(_I)]
    lib.maze_batch_autotune.argtypes = [P, _I, ctypes.POINTER(MazeTuneEntry), _I, ctypes.POINTER(_I)]
    lib.maze_last_error.restype = ctypes.c_char_p
    lib.maze_version.restype = ctypes.c_char_p
    for name in EXPORTS:
        if name not in ("maze_destroy", "maze_last_error", "maze_version", "maze_batch_destroy"):
            getattr(lib, name).restype = ctypes.c_int
    _lib = lib
    return lib


def _check(status):
    if status != MAZE_OK:
        raise MazeError(status, load().maze_last_error().decode())


def _dptr(a):
    return a.ctypes.data_as(ctypes.POINTER(_D))


# ---- C-named functions -----------------------------------------------------

def maze_create(cfg: MazeConfig):
    h = ctypes.c_void_p()
    _check(load().maze_create(ctypes.byref(cfg), ctypes.byref(h)))
    return h


def maze_spread(h):
    _check(load().maze_spread(h))


def maze_solve(h):
    it, res = _I(), _D()
    st = load().maze_solve(h, ctypes.byref(it), ctypes.byref(res))
    return st, it.value, res.value


def maze_gather(h):
    _check(load().maze_gather(h))


def maze_step(h, nsteps: int):
    return load().maze_step(h, int(nsteps))


def maze_step_async(h, nsteps: int):
    _check(load().maze_step_async(h, int(nsteps)))


def maze_get(h, what: int, out: np.ndarray):
    _check(load().maze_get(h, what, _dptr(out)))
    return out


def maze_set(h, what: int, arr: np.ndarray):
    arr = np.ascontiguousarray(arr, dtype=np.float64)
    _check(load().maze_set(h, what, _dptr(arr)))


def maze_get_stats(h) -> MazeStats:
    s = MazeStats()
    _check(load().maze_get_stats(h, ctypes.byref(s)))
    return s


def _ion_ptr(a, n, writable):
    """Address of an [n][3] float64 C-contiguous array (None -> NULL)."""
    if a is None:
        return None
    if (type(a) is not np.ndarray or a.dtype != np.float64 or a.shape != (n, 3)
            or not a.flags.c_contiguous or (writable and not a.flags.writeable)):
        raise ValueError(f"expected a C-contiguous float64 array of shape ({n}, 3)")
    return a.ctypes.data


def maze_step_io(h, n: int, pos_in, vel_in, nsteps: int, pos_out, vel_out, stats=None):
    """maze_step_io: inputs, steps and outputs in one call (arrays [n][3] or
    None; stats a MazeStats or None). Returns the status, as maze_step."""
    return load().maze_step_io(h, _ion_ptr(pos_in, n, False), _ion_ptr(vel_in, n, False), int(nsteps),
                               _ion_ptr(pos_out, n, True), _ion_ptr(vel_out, n, True),
                               None if stats is None else ctypes.byref(stats))


def maze_get_state(h) -> bytes:
    n = ctypes.c_size_t(0)
    _check(load().maze_get_state(h, None, ctypes.byref(n)))
    buf = ctypes.create_string_buffer(n.value)
    _check(load().maze_get_state(h, buf, ctypes.byref(n)))
    return buf.raw


def maze_set_state(h, blob: bytes):
    buf = ctypes.create_string_buffer(blob, len(blob))
    _check(load().maze_set_state(h, buf, len(blob)))


def maze_set_timing(h, on: bool):
    _check(load().maze_set_timing(h, int(bool(on))))


def maze_get_timing(h):
    """Phase times (ms) of the last step: spread, cells, solve, forces."""
    out = np.zeros(4)
    _check(load().maze_get_timing(h, _dptr(out)))
    return out


def maze_solve_shake_noalloc(grid_N: int, sigma_ptr: int, y_ptr: int, tol: float, max_iter: int,
                             stream: int | None = None):
    """Allocation-free M y = sigma_p solve on caller-owned device memory
    (raw device pointers, e.g. ``tensor.data_ptr()``). Returns (status, iters, resid)."""
    it, res = _I(), _D()
    st = load().maze_solve_shake_noalloc(int(grid_N), ctypes.c_void_p(sigma_ptr), ctypes.c_void_p(y_ptr),
                                         float(tol), int(max_iter), ctypes.c_void_p(stream or 0),
                                         ctypes.byref(it), ctypes.byref(res))
    return st, it.value, res.value


def maze_wait_probe(which: int, stream: int | None = None):
    """Run one bounded device wait that cannot complete (0 grid barrier, 1 grid
    reduction of doubles, 2 of 64-bit integers). Returns (call status,
    status recorded by the kernel)."""
    out = _I()
    st = load().maze_wait_probe(int(which), ctypes.c_void_p(stream or 0), ctypes.byref(out))
    return st, out.value


def maze_convert_probe(x):
    """The integer-pipe conversions of the FP64 kernels beside the conversion
    instructions, for a float64 array x. Returns (status, dict of arrays:
    f_own, f_hw, d_own, d_hw, floor_own, floor_hw, fix_own, fix_hw)."""
    x = np.ascontiguousarray(x, dtype=np.float64)
    n = x.size
    out = {"f_own": np.zeros(n, np.float32), "f_hw": np.zeros(n, np.float32), "d_own": np.zeros(n),
           "d_hw": np.zeros(n), "floor_own": np.zeros(n, np.int64), "floor_hw": np.zeros(n, np.int64),
           "fix_own": np.zeros(n), "fix_hw": np.zeros(n)}
    ptr = lambda a: a.ctypes.data_as(ctypes.c_void_p)
    st = load().maze_convert_probe(ptr(x), int(n), *(ptr(out[k]) for k in ("f_own", "f_hw", "d_own", "d_hw",
                                                                            "floor_own", "floor_hw", "fix_own",
                                                                            "fix_hw")))
    return st, out


def maze_exp_probe(x):
    """The pair forces' table-driven exp beside CUDA's exp() for a float64
    array x. Returns (status, own, ref)."""
    x = np.ascontiguousarray(x, dtype=np.float64)
    own, ref = np.zeros(x.size), np.zeros(x.size)
    ptr = lambda a: a.ctypes.data_as(ctypes.c_void_p)
    st = load().maze_exp_probe(ptr(x), int(x.size), ptr(own), ptr(ref))
    return st, own, ref


def maze_df_probe(what, x, kind=None, tf=None, r_cut=9.0):
    """The double-float exponential (what 0) or Tosi-Fumi pair (what 1; FP64
    form: what 2) of the FP64 boxes' pair kernel on the float64 array x, each
    value split into (hi, lo) floats first; kind and the table tf (with
    r_cut) for the pair. Returns (status, out0, out1)."""
    x = np.ascontiguousarray(x, dtype=np.float64)
    n = x.size
    o0, o1 = np.zeros(n), np.zeros(n)
    ptr = lambda a: a.ctypes.data_as(ctypes.c_void_p)
    cfg = None
    k = np.zeros(n, np.int32) if kind is None else np.ascontiguousarray(kind, dtype=np.int32)
    if tf is not None:
        cfg = MazeConfig()
        cfg.tf_A[:] = list(tf.A)
        cfg.tf_B = tf.B
        cfg.tf_s[:] = list(tf.s)
        cfg.tf_C[:] = list(tf.C)
        cfg.tf_D[:] = list(tf.D)
        cfg.r_cut = float(r_cut)
    st = load().maze_df_probe(ctypes.byref(cfg) if cfg is not None else None, int(what), ptr(x), ptr(k), int(n),
                              ptr(o0), ptr(o1))
    return st, o0, o1


def maze_destroy(h):
    load().maze_destroy(h)


def maze_last_error() -> str:
    return load().maze_last_error().decode()


def maze_version() -> str:
    return load().maze_version().decode()


# ---- convenience wrapper ---------------------------------------------------

def make_config(pos, vel, types, L, N, tf, *, r_cut, dt=1.0, tol=1e-10, max_iter=10000,
                solver=MAZE_SOLVER_CG, order=4, precision=MAZE_FP64, charge=(1.0, -1.0),
                mass=(22.98977, 35.453), mg_pre=2, mg_post=2, stream=None, scheme=MAZE_SCHEME_MAZE,
                force_estimator=MAZE_FORCE_CD, langevin_gamma=0.0, langevin_T=0.0, seed=0):
    """Build a MazeConfig; the returned tuple keeps the host arrays alive."""
    pos = np.ascontiguousarray(pos, dtype=np.float64)
    vel = np.ascontiguousarray(vel, dtype=np.float64)
    types = np.ascontiguousarray(types, dtype=np.int32)
    c = MazeConfig()
    c.n_ions = pos.shape[0]
    c.grid_N = int(N)
    c.box_L = float(L)
    c.pos = _dptr(pos)
    c.vel = _dptr(vel)
    c.type = types.ctypes.data_as(ctypes.POINTER(_I))
    c.charge[:] = list(charge)
    c.mass[:] = list(mass)
    c.tf_A[:] = list(tf.A)
    c.tf_B = tf.B
    c.tf_s[:] = list(tf.s)
    c.tf_C[:] = list(tf.C)
    c.tf_D[:] = list(tf.D)
    c.r_cut = float(r_cut)
    c.dt = float(dt)
    c.tol = float(tol)
    c.max_iter = int(max_iter)
    c.solver = int(solver)
    c.mg_pre = int(mg_pre)
    c.mg_post = int(mg_post)
    c.order_P = int(order)
    c.precision = int(precision)
    c.scheme = int(scheme)
    c.force_estimator = int(force_estimator)
    c.langevin_gamma = float(langevin_gamma)
    c.langevin_T = float(langevin_T)
    c.seed = int(seed)
    c.cuda_stream = stream
    return c, (pos, vel, types)


class ExchangeBuffers:
    """Pinned host buffers for a host-driven loop of maze_step_io exchanges:
    positions and velocities ([n][3], read as the step's inputs and
    overwritten with its results) and the step record, with their addresses
    taken once (MazeSim.exchange)."""

    def __init__(self, n: int):
        import torch
        self._keep = [torch.empty((n, 3), dtype=torch.float64).pin_memory() for _ in range(2)]
        self.pos, self.vel = (t.numpy() for t in self._keep)
        self.stats = MazeStats()
        self._args = (self.pos.ctypes.data, self.vel.ctypes.data, ctypes.byref(self.stats))


class MazeSim:
    """One MaZe simulation context on the current CUDA device."""

    def __init__(self, pos, vel, types, L, N, tf, **kw):
        cfg, keep = make_config(pos, vel, types, L, N, tf, **kw)
        self.n = cfg.n_ions
        self.N = int(N)
        self.h = maze_create(cfg)
        del keep

    def close(self):
        if self.h:
            maze_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _ion(self):
        return np.empty((self.n, 3))

    def _grid(self):
        return np.empty((self.N, self.N, self.N))

    def get(self, what):
        out = self._ion() if what <= MAZE_FORCE_EL else self._grid()
        return maze_get(self.h, what, out)

    def set(self, what, arr):
        maze_set(self.h, what, arr)

    def step(self, nsteps=1):
        _check(maze_step(self.h, nsteps))

    def step_async(self, nsteps=1):
        maze_step_async(self.h, nsteps)

    def exchange_buffers(self) -> ExchangeBuffers:
        """Pinned exchange buffers holding the current positions and velocities."""
        io = ExchangeBuffers(self.n)
        maze_get(self.h, MAZE_POS, io.pos)
        maze_get(self.h, MAZE_VEL, io.vel)
        return io

    def exchange(self, io: ExchangeBuffers, nsteps: int = 1):
        """maze_step_io with io's positions and velocities in and out and its
        record filled: one call, one synchronisation."""
        p, v, st = io._args
        status = load().maze_step_io(self.h, p, v, nsteps, p, v, st)
        if status:
            _check(status)

    def step_io(self, nsteps=1, pos=None, vel=None, out_pos=None, out_vel=None, stats=None):
        """Upload pos / vel (if given), run nsteps steps, fill out_pos / out_vel
        / stats (if given): one call, one synchronisation."""
        _check(maze_step_io(self.h, self.n, pos, vel, nsteps, out_pos, out_vel, stats))

    def spread(self):
        maze_spread(self.h)

    def solve(self, check=True):
        st, it, res = maze_solve(self.h)
        if check:
            _check(st)
        return it, res

    def gather(self):
        maze_gather(self.h)

    def stats(self) -> dict:
        return maze_get_stats(self.h).as_dict()

    def set_timing(self, on=True):
        maze_set_timing(self.h, on)

    def timing(self):
        return maze_get_timing(self.h)

    def get_state(self) -> bytes:
        return maze_get_state(self.h)

    def set_state(self, blob: bytes):
        maze_set_state(self.h, blob)


# ---- batched simulations -----------------------------------------------------

def maze_batch_box_bytes(cfg: MazeConfig) -> int:
    n = ctypes.c_size_t()
    _check(load().maze_batch_box_bytes(ctypes.byref(cfg), ctypes.byref(n)))
    return n.value


class MazeBatch:
    """Many independent MaZe simulations advanced together (maze_batch_*).

    Every simulation runs mixed precision with the multigrid solver; ids are
    slot numbers. ``add`` takes the same arguments as :class:`MazeSim`.
    """

    def __init__(self, arena_bytes: int, max_sims: int, cluster_ctas: int = 0, stream=None):
        c = MazeBatchConfig()
        c.arena_bytes = int(arena_bytes)
        c.max_sims = int(max_sims)
        c.cluster_ctas = int(cluster_ctas)
        c.cuda_stream = stream
        self.h = ctypes.c_void_p()
        _check(load().maze_batch_create(ctypes.byref(c), ctypes.byref(self.h)))
        self.shape = {}
        self.max_sims = int(max_sims)

    def close(self):
        if self.h:
            load().maze_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @staticmethod
    def config(pos, vel, types, L, N, tf, **kw):
        kw.setdefault("solver", MAZE_SOLVER_MG)
        kw.setdefault("precision", MAZE_MIXED)
        return make_config(pos, vel, types, L, N, tf, **kw)

    @staticmethod
    def box_bytes(pos, vel, types, L, N, tf, **kw) -> int:
        """Arena bytes one simulation of this configuration takes."""
        cfg, keep = MazeBatch.config(pos, vel, types, L, N, tf, **kw)
        return maze_batch_box_bytes(cfg)

    def add(self, pos, vel, types, L, N, tf, **kw) -> int:
        """Admit one simulation (runs its step 0); raises MazeError with status
        MAZE_ERR_OOM when no slot or arena room is free."""
        cfg, keep = self.config(pos, vel, types, L, N, tf, **kw)
        i = _I()
        _check(load().maze_batch_add(self.h, ctypes.byref(cfg), ctypes.byref(i)))
        self.shape[i.value] = (cfg.n_ions, int(N))
        return i.value

    def try_add(self, pos, vel, types, L, N, tf, **kw):
        """As add, but returns None instead of raising when the batch is full."""
        try:
            return self.add(pos, vel, types, L, N, tf, **kw)
        except MazeError as e:
            if e.status == MAZE_ERR_OOM:
                return None
            raise

    def remove(self, i: int):
        _check(load().maze_batch_remove(self.h, int(i)))
        self.shape.pop(int(i), None)

    def free_bytes(self):
        a, b = ctypes.c_size_t(), ctypes.c_size_t()
        _check(load().maze_batch_free_bytes(self.h, ctypes.byref(a), ctypes.byref(b)))
        return a.value, b.value

    def info(self) -> dict:
        n, c, k = _I(), _I(), _I()
        _check(load().maze_batch_info(self.h, ctypes.byref(n), ctypes.byref(c), ctypes.byref(k)))
        return {"count": n.value, "cluster_ctas": c.value, "clusters": k.value}

    def step(self, nsteps: int = 1):
        _check(load().maze_batch_step(self.h, int(nsteps)))

    def step_status(self, nsteps: int = 1) -> int:
        return load().maze_batch_step(self.h, int(nsteps))

    def step_async(self, nsteps: int = 1):
        _check(load().maze_batch_step_async(self.h, int(nsteps)))

    def step_ready_async(self, nsteps: int = 1):
        """Queue steps of the simulations whose admission has finished."""
        _check(load().maze_batch_step_ready_async(self.h, int(nsteps)))

    def refresh(self) -> list:
        """Ids of the simulations whose admission finished since the last call
        (they now advance with step_ready_async)."""
        arr = (_I * self.max_sims)()
        n = _I()
        _check(load().maze_batch_refresh(self.h, arr, self.max_sims, ctypes.byref(n)))
        return [arr[k] for k in range(n.value)]

    def sync_status(self) -> int:
        """Wait for the queued steps; the first failing status among them."""
        return load().maze_batch_sync(self.h)

    def get(self, i: int, what: int) -> np.ndarray:
        n, N = self.shape[int(i)]
        out = np.empty((n, 3)) if what <= MAZE_FORCE_EL else np.empty((N, N, N))
        _check(load().maze_batch_get(self.h, int(i), int(what), _dptr(out)))
        return out

    def set(self, i: int, what: int, arr):
        arr = np.ascontiguousarray(arr, dtype=np.float64)
        _check(load().maze_batch_set(self.h, int(i), int(what), _dptr(arr)))

    def stats(self, i: int) -> dict:
        s = MazeStats()
        _check(load().maze_batch_get_stats(self.h, int(i), ctypes.byref(s)))
        return s.as_dict()

    def all_stats(self) -> list:
        """Statistics of every slot (a free slot has step == -1), one call."""
        arr = (MazeStats * self.max_sims)()
        _check(load().maze_batch_get_all_stats(self.h, arr, self.max_sims))
        return [arr[i].as_dict() for i in range(self.max_sims)]

    def tune(self, steps_per_trial: int = 5):
        c, ms = _I(), _D()
        _check(load().maze_batch_tune(self.h, int(steps_per_trial), ctypes.byref(c), ctypes.byref(ms)))
        return c.value, ms.value

    def autotune(self, steps_per_trial: int = 5) -> list:
        """Per-size-class choice of CTAs per box, V-cycle schedule and coarse
        tail; returns the table (one dict per grid size)."""
        arr = (MazeTuneEntry * 64)()
        n = _I()
        _check(load().maze_batch_autotune(self.h, int(steps_per_trial), arr, 64, ctypes.byref(n)))
        return [arr[k].as_dict() for k in range(n.value)]
