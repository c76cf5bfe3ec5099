"""The FP32/FP64 conversions that the FP64 kernels perform with integer
operations (dbl_to_flt, flt_to_dbl, floor_ll, fix_to_dbl) equal the GPU's
conversion instructions bit for bit, on edge cases and on random values
across the exponent range."""
import numpy as np
import pytest

from paper_2505_20418_gb300 import maze as M

pytestmark = pytest.mark.gpu


def inputs():
    f32 = np.float32
    tiny = [0.0, -0.0, 5e-324, -5e-324, 2.0 ** -1022, 2.0 ** -126, 2.0 ** -127, 2.0 ** -149, 2.0 ** -150,
            1.5 * 2.0 ** -150, 2.0 ** -151, 3 * 2.0 ** -151, 1.0000001 * 2.0 ** -149, -2.0 ** -149,
            float(np.finfo(f32).tiny) * (1 - 2.0 ** -24), float(np.finfo(f32).tiny) * (1 - 2.0 ** -25)]
    big = [float(np.finfo(f32).max), float(np.finfo(f32).max) * (1 + 2.0 ** -25),
           float(np.finfo(f32).max) * (1 + 2.0 ** -24), 2.0 ** 128, 1e300, -1e300, np.inf, -np.inf, np.nan]
    # ties: halfway between neighbouring floats (even and odd lower neighbours)
    base = np.array([1.0, 1.0 + 2.0 ** -23, 3.0, 1e-3, 123.456, -7.5, 2.0 ** -140], dtype=np.float64)
    ulp = np.abs(np.spacing(base.astype(f32)).astype(np.float64))
    ties = np.concatenate([base + ulp / 2, base - ulp / 2, base + ulp / 2 * (1 + 2.0 ** -30)])
    floors = [0.5, -0.5, -1e-300, 1.0, -1.0, 2.5, -2.5, 1e15 + 0.5, -1e15 - 0.5, 2.0 ** 52, 2.0 ** 53 + 2,
              -(2.0 ** 60), 3.9e18, 0.49999999999999994, -0.9999999999999999]
    rng = np.random.default_rng(11)
    r = rng.standard_normal(200000) * 2.0 ** rng.integers(-160, 140, 200000)
    r2 = rng.uniform(-1e6, 1e6, 100000)
    return np.concatenate([np.array(tiny + big + floors), ties, r, r2])


def test_integer_pipe_conversions_equal_the_instructions():
    x = inputs()
    st, o = M.maze_convert_probe(x)
    assert st == M.MAZE_OK, M.maze_last_error()
    nan = np.isnan(o["f_hw"])
    assert np.array_equal(nan, np.isnan(o["f_own"]))
    assert np.array_equal(o["f_own"][~nan].view(np.uint32), o["f_hw"][~nan].view(np.uint32))
    ok = ~np.isnan(o["d_hw"])
    assert np.array_equal(o["d_own"][ok].view(np.uint64), o["d_hw"][ok].view(np.uint64))
    assert np.isnan(o["d_own"][~ok]).all()
    assert np.array_equal(o["floor_own"], o["floor_hw"])
    assert np.array_equal(o["fix_own"].view(np.uint64), o["fix_hw"].view(np.uint64))
    # the hardware rounding is IEEE nearest-even: the FP32 results are numpy's
    fin = np.isfinite(x)
    with np.errstate(over="ignore"):
        ref = x[fin].astype(np.float32)
    assert np.array_equal(o["f_hw"][fin].view(np.uint32), ref.view(np.uint32))


def ulp_distance(a, b):
    """Distance in units in the last place between doubles of the same sign."""
    ia = a.view(np.int64).astype(object)
    ib = b.view(np.int64).astype(object)
    return np.array([abs(x - y) for x, y in zip(ia, ib)], dtype=np.float64)


def test_table_exp_within_two_ulp_of_exp():
    """The pair forces' exponential (Tang's table-driven method) against the
    CUDA math library's exp(): within 2 ulp over the arguments of the
    Tosi-Fumi repulsion and far beyond, at the table's breakpoints, and exp()
    itself outside |x| < 512 and for non-finite x."""
    rng = np.random.default_rng(3)
    ln2_64 = np.log(2.0) / 64
    k = np.arange(-2000, 2000)
    edges = np.concatenate([k * ln2_64, (k + 0.5) * ln2_64, np.nextafter((k + 0.5) * ln2_64, np.inf),
                            np.nextafter((k + 0.5) * ln2_64, -np.inf)])
    x = np.concatenate([rng.uniform(-40, 15, 200000), rng.uniform(-511.9, 511.9, 50000), edges,
                        [0.0, -0.0, 1e-300, -1e-300, 511.99, -511.99]])
    st, own, ref = M.maze_exp_probe(x)
    assert st == M.MAZE_OK, M.maze_last_error()
    assert (own > 0).all() and (ref > 0).all()
    assert ulp_distance(own, ref).max() <= 2
    y = np.array([512.0, -512.0, 700.0, -745.0, 1000.0, -1000.0, np.inf, -np.inf, np.nan])
    st, own, ref = M.maze_exp_probe(y)
    assert st == M.MAZE_OK
    assert np.array_equal(own[:-1], ref[:-1]) and np.isnan(own[-1]) and np.isnan(ref[-1])


def split_df(x):
    """x as the (hi, lo) float pair the GPU forms, and their exact sum."""
    h = x.astype(np.float32).astype(np.float64)
    l = (x - h).astype(np.float32).astype(np.float64)
    return h + l


def test_double_float_exp_against_numpy():
    """The double-float exponential of the FP64 boxes' pair kernel (Tang's
    table method with a 2^(j/64) table held as float pairs) against numpy's
    FP64 exp of the same (hi, lo) input: within 3e-14 relative across the
    pair repulsion's arguments, the table breakpoints and -70 <= x < 87 (below
    -70 the lo float turns subnormal); 0 and infinity beyond |x| = 87."""
    rng = np.random.default_rng(5)
    ln2_64 = np.log(2.0) / 64
    k = np.arange(-5000, 5000)
    x = np.concatenate([rng.uniform(-30, 12, 200000), rng.uniform(-70, 86.9, 50000), k * ln2_64,
                        (k + 0.5) * ln2_64, [0.0, -0.0, 1e-30, -1e-30, 86.9, -70.0]])
    st, own, _ = M.maze_df_probe(0, x)
    assert st == M.MAZE_OK, M.maze_last_error()
    ref = np.exp(split_df(x))
    rel = np.abs(own - ref) / ref
    assert rel.max() < 3e-14, rel.max()
    st, own, _ = M.maze_df_probe(0, np.array([88.0, 100.0, -88.0, -100.0]))
    assert st == M.MAZE_OK
    assert np.isinf(own[0]) and np.isinf(own[1]) and own[2] == 0 and own[3] == 0


def test_double_float_tosi_fumi_pair_against_oracle():
    """The Tosi-Fumi pair in double-float arithmetic (and in FP64, the other
    kernels' form) against the oracle's pair formula in FP64 on the same
    squared distance, every pair kind, 0.6 A to r_cut: -(dV/dr)/r and the
    shifted energy within 5e-13 of the sum of their terms' magnitudes (the
    double-float products keep ~2^-47; the FP64 force bar is 1e-10)."""
    from oracle import maze_oracle as O
    from paper_2505_20418_gb300 import synth
    tf = synth.tosi_fumi_nacl()
    rc = 9.0
    rng = np.random.default_rng(8)
    r = np.concatenate([rng.uniform(0.6, rc, 60000), np.linspace(1.5, rc * (1 - 1e-12), 3000)])
    r2 = r * r
    kind = rng.integers(0, 3, r.size).astype(np.int32)
    rr = np.sqrt(split_df(r2))
    V, f = O._tf_pair(rr, kind, tf)
    Vc, _ = O._tf_pair(np.full(r.size, rc), kind, tf)
    A, s, C, D = (np.asarray(v)[kind] for v in (tf.A, tf.s, tf.C, tf.D))
    ex = A * np.exp(tf.B * (s - rr))
    f_scale = (tf.B * ex + 6 * C / rr ** 7 + 8 * D / rr ** 9) / rr
    v_scale = ex + C / rr ** 6 + D / rr ** 8 + np.abs(Vc)
    for what in (1, 2):
        st, fr, vv = M.maze_df_probe(what, r2, kind, tf, rc)
        assert st == M.MAZE_OK, M.maze_last_error()
        ef = np.abs(fr - f / rr) / f_scale
        ev = np.abs(vv - (V - Vc)) / v_scale
        assert ef.max() < 5e-13 and ev.max() < 5e-13, (what, ef.max(), ev.max())
    st, _, _ = M.maze_df_probe(1, r2[:4], np.array([0, 1, 2, 3], np.int32), tf, rc)
    assert st == M.MAZE_ERR_INVALID
