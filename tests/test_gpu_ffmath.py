"""The float-float (about 48-bit) arithmetic that evaluates the refined edge
costs, against FP64 references (numpy's float64 functions, within one unit
of 2^-53 of the exact results) on the same float-float-rounded inputs: every
result within a few units of 2^-48 (2.5e-14) of the reference."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from paper_2603_16103_gb300 import binding as B
    c = B.Context()
    yield c
    c.close()


def ff_round(x):
    """The float-float value the library makes of a float64 input."""
    x = np.asarray(x, dtype=np.float64)
    h = x.astype(np.float32).astype(np.float64)
    l = (x - h).astype(np.float32).astype(np.float64)
    return h + l


def rng_vals(seed, lo, hi, n, log=False):
    r = np.random.default_rng(seed)
    if log:
        return np.exp(r.uniform(np.log(lo), np.log(hi), n))
    return r.uniform(lo, hi, n)


def test_exp(ctx):
    x = ff_round(np.concatenate([rng_vals(1, -69.0, 85.0, 200000), rng_vals(2, -1e-3, 1e-3, 20000),
                                 [0.0, 1.0, -1.0, 0.5 * np.log(2.0), -12.0, 2.0]]))
    got = ctx.selftest_ff(0, x)
    ref = np.exp(x)
    rel = np.abs(got - ref) / ref
    assert np.all(rel <= 8e-15 * (1.0 + np.abs(x))), rel.max()
    # below e^-69 the tail float would be subnormal (flushed to zero):
    # absolute accuracy only, far below anything the cost can see
    xs = ff_round(rng_vals(14, -102.0, -69.0, 20000))
    assert np.all(np.abs(ctx.selftest_ff(0, xs) - np.exp(xs)) <= 1e-37)
    # below the float range the result is 0, above it infinity
    assert np.all(ctx.selftest_ff(0, np.array([-104.0, -200.0])) == 0.0)
    assert np.all(np.isinf(ctx.selftest_ff(0, np.array([89.0]))))


def test_log(ctx):
    x = ff_round(np.concatenate([rng_vals(3, 1e-30, 1e30, 200000, log=True),
                                 rng_vals(4, 0.999, 1.001, 20000), [1.0, 2.0, 0.5, np.sqrt(0.5)]]))
    got = ctx.selftest_ff(1, x)
    ref = np.log(x)
    err = np.abs(got - ref)
    assert np.all(err <= 2.5e-14 * np.maximum(1.0, np.abs(ref))), err.max()
    assert ctx.selftest_ff(1, np.array([1.0]))[0] == 0.0


def test_log1p(ctx):
    x = ff_round(np.concatenate([rng_vals(5, 0.0, 1.0, 100000), rng_vals(6, 1e-30, 1e-3, 20000, log=True),
                                 [0.0]]))
    got = ctx.selftest_ff(2, x)
    ref = np.log1p(x)
    # absolute accuracy: 1 + x is formed with an error of about 2^-48
    assert np.all(np.abs(got - ref) <= 2.5e-14), np.abs(got - ref).max()
    small = x < 1e-10
    assert np.all(np.abs(got[small] - ref[small]) <= 1e-7 * ref[small])


def test_sqrt_div_mul(ctx):
    x = ff_round(rng_vals(7, 1e-30, 1e30, 100000, log=True))
    y = ff_round(rng_vals(8, 1e-10, 1e10, 100000, log=True) * np.where(rng_vals(9, 0, 1, 100000) < 0.5, -1, 1))
    s = ctx.selftest_ff(3, x)
    assert np.all(np.abs(s - np.sqrt(x)) <= 2.5e-14 * np.sqrt(x))
    assert ctx.selftest_ff(3, np.array([0.0]))[0] == 0.0
    x = ff_round(rng_vals(15, 1e-10, 1e10, 100000, log=True))
    q = ctx.selftest_ff(4, x, y)
    assert np.all(np.abs(q - x / y) <= 2.5e-14 * np.abs(x / y))
    m = ctx.selftest_ff(7, ff_round(rng_vals(10, -1e3, 1e3, 100000)), y[:100000] * 1e-10)
    ref = ff_round(rng_vals(10, -1e3, 1e3, 100000)) * (y[:100000] * 1e-10)
    assert np.all(np.abs(m - ref) <= 2.5e-14 * np.abs(ref))


def test_softplus_lse(ctx):
    x = ff_round(np.concatenate([rng_vals(11, -80.0, 80.0, 100000), [0.0, -1e-8, 1e-8]]))
    got = ctx.selftest_ff(5, x)
    ref = np.logaddexp(0.0, x)
    assert np.all(np.abs(got - ref) <= 2.5e-14 * np.maximum(1.0, np.abs(ref)))
    a = ff_round(rng_vals(12, -50.0, 50.0, 100000))
    b = ff_round(np.concatenate([rng_vals(13, -50.0, 50.0, 99990), a[:10]]))
    got = ctx.selftest_ff(6, a, b)
    ref = np.logaddexp(a, b)
    assert np.all(np.abs(got - ref) <= 2.5e-14 * np.maximum(1.0, np.abs(ref)))


def test_selftest_rejects_bad_arguments(ctx):
    from paper_2603_16103_gb300 import binding as B
    with pytest.raises(B.NgsError):
        ctx.selftest_ff(8, np.zeros(4))
    with pytest.raises(B.NgsError):
        ctx.selftest_ff(4, np.zeros(4))  # division needs y
