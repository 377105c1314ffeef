"""The FP64 weight kernel's own exp, expm1 and reciprocal (Tang's table-driven
exponential; seeded Newton reciprocal) against the host's libm (numpy), against
CUDA's own exp (torch on the GPU), and against their error bounds.

The exponentials reduce their argument with one constant, fl(ln2/2048), whose
relative error (that of fl(ln 2), 3.35e-17) adds |x| 3.35e-17 relative error to
exp(x): at most 0.31 |x| ulp on top of the table method's 2 ulp.  exp takes its
table index near floor(x 2048/ln2) from FP32 arithmetic and assembles
T_hi (1 + e^r - 1 - r) + T_lo from bits, which bounds it by one ulp for a result
in [1, 2) times a power of two, and 1.5 ulp just below a power of two (table
entry 0 with r < 0); libm adds up to half an ulp of its own."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1904_02863_gb300 import binding as B
    from paper_1904_02863_gb300 import build
    build.build()
    c = B.pop_create(0)
    yield c
    B.pop_destroy(c)


def ulps(a, b):
    """|a - b| in units of the last place of b."""
    return np.abs(a - b) / np.spacing(np.abs(b))


def test_exp_within_two_ulp_of_libm(ctx):
    from paper_1904_02863_gb300 import binding as B
    rng = np.random.default_rng(1)
    x = np.concatenate([rng.uniform(-700, 709, 200000), rng.uniform(-1, 1, 100000),
                        rng.uniform(-1e-6, 1e-6, 20000), np.arange(-40, 41) * np.log(2) / 2048,
                        [0.0, -0.0, 1e-300, -1e-300, 709.5, -706.9]])
    y = B.pop_math_check(ctx, 0, x)
    e = ulps(y, np.exp(x))
    assert (e <= 2.0 + 0.31 * np.abs(x)).all(), np.max(e - 0.31 * np.abs(x))
    small = np.abs(x) <= 1.0
    assert np.max(e[small]) <= 2.0 and np.mean(e[small]) < 0.5


def test_exp_against_cuda_exp(ctx):
    import torch
    from paper_1904_02863_gb300 import binding as B
    x = np.random.default_rng(2).uniform(-50, 50, 100000)
    y = B.pop_math_check(ctx, 0, x)
    ref = torch.exp(torch.from_numpy(x).cuda()).cpu().numpy()
    assert (ulps(y, ref) <= 3.0 + 0.31 * np.abs(x)).all()


def test_exp_range_ends(ctx):
    from paper_1904_02863_gb300 import binding as B
    x = np.array([-707.5, -1e30, -np.inf, 710.0, 1e30, np.inf])
    y = B.pop_math_check(ctx, 0, x)
    np.testing.assert_array_equal(y, [0.0, 0.0, 0.0, np.inf, np.inf, np.inf])


def test_expm1_relative_accuracy(ctx):
    from paper_1904_02863_gb300 import binding as B
    rng = np.random.default_rng(3)
    x = np.concatenate([rng.uniform(-20, 5, 200000), rng.uniform(-1e-3, 1e-3, 100000),
                        -np.logspace(-300, 1, 5000), np.logspace(-300, 1, 5000), [0.0]])
    y = B.pop_math_check(ctx, 1, x)
    ref = np.expm1(x)
    nz = ref != 0
    # the reduction's error is |x| 3.35e-17 of exp(x), i.e. of exp(x) / |expm1(x)| times the result
    bound = 2.0 + 0.31 * np.abs(x[nz]) * np.exp(x[nz]) / np.abs(ref[nz])
    assert (ulps(y[nz], ref[nz]) <= bound).all()
    assert y[~nz].tolist() == [0.0] * int((~nz).sum())
    assert B.pop_math_check(ctx, 1, np.array([-800.0]))[0] == -1.0


def test_reciprocal_correct_to_half_ulp_bound(ctx):
    from paper_1904_02863_gb300 import binding as B
    rng = np.random.default_rng(4)
    x = np.concatenate([10 ** rng.uniform(-300, 300, 200000), rng.uniform(1e-3, 10, 100000)])
    y = B.pop_math_check(ctx, 2, x)
    assert np.max(ulps(y, 1.0 / x)) <= 1.0


def test_exp_at_the_index_switches_and_range_ends(ctx):
    """Arguments within a few ulp of multiples of ln2/2048 (where the floor index changes), of
    multiples of ln2 (table entry 0, whose r can be slightly negative: results just below a
    power of two), and near both ends of the range."""
    from paper_1904_02863_gb300 import binding as B
    rng = np.random.default_rng(6)
    step = np.log(2) / 2048
    ks = np.concatenate([np.arange(-3000, 3000), rng.integers(-2_088_000, 2_096_000, 20000)])
    base = ks * step
    base = base[(base > -706.9) & (base < 709.6)]
    eps = np.array([-1e-9, -1e-12, -1e-15, 0.0, 1e-15, 1e-12, 1e-9])
    x = (base[:, None] * (1.0 + eps[None, :]) + eps[None, :]).ravel()
    m = np.arange(-1019, 1024) * np.log(2)
    m = m[(m > -706.9) & (m < 709.6)]
    x = np.concatenate([x, m, np.nextafter(m, -np.inf), np.nextafter(m, np.inf), m - 1e-13, m + 1e-13,
                        np.linspace(709.0, 709.69, 2000), np.linspace(-706.99, -706.0, 2000)])
    y = B.pop_math_check(ctx, 0, x)
    e = ulps(y, np.exp(x))
    assert (e <= 2.0 + 0.31 * np.abs(x)).all(), np.max(e - 0.31 * np.abs(x))
    small = np.abs(x) <= 1.0
    assert np.max(e[small]) <= 2.0


def test_log_against_libm(ctx):
    """The finalise's ln x (Tang's table-driven logarithm, 129 entries) within 2 ulp of libm, with
    the library's log for zero, subnormal, infinite and negative arguments."""
    from paper_1904_02863_gb300 import binding as B
    rng = np.random.default_rng(9)
    x = np.concatenate([10.0 ** rng.uniform(-307, 308, 200000), rng.uniform(0.25, 4.0, 100000),
                        1.0 + rng.uniform(-2.0 ** -6, 2.0 ** -6, 100000),
                        1.0 + np.array([2.0 ** -8, -2.0 ** -8, 2.0 ** -9, -2.0 ** -9, 1e-12, -1e-12, 2.0 ** -52]),
                        [np.nextafter(1.0, 0.0), 1.0, 2.0, 0.5, 4096.0, 1.0 / 3.0],
                        2.0 ** np.arange(-1022.0, 1024.0) * (1.0 + 2.0 ** -8)])
    y = B.pop_math_check(ctx, 8, x)
    ref = np.log(x)
    nz = ref != 0.0
    e = ulps(y[nz], ref[nz])
    assert e.max() <= 2.0 and e.mean() < 0.4, (e.max(), e.mean())
    assert (y[~nz] == 0.0).all()
    special = np.array([0.0, 5e-324, 1e-310, np.inf, -1.0, np.nan])
    ys = B.pop_math_check(ctx, 8, special)
    with np.errstate(divide="ignore"):
        np.testing.assert_allclose(ys[:4], np.log(special[:4]), rtol=1e-15)
    assert np.isnan(ys[4]) and np.isnan(ys[5])
