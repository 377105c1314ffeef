"""The pipe-rate diagnostic behind the kernels' rooflines (pop_pipe_rates): thread operations
per SM clock for FP64 fma, FP32 fma, MUFU ex2 and MUFU rcp, FP32 lanes of the packed fma, and
warp-wide 16-byte shared loads per SM clock.

GB300 has 2 FP64 fma lanes and 128 FP32 fma lanes per SM per clock, so the measured rates must
lie at or below those and above half of them; the MUFU rates must order ex2 >= rcp and lie
within the 4..64 per clock that any recent SM has.  A 16-byte load of a whole warp moves 512
bytes, so at 128 bytes per clock it takes at least 4 clocks when the 32 addresses differ, and
sharing addresses cannot make it slower.  A rate far outside means the chains were optimised
away or the CTAs shared SMs."""
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    torch.cuda.set_device(0)
    from paper_1904_02863_gb300 import binding, build
    build.build()
    binding.load_library()
    return binding


def test_pipe_rates(B):
    r = B.pop_pipe_rates(0)
    print("pipe rates (thread ops per SM clock):", r)
    assert 1.0 <= r["dfma"] <= 2.05, r
    assert 64.0 <= r["ffma"] <= 129.0, r
    assert 4.0 <= r["rcp"] <= r["ex2"] <= 64.0, r
    assert 64.0 <= r["ffma2_lanes"] <= 129.0, r
    assert 0.1 <= r["lds128_32addr"] <= 0.26, r
    assert r["lds128_32addr"] * 0.95 <= r["lds128_4addr"] <= 1.01, r
    with pytest.raises(B.PopError):
        B.pop_pipe_rates(-1)


def test_pipe_rates_n_writes_only_what_is_asked(B):
    import ctypes
    import numpy as np
    lib = B.load_library()
    r = np.full(9, -7.0)
    assert lib.pop_pipe_rates_n(0, r.ctypes.data_as(ctypes.c_void_p), 2) == B.POP_OK
    assert 1.0 <= r[0] <= 2.05 and 64.0 <= r[1] <= 129.0 and (r[2:] == -7.0).all(), r
    assert lib.pop_pipe_rates_n(0, r.ctypes.data_as(ctypes.c_void_p), 9) == B.POP_OK   # clamped to 7
    assert (r[7:] == -7.0).all() and 0.1 <= r[5] <= 0.26, r
    assert lib.pop_pipe_rates_n(0, r.ctypes.data_as(ctypes.c_void_p), 0) == B.POP_EINVAL
    assert lib.pop_pipe_rates_n(0, None, 3) == B.POP_EINVAL
