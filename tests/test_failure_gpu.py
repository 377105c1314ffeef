"""Failure detection without a GPU fault.

The grid contraction's shared-memory copies complete on mbarriers, and each wait on one is
bounded: it gives up after a fixed number of polls, raises a device error word and returns, and
the host reports POP_ETIMEOUT. pop_wait_check runs that same wait on a barrier that nothing
completes, so the wait runs out; the test checks the status and that the context then still
computes ln L to the FP64 parity bar.
"""
import time

import pytest

from test_parity_gpu import assert_f64_parity

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


def test_bounded_wait_gives_up_and_the_context_stays_usable(B, oracle):
    from paper_1904_02863_gb300 import synth
    cat = synth.make_catalog(4, 800, 6, seed=651)
    inj = synth.make_injections(20000, 6, seed=652)
    lam = synth.make_lambdas(9, 11, seed=653)
    like = B.Likelihood(0).load(cat, inj)
    B.pop_wait_check(like.ctx, True, 64)  # a completed phase: the wait succeeds
    for polls in (1, 4096):
        t0 = time.perf_counter()
        with pytest.raises(B.PopError) as e:
            B.pop_wait_check(like.ctx, False, polls)
        dt = time.perf_counter() - t0
        assert e.value.status == B.POP_ETIMEOUT and "gave up" in str(e.value)
        assert dt < 5.0, dt
        print(f"wait of {polls} polls gave up after {dt * 1e3:.2f} ms (host time of the call)")
    assert_f64_parity(like(lam, B.POP_MODE_F64), oracle.loglik(cat, inj, lam), cat.n_events)
    with pytest.raises(B.PopError) as e:
        B.pop_wait_check(like.ctx, False, 0)
    assert e.value.status == B.POP_EINVAL
    B.pop_wait_check(like.ctx, True, B.POP_WAIT_CHECK_MAX_POLLS)
    like.close()
