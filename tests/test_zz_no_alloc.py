"""pop_loglik_f64_noalloc, the entry point for callers that cannot allocate.

Some callers cannot call cudaMalloc: their device memory all belongs to an
outer pool or framework, or their sampler loop must not allocate while it
runs.  They pass their own device buffers to pop_loglik_f64_noalloc, whose
scratch is one static device array inside libpop.so.  Through the C-ABI, two
calls in a row (different Lambda batches, so the second reuses scratch the
first wrote) must reproduce the context-based pop_loglik in FP64 within the
tolerance of the other FP64 parity tests, and a call too big for the array
must be refused.
"""
import numpy as np
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


def f64_close(got, ref, n_events):
    lnL, lnxi, neff, flags = got
    r_lnL, r_lnxi, r_neff, r_flags = ref
    np.testing.assert_array_equal(flags, r_flags)
    fin = np.isfinite(r_lnL)
    np.testing.assert_array_equal(np.isfinite(lnL), fin)
    scale = np.abs(np.where(fin, r_lnL, 0.0) + n_events * r_lnxi) + n_events * np.abs(r_lnxi)
    assert (np.abs(lnL[fin] - r_lnL[fin]) <= 1e-12 * scale[fin] + 1e-13).all()
    xf = np.isfinite(r_lnxi)
    np.testing.assert_allclose(lnxi[xf], r_lnxi[xf], rtol=1e-12, atol=1e-13)
    nf = np.isfinite(r_neff) & (r_neff > 0)
    np.testing.assert_allclose(neff[nf], r_neff[nf], rtol=1e-8)


@pytest.mark.parametrize("n_dims", [6, 7])
def test_noalloc_matches_pop_loglik_on_two_calls(B, n_dims):
    import torch
    from paper_1904_02863_gb300 import synth
    sizes = np.array([1, 4095, 4096, 5000, 9000, 300, 12289, 64])
    cat = synth.make_catalog(len(sizes), sizes, n_dims, seed=301 + n_dims)
    inj = synth.make_injections(60000, n_dims, seed=302)
    P = 11 + (n_dims == 7)
    batches = [synth.make_lambdas(37, P, seed=303), synth.make_lambdas(100, P, seed=304)]
    batches[1][3, 6] = -1.0   # an invalid row
    like = B.Likelihood(0).load(cat, inj, storage=B.POP_STORE_F64)
    refs = [like(L, B.POP_MODE_F64) for L in batches]
    like.close()

    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    off, th, pr, ith, pd = t(cat.offsets), t(cat.theta), t(cat.prior), t(inj.theta), t(inj.p_draw)
    for L, ref in zip(batches, refs):
        K = len(L)
        out = (torch.empty(K, dtype=torch.float64, device="cuda"), torch.empty(K, dtype=torch.float64, device="cuda"),
               torch.empty(K, dtype=torch.float64, device="cuda"), torch.empty(K, dtype=torch.int32, device="cuda"))
        B.pop_loglik_f64_noalloc(off, th, pr, inj.n_draw, ith, pd, t(L), out)
        got = [o.cpu().numpy() for o in out]
        got[3] = got[3].view(np.uint32)
        f64_close(got, ref, cat.n_events)


def test_noalloc_refuses_batches_beyond_the_scratch_array(B):
    import torch
    from paper_1904_02863_gb300 import synth
    cat = synth.make_catalog(1000, 4, 6, seed=311)
    inj = synth.make_injections(20000, 6, seed=312)
    K = 4096   # 4096 * 8 * (1000 + 2 * 2) bytes > 16 MiB
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    L = t(synth.make_lambdas(K, 11, seed=313))
    out = (torch.empty(K, dtype=torch.float64, device="cuda"), torch.empty(K, dtype=torch.float64, device="cuda"),
           torch.empty(K, dtype=torch.float64, device="cuda"), torch.empty(K, dtype=torch.int32, device="cuda"))
    with pytest.raises(B.PopError) as e:
        B.pop_loglik_f64_noalloc(t(cat.offsets), t(cat.theta), t(cat.prior), inj.n_draw, t(inj.theta),
                                 t(inj.p_draw), L, out)
    assert e.value.status == B.POP_EINVAL and "scratch" in str(e.value)
