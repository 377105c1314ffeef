"""pop_loglik_f64_noalloc, the entry point for callers that cannot allocate.

Some callers cannot call cudaMalloc: their device memory all belongs to an
outer pool or framework, or their sampler loop must not allocate while it
runs.  They pass their own device buffers to pop_loglik_f64_noalloc, whose
scratch is one static device array inside libpop.so.  Through the C-ABI, two
calls in a row (different Lambda batches, so the second reuses scratch the
first wrote) must reproduce the context-based pop_loglik and the FP64 CPU
oracle within the tolerance of the other FP64 parity tests; a call too big for
the array, malformed inputs and host memory must be refused; and a call must
leave free device memory unchanged.
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


def _outs(K):
    import torch
    return (torch.empty(K, dtype=torch.float64, device="cuda"), torch.empty(K, dtype=torch.float64, device="cuda"),
            torch.empty(K, dtype=torch.float64, device="cuda"), torch.empty(K, dtype=torch.int32, device="cuda"))


def _host(out):
    got = [o.cpu().numpy() for o in out]
    got[3] = got[3].view(np.uint32)
    return got


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
        out = _outs(len(L))
        B.pop_loglik_f64_noalloc(off, th, pr, inj.n_draw, ith, pd, t(L), out)
        f64_close(_host(out), ref, cat.n_events)


@pytest.mark.parametrize("n_dims", [6, 7])
def test_noalloc_matches_the_oracle(B, n_dims):
    """This entry point has its own weight kernel (raw samples, CUDA's exp): compare it with the
    FP64 CPU oracle directly, on two calls in a row."""
    import torch
    import oracle
    from paper_1904_02863_gb300 import synth
    sizes = np.array([1, 700, 4097, 33, 2500, 5])
    cat = synth.make_catalog(len(sizes), sizes, n_dims, seed=321 + n_dims)
    inj = synth.make_injections(40000, n_dims, seed=322)
    P = 11 + (n_dims == 7)
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    off, th, pr, ith, pd = t(cat.offsets), t(cat.theta), t(cat.prior), t(inj.theta), t(inj.p_draw)
    for seed, K in ((323, 29), (324, 64)):
        L = synth.make_lambdas(K, P, seed=seed)
        L[5, 3] = L[5, 2] - 1.0   # mmax < mmin: an invalid row
        out = _outs(K)
        B.pop_loglik_f64_noalloc(off, th, pr, inj.n_draw, ith, pd, t(L), out)
        f64_close(_host(out), oracle.loglik(cat, inj, L), cat.n_events)


def test_noalloc_refuses_malformed_inputs_and_recovers(B):
    """Malformed CSR offsets and a non-positive prior give POP_EINVAL (the kernels skip what they
    cannot read); the next well-formed call still matches the oracle."""
    import torch
    import oracle
    from paper_1904_02863_gb300 import synth
    cat = synth.make_catalog(5, [10, 300, 41, 7, 2000], 6, seed=331)
    inj = synth.make_injections(30000, 6, seed=332)
    L = synth.make_lambdas(16, 11, seed=333)
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    good = dict(offsets=t(cat.offsets), theta=t(cat.theta), prior=t(cat.prior), n_draw=inj.n_draw,
                inj_theta=t(inj.theta), p_draw=t(inj.p_draw), lambdas=t(L))
    bad_prior = cat.prior.copy()
    bad_prior[400] = 0.0
    short_end = cat.offsets.copy()
    short_end[-1] -= 1                     # offsets[N] != n_samples
    past_end = cat.offsets.copy()
    past_end[-1] += 5                      # last event ends beyond the samples
    backwards = cat.offsets.copy()
    backwards[2] = backwards[3] + 1        # event 2 has end <= start
    cases = [dict(prior=t(bad_prior)), dict(offsets=t(short_end)), dict(offsets=t(past_end)),
             dict(offsets=t(backwards))]
    for change in cases:
        args = {**good, **change}
        with pytest.raises(B.PopError) as e:
            B.pop_loglik_f64_noalloc(out=_outs(len(L)), **args)
        assert e.value.status == B.POP_EINVAL, str(e.value)
    out = _outs(len(L))
    B.pop_loglik_f64_noalloc(out=out, **good)
    f64_close(_host(out), oracle.loglik(cat, inj, L), cat.n_events)


def test_noalloc_refuses_host_memory_before_any_launch(B):
    """A pinned host buffer in place of a device one is refused by the library's pointer check."""
    import ctypes
    import torch
    from paper_1904_02863_gb300 import synth
    cat = synth.make_catalog(2, 50, 6, seed=341)
    inj = synth.make_injections(20000, 6, seed=342)
    L = synth.make_lambdas(4, 11, seed=343)
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    host_theta = torch.from_numpy(cat.theta).pin_memory()
    out = _outs(4)
    p = lambda x: ctypes.c_void_p(x.data_ptr())
    msg = ctypes.create_string_buffer(256)
    off, pr, ith, pd, lam = t(cat.offsets), t(cat.prior), t(inj.theta), t(inj.p_draw), t(L)
    rc = B.load_library().pop_loglik_f64_noalloc(
        0, None, 2, p(off), cat.theta.shape[0], 6, p(host_theta), p(pr), inj.theta.shape[0], inj.n_draw,
        p(ith), p(pd), 4, 11, p(lam), p(out[0]), p(out[1]), p(out[2]), p(out[3]), msg, 256)
    assert rc == B.POP_EINVAL and b"theta" in msg.value, msg.value
    with pytest.raises(ValueError):
        B.pop_loglik_f64_noalloc(off, host_theta, pr, inj.n_draw, ith, pd, lam, out)


def test_noalloc_allocates_nothing(B):
    """Free device memory is the same before and after a call (after one warm-up call, which may
    load the library's kernels)."""
    import torch
    from paper_1904_02863_gb300 import synth
    cat = synth.make_catalog(20, 3000, 6, seed=351)
    inj = synth.make_injections(50000, 6, seed=352)
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    args = (t(cat.offsets), t(cat.theta), t(cat.prior), inj.n_draw, t(inj.theta), t(inj.p_draw),
            t(synth.make_lambdas(256, 11, seed=353)))
    out = _outs(256)
    B.pop_loglik_f64_noalloc(*args, out)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(3):
        B.pop_loglik_f64_noalloc(*args, out)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0, (free0, free1)


def test_noalloc_refuses_batches_beyond_the_scratch_array(B):
    import torch
    from paper_1904_02863_gb300 import synth
    cat = synth.make_catalog(1000, 4, 6, seed=311)
    inj = synth.make_injections(20000, 6, seed=312)
    K = 4096   # 4096 * 8 * (1000 + 2 * 2) bytes > 16 MiB
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    L = t(synth.make_lambdas(K, 11, seed=313))
    out = _outs(K)
    with pytest.raises(B.PopError) as e:
        B.pop_loglik_f64_noalloc(t(cat.offsets), t(cat.theta), t(cat.prior), inj.n_draw, t(inj.theta),
                                 t(inj.p_draw), L, out)
    assert e.value.status == B.POP_EINVAL and "scratch" in str(e.value)
