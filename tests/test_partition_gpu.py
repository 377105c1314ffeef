"""The event-partition path on the GPU: two contexts each hold a disjoint range of
events and share of injections (as two ranks would); their pop_loglik_parts add up,
through replicas.combine_parts, to the single-context ln L within 1e-13 relative
(FP64), and within the FP32 budget in FP32 mode."""
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


def test_two_partitions_match_one_context(B, oracle):
    from paper_1904_02863_gb300 import replicas, synth
    sizes = np.array([4097, 1, 300, 9000, 64, 4096, 2500, 777])
    cat = synth.make_catalog(len(sizes), sizes, 7, seed=801)
    inj = synth.make_injections(300000, 7, seed=802)
    lam = synth.make_lambdas(50, 12, seed=803)
    lam[4, 6] = -1.0
    whole = B.Likelihood(0).load(cat, inj)
    world = 2
    parts = [replicas.EventPartition(cat, inj, r, world, device=0) for r in range(world)]
    for mode in (B.POP_MODE_F64, B.POP_MODE_F32):
        ref = whole(lam, mode)
        got = [B.pop_loglik_parts(p.like.ctx, lam, mode) for p in parts]
        tot = [sum(g[i] for g in got) for i in range(3)]
        lnL, lnxi, neff, flags = replicas.combine_parts(*tot, cat.n_events, inj.n_draw, (got[0][3] & 1) != 0)
        np.testing.assert_array_equal(flags, ref[3])
        fin = np.isfinite(ref[0])
        np.testing.assert_array_equal(np.isfinite(lnL), fin)
        scale = np.abs(ref[0][fin] + cat.n_events * ref[1][fin]) + cat.n_events * np.abs(ref[1][fin])
        if mode == B.POP_MODE_F64:
            assert (np.abs(lnL[fin] - ref[0][fin]) <= 1e-13 * scale + 1e-12).all()
            np.testing.assert_allclose(lnxi[fin], ref[1][fin], rtol=1e-13)
        else:
            # the injection chunks split at other places: FP32 chunk sums round differently
            assert np.abs(lnL[fin] - ref[0][fin]).max() <= 1e-5 * cat.n_events
    # the partition class itself (one rank: no collective) gives the same as the whole
    one = replicas.EventPartition(cat, inj, 0, 1, device=0)
    r1, rw = one(lam), whole(lam)
    np.testing.assert_array_equal(r1[3], rw[3])
    fin = np.isfinite(rw[0])
    np.testing.assert_array_equal(r1[0][~fin], rw[0][~fin])
    assert np.abs(r1[0][fin] - rw[0][fin]).max() <= 1e-9
    for p in parts + [one]:
        p.close()
    whole.close()


def test_parts_refuse_the_grid_and_the_surrogate(B):
    from paper_1904_02863_gb300 import synth
    cat = synth.make_catalog(3, 100, 6, seed=804)
    inj = synth.make_injections(5000, 6, seed=805)
    like = B.Likelihood(0).load(cat, inj)
    lam = synth.make_lambdas(4, 11, seed=806)
    with pytest.raises(B.PopError):
        B.pop_loglik_parts(like.ctx, lam, B.POP_MODE_F32_SURROGATE)
    m1, q, pdet = synth.campaign_vt_grid(50, 20)
    B.pop_load_vt_grid(like.ctx, m1, q, pdet)
    B.pop_set_xi_source(like.ctx, B.POP_XI_GRID)
    with pytest.raises(B.PopError):
        B.pop_loglik_parts(like.ctx, lam)
    like.close()
