"""The host-array batch entry point, the plan description and the FP32
throughput probe, through the C ABI."""
import numpy as np
import pytest

from paper_2609_34622_b300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    import paper_2609_34622_b300.bmnd as bm
    from paper_2609_34622_b300 import build as B
    B.build()
    c = bm.Context(0)
    yield c
    c.close()


def test_host_batch_equals_device_batch(ctx):
    """bmnd_denoise_batch_host returns, in host memory, bitwise the results
    of bmnd_denoise_batch on the same arrays (mixed noise kinds and shapes);
    a second call reuses its device buffers."""
    import torch
    jobs = synth.config3(n_images=3, size=96)
    ys = [j.y for j in jobs]
    cfgs = [dict(j.cfg, search=(19, 19)) for j in jobs]
    dy = [torch.from_numpy(y).cuda() for y in ys]
    do = [torch.empty_like(y) for y in dy]
    ctx.bmnd_denoise_batch(dy, do, cfgs)
    ref = [o.cpu().numpy() for o in do]
    for _ in range(2):
        outs = [np.full_like(y, np.nan) for y in ys]
        ctx.bmnd_denoise_batch_host(ys, outs, cfgs)
        for a, b in zip(outs, ref):
            np.testing.assert_array_equal(a, b)


def test_host_batch_rejects_bad_arrays(ctx):
    import paper_2609_34622_b300.bmnd as bm
    y = np.zeros((16, 16), np.float32)
    with pytest.raises(ValueError):
        ctx.bmnd_denoise_batch_host([y], [np.zeros((16, 16), np.float64)], [dict(noise=("gaussian", 0.1),
                                    patch=(4, 4), step=(2, 2), search=(5, 5))])
    with pytest.raises(bm.BmndError):
        ctx.bmnd_denoise_batch_host([y], [np.zeros_like(y)], [dict(noise=("gaussian", 0.1), patch=(4, 4),
                                    step=(2, 2), search=(4, 4))])


def test_plan_info(ctx):
    """The plan of the 1-D 262144-sample workload: tiles x core covers the
    reference origins, a region is the core plus the search halo and the
    patch extent."""
    inf = ctx.bmnd_plan_info((262144,), (32,), (4,), (129,))
    (C,) = inf["core"]
    assert inf["axes"] == 1
    assert inf["tiles"] * C >= 262144 - 32 + 1
    assert inf["region"] == C + 2 * 64 + 32 - 1


def test_fp32_peak_sane():
    """The FMA probe reports between half and 1.2 times the nominal
    148 SMs x 128 lanes x 2 flop at the maximum SM clock."""
    import paper_2609_34622_b300.bmnd as bm
    v = bm.bmnd_fp32_fma_peak(0)
    nominal = 148 * 128 * 2 * 2.032e9 / 1e12
    assert 0.5 * nominal < v < 1.2 * nominal, v


def test_mixed_rank_batch_equals_single():
    """A batch of 1-D, 2-D and 3-D arrays in one call: each array gets the
    bits of its own call (the rank classes run one after another)."""
    import torch
    import paper_2609_34622_b300.bmnd as bm
    rng = np.random.default_rng(77)
    x1 = synth.ecg_signal(4000, 250.0, rng)
    y1, s1 = synth.poisson_observe(x1, 30.0, rng)
    x2 = synth.disc_rect_image((70, 66), rng)
    y2, s2 = synth.poisson_observe(x2, 10.0, rng)
    lam = synth.ellipsoid_phantom((20, 18, 16), rng)
    y3, s3 = synth.poisson_observe(lam / lam.max(), 4.0, rng)
    jobs = [(y2, dict(noise=("poisson", s2), patch=(8, 8), step=(3, 3), search=(15, 15))),
            (y1, dict(noise=("poisson", s1), patch=(32,), step=(4,), search=(65,))),
            (y3, dict(noise=("poisson", s3), patch=(4, 4, 4), step=(2, 2, 2), search=(7, 7, 7))),
            (y2[::-1].copy(), dict(noise=("poisson", s2), patch=(8, 8), step=(3, 3), search=(15, 15)))]
    ctx = bm.Context(0)
    ys = [torch.from_numpy(np.ascontiguousarray(y, np.float32)).cuda() for y, _ in jobs]
    outs = [torch.empty_like(y) for y in ys]
    cfgs = [dict(c, group_size=(16, 32), stages=2, mass_conserve=0) for _, c in jobs]
    ctx.bmnd_denoise_batch(ys, outs, cfgs)
    for y, o, c in zip(ys, outs, cfgs):
        single = torch.empty_like(y)
        ctx.bmnd_denoise(y, single, c["noise"], c["patch"], c["step"], c["search"], c["group_size"], 2, 0)
        assert torch.equal(single, o)
