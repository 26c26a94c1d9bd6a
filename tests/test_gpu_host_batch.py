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
