"""Tile autotuning (bmnd_autotune): the chosen core is kept by the context and
used by later calls, whose output then equals the tuner's own final output
bitwise; against the planner's tiling the output differs only by the order of
floating-point additions."""
import numpy as np
import pytest

from paper_2609_34622_b300 import synth

pytestmark = pytest.mark.gpu


def _case(k):
    rng = np.random.default_rng(97)
    if k == 0:
        x = synth.ecg_signal(12000, 250.0, rng)
        y, sp = synth.poisson_observe(x, 50.0, rng)
        return y, dict(noise=("poisson", sp), patch=(32,), step=(4,), search=(129,))
    x = synth.disc_rect_image((72, 90), rng)
    y, sp = synth.poisson_observe(x, 10.0, rng)
    return y, dict(noise=("poisson", sp), patch=(8, 8), step=(3, 3), search=(19, 19))


@pytest.mark.parametrize("k", [0, 1])
def test_autotune_kept_and_close_to_planner(k):
    import torch
    import paper_2609_34622_b300.bmnd as bm
    y_np, c = _case(k)
    y = torch.from_numpy(np.ascontiguousarray(y_np, np.float32)).cuda()
    args = (c["noise"], c["patch"], c["step"], c["search"], (16, 32), 2, 0)
    ref_ctx = bm.Context(0)
    planned = torch.empty_like(y)
    ref_ctx.bmnd_denoise(y, planned, *args)
    ctx = bm.Context(0)
    tuned = torch.empty_like(y)
    core = ctx.bmnd_autotune(y, tuned, *args)
    assert len(core) == y.dim() and all(1 <= v <= s for v, s in zip(core, y.shape))
    again = torch.empty_like(y)
    ctx.bmnd_denoise(y, again, *args)
    g_out = torch.empty_like(y)
    g = ctx.bmnd_graph_create(y, g_out, *args)
    g.bmnd_graph_launch()
    torch.cuda.synchronize()
    np.testing.assert_array_equal(again.cpu().numpy(), tuned.cpu().numpy())
    np.testing.assert_array_equal(g_out.cpu().numpy(), tuned.cpu().numpy())
    d = np.abs(tuned.cpu().numpy().astype(np.float64) - planned.cpu().numpy())
    assert d.max() <= 1e-4, d.max()
    g.close()
    ctx.close()
    ref_ctx.close()


def test_autotune_batch_kept_and_bitwise():
    """bmnd_autotune_batch: the core chosen on the whole batch is kept for the
    problem key; the tuner's outputs, a later batched call and a later call per
    array all give the same bits (a job's result does not depend on the batch
    it runs in)."""
    import torch
    import paper_2609_34622_b300.bmnd as bm
    rng = np.random.default_rng(98)
    ys, cfgs = [], []
    for k in range(4):
        x = synth.disc_rect_image((72, 90), rng)
        y, sp = synth.poisson_observe(x, 5.0 + 5 * k, rng)
        ys.append(torch.from_numpy(np.ascontiguousarray(y, np.float32)).cuda())
        cfgs.append(dict(noise=("poisson", sp), patch=(8, 8), step=(3, 3), search=(19, 19), group_size=(16, 32),
                         stages=2, mass_conserve=0))
    ctx = bm.Context(0)
    tuned = [torch.empty_like(y) for y in ys]
    core = ctx.bmnd_autotune_batch(ys, tuned, cfgs)
    assert len(core) == 2 and all(1 <= v <= s for v, s in zip(core, ys[0].shape))
    again = [torch.empty_like(y) for y in ys]
    ctx.bmnd_denoise_batch(ys, again, cfgs)
    for a, b in zip(tuned, again):
        assert torch.equal(a, b)
    for y, c, a in zip(ys, cfgs, again):
        single = torch.empty_like(y)
        ctx.bmnd_denoise(y, single, c["noise"], c["patch"], c["step"], c["search"], c["group_size"], 2, 0)
        assert torch.equal(single, a)
