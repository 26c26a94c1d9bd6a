"""Replayable graphs (bmnd_graph_*): a recorded call must give bitwise the
output of bmnd_denoise_ex on the same input, launch after launch, and follow
new data written into its bound input."""
import numpy as np
import pytest

from paper_2609_34622_b300 import synth

pytestmark = pytest.mark.gpu


def _cases():
    rng = np.random.default_rng(91)
    cases = []
    x = synth.ecg_signal(6000, 250.0, rng)
    ys = [synth.poisson_observe(x, 30.0, rng)[0] for _ in range(2)]
    sp = synth.poisson_observe(x, 30.0, rng)[1]
    cases.append((ys, dict(noise=("poisson", sp), patch=(32,), step=(4,), search=(129,), group_size=(16, 32),
                           mass_conserve=0)))
    x = synth.disc_rect_image((70, 83), rng)
    cases.append(([synth.gaussian_observe(x, 25 / 255, rng) for _ in range(2)],
                  dict(noise=("gaussian", 25 / 255), patch=(8, 8), step=(3, 3), search=(19, 19),
                       group_size=(16, 32), mass_conserve=0)))
    lam = synth.ellipsoid_phantom((22, 20, 24), rng)
    lam = lam / lam.max()
    obs = [synth.poisson_observe(lam, 5.0, rng) for _ in range(2)]
    cases.append(([o[0] for o in obs], dict(noise=("poisson", obs[0][1]), patch=(4, 4, 4), step=(2, 2, 2),
                                            search=(7, 7, 7), group_size=(16, 32), mass_conserve=3)))
    return cases


@pytest.mark.parametrize("k", [0, 1, 2])
def test_graph_replay_equals_call(k):
    import torch
    import paper_2609_34622_b300.bmnd as bm
    ys, c = _cases()[k]
    ctx = bm.Context(0)
    ref = []
    for y in ys:
        t = torch.from_numpy(np.ascontiguousarray(y, np.float32)).cuda()
        o = torch.empty_like(t)
        ctx.bmnd_denoise(t, o, c["noise"], c["patch"], c["step"], c["search"], c["group_size"], 2,
                         c["mass_conserve"])
        ref.append(o.cpu().numpy())
    y_dev = torch.from_numpy(np.ascontiguousarray(ys[0], np.float32)).cuda()
    out = torch.full_like(y_dev, float("nan"))
    g = ctx.bmnd_graph_create(y_dev, out, c["noise"], c["patch"], c["step"], c["search"], c["group_size"], 2,
                              c["mass_conserve"])
    for _ in range(2):
        g.bmnd_graph_launch()
        torch.cuda.synchronize()
        np.testing.assert_array_equal(out.cpu().numpy(), ref[0])
    y_dev.copy_(torch.from_numpy(np.ascontiguousarray(ys[1], np.float32)))
    g.bmnd_graph_launch()
    torch.cuda.synchronize()
    np.testing.assert_array_equal(out.cpu().numpy(), ref[1])
    g.close()
    ctx.close()


def test_graph_rejects_overlap():
    import torch
    import paper_2609_34622_b300.bmnd as bm
    ctx = bm.Context(0)
    y = torch.zeros(1000, device="cuda")
    with pytest.raises(bm.BmndError) as e:
        ctx.bmnd_graph_create(y, y, ("poisson", 0.1), (32,), (4,), (33,))
    assert e.value.status == bm.EINVAL
    ctx.close()
