"""Parity of the bior1.5 spatial transform of the hard-threshold stage (App. A,
"Transforms" row) of the CUDA path with the oracle, through the C ABI: stage
1 alone, both stages, mass conservation, the windowed weights, the partial
shared-source variance, and the rejection of patch sides that are not powers
of two.  Matching does not involve the spatial transform, so stage-1 groups
are those of the DCT path; the outputs follow the voxel contract."""
import numpy as np
import pytest

from paper_2609_34622_b300 import synth
from tests import parity as PT

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    import paper_2609_34622_b300.bmnd as bm
    from paper_2609_34622_b300 import build as B
    B.build()
    c = bm.Context(0)
    yield c
    c.close()


def _cuda(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a, np.float32)).to("cuda:0")


def _cases():
    cases = []
    j1 = synth.config1()
    cases.append(("c1-2d-64", j1.y, j1.x, j1.cfg))
    rng = np.random.default_rng(41)
    x = synth.ecg_signal(3001, 250.0, rng)
    y, sp = synth.poisson_observe(x, 50.0, rng)
    cases.append(("1d-3001-p32", y, x, dict(noise=("poisson", sp), patch=(32,), step=(4,), search=(65,),
                                            group_size=(16, 32))))
    rng = np.random.default_rng(42)
    lam = synth.ellipsoid_phantom((22, 19, 17), rng)
    x = lam / lam.max()
    y, sp = synth.poisson_observe(x, 5.0, rng)
    cases.append(("3d-22x19x17", y, x, dict(noise=("poisson", sp), patch=(4, 4, 4), step=(2, 2, 2),
                                            search=(7, 7, 7), group_size=(16, 32))))
    rng = np.random.default_rng(43)
    x = synth.texture_edge_image((53, 71), rng)
    cases.append(("2d-gauss-53x71", synth.gaussian_observe(x, 25 / 255, rng), x,
                  dict(noise=("gaussian", 25 / 255), patch=(8, 8), step=(3, 3), search=(15, 15),
                       group_size=(16, 32))))
    rng = np.random.default_rng(44)
    x = synth.disc_rect_image((45, 39), rng)
    y, sp = synth.poisson_observe(x, 20.0, rng)
    cases.append(("2d-16x4", y, x, dict(noise=("poisson", sp), patch=(16, 4), step=(5, 2), search=(9, 11),
                                        group_size=(8, 16))))
    return cases


CASES = _cases()


def _op(oracle, y, cfg, mc=0, **kw):
    return oracle.params(y.shape, cfg["patch"], cfg["step"], cfg["search"], cfg["noise"], cfg["group_size"], 2, mc,
                         spatial_transform="bior1.5", **kw)


def _prm(**kw):
    import paper_2609_34622_b300.bmnd as bm
    return bm.params(spatial_transform="bior1.5", **kw)


@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_stage1_bior_parity(ctx, oracle, case):
    import torch
    name, y, x, cfg = case
    ref = oracle.stage(_op(oracle, y, cfg), y, None, 1)
    dct = oracle.stage(oracle.params(y.shape, cfg["patch"], cfg["step"], cfg["search"], cfg["noise"],
                                     cfg["group_size"], 2, 0), y, None, 1)
    out = torch.empty(y.shape, dtype=torch.float32, device="cuda:0")
    ctx.bmnd_stage(_cuda(y), None, out, cfg["noise"], cfg["patch"], cfg["step"], cfg["search"],
                   cfg["group_size"][0], 1, 0, _prm())
    got = out.cpu().numpy()
    PT.assert_voxels(got, ref, 1.0, what=name)
    assert abs(PT.psnr(got, x) - PT.psnr(ref, x)) <= PT.PSNR_DB
    # the transform matters: the DCT stage differs (patch sides of 8 and more;
    # on 4-sample axes bior1.5 is the Haar transform, still not the DCT)
    assert np.max(np.abs(ref - dct)) > 1e-3


@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_denoise_bior_two_stages(ctx, oracle, case):
    import torch
    name, y, x, cfg = case
    p = _op(oracle, y, cfg)
    out = torch.empty(y.shape, dtype=torch.float32, device="cuda:0")
    ctx.bmnd_denoise(_cuda(y), out, cfg["noise"], cfg["patch"], cfg["step"], cfg["search"], cfg["group_size"], 2,
                     0, _prm())
    frac = PT.two_stage_contract(ctx, oracle, p, y, x, cfg, out.cpu().numpy(), _cuda, _prm(), what=name)
    assert frac >= 0.5


@pytest.mark.parametrize("case", CASES[:3], ids=[c[0] for c in CASES[:3]])
def test_denoise_bior_mass_conserving(ctx, oracle, case):
    import torch
    name, y, x, cfg = case
    p = _op(oracle, y, cfg, 3)
    out = torch.empty(y.shape, dtype=torch.float32, device="cuda:0")
    ctx.bmnd_denoise(_cuda(y), out, cfg["noise"], cfg["patch"], cfg["step"], cfg["search"], cfg["group_size"], 2,
                     3, _prm())
    got = out.cpu().numpy()
    frac = PT.two_stage_contract(ctx, oracle, p, y, x, cfg, got, _cuda, _prm(), what=name)
    assert frac >= 0.3
    assert float(got.astype(np.float64).sum()) == pytest.approx(float(y.astype(np.float64).sum()), rel=1e-4)


@pytest.mark.parametrize("case", [CASES[0], CASES[4]], ids=[CASES[0][0], CASES[4][0]])
@pytest.mark.parametrize("kw", [dict(weight_domain="windowed_synthesis"), dict(cov_planes=4),
                                dict(ht_rule="soft")], ids=["windowed", "shared-source-4", "soft"])
def test_stage1_bior_variants(ctx, oracle, case, kw):
    import torch
    name, y, x, cfg = case
    ref = oracle.stage(_op(oracle, y, cfg, **kw), y, None, 1)
    out = torch.empty(y.shape, dtype=torch.float32, device="cuda:0")
    ctx.bmnd_stage(_cuda(y), None, out, cfg["noise"], cfg["patch"], cfg["step"], cfg["search"],
                   cfg["group_size"][0], 1, 0, _prm(**kw))
    got = out.cpu().numpy()
    PT.assert_voxels(got, ref, 1.0, what=name)
    assert abs(PT.psnr(got, x) - PT.psnr(ref, x)) <= PT.PSNR_DB


def test_bior_batched_equals_single(ctx):
    """A batch mixing bior1.5 arrays of two shapes gives each array the bits
    of its own call."""
    import torch
    a, b = CASES[0], CASES[4]
    ys = [_cuda(a[1]), _cuda(b[1])]
    outs = [torch.empty_like(t) for t in ys]
    cfgs = [dict(a[3], stages=2, mass_conserve=0), dict(b[3], stages=2, mass_conserve=0)]
    ctx.bmnd_denoise_batch(ys, outs, cfgs, _prm())
    for y, o, c in zip(ys, outs, cfgs):
        single = torch.empty_like(y)
        ctx.bmnd_denoise(y, single, c["noise"], c["patch"], c["step"], c["search"], c["group_size"], 2, 0, _prm())
        assert torch.equal(single, o)


def test_bior_rejects_non_power_of_two_patch(ctx):
    import torch
    import paper_2609_34622_b300.bmnd as bm
    y = torch.zeros((37, 29), device="cuda:0")
    with pytest.raises(bm.BmndError):
        ctx.bmnd_denoise(y, torch.empty_like(y), ("poisson", 0.1), (5, 4), (3, 2), (9, 7), prm=_prm())
    with pytest.raises(bm.BmndError):
        ctx.bmnd_denoise(y, torch.empty_like(y), ("poisson", 0.1), (8, 8), (3, 3), (9, 9),
                         prm=bm.params(spatial_transform=2))
