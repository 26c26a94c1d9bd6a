"""Parity of the windowed synthesized-domain aggregation weights (Sec. 7.3,
Def. "Windowed synthesized-domain weighting models") of the CUDA path with
the oracle, through the C ABI: both stages, the weighting models of each
stage, patch and group scope, hard and soft thresholding."""
import numpy as np
import pytest

from tests import parity as PT
from tests.test_gpu_parity import CASES

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


def _op(oracle, y, cfg, mc=0, **kw):
    return oracle.params(y.shape, cfg["patch"], cfg["step"], cfg["search"], cfg["noise"], cfg["group_size"], 2, mc,
                         weight_domain="windowed_synthesis", **kw)


@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
@pytest.mark.parametrize("kw", [dict(), dict(weight_model="classic", weight_scope="group"), dict(ht_rule="soft")],
                         ids=["variance-patch", "classic-group", "soft"])
def test_stage1_windowed_parity(ctx, oracle, case, kw):
    import torch
    import paper_2609_34622_b300.bmnd as bm
    name, y, x, cfg = case
    ref = oracle.stage(_op(oracle, y, cfg, **kw), y, None, 1)
    out = torch.empty(y.shape, dtype=torch.float32, device="cuda:0")
    ctx.bmnd_stage(_cuda(y), None, out, cfg["noise"], cfg["patch"], cfg["step"], cfg["search"],
                   cfg["group_size"][0], 1, 0, bm.params(weight_domain="windowed_synthesis", **kw))
    got = out.cpu().numpy()
    PT.assert_voxels(got, ref, 1.0, what=name)
    assert abs(PT.psnr(got, x) - PT.psnr(ref, x)) <= PT.PSNR_DB


@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
@pytest.mark.parametrize("model", ["variance", "risk", "classic"])
def test_stage2_windowed_parity_same_pilot(ctx, oracle, case, model):
    import torch
    import paper_2609_34622_b300.bmnd as bm
    name, y, x, cfg = case
    p = _op(oracle, y, cfg, weight_model=model)
    pilot = oracle.stage(p, y, None, 1).astype(np.float32)
    ref = oracle.stage(p, y, pilot.astype(np.float64), 2)
    out = torch.empty(y.shape, dtype=torch.float32, device="cuda:0")
    ctx.bmnd_stage(_cuda(y), _cuda(pilot), out, cfg["noise"], cfg["patch"], cfg["step"], cfg["search"],
                   cfg["group_size"][1], 2, 0, bm.params(weight_domain="windowed_synthesis", weight_model=model))
    got = out.cpu().numpy()
    PT.assert_voxels(got, ref, 1.0, what=name)
    assert abs(PT.psnr(got, x) - PT.psnr(ref, x)) <= PT.PSNR_DB


@pytest.mark.parametrize("case", CASES[1:3], ids=[c[0] for c in CASES[1:3]])
def test_denoise_windowed_mass_conserving(ctx, oracle, case):
    import torch
    import paper_2609_34622_b300.bmnd as bm
    name, y, x, cfg = case
    ref = PT.oracle_two_stages_f32_pilot(oracle, _op(oracle, y, cfg, 3), y)
    out = torch.empty(y.shape, dtype=torch.float32, device="cuda:0")
    ctx.bmnd_denoise(_cuda(y), out, cfg["noise"], cfg["patch"], cfg["step"], cfg["search"], cfg["group_size"], 2,
                     3, bm.params(weight_domain="windowed_synthesis"))
    got = out.cpu().numpy()
    PT.assert_voxels(got, ref, 1.0, what=name)
    assert float(got.astype(np.float64).sum()) == pytest.approx(float(y.astype(np.float64).sum()), rel=1e-4)


def test_unknown_domain_rejected(ctx):
    import torch
    import paper_2609_34622_b300.bmnd as bm
    y = torch.zeros((32, 32), device="cuda:0")
    with pytest.raises(bm.BmndError):
        ctx.bmnd_denoise(y, torch.empty_like(y), ("poisson", 0.1), (8, 8), (3, 3), (9, 9),
                         prm=bm.params(weight_domain=2))
