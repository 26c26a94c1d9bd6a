"""Parity of stage-1 soft thresholding (Def. "Coefficient thresholding",
Eq. soft-threshold, with the |a_k|^2 weighting models) of the CUDA path with
the oracle, through the C ABI, on the parity cases of the hard rule."""
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
                         ht_rule="soft", **kw)


@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
@pytest.mark.parametrize("wmodel", ["variance", "classic"])
def test_stage1_soft_parity(ctx, oracle, case, wmodel):
    import torch
    import paper_2609_34622_b300.bmnd as bm
    name, y, x, cfg = case
    ref = oracle.stage(_op(oracle, y, cfg, weight_model=wmodel), y, None, 1)
    out = torch.empty(y.shape, dtype=torch.float32, device="cuda:0")
    ctx.bmnd_stage(_cuda(y), None, out, cfg["noise"], cfg["patch"], cfg["step"], cfg["search"],
                   cfg["group_size"][0], 1, 0, bm.params(ht_rule="soft", weight_model=wmodel))
    got = out.cpu().numpy()
    PT.assert_voxels(got, ref, 1.0, what=name)
    assert abs(PT.psnr(got, x) - PT.psnr(ref, x)) <= PT.PSNR_DB


@pytest.mark.parametrize("case", CASES[1:3], ids=[c[0] for c in CASES[1:3]])
@pytest.mark.parametrize("mc", [0, 3])
def test_denoise_soft_end_to_end(ctx, oracle, case, mc):
    import torch
    import paper_2609_34622_b300.bmnd as bm
    name, y, x, cfg = case
    ref = PT.oracle_two_stages_f32_pilot(oracle, _op(oracle, y, cfg, mc), y)
    ref64, _ = oracle.denoise(_op(oracle, y, cfg, mc), y)
    out = torch.empty(y.shape, dtype=torch.float32, device="cuda:0")
    ctx.bmnd_denoise(_cuda(y), out, cfg["noise"], cfg["patch"], cfg["step"], cfg["search"], cfg["group_size"], 2,
                     mc, bm.params(ht_rule="soft"))
    got = out.cpu().numpy()
    PT.assert_voxels(got, ref, 1.0, what=name)
    assert abs(PT.psnr(got, x) - PT.psnr(ref64, x)) <= PT.PSNR_DB
    if mc == 3:
        assert float(got.astype(np.float64).sum()) == pytest.approx(float(y.astype(np.float64).sum()), rel=1e-4)


def test_soft_with_poisson_deviance(ctx, oracle):
    """Soft thresholding together with deviance matching under the reference
    finite-count rule (two ablation factors of App. B at once)."""
    import torch
    import paper_2609_34622_b300.bmnd as bm
    name, y, x, cfg = CASES[1]
    kw = dict(match_metric="poisson_deviance", match_policy="reference_finite_count")
    ref = oracle.stage(_op(oracle, y, cfg, **kw), y, None, 1)
    out = torch.empty(y.shape, dtype=torch.float32, device="cuda:0")
    ctx.bmnd_stage(_cuda(y), None, out, cfg["noise"], cfg["patch"], cfg["step"], cfg["search"],
                   cfg["group_size"][0], 1, 0, bm.params(ht_rule="soft", **kw))
    PT.assert_voxels(out.cpu().numpy(), ref, 1.0, what=name)


def test_soft_rule_rejected_when_unknown(ctx):
    import torch
    import paper_2609_34622_b300.bmnd as bm
    y = torch.zeros((32, 32), device="cuda:0")
    with pytest.raises(bm.BmndError):
        ctx.bmnd_denoise(y, torch.empty_like(y), ("poisson", 0.1), (8, 8), (3, 3), (9, 9), prm=bm.params(ht_rule=2))
