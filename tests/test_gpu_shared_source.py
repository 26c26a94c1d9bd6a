"""Parity of the partial shared-source Poisson variance (Sec. 5, Def.
"Partial shared-source Poisson variance model") of the CUDA path with the
oracle, through the C ABI: stage 1 and stage 2 (same pilot) for 1, 4 and 32
exact planes on the Poisson parity cases, Haar and DCT group transforms."""
import numpy as np
import pytest

from tests import parity as PT
from tests.test_gpu_parity import CASES

pytestmark = pytest.mark.gpu

POISSON = [c for c in CASES if c[3]["noise"][0] == "poisson"]


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


def _op(oracle, y, cfg, **kw):
    return oracle.params(y.shape, cfg["patch"], cfg["step"], cfg["search"], cfg["noise"], cfg["group_size"], 2, 0,
                         **kw)


@pytest.mark.parametrize("case", POISSON, ids=[c[0] for c in POISSON])
@pytest.mark.parametrize("kex", [1, 4, 32])
def test_stage1_shared_source_parity(ctx, oracle, case, kex):
    import torch
    import paper_2609_34622_b300.bmnd as bm
    name, y, x, cfg = case
    ref = oracle.stage(_op(oracle, y, cfg, cov_planes=kex), y, None, 1)
    out = torch.empty(y.shape, dtype=torch.float32, device="cuda:0")
    ctx.bmnd_stage(_cuda(y), None, out, cfg["noise"], cfg["patch"], cfg["step"], cfg["search"],
                   cfg["group_size"][0], 1, 0, bm.params(cov_planes=kex))
    got = out.cpu().numpy()
    PT.assert_voxels(got, ref, 1.0, what=name)
    assert abs(PT.psnr(got, x) - PT.psnr(ref, x)) <= PT.PSNR_DB
    # the model changes the result (overlapping members share voxels)
    diag = oracle.stage(_op(oracle, y, cfg), y, None, 1)
    assert np.max(np.abs(diag - ref)) > 1e-6


@pytest.mark.parametrize("case", POISSON, ids=[c[0] for c in POISSON])
def test_stage2_shared_source_parity_same_pilot(ctx, oracle, case):
    import torch
    import paper_2609_34622_b300.bmnd as bm
    name, y, x, cfg = case
    p = _op(oracle, y, cfg, cov_planes=4)
    pilot = oracle.stage(p, y, None, 1).astype(np.float32)
    ref = oracle.stage(p, y, pilot.astype(np.float64), 2)
    out = torch.empty(y.shape, dtype=torch.float32, device="cuda:0")
    ctx.bmnd_stage(_cuda(y), _cuda(pilot), out, cfg["noise"], cfg["patch"], cfg["step"], cfg["search"],
                   cfg["group_size"][1], 2, 0, bm.params(cov_planes=4))
    got = out.cpu().numpy()
    PT.assert_voxels(got, ref, 1.0, what=name)
    assert abs(PT.psnr(got, x) - PT.psnr(ref, x)) <= PT.PSNR_DB


def test_shared_source_dct_group_transform(ctx, oracle):
    import torch
    import paper_2609_34622_b300.bmnd as bm
    name, y, x, cfg = POISSON[-1]
    ref = oracle.stage(_op(oracle, y, cfg, cov_planes=4, group_transform="dct"), y, None, 1)
    out = torch.empty(y.shape, dtype=torch.float32, device="cuda:0")
    ctx.bmnd_stage(_cuda(y), None, out, cfg["noise"], cfg["patch"], cfg["step"], cfg["search"],
                   cfg["group_size"][0], 1, 0, bm.params(cov_planes=4, group_transform="dct"))
    PT.assert_voxels(out.cpu().numpy(), ref, 1.0, what=name)


def test_shared_source_rejections(ctx):
    import torch
    import paper_2609_34622_b300.bmnd as bm
    y = torch.zeros((32, 32), device="cuda:0")
    with pytest.raises(bm.BmndError):
        ctx.bmnd_denoise(y, torch.empty_like(y), ("gaussian", 0.1), (8, 8), (3, 3), (9, 9),
                         prm=bm.params(cov_planes=4))
    with pytest.raises(bm.BmndError):
        ctx.bmnd_denoise(y, torch.empty_like(y), ("poisson", 0.1), (8, 8), (3, 3), (9, 9),
                         prm=bm.params(cov_planes=33))
