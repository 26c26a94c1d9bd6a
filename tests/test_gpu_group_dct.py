"""Parity of the DCT along the group axis and of the group-scope aggregation
weights (Sec. 5, Def. "Separable group transform", with the weight scopes of
the aggregation) of the CUDA path with the oracle, through the C ABI, on the
parity cases of the default profile.  With the DCT the group sizes are not
rounded to powers of two, so these cases also run groups of every size."""
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
                         **kw)


PROFILES = {
    "dct": dict(group_transform="dct"),
    "dct-group-scope": dict(group_transform="dct", weight_scope="group"),
    "haar-group-scope": dict(weight_scope="group"),
}


@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
@pytest.mark.parametrize("prof", list(PROFILES), ids=list(PROFILES))
def test_stage1_parity(ctx, oracle, case, prof):
    import torch
    import paper_2609_34622_b300.bmnd as bm
    name, y, x, cfg = case
    kw = PROFILES[prof]
    ref = oracle.stage(_op(oracle, y, cfg, **kw), y, None, 1)
    out = torch.empty(y.shape, dtype=torch.float32, device="cuda:0")
    ctx.bmnd_stage(_cuda(y), None, out, cfg["noise"], cfg["patch"], cfg["step"], cfg["search"],
                   cfg["group_size"][0], 1, 0, bm.params(**kw))
    got = out.cpu().numpy()
    PT.assert_voxels(got, ref, 1.0, what=name)
    assert abs(PT.psnr(got, x) - PT.psnr(ref, x)) <= PT.PSNR_DB


@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
@pytest.mark.parametrize("prof", list(PROFILES), ids=list(PROFILES))
def test_stage2_parity_same_pilot(ctx, oracle, case, prof):
    import torch
    import paper_2609_34622_b300.bmnd as bm
    name, y, x, cfg = case
    kw = PROFILES[prof]
    p = _op(oracle, y, cfg, **kw)
    pilot = oracle.stage(p, y, None, 1).astype(np.float32)
    ref = oracle.stage(p, y, pilot.astype(np.float64), 2)
    out = torch.empty(y.shape, dtype=torch.float32, device="cuda:0")
    ctx.bmnd_stage(_cuda(y), _cuda(pilot), out, cfg["noise"], cfg["patch"], cfg["step"], cfg["search"],
                   cfg["group_size"][1], 2, 0, bm.params(**kw))
    got = out.cpu().numpy()
    PT.assert_voxels(got, ref, 1.0, what=name)
    assert abs(PT.psnr(got, x) - PT.psnr(ref, x)) <= PT.PSNR_DB


@pytest.mark.parametrize("case", CASES[1:4], ids=[c[0] for c in CASES[1:4]])
@pytest.mark.parametrize("mc", [0, 3])
def test_denoise_group_dct_end_to_end(ctx, oracle, case, mc):
    import torch
    import paper_2609_34622_b300.bmnd as bm
    name, y, x, cfg = case
    kw = PROFILES["dct"]
    ref = PT.oracle_two_stages_f32_pilot(oracle, _op(oracle, y, cfg, mc, **kw), y)
    out = torch.empty(y.shape, dtype=torch.float32, device="cuda:0")
    ctx.bmnd_denoise(_cuda(y), out, cfg["noise"], cfg["patch"], cfg["step"], cfg["search"], cfg["group_size"], 2,
                     mc, bm.params(**kw))
    got = out.cpu().numpy()
    PT.assert_voxels(got, ref, 1.0, what=name)
    if mc == 3:
        assert float(got.astype(np.float64).sum()) == pytest.approx(float(y.astype(np.float64).sum()), rel=1e-4)
