"""Parity with the FP64 oracle at the full configurations of the workloads,
through the C ABI: the 2-D batch's 39x39 search window (128x128 crops of its
images of each noise type, element by element, and sampled locations of
whole 512x512 images), and the 3-D volume's 11^3 window with mass
conservation in both stages (a 40^3 crop element by element, sampled
locations of the whole 128^3 volume)."""
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


@pytest.fixture(scope="module")
def batch():
    return synth.config3()


# image 0: Poisson peak 1 (dyadic data, exact FP32 tiles); 2: peak 5; 16: Gaussian
CROPS = [0, 2, 16]


def _crop(job, lo=128, n=128):
    sl = tuple(slice(lo, lo + n) for _ in range(job.y.ndim))
    return np.ascontiguousarray(job.y[sl]), np.ascontiguousarray(job.x[sl])


@pytest.mark.parametrize("idx", CROPS)
def test_batch_crop_stage1(ctx, oracle, batch, idx):
    """Stage 1 at search 39x39: groups identical except at near-ties, every
    voxel under the voxel contract, PSNR within 0.01 dB."""
    import torch
    job = batch[idx]
    y, x = _crop(job)
    cfg = job.cfg
    p = oracle.params(y.shape, cfg["patch"], cfg["step"], cfg["search"], cfg["noise"], cfg["group_size"], 2, 0)
    ref, _, og, oc = oracle.stage(p, y, None, 1, want_den=True, want_groups=True)
    gpu = PT.groups_of(ctx, _cuda(y), cfg, 1)
    oo = oracle.schedule(p)
    P = int(np.prod(cfg["patch"]))
    ne, nt, nb, bad = PT.group_agreement(gpu, (oo, og[:, :16], oc), y.astype(np.float64), cfg["patch"],
                                         cfg["search"], cfg["noise"], 3.0, 3000.0 * P / 255.0 ** 2,
                                         max_explain=len(oo))
    assert nb == 0, bad
    assert ne == len(oo)
    out = torch.empty(y.shape, dtype=torch.float32, device="cuda:0")
    ctx.bmnd_stage(_cuda(y), None, out, cfg["noise"], cfg["patch"], cfg["step"], cfg["search"], 16, 1)
    got = out.cpu().numpy()
    PT.assert_voxels(got, ref, 1.0, what=job.name)
    assert abs(PT.psnr(got, x) - PT.psnr(ref, x)) <= PT.PSNR_DB


@pytest.mark.parametrize("idx", CROPS)
def test_batch_crop_both_stages(ctx, oracle, batch, idx):
    import torch
    job = batch[idx]
    y, x = _crop(job)
    cfg = job.cfg
    p = oracle.params(y.shape, cfg["patch"], cfg["step"], cfg["search"], cfg["noise"], cfg["group_size"], 2, 0)
    out = torch.empty(y.shape, dtype=torch.float32, device="cuda:0")
    ctx.bmnd_denoise(_cuda(y), out, cfg["noise"], cfg["patch"], cfg["step"], cfg["search"], cfg["group_size"], 2, 0)
    frac = PT.two_stage_contract(ctx, oracle, p, y, x, cfg, out.cpu().numpy(), _cuda, what=job.name)
    print("%s: %.4f of voxels compared" % (job.name, frac))
    assert frac >= 0.9


@pytest.mark.parametrize("idx", [3, 19])
def test_batch_whole_image_sampled(ctx, oracle, batch, idx):
    """Stage 1 on a whole 512x512 image of the batch in the batched launch
    the benchmark times (all 32 images), at 24 locations (corners, edges,
    random) evaluated one by one by the oracle."""
    import torch
    import paper_2609_34622_b300.bmnd as bm
    ys = [_cuda(j.y) for j in batch]
    outs = [torch.empty_like(y) for y in ys]
    cfgs = [dict(j.cfg, stages=1) for j in batch]
    ctx.bmnd_denoise_batch(ys, outs, cfgs)
    job = batch[idx]
    cfg = job.cfg
    p = oracle.params(job.y.shape, cfg["patch"], cfg["step"], cfg["search"], cfg["noise"], cfg["group_size"], 1, 0)
    rng = np.random.default_rng(80 + idx)
    pts = np.concatenate([[0, 511, 511 * 512, 512 * 512 - 1, 255 * 512 + 256, 3, 512 * 7],
                          rng.integers(0, 512 * 512, 17)])
    ref = oracle.stage_points(p, job.y, None, 1, pts)
    got = outs[idx].cpu().numpy().ravel()[pts].astype(np.float64)
    np.testing.assert_allclose(got, ref, atol=PT.VOXEL_ABS, rtol=0)


@pytest.fixture(scope="module")
def volume():
    return synth.config4()


def test_volume_crop_mass_conservation(ctx, oracle, volume):
    """A 40^3 crop of the 3-D volume with its parameters (patch 4^3, step 2,
    search 11^3, mass conservation in both stages): stage 1 with its two
    sweeps under the voxel contract; both stages under the two-stage
    contract; the output sums to the input's sum."""
    import torch
    y, x = _crop(volume, 44, 40)
    cfg = volume.cfg
    p = oracle.params(y.shape, cfg["patch"], cfg["step"], cfg["search"], cfg["noise"], cfg["group_size"], 2, 3)
    ref1 = oracle.stage(p, y, None, 1)
    out1 = torch.empty(y.shape, dtype=torch.float32, device="cuda:0")
    ctx.bmnd_stage(_cuda(y), None, out1, cfg["noise"], cfg["patch"], cfg["step"], cfg["search"], 16, 1, 1)
    got1 = out1.cpu().numpy()
    PT.assert_voxels(got1, ref1, 1.0, what="stage 1 mc")
    out = torch.empty(y.shape, dtype=torch.float32, device="cuda:0")
    ctx.bmnd_denoise(_cuda(y), out, cfg["noise"], cfg["patch"], cfg["step"], cfg["search"], cfg["group_size"], 2, 3)
    got = out.cpu().numpy()
    assert float(got.astype(np.float64).sum()) == pytest.approx(float(y.astype(np.float64).sum()), rel=1e-5)
    frac = PT.two_stage_contract(ctx, oracle, p, y, x, cfg, got, _cuda, what="40^3 mc")
    print("40^3 both stages: %.4f of voxels compared" % frac)
    # stage-2 matching on the flat low-count pilot has many near-ties (the
    # contract checks they are near-ties), and mass conservation spreads each
    # one over the patches its corrections reach
    assert frac >= 0.3


def test_volume_whole_sampled(ctx, oracle, volume):
    """Stage 1 (no mass conservation: the oracle's point evaluation has none)
    on the whole 128^3 volume at 12 locations evaluated one by one."""
    import torch
    cfg = volume.cfg
    y = volume.y
    out = torch.empty(y.shape, dtype=torch.float32, device="cuda:0")
    ctx.bmnd_stage(_cuda(y), None, out, cfg["noise"], cfg["patch"], cfg["step"], cfg["search"], 16, 1, 0)
    p = oracle.params(y.shape, cfg["patch"], cfg["step"], cfg["search"], cfg["noise"], cfg["group_size"], 1, 0)
    rng = np.random.default_rng(90)
    n = 128 ** 3
    pts = np.concatenate([[0, n - 1, 64 * 128 * 128 + 64 * 128 + 64, 127], rng.integers(0, n, 8)])
    ref = oracle.stage_points(p, y, None, 1, pts)
    got = out.cpu().numpy().ravel()[pts].astype(np.float64)
    np.testing.assert_allclose(got, ref, atol=PT.VOXEL_ABS, rtol=0)
