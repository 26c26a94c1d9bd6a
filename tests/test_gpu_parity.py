"""Parity of the CUDA path (through the C ABI) with the FP64 oracle."""
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


def _small_cases():
    """(name, y, x, cfg) with shapes spanning several tiles and ragged tails."""
    cases = []
    j1 = synth.config1()
    cases.append(("c1-2d-64", j1.y, j1.x, j1.cfg))
    rng = np.random.default_rng(11)
    x = synth.ecg_signal(5000, 250.0, rng)
    y, sp = synth.poisson_observe(x, 50.0, rng)
    cases.append(("1d-5000", y, x, dict(noise=("poisson", sp), patch=(32,), step=(4,), search=(129,),
                                        group_size=(16, 32), stages=2, mass_conserve=0)))
    rng = np.random.default_rng(12)
    lam = synth.ellipsoid_phantom((22, 19, 17), rng)
    x = lam / lam.max()
    y, sp = synth.poisson_observe(x, 5.0, rng)
    cases.append(("3d-22x19x17", y, x, dict(noise=("poisson", sp), patch=(4, 4, 4), step=(2, 2, 2),
                                            search=(7, 7, 7), group_size=(16, 32), stages=2, mass_conserve=0)))
    rng = np.random.default_rng(13)
    x = synth.texture_edge_image((53, 71), rng)
    cases.append(("2d-gauss-53x71", synth.gaussian_observe(x, 25 / 255, rng), x,
                  dict(noise=("gaussian", 25 / 255), patch=(8, 8), step=(3, 3), search=(15, 15),
                       group_size=(16, 32), stages=2, mass_conserve=0)))
    rng = np.random.default_rng(14)
    x = synth.disc_rect_image((37, 29), rng)
    y, sp = synth.poisson_observe(x, 20.0, rng)
    cases.append(("2d-ragged-5x4", y, x, dict(noise=("poisson", sp), patch=(5, 4), step=(3, 2), search=(9, 7),
                                              group_size=(8, 16), stages=2, mass_conserve=0)))
    return cases


CASES = _small_cases()


def _oparams(oracle, y, cfg, **kw):
    return oracle.params(y.shape, cfg["patch"], cfg["step"], cfg["search"], cfg["noise"], cfg["group_size"],
                         cfg.get("stages", 2), cfg.get("mass_conserve", 0), **kw)


@pytest.mark.parametrize("shape,patch,step,sched", [
    ((64, 64), (8, 8), (3, 3), "generated"), ((262144,), (32,), (4,), "generated"),
    ((40, 33, 29), (4, 4, 4), (2, 2, 2), "generated"), ((37, 29), (5, 4), (3, 2), "balanced"),
    ((1, 40, 17), (1, 6, 5), (1, 4, 3), "sparse"), ((23, 31), (6, 6), (4, 5), "off"),
    ((300, 1), (16, 1), (4, 1), "generated"), ((9, 7, 5, 6), (3, 2, 2, 3), (2, 1, 2, 2), "generated")])
def test_schedule_bit_exact(ctx, oracle, shape, patch, step, sched):
    import paper_2609_34622_b300.bmnd as bm
    got = np.sort(ctx.bmnd_schedule(shape, patch, step, bm.params(schedule=sched)).cpu().numpy())
    p = oracle.params(shape, patch, step, (1,) * len(shape), schedule=sched)
    np.testing.assert_array_equal(got, oracle.schedule(p))


def _gpu_groups(ctx, guide, cfg, stage, prm=None):
    M = cfg["group_size"][stage - 1]
    o, g, c = ctx.bmnd_match(_cuda(guide), cfg["noise"], cfg["patch"], cfg["step"], cfg["search"], M, stage, prm)
    o, g, c = o.cpu().numpy(), g.cpu().numpy(), c.cpu().numpy()
    order = np.argsort(o)
    return o[order], g[order], c[order]


@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
@pytest.mark.parametrize("stage", [1, 2])
def test_group_membership(ctx, oracle, case, stage):
    name, y, x, cfg = case
    p = _oparams(oracle, y, cfg)
    guide = y.astype(np.float64)
    if stage == 2:
        _, pilot = oracle.denoise(p, y)
        guide = pilot.astype(np.float32).astype(np.float64)
        _, _, og, oc = oracle.stage(p, y, guide, 2, want_den=True, want_groups=True)
    else:
        _, _, og, oc = oracle.stage(p, y, None, 1, want_den=True, want_groups=True)
    oo = oracle.schedule(p)
    gpu = _gpu_groups(ctx, guide.astype(np.float32), cfg, stage)
    M = cfg["group_size"][stage - 1]
    gamma = 3.0 if stage == 1 else 0.0
    P = int(np.prod(cfg["patch"]))
    tau = (3000.0 if stage == 1 else 400.0) * P / 255.0 ** 2
    ne, nt, nb, bad = PT.group_agreement(gpu, (oo, og[:, :M], oc), guide.reshape(y.shape), cfg["patch"],
                                         cfg["search"], cfg["noise"], gamma, tau)
    print("%s stage %d: %d exact, %d near-tie, %d unexplained of %d" % (name, stage, ne, nt, nb, len(oo)))
    # the contract: identical except at near-ties of the FP64 scores.  The
    # kernels re-take in double precision every decision their FP32 error
    # bound cannot separate, so in practice every group is identical
    assert nb == 0, bad
    assert ne == len(oo), "%d of %d groups differ at near-ties" % (len(oo) - ne, len(oo))


@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_stage1_parity(ctx, oracle, case):
    import torch
    name, y, x, cfg = case
    p = _oparams(oracle, y, cfg)
    ref = oracle.stage(p, y, None, 1)
    out = torch.empty(y.shape, dtype=torch.float32, device="cuda:0")
    ctx.bmnd_stage(_cuda(y), None, out, cfg["noise"], cfg["patch"], cfg["step"], cfg["search"],
                   cfg["group_size"][0], 1)
    got = out.cpu().numpy()
    frac, dmax = PT.assert_voxels(got, ref, 1.0, what=name)
    assert abs(PT.psnr(got, x) - PT.psnr(ref, x)) <= PT.PSNR_DB
    print("%s stage 1: %.5f within 1e-4, max diff %.3g" % (name, frac, dmax))


@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_stage2_parity_same_pilot(ctx, oracle, case):
    import torch
    name, y, x, cfg = case
    p = _oparams(oracle, y, cfg)
    pilot = oracle.stage(p, y, None, 1).astype(np.float32)
    ref = oracle.stage(p, y, pilot.astype(np.float64), 2)
    out = torch.empty(y.shape, dtype=torch.float32, device="cuda:0")
    ctx.bmnd_stage(_cuda(y), _cuda(pilot), out, cfg["noise"], cfg["patch"], cfg["step"], cfg["search"],
                   cfg["group_size"][1], 2)
    got = out.cpu().numpy()
    frac, dmax = PT.assert_voxels(got, ref, 1.0, what=name)
    assert abs(PT.psnr(got, x) - PT.psnr(ref, x)) <= PT.PSNR_DB


@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_denoise_end_to_end(ctx, oracle, case):
    """Both stages, under the end-to-end contract of tests/parity.py: stage-2
    groups identical except at near-ties, the voxel contract outside the
    patches of the groups that differ, PSNR within 0.01 dB."""
    import torch
    name, y, x, cfg = case
    p = _oparams(oracle, y, cfg)
    out = torch.empty(y.shape, dtype=torch.float32, device="cuda:0")
    ctx.bmnd_denoise(_cuda(y), out, cfg["noise"], cfg["patch"], cfg["step"], cfg["search"], cfg["group_size"], 2, 0)
    frac_cmp, within = PT.end_to_end_contract(ctx, oracle, p, y, x, cfg, out.cpu().numpy(), _cuda, what=name)
    print("%s: %.4f of voxels compared, %.5f of them within 1e-4" % (name, frac_cmp, within))
    # near-ties of stage 2 leave most of the array under the voxel contract
    assert frac_cmp >= 0.5


@pytest.mark.parametrize("mc", [1, 2, 3])
def test_mass_conservation_parity(ctx, oracle, mc):
    import torch
    rng = np.random.default_rng(21)
    lam = synth.ellipsoid_phantom((20, 18, 21), rng, 0.05, 0.5)
    x = lam / lam.max()
    y, sp = synth.poisson_observe(x, 0.5 / 1.0 * 2, rng)
    cfg = dict(noise=("poisson", sp), patch=(4, 4, 4), step=(2, 2, 2), search=(7, 7, 7), group_size=(16, 32))
    p = oracle.params(y.shape, cfg["patch"], cfg["step"], cfg["search"], cfg["noise"], cfg["group_size"], 2, mc)
    ref = PT.oracle_two_stages_f32_pilot(oracle, p, y)
    out = torch.empty(y.shape, dtype=torch.float32, device="cuda:0")
    ctx.bmnd_denoise(_cuda(y), out, cfg["noise"], cfg["patch"], cfg["step"], cfg["search"], cfg["group_size"], 2, mc)
    got = out.cpu().numpy()
    PT.assert_voxels(got, ref, 1.0, what="mc%d" % mc)
    if mc & 2:
        assert got.astype(np.float64).sum() == pytest.approx(y.astype(np.float64).sum(), rel=1e-5)


def test_determinism_and_batch_equals_single(ctx):
    import torch
    jobs = [synth.config1()]
    rng = np.random.default_rng(31)
    for s in [(50, 61), (64, 64), (33, 90)]:
        x = synth.disc_rect_image(s, rng)
        y, sp = synth.poisson_observe(x, 10.0, rng)
        jobs.append(synth.Job(y, x, ("poisson", sp), (8, 8), (3, 3), (19, 19)))
    ys = [_cuda(j.y) for j in jobs]
    singles = []
    for j, y in zip(jobs, ys):
        o = torch.empty_like(y)
        ctx.bmnd_denoise(y, o, j.noise, j.patch, j.step, j.search, j.group_size, 2, 0)
        singles.append(o.cpu().numpy())
    o2 = torch.empty_like(ys[0])
    ctx.bmnd_denoise(ys[0], o2, jobs[0].noise, jobs[0].patch, jobs[0].step, jobs[0].search, (16, 32), 2, 0)
    np.testing.assert_array_equal(o2.cpu().numpy(), singles[0])
    outs = [torch.empty_like(y) for y in ys]
    ctx.bmnd_denoise_batch(ys, outs, [j.cfg for j in jobs])
    for a, b in zip(outs, singles):
        np.testing.assert_array_equal(a.cpu().numpy(), b)


def test_identity_zero_noise(ctx):
    import paper_2609_34622_b300.bmnd as bm
    import torch
    rng = np.random.default_rng(41)
    y = rng.uniform(0, 1, size=(40, 36)).astype(np.float32)
    out = torch.empty(y.shape, dtype=torch.float32, device="cuda:0")
    ctx.bmnd_denoise(_cuda(y), out, ("gaussian", 0.0), (4, 4), (2, 2), (7, 7), (8, 16), 2, 0,
                     bm.params(lambda_ht=0.0))
    np.testing.assert_allclose(out.cpu().numpy(), y, atol=2e-6)


def test_edge_shapes(ctx, oracle):
    """Patch equal to the array, singleton axes, search 1, group size 1."""
    import torch
    rng = np.random.default_rng(51)
    for shape, patch, step, search, gs in [((8, 8), (8, 8), (3, 3), (19, 19), (16, 32)),
                                           ((1, 300), (1, 16), (1, 4), (1, 33), (16, 32)),
                                           ((300, 1), (16, 1), (4, 1), (33, 1), (16, 32)),
                                           ((30, 30), (4, 4), (2, 2), (1, 1), (16, 32)),
                                           ((30, 30), (4, 4), (2, 2), (5, 5), (1, 1)),
                                           ((17,), (17,), (1,), (3,), (2, 2))]:
        x = rng.uniform(0.2, 1.0, size=shape)
        y, sp = synth.poisson_observe(x, 20.0, rng)
        cfg = dict(noise=("poisson", sp), patch=patch, step=step, search=search, group_size=gs)
        p = oracle.params(shape, patch, step, search, cfg["noise"], gs, 2, 0)
        ref, _ = oracle.denoise(p, y)
        out = torch.empty(shape, dtype=torch.float32, device="cuda:0")
        ctx.bmnd_denoise(_cuda(y), out, cfg["noise"], patch, step, search, gs, 2, 0)
        PT.assert_voxels(out.cpu().numpy(), ref, 1.0, what=str(shape))


def test_invalid_arguments(ctx):
    import paper_2609_34622_b300.bmnd as bm
    import torch
    y = torch.zeros(16, 16, device="cuda:0")
    o = torch.zeros(16, 16, device="cuda:0")
    bad = [dict(patch=(8, 8), step=(3, 3), search=(18, 19)),   # even search
           dict(patch=(8, 8), step=(9, 3), search=(19, 19)),   # step > patch
           dict(patch=(17, 8), step=(3, 3), search=(19, 19)),  # patch > shape
           dict(patch=(8, 8), step=(3, 3), search=(19, 19), gs=(12, 32))]  # not a power of two
    for b in bad:
        with pytest.raises(bm.BmndError) as e:
            ctx.bmnd_denoise(y, o, ("poisson", 0.1), b["patch"], b["step"], b["search"], b.get("gs", (16, 32)))
        assert e.value.status == bm.EINVAL
    with pytest.raises(bm.BmndError):
        ctx.bmnd_denoise(y, y, ("poisson", 0.1), (8, 8), (3, 3), (19, 19))       # out aliases y
    with pytest.raises(bm.BmndError):
        ctx.bmnd_denoise(y, o, ("poisson", -1.0), (8, 8), (3, 3), (19, 19))      # bad scale


def test_full_size_1d_sampled(ctx, oracle):
    """The 1-D workload at its full size (262144 samples) in the benchmark's
    launch configuration, checked at sampled locations one by one."""
    import torch
    job = synth.config2()
    cfg = job.cfg
    p = _oparams(oracle, job.y, cfg)
    y = _cuda(job.y)
    pilot = torch.empty_like(y)
    out = torch.empty_like(y)
    ctx.bmnd_stage(y, None, pilot, cfg["noise"], cfg["patch"], cfg["step"], cfg["search"], 16, 1)
    ctx.bmnd_stage(y, pilot, out, cfg["noise"], cfg["patch"], cfg["step"], cfg["search"], 32, 2)
    full = torch.empty_like(y)
    ctx.bmnd_denoise(y, full, cfg["noise"], cfg["patch"], cfg["step"], cfg["search"], (16, 32), 2, 0)
    np.testing.assert_array_equal(full.cpu().numpy(), out.cpu().numpy())
    rng = np.random.default_rng(61)
    pts = np.concatenate([[0, 1, 2, 3, 262143, 262142, 262112, 262111], rng.integers(0, 262144, 2040)])
    pl = pilot.cpu().numpy().astype(np.float64)
    r1 = oracle.stage_points(p, job.y, None, 1, pts)
    r2 = oracle.stage_points(p, job.y, pl, 2, pts)
    g1 = pl[pts]
    g2 = out.cpu().numpy().astype(np.float64)[pts]
    # the voxel contract on the samples: at least 99.9 % within 1e-4
    PT.assert_voxels(g1, r1, 1.0, what="1-D stage 1 at %d samples" % len(pts))
    PT.assert_voxels(g2, r2, 1.0, what="1-D stage 2 at %d samples" % len(pts))


@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
@pytest.mark.parametrize("mode", ["noise_floor", "variance_scaled"])
def test_stage2_pilot_power_modes(ctx, oracle, case, mode):
    """Def. "Pilot-power modes": the Wiener gain with a = 1 (noise floor) and
    a = s_v (variance scaled), stage 2 on the same pilot, under the voxel
    contract."""
    import torch
    import paper_2609_34622_b300.bmnd as bm
    name, y, x, cfg = case
    p = _oparams(oracle, y, cfg, power_mode=mode)
    pilot = oracle.stage(p, y, None, 1).astype(np.float32)
    ref = oracle.stage(p, y, pilot.astype(np.float64), 2)
    out = torch.empty(y.shape, dtype=torch.float32, device="cuda:0")
    ctx.bmnd_stage(_cuda(y), _cuda(pilot), out, cfg["noise"], cfg["patch"], cfg["step"], cfg["search"],
                   cfg["group_size"][1], 2, 0, bm.params(power_mode=mode))
    got = out.cpu().numpy()
    PT.assert_voxels(got, ref, 1.0, what="%s %s" % (name, mode))
    assert abs(PT.psnr(got, x) - PT.psnr(ref, x)) <= PT.PSNR_DB
