"""Parity of the Poisson-aware stage-1 matching (Secs. 4.2-4.3) of the CUDA
path with the oracle: the three distances (deviance, Pearson, Anscombe-SSD)
under the three acceptance policies (fixed, reference finite-count,
candidate-standardized), through the C ABI.

The oracle scores in double precision from its own closed forms (libm's
logarithm) with exact sums; on count data the kernels sum fixed-point table
values exactly, so groups must agree except at near-ties of the oracle's
scores (in practice everywhere); the stage outputs then follow the voxel
contract of the SSD path."""
import numpy as np
import pytest

from paper_2609_34622_b300 import synth
from tests import parity as PT

pytestmark = pytest.mark.gpu

METRICS = ("poisson_deviance", "pearson", "anscombe_ssd")
POLICIES = ("fixed", "reference_finite_count", "candidate_standardized")


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
    rng = np.random.default_rng(31)
    x = synth.ecg_signal(3001, 250.0, rng)
    y, sp = synth.poisson_observe(x, 20.0, rng)
    cases.append(("1d-3001", y, x, dict(noise=("poisson", sp), patch=(16,), step=(4,), search=(41,),
                                        group_size=(16, 32))))
    rng = np.random.default_rng(32)
    x = synth.disc_rect_image((40, 37), rng)
    y, sp = synth.poisson_observe(x, 8.0, rng)
    cases.append(("2d-40x37", y, x, dict(noise=("poisson", sp), patch=(6, 5), step=(3, 2), search=(9, 11),
                                         group_size=(8, 16))))
    rng = np.random.default_rng(33)
    lam = synth.ellipsoid_phantom((17, 15, 13), rng)
    x = lam / lam.max()
    y, sp = synth.poisson_observe(x, 4.0, rng)
    cases.append(("3d-17x15x13", y, x, dict(noise=("poisson", sp), patch=(3, 3, 3), step=(2, 2, 2),
                                            search=(5, 5, 5), group_size=(8, 16))))
    return cases


CASES = _cases()


def _scorer(oracle, y, cfg, metric, policy, t, beta=0.1, kappa=1.0):
    """FP64 candidate scores and threshold of one reference (near-tie
    classification of tests/parity.py)."""
    s_p = cfg["noise"][1]
    return lambda ref: PT.poisson_candidate_scores(y.astype(np.float64), ref, cfg["patch"], cfg["search"], s_p,
                                                   metric, policy, lambda n: oracle.moments(metric, n), t, beta,
                                                   kappa)


def _params(metric, policy, t):
    import paper_2609_34622_b300.bmnd as bm
    return bm.params(match_metric=metric, match_policy=policy, match_t=t)


def _oparams(oracle, y, cfg, metric, policy, t):
    return oracle.params(y.shape, cfg["patch"], cfg["step"], cfg["search"], cfg["noise"], cfg["group_size"],
                         2, 0, match_metric=metric, match_policy=policy, match_t=t)


@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
@pytest.mark.parametrize("policy", POLICIES)
@pytest.mark.parametrize("metric", METRICS)
def test_groups_identical(ctx, oracle, case, metric, policy):
    name, y, x, cfg = case
    t = 1.0
    p = _oparams(oracle, y, cfg, metric, policy, t)
    _, _, og, oc = oracle.stage(p, y, None, 1, want_den=True, want_groups=True)
    oo = oracle.schedule(p)
    M = cfg["group_size"][0]
    o, g, c = ctx.bmnd_match(_cuda(y), cfg["noise"], cfg["patch"], cfg["step"], cfg["search"], M, 1,
                             _params(metric, policy, t))
    o, g, c = o.cpu().numpy(), g.cpu().numpy(), c.cpu().numpy()
    order = np.argsort(o)
    o, g, c = o[order], g[order], c[order]
    scorer = _scorer(oracle, y, cfg, metric, policy, t)
    ne, nt, nb, bad = PT.group_agreement((o, g, c), (oo, og[:, :M], oc), y, cfg["patch"], cfg["search"],
                                         cfg["noise"], 0.0, 0.0, max_explain=len(oo), scorer=scorer,
                                         rel=PT.POISSON_TIE_REL, tol=PT.POISSON_TIE_REL)
    sizes = np.bincount(c, minlength=M + 1)
    print("%s %s/%s: %d groups (%d exact, %d near-tie), sizes %s" % (name, metric, policy, len(oo), ne, nt,
                                                                     sizes.tolist()))
    # the contract: identical except at ties of the FP64 scores to 1e-8:
    # ties in real arithmetic between different multisets of contributions
    # (e.g. phi(2, 0) = 2 phi(1, 0) for the deviance, 1/3 + 1/3 + 1/3 = 1 for
    # Pearson) are decided by rounding on either side.  Counts of 0..4 per
    # entry (the 3-D case) make them frequent.
    assert nb == 0, bad
    assert ne >= (0.5 if len(y.shape) == 3 else 0.95) * len(oo)


@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
@pytest.mark.parametrize("metric,policy", [("poisson_deviance", "reference_finite_count"),
                                           ("pearson", "candidate_standardized"), ("anscombe_ssd", "fixed")])
def test_stage1_parity(ctx, oracle, case, metric, policy):
    import torch
    name, y, x, cfg = case
    p = _oparams(oracle, y, cfg, metric, policy, 3.0)
    out = torch.empty(y.shape, dtype=torch.float32, device="cuda:0")
    prm = _params(metric, policy, 3.0)
    ctx.bmnd_stage(_cuda(y), None, out, cfg["noise"], cfg["patch"], cfg["step"], cfg["search"],
                   cfg["group_size"][0], 1, 0, prm)
    frac, ndiff = PT.stage1_poisson_contract(ctx, oracle, p, y, x, cfg, out.cpu().numpy(), _cuda, prm,
                                             _scorer(oracle, y, cfg, metric, policy, 3.0), name)
    print("%s: %d near-tie groups, %.4f of voxels compared" % (name, ndiff, frac))
    assert frac >= (0.2 if len(y.shape) == 3 else 0.9)


@pytest.mark.parametrize("case", CASES[:2], ids=[c[0] for c in CASES[:2]])
@pytest.mark.parametrize("mc", [0, 3])
def test_denoise_end_to_end(ctx, oracle, case, mc):
    """Both stages with the paper's finite-count configuration (deviance,
    reference finite-count, beta_s = 0.1, kappa_s = 1), with and without mass
    conservation."""
    import torch
    name, y, x, cfg = case
    p = oracle.params(y.shape, cfg["patch"], cfg["step"], cfg["search"], cfg["noise"], cfg["group_size"], 2, mc,
                      match_metric="poisson_deviance", match_policy="reference_finite_count")
    import paper_2609_34622_b300.bmnd as bm
    prm = bm.params(match_metric="poisson_deviance", match_policy="reference_finite_count")
    out = torch.empty(y.shape, dtype=torch.float32, device="cuda:0")
    ctx.bmnd_denoise(_cuda(y), out, cfg["noise"], cfg["patch"], cfg["step"], cfg["search"], cfg["group_size"], 2,
                     mc, prm)
    got = out.cpu().numpy()
    frac = PT.two_stage_poisson_contract(ctx, oracle, p, y, x, cfg, got, _cuda, prm,
                                         _scorer(oracle, y, cfg, "poisson_deviance", "reference_finite_count", 3.0),
                                         name)
    print("%s mc %d: %.4f of voxels compared" % (name, mc, frac))
    assert frac >= 0.3
    if mc == 3:
        assert float(got.astype(np.float64).sum()) == pytest.approx(float(y.astype(np.float64).sum()), rel=1e-4)


@pytest.mark.parametrize("kappa", [0.5, 2.0])
def test_structural_allowance_exponents(ctx, oracle, kappa):
    """Eq. (reference-threshold) with kappa_s off 1 (the sensitivity grid of
    Sec. 9.4) and a large beta_s, so that the allowance decides groups."""
    name, y, x, cfg = CASES[1]
    p = oracle.params(y.shape, cfg["patch"], cfg["step"], cfg["search"], cfg["noise"], cfg["group_size"], 2, 0,
                      match_metric="pearson", match_policy="reference_finite_count", match_t=0.5, beta_s=0.8,
                      kappa_s=kappa)
    _, _, og, oc = oracle.stage(p, y, None, 1, want_den=True, want_groups=True)
    import paper_2609_34622_b300.bmnd as bm
    prm = bm.params(match_metric="pearson", match_policy="reference_finite_count", match_t=0.5, beta_s=0.8,
                    kappa_s=kappa)
    M = cfg["group_size"][0]
    o, g, c = ctx.bmnd_match(_cuda(y), cfg["noise"], cfg["patch"], cfg["step"], cfg["search"], M, 1, prm)
    o = o.cpu().numpy()
    order = np.argsort(o)
    o, c, g = o[order], c.cpu().numpy()[order], g.cpu().numpy()[order]
    oo = oracle.schedule(p)
    scorer = _scorer(oracle, y, cfg, "pearson", "reference_finite_count", 0.5, 0.8, kappa)
    ne, nt, nb, bad = PT.group_agreement((o, g, c), (oo, og[:, :M], oc), y, cfg["patch"], cfg["search"],
                                         cfg["noise"], 0.0, 0.0, max_explain=len(oo), scorer=scorer,
                                         rel=PT.POISSON_TIE_REL, tol=PT.POISSON_TIE_REL)
    assert nb == 0, bad
    assert ne >= 0.95 * len(oo)


def test_full_size_1d_sampled(ctx, oracle):
    """The 1-D workload at full size (262144 samples) with the finite-count
    configuration, checked at sampled locations one by one."""
    import torch
    import paper_2609_34622_b300.bmnd as bm
    job = synth.config2()
    cfg = job.cfg
    p = oracle.params(job.y.shape, cfg["patch"], cfg["step"], cfg["search"], cfg["noise"], cfg["group_size"], 2, 0,
                      match_metric="poisson_deviance", match_policy="reference_finite_count")
    prm = bm.params(match_metric="poisson_deviance", match_policy="reference_finite_count")
    y = _cuda(job.y)
    pilot = torch.empty_like(y)
    ctx.bmnd_stage(y, None, pilot, cfg["noise"], cfg["patch"], cfg["step"], cfg["search"], 16, 1, 0, prm)
    rng = np.random.default_rng(62)
    pts = np.concatenate([[0, 1, 262143, 262112], rng.integers(0, 262144, 40)])
    r1 = oracle.stage_points(p, job.y, None, 1, pts)
    g1 = pilot.cpu().numpy().astype(np.float64)[pts]
    assert np.sum(np.abs(g1 - r1) > 1e-4) <= 1, np.abs(g1 - r1).max()


def test_rejections(ctx):
    import torch
    import paper_2609_34622_b300.bmnd as bm
    y = torch.zeros((32, 32), device="cuda:0")
    o = torch.empty_like(y)
    with pytest.raises(bm.BmndError):
        ctx.bmnd_denoise(y, o, ("gaussian", 0.1), (8, 8), (3, 3), (9, 9), prm=_params("pearson", "fixed", 3.0))
    with pytest.raises(bm.BmndError):
        ctx.bmnd_denoise(y, o, ("poisson", 0.1), (8, 8), (3, 3), (9, 9), prm=bm.params(match_metric=7))
    with pytest.raises(bm.BmndError):
        ctx.bmnd_denoise(y, o, ("poisson", 0.1), (8, 8), (3, 3), (9, 9),
                         prm=bm.params(match_metric="pearson", kappa_s=0.0))
