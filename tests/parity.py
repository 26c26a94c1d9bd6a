"""Comparison helpers shared by the GPU parity tests (test code only)."""
from __future__ import annotations

import itertools

import numpy as np

# Tolerances of the parity contract: group membership identical except at
# near-ties (scores closer than 1e-5 relative to their magnitude), >= 99.9%
# of output voxels within 1e-4 of the peak intensity, PSNR within 0.01 dB.
NEAR_TIE_REL = 1e-5
# Poisson distances on count data: the kernels' integer sums of fixed-point
# table values are within P 2^-33 of the exact sums, so a near-tie there is
# a difference below 1e-8 (|score| + 1): in practice a tie in real
# arithmetic between different multisets of contributions
POISSON_TIE_REL = 1e-8
VOXEL_ABS = 1e-4
VOXEL_FRAC = 0.999
PSNR_DB = 0.01


def voxel_report(got, ref, peak=1.0):
    d = np.abs(np.asarray(got, np.float64) - np.asarray(ref, np.float64))
    frac = float(np.mean(d <= VOXEL_ABS * peak))
    return frac, float(d.max())


def psnr(x, ref, peak=1.0):
    mse = float(np.mean((np.asarray(x, np.float64) - np.asarray(ref, np.float64)) ** 2))
    return 10 * np.log10(peak * peak / mse)


def assert_voxels(got, ref, peak=1.0, frac_min=VOXEL_FRAC, what=""):
    frac, dmax = voxel_report(got, ref, peak)
    assert frac >= frac_min, "%s: only %.5f of voxels within %g (max diff %g)" % (what, frac, VOXEL_ABS * peak, dmax)
    return frac, dmax


def candidate_scores(guide, ref_lin, patch, search, noise, gamma):
    """FP64 scores (d_SSD - gamma B) and magnitudes (d_SSD + gamma B) of every
    candidate in the clipped window of one reference (independent numpy)."""
    g = np.asarray(guide, np.float64)
    shape = g.shape
    ref = np.unravel_index(int(ref_lin), shape)
    ell = [L - j for L, j in zip(shape, patch)]
    rad = [(w - 1) // 2 for w in search]
    pref = g[tuple(slice(r, r + j) for r, j in zip(ref, patch))]
    P = pref.size
    out = {}
    ranges = [range(max(r - a, 0), min(r + a, e) + 1) for r, a, e in zip(ref, rad, ell)]
    for c in itertools.product(*ranges):
        q = g[tuple(slice(a, a + j) for a, j in zip(c, patch))]
        ssd = float(((q - pref) ** 2).sum())
        if noise[0] == "poisson":
            B = noise[1] * float(np.maximum(q + pref, 0).sum())
        else:
            B = 2 * P * noise[1] ** 2
        sc = ssd - gamma * B if gamma > 0 else ssd
        out[int(np.ravel_multi_index(c, shape))] = (sc, ssd + gamma * B + 1e-30)
    return out


def raw_counts(guide, s_p):
    """Eq. (raw-counts) with the integer reading of the oracle: y / s_P, the
    nearest integer when within a relative 2^-20 of it."""
    r = np.maximum(np.asarray(guide, np.float64) / s_p, 0.0)
    k = np.rint(r)
    return np.where(np.abs(r - k) <= np.ldexp(np.maximum(k, 1.0), -20), k, r)


def poisson_phi(metric, r, c):
    """phi_m(r, c) of Eq. (varphi) in FP64 (numpy, elementwise)."""
    r = np.asarray(r, np.float64)
    c = np.asarray(c, np.float64)
    n = r + c
    if metric == "poisson_deviance":
        with np.errstate(divide="ignore", invalid="ignore"):
            a = np.where(r > 0, r * np.log(np.where(r > 0, 2 * r, 1) / np.where(n > 0, n, 1)), 0.0)
            b = np.where(c > 0, c * np.log(np.where(c > 0, 2 * c, 1) / np.where(n > 0, n, 1)), 0.0)
        return np.where(n > 0, 2 * (a + b), 0.0)
    if metric == "pearson":
        return np.where(n > 0, (r - c) ** 2 / np.where(n > 0, n, 1), 0.0)
    d = 2 * np.sqrt(c + 0.375) - 2 * np.sqrt(r + 0.375)
    return 0.5 * d * d


def poisson_candidate_scores(guide, ref_lin, patch, search, s_p, metric, policy, moments, t=1.0, beta=0.1,
                             kappa=1.0, tau_fixed=None):
    """FP64 scores and magnitudes of every candidate of one reference under a
    Poisson distance (Sec. 4.2-4.3), and the acceptance threshold; moments(n)
    gives (mu, v) at a pooled count (capped at 4096)."""
    k = raw_counts(guide, s_p)
    shape = k.shape
    ref = np.unravel_index(int(ref_lin), shape)
    ell = [L - j for L, j in zip(shape, patch)]
    rad = [(w - 1) // 2 for w in search]
    pr = k[tuple(slice(a, a + j) for a, j in zip(ref, patch))].ravel()
    P = pr.size
    if policy == "fixed":
        thr = P * (tau_fixed if tau_fixed else 1 + t * np.sqrt(2.0 / P))
    elif policy == "candidate_standardized":
        thr = t
    else:
        mv = [moments(int(min(round(2 * x), 4096))) for x in pr]
        thr = sum(m for m, _ in mv) + t * np.sqrt(sum(v for _, v in mv)) + beta * P * np.mean(pr) ** kappa
    out = {}
    ranges = [range(max(r - a, 0), min(r + a, e) + 1) for r, a, e in zip(ref, rad, ell)]
    for cpos in itertools.product(*ranges):
        q = k[tuple(slice(a, a + j) for a, j in zip(cpos, patch))].ravel()
        phi = poisson_phi(metric, pr, q)
        acc = float(np.sum(phi))
        if policy == "candidate_standardized":
            mv = [moments(int(min(round(a + b), 4096))) for a, b in zip(pr, q)]
            vs = sum(v for _, v in mv)
            sc = (acc - sum(m for m, _ in mv)) / np.sqrt(vs) if vs > 0 else 0.0
            mag = abs(sc) + 1e-30
        else:
            sc, mag = acc, acc + 1e-30
        out[int(np.ravel_multi_index(cpos, shape))] = (sc, mag)
    return out, thr


def group_agreement(gpu, orc, guide, patch, search, noise, gamma, tau, max_explain=200, scorer=None,
                    rel=NEAR_TIE_REL, tol=0.0):
    """Compare per-reference groups.  gpu/orc: (origins[R], groups[R, M], counts[R])
    sorted by origin.  scorer(ref) -> ({origin: (score, magnitude)}, tau)
    replaces the SSD scores (candidate_scores) for other distances.  Returns
    (n_exact, n_near_tie, n_bad, bad_examples)."""
    go, gg, gc = gpu
    oo, og, oc = orc
    assert np.array_equal(go, oo), "reference origins differ"
    n_exact = n_tie = n_bad = 0
    bad = []
    for r in range(len(oo)):
        a = list(gg[r, : gc[r]])
        b = list(og[r, : oc[r]])
        if a == b:
            n_exact += 1
            continue
        if n_tie + n_bad >= max_explain:
            n_bad += 1
            continue
        if scorer is None:
            sc = candidate_scores(guide, oo[r], patch, search, noise, gamma)
        else:
            sc, tau = scorer(oo[r])
        ok = True
        for k in range(1, min(len(a), len(b))):
            if a[k] != b[k]:
                sa, ma = sc[a[k]]
                sb, mb = sc[b[k]]
                if abs(sa - sb) > rel * max(ma, mb) + tol:
                    ok = False
        if len(a) != len(b):
            # a different count is only legitimate if some candidate sits at
            # the acceptance threshold
            near_tau = any(abs(s - tau) <= rel * m + tol for k2, (s, m) in sc.items() if k2 != oo[r])
            ok = ok and near_tau
        if ok:
            n_tie += 1
        else:
            n_bad += 1
            if len(bad) < 5:
                bad.append((int(oo[r]), a, b))
    return n_exact, n_tie, n_bad, bad


def oracle_two_stages_f32_pilot(oracle, p, y):
    """The oracle's two stages with the stage-1 estimate stored in float32
    between them, as the library stores it (its arrays are float32).  The
    end-to-end voxel contract is checked against this; the PSNR contract
    against the oracle's double-precision run (oracle.denoise)."""
    pilot = oracle.stage(p, y, None, 1).astype(np.float32)
    if p.stages < 2:
        return pilot.astype(np.float64)
    return oracle.stage(p, y, pilot.astype(np.float64), 2)


def footprint_mask(shape, patch, origins):
    """Boolean mask of the union of the patches at the given linear origins."""
    mask = np.zeros(shape, bool)
    for o in origins:
        c = np.unravel_index(int(o), shape)
        mask[tuple(slice(a, a + j) for a, j in zip(c, patch))] = True
    return mask


def end_to_end_contract(ctx, oracle, p, y, x, cfg, got, cuda, prm=None, what=""):
    """Voxel and PSNR contract of both stages (no mass conservation).

    The library's stage-1 estimate differs from the oracle's by float32
    rounding, and stage-2 matching on the two estimates may order near-tied
    candidates differently, which the group contract allows.  So:
      - stage-2 groups: the GPU's, matched on its own estimate, against the
        oracle's on its estimate (float32), identical except at near-ties of
        the oracle's double-precision scores;
      - voxels outside the patches of the groups that differ: >= 99.9% within
        1e-4 of the peak of the oracle's two stages (float32 estimate between
        them);
      - PSNR within 0.01 dB of the oracle's double-precision run.
    Returns (fraction of voxels compared, fraction within tolerance)."""
    import torch
    opilot = oracle.stage(p, y, None, 1).astype(np.float32)
    ref = oracle.stage(p, y, opilot.astype(np.float64), 2)
    ref64, _ = oracle.denoise(p, y)
    gpilot = torch.empty(y.shape, dtype=torch.float32, device="cuda:0")
    ctx.bmnd_stage(cuda(y), None, gpilot, cfg["noise"], cfg["patch"], cfg["step"], cfg["search"],
                   cfg["group_size"][0], 1, 0, prm)
    M = cfg["group_size"][1]
    o, gg, gc = ctx.bmnd_match(gpilot, cfg["noise"], cfg["patch"], cfg["step"], cfg["search"], M, 2, prm)
    o, gg, gc = o.cpu().numpy(), gg.cpu().numpy(), gc.cpu().numpy()
    order = np.argsort(o)
    gpu = (o[order], gg[order], gc[order])
    _, _, og, oc = oracle.stage(p, y, opilot.astype(np.float64), 2, want_den=True, want_groups=True)
    oo = oracle.schedule(p)
    P = int(np.prod(cfg["patch"]))
    tau = 400.0 * P / 255.0 ** 2
    ne, nt, nb, bad = group_agreement(gpu, (oo, og[:, :M], oc), opilot.astype(np.float64), cfg["patch"],
                                      cfg["search"], cfg["noise"], 0.0, tau, max_explain=len(oo))
    assert nb == 0, bad
    differ = [r for r in range(len(oo)) if list(gpu[1][r, :gpu[2][r]]) != list(og[r, :oc[r]])]
    origins = [m for r in differ for m in list(gpu[1][r, :gpu[2][r]]) + list(og[r, :oc[r]])]
    mask = ~footprint_mask(y.shape, cfg["patch"], origins)
    frac_cmp = float(mask.mean())
    within = voxel_report(np.asarray(got)[mask], ref[mask])[0] if mask.any() else 1.0
    assert within >= VOXEL_FRAC, "%s: only %.5f of the compared voxels within %g" % (what, within, VOXEL_ABS)
    assert abs(psnr(got, x) - psnr(ref64, x)) <= PSNR_DB
    return frac_cmp, within


def groups_of(ctx, guide_cuda, cfg, stage, prm=None):
    """The library's groups (origins, groups, counts) sorted by origin."""
    M = cfg["group_size"][stage - 1]
    o, g, c = ctx.bmnd_match(guide_cuda, cfg["noise"], cfg["patch"], cfg["step"], cfg["search"], M, stage, prm)
    o, g, c = o.cpu().numpy(), g.cpu().numpy(), c.cpu().numpy()
    order = np.argsort(o)
    return o[order], g[order], c[order]


def differing_members(gpu, og, oc):
    """Member origins (both sides) of the references whose groups differ."""
    _, gg, gc = gpu
    out = []
    for r in range(len(gc)):
        a = list(gg[r, :gc[r]])
        b = list(og[r, :oc[r]])
        if a != b:
            out += a + b
    return out


def dilate(mask, widths):
    """Boolean dilation of mask by +-widths[d] along every axis d."""
    out = mask.copy()
    for d, w in enumerate(widths):
        acc = out.copy()
        for s in range(1, w + 1):
            acc[tuple(slice(s, None) if a == d else slice(None) for a in range(out.ndim))] |= \
                out[tuple(slice(None, -s) if a == d else slice(None) for a in range(out.ndim))]
            acc[tuple(slice(None, -s) if a == d else slice(None) for a in range(out.ndim))] |= \
                out[tuple(slice(s, None) if a == d else slice(None) for a in range(out.ndim))]
        out = acc
    return out


def assert_voxels_on(got, ref, mask, what=""):
    """The voxel contract on the voxels of mask."""
    if not mask.any():
        return 1.0
    frac = voxel_report(np.asarray(got)[mask], np.asarray(ref)[mask])[0]
    assert frac >= VOXEL_FRAC, "%s: only %.5f of the compared voxels within %g" % (what, frac, VOXEL_ABS)
    return frac


def stage1_poisson_contract(ctx, oracle, p, y, x, cfg, got, cuda, prm, scorer, what=""):
    """Stage 1 under a Poisson distance: groups identical except at near-ties
    of the oracle's FP64 scores (scorer), the voxel contract outside the
    patches of the groups that differ (either choice at a near-tie is
    correct, and they synthesize different patches), PSNR within 0.01 dB.
    Returns (fraction of voxels compared, number of differing groups)."""
    ref, _, og, oc = oracle.stage(p, y, None, 1, want_den=True, want_groups=True)
    M = cfg["group_size"][0]
    gpu = groups_of(ctx, cuda(y), cfg, 1, prm)
    oo = oracle.schedule(p)
    ne, nt, nb, bad = group_agreement(gpu, (oo, og[:, :M], oc), y, cfg["patch"], cfg["search"], cfg["noise"],
                                      0.0, 0.0, max_explain=len(oo), scorer=scorer, rel=POISSON_TIE_REL,
                                      tol=POISSON_TIE_REL)
    assert nb == 0, bad
    mask = ~footprint_mask(y.shape, cfg["patch"], differing_members(gpu, og[:, :M], oc))
    assert_voxels_on(got, ref, mask, what)
    assert abs(psnr(got, x) - psnr(ref, x)) <= PSNR_DB
    return float(mask.mean()), nt


def two_stage_contract(ctx, oracle, p, y, x, cfg, got, cuda, prm=None, scorer=None, what=""):
    """Both stages: stage-1 groups identical except at near-ties of the
    oracle's FP64 scores (scorer for a Poisson distance, else SSD with the
    noise-bias correction); the voxel contract against the oracle's stages
    (float32 pilot between them) outside the patches of the stage-1 groups
    that differ, dilated by the stage-2 search radius and patch (where the
    two pilots differ and stage-2 matching reads them; by one more patch with
    mass conservation, whose correction spreads over overlapping groups),
    and outside the patches of the stage-2 groups that differ; PSNR within
    0.01 dB of the oracle's double-precision run.  Returns the fraction of
    voxels compared."""
    import torch
    opilot = oracle.stage(p, y, None, 1).astype(np.float32)
    ref = oracle.stage(p, y, opilot.astype(np.float64), 2)
    ref64, _ = oracle.denoise(p, y)
    _, _, og1, oc1 = oracle.stage(p, y, None, 1, want_den=True, want_groups=True)
    M1, M2 = cfg["group_size"]
    gpu1 = groups_of(ctx, cuda(y), cfg, 1, prm)
    oo = oracle.schedule(p)
    P = int(np.prod(cfg["patch"]))
    if scorer is None:
        _, _, nb, bad = group_agreement(gpu1, (oo, og1[:, :M1], oc1), y.astype(np.float64), cfg["patch"],
                                        cfg["search"], cfg["noise"], 3.0, 3000.0 * P / 255.0 ** 2,
                                        max_explain=len(oo))
    else:
        _, _, nb, bad = group_agreement(gpu1, (oo, og1[:, :M1], oc1), y, cfg["patch"], cfg["search"], cfg["noise"],
                                        0.0, 0.0, max_explain=len(oo), scorer=scorer, rel=POISSON_TIE_REL,
                                        tol=POISSON_TIE_REL)
    assert nb == 0, bad
    gpilot = torch.empty(y.shape, dtype=torch.float32, device="cuda:0")
    ctx.bmnd_stage(cuda(y), None, gpilot, cfg["noise"], cfg["patch"], cfg["step"], cfg["search"], M1, 1,
                   p.mass_conserve & 1, prm)
    gpu2 = groups_of(ctx, gpilot, cfg, 2, prm)
    _, _, og2, oc2 = oracle.stage(p, y, opilot.astype(np.float64), 2, want_den=True, want_groups=True)
    a1 = footprint_mask(y.shape, cfg["patch"], differing_members(gpu1, og1[:, :M1], oc1))
    if not a1.any():
        # identical stage-1 groups: the two pilots differ by float rounding
        # only, so the stage-2 groups must agree except at near-ties of the
        # oracle's scores on its own pilot (SSD, tau of the Wiener stage)
        _, _, nb2, bad2 = group_agreement(gpu2, (oo, og2[:, :M2], oc2), opilot.astype(np.float64),
                                          cfg["patch"], cfg["search"], cfg["noise"], 0.0, 400.0 * P / 255.0 ** 2,
                                          max_explain=len(oo))
        assert nb2 == 0, bad2
    reach = [(w - 1) // 2 + j for w, j in zip(cfg["search"], cfg["patch"])]
    bad_area = dilate(a1, reach) | footprint_mask(y.shape, cfg["patch"], differing_members(gpu2, og2[:, :M2], oc2))
    if p.mass_conserve:
        bad_area = dilate(bad_area, list(cfg["patch"]))
    mask = ~bad_area
    assert_voxels_on(got, ref, mask, what)
    assert abs(psnr(got, x) - psnr(ref64, x)) <= PSNR_DB
    return float(mask.mean())


def two_stage_poisson_contract(ctx, oracle, p, y, x, cfg, got, cuda, prm, scorer, what=""):
    """two_stage_contract under a Poisson distance in stage 1."""
    return two_stage_contract(ctx, oracle, p, y, x, cfg, got, cuda, prm, scorer, what)
