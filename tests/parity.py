"""Comparison helpers shared by the GPU parity tests (test code only)."""
from __future__ import annotations

import itertools

import numpy as np

# Tolerances of the parity contract: group membership identical except at
# near-ties (scores closer than 1e-5 relative to their magnitude), >= 99.9%
# of output voxels within 1e-4 of the peak intensity, PSNR within 0.01 dB.
NEAR_TIE_REL = 1e-5
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


def group_agreement(gpu, orc, guide, patch, search, noise, gamma, tau, max_explain=200):
    """Compare per-reference groups.  gpu/orc: (origins[R], groups[R, M], counts[R])
    sorted by origin.  Returns (n_exact, n_near_tie, n_bad, bad_examples)."""
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
        sc = candidate_scores(guide, oo[r], patch, search, noise, gamma)
        ok = True
        for k in range(1, min(len(a), len(b))):
            if a[k] != b[k]:
                sa, ma = sc[a[k]]
                sb, mb = sc[b[k]]
                if abs(sa - sb) > NEAR_TIE_REL * max(ma, mb):
                    ok = False
        if len(a) != len(b):
            # a different count is only legitimate if some candidate sits at
            # the acceptance threshold
            near_tau = any(abs(s - tau) <= NEAR_TIE_REL * m for k2, (s, m) in sc.items() if k2 != oo[r])
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
