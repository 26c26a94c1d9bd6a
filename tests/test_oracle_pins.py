"""Pins of the FP64 oracle against facts that do not come from the oracle itself:
library routines (scipy DCT, numpy Kaiser, scipy Bessel I0), hand-derived values,
closed forms stated in the paper, brute force on tiny inputs, Monte-Carlo checks
of the variance propagation lemma, and invariants (orthonormality, identity at
zero threshold, mass conservation, N-D consistency).

Each test names the passage it pins.
"""
import itertools
import math

import numpy as np
import pytest
import scipy.fft
import scipy.special

from paper_2609_34622_b300 import synth


# ---------------------------------------------------------------------------
# transforms
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("n", [1, 2, 3, 4, 5, 8, 11, 16, 32])
def test_dct_matrix_matches_scipy(oracle, n):
    """Orthonormal DCT-II (App. A spatial transform) equals scipy's dct(norm='ortho')."""
    ref = scipy.fft.dct(np.eye(n), type=2, norm="ortho", axis=0)
    np.testing.assert_allclose(oracle.dct_matrix(n), ref, atol=1e-14)


def test_haar_hand_values(oracle):
    """Haar group transform (App. A): hand-written 1-, 2- and 4-point orthonormal Haar."""
    s = 1 / math.sqrt(2)
    np.testing.assert_allclose(oracle.haar_matrix(1), [[1.0]])
    np.testing.assert_allclose(oracle.haar_matrix(2), [[s, s], [s, -s]], atol=1e-15)
    h4 = np.array([[0.5, 0.5, 0.5, 0.5], [0.5, 0.5, -0.5, -0.5], [s, -s, 0, 0], [0, 0, s, -s]])
    np.testing.assert_allclose(oracle.haar_matrix(4), h4, atol=1e-15)


@pytest.mark.parametrize("n", [2, 4, 8, 16, 32, 64])
def test_haar_orthonormal_and_dyadic(oracle, n):
    H = oracle.haar_matrix(n)
    np.testing.assert_allclose(H @ H.T, np.eye(n), atol=1e-13)
    # every detail row is constant on the two halves of one dyadic block
    for row in H[1:]:
        nz = np.nonzero(row)[0]
        b = len(nz)
        assert b & (b - 1) == 0 and nz[0] % b == 0 and nz[-1] == nz[0] + b - 1
        np.testing.assert_allclose(row[nz[: b // 2]], 1 / math.sqrt(b))
        np.testing.assert_allclose(row[nz[b // 2:]], -1 / math.sqrt(b))


@pytest.mark.parametrize("n,beta", [(1, 2.0), (4, 2.0), (8, 2.0), (32, 2.0), (5, 0.5), (9, 6.0)])
def test_kaiser_matches_numpy(oracle, n, beta):
    """Kaiser aggregation window (App. A, beta = 2) equals numpy.kaiser."""
    np.testing.assert_allclose(oracle.kaiser(n, beta), np.kaiser(n, beta), rtol=1e-13)


def test_bessel_i0_matches_scipy(oracle):
    for x in [0.0, 0.3, 1.0, 2.0, 5.5, 12.0]:
        assert oracle.bessel_i0(x) == pytest.approx(scipy.special.i0(x), rel=1e-14)


def _full_T(oracle, count, patch, group_transform="haar"):
    """Full matrix of the group transform, built with numpy.kron from matrices
    that come from scipy (DCT) and from the hand-checked Haar."""
    A0 = scipy.fft.dct(np.eye(count), norm="ortho", axis=0) if group_transform == "dct" \
        else oracle.haar_matrix(count)
    T = A0
    for j in patch:
        T = np.kron(T, scipy.fft.dct(np.eye(j), norm="ortho", axis=0))
    return T


@pytest.mark.parametrize("count,patch,gt", [(4, (3, 2), "haar"), (2, (4,), "haar"), (3, (2, 2, 2), "dct"),
                                            (8, (2, 3), "haar"), (1, (5,), "haar")])
def test_group_transform_is_kronecker_and_orthonormal(oracle, count, patch, gt):
    """Patch-group observation model: T = (group axis) (x) DCT_j0 (x) ...;
    T T^T = I, mode 1 inverts, mode 2 is the entrywise square (the factor of
    Eq. transformed-coefficient-variance for diagonal covariance)."""
    D = len(patch)
    p = oracle.params(tuple(4 * j for j in patch), patch, (1,) * D, (3,) * D, group_transform=gt)
    d = count * int(np.prod(patch))
    E = np.eye(d).reshape((d, count) + patch)
    Tcols = np.stack([oracle.group_transform(p, E[i], 0).ravel() for i in range(d)], axis=1)
    T = _full_T(oracle, count, patch, gt)
    np.testing.assert_allclose(Tcols, T, atol=1e-13)
    np.testing.assert_allclose(T @ T.T, np.eye(d), atol=1e-13)
    x = np.random.default_rng(1).normal(size=(count,) + patch)
    y = oracle.group_transform(p, x, 0)
    np.testing.assert_allclose(oracle.group_transform(p, y, 1), x, atol=1e-13)
    np.testing.assert_allclose(oracle.group_transform(p, x, 2).ravel(), (T * T) @ x.ravel(), atol=1e-13)


# ---------------------------------------------------------------------------
# reference schedule (Sec. 4.1)
# ---------------------------------------------------------------------------

def test_shift_list_example_2d(oracle):
    """Eq. number-shifts / candidate-shift-list for j = 8, h = 3, rho_s = 2 give
    n = ceil(2*7/3) = 5 and S = (0, 2, 4, 5, 7) (hand derived).  Under the
    generated schedule axis 0 is shifted by S[(q_1 + k) mod 5], so an interior
    axis-0 slot q_0 (nominal 3 q_0) yields exactly the origins 3 q_0 - S."""
    p = oracle.params((64, 64), (8, 8), (3, 3), (19, 19))
    R = oracle.schedule(p)
    r0, r1 = R // 64, R % 64
    S = (0, 2, 4, 5, 7)
    for q1 in range(5, 12):
        # the last axis is unshifted: column r1 = 3 q1 holds slot q1's origins
        col = sorted(r0[(r1 == 3 * q1) & (r0 >= 12) & (r0 <= 36)].tolist())
        expect = sorted({3 * q0 - S[(q1 + k) % 5] for q0 in range(0, 20) for k in (0, 1)} & set(range(12, 37)))
        assert col == expect, (q1, col, expect)


def test_off_schedule_1d_lattice(oracle):
    """Def. off reference schedule: 0, h, 2h, ..., l, with l appended.  In 1-D
    the generated schedule leaves its only (last) axis unshifted, so it gives
    the same lattice."""
    L, j, h = 100, 8, 3
    ell = L - j
    expect = list(range(0, ell + 1, h))
    if expect[-1] != ell:
        expect.append(ell)
    for sched in ("off", "generated"):
        p = oracle.params((L,), (j,), (h,), (9,), schedule=sched)
        assert oracle.schedule(p).tolist() == expect


@pytest.mark.parametrize("shape,patch,step,sched", [
    ((64, 64), (8, 8), (3, 3), "generated"), ((37, 29), (5, 4), (3, 2), "generated"),
    ((20, 18, 16), (4, 4, 4), (2, 2, 2), "generated"), ((37, 29), (5, 4), (3, 2), "balanced"),
    ((1, 40, 17), (1, 6, 5), (1, 4, 3), "sparse"), ((23, 31), (6, 6), (4, 5), "off")])
def test_schedule_valid_and_covering(oracle, shape, patch, step, sched):
    """Clipped reference origin: every origin is valid, the far boundary l_d is
    reached on every axis, there are at most K_s prod Z_d distinct origins,
    and the reference patches cover the whole array (steps <= patch sizes)."""
    p = oracle.params(shape, patch, step, (3,) * len(shape), schedule=sched)
    R = oracle.schedule(p)
    coords = np.stack(np.unravel_index(R, shape), axis=1)
    ell = np.array(shape) - np.array(patch)
    assert (coords >= 0).all() and (coords <= ell).all()
    assert len(np.unique(R)) == len(R) and (np.diff(R) > 0).all()
    for d in range(len(shape)):
        assert (coords[:, d] == ell[d]).any() and (coords[:, d] == 0).any()
    Z = [math.ceil(e / h) + 1 for e, h in zip(ell, step)]
    assert len(R) <= 2 * int(np.prod(Z))
    cov = np.zeros(shape, np.int32)
    for c in coords:
        cov[tuple(slice(int(a), int(a) + j) for a, j in zip(c, patch))] += 1
    assert (cov > 0).all()


def test_generated_vs_sparse_singleton(oracle):
    """Sparse schedule (Def.): singleton axes leave the hierarchy.  With a
    leading singleton axis both schedules coincide with the 1-D lattice; the
    survey reading notes that a trailing singleton axis changes the generated
    schedule but not the sparse one."""
    L = 50
    p1 = oracle.params((L,), (6,), (4,), (9,))
    base = oracle.schedule(p1).tolist()
    for sched in ("generated", "sparse"):
        p = oracle.params((1, L), (1, 6), (1, 4), (1, 9), schedule=sched)
        assert oracle.schedule(p).tolist() == base
    p = oracle.params((L, 1), (6, 1), (4, 1), (9, 1), schedule="sparse")
    assert oracle.schedule(p).tolist() == base


# ---------------------------------------------------------------------------
# block matching (Sec. 4.2, 4.4; App. A group rules), brute force
# ---------------------------------------------------------------------------

def _brute_match(y, ref, patch, search, noise, gamma, tau, M, min_group=2, pow2=True):
    """Independent numpy brute force: score every origin in the clipped window."""
    shape = y.shape
    ell = [L - j for L, j in zip(shape, patch)]
    rad = [(w - 1) // 2 for w in search]
    pref = y[tuple(slice(r, r + j) for r, j in zip(ref, patch))].astype(np.float64)
    cands = []
    ranges = [range(max(r - a, 0), min(r + a, e) + 1) for r, a, e in zip(ref, rad, ell)]
    for c in itertools.product(*ranges):
        if tuple(c) == tuple(ref):
            continue
        q = y[tuple(slice(a, a + j) for a, j in zip(c, patch))].astype(np.float64)
        ssd = float(((q - pref) ** 2).sum())
        if noise[0] == "poisson":
            B = noise[1] * float(np.maximum(q + pref, 0).sum())
        else:
            B = 2 * pref.size * noise[1] ** 2
        s = ssd - gamma * B if gamma > 0 else ssd
        cands.append((s, int(np.ravel_multi_index(c, shape))))
    cands.sort()
    nacc = sum(1 for s, _ in cands if s < tau)
    take = min(nacc, M - 1)
    if 1 + take < min_group:
        take = min(min_group - 1, M - 1, len(cands))
    cnt = 1 + take
    if pow2:
        cnt = 1 << (cnt.bit_length() - 1)
    return [int(np.ravel_multi_index(tuple(ref), shape))] + [l for _, l in cands[: cnt - 1]]


@pytest.mark.parametrize("case", range(4))
def test_matching_brute_force(oracle, case):
    rng = np.random.default_rng(10 + case)
    # dyadic data (counts times 2^-k, or multiples of 1/64) keep every score
    # exact in double precision, so exact ties are broken by the index rule
    # on both sides rather than by summation order
    if case == 0:
        shape, patch, search, noise, M = (12, 12), (3, 3), (5, 5), ("poisson", 0.25), 8
    elif case == 1:
        shape, patch, search, noise, M = (16,), (4,), (7,), ("poisson", 0.5), 4
    elif case == 2:
        shape, patch, search, noise, M = (6, 6, 6), (2, 2, 2), (3, 3, 3), ("poisson", 0.25), 16
    else:
        shape, patch, search, noise, M = (12, 10), (3, 2), (7, 5), ("gaussian", 0.125), 8
    x = rng.uniform(0.2, 1.0, size=shape)
    if noise[0] == "poisson":
        y = rng.poisson(x / noise[1]) * noise[1]
    else:
        y = np.round(64 * (x + rng.normal(0, noise[1], shape))) / 64
    for stage in (1, 2):
        for tau in (0.0, 0.05, 1e9):
            p = oracle.params(shape, patch, (1,) * len(shape), search, noise, (M, M),
                              tau_ht=tau if tau > 0 else 1e-300, tau_wie=tau if tau > 0 else 1e-300)
            gamma = 3.0 if stage == 1 else 0.0
            t = tau if tau > 0 else 1e-300
            for ref in [(0,) * len(shape), tuple(s // 2 for s in shape), tuple(s - j for s, j in zip(shape, patch))]:
                rl = int(np.ravel_multi_index(ref, shape))
                mem, _ = oracle.match_ref(p, y, stage, rl)
                assert mem.tolist() == _brute_match(y, ref, patch, search, noise, gamma, t, M)


# ---------------------------------------------------------------------------
# variances (Lemma covariance propagation, Cor. white noise, Prop. diagonal Poisson)
# ---------------------------------------------------------------------------

def _group_setup(oracle, noise, shape=(16, 16), patch=(4, 4), seed=0):
    rng = np.random.default_rng(seed)
    x = rng.uniform(0.1, 1.0, size=shape)
    p = oracle.params(shape, patch, (2, 2), (7, 7), noise, (8, 8))
    members = np.array([np.ravel_multi_index(c, shape) for c in [(3, 3), (5, 4), (0, 9), (10, 2)]])
    return p, x, members, rng


def test_white_noise_variance(oracle):
    """Cor. white-noise transform variance: sigma_k^2 = sigma^2 for every k."""
    p, x, members, _ = _group_setup(oracle, ("gaussian", 0.3))
    g = oracle.filter_group(p, 1, x, None, members)
    np.testing.assert_allclose(g["var"], 0.09, rtol=1e-13)


def test_poisson_variance_monte_carlo(oracle):
    """Lemma covariance propagation / Prop. diagonal Poisson variance: with the
    exact clean mean as surrogate, sum_i T_ki^2 s_P X(u_i) is the variance of
    the transformed coefficient of Poisson observations (independent counts,
    distinct source voxels).  Checked against 20000 Monte-Carlo draws."""
    s_p = 0.05
    p, x, _, rng = _group_setup(oracle, ("poisson", s_p))
    offs = [np.ravel_multi_index((a, b), x.shape) for a in range(4) for b in range(4)]

    def empirical(members, n=20000):
        Ys = []
        idx = np.array([[m + o for o in offs] for m in members]).ravel()
        for _ in range(n // 500):
            y = rng.poisson(x[None] / s_p, size=(500,) + x.shape) * s_p
            grp = y.reshape(500, -1)[:, idx].reshape(500, 4, 4, 4)
            Ys.append(np.stack([oracle.group_transform(p, gi, 0).ravel() for gi in grp]))
        return np.concatenate(Ys).var(axis=0, ddof=1)

    disjoint = np.array([np.ravel_multi_index(c, x.shape) for c in [(0, 0), (0, 9), (6, 4), (10, 11)]])
    var = oracle.filter_group(p, 1, x, None, disjoint)["var"].ravel()
    # relative standard error of a variance estimate ~ sqrt(2/n) ~ 1%
    np.testing.assert_allclose(empirical(disjoint), var, rtol=0.06)
    # overlapping patches share source voxels: there the diagonal model is an
    # approximation (Eq. shared-voxel-group-covariance), and it visibly misses
    overlap = np.array([np.ravel_multi_index(c, x.shape) for c in [(3, 3), (4, 3), (3, 4), (4, 4)]])
    var_o = oracle.filter_group(p, 1, x, None, overlap)["var"].ravel()
    assert np.max(np.abs(empirical(overlap) / var_o - 1)) > 0.2


def test_patch_weights_equal_exact_synthesized_noise(oracle):
    """Def. coefficient-domain hard-thresholding weighting (variance model,
    patch scope) under white noise: R_j = sum_l |V_jl|^2 sum_q a_lq sigma^2
    equals the trace of the noise covariance of synthesized patch j,
    computed here with the full matrices U A T sigma^2 T^T A U^T."""
    sig = 0.2
    p, x, members, rng = _group_setup(oracle, ("gaussian", sig))
    y = x + rng.normal(0, sig, x.shape)
    g = oracle.filter_group(p, 1, y, None, members)
    a = (g["C"].ravel() != 0).astype(float)
    T = _full_T(oracle, 4, (4, 4))
    U = T.T
    cov = U @ np.diag(a) @ (sig ** 2 * np.eye(64)) @ np.diag(a) @ U.T
    R = np.array([np.trace(cov[j * 16:(j + 1) * 16, j * 16:(j + 1) * 16]) for j in range(4)])
    np.testing.assert_allclose(g["w"], 1.0 / R, rtol=1e-12)


def test_hard_threshold_exact_tie(oracle):
    """Def. coefficient thresholding at an exact tie: with s_P = 1 and two
    one-sample members y = (9, 0), Haar gives Y = (9/sqrt 2, 9/sqrt 2) and
    sigma^2 = ((9 + 0)/2, (9 + 0)/2), so |Y_k| = 3 sigma_k for both
    coefficients in real arithmetic and the strict inequality zeroes them;
    a count of 9 + 1e-6 lifts both above the threshold."""
    y = np.array([9.0, 0.0, 0.0])
    p = oracle.params(y.shape, (1,), (1,), (3,), ("poisson", 1.0), (2, 2))
    g = oracle.filter_group(p, 1, y, None, [0, 1])
    np.testing.assert_allclose(np.abs(g["Y"].ravel()), 9 / np.sqrt(2), rtol=1e-15)
    np.testing.assert_allclose(np.sqrt(g["var"].ravel()), np.sqrt(4.5), rtol=1e-15)
    assert np.all(g["C"] == 0.0)
    y[0] = 9.0 + 1e-6
    g = oracle.filter_group(p, 1, y, None, [0, 1])
    np.testing.assert_array_equal(g["C"], g["Y"])


def test_hard_threshold_mask(oracle):
    """Def. coefficient thresholding: C_k = Y_k if |Y_k| > lambda sigma_k else 0."""
    p, x, members, rng = _group_setup(oracle, ("poisson", 0.1))
    y = rng.poisson(x / 0.1) * 0.1
    g = oracle.filter_group(p, 1, y, None, members)
    keep = np.abs(g["Y"]) - 3.0 * np.sqrt(g["var"]) > 1e-12 * 3.0 * np.sqrt(g["var"])
    np.testing.assert_array_equal(g["C"], np.where(keep, g["Y"], 0.0))


@pytest.mark.parametrize("mode,a", [("noise_floor", 1.0), ("variance_scaled", 0.4)])
def test_wiener_dead_zone_closed_form(oracle, mode, a):
    """Prop. corrected pilot-power Wiener gain: G = 0 for |Gamma|^2 <= a sigma^2,
    else (|Gamma|^2 - a sigma^2) / (|Gamma|^2 - a sigma^2 + s_v sigma^2)."""
    sig = 0.15
    shape, patch = (16, 16), (4, 4)
    rng = np.random.default_rng(3)
    x = rng.uniform(0.1, 1.0, size=shape)
    y = x + rng.normal(0, sig, shape)
    pilot = x + rng.normal(0, 0.05, shape)
    p = oracle.params(shape, patch, (2, 2), (7, 7), ("gaussian", sig), (8, 8), power_mode=mode)
    members = np.array([np.ravel_multi_index(c, shape) for c in [(3, 3), (5, 4), (0, 9), (10, 2)]])
    g = oracle.filter_group(p, 2, y, pilot, members)
    offs = [np.ravel_multi_index((i, j), shape) for i in range(4) for j in range(4)]
    T = _full_T(oracle, 4, patch)
    gam = T @ pilot.ravel()[np.array([[m + o for o in offs] for m in members]).ravel()]
    s2 = sig ** 2
    G = np.where(gam ** 2 <= a * s2, 0.0, (gam ** 2 - a * s2) / (gam ** 2 - a * s2 + 0.4 * s2))
    np.testing.assert_allclose(g["C"].ravel(), G * g["Y"].ravel(), atol=1e-13)


# ---------------------------------------------------------------------------
# whole-stage invariants
# ---------------------------------------------------------------------------

def test_identity_at_zero_threshold(oracle):
    """With sigma = 0 and lambda_HT = 0 every nonzero coefficient passes, every
    Wiener gain is 1 where the coefficient is nonzero, and weighted overlap-add
    of unmodified patches returns the observation exactly."""
    rng = np.random.default_rng(5)
    y = rng.uniform(0, 1, size=(24, 20))
    p = oracle.params(y.shape, (4, 4), (2, 2), (7, 7), ("gaussian", 0.0), (8, 16), lambda_ht=0.0)
    out, pilot = oracle.denoise(p, y)
    np.testing.assert_allclose(pilot, y, atol=1e-12)
    np.testing.assert_allclose(out, y, atol=1e-12)


def test_constant_array_closed_form(oracle):
    """A constant group has only its all-axis DC coefficient Y = c sqrt(n P).
    Stage 1: it survives the threshold, so overlap-add returns c (Def. weighted
    overlap-add).  Stage 2 (classic power): every group is full (n = 16, all
    distances 0), the gain is G = Y^2 / (Y^2 + s_v sigma^2) (Def. practical
    Wiener gain), so the output is the constant c G."""
    c, sig = 0.7, 0.05
    y = np.full((20, 22), c)
    p = oracle.params(y.shape, (4, 4), (3, 3), (7, 7), ("gaussian", sig), (8, 16))
    out, pilot = oracle.denoise(p, y)
    np.testing.assert_allclose(pilot, c, atol=1e-12)
    Y2 = c * c * 16 * 16
    np.testing.assert_allclose(out, c * Y2 / (Y2 + 0.4 * sig * sig), atol=1e-12)


@pytest.mark.parametrize("noise", [("poisson", 0.2), ("gaussian", 0.1)])
def test_mass_conservation(oracle, noise):
    """Thm. mass conservation after normalized overlap-add: with the two-sweep
    correction in both stages, sum x^ = sum y; without it the sums differ."""
    rng = np.random.default_rng(7)
    x = synth.disc_rect_image((28, 30), rng)
    y = rng.poisson(x / noise[1]) * noise[1] if noise[0] == "poisson" else x + rng.normal(0, noise[1], x.shape)
    for mc in (1, 2, 3):
        p = oracle.params(y.shape, (4, 4), (2, 2), (9, 9), noise, (8, 16), mass_conserve=mc)
        out, pilot = oracle.denoise(p, y)
        if mc & 1:
            assert pilot.sum() == pytest.approx(y.sum(), rel=1e-12)
        if mc & 2:
            assert out.sum() == pytest.approx(y.sum(), rel=1e-12)
    p = oracle.params(y.shape, (4, 4), (2, 2), (9, 9), noise, (8, 16), mass_conserve=0)
    out, _ = oracle.denoise(p, y)
    assert abs(out.sum() - y.sum()) > 1e-6 * abs(y.sum())


def test_nd_consistency_singleton_axis(oracle):
    """A 2-D array with a leading axis of length 1 gives the 1-D result."""
    rng = np.random.default_rng(9)
    x = synth.ecg_signal(600, 250.0, rng)
    y = rng.poisson(x * 20) / 20.0
    p1 = oracle.params((600,), (16,), (4,), (33,), ("poisson", 0.05), (16, 32))
    p2 = oracle.params((1, 600), (1, 16), (1, 4), (1, 33), ("poisson", 0.05), (16, 32))
    o1, pl1 = oracle.denoise(p1, y)
    o2, pl2 = oracle.denoise(p2, y[None])
    np.testing.assert_allclose(pl2[0], pl1, atol=1e-12)
    np.testing.assert_allclose(o2[0], o1, atol=1e-12)


def test_stage_points_agree_with_full_stage(oracle):
    job = synth.config1()
    p = oracle.params(job.y.shape, job.patch, job.step, job.search, job.noise, job.group_size)
    full, pilot = oracle.denoise(p, job.y)
    pts = np.array([0, 63, 64 * 31 + 17, 64 * 64 - 1, 64 * 40 + 3])
    np.testing.assert_allclose(oracle.stage_points(p, job.y, None, 1, pts), pilot.ravel()[pts], rtol=1e-13)
    np.testing.assert_allclose(oracle.stage_points(p, job.y, pilot, 2, pts), full.ravel()[pts], rtol=1e-13)


def test_group_scope_and_dct_group_transform(oracle):
    """Group scope gives one weight per group; the DCT group transform keeps
    non-power-of-two group sizes (no truncation)."""
    p, x, members, rng = _group_setup(oracle, ("poisson", 0.1))
    p2 = oracle.params(x.shape, (4, 4), (2, 2), (7, 7), ("poisson", 0.1), (8, 8), weight_scope="group")
    g = oracle.filter_group(p2, 1, x, None, members)
    assert np.allclose(g["w"], g["w"][0])
    y = rng.poisson(x / 0.1) * 0.1
    p3 = oracle.params(x.shape, (4, 4), (1, 1), (7, 7), ("poisson", 0.1), (7, 7), group_transform="dct",
                       tau_ht=1e9)
    mem, _ = oracle.match_ref(p3, y, 1, 5 * 16 + 5)
    assert len(mem) == 7


def test_classic_group_weight_is_retained_count(oracle):
    """Def. hard-thresholding weighting: the classic group-scope surrogate is
    R = sum_k a_k = N_g^HT (Def. retained coefficient count)."""
    p0, x, members, rng = _group_setup(oracle, ("poisson", 0.1))
    y = rng.poisson(x / 0.1) * 0.1
    p = oracle.params(x.shape, (4, 4), (2, 2), (7, 7), ("poisson", 0.1), (8, 8),
                      weight_model="classic", weight_scope="group")
    g = oracle.filter_group(p, 1, y, None, members)
    n_ht = int(np.count_nonzero(g["C"]))
    np.testing.assert_allclose(g["w"], 1.0 / n_ht, rtol=1e-14)


def test_wiener_risk_weight_minimum_risk(oracle):
    """Thm. optimal scalar Wiener gain: at G = S / (S + sigma^2) the risk
    (1-G)^2 S + G^2 sigma^2 equals G sigma^2.  With s_v = 1 and the classic
    pilot power, the risk model in group scope therefore gives
    w = 1 / sum_k G_k sigma^2 with G_k = Gamma_k^2 / (Gamma_k^2 + sigma^2)."""
    sig = 0.2
    shape, patch = (16, 16), (4, 4)
    rng = np.random.default_rng(4)
    x = rng.uniform(0.1, 1.0, size=shape)
    y = x + rng.normal(0, sig, shape)
    pilot = x + rng.normal(0, 0.05, shape)
    p = oracle.params(shape, patch, (2, 2), (7, 7), ("gaussian", sig), (8, 8), s_v=1.0,
                      weight_model="risk", weight_scope="group")
    members = np.array([np.ravel_multi_index(c, shape) for c in [(3, 3), (5, 4), (0, 9), (10, 2)]])
    g = oracle.filter_group(p, 2, y, pilot, members)
    offs = [np.ravel_multi_index((i, j), shape) for i in range(4) for j in range(4)]
    gam = _full_T(oracle, 4, patch) @ pilot.ravel()[np.array([[m + o for o in offs] for m in members]).ravel()]
    G = gam ** 2 / (gam ** 2 + sig ** 2)
    np.testing.assert_allclose(g["w"], 1.0 / np.sum(G * sig ** 2), rtol=1e-12)


# ---------------------------------------------------------------------------
# soft thresholding (Def. "Coefficient thresholding", Eq. soft-threshold)
# ---------------------------------------------------------------------------

def _soft_params(oracle, noise, **kw):
    return oracle.params((16, 16), (4, 4), (2, 2), (7, 7), noise, (8, 8), ht_rule="soft", **kw)


def test_soft_threshold_coefficients(oracle):
    """Eq. (soft-threshold): C_k = sgn(Y_k) [|Y_k| - lambda sigma_k]_+, written
    here with numpy from the group's coefficients and variances."""
    _, x, members, rng = _group_setup(oracle, ("poisson", 0.1))
    p = _soft_params(oracle, ("poisson", 0.1))
    y = rng.poisson(x / 0.1) * 0.1
    g = oracle.filter_group(p, 1, y, None, members)
    want = np.sign(g["Y"]) * np.maximum(np.abs(g["Y"]) - 3.0 * np.sqrt(g["var"]), 0.0)
    np.testing.assert_allclose(g["C"], want, rtol=1e-13, atol=1e-15)
    assert np.count_nonzero(g["C"]) > 0 and np.count_nonzero(g["C"]) < g["C"].size


def test_soft_threshold_weights_are_synthesized_noise(oracle):
    """Def. "Coefficient-domain hard-thresholding weighting models" with the
    soft attenuation a_k = C_k / Y_k (variance model, patch scope, white
    noise): R_j = sum_l |V_jl|^2 sum_q |a_lq|^2 sigma^2 equals the trace of the
    noise covariance of synthesized patch j, U A sigma^2 I A U^T, full matrices."""
    sig = 0.2
    _, x, members, rng = _group_setup(oracle, ("gaussian", sig))
    p = _soft_params(oracle, ("gaussian", sig))
    y = x + rng.normal(0, sig, x.shape)
    g = oracle.filter_group(p, 1, y, None, members)
    Y, C = g["Y"].ravel(), g["C"].ravel()
    a = np.where(Y != 0, C / np.where(Y != 0, Y, 1.0), 0.0)
    assert np.any((a > 0) & (a < 1))
    U = _full_T(oracle, 4, (4, 4)).T
    cov = U @ np.diag(a) @ (sig ** 2 * np.eye(64)) @ np.diag(a) @ U.T
    R = np.array([np.trace(cov[j * 16:(j + 1) * 16, j * 16:(j + 1) * 16]) for j in range(4)])
    np.testing.assert_allclose(g["w"], 1.0 / R, rtol=1e-12)


def test_soft_classic_group_weight(oracle):
    """Classic group-scope surrogate under soft attenuation: R = sum_k |a_k|^2."""
    _, x, members, rng = _group_setup(oracle, ("poisson", 0.1))
    p = _soft_params(oracle, ("poisson", 0.1), weight_model="classic", weight_scope="group")
    y = rng.poisson(x / 0.1) * 0.1
    g = oracle.filter_group(p, 1, y, None, members)
    Y, C = g["Y"].ravel(), g["C"].ravel()
    a = np.where(Y != 0, C / np.where(Y != 0, Y, 1.0), 0.0)
    np.testing.assert_allclose(g["w"], 1.0 / np.sum(a * a), rtol=1e-12)


def test_soft_identity_at_zero_threshold(oracle):
    """lambda_HT = 0: the soft rule keeps every coefficient unchanged, so the
    first stage returns the observation (as the hard rule does)."""
    rng = np.random.default_rng(5)
    y = rng.uniform(0, 1, size=(24, 20))
    p = oracle.params(y.shape, (4, 4), (2, 2), (7, 7), ("gaussian", 0.0), (8, 16), lambda_ht=0.0, ht_rule="soft")
    out, pilot = oracle.denoise(p, y)
    np.testing.assert_allclose(pilot, y, atol=1e-12)


def test_soft_shrinks_at_least_as_much_as_hard(oracle):
    """|C_soft| <= |C_hard| coefficient by coefficient, and they share their
    zero set away from the threshold."""
    _, x, members, rng = _group_setup(oracle, ("poisson", 0.1))
    y = rng.poisson(x / 0.1) * 0.1
    gh = oracle.filter_group(oracle.params((16, 16), (4, 4), (2, 2), (7, 7), ("poisson", 0.1), (8, 8)),
                             1, y, None, members)
    gs = oracle.filter_group(_soft_params(oracle, ("poisson", 0.1)), 1, y, None, members)
    assert np.all(np.abs(gs["C"]) <= np.abs(gh["C"]) + 1e-15)
    thr = 3.0 * np.sqrt(gh["var"])
    clear = np.abs(np.abs(gh["Y"]) - thr) > 1e-3 * thr
    np.testing.assert_array_equal((gs["C"] != 0)[clear], (gh["C"] != 0)[clear])


# ---------------------------------------------------------------------------
# windowed synthesized-domain weights (Sec. 7.3)
# ---------------------------------------------------------------------------

def _windowed_R(oracle, g, members, F, S2, extra=None, scope="patch"):
    """tr(H F Sigma F^H) (+ extra) with H = U^H Q_j^H W_p^H W_p Q_j U built from
    full matrices (Def. "Windowed synthesis metrics", Def. "Windowed
    synthesized-domain weighting models"): U = T^T (scipy DCT, hand Haar),
    W_p the Kaiser window (numpy, beta = 2)."""
    n, P = 4, 16
    U = _full_T(oracle, n, (4, 4)).T
    w1 = np.kaiser(4, 2.0)
    wp = np.outer(w1, w1).ravel()
    M = np.diag(F) @ np.diag(S2) @ np.diag(F)
    if extra is not None:
        M = M + extra
    R = []
    for j in range(n):
        Q = np.zeros((P, n * P))
        Q[:, j * P:(j + 1) * P] = np.eye(P)
        L = np.diag(wp) @ Q @ U
        R.append(np.trace(L.T @ L @ M))
    R = np.array(R)
    return R if scope == "patch" else np.full(n, R.sum())


@pytest.mark.parametrize("scope", ["patch", "group"])
@pytest.mark.parametrize("rule", ["hard", "soft"])
def test_windowed_ht_weights_full_matrices(oracle, scope, rule):
    """Hard or soft thresholding, variance model: R = tr(H A Sigma A^H)."""
    _, x, members, rng = _group_setup(oracle, ("poisson", 0.1))
    p = oracle.params((16, 16), (4, 4), (2, 2), (7, 7), ("poisson", 0.1), (8, 8), ht_rule=rule,
                      weight_domain="windowed_synthesis", weight_scope=scope)
    y = rng.poisson(x / 0.1) * 0.1
    g = oracle.filter_group(p, 1, y, None, members)
    Y, C, S2 = g["Y"].ravel(), g["C"].ravel(), g["var"].ravel()
    a = np.where(Y != 0, C / np.where(Y != 0, Y, 1.0), 0.0)
    R = _windowed_R(oracle, g, members, a, S2, scope=scope)
    np.testing.assert_allclose(g["w"], 1.0 / R, rtol=1e-11)


@pytest.mark.parametrize("model", ["classic", "variance", "risk"])
def test_windowed_wiener_weights_full_matrices(oracle, model):
    """Wiener stage: classic tr(H D D^H), variance tr(H D Sigma D^H), risk adds
    tr(H (D - I) diag(S) (D - I)^H) with S = [Gamma^2 - a sigma^2]_+ (classic
    pilot power, a = 0)."""
    sig = 0.15
    shape = (16, 16)
    rng = np.random.default_rng(3)
    x = rng.uniform(0.1, 1.0, size=shape)
    y = x + rng.normal(0, sig, shape)
    pilot = x + rng.normal(0, 0.05, shape)
    p = oracle.params(shape, (4, 4), (2, 2), (7, 7), ("gaussian", sig), (8, 8), weight_model=model,
                      weight_domain="windowed_synthesis")
    members = np.array([np.ravel_multi_index(c, shape) for c in [(3, 3), (5, 4), (0, 9), (10, 2)]])
    g = oracle.filter_group(p, 2, y, pilot, members)
    offs = [np.ravel_multi_index((i, j), shape) for i in range(4) for j in range(4)]
    T = _full_T(oracle, 4, (4, 4))
    gam = T @ pilot.ravel()[np.array([[m + o for o in offs] for m in members]).ravel()]
    s2 = np.full(64, sig ** 2)
    S = np.maximum(gam ** 2, 0.0)
    G = S / (S + 0.4 * s2)
    np.testing.assert_allclose(g["C"].ravel(), G * g["Y"].ravel(), atol=1e-12)
    if model == "classic":
        R = _windowed_R(oracle, g, members, G, np.ones(64))
    elif model == "variance":
        R = _windowed_R(oracle, g, members, G, s2)
    else:
        R = _windowed_R(oracle, g, members, G, s2, extra=np.diag((G - 1) ** 2 * S))
    np.testing.assert_allclose(g["w"], 1.0 / R, rtol=1e-11)


def test_windowed_equals_coefficient_domain_with_flat_window(oracle):
    """With a constant window (Kaiser beta = 0) and a unitary U, H = I and the
    windowed models reduce to the coefficient-domain ones (the remark closing
    Sec. 7.3)."""
    _, x, members, rng = _group_setup(oracle, ("poisson", 0.1))
    y = rng.poisson(x / 0.1) * 0.1
    kw = dict(kaiser_beta=0.0)
    pc = oracle.params((16, 16), (4, 4), (2, 2), (7, 7), ("poisson", 0.1), (8, 8), **kw)
    pw = oracle.params((16, 16), (4, 4), (2, 2), (7, 7), ("poisson", 0.1), (8, 8),
                       weight_domain="windowed_synthesis", **kw)
    np.testing.assert_allclose(oracle.filter_group(pw, 1, y, None, members)["w"],
                               oracle.filter_group(pc, 1, y, None, members)["w"], rtol=1e-12)


# ---------------------------------------------------------------------------
# reference coverage of a schedule (Sec. 9.3, "Shift Schedule Analysis")
# ---------------------------------------------------------------------------

def test_coverage_off_schedule_by_hand(oracle):
    """Def. "Off reference schedule" on 8 samples, patch 3, step 2: origins
    0, 2, 4 and the appended l = 5; C(x) counted by hand."""
    cov, n, cv = oracle.coverage(oracle.params((8,), (3,), (2,), (1,), schedule="off"))
    assert n == 4
    np.testing.assert_array_equal(cov, [1, 1, 2, 1, 2, 2, 2, 1])
    assert cv == pytest.approx(1 / 3, rel=1e-15)


def test_coverage_off_schedule_is_separable(oracle):
    """The off schedule is the product of the per-axis lattices, so its 2-D
    coverage is the outer product of the 1-D coverages."""
    c2, n2, _ = oracle.coverage(oracle.params((23, 17), (5, 4), (3, 2), (1, 1), schedule="off"))
    ca, na, _ = oracle.coverage(oracle.params((23,), (5,), (3,), (1,), schedule="off"))
    cb, nb, _ = oracle.coverage(oracle.params((17,), (4,), (2,), (1,), schedule="off"))
    assert n2 == na * nb
    np.testing.assert_array_equal(c2, np.outer(ca, cb))


@pytest.mark.parametrize("sched,rho,K", [("generated", 2.0, 2), ("balanced", 2.0, 2), ("sparse", 1.0, 1),
                                         ("generated", 4.0, 1), ("balanced", 4.0, 2)])
def test_coverage_counts_every_patch_once(oracle, sched, rho, K):
    """Sum of C(x) = |R| P (each reference covers its P entries once); the
    CV equals numpy's population std / mean of the map.  Two passes cover
    every location; one pass with shifts wider than the step can leave a
    gap before the clipped far origin l_d (Def. "Clipped reference origin"),
    as it does here for rho = 4, K = 1 at one location."""
    shape, patch = (41, 37), (8, 8)
    p = oracle.params(shape, patch, (3, 3), (1, 1), schedule=sched, shift_density=rho, passes=K)
    cov, n, cv = oracle.coverage(p)
    assert n == len(oracle.schedule(p))
    assert int(cov.sum()) == n * 64
    assert cv == pytest.approx(cov.std() / cov.mean(), rel=1e-12)
    if K == 2:
        assert cov.min() >= 1
    elif (sched, rho) == ("generated", 4.0):
        assert np.argwhere(cov == 0).tolist() == [[32, 23]]


def test_schedule_analysis_statements(oracle):
    """Sec. 9.3 statements on 2-D shapes of the paper's test sets (8x8
    patches, step 3): the sparse schedule generates the same origins as the
    generated one when no axis is a singleton, and balanced (2, 2) has the
    most uniform coverage (lowest CV) of the configurations compared; no
    shifts (shift density 0) reduce to the off lattice."""
    shapes = [(481, 321), (256, 256)]
    def stats(sched, rho, K):
        out = []
        for sh in shapes:
            p = oracle.params(sh, (8, 8), (3, 3), (1, 1), schedule=sched, shift_density=rho, passes=K)
            out.append(oracle.coverage(p)[1:])
        return out
    for sh in shapes:
        g = oracle.schedule(oracle.params(sh, (8, 8), (3, 3), (1, 1), schedule="generated"))
        sp = oracle.schedule(oracle.params(sh, (8, 8), (3, 3), (1, 1), schedule="sparse"))
        np.testing.assert_array_equal(g, sp)
        g0 = oracle.schedule(oracle.params(sh, (8, 8), (3, 3), (1, 1), schedule="generated", shift_density=0.0))
        off = oracle.schedule(oracle.params(sh, (8, 8), (3, 3), (1, 1), schedule="off"))
        np.testing.assert_array_equal(g0, off)
    cv = {c: np.median([s[1] for s in stats(*c)]) for c in
          [("off", 2.0, 1), ("generated", 2.0, 2), ("generated", 1.0, 2), ("balanced", 2.0, 2), ("balanced", 4.0, 2),
           ("balanced", 2.0, 1)]}
    assert min(cv, key=cv.get) == ("balanced", 2.0, 2)


# ---------------------------------------------------------------------------
# partial shared-source variance (Sec. 5, Def. "Partial shared-source
# Poisson variance model")
# ---------------------------------------------------------------------------

def _overlap_members(shape):
    return np.array([np.ravel_multi_index(c, shape) for c in [(3, 3), (4, 3), (3, 5), (5, 4)]])


def test_shared_source_all_planes_equals_full_covariance(oracle):
    """k_ex = n: sigma_k^2 = (T Sigma_g T^T)_kk with (Sigma_g)_ij = m_v(u_i) when
    u_i = u_j and 0 otherwise (Eq. shared-voxel-group-covariance), built with
    full matrices (scipy DCT, hand Haar) from the plug-in m_v = s_P [y]_+."""
    s_p = 0.1
    _, x, _, rng = _group_setup(oracle, ("poisson", s_p))
    y = rng.poisson(x / s_p) * s_p
    members = _overlap_members(x.shape)
    p = oracle.params((16, 16), (4, 4), (2, 2), (7, 7), ("poisson", s_p), (8, 8), cov_planes=4)
    g = oracle.filter_group(p, 1, y, None, members)
    offs = [np.ravel_multi_index((a, b), x.shape) for a in range(4) for b in range(4)]
    u = np.array([[m + o for o in offs] for m in members]).ravel()
    mv = s_p * np.maximum(y.ravel()[u], 0)
    Sigma = np.where(u[:, None] == u[None, :], mv[:, None], 0.0)
    T = _full_T(oracle, 4, (4, 4))
    np.testing.assert_allclose(g["var"].ravel(), np.diag(T @ Sigma @ T.T), rtol=1e-11, atol=1e-14)
    # the hard threshold of the filter uses these variances
    keep = np.abs(g["Y"]) - 3.0 * np.sqrt(g["var"]) > 1e-12 * 3.0 * np.sqrt(g["var"])
    np.testing.assert_array_equal(g["C"], np.where(keep, g["Y"], 0.0))


def test_shared_source_leading_planes_only(oracle):
    """k_ex = 1: plane 0 takes the shared-source variance, planes 1..n-1 keep
    the diagonal model sum_i T_ki^2 m_v(u_i) (Remark "Limiting cases": k_ex = 0
    is the diagonal model)."""
    s_p = 0.1
    _, x, _, rng = _group_setup(oracle, ("poisson", s_p))
    y = rng.poisson(x / s_p) * s_p
    members = _overlap_members(x.shape)
    mk = lambda k: oracle.params((16, 16), (4, 4), (2, 2), (7, 7), ("poisson", s_p), (8, 8), cov_planes=k)
    v0 = oracle.filter_group(mk(0), 1, y, None, members)["var"]
    v1 = oracle.filter_group(mk(1), 1, y, None, members)["var"]
    v4 = oracle.filter_group(mk(4), 1, y, None, members)["var"]
    np.testing.assert_array_equal(v1[1:], v0[1:])
    np.testing.assert_allclose(v1[0], v4[0], rtol=1e-14)
    assert np.max(np.abs(v1[0] / v0[0] - 1)) > 0.1


def test_shared_source_variance_monte_carlo(oracle):
    """On overlapping patches, where the diagonal model visibly misses, the
    shared-source model with the exact clean mean as surrogate is the
    variance of the transformed Poisson group (20000 draws)."""
    s_p = 0.05
    _, x, _, rng = _group_setup(oracle, ("poisson", s_p))
    members = _overlap_members(x.shape)
    offs = [np.ravel_multi_index((a, b), x.shape) for a in range(4) for b in range(4)]
    idx = np.array([[m + o for o in offs] for m in members]).ravel()
    p = oracle.params((16, 16), (4, 4), (2, 2), (7, 7), ("poisson", s_p), (8, 8), cov_planes=4)
    Ys = []
    for _ in range(40):
        yy = rng.poisson(x[None] / s_p, size=(500,) + x.shape) * s_p
        grp = yy.reshape(500, -1)[:, idx].reshape(500, 4, 4, 4)
        Ys.append(np.stack([oracle.group_transform(p, gi, 0).ravel() for gi in grp]))
    emp = np.concatenate(Ys).var(axis=0, ddof=1)
    var = oracle.filter_group(p, 1, x, None, members)["var"].ravel()
    big = var > 0.05 * var.max()
    np.testing.assert_allclose(emp[big], var[big], rtol=0.08)


def test_ssd_is_the_exact_sum_rounded_once(oracle):
    """Eq. (ssd) with exact summation: the oracle's score of every candidate
    equals the exact rational SSD of the float32 inputs rounded once to
    double (fractions.Fraction), on data spanning 2^-20 to 2^4, where the
    squares need more than 53 bits and a sum of rounded squares would miss."""
    from fractions import Fraction
    rng = np.random.default_rng(17)
    y = (rng.uniform(0, 16, 24) * np.where(rng.uniform(size=24) < 0.3, 2.0 ** -24, 1.0)).astype(np.float32)
    yd = y.astype(np.float64)
    p = oracle.params(y.shape, (4,), (1,), (21,), ("gaussian", 0.0), (16, 16), gamma_ht=0.0, tau_ht=1e30,
                      group_transform="dct")
    mem, sc = oracle.match_ref(p, yd, 1, 10)
    misses = 0
    for m, s in zip(mem[1:], sc[1:]):
        exact = sum((Fraction(float(yd[m + i])) - Fraction(float(yd[10 + i]))) ** 2 for i in range(4))
        assert s == float(exact), (m, s, float(exact))
        rounded = 0.0
        for i in range(4):
            rounded += (yd[m + i] - yd[10 + i]) ** 2
        misses += rounded != float(exact)
    assert misses > 0


# ---------------------------------------------------------------------------
# bior1.5 spatial transform of the hard-threshold stage (App. A)
# ---------------------------------------------------------------------------

def _bior_hand(n):
    """bior1.5 analysis matrices derived by hand (periodic, full depth,
    coarsest first).  n = 2 and n = 4: the wrapped lowpass taps pair up to the
    Haar filter, so the matrix is the Haar matrix.  n = 8: the level-1
    approximations are a1[i] = (x[2i] + x[2i+1] + c (x[2i+2] - x[2i+3]
    - x[2i-2] + x[2i-1])) / sqrt 2 with c = 22/128 (indices mod 8; the taps
    +-3/128 cancel on a period of 8), and the coarser levels are Haar steps
    on them."""
    r2 = math.sqrt(2.0)
    if n == 2:
        return np.array([[1, 1], [1, -1]]) / r2
    if n == 4:
        return np.array([[.5, .5, .5, .5], [.5, .5, -.5, -.5], [1 / r2, -1 / r2, 0, 0], [0, 0, 1 / r2, -1 / r2]])
    c = 11.0 / 64.0
    T = np.zeros((8, 8))
    T[0] = 1 / math.sqrt(8)
    T[1] = np.array([1 - 2 * c, 1 + 2 * c, 1 + 2 * c, 1 - 2 * c, -1 + 2 * c, -1 - 2 * c, -1 - 2 * c, -1 + 2 * c]) / (2 * r2)
    T[2] = np.array([1 + c, 1 - c, c - 1, -c - 1, -c, c, -c, c]) / 2
    T[3] = np.array([-c, c, -c, c, 1 + c, 1 - c, c - 1, -c - 1]) / 2
    for i in range(4):
        T[4 + i, 2 * i], T[4 + i, 2 * i + 1] = 1 / r2, -1 / r2
    return T


@pytest.mark.parametrize("n", [2, 4, 8])
def test_bior15_hand_values(oracle, n):
    """App. A's bior1.5 on periodic patch axes of 2, 4 and 8 samples against
    the hand derivation above."""
    np.testing.assert_allclose(oracle.bior15_matrix(n), _bior_hand(n), atol=1e-15)


@pytest.mark.parametrize("n", [2, 4, 8, 16, 32])
def test_bior15_perfect_reconstruction(oracle, n):
    """The synthesis cascade (from the synthesis filters alone) inverts the
    analysis cascade on both sides: U T = T U = I, the biorthogonality of the
    pair; T is not orthonormal for n >= 8 (rows of norm != 1)."""
    T, U = oracle.bior15_matrix(n), oracle.bior15_synthesis(n)
    np.testing.assert_allclose(U @ T, np.eye(n), atol=1e-13)
    np.testing.assert_allclose(T @ U, np.eye(n), atol=1e-13)
    if n >= 8:
        assert np.max(np.abs(np.linalg.norm(T, axis=1) - 1)) > 0.02
        assert np.max(np.abs(U - T.T)) > 0.05
    # DC row 1/sqrt n; every detail row annihilates constants
    np.testing.assert_allclose(T[0], 1 / math.sqrt(n), atol=1e-15)
    np.testing.assert_allclose(T[1:].sum(axis=1), 0.0, atol=1e-14)


def test_bior15_synthesis_wavelet_vanishing_moments(oracle):
    """The family's defining property (N~ = 5): the synthesis highpass g has
    five vanishing moments, sum_k g[k] k^p = 0 for p = 0..4 (and not for
    p = 5).  g is read from the synthesis matrix of a 32-sample axis: the
    column of the finest detail d_1[j] holds g[k] at 2j + k, k = -4..5."""
    U = oracle.bior15_synthesis(32)
    j = 8
    col = U[:, 16 + j]
    k = np.arange(-4, 6)
    g = col[2 * j + k]
    assert np.count_nonzero(np.abs(col) > 1e-15) == 10
    mom = [np.sum(g * k.astype(float) ** p) for p in range(6)]
    np.testing.assert_allclose(mom[:5], 0.0, atol=1e-13)
    assert abs(mom[5]) > 1.0
    # and the synthesis lowpass is the box: the column of a_m is constant
    np.testing.assert_allclose(U[:, 0], 1 / math.sqrt(32), atol=1e-15)


def _bior_group(oracle, **kw):
    rng = np.random.default_rng(21)
    x = rng.uniform(0.1, 1.0, size=(24, 24))
    s_p = 0.05
    y = rng.poisson(x / s_p) * s_p
    p = oracle.params((24, 24), (8, 8), (3, 3), (9, 9), ("poisson", s_p), (8, 8), spatial_transform="bior1.5", **kw)
    members = np.array([np.ravel_multi_index(c, (24, 24)) for c in [(3, 3), (5, 12), (14, 1), (10, 10)]])
    offs = [np.ravel_multi_index((a, b), (24, 24)) for a in range(8) for b in range(8)]
    u = np.array([[m + o for o in offs] for m in members]).ravel()
    A = _bior_hand(8)
    T = np.kron(oracle.haar_matrix(4), np.kron(A, A))
    return p, y, members, u, T, s_p


def test_bior15_group_coefficients_and_variances(oracle):
    """Stage 1 with the bior1.5 spatial transform: Y = T y_g and sigma_k^2 =
    sum_i T_ki^2 m_v(u_i) (Lemma "Covariance propagation", Prop. "Diagonal
    Poisson variance propagation") with T = Haar (x) A (x) A from the hand
    matrix A; at lambda = 0 the filter returns the group itself (synthesis =
    exact inverse); stage 2 keeps the DCT."""
    p, y, members, u, T, s_p = _bior_group(oracle)
    g = oracle.filter_group(p, 1, y, None, members)
    yg = y.ravel()[u]
    np.testing.assert_allclose(g["Y"].ravel(), T @ yg, atol=1e-12)
    np.testing.assert_allclose(g["var"].ravel(), (T * T) @ (s_p * yg), rtol=1e-12)
    p0, *_ = _bior_group(oracle, lambda_ht=0.0)
    g0 = oracle.filter_group(p0, 1, y, None, members)
    np.testing.assert_allclose(g0["p"].ravel(), yg, atol=1e-12)
    g2 = oracle.filter_group(p, 2, y, y, members)
    Td = _full_T(oracle, 4, (8, 8))
    np.testing.assert_allclose(g2["Y"].ravel(), Td @ yg, atol=1e-12)


def test_bior15_coefficient_domain_patch_weights(oracle):
    """Variance model, patch scope, with a non-orthonormal spatial transform:
    the coefficient-domain surrogate R_j = sum_l |V_jl|^2 sum_q a_lq
    sigma_lq^2 (Def. "Coefficient-domain hard-thresholding weighting models")
    from the diagonal variances, checked with full matrices."""
    p, y, members, u, T, s_p = _bior_group(oracle)
    g = oracle.filter_group(p, 1, y, None, members)
    a = (g["C"].ravel() != 0).astype(float)
    S2 = (T * T) @ (s_p * y.ravel()[u])
    V = oracle.haar_matrix(4).T
    r = (a * S2).reshape(4, 64).sum(axis=1)
    R = (V * V) @ r
    np.testing.assert_allclose(g["w"], 1.0 / R, rtol=1e-12)


@pytest.mark.parametrize("scope", ["patch", "group"])
def test_bior15_windowed_weights_full_matrices(oracle, scope):
    """Windowed synthesized-domain weights with the bior1.5 synthesis: R =
    tr(H A Sigma A^H), H = U^H Q_j^H W_p^H W_p Q_j U with U = the inverse of
    the hand-built T (numpy) and W_p the Kaiser window (numpy, beta 2)."""
    p, y, members, u, T, s_p = _bior_group(oracle, weight_domain="windowed_synthesis", weight_scope=scope)
    g = oracle.filter_group(p, 1, y, None, members)
    a = (g["C"].ravel() != 0).astype(float)
    S2 = (T * T) @ (s_p * y.ravel()[u])
    U = np.linalg.inv(T)
    w1 = np.kaiser(8, 2.0)
    wp = np.outer(w1, w1).ravel()
    Mx = np.diag(a * S2)
    R = []
    for j in range(4):
        Q = np.zeros((64, 256))
        Q[:, j * 64:(j + 1) * 64] = np.eye(64)
        L = np.diag(wp) @ Q @ U
        R.append(np.trace(L.T @ L @ Mx))
    R = np.array(R) if scope == "patch" else np.full(4, np.sum(R))
    np.testing.assert_allclose(g["w"], 1.0 / R, rtol=1e-11)


def test_bior15_identity_and_mass_conservation(oracle):
    """Whole denoiser with the bior1.5 stage-1 transform: identity at sigma =
    0, lambda = 0 (exact synthesis); Thm. "Mass conservation after normalized
    overlap-add" with the two-sweep correction, whose residual needs the
    synthesis adjoint U^T, not T (Def. "Aggregation-aware constant-synthesis
    correction")."""
    rng = np.random.default_rng(9)
    y = rng.uniform(0, 1, size=(26, 30))
    p = oracle.params(y.shape, (8, 8), (3, 3), (9, 9), ("gaussian", 0.0), (8, 16), lambda_ht=0.0,
                      spatial_transform="bior1.5")
    out, pilot = oracle.denoise(p, y)
    np.testing.assert_allclose(pilot, y, atol=1e-12)
    x = synth.disc_rect_image((30, 28), rng)
    yp = rng.poisson(x / 0.2) * 0.2
    p = oracle.params(yp.shape, (8, 8), (3, 3), (9, 9), ("poisson", 0.2), (8, 16), mass_conserve=3,
                      spatial_transform="bior1.5")
    out, pilot = oracle.denoise(p, yp)
    assert pilot.sum() == pytest.approx(yp.sum(), rel=1e-12)
    assert out.sum() == pytest.approx(yp.sum(), rel=1e-12)
    p0 = oracle.params(yp.shape, (8, 8), (3, 3), (9, 9), ("poisson", 0.2), (8, 16), mass_conserve=3)
    out0, pilot0 = oracle.denoise(p0, yp)
    assert np.max(np.abs(pilot - pilot0)) > 1e-3


def test_bior15_shared_source_all_planes(oracle):
    """Partial shared-source variance with the bior1.5 spatial factors: with
    every plane exact, sigma_k^2 = (T Sigma_g T^T)_kk for the repeated-voxel
    covariance (Eq. shared-voxel-group-covariance), full matrices from the
    hand-built T."""
    p, y, _, _, _, s_p = _bior_group(oracle, cov_planes=4)
    members = np.array([np.ravel_multi_index(c, (24, 24)) for c in [(3, 3), (4, 5), (6, 3), (9, 9)]])
    offs = [np.ravel_multi_index((a, b), (24, 24)) for a in range(8) for b in range(8)]
    u = np.array([[m + o for o in offs] for m in members]).ravel()
    A = _bior_hand(8)
    T = np.kron(oracle.haar_matrix(4), np.kron(A, A))
    g = oracle.filter_group(p, 1, y, None, members)
    mv = s_p * np.maximum(y.ravel()[u], 0)
    Sigma = np.where(u[:, None] == u[None, :], mv[:, None], 0.0)
    np.testing.assert_allclose(g["var"].ravel(), np.diag(T @ Sigma @ T.T), rtol=1e-11, atol=1e-14)
