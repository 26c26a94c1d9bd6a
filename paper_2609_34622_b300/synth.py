"""Seeded synthetic inputs and workload definitions.

This module holds no step of the denoiser: it only draws clean signals and
their noisy observations, and names the five workloads with their parameters.
Both the CUDA path's tests/benchmark and the FP64 oracle's tests take their
inputs from here.

Noise conventions follow the paper's experiment section ("Noise Models"):
clean intensities x in [0, 1]; Gaussian observations y = x + n with
sigma = sigma_255 / 255; scaled-Poisson observations K ~ Poi(lambda_pk x) and
y = s_P K with s_P = 1 / lambda_pk.

The generators are stand-ins for the paper's datasets (generated 2-D/3-D
images, natural images, fluorescence microscopy, MIT-BIH ECG), none of which
is reproduced here.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np


def rng_for(config: int, item: int = 0) -> np.random.Generator:
    """Seed = 1000 * config + item (PCG64)."""
    return np.random.Generator(np.random.PCG64(1000 * config + item))


# --------------------------------------------------------------------------
# clean signals
# --------------------------------------------------------------------------

def disc_rect_image(shape=(64, 64), rng=None) -> np.ndarray:
    """Piecewise-constant discs and rectangles over a smooth gradient, in [0, 1]."""
    rng = rng or np.random.default_rng(0)
    H, W = shape
    yy, xx = np.meshgrid(np.arange(H) / max(H - 1, 1), np.arange(W) / max(W - 1, 1), indexing="ij")
    a, b = rng.uniform(-0.25, 0.25, size=2)
    img = 0.35 + a * yy + b * xx
    for _ in range(int(rng.integers(3, 7))):
        cy, cx = rng.uniform(0, H), rng.uniform(0, W)
        rad = rng.uniform(0.06, 0.22) * min(H, W)
        img = np.where((yy * (H - 1) - cy) ** 2 + (xx * (W - 1) - cx) ** 2 <= rad ** 2, rng.uniform(0.05, 0.95), img)
    for _ in range(int(rng.integers(3, 7))):
        y0, x0 = rng.uniform(0, H), rng.uniform(0, W)
        h, w = rng.uniform(0.1, 0.4) * H, rng.uniform(0.1, 0.4) * W
        m = (yy * (H - 1) >= y0) & (yy * (H - 1) < y0 + h) & (xx * (W - 1) >= x0) & (xx * (W - 1) < x0 + w)
        img = np.where(m, rng.uniform(0.05, 0.95), img)
    return np.clip(img, 0.0, 1.0)


def ecg_signal(n=262144, fs=250.0, rng=None) -> np.ndarray:
    """ECG-shaped pulse train: Gaussian P, Q, R, S and T waves per beat, beat
    rate drawn from 60-100 bpm with per-beat jitter, plus baseline wander;
    offset and scaled to [0.02, 1]."""
    rng = rng or np.random.default_rng(0)
    t = np.arange(n) / fs
    sig = np.zeros(n)
    waves = [(-0.20, 0.12, 0.025), (-0.035, -0.12, 0.010), (0.0, 1.0, 0.012),
             (0.035, -0.25, 0.012), (0.28, 0.30, 0.045)]
    tb = rng.uniform(0.2, 0.8)
    hr = rng.uniform(60, 100)
    while tb < t[-1] + 1.0:
        amp = rng.uniform(0.85, 1.15)
        c0 = int(tb * fs)
        lo, hi = max(c0 - int(0.5 * fs), 0), min(c0 + int(0.7 * fs), n)
        if lo < hi:
            tt = t[lo:hi] - tb
            for (mu, a, s) in waves:
                sig[lo:hi] += amp * a * np.exp(-0.5 * ((tt - mu) / s) ** 2)
        hr = float(np.clip(hr + rng.normal(0, 2.0), 60, 100))
        tb += 60.0 / hr * rng.uniform(0.95, 1.05)
    wander = 0.15 * np.sin(2 * np.pi * rng.uniform(0.15, 0.35) * t + rng.uniform(0, 2 * np.pi))
    wander += 0.05 * np.sin(2 * np.pi * rng.uniform(0.02, 0.06) * t + rng.uniform(0, 2 * np.pi))
    sig += wander
    sig = (sig - sig.min()) / (sig.max() - sig.min())
    return 0.02 + 0.98 * sig


def texture_edge_image(shape=(512, 512), rng=None) -> np.ndarray:
    """Procedural texture (modulated oriented sinusoids) plus piecewise-constant
    regions with sharp edges, in [0, 1]."""
    rng = rng or np.random.default_rng(0)
    H, W = shape
    yy, xx = np.meshgrid(np.arange(H, dtype=np.float64), np.arange(W, dtype=np.float64), indexing="ij")
    img = np.zeros(shape)
    for _ in range(4):
        th = rng.uniform(0, np.pi)
        f = rng.uniform(0.02, 0.25)
        env = 0.5 + 0.5 * np.cos(2 * np.pi * (rng.uniform(0.001, 0.004) * xx + rng.uniform(0.001, 0.004) * yy)
                                 + rng.uniform(0, 2 * np.pi))
        img += rng.uniform(0.05, 0.15) * env * np.sin(2 * np.pi * f * (np.cos(th) * xx + np.sin(th) * yy)
                                                     + rng.uniform(0, 2 * np.pi))
    base = np.full(shape, rng.uniform(0.3, 0.6))
    for _ in range(int(rng.integers(5, 10))):
        # half-planes and rectangles with constant offsets
        if rng.uniform() < 0.5:
            th = rng.uniform(0, 2 * np.pi)
            c = rng.uniform(0.2, 0.8) * np.array([H, W])
            m = (np.cos(th) * (yy - c[0]) + np.sin(th) * (xx - c[1])) > 0
        else:
            y0, x0 = rng.uniform(0, H), rng.uniform(0, W)
            h, w = rng.uniform(0.05, 0.3) * H, rng.uniform(0.05, 0.3) * W
            m = (yy >= y0) & (yy < y0 + h) & (xx >= x0) & (xx < x0 + w)
        base = np.where(m, base + rng.uniform(-0.25, 0.25), base)
    img = base + img
    img = (img - img.min()) / (img.max() - img.min())
    return img


def ellipsoid_phantom(shape=(128, 128, 128), rng=None, lo=0.5, hi=5.0) -> np.ndarray:
    """Event-rate field (counts per voxel) made of random ellipsoids with rates
    in [lo, hi] over a background of rate lo."""
    rng = rng or np.random.default_rng(0)
    grids = np.meshgrid(*[np.arange(n, dtype=np.float64) for n in shape], indexing="ij")
    lam = np.full(shape, lo)
    for _ in range(int(rng.integers(10, 20))):
        c = [rng.uniform(0.15, 0.85) * n for n in shape]
        r = [rng.uniform(0.05, 0.3) * n for n in shape]
        q = sum(((g - ci) / ri) ** 2 for g, ci, ri in zip(grids, c, r))
        lam = np.where(q <= 1.0, rng.uniform(lo, hi), lam)
    return lam


# --------------------------------------------------------------------------
# noise
# --------------------------------------------------------------------------

def poisson_observe(x: np.ndarray, lam_pk: float, rng) -> tuple[np.ndarray, float]:
    """K ~ Poi(lam_pk x), y = K / lam_pk; returns (y float32, s_P)."""
    k = rng.poisson(lam_pk * np.clip(x, 0.0, None))
    s_p = 1.0 / lam_pk
    return (k * s_p).astype(np.float32), s_p


def gaussian_observe(x: np.ndarray, sigma: float, rng) -> np.ndarray:
    return (x + rng.normal(0.0, sigma, size=x.shape)).astype(np.float32)


# --------------------------------------------------------------------------
# workloads
# --------------------------------------------------------------------------

@dataclass
class Job:
    """One denoising problem: observation, clean signal and parameters."""
    y: np.ndarray
    x: np.ndarray
    noise: tuple
    patch: tuple
    step: tuple
    search: tuple
    group_size: tuple = (16, 32)
    stages: int = 2
    mass_conserve: int = 0
    peak: float = 1.0
    name: str = ""

    @property
    def cfg(self) -> dict:
        return dict(noise=self.noise, patch=self.patch, step=self.step, search=self.search,
                    group_size=self.group_size, stages=self.stages, mass_conserve=self.mass_conserve)


def config1(item=0) -> Job:
    """2-D 64x64, discs/rectangles over a gradient, peak 10, Poisson; 8x8, step 3,
    search 19x19, groups 16/32, both stages, no mass conservation."""
    rng = rng_for(1, item)
    x = disc_rect_image((64, 64), rng)
    y, s_p = poisson_observe(x, 10.0, rng)
    return Job(y, x, ("poisson", s_p), (8, 8), (3, 3), (19, 19), (16, 32), 2, 0, 1.0, "c1-2d-64")


def config2(item=0, n=262144) -> Job:
    """1-D ECG-like signal of 262144 samples, peak 50, Poisson; patch 32, step 4,
    search 129, groups 16/32, both stages."""
    rng = rng_for(2, item)
    x = ecg_signal(n, 250.0, rng)
    y, s_p = poisson_observe(x, 50.0, rng)
    return Job(y, x, ("poisson", s_p), (32,), (4,), (129,), (16, 32), 2, 0, 1.0, "c2-1d-262144")


C3_PEAKS = (1.0, 2.0, 5.0, 10.0, 30.0)


def config3(n_images=16, size=512) -> list[Job]:
    """16 images of 512x512 (textures plus edges) with Poisson peaks cycled over
    {1,2,5,10,30}, plus the same images with Gaussian sigma = 25/255; 8x8,
    step 3, search 39x39, groups 16/32, both stages."""
    jobs = []
    xs = [texture_edge_image((size, size), rng_for(3, i)) for i in range(n_images)]
    for i, x in enumerate(xs):
        rng = rng_for(3, 100 + i)
        pk = C3_PEAKS[i % len(C3_PEAKS)]
        y, s_p = poisson_observe(x, pk, rng)
        jobs.append(Job(y, x, ("poisson", s_p), (8, 8), (3, 3), (39, 39), (16, 32), 2, 0, 1.0,
                        "c3-poisson-%d" % i))
    for i, x in enumerate(xs):
        rng = rng_for(3, 200 + i)
        sig = 25.0 / 255.0
        jobs.append(Job(gaussian_observe(x, sig, rng), x, ("gaussian", sig), (8, 8), (3, 3), (39, 39),
                        (16, 32), 2, 0, 1.0, "c3-gauss-%d" % i))
    return jobs


def config4(item=0, n=128) -> Job:
    """3-D 128^3 ellipsoid phantom with 0.5-5 counts per voxel, Poisson; 4x4x4,
    step 2, search 11x11x11, groups 16/32, both stages with mass conservation."""
    rng = rng_for(4, item)
    lam = ellipsoid_phantom((n, n, n), rng)
    s_p = 1.0 / float(lam.max())
    k = rng.poisson(lam)
    y = (k * s_p).astype(np.float32)
    return Job(y, lam * s_p, ("poisson", s_p), (4, 4, 4), (2, 2, 2), (11, 11, 11), (16, 32), 2, 3,
               1.0, "c4-3d-128")


@dataclass
class Request:
    arrival_s: float
    job: Job


def config5(n_requests=512, rate=200.0, seed_item=0) -> list[Request]:
    """Serving mix: Poisson-process arrivals at 200 req/s; 40% 1-D (8k-262k
    samples), 45% 2-D (64^2-1024^2), 15% 3-D (32^3-128^3); Poisson peaks
    log-uniform in [1, 50]; parameters of configs 2 / 1 / 4 by dimension."""
    rng = rng_for(5, seed_item)
    t = 0.0
    reqs = []
    for i in range(n_requests):
        t += rng.exponential(1.0 / rate)
        u = rng.uniform()
        pk = float(math.exp(rng.uniform(math.log(1.0), math.log(50.0))))
        r2 = rng_for(5, 1000 + i)
        if u < 0.40:
            n = int(round(math.exp(rng.uniform(math.log(8192), math.log(262144)))))
            x = ecg_signal(n, 250.0, r2)
            y, s_p = poisson_observe(x, pk, r2)
            job = Job(y, x, ("poisson", s_p), (32,), (4,), (129,), (16, 32), 2, 0, 1.0, "req%d-1d" % i)
        elif u < 0.85:
            s = int(round(math.exp(rng.uniform(math.log(64), math.log(1024)))))
            x = disc_rect_image((s, s), r2)
            y, s_p = poisson_observe(x, pk, r2)
            job = Job(y, x, ("poisson", s_p), (8, 8), (3, 3), (19, 19), (16, 32), 2, 0, 1.0, "req%d-2d" % i)
        else:
            s = int(round(math.exp(rng.uniform(math.log(32), math.log(128)))))
            lam = ellipsoid_phantom((s, s, s), r2)
            x = lam / lam.max()
            y, s_p = poisson_observe(x, pk, r2)
            job = Job(y, x, ("poisson", s_p), (4, 4, 4), (2, 2, 2), (11, 11, 11), (16, 32), 2, 0, 1.0,
                      "req%d-3d" % i)
        reqs.append(Request(t, job))
    return reqs


def psnr(x: np.ndarray, ref: np.ndarray, peak: float = 1.0) -> float:
    mse = float(np.mean((np.asarray(x, np.float64) - np.asarray(ref, np.float64)) ** 2))
    return 10.0 * math.log10(peak * peak / mse) if mse > 0 else float("inf")
