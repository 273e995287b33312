"""Seeded synthetic inputs for sparse w-projection imaging.

This module only draws random inputs (sky images, (u, v, w) baselines, noise).
It holds none of the imaging method's arithmetic, so both the FP64 oracle tests
and the CUDA path can take their inputs from it.

Set-up follows Section 4.1 of Wolz et al. 2013 (arXiv:1307.3424):
  * field of view: opening angle 2 deg, planar FoV L = 2 sin(theta/2);
  * band limit of an N-pixel image: B = N / (2L);
  * w in the paper's normalised unit w_d = w L^2 / N, so w = w_d N / L^2;
  * i.i.d. Gaussian noise with sigma_n = 10^(-SNR_in/20) * std(x), SNR_in = 30 dB.
The paper's test images (M31, 30Dor) are not available; a sum of Gaussian
blobs stands in for them (amplitudes U[0,1], widths U[1,4] px).

Random numbers are drawn from numpy.random.Generator(PCG64(seed)) in the fixed
order sky -> uv -> w -> noise.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

THETA_DEG = 2.0


def fov_L(theta_deg: float = THETA_DEG) -> float:
    """Planar field of view L = 2 sin(theta/2) (Section 4.1)."""
    return 2.0 * math.sin(math.radians(theta_deg) / 2.0)


def band_limit(N: int, L: float) -> float:
    """B = N / (2L) (Section 4.1)."""
    return N / (2.0 * L)


def w_from_wd(wd, N: int, L: float):
    """Invert w_d = w L^2 / N (Section 4.1)."""
    return np.asarray(wd, dtype=np.float64) * N / (L * L)


@dataclass
class Workload:
    name: str
    N: int
    n_blobs: int
    M: int
    uv: str = "uniform"          # "uniform" disk or "gaussian" (sigma_uv * B, truncated to the disk)
    sigma_uv: float = 0.25
    wd_max: float = 1.0
    e: float = 0.99
    W: int = 4
    dr_iters: int = 50
    inner_iters: int = 10
    snr_in_db: float = 30.0
    powerlaw: bool = False
    w_unit: str = "wd"       # "wd": w = w_d N / L^2;  "cells": chirp half-band h = 2 w_c cells, w = h / L^2
    box: str = "G"           # kernel box: "G" (exact) or "rule" (S(w))
    extra: dict = field(default_factory=dict)


# Small case the oracle finishes in seconds: 64x64, 20 blobs, M = 0.3 N^2.
SMALL = Workload("blobs64_m1229", N=64, n_blobs=20, M=1229, uv="uniform",
                 wd_max=1.0, e=0.99, dr_iters=50)
# The paper-scale case: 256x256, 200 blobs, M = 0.5 N^2, radially Gaussian uv.
PAPER_SCALE = Workload("blobs256_m32768", N=256, n_blobs=200, M=32768,
                       uv="gaussian", sigma_uv=0.25, wd_max=1.0, e=0.99,
                       dr_iters=300)
# The precision-form case: 1024x1024, 2000 blobs plus a power-law diffuse part,
# M = 2^21, w_c ~ U[0, 4] grid cells (chirp half-band h = 2 w_c), box rule S(w).
PRECISION = Workload("blobs1024_m2097152", N=1024, n_blobs=2000, M=2 ** 21, uv="uniform",
                     wd_max=4.0, e=0.99, dr_iters=50, powerlaw=True, w_unit="cells", box="rule")


def blob_sky(rng: np.random.Generator, N: int, n_blobs: int) -> np.ndarray:
    """Sum of isotropic Gaussian blobs; centres U[0,N)^2, amplitude U[0,1],
    width (Gaussian sigma in pixels) U[1,4]."""
    cx = rng.uniform(0.0, N, n_blobs)
    cy = rng.uniform(0.0, N, n_blobs)
    amp = rng.uniform(0.0, 1.0, n_blobs)
    sig = rng.uniform(1.0, 4.0, n_blobs)
    x = np.zeros((N, N), dtype=np.float64)
    for b in range(n_blobs):
        # each blob within +-8 sigma of its centre (the rest is below 1e-13 of its peak)
        r = int(np.ceil(8.0 * sig[b]))
        pu = np.arange(max(0, int(cx[b]) - r), min(N, int(cx[b]) + r + 2), dtype=np.float64)
        pv = np.arange(max(0, int(cy[b]) - r), min(N, int(cy[b]) + r + 2), dtype=np.float64)
        gx = np.exp(-((pu - cx[b]) ** 2) / (2.0 * sig[b] ** 2))
        gy = np.exp(-((pv - cy[b]) ** 2) / (2.0 * sig[b] ** 2))
        x[int(pu[0]):int(pu[-1]) + 1, int(pv[0]):int(pv[-1]) + 1] += amp[b] * np.outer(gx, gy)
    return x


def powerlaw_field(rng: np.random.Generator, N: int, exponent: float = -2.5,
                   top: float = 0.1) -> np.ndarray:
    """Gaussian random field with P(k) ~ k^exponent, min-max scaled to [0, top]."""
    k = np.fft.fftfreq(N)
    kk = np.sqrt(k[:, None] ** 2 + k[None, :] ** 2)
    kk[0, 0] = 1.0
    amp = kk ** (exponent / 2.0)
    amp[0, 0] = 0.0
    noise = rng.standard_normal((N, N)) + 1j * rng.standard_normal((N, N))
    f = np.fft.ifft2(noise * amp).real
    f -= f.min()
    return top * f / max(f.max(), 1e-300)


def uv_points(rng: np.random.Generator, M: int, B: float, N: int, kind: str,
              sigma_uv: float = 0.25) -> np.ndarray:
    """(u, v) in wavelengths inside the disk |uv| < B (1 - 1/N)."""
    rmax = B * (1.0 - 1.0 / N)
    if kind == "uniform":
        r = rmax * np.sqrt(rng.uniform(0.0, 1.0, M))
        th = rng.uniform(0.0, 2.0 * np.pi, M)
        return np.stack([r * np.cos(th), r * np.sin(th)], axis=1)
    if kind == "gaussian":
        out = np.empty((0, 2))
        while out.shape[0] < M:
            cand = rng.normal(0.0, sigma_uv * B, (2 * M, 2))
            keep = np.hypot(cand[:, 0], cand[:, 1]) < rmax
            out = np.concatenate([out, cand[keep]], axis=0)
        return out[:M]
    raise ValueError(kind)


def complex_noise(rng: np.random.Generator, M: int, sigma_n: float) -> np.ndarray:
    """Circular complex Gaussian noise, total std sigma_n (sigma_n/sqrt(2) per part)."""
    s = sigma_n / math.sqrt(2.0)
    return s * rng.standard_normal(M) + 1j * s * rng.standard_normal(M)


def noise_sigma(x: np.ndarray, snr_in_db: float) -> float:
    """sigma_n = 10^(-SNR_in/20) * std(x), population std (Section 4.1)."""
    return 10.0 ** (-snr_in_db / 20.0) * float(np.std(x))


@dataclass
class Problem:
    wl: Workload
    L: float
    x: np.ndarray          # N x N float64 sky
    uvw: np.ndarray        # M x 3 float64, wavelengths
    wd: np.ndarray         # M normalised w
    rng: np.random.Generator   # positioned after w; the next draw is the noise


def make_problem(wl: Workload, seed: int = 0, M: int | None = None,
                 wd_const: float | None = None) -> Problem:
    """Draw sky, then uv, then w (the noise is drawn later by `draw_noise`)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    L = fov_L()
    N = wl.N
    M = wl.M if M is None else M
    x = blob_sky(rng, N, wl.n_blobs)
    if wl.powerlaw:
        x = x + powerlaw_field(rng, N)
    B = band_limit(N, L)
    uv = uv_points(rng, M, B, N, wl.uv, wl.sigma_uv)
    if wd_const is None:
        wd = rng.uniform(0.0, wl.wd_max, M)
    else:
        wd = np.full(M, float(wd_const))
    if wl.w_unit == "cells":
        w = 2.0 * wd / (L * L)          # h = 2 w_c cells; h = |w| L^2
    else:
        w = w_from_wd(wd, N, L)
    uvw = np.ascontiguousarray(np.concatenate([uv, w[:, None]], axis=1))
    return Problem(wl, L, x, uvw, wd, rng)


def draw_noise(prob: Problem, M: int | None = None) -> tuple[np.ndarray, float]:
    """Noise for the visibilities of `prob` (drawn after sky, uv and w)."""
    sigma_n = noise_sigma(prob.x, prob.wl.snr_in_db)
    M = prob.uvw.shape[0] if M is None else M
    return complex_noise(prob.rng, M, sigma_n), sigma_n


def random_uvw(rng: np.random.Generator, M: int, N: int, L: float,
               wd_max: float = 1.0) -> np.ndarray:
    """Uniform-disk (u,v) and uniform w_d in [0, wd_max], as an M x 3 array."""
    B = band_limit(N, L)
    uv = uv_points(rng, M, B, N, "uniform")
    w = w_from_wd(rng.uniform(0.0, wd_max, M), N, L)
    return np.ascontiguousarray(np.concatenate([uv, w[:, None]], axis=1))


# The learned-kernel deployment: 2048x2048 (8000 blobs plus the power-law part),
# M = 2^23, w_c ~ U[0, 4] cells, box rule S(w).
LEARNED = Workload("blobs2048_m8388608", N=2048, n_blobs=8000, M=2 ** 23, uv="uniform",
                   wd_max=4.0, e=0.99, dr_iters=50, powerlaw=True, w_unit="cells", box="rule")


# The batched form: many independent problems of uneven size.  Image sides are
# drawn log-uniformly from the powers of two 64 .. 512 (the FFTs are radix 2/4),
# M = f N^2 with f ~ U[0.1, 1], a per-problem w_c,max ~ U[0, 2] cells with
# w_c ~ U[0, w_c,max] per visibility (chirp half-band h = 2 w_c), uniform-disk
# (u, v), blob skies with 20 (N/64)^2 blobs, box rule S(w), e = 0.99.
@dataclass
class BatchWorkload:
    name: str
    n_problems: int
    sides: tuple = (64, 128, 256, 512)
    mfrac: tuple = (0.1, 1.0)
    wc_max: float = 2.0
    e: float = 0.99
    dr_iters: int = 200
    inner_iters: int = 10
    snr_in_db: float = 30.0


BATCHED = BatchWorkload("batch256_n64-512", n_problems=256)


def make_batch(bw: BatchWorkload, seed: int = 0, n_problems: int | None = None,
               max_side: int | None = None) -> list[Problem]:
    """Problems of a batch; problem i is drawn from PCG64(seed * 1_000_003 + i)
    in the order side -> M -> w_c,max -> sky -> uv -> w (noise: draw_noise)."""
    n_problems = bw.n_problems if n_problems is None else n_problems
    sides = [s for s in bw.sides if max_side is None or s <= max_side]
    L = fov_L()
    out = []
    for i in range(n_problems):
        rng = np.random.Generator(np.random.PCG64(seed * 1_000_003 + i))
        N = int(sides[rng.integers(0, len(sides))])
        M = max(1, int(round(rng.uniform(*bw.mfrac) * N * N)))
        wcm = rng.uniform(0.0, bw.wc_max)
        wl = Workload(f"{bw.name}[{i}]", N=N, n_blobs=max(1, 20 * (N // 64) ** 2), M=M, uv="uniform",
                      wd_max=wcm, e=bw.e, dr_iters=bw.dr_iters, inner_iters=bw.inner_iters,
                      snr_in_db=bw.snr_in_db, w_unit="cells", box="rule")
        x = blob_sky(rng, N, wl.n_blobs)
        uv = uv_points(rng, M, band_limit(N, L), N, "uniform")
        wc = rng.uniform(0.0, wcm, M)
        w = 2.0 * wc / (L * L)
        uvw = np.ascontiguousarray(np.concatenate([uv, w[:, None]], axis=1))
        out.append(Problem(wl, L, x, uvw, wc, rng))
    return out


def mlp_init_params(seed: int = 0) -> np.ndarray:
    """Initial parameters of the learned-kernel network (flat float32, layout of
    include/wproj.h): weights N(0, 1/fan_in) (1/3 for the 3-wide input layer),
    biases zero."""
    rng = np.random.Generator(np.random.PCG64(seed))
    parts = []
    for out_f, in_f in ((256, 3), (256, 256), (256, 256), (3072, 256)):
        parts.append(rng.standard_normal(out_f * in_f) / math.sqrt(in_f))
        parts.append(np.zeros(out_f))
    return np.concatenate(parts).astype(np.float32)


def mlp_samples(m: int, seed: int, wc_max: float = 4.0) -> tuple[np.ndarray, np.ndarray]:
    """uvw rows for training the learned-kernel network on an N-pixel grid:
    sub-grid offsets U[0,1)^2 around random cells, w_c ~ U[0, wc_max] cells
    (h = 2 w_c).  Returns (offsets, w_c); `mlp_uvw` places them on a grid."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return rng.uniform(0.0, 1.0, (m, 2)), rng.uniform(0.0, wc_max, m)


def mlp_uvw(offsets: np.ndarray, wc: np.ndarray, N: int, L: float, seed: int = 1) -> np.ndarray:
    """(u, v, w) in wavelengths for cells drawn uniformly inside |g| < N/2 - 16."""
    rng = np.random.Generator(np.random.PCG64(seed))
    m = wc.shape[0]
    du = 1.0 / (2.0 * L)
    cells = rng.integers(-(N // 2 - 16), N // 2 - 16, (m, 2))
    uv = (cells + offsets) * du
    w = 2.0 * wc / (L * L)
    return np.ascontiguousarray(np.concatenate([uv, w[:, None]], axis=1))


def paper_problem(N: int, coverage: float, seed: int = 0, wd: float | None = None, n_blobs: int = 20,
                  L: float | None = None) -> Problem:
    """The paper's own set-up (Section 4.1): visibilities on the 2N x 2N grid
    (cells 1/L), a fraction `coverage` of all grid cells drawn uniformly
    without replacement, w_d ~ U[0, 1] (or the constant `wd`), w = w_d N / L^2.
    (u, v) = (j + 1e-9) / L for grid cell j in [-N, N), so that floor(u L) = j
    exactly.  Order: sky -> cells -> w (noise: draw_noise)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    L = fov_L() if L is None else L
    G = 2 * N
    x = blob_sky(rng, N, n_blobs)
    M = max(1, int(round(coverage * G * G)))
    flat = rng.choice(G * G, M, replace=False)
    cells = np.stack([flat // G - N, flat % G - N], axis=1).astype(np.float64)
    wdv = rng.uniform(0.0, 1.0, M) if wd is None else np.full(M, float(wd))
    w = wdv * N / (L * L)
    uvw = np.ascontiguousarray(np.concatenate([(cells + 1e-9) / L, w[:, None]], axis=1))
    wl = Workload(f"paper{N}_cov{coverage}", N=N, n_blobs=n_blobs, M=M, uv="grid", wd_max=1.0, e=0.75)
    return Problem(wl, L, x, uvw, wdv, rng)


def dde_screens(n_screens: int, N: int, L: float, seed: int = 0, beam_fwhm: float = 1.2,
                pointing: float = 0.05, phase_rad: float = 0.5, modes: int = 3) -> np.ndarray:
    """Synthetic direction-dependent screens (A-projection style), n x G x G
    complex64 on the chirp's sample points of the padded field of view: index P
    holds offset P - G/2, i.e. l = (P - G/2) L / N (pixel p of the image at
    index p + N/2).  Each screen is a Gaussian primary beam of full width at
    half maximum beam_fwhm * L, pointed off centre by up to pointing * L, times
    a smooth phase screen of `modes` plane waves of at most two cycles across
    the field of view and amplitude phase_rad radians each."""
    rng = np.random.Generator(np.random.PCG64(seed))
    G = 2 * N
    l = (np.arange(G) - G // 2) * (L / N)
    sig = beam_fwhm * L / (2.0 * math.sqrt(2.0 * math.log(2.0)))
    out = np.empty((n_screens, G, G), dtype=np.complex64)
    for j in range(n_screens):
        l0, m0 = rng.uniform(-pointing, pointing, 2) * L
        beam = np.exp(-((l[:, None] - l0) ** 2 + (l[None, :] - m0) ** 2) / (2.0 * sig * sig))
        phase = np.zeros((G, G))
        for _ in range(modes):
            ku, kv = rng.uniform(-2.0, 2.0, 2) / L
            phase += phase_rad * np.cos(2.0 * math.pi * (ku * l[:, None] + kv * l[None, :]) + rng.uniform(0, 2 * math.pi))
        out[j] = (beam * np.exp(1j * phase)).astype(np.complex64)
    return out
