"""Seeded synthetic plane-wave channel data: the inputs both sides are fed.

This module only *generates inputs*.  It simulates the acquisition that the
paper's handheld front end performs (Sec. II-A, II-C: 64-channel receive of a
nonsteered plane-wave transmit, 10-bit ADC, Table I) on a synthetic phantom,
because the paper's PVA phantom and in-vivo recordings are not available.  It
holds none of the beamformer's arithmetic: no delay tables, no interpolation,
no combiner, no envelope.  The forward model is the physics of a point
scatterer in a homogeneous medium insonified by a plane wave; the beamformer
under test has to invert it.

Recipe (all seeded with numpy's PCG64):

* pulse  p(t) = exp(-t^2 / (2 s^2)) cos(2 pi f0 t), s = 2 / (2.3548 f0)
  (envelope FWHM of two cycles), truncated at |t| <= 4 s;
* echo of scatterer k at element i for a plane wave at angle theta:
  t_k,i = (x_k sin(theta) + z_k cos(theta)) / c + sqrt((x_k - x_i)^2 + z_k^2) / c,
  time zero when the wavefront crosses the array centre; sample n is at n/fs;
* speckle: 10^4 scatterers uniform over the field of view widened by 2 mm on
  every side, amplitude Rayleigh(sigma=1) times a random sign;
* point targets (wires) with amplitude 20, an anechoic cyst that removes the
  speckle inside its disk;
* white Gaussian noise at 40 dB SNR relative to the global RMS of the clean
  echoes, then scaling so that max|u| = 0.9 * 32767, round-half-even and
  saturation to int16 (optionally rounding to multiples of 64 to mimic the
  10-bit converter of Table I).
"""
from __future__ import annotations

import dataclasses
import math
from typing import Optional, Sequence

import numpy as np

BASE_SEED = 231100482


@dataclasses.dataclass(frozen=True)
class Acquisition:
    """Probe, sampling and grid description of one synthetic workload."""

    n_elements: int = 64
    pitch_m: float = 0.3e-3
    f0_hz: float = 5e6
    fs_hz: float = 20e6
    c_mps: float = 1540.0
    n_samples: int = 1024
    angles_deg: tuple = (0.0,)
    nx: int = 128
    nz: int = 128
    x0_m: float = -9.6e-3
    x1_m: float = 9.6e-3
    z0_m: float = 5e-3
    z1_m: float = 40e-3
    f_number: float = 1.5

    @property
    def angles_rad(self) -> np.ndarray:
        return np.deg2rad(np.asarray(self.angles_deg, dtype=np.float64))

    def x_elements(self) -> np.ndarray:
        i = np.arange(self.n_elements, dtype=np.float64)
        return (i - 0.5 * (self.n_elements - 1)) * self.pitch_m

    def with_(self, **kw) -> "Acquisition":
        return dataclasses.replace(self, **kw)


@dataclasses.dataclass
class Phantom:
    x: np.ndarray
    z: np.ndarray
    amp: np.ndarray
    cysts: list  # [(xc, zc, radius)]
    points: np.ndarray  # [K, 2] wire / point positions (m)


def angles_linspace(n: int, span_deg: float = 10.0) -> tuple:
    """n plane waves evenly spread over [-span, +span] degrees; one wave is 0 deg."""
    if n == 1:
        return (0.0,)
    return tuple(float(a) for a in np.linspace(-span_deg, span_deg, n))


def make_phantom(acq: Acquisition, rng: np.random.Generator, *, n_speckle: int = 10_000,
                 points: Optional[np.ndarray] = None, n_random_points: int = 0,
                 point_box: Optional[tuple] = None, cysts: Sequence = (),
                 point_amp: float = 20.0, margin_m: float = 2e-3) -> Phantom:
    """Speckle + point targets + anechoic cysts (scatterer list)."""
    xs = rng.uniform(acq.x0_m - margin_m, acq.x1_m + margin_m, n_speckle)
    zs = rng.uniform(acq.z0_m - margin_m, acq.z1_m + margin_m, n_speckle)
    amp = rng.rayleigh(1.0, n_speckle) * rng.choice(np.array([-1.0, 1.0]), n_speckle)
    keep = np.ones(n_speckle, dtype=bool)
    for (xc, zc, r) in cysts:
        keep &= (xs - xc) ** 2 + (zs - zc) ** 2 > r * r
    xs, zs, amp = xs[keep], zs[keep], amp[keep]
    pts = [] if points is None else [np.asarray(points, dtype=np.float64).reshape(-1, 2)]
    if n_random_points:
        (bx0, bx1, bz0, bz1) = point_box
        pts.append(np.stack([rng.uniform(bx0, bx1, n_random_points),
                             rng.uniform(bz0, bz1, n_random_points)], axis=1))
    pts = np.concatenate(pts, axis=0) if pts else np.zeros((0, 2))
    return Phantom(x=np.concatenate([xs, pts[:, 0]]), z=np.concatenate([zs, pts[:, 1]]),
                   amp=np.concatenate([amp, np.full(len(pts), point_amp)]),
                   cysts=list(cysts), points=pts)


def pulse(t: np.ndarray, f0: float) -> np.ndarray:
    s = 2.0 / (2.3548 * f0)
    p = np.exp(-t * t / (2 * s * s)) * np.cos(2 * math.pi * f0 * t)
    return np.where(np.abs(t) <= 4 * s, p, 0.0)


def clean_echoes(acq: Acquisition, ph: Phantom) -> np.ndarray:
    """Noise-free float64 echoes [A][N][Ns] of a scatterer list."""
    s = 2.0 / (2.3548 * acq.f0_hz)
    half = 4 * s
    width = int(math.ceil(2 * half * acq.fs_hz)) + 2
    taps = np.arange(width)
    xe = acq.x_elements()
    out = np.zeros((len(acq.angles_deg), acq.n_elements, acq.n_samples))
    for a, th in enumerate(acq.angles_rad):
        t_tx = (ph.x * math.sin(th) + ph.z * math.cos(th)) / acq.c_mps
        for i in range(acq.n_elements):
            t = t_tx + np.sqrt((ph.x - xe[i]) ** 2 + ph.z ** 2) / acq.c_mps
            n0 = np.ceil((t - half) * acq.fs_hz).astype(np.int64)
            n = n0[:, None] + taps[None, :]
            w = ph.amp[:, None] * pulse(n / acq.fs_hz - t[:, None], acq.f0_hz)
            ok = (n >= 0) & (n < acq.n_samples) & (w != 0.0)
            out[a, i] = np.bincount(n[ok], weights=w[ok], minlength=acq.n_samples)
    return out


def quantise(x: np.ndarray, *, ten_bit: bool = False) -> np.ndarray:
    """Scale to 0.9 of int16 full range, round half to even, saturate."""
    peak = float(np.max(np.abs(x)))
    scale = 0.0 if peak == 0.0 else 0.9 * 32767.0 / peak
    y = x * scale
    y = np.rint(y / 64.0) * 64.0 if ten_bit else np.rint(y)
    return np.clip(y, -32768, 32767).astype(np.int16)


def synth_rf(acq: Acquisition, ph: Phantom, rng: np.random.Generator, *, snr_db: float = 40.0,
             ten_bit: bool = False) -> np.ndarray:
    """int16 RF [A][N][Ns] with AWGN at the given SNR (global RMS)."""
    clean = clean_echoes(acq, ph)
    rms = float(np.sqrt(np.mean(clean * clean)))
    noisy = clean + rng.normal(0.0, rms * 10 ** (-snr_db / 20.0), clean.shape) if snr_db is not None else clean
    return quantise(noisy, ten_bit=ten_bit)


# --- named workloads (sizes and phantoms of the paper-shaped acquisitions) ---

SPECKLE_POINTS_128 = Acquisition()  # 128x128 grid, 1024 samples, one 0 deg wave, DAS
CYST_WIRES_512 = Acquisition(n_samples=2048, nx=512, nz=512)  # 512x512, 2048 samples
PRECISION_1024 = Acquisition(n_elements=128, n_samples=4096, angles_deg=angles_linspace(7),
                             nx=1024, nz=1024, x0_m=-19.2e-3, x1_m=19.2e-3, z0_m=5e-3, z1_m=30e-3)
# Grid sizes timed in Sec. II-D (depth x lateral), 50 MHz sampling, 7.5 MHz probe, 3 cm depth.
PAPER_GRIDS = ((128, 32), (256, 32), (512, 64), (1024, 64), (1750, 64))


def speckle_points_frame(acq: Acquisition = SPECKLE_POINTS_128, seed: int = BASE_SEED + 0):
    """20 random point targets + speckle + noise (the 128x128 DAS workload)."""
    rng = np.random.default_rng(seed)
    ph = make_phantom(acq, rng, n_random_points=20, point_box=(-8e-3, 8e-3, 7e-3, 38e-3))
    return synth_rf(acq, ph, rng), ph


def cyst_wires_frame(acq: Acquisition = CYST_WIRES_512, seed: int = BASE_SEED + 1, *,
                     cyst=(0.0, 22.5e-3, 2e-3), wire_z_mm=(8, 12, 16, 20, 26, 30, 34, 38),
                     wire_x_mm=(0.0,), ten_bit: bool = False):
    """Anechoic 4 mm cyst + wire targets + speckle + noise."""
    rng = np.random.default_rng(seed)
    pts = np.array([(x * 1e-3, z * 1e-3) for z in wire_z_mm for x in wire_x_mm])
    ph = make_phantom(acq, rng, points=pts, cysts=[cyst])
    return synth_rf(acq, ph, rng, ten_bit=ten_bit), ph


def precision_frame(acq: Acquisition = PRECISION_1024, seed: int = BASE_SEED + 3):
    """128-element, 7-angle, 1024x1024 workload with a cyst at 17.5 mm and wires."""
    return cyst_wires_frame(acq, seed, cyst=(0.0, 17.5e-3, 2e-3), wire_z_mm=(8, 12, 24, 28),
                            wire_x_mm=(-8.0, 0.0, 8.0))


def point_frame(acq: Acquisition, x_m: float, z_m: float, amp: float = 1.0):
    """Noise-free single point scatterer (for localisation checks), quantised."""
    ph = Phantom(x=np.array([x_m]), z=np.array([z_m]), amp=np.array([amp]), cysts=[],
                 points=np.array([[x_m, z_m]]))
    return quantise(clean_echoes(acq, ph)), ph


def mixed_batch_specs(n_frames: int = 256, seed: int = BASE_SEED + 2, *, nmin=64, nmax=1024,
                      amax=11):
    """Grid sizes and angle counts of the uneven 256-frame batch (uniform draws)."""
    rng = np.random.default_rng(seed)
    nx = rng.integers(nmin, nmax + 1, n_frames)
    nz = rng.integers(nmin, nmax + 1, n_frames)
    na = rng.integers(1, amax + 1, n_frames)
    return [dict(nx=int(a), nz=int(b), n_angles=int(c)) for a, b, c in zip(nx, nz, na)]
