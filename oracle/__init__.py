"""FP64 CPU oracle for plane-wave beamforming, envelope, log compression and metrics.

TEST INFRASTRUCTURE ONLY: the test-suite, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline / reference leg are the only importers.  The product
package never imports it, and it imports nothing from the product package.

* ``beamform`` / ``beamform_pdas`` / ``beamform_iq`` / ``delayed_samples`` wrap
  ``bf_oracle.c``; ``demodulate`` forms the complex baseband records of IQ beamforming (double precision,
  plain loops over pixels, angles and channels; see that file's header for
  the exact definition it follows, Eq. (1) and Sec. II-B of the paper).
* ``envelope`` is the analytic-signal magnitude along depth computed with a
  library FFT in float64 (one-sided spectrum, scipy.signal.hilbert
  convention); the DMAS image additionally keeps only the band [f0, 3 f0]
  around its second harmonic.
* ``log_compress`` maps the envelope to decibels against the frame maximum
  and clips at the -70 dB dynamic range the paper's images use (Fig. 3).
* ``fwhm``, ``contrast`` implement the resolution and contrast metrics of
  Sec. II-D (FWHM at -6 dB, CR, CNR).
* ``fk_migrate`` is the plane-wave f-k migration (Sec. II-B-3) with the exact
  wavenumber mapping of the delay model above, numpy FFTs in float64.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "bf_oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

DAS, DMAS, CF = "das", "dmas", "cf"


def build(force: bool = False) -> str:
    """Compile bf_oracle.c into liboracle.so next to it (gcc, OpenMP, no FMA contraction)."""
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + ".tmp%d" % os.getpid()
    cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fopenmp", "-fPIC",
           "-shared", _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _bind(lib):
    d, i32, i64 = ctypes.c_double, ctypes.c_int32, ctypes.c_int64
    p = ctypes.c_void_p
    lib.oracle_beamform.argtypes = [p, i32, i32, i32, p, p, i32, i32, d, d, d, d, d, d, d,
                                    p, i64, p, p, p, p, i32]
    lib.oracle_beamform.restype = ctypes.c_int
    lib.oracle_delayed_samples.argtypes = [p, i32, i32, i32, p, p, i32, i32, d, d, d, d,
                                           i32, i32, d, d, d, p, p, p]
    lib.oracle_delayed_samples.restype = ctypes.c_int
    lib.oracle_beamform_pdas.argtypes = [p, i32, i32, i32, p, p, i32, i32, d, d, d, d, d, d, d,
                                         d, p, i64, p, i32]
    lib.oracle_beamform_pdas.restype = ctypes.c_int
    lib.oracle_beamform_iq.argtypes = [p, p, i32, i32, i32, p, p, i32, i32, d, d, d, d, d, d, d,
                                       d, p, i64, p, p, i32]
    lib.oracle_beamform_iq.restype = ctypes.c_int
    lib.oracle_max_threads.restype = ctypes.c_int32
    return lib


def _load():
    global _lib
    with _lock:
        if _lib is None:
            _lib = _bind(ctypes.CDLL(build()))
    return _lib


class use_library:
    """Context manager that routes this module through another build of
    bf_oracle.c (the mutation tests plant mistakes in a copy of the source)."""

    def __init__(self, path):
        self.path = path

    def __enter__(self):
        global _lib
        _load()
        self.saved = _lib
        _lib = _bind(ctypes.CDLL(self.path))
        return self

    def __exit__(self, *exc):
        global _lib
        _lib = self.saved
        return False


def max_threads() -> int:
    return int(_load().oracle_max_threads())


def _ptr(a):
    return None if a is None else a.ctypes.data


def _grid(grid):
    nx, nz, x0, x1, z0, z1 = grid
    return int(nx), int(nz), float(x0), float(x1), float(z0), float(z1)


def grid_coords(grid):
    """Pixel coordinates (inclusive linspaces, float64)."""
    nx, nz, x0, x1, z0, z1 = _grid(grid)

    def ls(lo, hi, n):
        if n == 1:
            return np.array([lo])
        return lo + np.arange(n, dtype=np.float64) * ((hi - lo) / (n - 1))

    return ls(x0, x1, nx), ls(z0, z1, nz)


def beamform(rf, x_elem, angles_rad, grid, fs, c, f_number, *, pixels=None, threads=0):
    """DAS, DMAS and CF-DAS images (float64) plus the active-channel count.

    rf: int16 [A][N][Ns]; grid = (nx, nz, x0, x1, z0, z1) in metres.
    pixels: optional int64 array of linear indices ix * nz + iz; outputs are
    then 1-D in that order, otherwise [nx][nz].
    """
    rf = np.ascontiguousarray(rf, dtype=np.int16)
    na, ne, ns = rf.shape
    x_elem = np.ascontiguousarray(x_elem, dtype=np.float64)
    th = np.ascontiguousarray(np.atleast_1d(angles_rad), dtype=np.float64)
    assert x_elem.shape == (ne,) and th.shape == (na,)
    nx, nz, x0, x1, z0, z1 = _grid(grid)
    if pixels is None:
        shape, pix, npix = (nx, nz), None, nx * nz
    else:
        pix = np.ascontiguousarray(pixels, dtype=np.int64)
        shape, npix = pix.shape, pix.size
    out = {k: np.empty(shape, np.float64) for k in (DAS, DMAS, CF)}
    m = np.empty(shape, np.int32)
    rc = _load().oracle_beamform(_ptr(rf), na, ne, ns, _ptr(x_elem), _ptr(th), nx, nz, x0, x1,
                                 z0, z1, float(fs), float(c), float(f_number), _ptr(pix), npix,
                                 _ptr(out[DAS]), _ptr(out[DMAS]), _ptr(out[CF]), _ptr(m),
                                 int(threads))
    if rc != 0:
        raise ValueError("oracle_beamform rejected its arguments (rc=%d)" % rc)
    out["m"] = m
    return out


def beamform_pdas(rf, x_elem, angles_rad, grid, fs, c, f_number, p, *, pixels=None, threads=0):
    """pDAS image (float64, Eq. (2)-(3)): per angle sign(yt) |yt|^p with
    yt = sum over active channels of sign(v) |v|^(1/p), summed over angles.
    Shapes as ``beamform``."""
    rf = np.ascontiguousarray(rf, dtype=np.int16)
    na, ne, ns = rf.shape
    x_elem = np.ascontiguousarray(x_elem, dtype=np.float64)
    th = np.ascontiguousarray(np.atleast_1d(angles_rad), dtype=np.float64)
    assert x_elem.shape == (ne,) and th.shape == (na,)
    nx, nz, x0, x1, z0, z1 = _grid(grid)
    if pixels is None:
        shape, pix, npix = (nx, nz), None, nx * nz
    else:
        pix = np.ascontiguousarray(pixels, dtype=np.int64)
        shape, npix = pix.shape, pix.size
    out = np.empty(shape, np.float64)
    rc = _load().oracle_beamform_pdas(_ptr(rf), na, ne, ns, _ptr(x_elem), _ptr(th), nx, nz, x0,
                                      x1, z0, z1, float(fs), float(c), float(f_number), float(p),
                                      _ptr(pix), npix, _ptr(out), int(threads))
    if rc != 0:
        raise ValueError("oracle_beamform_pdas rejected its arguments (rc=%d)" % rc)
    return out


def demodulate(rf, fs, f0):
    """Complex baseband records IQ[k] = a[k] exp(-j 2 pi f0 k / fs), a the analytic
    signal of each channel record along its samples (one-sided spectrum, the
    scipy.signal.hilbert convention), in float64.  rf: [..., Ns]."""
    u = np.asarray(rf, dtype=np.float64)
    ns = u.shape[-1]
    a = np.fft.ifft(np.fft.fft(u, axis=-1) * spectral_mask(ns), axis=-1)
    k = np.arange(ns, dtype=np.float64)
    return a * np.exp(-2j * np.pi * f0 * k / fs)


def beamform_iq(iq, x_elem, angles_rad, grid, fs, c, f_number, f0, *, pixels=None, threads=0):
    """|IQ-DAS| and |BB-DMAS| (Eq. (4)) images in float64 from complex baseband
    records iq [A][N][Ns] (``demodulate``).  Shapes as ``beamform``."""
    iq = np.asarray(iq)
    na, ne, ns = iq.shape
    re = np.ascontiguousarray(iq.real, dtype=np.float64)
    im = np.ascontiguousarray(iq.imag, dtype=np.float64)
    x_elem = np.ascontiguousarray(x_elem, dtype=np.float64)
    th = np.ascontiguousarray(np.atleast_1d(angles_rad), dtype=np.float64)
    assert x_elem.shape == (ne,) and th.shape == (na,)
    nx, nz, x0, x1, z0, z1 = _grid(grid)
    if pixels is None:
        shape, pix, npix = (nx, nz), None, nx * nz
    else:
        pix = np.ascontiguousarray(pixels, dtype=np.int64)
        shape, npix = pix.shape, pix.size
    out = {"iqdas": np.empty(shape, np.float64), "bbdmas": np.empty(shape, np.float64)}
    rc = _load().oracle_beamform_iq(_ptr(re), _ptr(im), na, ne, ns, _ptr(x_elem), _ptr(th), nx, nz,
                                    x0, x1, z0, z1, float(fs), float(c), float(f_number), float(f0),
                                    _ptr(pix), npix, _ptr(out["iqdas"]), _ptr(out["bbdmas"]),
                                    int(threads))
    if rc != 0:
        raise ValueError("oracle_beamform_iq rejected its arguments (rc=%d)" % rc)
    return out


def fk_sizes(n_elements, n_samples):
    """Transform lengths of the f-k migration: records zero-padded to twice
    their length and the aperture to twice its width, rounded up to powers of two."""
    nt = 1 << int(np.ceil(np.log2(2 * n_samples)))
    nk = 1 << int(np.ceil(np.log2(2 * n_elements)))
    return nt, nk


def fk_migrate(rf, pitch, angles_rad, fs, c):
    """Plane-wave f-k migration (exact mapping of the delay model of Eq. (1) with
    the plane-wave transmit), compounded over angles; returns |image| on the
    native grid [N][Ns]: column i at element i, row m at depth m dz, dz = c / (2 fs).

    Per angle theta (s = sin, c_ = cos), in float64:
      1. D(b, x_i) = DFT over n of u_i[n] (records zero-padded to nt), bins
         b = 0 .. nt/2 (frequency b fs / nt);
      2. the transmit's lateral delay is removed:
         D *= exp(+j 2 pi (b fs / nt) x_i s / c) = exp(+j pi b x_i s / (nt dz));
      3. DFT over the elements (zero-padded to nk): D(b, m), lateral wavenumber
         Kx = 2 pi m_s / (nk pitch) with m_s the signed index of bin m;
      4. the output spectrum at (m, q), depth wavenumber Kz = 2 pi q / (nt dz),
         q = 1 .. nt/2, takes the temporal bin where the transmit wave
         k (s, c_) plus a receive wave of lateral wavenumber Kx - k s reach
         (Kx, Kz): k = (Kx^2 + Kz^2) / (2 (Kx s + Kz c_)).  In bins, with
         X = m_s nt dz / (nk pitch) and Q = q:
             pos = (X^2 + Q^2) / (X s + Q c_),
         kept where X s + Q c_ > 0, |2 X - pos s| <= pos (a propagating
         receive wave) and 0 <= pos < nt / 2; D(., m) is interpolated linearly
         at pos and weighted by dk/dKz = (1/2) dpos/dQ
             = (Q (X s + Q c_) - (X^2 + Q^2) c_ / 2) / (X s + Q c_)^2;
      5. the spectra of all angles are summed, inverse 2-D DFT, magnitude.
    """
    rf = np.asarray(rf, dtype=np.float64)
    na, ne, ns = rf.shape
    nt, nk = fk_sizes(ne, ns)
    dz = c / (2.0 * fs)
    x = (np.arange(ne) - 0.5 * (ne - 1)) * pitch
    b = np.arange(nt // 2 + 1, dtype=np.float64)
    ms = np.where(np.arange(nk) < nk // 2, np.arange(nk), np.arange(nk) - nk).astype(np.float64)
    X = ms * (nt * dz / (nk * pitch))                         # [nk]
    Q = np.arange(1, nt // 2 + 1, dtype=np.float64)           # [nt/2]
    XX, QQ = np.meshgrid(X, Q)                                # [q][m]
    spec = np.zeros((nt, nk), dtype=np.complex128)            # [Kz bin][Kx bin]
    cols = np.broadcast_to(np.arange(nk)[None, :], XX.shape)
    for a in range(na):
        st, ct = np.sin(angles_rad[a]), np.cos(angles_rad[a])
        D = np.fft.rfft(rf[a], n=nt, axis=1)                  # [N][nt/2+1]
        D = D * np.exp(1j * np.pi * b[None, :] * x[:, None] * st / (nt * dz))
        D = np.fft.fft(D, n=nk, axis=0)                       # [nk][nt/2+1]
        den = XX * st + QQ * ct
        num = XX * XX + QQ * QQ
        with np.errstate(divide="ignore", invalid="ignore"):
            pos = num / den
            w = (QQ * den - 0.5 * num * ct) / (den * den)
        ok = (den > 0) & (np.abs(2.0 * XX - pos * st) <= pos) & (pos >= 0) & (pos < nt // 2)
        pos = np.where(ok, pos, 0.0)
        i0 = np.floor(pos).astype(np.int64)
        al = pos - i0
        i1 = np.minimum(i0 + 1, nt // 2)
        val = (1 - al) * D[cols, i0] + al * D[cols, i1]
        spec[1:nt // 2 + 1] += np.where(ok, val * w, 0.0)
    img = np.fft.ifft2(spec)                                  # [z][x]
    return np.abs(img[:ns, :ne]).T.copy()


def fk_stolt(rf, pitch, angles_rad, fs, c):
    """Stolt's f-k migration for plane waves (Sec. II-B-3): the exploding
    reflector model fitted to the plane-wave two-way time, migrated with Stolt's
    mapping and mapped back onto the native grid [N][Ns] (column i at element
    i, row m at depth m dz, dz = c / (2 fs)); |image|, compounded over angles.

    The fit (the reading this library takes; the paper cites the method): after
    the transmit's lateral delay x_i sin(theta) / c is removed, a scatterer at
    (x0, z0) draws c t(u) = z0 (1 + cos) - u sin + sqrt(u^2 + z0^2), u = x - x0.
    An exploding reflector at (x0', z0') seen with velocity v draws
    v t = sqrt((x - x0')^2 + z0'^2).  Matching the two in value, slope and
    curvature at u = 0 gives
        v = c / beta, beta = sqrt(1 + cos - sin^2 / 2),
        z0' = beta z0, x0' = x0 + z0 sin.
    Stolt's mapping for that model takes the output wavenumbers (Kx, Kz') to
    the temporal frequency w = v sqrt(Kx^2 + Kz'^2); the image is then mapped
    back by the shear and scale (x, z) -> (x + z sin, beta z), which in the
    spectrum reads Kz' = (Kz - Kx sin) / beta.  In bins (X, Q as in
    fk_migrate): Q' = (Q - X sin) / beta, the temporal bin
        pos = (2 / beta) sqrt(X^2 + Q'^2),
    kept where Q' > 0 and 0 <= pos < nt / 2, interpolated linearly as in
    fk_migrate and weighted by (1/2) dpos/dQ = Q' / (beta^2 sqrt(X^2 + Q'^2)).
    """
    rf = np.asarray(rf, dtype=np.float64)
    na, ne, ns = rf.shape
    nt, nk = fk_sizes(ne, ns)
    dz = c / (2.0 * fs)
    x = (np.arange(ne) - 0.5 * (ne - 1)) * pitch
    b = np.arange(nt // 2 + 1, dtype=np.float64)
    ms = np.where(np.arange(nk) < nk // 2, np.arange(nk), np.arange(nk) - nk).astype(np.float64)
    X = ms * (nt * dz / (nk * pitch))                         # [nk]
    Q = np.arange(1, nt // 2 + 1, dtype=np.float64)           # [nt/2]
    XX, QQ = np.meshgrid(X, Q)                                # [q][m]
    spec = np.zeros((nt, nk), dtype=np.complex128)            # [Kz bin][Kx bin]
    cols = np.broadcast_to(np.arange(nk)[None, :], XX.shape)
    for a in range(na):
        st, ct = np.sin(angles_rad[a]), np.cos(angles_rad[a])
        D = np.fft.rfft(rf[a], n=nt, axis=1)                  # [N][nt/2+1]
        D = D * np.exp(1j * np.pi * b[None, :] * x[:, None] * st / (nt * dz))
        D = np.fft.fft(D, n=nk, axis=0)                       # [nk][nt/2+1]
        bet = np.sqrt(1.0 + ct - 0.5 * st * st)
        Qp = (QQ - st * XX) / bet
        rad = np.sqrt(XX * XX + Qp * Qp)
        with np.errstate(divide="ignore", invalid="ignore"):
            pos = (2.0 / bet) * rad
            w = Qp / (bet * bet * rad)
        ok = (Qp > 0) & (pos >= 0) & (pos < nt // 2)
        pos = np.where(ok, pos, 0.0)
        i0 = np.floor(pos).astype(np.int64)
        al = pos - i0
        i1 = np.minimum(i0 + 1, nt // 2)
        val = (1 - al) * D[cols, i0] + al * D[cols, i1]
        spec[1:nt // 2 + 1] += np.where(ok, val * w, 0.0)
    img = np.fft.ifft2(spec)                                  # [z][x]
    return np.abs(img[:ns, :ne]).T.copy()


def delayed_samples(rf, x_elem, angles_rad, grid, ix, iz, fs, c, f_number):
    """Per (angle, channel) interpolated samples of one pixel and their flags."""
    rf = np.ascontiguousarray(rf, dtype=np.int16)
    na, ne, ns = rf.shape
    x_elem = np.ascontiguousarray(x_elem, dtype=np.float64)
    th = np.ascontiguousarray(np.atleast_1d(angles_rad), dtype=np.float64)
    nx, nz, x0, x1, z0, z1 = _grid(grid)
    v = np.empty((na, ne), np.float64)
    act = np.empty((na, ne), np.uint8)
    rec = np.empty((na, ne), np.uint8)
    rc = _load().oracle_delayed_samples(_ptr(rf), na, ne, ns, _ptr(x_elem), _ptr(th), nx, nz, x0,
                                        x1, z0, z1, int(ix), int(iz), float(fs), float(c),
                                        float(f_number), _ptr(v), _ptr(act), _ptr(rec))
    if rc != 0:
        raise ValueError("pixel out of the grid")
    return v, act.astype(bool), rec.astype(bool)


def spectral_mask(length, *, bandpass=False, dz=None, c=None, f0=None):
    """One-sided analytic-signal mask H[k] times the optional band-pass B[k].

    H[0] = 1, H[k] = 2 for 0 < k < L/2, H[L/2] = 1 when L is even, 0 for the
    negative frequencies.  B[k] = 1 iff f0 <= k c / (2 L dz) <= 3 f0 and
    B[0] = 0: bin k of a depth axis of spacing dz is the RF frequency
    k c / (2 L dz) (two-way travel)."""
    L = int(length)
    h = np.zeros(L)
    h[0] = 1.0
    if L % 2 == 0:
        h[1:L // 2] = 2.0
        h[L // 2] = 1.0
    else:
        h[1:(L + 1) // 2] = 2.0
    if bandpass:
        k = np.arange(L, dtype=np.float64)
        f = k * c / (2.0 * L * dz) if L > 1 else np.zeros(1)
        b = ((f >= f0) & (f <= 3.0 * f0)).astype(np.float64)
        b[0] = 0.0
        h = h * b
    return h


def envelope(y, *, bandpass=False, dz=None, c=None, f0=None):
    """|analytic signal| of each column of y [..., nz] along the last axis (float64)."""
    y = np.asarray(y, dtype=np.float64)
    L = y.shape[-1]
    X = np.fft.fft(y, axis=-1)
    X = X * spectral_mask(L, bandpass=bandpass, dz=dz, c=c, f0=f0)
    return np.abs(np.fft.ifft(X, axis=-1))


def log_compress(env, dynamic_range_db=70.0):
    """20 log10(env / max env), clipped to [-DR, 0]; a zero envelope maps to -DR."""
    env = np.asarray(env, dtype=np.float64)
    peak = env.max() if env.size else 0.0
    out = np.full(env.shape, -float(dynamic_range_db))
    if peak > 0.0:
        with np.errstate(divide="ignore"):
            db = 20.0 * np.log10(env / peak)
        out = np.clip(db, -float(dynamic_range_db), 0.0)
    return out


def fwhm(profile, spacing=1.0, drop_db=6.0):
    """Width at -drop_db below the peak of a sampled profile (linear envelope).

    Crossings are located by linear interpolation between the samples that
    straddle the threshold, walking outwards from the peak; NaN when the
    profile never drops below the threshold on one side."""
    p = np.asarray(profile, dtype=np.float64)
    m = int(np.argmax(p))
    thr = p[m] * 10.0 ** (-drop_db / 20.0)
    j = m
    while j > 0 and p[j - 1] >= thr:
        j -= 1
    if j == 0:
        return float("nan")
    left = (j - 1) + (thr - p[j - 1]) / (p[j] - p[j - 1])
    j = m
    while j < len(p) - 1 and p[j + 1] >= thr:
        j += 1
    if j == len(p) - 1:
        return float("nan")
    right = j + (p[j] - thr) / (p[j] - p[j + 1])
    return float((right - left) * spacing)


def cyst_regions(grid, xc, zc, radius, *, inner=0.8, offset=2.5):
    """Masks [nx][nz]: a disk of inner*radius at the cyst centre and two disks
    of the same size at the same depth, offset*radius to either side."""
    xs, zs = grid_coords(grid)
    X, Z = np.meshgrid(xs, zs, indexing="ij")
    r2 = (inner * radius) ** 2
    inside = (X - xc) ** 2 + (Z - zc) ** 2 <= r2
    outside = (((X - xc - offset * radius) ** 2 + (Z - zc) ** 2 <= r2)
               | ((X - xc + offset * radius) ** 2 + (Z - zc) ** 2 <= r2))
    return inside, outside


def contrast(env, inside, outside):
    """CR (dB) and CNR of Sec. II-D from a linear envelope image.

    cnr uses the pooled deviation sqrt((s_in^2 + s_out^2)/2); cnr_printed is
    the expression exactly as typeset, sqrt(s_in^2 + s_out^2/2)."""
    a = np.asarray(env, dtype=np.float64)[inside]
    b = np.asarray(env, dtype=np.float64)[outside]
    mi, mo = a.mean(), b.mean()
    si, so = a.std(), b.std()
    return dict(cr_db=float(20 * np.log10(mi / mo)),
                cnr=float(abs(mi - mo) / np.sqrt((si * si + so * so) / 2.0)),
                cnr_printed=float((mi - mo) / np.sqrt(si * si + so * so / 2.0)),
                mu_in=float(mi), mu_out=float(mo), sigma_in=float(si), sigma_out=float(so))
