"""Seeded synthetic inputs for the messenger mapmaker: sky, scan pointing, 1/f noise.

This module only *generates data* (the forward model d = P m_true + n of Sec. 2, Eq. 1).
It holds none of the solver's arithmetic and is shared by the CUDA path, the tests and
the CPU oracle as a pure input source.

Workload shapes (the paper's own simulation, Sec. 2.3, uses a 2-degree patch with
compact sources that is not reproduced; these synthetic stand-ins keep its structure:
cross-linked rasters, polarised detectors at several angles, N(f) = s^2 (1 + (fk/f)^a)):

* ``config_temperature_64``   64x64 T-only map, one detector, 64 horizontal then 64
  vertical sweeps of 256 samples at 4 samples/pixel (32768 samples, 100 Hz).
* ``config_iqu(...)``         W x W IQU map, D detectors of n samples each at 200 Hz,
  alternating horizontal / vertical sweeps (4 samples per pixel), detector angles
  0, 180/D, ... degrees plus a 0.5 Hz half-wave-plate rotation.
* ``config_uneven(...)``      chunks of uneven 2-3-5-smooth lengths, each with its own
  noise spectrum and raster angle, on one IQU map (1024^2, 64 chunks of 2^16..2^20).
* ``config_crosslinked(...)`` 2048^2 IQU, 32 detectors x 2^24 samples on rasters at four
  angles, FP16 weights.

Noise draws use a circulant covariance per chunk: n = irfft(sqrt(N_k) * rfft(w)),
w ~ N(0, 1), whose covariance is exactly F^-1 diag(N_k) F.
"""
from __future__ import annotations

import os
from concurrent.futures import ThreadPoolExecutor

import numpy as np

SEED_BASE = 1705_0000


def _rng(seed: int, stream: int) -> np.random.Generator:
    return np.random.default_rng([int(seed), int(stream)])


def _pmap(fn, items):
    """[fn(x) for x in items] on a thread pool (NumPy's FFTs, random draws and elementwise
    kernels release the GIL); every chunk has its own random stream, so the result does not
    depend on the number of threads."""
    items = list(items)
    workers = min(len(items), os.cpu_count() or 1, 16)
    if workers <= 1:
        return [fn(x) for x in items]
    with ThreadPoolExecutor(workers) as ex:
        return list(ex.map(fn, items))


def grf_map(nx: int, ny: int, seed: int, stream: int, rms: float = 1.0) -> np.ndarray:
    """Gaussian random field with power ~ l^-2 (amplitude ~ 1/|l|), zero mean, given rms."""
    w = _rng(seed, stream).standard_normal((ny, nx))
    W = np.fft.rfft2(w)
    ly = np.fft.fftfreq(ny)[:, None] * ny
    lx = np.fft.rfftfreq(nx)[None, :] * nx
    ell = np.sqrt(lx * lx + ly * ly)
    amp = np.zeros_like(ell)
    amp[ell > 0] = 1.0 / ell[ell > 0]
    m = np.fft.irfft2(W * amp, s=(ny, nx))
    m -= m.mean()
    m *= rms / m.std()
    return m


def sky(width: int, ncomp: int, seed: int) -> np.ndarray:
    """[width*width, ncomp] float64 sky: T unit rms; Q, U independent GRFs at 0.1 T rms."""
    t = grf_map(width, width, seed, 1, 1.0).ravel()
    if ncomp == 1:
        return t[:, None].copy()
    q = grf_map(width, width, seed, 2, 0.1).ravel()
    u = grf_map(width, width, seed, 3, 0.1).ravel()
    return np.stack([t, q, u], axis=1)


def noise_psd(n: int, fs: float, sigma: float, fknee: float, alpha: float) -> np.ndarray:
    """PSD on the rfft bins k = 0..n//2 used to *draw* noise; DC floored at bin 1."""
    f = np.arange(n // 2 + 1) * (fs / n)
    N = np.empty(n // 2 + 1)
    N[1:] = sigma * sigma * (1.0 + (fknee / f[1:]) ** alpha)
    N[0] = N[1]
    return N


def draw_noise(n: int, psd: np.ndarray, seed: int, stream: int) -> np.ndarray:
    w = _rng(seed, stream).standard_normal(n)
    return np.fft.irfft(np.sqrt(psd) * np.fft.rfft(w), n)


def raster_temperature(width: int, spp: int) -> np.ndarray:
    """width horizontal sweeps (row s, sample j -> column j//spp) then width vertical ones."""
    j = np.arange(width * spp) // spp
    rows = [s * width + j for s in range(width)]
    cols = [j * width + s for s in range(width)]
    return np.concatenate(rows + cols).astype(np.int32)


def raster_alternating(width: int, spp: int, n: int, phase: int) -> np.ndarray:
    """Sweeps of width*spp samples alternating horizontal / vertical, advancing one
    row / column every two sweeps, starting ``phase`` rows/columns in."""
    per = width * spp
    nsweep = -(-n // per)
    j = np.arange(per) // spp
    out = np.empty(nsweep * per, dtype=np.int64)
    for s in range(nsweep):
        line = (s // 2 + phase) % width
        out[s * per:(s + 1) * per] = line * width + j if s % 2 == 0 else j * width + line
    return out[:n].astype(np.int32)


def raster_angled(width: int, spp: int, n: int, angle_rad: float, phase: int,
                  cross_offset: float = 0.0) -> np.ndarray:
    """Back-and-forth sweeps across the map along direction (cos a, sin a) through its
    centre, each sweep one pixel further along the cross direction (wrapping after the
    map's extent, width (|cos a| + |sin a|), in that direction), spp samples per pixel of
    path; coordinates in float64, nearest pixel floor(x) + width floor(y), samples outside
    the map get -1.  cross_offset shifts the beam across the scan direction (pixels)."""
    ca, sa = np.cos(angle_rad), np.sin(angle_rad)
    span = int(np.ceil(width * (abs(ca) + abs(sa)) - 1e-9))
    per = span * spp
    s = np.arange(n) // per
    j = np.arange(n) % per
    xi = -0.5 * span + (j + 0.5) / spp
    xi = np.where(s % 2 == 0, xi, -xi)
    eta = -0.5 * span + ((s // 2 + phase) % span) + 0.5 + cross_offset
    x = 0.5 * width + xi * ca - eta * sa
    y = 0.5 * width + xi * sa + eta * ca
    inside = (x >= 0) & (x < width) & (y >= 0) & (y < width)
    pix = np.floor(x).astype(np.int64) + width * np.floor(y).astype(np.int64)
    return np.where(inside, pix, -1).astype(np.int32)


def smooth235_lengths(lo: int, hi: int) -> np.ndarray:
    """All n in [lo, hi] whose prime factors are 2, 3 and 5."""
    out = []
    a = 1
    while a <= hi:
        b = a
        while b <= hi:
            c = b
            while c <= hi:
                if c >= lo:
                    out.append(c)
                c *= 5
            b *= 3
        a *= 2
    return np.array(sorted(out), dtype=np.int64)


def _project(m: np.ndarray, pix: np.ndarray, c: np.ndarray | None, s: np.ndarray | None) -> np.ndarray:
    """Signal timestream of Eq. 1 (T, or T + Q cos2psi + U sin2psi) for the data model."""
    good = pix >= 0
    out = np.zeros(pix.shape[0])
    p = pix[good]
    out[good] = m[p, 0]
    if m.shape[1] == 3:
        out[good] += m[p, 1] * c[good] + m[p, 2] * s[good]
    return out


def make_problem(width: int, ncomp: int, pix_chunks, fs: float, sigmas, fknees, alphas,
                 angles_deg, hwp_hz: float, seed: int, weight_dtype=np.float32,
                 noiseless: bool = False):
    """Assemble concatenated chunk arrays.  Returns a dict of numpy arrays:
    pix int32 [n], cos/sin weight_dtype [n] (None for T-only), tod float32 [n],
    offsets int64 [n_chunks+1], params float64 [n_chunks, 4] = (sigma, fknee, alpha, fs),
    m_true float64 [npix, ncomp]."""
    m_true = sky(width, ncomp, seed)
    nchunk = len(pix_chunks)
    lens = [len(p) for p in pix_chunks]
    offsets = np.zeros(nchunk + 1, dtype=np.int64)
    offsets[1:] = np.cumsum(lens)
    pix = np.concatenate(pix_chunks).astype(np.int32)
    cos = sin = None
    if ncomp == 3:
        cos = np.empty(offsets[-1], dtype=weight_dtype)
        sin = np.empty(offsets[-1], dtype=weight_dtype)
    tod = np.empty(offsets[-1], dtype=np.float32)
    params = np.zeros((nchunk, 4))
    def fill(c):
        a, b = offsets[c], offsets[c + 1]
        n = b - a
        cc = ss = None
        if ncomp == 3:
            t = np.arange(n) / fs
            psi = np.deg2rad(angles_deg[c]) + 2.0 * np.pi * hwp_hz * t
            cos[a:b] = np.cos(2.0 * psi)
            sin[a:b] = np.sin(2.0 * psi)
            cc = cos[a:b].astype(np.float64)
            ss = sin[a:b].astype(np.float64)
        sig = _project(m_true, pix[a:b], cc, ss)
        if not noiseless:
            sig = sig + draw_noise(n, noise_psd(n, fs, sigmas[c], fknees[c], alphas[c]), seed, 100 + c)
        tod[a:b] = sig
        params[c] = (sigmas[c], fknees[c], alphas[c], fs)

    _pmap(fill, range(nchunk))
    return dict(width=width, npix=width * width, ncomp=ncomp, pix=pix, cos=cos, sin=sin,
                tod=tod, offsets=offsets, params=params, m_true=m_true)


def config_temperature_64(seed: int = SEED_BASE + 0, noiseless: bool = False):
    """64x64 T-only map, 1 detector, 32768 samples at 100 Hz, sigma 1, fknee 1 Hz, alpha 2."""
    pix = raster_temperature(64, 4)
    return make_problem(64, 1, [pix], 100.0, [1.0], [1.0], [2.0], [0.0], 0.0, seed,
                        noiseless=noiseless)


def config_iqu(width: int, n_det: int, n_per_det: int, seed: int, fs: float = 200.0,
               spp: int = 4, fknee_range=(0.1, 2.0), alpha_range=(1.0, 3.0),
               weight_dtype=np.float32, noiseless: bool = False, phase_step: int | None = None):
    """IQU raster of n_det detectors at angles k*180/n_det degrees with a 0.5 Hz HWP.
    Per-detector 1/f noise: sigma 1, fknee ~ U(fknee_range), alpha ~ U(alpha_range)."""
    rng = _rng(seed, 7)
    fknees = rng.uniform(*fknee_range, size=n_det)
    alphas = rng.uniform(*alpha_range, size=n_det)
    if phase_step is None:
        phase_step = max(1, width // n_det)
    chunks = _pmap(lambda d: raster_alternating(width, spp, n_per_det, d * phase_step),
                   range(n_det))
    angles = [180.0 * d / n_det for d in range(n_det)]
    return make_problem(width, 3, chunks, fs, [1.0] * n_det, fknees, alphas, angles, 0.5,
                        seed, weight_dtype=weight_dtype, noiseless=noiseless)


def config_iqu_512(seed: int = SEED_BASE + 1):
    """512x512 IQU map, 8 detectors x 2^22 samples at 200 Hz, FP32 cos2psi/sin2psi."""
    return config_iqu(512, 8, 1 << 22, seed)


def config_iqu_256(seed: int = SEED_BASE + 3):
    """256x256 IQU map, 4 detectors x 2^20 samples at 200 Hz."""
    return config_iqu(256, 4, 1 << 20, seed)


def config_uneven(width: int = 1024, n_chunks: int = 64, lo: int = 1 << 16, hi: int = 1 << 20,
                  seed: int = SEED_BASE + 2, fs: float = 200.0, spp: int = 2):
    """Batched uneven chunks: lengths drawn uniformly from the 2-3-5-smooth integers in
    [lo, hi], each chunk its own 1/f spectrum (f_knee ~ U(0.05, 3) Hz, alpha ~ U(1, 3),
    sigma ~ U(0.5, 2)), its own raster angle ~ U(0, pi) and detector angle ~ U(0, 180) deg
    plus a 0.5 Hz half-wave plate, all scanning one width x width IQU map."""
    rng = _rng(seed, 11)
    cand = smooth235_lengths(lo, hi)
    lens = rng.choice(cand, size=n_chunks)
    fknees = rng.uniform(0.05, 3.0, size=n_chunks)
    alphas = rng.uniform(1.0, 3.0, size=n_chunks)
    sigmas = rng.uniform(0.5, 2.0, size=n_chunks)
    raster = rng.uniform(0.0, np.pi, size=n_chunks)
    angles = rng.uniform(0.0, 180.0, size=n_chunks)
    phases = rng.integers(0, 1 << 20, size=n_chunks)
    chunks = _pmap(lambda c: raster_angled(width, spp, int(lens[c]), raster[c], int(phases[c])),
                   range(n_chunks))
    return make_problem(width, 3, chunks, fs, sigmas, fknees, alphas, angles, 0.5, seed)


def config_crosslinked(width: int = 2048, n_det: int = 32, n_per_det: int = 1 << 24,
                       seed: int = SEED_BASE + 4, fs: float = 200.0, spp: int = 2,
                       weight_dtype=np.float16):
    """Large single-GPU run: n_det detectors on cross-linked rasters at 0, 45, 90 and 135
    degrees (detector d at 45 (d mod 4) degrees), detector angles d * 180 / n_det plus a
    0.5 Hz half-wave plate, 1/f noise f_knee 0.5 Hz, alpha 2, sigma 1, FP16 weights."""
    step = max(1, width // max(1, n_det // 4))
    chunks = _pmap(lambda d: raster_angled(width, spp, n_per_det, np.deg2rad(45.0 * (d % 4)),
                                           (d // 4) * step), range(n_det))
    angles = [180.0 * d / n_det for d in range(n_det)]
    return make_problem(width, 3, chunks, fs, [1.0] * n_det, [0.5] * n_det, [2.0] * n_det,
                        angles, 0.5, seed, weight_dtype=weight_dtype)


def config_differential(width: int = 32, n_chunks: int = 9, n_per: int = 1 << 13,
                        sep: float = 3.0, seed: int = SEED_BASE + 5, fs: float = 100.0,
                        spp: int = 2, fknee: float = 1.0, alpha: float = 2.0,
                        sigma: float = 1.0, noiseless: bool = False):
    """Differencing instrument (App. B test): one T-only detector with two beams offset by
    +-sep/2 pixels across the scan direction, data d = m(beam A) - m(beam B) + n, rasters at
    n_chunks orientations k pi / n_chunks (one chunk each), 1/f noise.  Returns the fields
    of make_problem plus pix_b, gain_a = 1, gain_b = -1."""
    m_true = sky(width, 1, seed)
    offsets = np.arange(n_chunks + 1, dtype=np.int64) * n_per
    pa, pb, tod = [], [], []
    rng = _rng(seed, 13)
    phases = rng.integers(0, 1 << 20, size=n_chunks)
    for c in range(n_chunks):
        ang = np.pi * c / n_chunks
        a = raster_angled(width, spp, n_per, ang, int(phases[c]), 0.5 * sep)
        b = raster_angled(width, spp, n_per, ang, int(phases[c]), -0.5 * sep)
        sig = np.where(a >= 0, m_true[np.maximum(a, 0), 0], 0.0) - \
            np.where(b >= 0, m_true[np.maximum(b, 0), 0], 0.0)
        if not noiseless:
            sig = sig + draw_noise(n_per, noise_psd(n_per, fs, sigma, fknee, alpha), seed, 200 + c)
        pa.append(a)
        pb.append(b)
        tod.append(sig)
    params = np.tile([sigma, fknee, alpha, fs], (n_chunks, 1)).astype(np.float64)
    return dict(width=width, npix=width * width, ncomp=1, pix=np.concatenate(pa).astype(np.int32),
                pix_b=np.concatenate(pb).astype(np.int32), gain_a=1.0, gain_b=-1.0, cos=None,
                sin=None, tod=np.concatenate(tod).astype(np.float32), offsets=offsets,
                params=params, m_true=m_true)
