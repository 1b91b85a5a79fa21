"""Seeded synthetic inputs shaped like the paper's analysis segments.

This module is shared by the CUDA path's tests/benchmark and by the CPU
oracle's tests.  It holds none of the likelihood arithmetic (no Cholesky, no
solve, no quadratic form): it only produces the *inputs* of the method --
an autocovariance sequence (ACF), a gap mask, coloured-noise data and
residual batches R = d - h(theta).

Conventions (paper Sec. II and Sec. II.B; the paper fixes no numeric
convention, so these are stated readings):

* One-sided PSD  S(f) = x**a + floor + 2 x**2,  x = f / 100 Hz, held at
  S(20 Hz) for f < 20 Hz (including f = 0).  Defaults a = -4, floor = 2.
* ACF of a segment of N samples: acf = irfft(S_k, n=2N)[:N] with
  S_k = S(k fs / (2N)), k = 0..N (numpy's 1/(2N) normalisation, no fs/2
  factor).  The N x N Toeplitz matrix C_ij = acf[|i-j|] (Sec. II,
  C_ij = rho(|i-j|)) is then the leading block of the 2N-point circulant
  whose eigenvalues are S_k, so every eigenvalue of C (and of any principal
  submatrix, by interlacing) lies in [min S_k, max S_k].
* Noise with covariance exactly C is drawn by circulant embedding (the
  2N-circulant above is positive semi-definite, so a stationary periodic
  Gaussian process of length 2N restricted to its first N samples has
  covariance C).  This is equal in distribution to the paper's L n~ draw
  (Sec. V.A.1, "Gaussian noise injection") without needing the factor.
* Chirp: leading-order (Newtonian) inspiral,
  h(t) = A tau**(-1/4) cos(phi_c - 2 (tau / (5 Tsun Mc))**(5/8)),
  tau = t_c - t, h = 0 for tau <= 1/fs.  A is fixed once per data draw so
  that the chirp's circulant-embedding (Whittle) SNR against the 2N
  spectrum is 10; templates h(theta_k) reuse that A.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

TSUN = 4.925491025543576e-06  # G Msun / c^3 in seconds


# ----------------------------------------------------------------------------
# PSD / ACF
# ----------------------------------------------------------------------------
def psd(f: np.ndarray, a: float = -4.0, floor: float = 2.0,
        fref: float = 100.0, flow: float = 20.0) -> np.ndarray:
    """One-sided PSD S(f) = (f/fref)^a + floor + 2 (f/fref)^2, held below flow."""
    f = np.asarray(f, dtype=np.float64)
    fe = np.maximum(f, flow)
    x = fe / fref
    return x ** a + floor + 2.0 * x * x


def psd_grid(n: int, fs: float, a: float = -4.0, floor: float = 2.0) -> np.ndarray:
    """S_k = S(k fs / (2n)), k = 0..n (the 2n-point one-sided grid)."""
    k = np.arange(n + 1, dtype=np.float64)
    return psd(k * fs / (2.0 * n), a=a, floor=floor)


def acf_from_psd(n: int, fs: float, a: float = -4.0, floor: float = 2.0,
                 scale: float = 1.0) -> np.ndarray:
    """ACF with n lags: irfft over 2n points of the one-sided PSD, truncated."""
    s = psd_grid(n, fs, a=a, floor=floor) * scale
    return np.fft.irfft(s, n=2 * n)[:n].copy()


def white_acf(n: int, sigma2: float) -> np.ndarray:
    acf = np.zeros(n)
    acf[0] = sigma2
    return acf


def ar1_acf(n: int, phi: float, sigma2: float) -> np.ndarray:
    """ACF of x_t = phi x_{t-1} + e_t, Var(e) = sigma2: sigma2 phi^k / (1 - phi^2)."""
    k = np.arange(n, dtype=np.float64)
    return sigma2 * phi ** k / (1.0 - phi * phi)


# ----------------------------------------------------------------------------
# gaps
# ----------------------------------------------------------------------------
def gap_mask(n: int, n_gaps: int, gap_len: int, rng: np.random.Generator) -> np.ndarray:
    """u8 mask (1 = kept).  Gaps of gap_len samples at seeded offsets drawn
    uniformly, rejected if they overlap or touch another gap."""
    mask = np.ones(n, dtype=np.uint8)
    if n_gaps == 0:
        return mask
    if n_gaps * (gap_len + 1) >= n:
        raise ValueError("gaps do not fit")
    starts: list[int] = []
    tries = 0
    while len(starts) < n_gaps:
        tries += 1
        if tries > 100000:
            raise RuntimeError("could not place gaps")
        s = int(rng.integers(0, n - gap_len + 1))
        if all(s + gap_len < t or t + gap_len < s for t in starts):
            starts.append(s)
    for s in starts:
        mask[s:s + gap_len] = 0
    return mask


def kept_index(mask: np.ndarray | None, n: int) -> np.ndarray:
    if mask is None:
        return np.arange(n, dtype=np.int64)
    return np.flatnonzero(np.asarray(mask) != 0).astype(np.int64)


# ----------------------------------------------------------------------------
# noise by circulant embedding
# ----------------------------------------------------------------------------
def noise_draw(n: int, fs: float, rng: np.random.Generator, a: float = -4.0,
               floor: float = 2.0, scale: float = 1.0, count: int = 1) -> np.ndarray:
    """`count` independent length-n draws whose covariance is exactly the
    Toeplitz matrix of acf_from_psd(n, fs, a, floor, scale).  Returns (count, n)."""
    m = 2 * n
    s = psd_grid(n, fs, a=a, floor=floor) * scale            # eigenvalues, k = 0..n
    lam = np.concatenate([s, s[-2:0:-1]])                     # full length-2n spectrum
    out = np.empty((count, n))
    sq = np.sqrt(lam)
    for c in range(count):
        eps = (rng.standard_normal(m) + 1j * rng.standard_normal(m)) / math.sqrt(2.0)
        y = np.fft.ifft(sq * eps) * math.sqrt(m)              # covariance = circulant (complex)
        out[c] = math.sqrt(2.0) * y.real[:n]
    return out


# ----------------------------------------------------------------------------
# Newtonian chirp
# ----------------------------------------------------------------------------
@dataclasses.dataclass
class ChirpPrior:
    mc_lo: float = 5.0
    mc_hi: float = 30.0
    tc_lo: float = 0.70   # fraction of T
    tc_hi: float = 0.95


def chirp(n: int, fs: float, mc: float, tc: float, phic: float, amp: float = 1.0) -> np.ndarray:
    """Leading-order PN chirp sampled at t_j = j/fs, zero for tau <= 1/fs."""
    t = np.arange(n, dtype=np.float64) / fs
    tau = tc - t
    h = np.zeros(n)
    on = tau > 1.0 / fs
    ta = tau[on]
    phase = phic - 2.0 * (ta / (5.0 * TSUN * mc)) ** 0.625
    h[on] = amp * ta ** (-0.25) * np.cos(phase)
    return h


def draw_theta(rng: np.random.Generator, T: float, count: int,
               prior: ChirpPrior = ChirpPrior()) -> np.ndarray:
    """(count, 3) array of (Mc, t_c, phi_c) from the chirp priors."""
    mc = rng.uniform(prior.mc_lo, prior.mc_hi, count)
    tc = rng.uniform(prior.tc_lo, prior.tc_hi, count) * T
    ph = rng.uniform(0.0, 2.0 * math.pi, count)
    return np.stack([mc, tc, ph], axis=1)


def whittle_snr(h: np.ndarray, n: int, fs: float, a: float = -4.0, floor: float = 2.0,
                scale: float = 1.0) -> float:
    """SNR of h against the 2n-circulant with eigenvalues S_k (amplitude setting
    only; the exact time-domain SNR of the segment differs slightly)."""
    m = 2 * n
    s = psd_grid(n, fs, a=a, floor=floor) * scale
    lam = np.concatenate([s, s[-2:0:-1]])
    hp = np.zeros(m)
    hp[:n] = h
    H = np.fft.fft(hp)
    return math.sqrt(float(np.sum(np.abs(H) ** 2 / lam)) / m)


# ----------------------------------------------------------------------------
# one segment's workload
# ----------------------------------------------------------------------------
@dataclasses.dataclass
class Segment:
    n: int
    fs: float
    acf: np.ndarray          # float64[n]
    mask: np.ndarray | None  # uint8[n] or None (no gaps)
    kept: np.ndarray         # int64[n']
    d: np.ndarray            # float64[n] data (noise + injected chirp)
    amp: float               # chirp amplitude (Whittle SNR 10)
    a: float = -4.0
    floor: float = 2.0
    scale: float = 1.0

    @property
    def n_kept(self) -> int:
        return int(self.kept.size)


def make_segment(n: int, fs: float, seed: int, n_gaps: int = 0, gap_len: int = 512,
                 a: float = -4.0, floor: float = 2.0, scale: float = 1.0,
                 snr: float = 10.0) -> Segment:
    rng = np.random.default_rng(seed)
    acf = acf_from_psd(n, fs, a=a, floor=floor, scale=scale)
    mask = gap_mask(n, n_gaps, gap_len, rng) if n_gaps > 0 else None
    kept = kept_index(mask, n)
    T = n / fs
    th = draw_theta(rng, T, 1)[0]
    h0 = chirp(n, fs, th[0], th[1], th[2])
    amp = snr / max(whittle_snr(h0, n, fs, a=a, floor=floor, scale=scale), 1e-300)
    noise = noise_draw(n, fs, rng, a=a, floor=floor, scale=scale, count=1)[0]
    d = noise + amp * h0
    return Segment(n=n, fs=fs, acf=acf, mask=mask, kept=kept, d=d, amp=amp,
                   a=a, floor=floor, scale=scale)


def residual_batch(seg: Segment, K: int, seed: int) -> np.ndarray:
    """R (K, n') float32, row k = kept samples of d - h(theta_k).  As a flat
    buffer this is the n' x K column-major matrix with leading dimension n'."""
    rng = np.random.default_rng(seed)
    T = seg.n / seg.fs
    th = draw_theta(rng, T, K)
    R = np.empty((K, seg.n_kept), dtype=np.float32)
    for k in range(K):
        h = chirp(seg.n, seg.fs, th[k, 0], th[k, 1], th[k, 2], amp=seg.amp)
        R[k] = (seg.d - h)[seg.kept].astype(np.float32)
    return R


def template_batch(seg: Segment, K: int, seed: int) -> np.ndarray:
    """H (K, n') float32, row k = kept samples of the template h(theta_k), theta_k
    from the chirp priors, with the segment's injection amplitude."""
    rng = np.random.default_rng(seed)
    T = seg.n / seg.fs
    th = draw_theta(rng, T, K)
    H = np.empty((K, seg.n_kept), dtype=np.float32)
    for k in range(K):
        H[k] = chirp(seg.n, seg.fs, th[k, 0], th[k, 1], th[k, 2], amp=seg.amp)[seg.kept].astype(np.float32)
    return H


def polarization_batch(seg: Segment, K: int, lw: int, seed: int):
    """Polarizations of K chirps on a waveform grid of lw samples at the
    segment's rate, with the coalescence on the last sample (h_plus with the
    cos phase, h_cross with the sin phase, the segment's injection amplitude),
    and per-template detector inputs: antenna factors F_plus, F_cross uniform
    in [-1, 1] and integer offsets (segment sample of waveform sample 0) that
    put the coalescence anywhere from before the segment's start to after its
    end.  Returns hp, hc float32 (K, lw); fp, fc float64 (K,); off int64 (K,)."""
    rng = np.random.default_rng(seed)
    th = draw_theta(rng, seg.n / seg.fs, K)
    t = np.arange(lw, dtype=np.float64) / seg.fs
    tc = lw / seg.fs
    hp = np.zeros((K, lw), dtype=np.float32)
    hc = np.zeros((K, lw), dtype=np.float32)
    for k in range(K):
        tau = tc - t
        on = tau > 1.0 / seg.fs
        ta = tau[on]
        phase = th[k, 2] - 2.0 * (ta / (5.0 * TSUN * th[k, 0])) ** 0.625
        amp = seg.amp * ta ** (-0.25)
        hp[k, on] = (amp * np.cos(phase)).astype(np.float32)
        hc[k, on] = (amp * np.sin(phase)).astype(np.float32)
    fp = rng.uniform(-1.0, 1.0, K)
    fc = rng.uniform(-1.0, 1.0, K)
    off = rng.integers(-lw // 4, seg.n - lw + lw // 4, K).astype(np.int64)
    return hp, hc, fp, fc, off


def noise_residuals(n: int, fs: float, K: int, seed: int, mask: np.ndarray | None = None,
                    a: float = -4.0, floor: float = 2.0, scale: float = 1.0) -> np.ndarray:
    """K pure-noise residuals on the kept samples, float32 (K, n')."""
    rng = np.random.default_rng(seed)
    x = noise_draw(n, fs, rng, a=a, floor=floor, scale=scale, count=K)
    kept = kept_index(mask, n)
    return np.ascontiguousarray(x[:, kept], dtype=np.float32)


def ar1_noise(n: int, phi: float, sigma2: float, K: int, seed: int,
              mask: np.ndarray | None = None) -> np.ndarray:
    """K draws of the stationary AR(1) process x_t = phi x_{t-1} + e_t,
    Var(e) = sigma2 (x_0 from the stationary law), on the kept samples,
    float32 (K, n')."""
    rng = np.random.default_rng(seed)
    e = rng.standard_normal((K, n)) * math.sqrt(sigma2)
    x = np.empty((K, n))
    x[:, 0] = e[:, 0] / math.sqrt(1.0 - phi * phi)
    for t in range(1, n):
        x[:, t] = phi * x[:, t - 1] + e[:, t]
    return np.ascontiguousarray(x[:, kept_index(mask, n)], dtype=np.float32)


# ----------------------------------------------------------------------------
# the configurations of the benchmark suite (shapes of the paper's segments)
# ----------------------------------------------------------------------------
SINGLE_N1024 = dict(name="single_n1024", n=1024, fs=1024.0, K=1, n_gaps=0, seed=1001)
GAPFREE_N8192_K4096 = dict(name="gapfree_n8192_k4096", n=8192, fs=2048.0, K=4096, n_gaps=0, seed=2002)
GAPPED_N16384_3DET = dict(name="gapped_n16384_3det_k1024", n=16384, fs=2048.0, K=1024, n_gaps=3,
            gap_len=512, scales=(1.0, 1.3, 2.1), seed=3003)


def serving_fleet(seed: int = 5005, count: int = 200) -> list[dict]:
    """The serving workload's resident segments: N uniform over {4096, 8192,
    16384, 32768} at 2048 Hz, 0-3 gaps of 512 samples each (seeded offsets),
    the reference PSD."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        n = int(rng.choice([4096, 8192, 16384, 32768]))
        g = int(rng.integers(0, 4))
        mask = gap_mask(n, g, 512, rng) if g else None
        out.append(dict(n=n, fs=2048.0, gaps=g, mask=mask, index=i))
    return out


def serving_pool(n: int, fs: float = 2048.0, count: int = 512, seed: int = 5151) -> np.ndarray:
    """Full-length residual pool shared by the serving workload's segments of
    length n: count coloured-noise draws, float32 (count, n); a segment's
    requests take the first K columns of pool[:, kept samples]."""
    return noise_residuals(n, fs, count, seed + n)


def mix64_segments(seed: int = 4004, count: int = 64) -> list[dict]:
    """64 disjoint segments: N log-uniform in [512, 32768] at 4096 Hz, K uniform
    in [16, 512], PSD exponent -4 +- 0.5 and floor 2 +- 1."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        n = int(round(math.exp(rng.uniform(math.log(512), math.log(32768)))))
        K = int(rng.integers(16, 513))
        a = float(rng.uniform(-4.5, -3.5))
        fl = float(rng.uniform(1.0, 3.0))
        out.append(dict(n=n, fs=4096.0, K=K, a=a, floor=fl, seed=seed * 1000 + i))
    return out
