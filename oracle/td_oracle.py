"""CPU FP64 oracle for the time-domain Gaussian likelihood.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path imports, calls or
links this module: only tests/, __graft_entry__.smoke() and bench.py's CPU
baseline leg use it.  It shares no code with the CUDA path.

It is a plain, slow, direct statement of the likelihood of paper Sec. II:

* C_ij = rho(|t_i - t_j|) over the kept sample indices t (Sec. II, the
  stationary-noise covariance; Sec. II.B items 1-2, segments and gaps:
  gap samples are deleted, so C is the kept x kept principal submatrix of
  the segment's Toeplitz matrix).
* C = L L^T with L lower triangular (Sec. II.A, Cholesky whitening).
* W = L^{-1} R, one column per residual r = d - h(theta) (Sec. II.A, the
  whitened residual; Eq. eq:td_like_whitened).
* chi2_k = sum_i W_ik^2  (= r^T C^{-1} r, Eq. eqn:ip).
* logdet C = 2 sum_i log L_ii.
* logL_k = -chi2_k / 2 - logdet / 2 - (N'/2) log(2 pi)  (Eq. eqn:lik and
  eq:td_like_whitened with the constant written out; N' = kept count).
* Joint multi-detector logL = sum of per-detector logL (Sec. II.B item 3).

Library primitives serve as steps: LAPACK dpotrf for the Cholesky and
dtrtrs for the forward substitution (via scipy), numpy pairwise summation
for the FP64 chi2.  No blocking, fusion or reordering is added.

Residuals arrive as float32 and are promoted exactly to float64 (the FP32
rounding of d - h is part of the input, not an error of the method).

Also here (the NEXT rows of the hot path, Sec. II.B item 7 and Sec. III.A):
matched-filter and effective SNR definitions, and the detector projection and
placement of a template (Sec. II.B waveform conditioning, Sec. III.A data
projection and conditioning).
"""
from __future__ import annotations

import math
import os
import time

import numpy as np
import scipy.linalg as sla

LOG2PI = math.log(2.0 * math.pi)


class NotPositiveDefinite(ValueError):
    def __init__(self, pivot: int):
        super().__init__(f"covariance not positive definite at pivot {pivot}")
        self.pivot = pivot   # 0-based index of the first failing pivot


def kept_indices(n: int, mask) -> np.ndarray:
    """Kept sample indices t_0 < ... < t_{N'-1} (Sec. II.B item 2)."""
    if mask is None:
        return np.arange(n, dtype=np.int64)
    mask = np.asarray(mask)
    if mask.shape != (n,):
        raise ValueError("mask must have n entries")
    return np.flatnonzero(mask != 0).astype(np.int64)


def build_cov(acf, mask=None) -> np.ndarray:
    """Dense FP64 C_kept[i, j] = acf[|t_i - t_j|] (Sec. II and II.B)."""
    acf = np.asarray(acf, dtype=np.float64)
    n = acf.shape[0]
    t = kept_indices(n, mask)
    lag = np.abs(t[:, None] - t[None, :])
    return acf[lag]


def cholesky(C: np.ndarray) -> np.ndarray:
    """Lower-triangular L with C = L L^T (Sec. II.A).  LAPACK dpotrf."""
    L, info = sla.lapack.dpotrf(np.asarray(C, dtype=np.float64), lower=1, clean=1,
                                overwrite_a=0)
    if info > 0:
        raise NotPositiveDefinite(info - 1)
    if info < 0:
        raise ValueError("dpotrf argument error")
    return L


def logdet(L: np.ndarray) -> float:
    """log det C = 2 sum log L_ii (the constant of Eq. eqn:lik)."""
    return 2.0 * float(np.sum(np.log(np.diag(L))))


def whiten(L: np.ndarray, R) -> np.ndarray:
    """W = L^{-1} R by forward substitution (Sec. II.A).  R: (N', K) or (N',).
    LAPACK dtrtrs through scipy."""
    R64 = np.asarray(R, dtype=np.float64)
    return sla.solve_triangular(L, R64, lower=True, check_finite=False)


def chi2(W: np.ndarray) -> np.ndarray:
    """chi2_k = sum_i W_ik^2 in FP64 (pairwise summation along i)."""
    W = np.asarray(W, dtype=np.float64)
    if W.ndim == 1:
        return np.asarray(np.sum(W * W))
    Wt = np.ascontiguousarray(W.T)          # sum along a contiguous axis -> pairwise
    return np.sum(Wt * Wt, axis=1)


def loglike_from_chi2(chi2_k, logdet_c: float, n_kept: int):
    """logL = -chi2/2 - logdet/2 - (N'/2) log 2 pi."""
    return -0.5 * np.asarray(chi2_k) - 0.5 * logdet_c - 0.5 * n_kept * LOG2PI


class OracleSegment:
    """One segment (one detector, one time window) of the FP64 oracle."""

    def __init__(self, acf, mask=None):
        self.acf = np.asarray(acf, dtype=np.float64).copy()
        self.n = self.acf.shape[0]
        self.mask = None if mask is None else np.asarray(mask, dtype=np.uint8).copy()
        self.kept = kept_indices(self.n, self.mask)
        self.C = build_cov(self.acf, self.mask)
        self.L = cholesky(self.C)
        self.logdet = logdet(self.L)

    @property
    def n_kept(self) -> int:
        return int(self.kept.size)

    def whiten(self, R_kn) -> np.ndarray:
        """R given as (K, N') rows (column-major N' x K buffer) -> W (N', K)."""
        R_kn = np.atleast_2d(np.asarray(R_kn))
        return whiten(self.L, R_kn.T)

    def chi2(self, R_kn) -> np.ndarray:
        return chi2(self.whiten(R_kn))

    def loglike(self, R_kn) -> np.ndarray:
        return loglike_from_chi2(self.chi2(R_kn), self.logdet, self.n_kept)


def joint_loglike(segments, residuals) -> np.ndarray:
    """Multi-detector logL: per-detector logL summed (Sec. II.B item 3)."""
    total = None
    for seg, R in zip(segments, residuals):
        ll = seg.loglike(R)
        total = ll if total is None else total + ll
    return total


# ---------------------------------------------------------------------------
# SNR definitions (Sec. II.B item 7)
# ---------------------------------------------------------------------------
def inner(seg: OracleSegment, s, h) -> float:
    """<s, h> = s^T C^{-1} h (Eq. eqn:ip), via the whitened vectors."""
    ws = seg.whiten(np.asarray(s)[None, :])[:, 0]
    wh = seg.whiten(np.asarray(h)[None, :])[:, 0]
    return float(np.dot(ws, wh))


def mf_snr(seg: OracleSegment, d, h) -> float:
    """rho_mf = <d, h> / sqrt(<h, h>)."""
    return inner(seg, d, h) / math.sqrt(inner(seg, h, h))


def eff_snr2(seg: OracleSegment, d, h) -> float:
    """rho_eff^2 = <d, d> - <r, r>, r = d - h."""
    r = np.asarray(d) - np.asarray(h)
    return inner(seg, d, d) - inner(seg, r, r)


# ---------------------------------------------------------------------------
# Detector projection and placement of a template (Sec. II.B, waveform
# conditioning; Sec. III.A, data projection and conditioning)
# ---------------------------------------------------------------------------
def project_template(n: int, hp, hc, fp: float, fc: float, offset: int) -> np.ndarray:
    """Detector-frame template on the segment's n sample times, FP64.

    The polarizations are combined with the detector's antenna factors,
    h = fp h_plus + fc h_cross, and the result is placed so that waveform
    sample u lands on segment sample t = u + offset; segment samples that no
    waveform sample reaches are zero (the zero padding that positions the
    peak).  Waveform samples that fall outside the segment are dropped.
    hc = None means no cross polarization."""
    hp = np.asarray(hp, dtype=np.float64)
    lw = hp.shape[0]
    h = np.zeros(n)
    t = np.arange(n)
    u = t - int(offset)
    on = (u >= 0) & (u < lw)
    h[on] = fp * hp[u[on]]
    if hc is not None:
        h[on] = h[on] + fc * np.asarray(hc, dtype=np.float64)[u[on]]
    return h


def projected_residual(seg: OracleSegment, d_kept, hp, hc, fp: float, fc: float, offset: int) -> np.ndarray:
    """r = d - h over the kept samples, FP64 (d given on the kept samples)."""
    h = project_template(seg.n, hp, hc, fp, fc, offset)
    return np.asarray(d_kept, dtype=np.float64) - h[seg.kept]


# ---------------------------------------------------------------------------
# CPU timing of the per-evaluation path (used only by bench.py's baseline leg)
# ---------------------------------------------------------------------------
def time_per_eval_path(seg: OracleSegment, R_kn, threads: int | None = None,
                       min_seconds: float = 0.0):
    """Time whiten + chi2 + logL for the columns of R_kn on `threads` BLAS
    threads (default: all host cores).  Returns (seconds, threads_used)."""
    import contextlib
    ncpu = os.cpu_count() or 1
    threads = threads or ncpu
    try:
        from threadpoolctl import threadpool_limits
        ctx = threadpool_limits(limits=threads)
    except ImportError:
        if threads < ncpu:       # a thread count below the BLAS default cannot be honoured
            raise RuntimeError("threadpoolctl is needed to time the oracle on fewer than all host cores")
        ctx = contextlib.nullcontext()
    with ctx:
        reps = 0
        t0 = time.perf_counter()
        while True:
            seg.loglike(R_kn)
            reps += 1
            el = time.perf_counter() - t0
            if el >= min_seconds:
                break
    return el / reps, threads
