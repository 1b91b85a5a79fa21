"""Independent pins for the CPU oracle.

Each check takes an oracle-like namespace (anything with an OracleSegment
class) and raises AssertionError if the oracle disagrees with a result fixed
by mathematics rather than by the oracle itself:

* closed forms -- white noise, AR(1) with and without gaps (the whitened
  vector itself, not only chi2);
* brute force -- exact rational Gaussian elimination (N <= 24) and an
  80-bit Gauss-Jordan inverse (N = 64);
* Levinson-Durbin innovations and prediction-error variances (gap-free
  Toeplitz; Sec. II.B item 6 cites Levinson/Durbin for re-truncating the ACF);
* Gohberg-Semencul with FFT circulant-embedded Toeplitz products
  (Sec. III.A, GS formula and Eq. eq:toeplitz_fft), with C^{-1} e1 found by
  conjugate gradients on FFT matvecs;
* invariants -- PSD scale, time reversal, mirrored gaps, spectral bounds;
* a library density -- scipy's multivariate-normal log-density of the
  block-diagonal covariance of two gapped detectors (Sec. II.B item 3);
* LU on a gapped coloured segment (N' = 1299) -- chi2 and log det by numpy
  solve / slogdet;
* detector projection and placement -- energy of a placed waveform, nothing
  subtracted outside the segment or inside a gap, the plain template form as
  a special case, linearity in the antenna factors.

None of these call the oracle's own routines to produce an expected value.
"""
from __future__ import annotations

import math
from fractions import Fraction

import numpy as np

from paper_2603_06010_b300 import inputs

LOG2PI = math.log(2.0 * math.pi)


def _rel(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.max(np.abs(a - b) / np.maximum(np.abs(b), 1e-300)))


# ---------------------------------------------------------------------------
# white noise: C = sigma^2 I
# ---------------------------------------------------------------------------
def check_white(orc, n=96, sigma2=2.7, K=5, seed=11, gaps=True):
    rng = np.random.default_rng(seed)
    acf = inputs.white_acf(n, sigma2)
    mask = None
    if gaps:
        mask = np.ones(n, np.uint8)
        mask[10:17] = 0
        mask[40:41] = 0
        mask[n - 5:] = 0
    seg = orc.OracleSegment(acf, mask)
    nk = int(n if mask is None else mask.sum())
    R = rng.standard_normal((K, nk)).astype(np.float32)
    R64 = R.astype(np.float64)
    expect = -np.sum(R64 * R64, axis=1) / (2 * sigma2) - 0.5 * nk * math.log(2 * math.pi * sigma2)
    got = seg.loglike(R)
    assert np.allclose(got, expect, rtol=1e-13, atol=1e-10), (got, expect)
    assert abs(seg.logdet - nk * math.log(sigma2)) < 1e-10


# ---------------------------------------------------------------------------
# AR(1): x_t = phi x_{t-1} + e_t, Var e = s2.  Markov property gives the
# whitening of any kept subsequence in closed form.
# ---------------------------------------------------------------------------
def ar1_whiten_closed_form(r, t, phi, s2):
    """Sequential standardized innovations of kept samples t (increasing)."""
    r = np.asarray(r, dtype=np.float64)
    w = np.empty_like(r)
    var0 = s2 / (1 - phi * phi)
    w[0] = r[0] / math.sqrt(var0)
    logdet = math.log(var0)
    for i in range(1, len(t)):
        dlt = int(t[i] - t[i - 1])
        pd = phi ** dlt
        v = s2 * (1 - pd * pd) / (1 - phi * phi)
        w[i] = (r[i] - pd * r[i - 1]) / math.sqrt(v)
        logdet += math.log(v)
    return w, logdet


def check_ar1(orc, n=200, phi=0.83, s2=1.7, K=3, seed=12, gaps=False):
    rng = np.random.default_rng(seed)
    acf = inputs.ar1_acf(n, phi, s2)
    if gaps:
        mask = np.ones(n, np.uint8)
        mask[0:3] = 0
        mask[50:61] = 0
        mask[62:64] = 0     # adjacent-ish gaps, one kept sample between
        mask[120:121] = 0
        mask[n - 7:] = 0
    else:
        mask = None
    seg = orc.OracleSegment(acf, mask)
    t = np.arange(n) if mask is None else np.flatnonzero(mask)
    R = (rng.standard_normal((K, len(t))) * 3).astype(np.float32)
    W = seg.whiten(R)
    for k in range(K):
        w, ld = ar1_whiten_closed_form(R[k].astype(np.float64), t, phi, s2)
        assert np.allclose(W[:, k], w, rtol=1e-11, atol=1e-11), k
        assert abs(seg.logdet - ld) < 1e-9 * max(1.0, abs(ld))
    if mask is None:
        # the textbook gap-free log det: N log s2 - log(1 - phi^2)
        assert abs(seg.logdet - (n * math.log(s2) - math.log(1 - phi * phi))) < 1e-9
    ll = seg.loglike(R)
    chi = np.sum(W * W, axis=0)
    assert np.allclose(ll, -0.5 * chi - 0.5 * seg.logdet - 0.5 * len(t) * LOG2PI, rtol=1e-13)


# ---------------------------------------------------------------------------
# brute force: exact rationals
# ---------------------------------------------------------------------------
def _exact_solve_det(A, b):
    n = len(A)
    M = [[Fraction(A[i][j]) for j in range(n)] + [Fraction(b[i])] for i in range(n)]
    det = Fraction(1)
    for c in range(n):
        p = next(i for i in range(c, n) if M[i][c] != 0)
        if p != c:
            M[c], M[p] = M[p], M[c]
            det = -det
        det *= M[c][c]
        inv = 1 / M[c][c]
        for i in range(c + 1, n):
            f = M[i][c] * inv
            if f:
                for j in range(c, n + 1):
                    M[i][j] -= f * M[c][j]
    x = [Fraction(0)] * n
    for i in range(n - 1, -1, -1):
        s = M[i][n] - sum(M[i][j] * x[j] for j in range(i + 1, n))
        x[i] = s / M[i][i]
    return x, det


def check_bruteforce_exact(orc, seed=13):
    rng = np.random.default_rng(seed)
    # small-integer diagonally dominant symmetric Toeplitz -> SPD
    for n, mask in ((16, None), (22, np.array([1] * 4 + [0] * 3 + [1] * 9 + [0] + [1] * 5, np.uint8))):
        acf = np.zeros(n)
        acf[0] = 40
        acf[1:6] = [9, -7, 5, 3, -2]
        t = np.arange(n) if mask is None else np.flatnonzero(mask)
        A = [[int(acf[abs(int(t[i]) - int(t[j]))]) for j in range(len(t))] for i in range(len(t))]
        r = rng.integers(-9, 10, len(t))
        x, det = _exact_solve_det(A, [int(v) for v in r])
        chi_exact = float(sum(Fraction(int(r[i])) * x[i] for i in range(len(t))))
        seg = orc.OracleSegment(acf, mask)
        got = float(seg.chi2(r.astype(np.float32)[None, :])[0])
        assert abs(got - chi_exact) <= 1e-12 * abs(chi_exact), (got, chi_exact)
        assert abs(seg.logdet - math.log(float(det))) < 1e-12 * max(1, abs(seg.logdet))


def _gauss_jordan_inverse_ld(A):
    A = np.array(A, dtype=np.longdouble)
    n = A.shape[0]
    M = np.concatenate([A, np.eye(n, dtype=np.longdouble)], axis=1)
    logdet = np.longdouble(0)
    for c in range(n):
        p = c + int(np.argmax(np.abs(M[c:, c])))
        if p != c:
            M[[c, p]] = M[[p, c]]
        piv = M[c, c]
        logdet += np.log(np.abs(piv))
        M[c] = M[c] / piv
        for i in range(n):
            if i != c:
                M[i] = M[i] - M[i, c] * M[c]
    return M[:, n:], logdet


def check_bruteforce_longdouble(orc, seed=14):
    rng = np.random.default_rng(seed)
    n = 64
    acf = inputs.acf_from_psd(n, 512.0)
    mask = np.ones(n, np.uint8)
    mask[20:28] = 0
    t = np.flatnonzero(mask)
    A = acf[np.abs(t[:, None] - t[None, :])]
    Ainv, ld = _gauss_jordan_inverse_ld(A)
    R = (rng.standard_normal((4, len(t))) * 5).astype(np.float32)
    seg = orc.OracleSegment(acf, mask)
    got = seg.chi2(R)
    for k in range(4):
        r = R[k].astype(np.longdouble)
        chi = float(r @ Ainv @ r)
        assert abs(got[k] - chi) < 1e-11 * chi, (got[k], chi)
    assert abs(seg.logdet - float(ld)) < 1e-11 * max(1, abs(float(ld)))


# ---------------------------------------------------------------------------
# Levinson-Durbin (gap-free Toeplitz)
# ---------------------------------------------------------------------------
def levinson_innovations(acf, r):
    """Forward prediction-error filter of the Toeplitz ACF applied to r.
    Returns (whitened innovations, prediction-error variances)."""
    g = np.asarray(acf, dtype=np.float64)
    n = len(g)
    r = np.asarray(r, dtype=np.float64)
    v = np.empty(n)
    w = np.empty(n)
    v[0] = g[0]
    w[0] = r[0] / math.sqrt(v[0])
    a = np.zeros(0)                      # a[j-1] = a_{t,j}, predictor of x_t from x_{t-j}
    for t in range(1, n):
        kap = (g[t] - np.dot(a, g[t - 1:0:-1])) / v[t - 1]
        a = np.concatenate([a - kap * a[::-1], [kap]])
        v[t] = v[t - 1] * (1 - kap * kap)
        e = r[t] - np.dot(a, r[t - 1::-1][:t])
        w[t] = e / math.sqrt(v[t])
    return w, v


def check_levinson(orc, n=384, fs=1024.0, seed=15):
    rng = np.random.default_rng(seed)
    acf = inputs.acf_from_psd(n, fs)
    seg = orc.OracleSegment(acf, None)
    R = (rng.standard_normal((3, n)) * 8).astype(np.float32)
    W = seg.whiten(R)
    for k in range(3):
        w, v = levinson_innovations(acf, R[k])
        assert np.allclose(W[:, k], w, rtol=1e-9, atol=1e-9 * np.max(np.abs(w)))
        if k == 0:
            assert abs(seg.logdet - float(np.sum(np.log(v)))) < 1e-9 * abs(seg.logdet)


# ---------------------------------------------------------------------------
# Gohberg-Semencul + circulant embedding (Sec. III.A)
# ---------------------------------------------------------------------------
def toeplitz_matvec_fft(col, row, v):
    """T v with T the Toeplitz matrix of first column col and first row row,
    via the 2n circulant embedding (Eq. eq:toeplitz_fft)."""
    n = len(col)
    m = 2 * n
    c = np.zeros(m)
    c[:n] = col
    c[n + 1:] = row[:0:-1]
    vp = np.zeros(m)
    vp[:n] = v
    return np.fft.irfft(np.fft.rfft(c) * np.fft.rfft(vp), n=m)[:n]


def cg_toeplitz(acf, b, tol=1e-15, maxit=5000):
    x = np.zeros_like(b)
    r = b.copy()
    p = r.copy()
    rr = r @ r
    nb = math.sqrt(b @ b)
    for _ in range(maxit):
        Ap = toeplitz_matvec_fft(acf, acf, p)
        al = rr / (p @ Ap)
        x += al * p
        r -= al * Ap
        rn = r @ r
        if math.sqrt(rn) < tol * nb:
            break
        p = r + (rn / rr) * p
        rr = rn
    return x


def gs_chi2(acf, x, r):
    """r^T C^{-1} r = (1/x1)(|L_x^T r|^2 - |R_x r|^2), C x = e1."""
    n = len(x)
    z = np.zeros(n)
    LxT_r = toeplitz_matvec_fft(np.r_[x[0], z[1:]], x, r)          # upper Toeplitz, first row x
    rrow = np.r_[0.0, x[:0:-1]]                                     # (0, x_n, ..., x_2)
    Rx_r = toeplitz_matvec_fft(z, rrow, r)
    return (LxT_r @ LxT_r - Rx_r @ Rx_r) / x[0]


def check_gs_formula_small():
    """The GS inverse formula itself against an explicit inverse (N = 12)."""
    n = 12
    acf = inputs.acf_from_psd(n, 256.0)
    C = acf[np.abs(np.arange(n)[:, None] - np.arange(n)[None, :])]
    Ci = np.linalg.inv(C)
    x = Ci[:, 0]
    Lx = np.array([[x[i - j] if i >= j else 0.0 for j in range(n)] for i in range(n)])
    rrow = np.r_[0.0, x[:0:-1]]
    Rx = np.array([[rrow[j - i] if j >= i else 0.0 for j in range(n)] for i in range(n)])
    G = (Lx @ Lx.T - Rx.T @ Rx) / x[0]
    assert np.allclose(G, Ci, rtol=1e-9, atol=1e-12 * np.max(np.abs(Ci)))


def check_gs(orc, n=2048, fs=2048.0, seed=16):
    rng = np.random.default_rng(seed)
    acf = inputs.acf_from_psd(n, fs)
    e1 = np.zeros(n)
    e1[0] = 1.0
    x = cg_toeplitz(acf, e1)
    seg = orc.OracleSegment(acf, None)
    R = (rng.standard_normal((2, n)) * 9).astype(np.float32)
    got = seg.chi2(R)
    for k in range(2):
        ref = gs_chi2(acf, x, R[k].astype(np.float64))
        assert abs(got[k] - ref) < 1e-9 * ref, (got[k], ref)


# ---------------------------------------------------------------------------
# invariants
# ---------------------------------------------------------------------------
def check_scaling(orc, n=300, fs=1024.0, s=2.1, seed=17):
    rng = np.random.default_rng(seed)
    mask = np.ones(n, np.uint8)
    mask[100:140] = 0
    a1 = inputs.acf_from_psd(n, fs)
    a2 = inputs.acf_from_psd(n, fs, scale=s)
    s1 = orc.OracleSegment(a1, mask)
    s2 = orc.OracleSegment(a2, mask)
    nk = int(mask.sum())
    R = (rng.standard_normal((3, nk)) * 6).astype(np.float32)
    assert abs(s2.logdet - (s1.logdet + nk * math.log(s))) < 1e-9 * abs(s1.logdet)
    assert np.allclose(s2.chi2(R), s1.chi2(R) / s, rtol=1e-10)


def check_reversal(orc, n=257, fs=1024.0, seed=18):
    rng = np.random.default_rng(seed)
    acf = inputs.acf_from_psd(n, fs)
    R = (rng.standard_normal((2, n)) * 6).astype(np.float32)
    seg = orc.OracleSegment(acf, None)
    assert np.allclose(seg.chi2(R), seg.chi2(R[:, ::-1].copy()), rtol=1e-10)
    mask = np.ones(n, np.uint8)
    mask[30:90] = 0
    mask[200:203] = 0
    g1 = orc.OracleSegment(acf, mask)
    g2 = orc.OracleSegment(acf, mask[::-1].copy())
    Rk = R[:, mask.astype(bool)]
    assert np.allclose(g1.chi2(Rk), g2.chi2(Rk[:, ::-1].copy()), rtol=1e-10)
    assert abs(g1.logdet - g2.logdet) < 1e-10 * abs(g1.logdet)


def check_spectral_bounds(orc, n=512, fs=2048.0):
    acf = inputs.acf_from_psd(n, fs)
    S = inputs.psd_grid(n, fs)
    mask = np.ones(n, np.uint8)
    mask[64:128] = 0
    C = orc.build_cov(acf, mask)
    ev = np.linalg.eigvalsh(C)
    assert ev.min() >= S.min() * (1 - 1e-9) and ev.max() <= S.max() * (1 + 1e-9)


def check_noise_chi2_distribution(orc, n=512, fs=2048.0, K=800, seed=19):
    """chi2 of noise-only residuals ~ chi-square(N'): mean N', variance 2N'.
    Noise comes from circulant embedding, independent of the oracle."""
    from scipy import stats
    mask = np.ones(n, np.uint8)
    mask[100:164] = 0
    nk = int(mask.sum())
    R = inputs.noise_residuals(n, fs, K, seed, mask=mask)
    seg = orc.OracleSegment(inputs.acf_from_psd(n, fs), mask)
    c = seg.chi2(R)
    assert abs(c.mean() - nk) < 5 * math.sqrt(2 * nk / K), (c.mean(), nk)
    assert abs(c.var() / (2 * nk) - 1) < 0.25
    assert stats.kstest(c, stats.chi2(nk).cdf).pvalue > 1e-3
    W = seg.whiten(R)
    assert abs(W.mean()) < 0.01 and abs(W.std() - 1) < 0.01


# ---------------------------------------------------------------------------
# library density: the full logL (whitening, log det and the constant) of two
# gapped detectors against scipy's multivariate-normal log-density of the
# block-diagonal covariance (an eigendecomposition, no Cholesky)
# ---------------------------------------------------------------------------
def check_mvn_joint(orc, seed=20):
    from scipy import linalg, stats
    rng = np.random.default_rng(seed)
    segs, blocks, Rs = [], [], []
    for n, fs, gap in ((180, 1024.0, (20, 55)), (137, 2048.0, (100, 104))):
        acf = inputs.acf_from_psd(n, fs)
        mask = np.ones(n, np.uint8)
        mask[gap[0]:gap[1]] = 0
        keep = np.flatnonzero(mask)
        blocks.append(linalg.toeplitz(acf)[np.ix_(keep, keep)])
        segs.append(orc.OracleSegment(acf, mask))
        Rs.append((rng.standard_normal((4, keep.size)) * 3).astype(np.float32))
    C = linalg.block_diag(*blocks)
    X = np.concatenate([R.astype(np.float64) for R in Rs], axis=1)
    expect = stats.multivariate_normal(mean=np.zeros(C.shape[0]), cov=C).logpdf(X)
    got = orc.joint_loglike(segs, Rs)
    assert np.allclose(got, expect, rtol=1e-10, atol=1e-8), (got, expect)


# ---------------------------------------------------------------------------
# detector projection and placement of a template (Sec. II.B waveform
# conditioning, Sec. III.A data projection and conditioning)
# ---------------------------------------------------------------------------
def check_projection(orc, seed=21):
    rng = np.random.default_rng(seed)
    n, lw, s2 = 160, 48, 1.9
    hp = rng.standard_normal(lw)
    hc = rng.standard_normal(lw)
    fp, fc = 0.62, -0.47
    white = orc.OracleSegment(inputs.white_acf(n, s2))
    zero = np.zeros(n)
    # placed fully inside the segment, anywhere: the energy of the detector
    # signal is fp^2|hp|^2 + 2 fp fc <hp, hc> + fc^2 |hc|^2, so with d = 0 and
    # white noise chi2 = that / s2 whatever the offset
    energy = fp * fp * (hp @ hp) + 2 * fp * fc * (hp @ hc) + fc * fc * (hc @ hc)
    for off in (0, 1, 37, n - lw):
        r = orc.projected_residual(white, zero, hp, hc, fp, fc, off)
        assert abs(float(white.chi2(r[None, :])[0]) - energy / s2) < 1e-10 * energy / s2, off
    # outside the segment entirely (before or after): nothing is subtracted
    d = rng.standard_normal(n)
    for off in (n, n + 5, -lw, -lw - 9):
        assert np.array_equal(orc.projected_residual(white, d, hp, hc, fp, fc, off), d), off
    # fp = 1, fc = 0, offset 0 and a waveform as long as the segment: the plain
    # template form d - h, sample for sample
    hfull = rng.standard_normal(n)
    r = orc.projected_residual(white, d, hfull, None, 1.0, 0.0, 0)
    assert np.array_equal(r, d - hfull)
    # partly outside: only the overlap is subtracted (first and last samples)
    r = orc.projected_residual(white, zero, hp, None, 1.0, 0.0, -10)
    assert np.array_equal(-r[:lw - 10], hp[10:]) and np.all(r[lw - 10:] == 0)
    r = orc.projected_residual(white, zero, hp, None, 1.0, 0.0, n - 10)
    assert np.array_equal(-r[n - 10:], hp[:10]) and np.all(r[:n - 10] == 0)
    # linear in the antenna factors
    a = orc.projected_residual(white, zero, hp, hc, 1.0, 0.0, 20)
    b = orc.projected_residual(white, zero, hp, hc, 0.0, 1.0, 20)
    c = orc.projected_residual(white, zero, hp, hc, fp, fc, 20)
    assert np.allclose(c, fp * a + fc * b, rtol=0, atol=1e-14)
    # gaps: a waveform that lies inside a gap subtracts nothing; one that
    # straddles the gap's edge keeps exactly its samples on kept times
    mask = np.ones(n, np.uint8)
    mask[60:120] = 0
    g = orc.OracleSegment(inputs.white_acf(n, s2), mask)
    dk = rng.standard_normal(int(mask.sum()))
    assert np.array_equal(orc.projected_residual(g, dk, hp, hc, fp, fc, 65), dk)
    r = orc.projected_residual(g, np.zeros(int(mask.sum())), hp, None, 1.0, 0.0, 40)
    assert np.array_equal(-r[40:60], hp[:20]) and np.all(r[60:] == 0) and np.all(r[:40] == 0)


# ---------------------------------------------------------------------------
# gapped coloured segment at moderate N': chi2 = r^T C^{-1} r and log det C by
# LU (numpy solve / slogdet), a factorisation the oracle does not use
# ---------------------------------------------------------------------------
def check_lu_gapped(orc, n=1500, fs=2048.0, seed=22):
    from scipy import linalg
    rng = np.random.default_rng(seed)
    mask = np.ones(n, np.uint8)
    mask[200:330] = 0
    mask[900:971] = 0
    keep = np.flatnonzero(mask)
    acf = inputs.acf_from_psd(n, fs)
    C = linalg.toeplitz(acf)[np.ix_(keep, keep)]
    R = (rng.standard_normal((3, keep.size)) * 5).astype(np.float32)
    seg = orc.OracleSegment(acf, mask)
    X = np.linalg.solve(C, R.astype(np.float64).T)
    chi2 = np.einsum("ij,ij->j", R.astype(np.float64).T, X)
    sign, ld = np.linalg.slogdet(C)
    assert sign > 0
    assert abs(seg.logdet - ld) < 1e-9 * abs(ld), (seg.logdet, ld)
    assert np.allclose(seg.chi2(R), chi2, rtol=1e-10), (seg.chi2(R), chi2)


ALL_CHECKS = [
    ("white", lambda o: (check_white(o, gaps=False), check_white(o, gaps=True))),
    ("ar1", lambda o: check_ar1(o, gaps=False)),
    ("ar1_gapped", lambda o: check_ar1(o, gaps=True)),
    ("bruteforce_exact", check_bruteforce_exact),
    ("bruteforce_longdouble", check_bruteforce_longdouble),
    ("levinson", check_levinson),
    ("gs", check_gs),
    ("scaling", check_scaling),
    ("reversal", check_reversal),
    ("mvn_joint", check_mvn_joint),
    ("projection", check_projection),
    ("lu_gapped", check_lu_gapped),
]
