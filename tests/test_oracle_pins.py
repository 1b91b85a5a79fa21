"""The CPU oracle against results fixed by mathematics (not by itself)."""
import types

import numpy as np
import pytest

import oracle
from oracle import td_oracle
from tests import pins


@pytest.mark.parametrize("name,check", pins.ALL_CHECKS, ids=[c[0] for c in pins.ALL_CHECKS])
def test_pin(name, check):
    check(oracle)


def test_gs_formula_itself():
    pins.check_gs_formula_small()


def test_spectral_bounds():
    pins.check_spectral_bounds(oracle)


def test_noise_chi2_distribution():
    pins.check_noise_chi2_distribution(oracle)


def test_not_positive_definite_pivot():
    acf = np.array([1.0, 2.0, 0.0, 0.0])
    with pytest.raises(oracle.NotPositiveDefinite) as e:
        oracle.OracleSegment(acf)
    assert e.value.pivot == 1


def test_whitening_round_trip():
    """d = L z  ->  L^{-1} d = z (the paper's noise draw, Sec. V.A.1)."""
    from paper_2603_06010_b300 import inputs
    acf = inputs.acf_from_psd(300, 1024.0)
    mask = np.ones(300, np.uint8)
    mask[40:90] = 0
    seg = oracle.OracleSegment(acf, mask)
    z = np.random.default_rng(3).standard_normal((seg.n_kept, 4))
    d = seg.L @ z
    W = td_oracle.whiten(seg.L, d)
    assert np.allclose(W, z, atol=1e-11)


def test_snr_definitions_white():
    """rho_mf and rho_eff for C = s2 I reduce to Euclidean products."""
    from paper_2603_06010_b300 import inputs
    n, s2 = 128, 3.0
    seg = oracle.OracleSegment(inputs.white_acf(n, s2))
    rng = np.random.default_rng(4)
    d = rng.standard_normal(n)
    h = rng.standard_normal(n)
    assert abs(oracle.mf_snr(seg, d, h) - (d @ h) / np.sqrt(s2 * (h @ h))) < 1e-12
    assert abs(oracle.eff_snr2(seg, d, h) - (2 * d @ h - h @ h) / s2) < 1e-11


# ---------------------------------------------------------------------------
# planted mistakes: every plausible slip in the oracle must fail some pin
# ---------------------------------------------------------------------------
def _mutant(kind):
    base = td_oracle.OracleSegment

    class Mut(base):
        def __init__(self, acf, mask=None):
            if kind == "gather_by_position":
                # C built from positions in the kept list, not sample times
                self.acf = np.asarray(acf, float)
                self.n = self.acf.shape[0]
                self.mask = mask
                self.kept = td_oracle.kept_indices(self.n, mask)
                i = np.arange(self.kept.size)
                self.C = self.acf[np.abs(i[:, None] - i[None, :])]
                self.L = td_oracle.cholesky(self.C)
                self.logdet = td_oracle.logdet(self.L)
            else:
                super().__init__(acf, mask)
                if kind == "logdet_half":
                    self.logdet = 0.5 * self.logdet
                if kind == "transposed_L":
                    self.L = np.ascontiguousarray(self.L.T)

        def whiten(self, R_kn):
            if kind == "transposed_L":
                import scipy.linalg as sla
                return sla.solve_triangular(self.L, np.atleast_2d(R_kn).T.astype(float), lower=False)
            return super().whiten(R_kn)

        def loglike(self, R_kn):
            ll = super().loglike(R_kn)
            if kind == "const_uses_n":
                ll = ll - 0.5 * (self.n - self.n_kept) * td_oracle.LOG2PI
            if kind == "sign_chi2":
                ll = ll + self.chi2(R_kn)
            return ll

    ns = types.SimpleNamespace(**{k: getattr(td_oracle, k) for k in dir(td_oracle) if not k.startswith("__")})
    ns.OracleSegment = Mut
    return ns


@pytest.mark.parametrize("kind", ["gather_by_position", "logdet_half", "transposed_L",
                                  "const_uses_n", "sign_chi2"])
def test_pins_catch_planted_mistake(kind):
    mut = _mutant(kind)
    failed = []
    for name, check in pins.ALL_CHECKS:
        try:
            check(mut)
        except AssertionError:
            failed.append(name)
    assert failed, f"no pin caught the planted mistake {kind}"


def _projection_mutant(kind):
    def project(n, hp, hc, fp, fc, offset):
        hp = np.asarray(hp, dtype=np.float64)
        hc = None if hc is None else np.asarray(hc, dtype=np.float64)
        lw = hp.shape[0]
        h = np.zeros(n)
        for t in range(n):
            u = {"off_by_one": t - offset + 1, "offset_sign": t + offset}.get(kind, t - offset)
            if kind == "wrap":
                u %= lw
            elif not 0 <= u < lw:
                continue
            v = fp * hp[u]
            if hc is not None and kind != "drop_cross":
                v += fc * (hp[u] if kind == "cross_on_plus" else hc[u])
            h[t] = v
        return h

    def projected_residual(seg, d_kept, hp, hc, fp, fc, offset):
        return np.asarray(d_kept, dtype=np.float64) - project(seg.n, hp, hc, fp, fc, offset)[seg.kept]

    ns = types.SimpleNamespace(**{k: getattr(td_oracle, k) for k in dir(td_oracle) if not k.startswith("__")})
    ns.project_template = project
    ns.projected_residual = projected_residual
    return ns


@pytest.mark.parametrize("kind", ["off_by_one", "offset_sign", "wrap", "drop_cross", "cross_on_plus"])
def test_projection_pin_catches_planted_mistake(kind):
    """Each plausible slip in the projection and placement fails the pin
    (the unmutated loop form of the same definition passes it)."""
    pins.check_projection(_projection_mutant("none"))
    with pytest.raises(AssertionError):
        pins.check_projection(_projection_mutant(kind))
