"""The library's host-side size analysis (Sec. 5) against the oracle's:
Rios' and Hillert's densities and the two fits, through the C ABI on the
host (no device needed)."""
import json
import os

import numpy as np
import pytest

from oracle import lsgg_oracle as O

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_constants.json")


@pytest.fixture(scope="module")
def L():
    L = pytest.importorskip("paper_1701_06658_gb300.lsgg")
    try:
        L.lib()
    except Exception as e:          # library not built here
        pytest.skip(f"library unavailable: {e}")
    return L


def test_rios_and_hillert_match_the_oracle(L):
    z = np.linspace(0.0, 3.0, 61)
    for nu, rho in ((3.106, 0.863), (2.0, 0.75), (3.99, 8.0 / 9.0)):
        got = np.array([L.rios_pdf(float(q), nu, rho) for q in z])
        assert np.allclose(got, O.rios_pdf(z, nu, rho), rtol=1e-13, atol=1e-15)
    got = np.array([L.hillert_pdf(float(q)) for q in z])
    assert np.allclose(got, O.hillert_pdf(z), rtol=1e-13, atol=1e-15)
    assert np.isnan(L.rios_pdf(1.0, 4.5, 0.8)) and np.isnan(L.rios_pdf(1.0, 3.0, -1.0))


def test_rios_nu_fit_matches_the_oracle(L):
    c = json.load(open(GOLDEN))["size_distribution"]
    rng = np.random.default_rng(3)
    n_bins, r_max = 25, 2.5
    zc = (np.arange(n_bins) + 0.5) * (r_max / n_bins)
    hist = O.rios_pdf(zc, c["steady_nu"], c["steady_rho"]) * (r_max / n_bins)
    assert abs(L.fit_rios_nu(hist, r_max, c["steady_rho"]) - c["steady_nu"]) < 1e-6
    noisy = hist * (1.0 + 0.05 * rng.standard_normal(n_bins))
    assert abs(L.fit_rios_nu(noisy, r_max, c["steady_rho"]) - O.fit_rios_nu(noisy, r_max, c["steady_rho"])) < 1e-6


def test_growth_exponent_fit_matches_the_oracle(L):
    t = np.linspace(0.0, 300.0, 50)
    for n, k, r0 in ((0.5, 0.4, 4.0), (0.448, 0.15, 6.0)):
        r = (r0 ** (1.0 / n) + k * t) ** n
        fn, fk = L.fit_growth_exponent(t, r)
        assert abs(fn - n) < 1e-6 and abs(fk - k) < 1e-5 * k
    rng = np.random.default_rng(4)
    r = (4.0 ** 2 + 0.4 * t) ** 0.5 * (1.0 + 0.003 * rng.standard_normal(t.size))
    fn, fk = L.fit_growth_exponent(t, r)
    on, ok = O.fit_growth_exponent(t, r)
    assert abs(fn - on) < 1e-5 and abs(fk - ok) < 1e-4 * ok
    with pytest.raises(L.LsggError):
        L.fit_growth_exponent(t[::-1], r)
