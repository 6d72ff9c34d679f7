"""Pins for the high-degree rational approximations the workloads use (paper
Sec. 2: separate rationals for the molecular dynamics and for the heatbath
and Metropolis steps), evaluated exactly (mpmath, 40 digits) from the stored
double coefficients of tests/golden/rationals.json:

  * Chebyshev alternation of the relative error e(x) = r(x) x^s - 1 on
    [m^2, 16 + m^2]: 2n+1 sign changes, 2n+2 extrema (both end points among
    them) of alternating sign, each of magnitude err up to the rounding of
    the coefficients to doubles;
  * positivity of the partial fractions (alpha_i > 0 for x^-s, every
    beta_i > 0, so each (A + beta_i) is positive definite);
  * the heatbath and Metropolis rationals of one flavour are consistent:
    r_hb(x)^2 r_met(x) = 1 within their two errors.

Rounding of the coefficients: each stored alpha_i, beta_i, a0 carries a
relative error <= 2^-53, so every term alpha_i / (x + beta_i) moves by a
relative <= 2^-52 and r by <= 2^-52 kappa(x) |r|, kappa(x) = (|a0| +
sum |alpha_i / (x + beta_i)|) / |r(x)|; hence |e_stored - e| <= 2^-52
kappa (1 + err).  For x^-s all terms are positive (kappa = 1); the
heatbath rationals of x^(+s/2) have alpha_i < 0 and cancel (kappa up to 91
for 16^4), so their stored doubles are accurate to 2^-52 kappa rather than
err (2.2e-15 for the 16^4 heatbath, far below its 1e-12 solver tolerance).
Where that rounding band exceeds err / 2 the alternation itself is not
resolvable in doubles, and the pin is the accuracy bound and the
consistency with the Metropolis rational.  The oracle's Remez stops when
the extrema agree to a relative 1e-6."""
import json
import os

import mpmath as mp
import numpy as np
import pytest

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "rationals.json")
ROUND = 2.0 ** -52


def _table():
    return json.load(open(GOLDEN))


def _coeffs(d):
    return mp.mpf(d["a0"]), [mp.mpf(a) for a in d["alpha"]], [mp.mpf(b) for b in d["beta"]], mp.mpf(d["s"])


def _target_inv(d, x):
    """1 / the approximated function at x: x^s, or (x / (x + delta))^s for a mass ratio."""
    s, delta = mp.mpf(d["s"]), mp.mpf(d.get("delta", 0.0))
    return x ** s if delta == 0 else (x / (x + delta)) ** s


def _err_fn(d):
    a0, al, be, s = _coeffs(d)

    def e(u):                      # u = log x
        x = mp.e ** u
        return (a0 + mp.fsum(a / (x + b) for a, b in zip(al, be))) * _target_inv(d, x) - 1
    return e


def _rounding_band(d, n_grid=800):
    """max over x of 2^-52 kappa(x) (1 + err) and of |e_stored(x)|."""
    with mp.workdps(40):
        a0, al, be, s = _coeffs(d)
        lo, hi = mp.log(mp.mpf(d["lo"])), mp.log(mp.mpf(d["hi"]))
        band = worst = 0.0
        for k in range(n_grid):
            x = mp.e ** (lo + (hi - lo) * k / (n_grid - 1))
            terms = [a / (x + b) for a, b in zip(al, be)]
            r = a0 + mp.fsum(terms)
            kappa = (abs(a0) + mp.fsum(abs(q) for q in terms)) / abs(r)
            band = max(band, float(kappa) * ROUND * (1 + d["err"]))
            worst = max(worst, float(abs(r * _target_inv(d, x) - 1)))
        return band, worst


def _extrema(d, n_grid=6000):
    """Extremum value of e in each interval between consecutive sign changes
    (and the end points), located on a log grid and refined by golden
    section."""
    with mp.workdps(40):
        e = _err_fn(d)
        lo, hi = mp.log(mp.mpf(d["lo"])), mp.log(mp.mpf(d["hi"]))
        us = [lo + (hi - lo) * k / (n_grid - 1) for k in range(n_grid)]
        es = [e(u) for u in us]
        cuts = [0] + [k for k in range(1, n_grid) if (es[k] > 0) != (es[k - 1] > 0)] + [n_grid]
        ext = []
        for a, b in zip(cuts[:-1], cuts[1:]):
            k = max(range(a, b), key=lambda j: abs(es[j]))
            if k in (0, n_grid - 1):           # the end points are extrema themselves
                ext.append(float(es[k]))
                continue
            x0, x1 = us[max(k - 1, 0)], us[min(k + 1, n_grid - 1)]
            g = (mp.sqrt(5) - 1) / 2
            c, dd = x1 - g * (x1 - x0), x0 + g * (x1 - x0)
            for _ in range(60):
                if abs(e(c)) > abs(e(dd)):
                    x1, dd = dd, c
                    c = x1 - g * (x1 - x0)
                else:
                    x0, c = c, dd
                    dd = x0 + g * (x1 - x0)
            ext.append(float(max((e(c), e(dd), es[k]), key=abs)))
        return ext, len(cuts) - 2


HIGH = ["c2_md", "c2_met", "c2_hb", "c3_light_md", "c3_light_met", "c3_light_hb", "c3_strange_md",
        "c3_strange_met", "c3_strange_hb", "c4_md", "c4_met", "c4_hb", "c1_met", "c1_hb",
        "t3_high_md", "t3_high_met", "t3_high_hb", "t3_low_md", "t3_low_met", "t3_low_hb",
        "c2_pf2_md", "c2_pf2_met", "c2_pf2_hb", "c2_pf3_md", "c2_pf3_met", "c2_pf3_hb",
        "c2_pf4_md", "c2_pf4_met", "c2_pf4_hb", "c2_heavy_md", "c2_heavy_met", "c2_heavy_hb",
        "c2_ratio_md", "c2_ratio_met", "c2_ratio_hb"]


@pytest.mark.parametrize("name", HIGH)
def test_stored_rational_is_accurate_to_its_error(name):
    """max |e_stored| <= err (1 + 1e-6) + the rounding band, everywhere."""
    d = _table()[name]
    band, worst = _rounding_band(d)
    assert worst <= d["err"] * (1 + 1e-6) + band, (worst, d["err"], band)
    if name.endswith("_met") or name.endswith("_md"):
        assert band <= 1.01 * ROUND * (1 + d["err"])       # no cancellation for x^-s


@pytest.mark.parametrize("name", HIGH)
def test_stored_rational_equioscillates(name):
    d = _table()[name]
    band, _ = _rounding_band(d)
    if band > 0.5 * d["err"]:
        pytest.skip(f"{name}: coefficient rounding {band:.1e} exceeds err/2 = {d['err'] / 2:.1e}")
    n = d["n"]
    ext, zeros = _extrema(d)
    assert zeros == 2 * n + 1, f"{name}: {zeros} sign changes, want {2 * n + 1}"
    assert len(ext) == 2 * n + 2
    assert all(np.sign(ext[k]) == -np.sign(ext[k - 1]) for k in range(1, len(ext)))
    tol = 1e-6 * d["err"] + band + 1e-3 * d["err"]     # Remez stop, coefficient rounding, refinement grid
    dev = max(abs(abs(v) - d["err"]) for v in ext)
    assert dev <= tol, f"{name}: extrema {min(map(abs, ext)):.3e}..{max(map(abs, ext)):.3e}, err {d['err']:.3e}"


@pytest.mark.parametrize("name", [k for k in HIGH if not k.endswith("_hb")])
def test_inverse_power_rationals_have_positive_partial_fractions(name):
    d = _table()[name]
    assert d["s"] > 0 and d["a0"] > 0
    assert min(d["alpha"]) > 0 and min(d["beta"]) > 0


@pytest.mark.parametrize("flavour", ["c1", "c2", "c3_light", "c3_strange", "c4", "t3_high", "t3_low", "c2_pf2",
                                     "c2_pf3", "c2_pf4", "c2_heavy", "c2_ratio"])
def test_heatbath_and_metropolis_rationals_are_inverse(flavour):
    """phi = r_hb(A) xi makes phi^dag r_met(A) phi = xi^dag xi exactly only
    if r_hb^2 r_met = 1; the stored pair meets it within twice the heatbath
    rational's stored accuracy plus the Metropolis one's, checked at 400
    points in exact arithmetic.  With the Metropolis rational pinned by its
    alternation, this pins the heatbath rational to the same function."""
    t = _table()
    hb, met = t[flavour + "_hb"], t[flavour + "_met"]
    assert hb["s"] == -met["s"] / 2 and hb["lo"] == met["lo"] and hb["hi"] == met["hi"]
    assert min(hb["beta"]) > 0
    band_hb, _ = _rounding_band(hb, 200)
    band_met, _ = _rounding_band(met, 200)
    bound = 2 * (hb["err"] * (1 + 1e-6) + band_hb) + met["err"] * (1 + 1e-6) + band_met
    with mp.workdps(40):
        def r(d, x):
            return mp.mpf(d["a0"]) + mp.fsum(mp.mpf(a) / (x + mp.mpf(b)) for a, b in zip(d["alpha"], d["beta"]))
        lo, hi = mp.log(mp.mpf(hb["lo"])), mp.log(mp.mpf(hb["hi"]))
        worst = 0.0
        for k in range(400):
            x = mp.e ** (lo + (hi - lo) * k / 399)
            worst = max(worst, float(abs(r(hb, x) ** 2 * r(met, x) - 1)))
    assert worst <= 1.01 * bound, (worst, bound)
