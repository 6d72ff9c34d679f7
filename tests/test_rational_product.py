"""The library's own Remez (host set-up of the C ABI's rational inputs)
against the oracle's, whose coefficients tests/golden/make_rationals.py
wrote: the relative-minimax approximation is unique, so both must agree
coefficient by coefficient."""
import json
import os

import numpy as np
import pytest

from paper_1010_5433_gb300 import rational

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "rationals.json")


def _close(r, g, tol):
    assert r.n == g["n"]
    np.testing.assert_allclose(r.beta, g["beta"], rtol=tol)
    np.testing.assert_allclose(r.alpha, g["alpha"], rtol=tol)
    assert abs(r.a0 - g["a0"]) <= tol * abs(g["a0"])
    assert abs(r.err - g["err"]) <= 1e-3 * g["err"]


@pytest.mark.parametrize("name", ["c1_md", "c2_md", "c4_md"])
def test_product_remez_matches_oracle(name):
    g = json.load(open(GOLDEN))[name]
    s, m, n = rational.WORKLOADS[name][:3]
    _close(rational.remez(s, m * m, 16 + m * m, n), g, 1e-9)


def test_shipped_table_matches_oracle():
    if not os.path.exists(rational.TABLE_PATH):
        pytest.skip("no shipped table")
    tab = json.load(open(rational.TABLE_PATH))
    gold = json.load(open(GOLDEN))
    common = [k for k in tab if k in gold]
    assert common
    for k in common:
        _close(rational.load(k), gold[k], 1e-8)


def test_positivity_and_heatbath_inverse():
    """x^(-s) approximations have alpha_i, beta_i > 0; r_hb(x)^2 r_met(x) = 1
    within the two approximation errors."""
    tab = json.load(open(GOLDEN))
    for k in ("c1_md", "c1_met", "c2_md"):
        assert min(tab[k]["alpha"]) > 0 and min(tab[k]["beta"]) > 0
    hb, met = tab["c1_hb"], tab["c1_met"]
    x = np.geomspace(hb["lo"], hb["hi"], 2001)
    rh = hb["a0"] + sum(a / (x + b) for a, b in zip(hb["alpha"], hb["beta"]))
    rm = met["a0"] + sum(a / (x + b) for a, b in zip(met["alpha"], met["beta"]))
    assert np.abs(rh * rh * rm - 1).max() < 3 * (2 * hb["err"] + met["err"]) + 1e-15


def test_golden_entry_is_what_the_committed_script_writes():
    """Provenance of the stored table: re-running the oracle's Remez with the
    script's own parameters reproduces the stored 4^4 MD entry to rounding."""
    import importlib.util
    spec = importlib.util.spec_from_file_location(
        "make_rationals", os.path.join(os.path.dirname(GOLDEN), "make_rationals.py"))
    mk = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mk)
    s, m, n = mk.TABLE["c1_md"]
    r = mk.remez(s, m * m, 16 + m * m, n, dps=60)
    g = json.load(open(GOLDEN))["c1_md"]
    np.testing.assert_allclose(r.beta, g["beta"], rtol=1e-13)
    np.testing.assert_allclose(r.alpha, g["alpha"], rtol=1e-13)
    assert abs(r.a0 - g["a0"]) <= 1e-13 * abs(g["a0"])


def test_improved_operator_rationals_cover_its_spectrum_bound():
    """The improved operator's workload rationals approximate on [m^2, m^2 + 64],
    which contains its A's spectrum bound m^2 + 58.8 (u0 = 1), and the shipped
    table agrees with the oracle's Remez there too."""
    import json as _json
    gold = _json.load(open(GOLDEN))
    for k in ("asqtad_md", "asqtad_met", "asqtad_hb"):
        r = rational.load(k)
        assert abs(r.lo - 0.02 ** 2) < 1e-15 and abs(r.hi - (64.0 + 0.02 ** 2)) < 1e-12
        assert r.hi - r.lo >= (4 * (5 / 8 + 6 / 16 + 24 / 64 + 48 / 384 + 6 / 16 + 1 / 24)) ** 2
        _close(r, gold[k], 1e-8)
