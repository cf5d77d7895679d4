"""The GPU step (FP64 fields, through the C ABI) against the numbers printed
in the paper's Tables 1-6 (tests/golden/paper_tables.json, cited): full runs
of the thin ellipse and thick shell problems at N up to 512.

Tolerances: E[div u; N] is printed with three digits: 1.5%.  Rates: the
velocity and marker rates within 0.08; the pressure rate, which depends on
the fine-to-coarse transfer the paper does not give (tests/paper_runs.py),
within 0.15.  Area loss at t = 4 and leakage rate over t in [2, 4] (Tables 3
and 4): 3% and 2% (measured within 2.3% and 0.9%); the relaxed membrane is a
circle of the ellipse's area, radius sqrt(r1 r2) = 1/4, to 0.5%.
"""
import json
import os

import numpy as np
import pytest

import paper_runs as R

pytestmark = pytest.mark.gpu

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_tables.json")))
TOL_RATE = {"u": 0.08, "X": 0.08, "p": 0.15}
_cache = {}


def thin(N, sigma, dt, t):
    key = ("thin", N, sigma)
    if key not in _cache:
        _cache[key] = R.thin_ellipse(N, sigma=sigma, dt=dt, t=t)
    return _cache[key]


def thick(N, mu, dt):
    key = ("thick", N, mu, dt)
    if key not in _cache:
        _cache[key] = R.thick_shell(N, mu=mu, dt=dt)
    return _cache[key]


@pytest.mark.parametrize("run", GOLD["table2_thin_ellipse_divergence"]["runs"], ids=lambda r: f"sigma{r['sigma']}")
def test_table2_divergence_error(run):
    for N, ref in run["E_div"].items():
        r = thin(int(N), run["sigma"], run["dt"], run["t"])
        assert R.l2_cells(r["div"], int(N)) == pytest.approx(ref, rel=0.015), (N, ref)


@pytest.mark.parametrize("run", GOLD["table1_thin_ellipse_rates"]["runs"], ids=lambda r: f"sigma{r['sigma']}")
def test_table1_convergence_rates(run):
    r = {N: thin(N, run["sigma"], run["dt"], run["t"]) for N in (64, 128, 256, 512)}
    got = {"R64": R.rate(r[64], r[128], r[256]), "R128": R.rate(r[128], r[256], r[512])}
    for which in ("R64", "R128"):
        for q, ref in run[which].items():
            assert abs(got[which][q] - ref) < TOL_RATE[q], (which, q, got[which][q], ref)


@pytest.mark.parametrize("run", GOLD["table6_thick_shell_divergence"]["runs"], ids=lambda r: f"dt{r['dt']}")
def test_table6_divergence_error(run):
    for N, ref in run["E_div"].items():
        r = thick(int(N), 0.01, run["dt"])
        assert R.l2_cells(r["div"], int(N)) == pytest.approx(ref, rel=0.015), (N, ref)


@pytest.mark.parametrize("run", GOLD["table5_thick_shell_rates"]["runs"], ids=lambda r: f"mu{r['mu']}")
def test_table5_convergence_rates(run):
    r = {N: thick(N, run["mu"], 0.08 / 512) for N in (128, 256, 512)}
    got = R.rate(r[128], r[256], r[512], fibers=3 * 128 // 8, thick=True)
    for q, ref in run["R128"].items():
        assert abs(got[q] - ref) < TOL_RATE[q], (q, got[q], ref)


@pytest.mark.parametrize("N", [64, 128])
@pytest.mark.parametrize("k", [0, 1])
def test_tables3_4_area_loss_and_leakage_rate(N, k):
    t3 = GOLD["table3_thin_ellipse_area_loss"]["runs"][k]
    t4 = GOLD["table4_thin_ellipse_leakage_rate"]["runs"][k]
    assert t3["dt"] == t4["dt"]
    ts, loss, X = R.thin_ellipse_area_history(N, t3["dt"])
    assert loss[-1] == pytest.approx(t3["loss"][str(N)], rel=0.03)
    rate = np.polyfit(ts, loss, 1)[0]
    assert rate == pytest.approx(t4["rate"][str(N)], rel=0.02)
    # equilibrium: a circle of radius sqrt(r1 r2) = 1/4 about the centroid
    r = np.linalg.norm(X - X.mean(0), axis=1)
    assert abs(r.mean() - 0.25) < 0.005 * 0.25
    assert (r.max() - r.min()) < 0.005 * 0.25
