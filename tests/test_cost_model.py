"""The cost sums of App. C against their stated asymptotics, and the fits
and interpolation the measured bond-dimension study uses."""
import numpy as np

from paper_2606_02930_gb300 import costmodel


def test_fixed_chi_gives_tau_max_over_log():
    # chi fixed: C_U = chi^3 2^m and C_L = chi^3 m exactly
    for m in (4, 10, 16):
        cu, cl = costmodel.appc_costs(m, lambda t: np.full_like(t, 7.0))
        assert cu == 343.0 * 2 ** m and cl == 343.0 * m


def test_log_growth_gives_stirling_and_quartic_sums():
    # chi = log2 tau: C_L = sum k^3 = (m (m + 1) / 2)^2 exactly, and C_U / (m^3 2^m) -> 1
    ratios = []
    for m in (8, 12, 16, 20):
        cu, cl = costmodel.appc_costs(m, np.log2)
        assert abs(cl - (m * (m + 1) / 2) ** 2) < 1e-6 * cl
        ratios.append(cu / (m ** 3 * 2 ** m))
    assert all(0.5 < r < 1.0 for r in ratios)
    assert all(b > a for a, b in zip(ratios, ratios[1:]))     # approaching 1 from below


def test_power_growth_gives_tau_max_reduction():
    # chi = tau^alpha: C_U ~ tau_max^(3 alpha + 1) / (3 alpha + 1) and
    # C_L ~ tau_max^(3 alpha) / (1 - 2^(-3 alpha)), so C_U / C_L / tau_max
    # tends to (1 - 2^(-3 alpha)) / (3 alpha + 1)
    alpha = 0.3
    want = (1 - 2 ** (-3 * alpha)) / (3 * alpha + 1)
    got = []
    for m in (10, 14, 18):
        cu, cl = costmodel.appc_costs(m, lambda t: t ** alpha)
        got.append(cu / cl / 2 ** m)
    assert abs(got[-1] - want) < 0.01 * want
    assert abs(got[-1] - want) < abs(got[0] - want)


def test_fits_recover_their_laws():
    tau = np.geomspace(0.1, 300, 40)
    a, p = costmodel.fit_power_law(tau, 2.5 * tau ** 1.7)
    assert abs(a - 2.5) < 1e-10 and abs(p - 1.7) < 1e-12
    g = costmodel.fit_growth(tau, 4.0 + 3.0 * np.log(tau) + 20.0)
    assert abs(g["log"]["b"] - 3.0) < 1e-10 and g["log"]["rms_rel"] < 1e-12
    assert g["power"]["rms_rel"] > 1e-3
    g = costmodel.fit_growth(tau, 5.0 * tau ** 0.4)
    assert abs(g["power"]["alpha"] - 0.4) < 1e-12 and g["power"]["rms_rel"] < 1e-12


def test_uniform_cost_on_a_measured_evolution():
    nodes = np.array([0.0, 0.5, 1.0, 2.0, 4.0])
    chis = [2, 4, 8, 16]
    # tau in (0, 0.5] -> 2, (0.5, 1] -> 4, (1, 2] -> 8, (2, 4] -> 16, beyond -> 16
    assert costmodel.chi_at([0.25, 0.5, 0.75, 1.5, 3.0, 9.0], nodes, chis).tolist() == \
        [2, 2, 4, 8, 16, 16]
    # dtau = 0.5 up to 4: chis 2, 4, 8, 8, 16, 16, 16, 16 at cost chi
    assert costmodel.uniform_cost(4.0, 0.5, nodes, chis, lambda c: c) == 86.0
