"""Cost of imaginary-time grids when the bond dimension grows (App. C).

App. C compares a uniform grid tau_k = k (k = 1 .. 2^m) with the logarithmic
grid tau_k = 2^k (k = 1 .. m) at a per-step cost chi(tau_k)^3:

    C_U = sum_{k=1}^{2^m} chi(k)^3,      C_L = sum_{k=1}^{m} chi(2^k)^3,

and finds C_U / C_L growing like tau_max = 2^m up to logarithmic factors for
a fixed chi, chi = log tau and chi = tau^alpha.  The main text adds the
observation that a step's cost does not depend on its size dtau, which is what
lets a step count stand for the cost.

This module holds those sums and the fits that the measured study (per-step
times t_k and bond dimensions chi_k of an evolution on the paper's panel grid)
feeds: a power law t(chi) = a chi^p for the step cost, the two growth laws for
chi(tau), and the cost that uniform stepping would have had on the same
evolution.  Host-side analysis only; nothing here runs on the device.
"""
import numpy as np


def appc_costs(m, chi_of_tau, power=3.0):
    """(C_U, C_L) of App. C for tau_max = 2^m and the growth law chi_of_tau."""
    k_u = np.arange(1, 2 ** m + 1, dtype=float)
    k_l = 2.0 ** np.arange(1, m + 1)
    return (float(np.sum(chi_of_tau(k_u) ** power)), float(np.sum(chi_of_tau(k_l) ** power)))


def fit_power_law(x, y):
    """Least squares of log y = log a + p log x; returns (a, p)."""
    lx, ly = np.log(np.asarray(x, float)), np.log(np.asarray(y, float))
    p, la = np.polyfit(lx, ly, 1)
    return float(np.exp(la)), float(p)


def fit_growth(tau, chi):
    """Both growth laws of App. C on (tau, chi) samples: chi = a + b ln tau and
    chi = c tau^alpha.  Returns a dict with the parameters and the root mean
    square relative residual of each."""
    tau, chi = np.asarray(tau, float), np.asarray(chi, float)
    b, a = np.polyfit(np.log(tau), chi, 1)
    res_log = np.sqrt(np.mean(((a + b * np.log(tau)) - chi) ** 2 / chi ** 2))
    c, alpha = fit_power_law(tau, chi)
    res_pow = np.sqrt(np.mean((c * tau ** alpha - chi) ** 2 / chi ** 2))
    return {"log": {"a": float(a), "b": float(b), "rms_rel": float(res_log)},
            "power": {"c": float(c), "alpha": float(alpha), "rms_rel": float(res_pow)}}


def chi_at(tau, nodes, chis):
    """Bond dimension at times tau from an evolution on `nodes` (t_0 = 0 <
    t_1 < ...) whose step k (ending at nodes[k]) left chis[k-1]: the value of
    the step whose interval holds tau (the last one beyond nodes[-1])."""
    nodes = np.asarray(nodes, float)
    idx = np.searchsorted(nodes[1:], np.asarray(tau, float), side="left")
    idx = np.minimum(idx, len(chis) - 1)
    return np.asarray(chis)[idx]


def uniform_cost(tau_max, dtau, nodes, chis, t_of_chi):
    """Cost of uniform steps of size dtau up to tau_max on the same evolution:
    sum over j of t(chi(j dtau)), chi from the measured steps and t from the
    fitted step cost (a step's cost taken independent of its size)."""
    n = int(round(tau_max / dtau))
    taus = dtau * np.arange(1, n + 1)
    return float(np.sum(t_of_chi(chi_at(taus, nodes, chis).astype(float))))
