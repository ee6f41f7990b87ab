"""Logarithmic imaginary-time grids.  Test infrastructure only.

* ``panel_grid``: the paper's grid (Method, panel construction): P panels with
  endpoints {0, tau_max / 2^(P-j) for j = 1..P} and n uniform steps on each
  panel.  The first panel is [0, tau_max / 2^(P-1)].
* ``geometric_grid``: a geometric grid a -> b with K steps: t_0 = 0 and
  t_k = a (b/a)^((k-1)/(K-1)) for k = 1..K, so the first step is 0 -> a and
  the last node is b (the reading used for the synthetic workloads).
"""
import numpy as np


def panel_grid(tau_max, P, n):
    ends = [0.0] + [tau_max / 2.0 ** (P - j) for j in range(1, P + 1)]
    nodes = [0.0]
    for p in range(P):
        a, b = ends[p], ends[p + 1]
        for i in range(1, n + 1):
            nodes.append(a + (b - a) * i / n)
    return np.array(nodes)


def geometric_grid(a, b, K):
    if K == 1:
        return np.array([0.0, float(b)])
    k = np.arange(1, K + 1)
    return np.concatenate([[0.0], a * (b / a) ** ((k - 1) / (K - 1))])


def steps(nodes):
    nodes = np.asarray(nodes, float)
    return nodes[1:] - nodes[:-1]
