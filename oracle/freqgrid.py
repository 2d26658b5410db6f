"""Logarithmic frequency grid (oracle), Eq. grid of Sec. 3.2.

  w_i = dw (s^(i-1) - 1)/(s - 1),            i = 1 .. N_max
  w_i = E_max exp[ln 3 (i - N_max)/(N_W - N_max)],   i = N_max+1 .. N_W
with N_max = (9 N_W)/10 (integer division) and s > 1 fixed by w_{N_max} = E_max.
The text prints the equation for s with a plus sign, which cannot meet its
own boundary conditions; the reading used here is the one that does:
  s^(N_max - 1) - (E_max/dw)(s - 1) = 1.
"""
import numpy as np
from scipy.optimize import brentq


def log_grid(e_max, n_total=70, dw=0.05 / 27.211386245988):
    n_max = (9 * n_total) // 10
    ratio = e_max / dw

    def g(s):
        return (s ** (n_max - 1) - 1.0) / (s - 1.0) - ratio

    s = brentq(g, 1.0 + 1e-12, 10.0, xtol=1e-15, rtol=1e-15, maxiter=500)
    i = np.arange(1, n_total + 1, dtype=np.float64)
    w = np.empty(n_total)
    lo = i <= n_max
    w[lo] = dw * (s ** (i[lo] - 1.0) - 1.0) / (s - 1.0)
    w[~lo] = e_max * np.exp(np.log(3.0) * (i[~lo] - n_max) / (n_total - n_max))
    return w, s
