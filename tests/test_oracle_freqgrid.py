"""Pins for the logarithmic frequency grid (Eq. grid, Sec. 3.2).

The four boundary conditions and the defaults the paper prints are stored in
tests/golden/freq_grid_defaults.json.
"""
import json
import os

import numpy as np

from oracle.freqgrid import log_grid

HARTREE_EV = 27.211386245988


def test_boundary_conditions():
    g = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "freq_grid_defaults.json")))
    dw = g["dw_eV"] / HARTREE_EV
    for e_max in (0.7, 1.9, 4.0):
        w, s = log_grid(e_max, g["N_Omega"], dw)
        nmax = g["N_max"]
        assert s > 1.0
        assert w[0] == g["w1"]
        assert abs(w[1] - dw) < 1e-15
        assert abs(w[nmax - 1] - e_max) < 1e-12 * e_max
        assert abs(w[-1] - g["last_over_Emax"] * e_max) < 1e-12 * e_max
        assert np.all(np.diff(w) > 0)
