"""Band lists of a metal for the pair layout (input preparation only, no arithmetic of the method).

The pair layout takes the first n_occ entries of a band list as the bands that may be occupied (at
k) and the next n_emp as those that may be empty (at k + q).  In a metal a partly filled band is
both, so its entry appears in each range: `metal_view` returns the list with the bands that reach
below the Fermi energy first and the bands that reach above it after them (the partly filled ones
twice), with n_occ and n_emp of that view.
"""
from dataclasses import replace

import numpy as np


def metal_bands(bands, fermi):
    """(o_end, a_begin): bands 0 .. o_end-1 have a state below `fermi` somewhere on the mesh,
    bands a_begin .. nband-1 a state above it."""
    e = bands.energy
    below = np.nonzero(e.min(axis=0) < fermi)[0]
    above = np.nonzero(e.max(axis=0) > fermi)[0]
    if len(below) == 0 or len(above) == 0:
        raise ValueError("the Fermi energy lies outside the bands")
    return int(below.max()) + 1, int(above.min())


def metal_view(bands, fermi, window=None):
    """(bands of the view, n_occ, n_emp): rows 0 .. o_end-1, then a_begin .. nband-1; with
    window = (lo, hi) only the bands lo .. hi-1 of each range (a band window around the Fermi
    energy)."""
    o_end, a_begin = metal_bands(bands, fermi)
    lo, hi = (0, bands.energy.shape[1]) if window is None else window
    rows = np.concatenate([np.arange(lo, o_end), np.arange(a_begin, hi)])
    view = replace(bands, coef=np.ascontiguousarray(bands.coef[:, rows]),
                   energy=np.ascontiguousarray(bands.energy[:, rows]),
                   meta=dict(bands.meta, metal_rows=rows.tolist(), fermi=float(fermi)))
    return view, o_end - lo, len(rows) - (o_end - lo)
