"""Intraband plasma frequency (Sec. 2.3, Eq. plasma) on the GPU through the C ABI against the oracle:
free-electron bands of a simple-cubic cell (where both tend to 4 pi n) and the empirical-
pseudopotential bands of the small workload with the Fermi energy inside a band, with and without
cRPA weights T.  FP64: 1e-12 of the largest component."""
import numpy as np
import pytest

from conftest import workload

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2001_02351_gb300 as rp  # noqa: E402
from oracle import plasma as OPL  # noqa: E402


def _ctx(b, nb, fft, T=None):
    ctx = rp.Context(b.cell.lat, b.kmesh, fft, b.ecut_psi, b.ecut_psi * 0.5)
    ctx.load_bands(1, b.npw, b.miller, b.coef[:, :nb], b.energy[:, :nb], None if T is None else T[:, :nb])
    return ctx


def test_plasma_free_electrons():
    import sys
    import os
    sys.path.insert(0, os.path.dirname(__file__))
    from test_oracle_plasma import _free_bands
    kf = 1.1
    b, nb = _free_bands(8, 4.0, ecut=0.5 * (kf + 2.2) ** 2)
    ef = 0.5 * kf * kf
    got = _ctx(b, nb, (16, 16, 16)).rp_plasma(ef)
    ref = OPL.plasma_tensor(b, ef, nb)
    assert np.abs(got - ref).max() <= 1e-12 * np.abs(ref).max()
    assert abs(got[0, 0] / (4 * np.pi * kf ** 3 / (3 * np.pi ** 2)) - 1) < 0.1


def test_plasma_epm_metal():
    wl = workload("small")
    b = wl.bands
    nb = b.energy.shape[1]
    ef = float(np.median(b.energy[:, 5]))                    # inside the sixth band
    rng = np.random.default_rng(9)
    T = rng.uniform(0, 1, size=b.energy.shape)
    for t in (None, T):
        got = _ctx(b, nb, wl.fft, t).rp_plasma(ef)
        ref = OPL.plasma_tensor(b, ef, nb, T=t)
        assert np.abs(got - ref).max() <= 1e-12 * np.abs(ref).max()
        assert np.abs(ref).max() > 0
