"""Metallic tetrahedron weights on the GPU (rp_set_fermi, Fermi-surface clipping) against the
oracle: the tiny set with the Fermi energy inside bands 6 and 7, a band window around it (bands
5-7 may be occupied, 6-9 may be empty; the partly filled bands 6 and 7 in both ranges, so their
intraband pairs are included).  Weights (FP64) and chi0 in the FP64 and BF16x3 tiers; turning the
clipping off again restores the band-index weights."""
from dataclasses import replace

import numpy as np
import pytest

from conftest import workload

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

import paper_2001_02351_gb300 as rp  # noqa: E402
from oracle import chi0 as OC, lattice as OL, pair_density as OP  # noqa: E402
from synth import metal_view  # noqa: E402

FERMI = -0.21


def _rel_fro(a, b):
    a = np.asarray(a).reshape(a.shape[0], -1)
    b = np.asarray(b).reshape(b.shape[0], -1)
    return np.linalg.norm(a - b, axis=1) / np.linalg.norm(b, axis=1)


@pytest.fixture(scope="module")
def metal():
    wl = workload("tiny")
    view, nocc, nemp = metal_view(wl.bands, FERMI, window=(5, 10))
    assert (nocc, nemp) == (3, 4)
    return replace(wl, bands=view, nocc=nocc, nemp=nemp)


@pytest.fixture(scope="module")
def metal_ref(metal):
    q = metal.q[0]
    G = OL.eps_sphere(metal.cell.lat, q, metal.ecut_eps[0])
    w = OC.pair_weights(metal, q, fermi=FERMI)
    M = OP.pair_density(metal.bands, metal.nocc, metal.nemp, q, G, fft=metal.fft)
    return w, OC.chi0(M, w)


def test_metal_weights_and_chi0(metal, metal_ref):
    w_ref, chi_ref = metal_ref
    q = metal.q[0]
    ctx = rp.context_for(metal)
    ctx.rp_set_fermi(FERMI)
    ax, od = rp.RP_AXIS_IMAG, rp.RP_TIME_ORDERED
    w = ctx.rp_tetra_weights(q, ax, od, metal.freq, metal.delta)
    nk = metal.bands.kfrac.shape[0]
    assert np.abs(w - w_ref).max() < 1e-11 * np.abs(w_ref).max()
    # the intraband pairs (band 6 with itself: a = 0, o = 1) carry weight
    assert np.abs(w.reshape(len(metal.freq), nk, metal.nemp, metal.nocc)[:, :, 0, 1]).max() > 0
    chi = ctx.rp_build_chi0(q, ax, od, metal.freq, metal.delta, rp.RP_FP64_NATIVE)
    assert np.all(_rel_fro(chi, chi_ref) < 1e-11)
    chi = ctx.rp_build_chi0(q, ax, od, metal.freq, metal.delta, rp.RP_BF16X3)
    assert np.all(_rel_fro(chi, chi_ref) < 1e-4)
    # NaN: band-index occupations again
    ctx.rp_set_fermi()
    w0 = ctx.rp_tetra_weights(q, ax, od, metal.freq, metal.delta)
    w0_ref = OC.pair_weights(metal, q, k_list=[0, 21])
    cols = np.concatenate([np.arange(k * metal.nemp * metal.nocc, (k + 1) * metal.nemp * metal.nocc) for k in (0, 21)])
    assert np.abs(w0[:, cols] - w0_ref).max() < 1e-11 * np.abs(w0_ref).max()
    with pytest.raises(rp.RPError) as e:
        ctx.rp_set_fermi(float("inf"))
    assert e.value.code == rp.RP_ERR_ARG
    ctx.close()
