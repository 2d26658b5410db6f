"""q -> 0 limit on the GPU through the C ABI against the oracle (Sec. 2.3, Eq. eps00, Eq. momentum,
Eqs. epsilonM, eels, optical-conductivity, reflectance): the extended chi0 with the head and wings
from the k.p limit (FP64 and BF16x3), the extended Dyson step, and the optical quantities from
its head.  Real axis with broadening (small workload) and imaginary axis (tiny)."""
import numpy as np
import pytest

from conftest import workload

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2001_02351_gb300 as rp  # noqa: E402
from oracle import chi0 as OC, dyson as OD, head as OH, lattice as OL, pair_density as OP  # noqa: E402

QHAT = np.array([0.3, -0.5, 0.8])


def _rel_fro(a, b):
    a = np.asarray(a).reshape(a.shape[0], -1)
    b = np.asarray(b).reshape(b.shape[0], -1)
    return np.linalg.norm(a - b, axis=1) / np.linalg.norm(b, axis=1)


# band counts whose occupied set ends in a gap at every mesh point (the k.p head divides by the
# transition energy at q = 0)
INSULATING = {"tiny": dict(nocc=6, nemp=6), "small": dict(nocc=3, nemp=8)}


@pytest.mark.parametrize("name", ["tiny", "small"])
def test_head_and_wings_against_oracle(name):
    wl = workload(name, **INSULATING[name])
    E = wl.bands.energy
    assert (E[:, wl.nocc] - E[:, wl.nocc - 1]).min() > 1e-3
    q = np.zeros(3)
    G = OL.eps_sphere(wl.cell.lat, q, wl.ecut_eps[0])
    M = OP.pair_density(wl.bands, wl.nocc, wl.nemp, q, G, fft=wl.fft)
    w = OC.pair_weights(wl, q)
    Mx = OH.extended_rows(OH.head_row(wl, QHAT), M)
    chi_ref = OC.chi0(Mx, w)
    W_ref = OD.screened(chi_ref, OH.coulomb_sqrt_ext(wl.cell.lat, G))
    ctx = rp.context_for(wl)
    axis = rp.RP_AXIS_IMAG if wl.axis == "imag" else rp.RP_AXIS_REAL
    chi = ctx.rp_build_chi0_q0(2.5 * QHAT, axis, rp.RP_TIME_ORDERED, wl.freq, wl.delta, rp.RP_FP64_NATIVE)
    assert chi.shape == (len(wl.freq), len(G) + 1, len(G) + 1)
    assert np.all(_rel_fro(chi, chi_ref) < 1e-11)
    # the head and the wings themselves (a small part of the Frobenius norm)
    assert np.abs(chi[:, 0, 0] - chi_ref[:, 0, 0]).max() <= 1e-11 * np.abs(chi_ref[:, 0, 0]).max()
    assert np.abs(chi[:, 1:, 0] - chi_ref[:, 1:, 0]).max() <= 1e-11 * np.abs(chi_ref[:, 1:, 0]).max()
    W = ctx.rp_solve_w_q0(chi)
    assert np.all(_rel_fro(W, W_ref) < 1e-11)
    assert np.abs(W[:, 0, 0] - W_ref[:, 0, 0]).max() <= 1e-11 * np.abs(W_ref[:, 0, 0]).max()
    opt = ctx.rp_optics(wl.freq, W[:, 0, 0])
    em, loss, sig, refl = OH.macroscopic(wl.freq, W_ref[:, 0, 0] * wl.cell.omega / (4 * np.pi))
    ref = np.stack([em.real, em.imag, loss, sig, refl], axis=1)
    assert np.abs(opt - ref).max() <= 1e-10 * np.abs(ref).max()
    assert np.all(opt[:, 0] > 1.0) if wl.axis == "imag" else True   # eps_M(i nu) > 1 for an insulator
    # the split tier on the same extended rows
    chi = ctx.rp_build_chi0_q0(QHAT, axis, rp.RP_TIME_ORDERED, wl.freq, wl.delta, rp.RP_BF16X3)
    assert np.all(_rel_fro(chi, chi_ref) < 1e-4)
    with pytest.raises(rp.RPError) as e:
        ctx.rp_build_chi0_q0(np.zeros(3), axis, rp.RP_TIME_ORDERED, wl.freq, wl.delta, rp.RP_FP64_NATIVE)
    assert e.value.code == rp.RP_ERR_ARG


def test_head_refuses_a_band_set_without_gap():
    wl = workload("tiny")                       # 8 + 8 bands: bands 8 and 9 touch at some k
    assert (wl.bands.energy[:, 8] - wl.bands.energy[:, 7]).min() < 1e-9
    ctx = rp.context_for(wl)
    with pytest.raises(rp.RPError) as e:
        ctx.rp_build_chi0_q0(QHAT, rp.RP_AXIS_IMAG, rp.RP_TIME_ORDERED, wl.freq, wl.delta, rp.RP_FP64_NATIVE)
    assert e.value.code == rp.RP_ERR_ARG
