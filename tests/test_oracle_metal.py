"""Pins of the metallic generalized tetrahedron method (oracle, Fermi-surface clipping).

Each tetrahedron contributes over its part where band o (at k) lies below the Fermi energy and
band a (at k + q) above it, both interpolated linearly; the part is cut into sub-tetrahedra on
which the unclipped vertex formula is applied.  Pinned here by:
- geometry: the pieces of {e < 0} and {e > 0} partition the tetrahedron (volumes and barycentric
  first moments add up to the whole) for every count of negative vertices;
- the clipped region's barycentric moments (1/V) int lambda_j over {E_o < E_F < E_a} against a
  Monte Carlo estimate from uniformly sampled points (independent of the clipping);
- the insulator limit: with the Fermi energy in a gap every piece is the whole tetrahedron and the
  weights equal the unclipped ones;
- nothing occupied (Fermi energy below the bands) gives zero;
- a metal (Fermi energy inside two bands of the tiny set, a band window with its partly filled
  bands in both ranges): chi0 on the imaginary axis is Hermitian and negative semidefinite (every
  clipped piece has D = E_a - E_o > 0), and the intraband pairs (a band with itself) contribute;
- the free-electron gas: chi_00(q, i nu) per volume from the clipped tetrahedra approaches the
  Lindhard function as the mesh grows (4^3 -> 6^3: relative error 0.13 -> 0.05 at nu = 0.5 Ha).
"""
from dataclasses import replace

import numpy as np
import pytest

from conftest import workload
from oracle import chi0 as C, lattice, pair_density as pd, tetra as T
from synth import metal_view

FERMI_TINY = -0.21      # inside bands 6 and 7 of the tiny set (widths -0.267..-0.191, -0.221..-0.191)


def _vol(pieces):
    return sum(abs(np.linalg.det(B)) for B in pieces)


def _moment(pieces):
    """(1/V) int lambda over the pieces: each piece's volume times the mean of its rows."""
    return sum(abs(np.linalg.det(B)) * B.mean(axis=0) for B in pieces)


@pytest.mark.parametrize("e", [[-1.0, 0.5, 0.7, 0.2], [-1.0, -0.3, 0.7, 0.2], [-1.0, -0.3, -0.7, 0.2],
                               [-1.0, -0.3, -0.7, -0.2], [1.0, 0.3, 0.7, 0.2], [-0.4, 0.4, -0.4, 0.4]])
def test_clip_partitions_the_tetrahedron(e):
    e = np.asarray(e)
    below, above = T.clip_negative(e), T.clip_negative(-e)
    assert len(below) == {0: 0, 1: 1, 2: 3, 3: 3, 4: 1}[int(np.sum(e < 0))]
    assert abs(_vol(below) + _vol(above) - 1.0) < 1e-14
    m = (_moment(below) if below else 0) + (_moment(above) if above else 0)
    assert np.allclose(m, 0.25, atol=1e-14)
    # every piece lies on its side: the function at each piece vertex has the right sign
    for B in below:
        assert np.all(B @ e <= 1e-15)
    for B in above:
        assert np.all(B @ e >= -1e-15)


def test_four_occupancy_regions_partition():
    """{E_o < F < E_a}, {E_o < F, E_a < F}, {E_o > F, E_a > F}, {E_o > F > E_a}: the four
    regions' pieces (through the two clips with the signs flipped) make up the tetrahedron."""
    rng = np.random.default_rng(11)
    for _ in range(20):
        eo, ea, F = rng.standard_normal(4), rng.standard_normal(4), 0.1 * rng.standard_normal()
        tot = 0.0
        for so in (1, -1):
            for sa in (1, -1):
                for B in T.clip_negative(so * (eo - F)):
                    tot += _vol([C_ @ B for C_ in T.clip_negative(B @ (sa * (F - ea)))])
        assert abs(tot - 1.0) < 1e-13


@pytest.mark.parametrize("seed", [1, 2, 3, 4])
def test_clipped_moments_against_monte_carlo(seed):
    rng = np.random.default_rng(seed)
    while True:
        # both bands cross the Fermi energy inside the tetrahedron, and their region is not empty
        eo, ea = rng.uniform(-1, 1, 4), rng.uniform(-1, 1, 4)
        pieces = T.occupied_pieces(eo, ea, 0.0)
        if 0 < np.sum(eo < 0) < 4 and 0 < np.sum(ea > 0) < 4 and _vol(pieces) > 0.02:
            break
    got = T.clipped_vertex_weights(ea - eo, pieces, lambda ds: np.full(ds.shape, 0.25))
    lam = rng.dirichlet(np.ones(4), size=2_000_000)             # uniform points of the tetrahedron
    inside = (lam @ eo < 0.0) & (lam @ ea > 0.0)
    ref = (lam * inside[:, None]).mean(axis=0)
    assert np.all(np.abs(got - ref) < 1.5e-3), (got, ref)
    assert abs(_vol(pieces) - inside.mean()) < 1.5e-3


def test_insulator_limit_equals_unclipped():
    # the lowest 6 bands of the tiny set are separated from the rest by a gap on the whole mesh
    wl = replace(workload("tiny"), nocc=6, nemp=6)
    b = wl.bands
    q = wl.q[0]
    kp, _ = lattice.umklapp(b.kmesh, q)
    e_occ, e_emp = b.energy[:, :wl.nocc], b.energy[kp, wl.nocc:wl.nocc + wl.nemp]
    gap_mid = 0.5 * (e_occ.max() + e_emp.min())
    assert e_occ.max() < gap_mid < e_emp.min()
    tets = T.tetrahedra(b.kmesh, b.cell.recip)
    z1, z2 = T.poles(wl.freq, wl.axis, wl.delta, wl.ordering)
    ks = [0, 21]
    ref = T.vertex_weights(e_occ, e_emp, tets, z1, z2, wl.delta_a, wl.delta_r, k_list=ks)
    got = T.metal_vertex_weights(e_occ, e_emp, tets, z1, z2, wl.delta_a, wl.delta_r, gap_mid, k_list=ks)
    assert np.abs(got - ref).max() < 1e-12 * np.abs(ref).max()
    none = T.metal_vertex_weights(e_occ, e_emp, tets, z1, z2, wl.delta_a, wl.delta_r, e_occ.min() - 1.0,
                                  k_list=ks)
    assert np.all(none == 0)


@pytest.fixture(scope="module")
def tiny_metal():
    # a band window around the Fermi energy: bands 4-7 may be occupied, 6-10 may be empty
    wl = workload("tiny")
    view, nocc, nemp = metal_view(wl.bands, FERMI_TINY, window=(4, 11))
    return replace(wl, bands=view, nocc=nocc, nemp=nemp)


def test_metal_view_of_the_tiny_set(tiny_metal):
    full, nocc, nemp = metal_view(workload("tiny").bands, FERMI_TINY)
    assert (nocc, nemp) == (8, 10) and full.meta["metal_rows"][8:10] == [6, 7]
    assert (tiny_metal.nocc, tiny_metal.nemp) == (4, 5)
    assert tiny_metal.bands.meta["metal_rows"] == [4, 5, 6, 7, 6, 7, 8, 9, 10]


def test_metal_chi0_hermitian_negative_semidefinite(tiny_metal):
    wl = tiny_metal
    q = wl.q[0]
    G = lattice.eps_sphere(wl.cell.lat, q, wl.ecut_eps[0])
    M = pd.pair_density(wl.bands, wl.nocc, wl.nemp, q, G, fft=wl.fft)
    w = C.pair_weights(wl, q, fermi=FERMI_TINY)
    chi = C.chi0(M, w)
    assert np.abs(chi - np.conj(np.transpose(chi, (0, 2, 1)))).max() < 1e-14 * np.abs(chi).max()
    for c in chi:
        ev = np.linalg.eigvalsh(c)
        assert ev.max() < 1e-12 * np.abs(ev).max() and ev.min() < 0
    # the intraband pairs (bands 6 and 7 with themselves: a = 0, o = 2 and a = 1, o = 3) carry weight
    nk = wl.bands.kfrac.shape[0]
    wk = w.reshape(len(wl.freq), nk, wl.nemp, wl.nocc)
    assert np.abs(wk[:, :, 0, 2]).max() > 0 and np.abs(wk[:, :, 1, 3]).max() > 0


def test_free_electron_lindhard_metallic_tetrahedron():
    """Plane-wave bands of an empty simple-cubic cell (a = 4 bohr), Fermi wave number 0.8, the lowest
    12 bands of each range, |q| = 2 pi / 8 bohr^-1 (Q / 2 k_F ~ 0.49): chi_00 from the metallic
    tetrahedron weights against the Lindhard function, on 4^3 and 6^3 meshes."""
    from test_oracle_chi0 import _pw_bands, lindhard_imag
    from synth import Workload
    nu = np.array([0.5])
    kf, nwin = 0.8, 12
    errs = []
    for n in (4, 6):
        bands, nb = _pw_bands(4.0, (n, n, n), ecut=0.5 * (kf + 2.6) ** 2)
        rows = np.concatenate([np.arange(nwin), nb + np.arange(nwin)])
        b2 = replace(bands, coef=bands.coef[:, rows], energy=bands.energy[:, rows])
        q = np.array([0.5, 0.0, 0.0])
        M = pd.pair_density(b2, nwin, nwin, q, np.zeros((1, 3), dtype=np.int64), fft=(16, 16, 16))
        wl = Workload(name="free", bands=b2, fft=(16, 16, 16), nocc=nwin, nemp=nwin, q=q[None, :],
                      ecut_eps=np.array([1.0]), axis="imag", freq=nu, delta=0.0)
        chi = C.chi0(M, C.pair_weights(wl, q, kind="tetra", fermi=0.5 * kf * kf))[:, 0, 0] / bands.cell.omega
        Q = np.linalg.norm(q @ bands.cell.recip)
        ref = lindhard_imag(Q, nu[0], kf)
        errs.append(abs(chi[0] - ref) / abs(ref))
    assert errs[1] < 0.08 and errs[1] < 0.5 * errs[0], errs
