"""GPU path vs the FP64 oracle, element by element, through the C ABI.

Tolerances (FP64 path): pair densities and weights agree to rounding of a few hundred
operations (1e-12 relative to the largest element); chi0 and W per frequency to a
relative Frobenius error of 1e-11, the bound the summation of ~1e4..1e6 FP64 terms and
the Gauss-Jordan inverse of a well-conditioned NG x NG matrix leave.
"""
import numpy as np
import pytest

from conftest import workload

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

import paper_2001_02351_gb300 as rp  # noqa: E402
from oracle import chi0 as OC, dyson as OD, lattice as OL, pair_density as OP  # noqa: E402


def _ctx(wl):
    return rp.context_for(wl)


def _axis(wl):
    return rp.RP_AXIS_IMAG if wl.axis == "imag" else rp.RP_AXIS_REAL


def _ordering(wl):
    return rp.RP_TIME_ORDERED if wl.ordering == "time" else rp.RP_RETARDED


def _rel_fro(a, b):
    a = np.asarray(a).reshape(a.shape[0], -1)
    b = np.asarray(b).reshape(b.shape[0], -1)
    return np.linalg.norm(a - b, axis=1) / np.linalg.norm(b, axis=1)


@pytest.fixture(scope="module")
def tiny():
    return workload("tiny")


def test_sphere_matches_oracle(tiny):
    ctx = _ctx(tiny)
    q = tiny.q[0]
    g, t = ctx.rp_sphere_size(q)
    assert np.array_equal(g, OL.eps_sphere(tiny.cell.lat, q, tiny.ecut_eps[0]))
    assert np.array_equal(t, OL.tail_sphere(tiny.cell.lat, q, tiny.ecut_eps[0], tiny.bands.ecut_psi))


@pytest.mark.parametrize("name,krange", [("micro", (0, 8)), ("tiny", (5, 13)), ("small", (0, 27))])
def test_pair_density(name, krange):
    wl = workload(name)
    ctx = _ctx(wl)
    q = wl.q[0]
    G = OL.eps_sphere(wl.cell.lat, q, wl.ecut_eps[0])
    ref = OP.pair_density(wl.bands, wl.nocc, wl.nemp, q, G, fft=wl.fft, k_list=range(*krange))
    got = ctx.rp_pair_density(q, *krange)
    assert got.shape == ref.shape
    assert np.abs(got - ref).max() <= 1e-12 * np.abs(ref).max()


@pytest.mark.parametrize("name,fft", [("tiny", (32, 32, 32)), ("small", (24, 24, 24))])
def test_pair_density_on_a_smaller_exact_grid(name, fft):
    """A requested grid larger than the product and the sphere need: the library transforms on
    a smaller grid on which nothing folds onto the sphere, so M is the oracle's convolution over
    the requested grid (both are the exact convolution of Eq. ism)."""
    from dataclasses import replace
    wl = replace(workload(name), fft=fft)
    ctx = _ctx(wl)
    q = wl.q[0]
    G = OL.eps_sphere(wl.cell.lat, q, wl.ecut_eps[0])
    ref = OP.pair_density(wl.bands, wl.nocc, wl.nemp, q, G, fft=wl.fft, k_list=range(0, 5))
    got = ctx.rp_pair_density(q, 0, 5)
    assert np.abs(got - ref).max() <= 1e-12 * np.abs(ref).max()
    # the split-precision path (FP32 transforms) on the same grid choice
    M = OP.pair_density(wl.bands, wl.nocc, wl.nemp, q, G, fft=wl.fft)
    chi_ref = OC.chi0(M, OC.pair_weights(wl, q))
    chi = ctx.rp_build_chi0(q, _axis(wl), _ordering(wl), wl.freq, wl.delta, rp.RP_BF16X3)
    assert np.all(_rel_fro(chi, chi_ref) < BF16X3_TOL)


# wide epsilon spheres (E_cut^eps just below E_cut^psi): on the 24-point grid the sphere reaches 6
# (window of half-width 6), on the 32-point grid it reaches 8 (half-width 8, 289 points, taken in
# passes of 256 by the x read-out) and 10 (half-width 11, 529 points)
WIDE = {
    "w24": ("small", dict(npw=700, ng=600, fft=(32, 32, 32)), 6),
    "w32": ("micro", dict(kmesh=(2, 2, 2), npw=1600, ng=1400, fft=(48, 48, 48)), 8),
    "w32b": ("micro", dict(kmesh=(2, 2, 2), npw=3000, ng=2600, fft=(48, 48, 48)), 10),
}


@pytest.mark.parametrize("case", sorted(WIDE))
def test_wide_sphere_window(case):
    """Pair densities and the split-tier chi0 on wide epsilon spheres: the FP32 pair kernels take
    the windows of half-width 6 (24-point grid), 8 and 11 (32-point grid).  chi0 of the split tier
    against the oracle, and the FP64 pair densities (residue masks) of two k points."""
    from dataclasses import replace
    base, kw, reach = WIDE[case]
    wl = workload(base, **kw)
    wl = replace(wl, freq=np.asarray(wl.freq)[:2])
    assert wl.ecut_eps[0] <= wl.bands.ecut_psi
    ctx = _ctx(wl)
    q = wl.q[0]
    G = OL.eps_sphere(wl.cell.lat, q, wl.ecut_eps[0])
    assert np.abs(G).max() == reach
    M = OP.pair_density(wl.bands, wl.nocc, wl.nemp, q, G, fft=wl.fft)
    npk = wl.nocc * wl.nemp
    got = ctx.rp_pair_density(q, 0, 2)
    assert np.abs(got - M[:, :2 * npk]).max() <= 1e-12 * np.abs(M).max()
    chi_ref = OC.chi0(M, OC.pair_weights(wl, q))
    chi = ctx.rp_build_chi0(q, _axis(wl), _ordering(wl), wl.freq, wl.delta, rp.RP_BF16X3)
    assert np.all(_rel_fro(chi, chi_ref) < BF16X3_TOL)


@pytest.mark.parametrize("name", ["micro", "small"])
def test_tetra_weights(name):
    wl = workload(name)
    ctx = _ctx(wl)
    q = wl.q[0]
    ref = OC.pair_weights(wl, q)
    got = ctx.rp_tetra_weights(q, _axis(wl), _ordering(wl), wl.freq, wl.delta, wl.delta_a, wl.delta_r)
    scale = np.abs(ref).max(axis=1, keepdims=True)
    assert np.all(np.abs(got - ref) <= 1e-11 * scale)


def test_tetra_weights_tiny_retarded_crpa():
    from dataclasses import replace
    wl = workload("tiny", crpa=True)
    wl = replace(wl, axis="real", ordering="retarded", delta=0.01, freq=np.array([-0.3, 0.0, 0.2, 0.6]))
    ctx = _ctx(wl)
    q = wl.q[0]
    ref = OC.pair_weights(wl, q, k_list=[0, 7, 21, 63])
    got = ctx.rp_tetra_weights(q, rp.RP_AXIS_REAL, rp.RP_RETARDED, wl.freq, wl.delta)
    cols = np.concatenate([np.arange(k * wl.nemp * wl.nocc, (k + 1) * wl.nemp * wl.nocc) for k in [0, 7, 21, 63]])
    scale = np.abs(ref).max(axis=1, keepdims=True)
    assert np.all(np.abs(got[:, cols] - ref) <= 1e-11 * scale)


@pytest.mark.parametrize("ng,K,nf", [(77, 1000, 3), (128, 64, 1), (5, 37, 2)])
def test_contract_fp64(ng, K, nf):
    rng = np.random.default_rng(ng * 1000 + K)
    M = rng.standard_normal((ng, K)) + 1j * rng.standard_normal((ng, K))
    w = rng.standard_normal((nf, K)) + 1j * rng.standard_normal((nf, K))
    ctx = _ctx(workload("micro"))
    got = ctx.rp_contract_chi0(M, w)
    ref = OC.chi0(M, w)
    assert np.all(_rel_fro(got, ref) < 1e-13)
    # device pointers give the same result
    Md = torch.from_numpy(M).cuda()
    wd = torch.from_numpy(w).cuda()
    gd = ctx.rp_contract_chi0(Md, wd)
    torch.cuda.synchronize()
    assert np.array_equal(gd.cpu().numpy(), got)


@pytest.fixture(scope="module")
def tiny_ref(tiny):
    q = tiny.q[0]
    G = OL.eps_sphere(tiny.cell.lat, q, tiny.ecut_eps[0])
    M = OP.pair_density(tiny.bands, tiny.nocc, tiny.nemp, q, G, fft=tiny.fft)
    w = OC.pair_weights(tiny, q)
    chi = OC.chi0(M, w)
    vs = OD.coulomb_sqrt(tiny.cell.lat, q, G)
    return chi, OD.screened(chi, vs)


def test_build_chi0_and_w_tiny(tiny, tiny_ref):
    chi_ref, W_ref = tiny_ref
    ctx = _ctx(tiny)
    q = tiny.q[0]
    chi = ctx.rp_build_chi0(q, _axis(tiny), _ordering(tiny), tiny.freq, tiny.delta, rp.RP_FP64_NATIVE)
    assert np.all(_rel_fro(chi, chi_ref) < 1e-11)
    W, tail = ctx.rp_solve_w(q, chi)
    assert np.all(_rel_fro(W, W_ref) < 1e-11)
    T = OL.tail_sphere(tiny.cell.lat, q, tiny.ecut_eps[0], tiny.bands.ecut_psi)
    assert np.allclose(tail, OD.tail(tiny.cell.lat, q, T), rtol=1e-14, atol=0)
    # the same through device pointers on torch's stream
    chi_d = torch.empty((len(tiny.freq),) + chi.shape[1:], dtype=torch.complex128, device="cuda")
    ctx.rp_build_chi0(q, _axis(tiny), _ordering(tiny), tiny.freq, tiny.delta, rp.RP_FP64_NATIVE, out=chi_d)
    W_d, _ = ctx.rp_solve_w(q, chi_d)
    torch.cuda.synchronize()
    assert np.all(_rel_fro(chi_d.cpu().numpy(), chi_ref) < 1e-11)
    assert np.all(_rel_fro(W_d.cpu().numpy(), W_ref) < 1e-11)


def test_retarded_symmetry_on_gpu():
    wl = workload("micro")
    ctx = _ctx(wl)
    q = wl.q[0]
    freq = np.array([0.1, 0.3, -0.1, -0.3])
    chi = ctx.rp_build_chi0(q, rp.RP_AXIS_REAL, rp.RP_RETARDED, freq, 0.02, rp.RP_FP64_NATIVE)
    assert np.abs(chi[2:] - np.conj(chi[:2])).max() < 1e-13 * np.abs(chi).max()


def test_errors_are_reported():
    wl = workload("micro")
    b = wl.bands
    ctx = rp.Context(b.cell.lat, b.kmesh, wl.fft, b.ecut_psi, float(wl.ecut_eps[0]))
    with pytest.raises(rp.RPError) as e:
        ctx.nk, ctx.nemp, ctx.nocc = 8, 4, 4
        ctx.rp_tetra_weights(wl.q[0], rp.RP_AXIS_IMAG, rp.RP_TIME_ORDERED, wl.freq, 0.0)
    assert e.value.code == rp.RP_ERR_STATE
    # more plane waves than grid points (at least 110 on 4^3): two of them share a grid point, and
    # the load is refused
    ws = workload("small")
    bs, nbs = ws.bands, ws.nocc + ws.nemp
    assert np.min(bs.npw) > 64
    narrow = rp.Context(bs.cell.lat, bs.kmesh, (4, 4, 4), bs.ecut_psi, float(ws.ecut_eps[0]))
    with pytest.raises(rp.RPError) as e:
        narrow.load_bands(ws.nocc, bs.npw, bs.miller, bs.coef[:, :nbs], bs.energy[:, :nbs])
    assert e.value.code == rp.RP_ERR_ARG and "does not fit" in str(e.value)
    ctx = _ctx(wl)
    with pytest.raises(rp.RPError) as e:
        ctx.rp_sphere_size([0.3, 0.0, 0.0])           # not a mesh vector
    assert e.value.code == rp.RP_ERR_ARG
    with pytest.raises(rp.RPError) as e:              # pole on the real axis
        ctx.rp_tetra_weights(wl.q[0], rp.RP_AXIS_REAL, rp.RP_TIME_ORDERED, wl.freq, 0.0)
    assert e.value.code == rp.RP_ERR_ARG
    # a non-finite chi0 makes the pivot search fail: reported, not faulted
    q = wl.q[0]
    G = OL.eps_sphere(wl.cell.lat, q, wl.ecut_eps[0])
    vs = OD.coulomb_sqrt(wl.cell.lat, q, G)
    chi = np.zeros((1, len(G), len(G)), dtype=np.complex128)
    chi[0, :, 0] = np.nan
    with pytest.raises(rp.RPError) as e:
        ctx.rp_solve_w(q, chi)
    assert e.value.code == rp.RP_ERR_NUMERIC
    # the context stays usable afterwards
    W, _ = ctx.rp_solve_w(q, np.zeros((1, len(G), len(G)), dtype=np.complex128))
    assert np.allclose(W[0], np.diag(vs * vs), rtol=1e-14, atol=0)


def test_bad_pivot_in_one_of_several_frequencies_cooperative():
    """The cooperative Dyson kernel runs all frequencies in one grid with shared barriers: one
    frequency with a non-finite chi0 is reported as RP_ERR_NUMERIC (through rp_check_numeric after
    an asynchronous call), while the other frequency's W is still exact (chi0 = 0 gives W = v).
    NG is about 150, so the cooperative form (several CTAs per frequency) is the one that runs."""
    from synth.configs import _mid_gap_cutoff
    wl = workload("tiny")
    b = wl.bands
    q = wl.q[0]
    cut = _mid_gap_cutoff(wl.cell.recip, q, 150, exclude_zero=True)
    assert cut < b.ecut_psi
    ctx = rp.Context(b.cell.lat, b.kmesh, wl.fft, b.ecut_psi, cut)
    nb = wl.nocc + wl.nemp
    ctx.load_bands(wl.nocc, b.npw, b.miller, b.coef[:, :nb], b.energy[:, :nb])
    G = OL.eps_sphere(wl.cell.lat, q, cut)
    assert len(G) >= 128
    vs = OD.coulomb_sqrt(wl.cell.lat, q, G)
    chi = torch.zeros((3, len(G), len(G)), dtype=torch.complex128, device="cuda")
    chi[1, :, 0] = float("nan")
    W, _ = ctx.rp_solve_w(q, chi)
    with pytest.raises(rp.RPError) as e:
        ctx.rp_check_numeric()
    assert e.value.code == rp.RP_ERR_NUMERIC
    Wh = W.cpu().numpy()
    for f in (0, 2):
        assert np.allclose(Wh[f], np.diag(vs * vs), rtol=1e-14, atol=0)
    # the flag was cleared: the next solve is clean
    W, _ = ctx.rp_solve_w(q, torch.zeros_like(chi))
    ctx.rp_check_numeric()
    assert np.allclose(W.cpu().numpy()[1], np.diag(vs * vs), rtol=1e-14, atol=0)


def test_dyson_hermitian_sweep():
    """rp_set_dyson_hermitian: the lower-triangle sweep without pivoting (eps Hermitian positive
    definite on the imaginary axis) against the oracle and the pivoted solve, on host buffers, on
    device buffers and in a packed batched launch over three q; a frequency whose eps is not positive
    definite is reported as RP_ERR_NUMERIC while the others stay exact."""
    from synth.configs import _mid_gap_cutoff
    wl = workload("tiny")
    b = wl.bands
    q = wl.q[0]
    cut = _mid_gap_cutoff(wl.cell.recip, q, 150, exclude_zero=True)
    ctx = rp.Context(b.cell.lat, b.kmesh, wl.fft, b.ecut_psi, cut)
    nb = wl.nocc + wl.nemp
    ctx.load_bands(wl.nocc, b.npw, b.miller, b.coef[:, :nb], b.energy[:, :nb])
    G = OL.eps_sphere(wl.cell.lat, q, cut)
    vs = OD.coulomb_sqrt(wl.cell.lat, q, G)
    chi = ctx.rp_build_chi0(q, _axis(wl), _ordering(wl), wl.freq, wl.delta, rp.RP_FP64_NATIVE)
    W_gj, _ = ctx.rp_solve_w(q, chi)
    W_ref = OD.screened(chi, vs)
    ctx.rp_set_dyson_hermitian(True)
    W_h, _ = ctx.rp_solve_w(q, chi)
    assert np.all(_rel_fro(W_h, W_ref) < 1e-11)
    assert np.all(_rel_fro(W_h, W_gj) < 1e-12)
    dW, _ = ctx.rp_solve_w(q, torch.from_numpy(chi).cuda())
    ctx.rp_check_numeric()
    assert np.all(_rel_fro(dW.cpu().numpy(), W_ref) < 1e-11)
    # eps = 1 - 2 at G = 0 for the second frequency: not positive definite
    bad = np.zeros((3, len(G), len(G)), dtype=np.complex128)
    bad[1, 0, 0] = 2.0 / vs[0] ** 2
    with pytest.raises(rp.RPError) as e:
        ctx.rp_solve_w(q, bad)
    assert e.value.code == rp.RP_ERR_NUMERIC
    dB, _ = ctx.rp_solve_w(q, torch.from_numpy(bad).cuda())
    with pytest.raises(rp.RPError) as e:
        ctx.rp_check_numeric()
    assert e.value.code == rp.RP_ERR_NUMERIC
    dB = dB.cpu().numpy()
    for f in (0, 2):
        assert np.allclose(dB[f], np.diag(vs * vs), rtol=1e-14, atol=0)
    ctx.close()
    # three q in one packed launch of the list kernel, device buffers, against the pivoted host solves
    ctx = _ctx(wl)
    qs = np.array([wl.q[0], [0.25, 0.25, 0.0], [0.5, 0.0, 0.25]])
    cuts = np.array([_mid_gap_cutoff(wl.cell.recip, qq, t, exclude_zero=True) for qq, t in zip(qs, (40, 60, 90))])
    chis = ctx.rp_build_chi0_batched(qs, _axis(wl), _ordering(wl), wl.freq, wl.delta, rp.RP_FP64_NATIVE,
                                     ecut_eps=cuts)
    ref = ctx.rp_solve_w_batched(qs, chis, ecut_eps=cuts)
    ctx.rp_set_dyson_hermitian(True)
    dW = ctx.rp_solve_w_batched(qs, [torch.from_numpy(c).cuda() for c in chis], ecut_eps=cuts)
    ctx.rp_check_numeric()
    for (W, _), d in zip(ref, dW):
        assert np.all(_rel_fro(d.cpu().numpy(), W) < 1e-12)
    ctx.close()


def test_bad_pivot_in_a_batched_device_solve():
    """The batched Dyson solve on device buffers packs the (q, w) matrices of several q into
    cooperative launches of the list kernel: one matrix with a non-finite chi0 is reported as
    RP_ERR_NUMERIC, and every other matrix of the batch (of both q, sharing the launch and its
    barriers) is still exact (chi0 = 0 gives W = v)."""
    from synth.configs import _mid_gap_cutoff
    wl = workload("tiny")
    b = wl.bands
    qs = np.array([wl.q[0], [0.25, 0.25, 0.0]])
    cuts = np.array([_mid_gap_cutoff(wl.cell.recip, q, t, exclude_zero=True) for q, t in zip(qs, (150, 90))])
    ctx = rp.Context(b.cell.lat, b.kmesh, wl.fft, b.ecut_psi, float(cuts[0]))
    nb = wl.nocc + wl.nemp
    ctx.load_bands(wl.nocc, b.npw, b.miller, b.coef[:, :nb], b.energy[:, :nb])
    Gs = [OL.eps_sphere(wl.cell.lat, q, c) for q, c in zip(qs, cuts)]
    chis = [torch.zeros((3, len(G), len(G)), dtype=torch.complex128, device="cuda") for G in Gs]
    chis[1][2, :, 0] = float("nan")
    Ws = ctx.rp_solve_w_batched(qs, chis, ecut_eps=cuts)
    with pytest.raises(rp.RPError) as e:
        ctx.rp_check_numeric()
    assert e.value.code == rp.RP_ERR_NUMERIC
    for i, (q, G, W) in enumerate(zip(qs, Gs, Ws)):
        vs = OD.coulomb_sqrt(wl.cell.lat, q, G)
        Wh = W.cpu().numpy()
        for f in range(3):
            if (i, f) != (1, 2):
                assert np.allclose(Wh[f], np.diag(vs * vs), rtol=1e-14, atol=0)
    ctx.close()


def test_contraction_wait_that_gives_up_is_reported():
    """With the wait limit set to zero the BF16x3 contraction's pipeline waits give up at once:
    the kernel returns through its teardown (in-flight copies and MMAs drained with the fixed
    limit) and the call reports RP_ERR_TIMEOUT, on host buffers directly and, for device buffers,
    through rp_check_numeric.  With the default limit restored the same context is correct again."""
    rng = np.random.default_rng(5)
    ng, K, nf = 150, 5000, 2
    M = rng.standard_normal((ng, K)) + 1j * rng.standard_normal((ng, K))
    w = rng.standard_normal((nf, K)) + 1j * rng.standard_normal((nf, K))
    ctx = _ctx(workload("micro"))
    ctx.rp_set_wait_limit(0)
    codes = []
    for _ in range(3):
        try:
            ctx.rp_contract_chi0(M, w, precision=rp.RP_BF16X3)
            codes.append(rp.RP_OK)
        except rp.RPError as ex:
            codes.append(ex.code)
    assert set(codes) <= {rp.RP_OK, rp.RP_ERR_TIMEOUT}
    assert rp.RP_ERR_TIMEOUT in codes
    Md = torch.from_numpy(M).cuda()
    wd = torch.from_numpy(w).cuda()
    seen = False
    for _ in range(3):
        ctx.rp_contract_chi0(Md, wd, precision=rp.RP_BF16X3)
        try:
            ctx.rp_check_numeric()
        except rp.RPError as ex:
            assert ex.code == rp.RP_ERR_TIMEOUT
            seen = True
    assert seen
    ctx.rp_set_wait_limit(2_000_000_000)
    got = ctx.rp_contract_chi0(M, w, precision=rp.RP_BF16X3)
    assert np.all(_rel_fro(got, OC.chi0(M, w)) < 1e-4)


# ---- BF16x3 split-precision contraction on tcgen05 ----
# Each operand is carried as two bf16 (16 significant bits); the dropped lo*lo term and the
# FP32 accumulation inside each 8192-real window bound the error near 2^-16 per product, which
# averages down over the sum: 1e-4 relative Frobenius is the stated bound.
BF16X3_TOL = 1e-4


@pytest.mark.parametrize("ng,K,nf", [(150, 5000, 2), (64, 100, 1), (7, 33, 3), (300, 9000, 1)])
def test_contract_bf16x3(ng, K, nf):
    rng = np.random.default_rng(7 * ng + K)
    M = rng.standard_normal((ng, K)) + 1j * rng.standard_normal((ng, K))
    w = rng.standard_normal((nf, K)) + 1j * rng.standard_normal((nf, K))
    ctx = _ctx(workload("micro"))
    got = ctx.rp_contract_chi0(M, w, precision=rp.RP_BF16X3)
    ref = OC.chi0(M, w)
    err = _rel_fro(got, ref)
    print("bf16x3 rel err", err)
    assert np.all(err < BF16X3_TOL)
    # a second call on the same context gives the same bits (no stale state)
    got2 = ctx.rp_contract_chi0(M, w, precision=rp.RP_BF16X3)
    assert np.array_equal(got, got2)


@pytest.mark.parametrize("bn", list(rp.TILE_WIDTHS))
@pytest.mark.parametrize("ng,K,nf", [(300, 3000, 6), (150, 2000, 5), (37, 700, 2), (520, 1500, 1)])
def test_contract_bf16x3_every_tile_width(bn, ng, K, nf):
    """Each built tile width BN of the BF16x3 kernel (set through rp_set_contraction_tile) against the
    oracle: NG below, across and above BN (the last tile moved back to end at NG), and frequency
    counts whose last group has only one live tile (nf = 6, 5, 2, 1: the other tile is skipped)."""
    rng = np.random.default_rng(13 * ng + K + bn)
    M = rng.standard_normal((ng, K)) + 1j * rng.standard_normal((ng, K))
    w = rng.standard_normal((nf, K)) + 1j * rng.standard_normal((nf, K))
    ctx = _ctx(workload("micro"))
    ctx.rp_set_contraction_tile(ng, bn)
    got = ctx.rp_contract_chi0(M, w, precision=rp.RP_BF16X3)
    assert np.all(_rel_fro(got, OC.chi0(M, w)) < BF16X3_TOL)


def test_contraction_tile_tuner():
    """rp_tune_contraction times every tile width on synthetic operands, keeps the fastest for this
    NG, and later contractions with that NG use it and stay correct; a width that is not built is
    refused."""
    ctx = _ctx(workload("micro"))
    ng, K, nf = 400, 20000, 4
    bn, ms = ctx.rp_tune_contraction(ng, K, nf)
    assert bn in rp.TILE_WIDTHS
    assert all(v > 0 for v in ms.values()) and ms[bn] == min(ms.values())
    rng = np.random.default_rng(3)
    M = rng.standard_normal((ng, 3000)) + 1j * rng.standard_normal((ng, 3000))
    w = rng.standard_normal((nf, 3000)) + 1j * rng.standard_normal((nf, 3000))
    got = ctx.rp_contract_chi0(M, w, precision=rp.RP_BF16X3)
    assert np.all(_rel_fro(got, OC.chi0(M, w)) < BF16X3_TOL)
    with pytest.raises(rp.RPError) as e:
        ctx.rp_set_contraction_tile(ng, 100)
    assert e.value.code == rp.RP_ERR_ARG


def test_build_chi0_bf16x3_tiny(tiny, tiny_ref):
    chi_ref, W_ref = tiny_ref
    ctx = _ctx(tiny)
    q = tiny.q[0]
    chi = ctx.rp_build_chi0(q, _axis(tiny), _ordering(tiny), tiny.freq, tiny.delta, rp.RP_BF16X3)
    e = _rel_fro(chi, chi_ref)
    print("bf16x3 chi0 rel err per frequency", e)
    assert np.all(e < BF16X3_TOL)
    W, _ = ctx.rp_solve_w(q, chi)
    assert np.all(_rel_fro(W, W_ref) < BF16X3_TOL)


# TF32x3: operands split into TF32 hi + lo (2^-22 relative left out), FP32 accumulation over
# chunks of 16 reals (at most 16 roundings of 2^-23 = 1.9e-6 relative) added into FP64: 2e-6.
TF32X3_TOL = 2e-6


@pytest.mark.parametrize("ng,K,nf", [(150, 5000, 2), (64, 100, 1), (7, 33, 3), (130, 20000, 1)])
def test_contract_tf32x3(ng, K, nf):
    rng = np.random.default_rng(11 * ng + K)
    M = rng.standard_normal((ng, K)) + 1j * rng.standard_normal((ng, K))
    w = rng.standard_normal((nf, K)) + 1j * rng.standard_normal((nf, K))
    ctx = _ctx(workload("micro"))
    got = ctx.rp_contract_chi0(M, w, precision=rp.RP_TF32X3)
    ref = OC.chi0(M, w)
    err = _rel_fro(got, ref)
    print("tf32x3 rel err", err)
    assert np.all(err < TF32X3_TOL)


def test_build_chi0_tf32x3_tiny(tiny, tiny_ref):
    chi_ref, W_ref = tiny_ref
    ctx = _ctx(tiny)
    q = tiny.q[0]
    chi = ctx.rp_build_chi0(q, _axis(tiny), _ordering(tiny), tiny.freq, tiny.delta, rp.RP_TF32X3)
    e = _rel_fro(chi, chi_ref)
    print("tf32x3 chi0 rel err per frequency", e)
    assert np.all(e < TF32X3_TOL)
    W, _ = ctx.rp_solve_w(q, chi)
    assert np.all(_rel_fro(W, W_ref) < TF32X3_TOL)


# ---- FP32 weights of the split-precision path (FP64 re-evaluation near degeneracies) ----
# FP32 rounding amplified by the divided-difference recursion of resonant node sets stays below
# 1e-4 of the largest weight of a frequency, the budget of the split-precision chi0.
FP32_WEIGHT_TOL = 1e-4

@pytest.mark.parametrize("name,axis,delta", [("micro", "imag", 0.0), ("small", "real", 0.02),
                                             ("small", "real", 0.05 / 27.211386245988)])
def test_tetra_weights_fp32_path(name, axis, delta):
    from dataclasses import replace
    wl = workload(name)
    freq = wl.freq if axis == wl.axis else (np.linspace(0.0, 0.8, 5) if axis == "real" else wl.freq)
    wl = replace(wl, axis=axis, delta=delta, freq=freq)
    ctx = _ctx(wl)
    q = wl.q[0]
    ref = OC.pair_weights(wl, q)
    got = ctx.rp_tetra_weights(q, _axis(wl), _ordering(wl), wl.freq, wl.delta, precision=rp.RP_BF16X3)
    scale = np.abs(ref).max(axis=1, keepdims=True)
    err = np.abs(got - ref).max(axis=1, keepdims=True) / scale
    print("fp32 weights max err / max |w|", err.ravel())
    assert np.all(np.isfinite(got))
    assert np.all(err < FP32_WEIGHT_TOL)


def test_build_chi0_bf16x3_real_axis_small_broadening():
    from dataclasses import replace
    wl = workload("small")
    wl = replace(wl, axis="real", delta=0.05 / 27.211386245988, freq=np.linspace(0.0, 0.7, 6))
    ctx = _ctx(wl)
    q = wl.q[0]
    G = OL.eps_sphere(wl.cell.lat, q, wl.ecut_eps[0])
    M = OP.pair_density(wl.bands, wl.nocc, wl.nemp, q, G, fft=wl.fft)
    chi_ref = OC.chi0(M, OC.pair_weights(wl, q))
    chi = ctx.rp_build_chi0(q, rp.RP_AXIS_REAL, rp.RP_TIME_ORDERED, wl.freq, wl.delta, rp.RP_BF16X3)
    e = _rel_fro(chi, chi_ref)
    print("bf16x3 real-axis chi0 rel err", e)
    assert np.all(e < BF16X3_TOL)


def test_batched_q_with_uneven_spheres_tiny():
    """rp_build_chi0_batched / rp_solve_w_batched over three q of the 4^3 mesh (Gamma excluded),
    each with its own epsilon cut-off (NG about 20, 50 and 80, cut-offs placed mid-gap), against
    the oracle per member."""
    from synth.configs import _mid_gap_cutoff
    wl = workload("tiny")
    ctx = _ctx(wl)
    qs = np.array([wl.q[0], [0.25, 0.25, 0.0], [0.5, 0.0, 0.25]])
    cuts = np.array([_mid_gap_cutoff(wl.cell.recip, q, t, exclude_zero=True) for q, t in zip(qs, (20, 50, 80))])
    assert np.all(cuts < wl.bands.ecut_psi)
    chis = ctx.rp_build_chi0_batched(qs, _axis(wl), _ordering(wl), wl.freq, wl.delta, rp.RP_FP64_NATIVE,
                                     ecut_eps=cuts)
    ws = ctx.rp_solve_w_batched(qs, chis, ecut_eps=cuts)
    sizes = []
    for q, cut, chi, (W, tail) in zip(qs, cuts, chis, ws):
        G = OL.eps_sphere(wl.cell.lat, q, cut)
        sizes.append(len(G))
        assert chi.shape == (len(wl.freq), len(G), len(G))
        M = OP.pair_density(wl.bands, wl.nocc, wl.nemp, q, G, fft=wl.fft)
        chi_ref = OC.chi0(M, OC.pair_weights(wl, q))
        assert np.all(_rel_fro(chi, chi_ref) < 1e-11)
        W_ref = OD.screened(chi_ref, OD.coulomb_sqrt(wl.cell.lat, q, G))
        assert np.all(_rel_fro(W, W_ref) < 1e-11)
        T = OL.tail_sphere(wl.cell.lat, q, cut, wl.bands.ecut_psi)
        assert np.allclose(tail, OD.tail(wl.cell.lat, q, T), rtol=1e-14, atol=0)
    # the same batch on device buffers: the (q, w) matrices of all three q in one packed launch of
    # the list kernel, the same W as the per-q host-buffer solves
    dev = [torch.from_numpy(c).cuda() for c in chis]
    dW = ctx.rp_solve_w_batched(qs, dev, ecut_eps=cuts)
    ctx.rp_check_numeric()
    for (W, _), d in zip(ws, dW):
        assert np.all(_rel_fro(d.cpu().numpy(), W) < 1e-13)
    assert len(set(sizes)) == 3


def test_kset_builds_partition_the_mesh(tiny, tiny_ref):
    """rp_build_chi0_kset: the chi0 of a k subset is the oracle's sum over those k points' pairs
    (full-mesh weights), and the subsets of a partition of the mesh add up to the whole build."""
    q = tiny.q[0]
    ctx = _ctx(tiny)
    nk = tiny.bands.kfrac.shape[0]
    ks = [41, 3, 17, 18, 19, 60]                 # unsorted, with a run of consecutive points
    G = OL.eps_sphere(tiny.cell.lat, q, tiny.ecut_eps[0])
    M = OP.pair_density(tiny.bands, tiny.nocc, tiny.nemp, q, G, fft=tiny.fft, k_list=sorted(ks))
    ref = OC.chi0(M, OC.pair_weights(tiny, q, k_list=sorted(ks)))
    for p, tol in ((rp.RP_FP64_NATIVE, 1e-11), (rp.RP_BF16X3, BF16X3_TOL)):
        got = ctx.rp_build_chi0_kset(q, ks, _axis(tiny), _ordering(tiny), tiny.freq, tiny.delta, p)
        assert np.all(_rel_fro(got, ref) < tol)
    parts = [list(range(0, nk, 2)), list(range(1, nk, 2))]
    tot = sum(ctx.rp_build_chi0_kset(q, part, _axis(tiny), _ordering(tiny), tiny.freq, tiny.delta,
                                     rp.RP_FP64_NATIVE) for part in parts)
    assert np.all(_rel_fro(tot, tiny_ref[0]) < 1e-11)
    with pytest.raises(rp.RPError) as e:
        ctx.rp_build_chi0_kset(q, [1, 1], _axis(tiny), _ordering(tiny), tiny.freq, tiny.delta, rp.RP_FP64_NATIVE)
    assert e.value.code == rp.RP_ERR_ARG


def test_gamma_point_build_and_w(tiny):
    """q = 0: k' = k with no umklapp, and the epsilon sphere leaves out G = 0 (its Coulomb factor
    diverges; the analytic head is not part of this path).  chi0 (FP64 and BF16x3) and W against
    the oracle with the same convention, and the sphere lists against the oracle's."""
    q = np.zeros(3)
    ctx = _ctx(tiny)
    g, t = ctx.rp_sphere_size(q)
    G = OL.eps_sphere(tiny.cell.lat, q, tiny.ecut_eps[0])
    assert np.array_equal(g, G) and not np.any(np.all(G == 0, axis=1))
    assert np.array_equal(t, OL.tail_sphere(tiny.cell.lat, q, tiny.ecut_eps[0], tiny.bands.ecut_psi))
    M = OP.pair_density(tiny.bands, tiny.nocc, tiny.nemp, q, G, fft=tiny.fft)
    chi_ref = OC.chi0(M, OC.pair_weights(tiny, q))
    W_ref = OD.screened(chi_ref, OD.coulomb_sqrt(tiny.cell.lat, q, G))
    chi = ctx.rp_build_chi0(q, _axis(tiny), _ordering(tiny), tiny.freq, tiny.delta, rp.RP_FP64_NATIVE)
    assert np.all(_rel_fro(chi, chi_ref) < 1e-11)
    W, _ = ctx.rp_solve_w(q, chi)
    assert np.all(_rel_fro(W, W_ref) < 1e-11)
    chi = ctx.rp_build_chi0(q, _axis(tiny), _ordering(tiny), tiny.freq, tiny.delta, rp.RP_BF16X3)
    assert np.all(_rel_fro(chi, chi_ref) < BF16X3_TOL)


def test_constrained_chi0_with_wannier_weights():
    """cRPA (Eq. chi with T of Eq. tak from the Wannier construction): a window of two occupied and two
    empty bands and two projected Gaussians, so 0 < T < 1 on the window and pairs inside it are
    partly removed; FP64 and BF16x3 against the oracle on the small workload."""
    from dataclasses import replace
    from synth.wannier import gaussian_wannier
    wl = workload("small")
    _, T = gaussian_wannier(wl.bands, 4, np.array([(0.1, 0.2, 0.0), (0.5, 0.4, 0.3)]), 1.6, first=wl.nocc - 2,
                            with_T=True)
    wl = replace(wl, T=T)
    ctx = _ctx(wl)
    q = wl.q[0]
    G = OL.eps_sphere(wl.cell.lat, q, wl.ecut_eps[0])
    M = OP.pair_density(wl.bands, wl.nocc, wl.nemp, q, G, fft=wl.fft)
    chi_ref = OC.chi0(M, OC.pair_weights(wl, q))
    chi_rpa = OC.chi0(M, OC.pair_weights(replace(wl, T=None), q))
    assert np.all(_rel_fro(chi_ref, chi_rpa) > 1e-3)         # the constraint changes chi0
    for p, tol in ((rp.RP_FP64_NATIVE, 1e-11), (rp.RP_BF16X3, BF16X3_TOL)):
        chi = ctx.rp_build_chi0(q, _axis(wl), _ordering(wl), wl.freq, wl.delta, p)
        assert np.all(_rel_fro(chi, chi_ref) < tol)


def test_rotation_to_reducible_q():
    """rp_rotate_q against the oracle's rotation of the same matrix, and the rotated GPU chi0 and W of
    q* against the GPU's direct build at q (6 + 6 bands of the 4^3 cell: both ends of the band list in
    gaps; Lorentz-exact k sums are checked by the oracle pin, the tetrahedron sum agrees to its
    integration error)."""
    from oracle import symmetry as SY
    from synth.epm import cubic_rotations
    wl = workload("tiny", nocc=6, nemp=6)
    ctx = _ctx(wl)
    qs = np.array([0.25, 0.0, 0.0])
    S = next(S for S in cubic_rotations(wl.cell.recip) if not np.allclose(np.mod(qs @ S, 1.0), qs))
    img = qs @ S
    q = np.mod(img, 1.0)
    g_s = np.rint(img - q).astype(np.int64)
    chi_s = ctx.rp_build_chi0(qs, _axis(wl), _ordering(wl), wl.freq, wl.delta, rp.RP_FP64_NATIVE)
    got = ctx.rp_rotate_q(qs, q, S, chi_s)
    Gs = OL.eps_sphere(wl.cell.lat, qs, wl.ecut_eps[0])
    G = OL.eps_sphere(wl.cell.lat, q, wl.ecut_eps[0])
    assert np.array_equal(got, SY.rotate(chi_s, SY.image_index(Gs, G, S, g_s)))
    direct = ctx.rp_build_chi0(q, _axis(wl), _ordering(wl), wl.freq, wl.delta, rp.RP_FP64_NATIVE)
    assert np.all(_rel_fro(got, direct) < 5e-2)
    W_s, _ = ctx.rp_solve_w(qs, chi_s)
    W_q, _ = ctx.rp_solve_w(q, got)
    assert np.all(_rel_fro(ctx.rp_rotate_q(qs, q, S, W_s), W_q) < 1e-12)
    with pytest.raises(rp.RPError) as e:
        ctx.rp_rotate_q(qs, np.array([0.0, 0.5, 0.0]), S, chi_s)
    assert e.value.code == rp.RP_ERR_ARG


def test_peak_probes_run():
    """rp_probe_peaks: the three probe kernels return and give rates of the right order for a GB300
    (FP64 about 1 TFLOP/s on both paths, bf16 tcgen05 some 1-2.5 PFLOP/s)."""
    p = rp.probe_peaks()
    assert 0.1 < p["fp64_fma"] < 20 and 0.1 < p["fp64_mma"] < 20
    assert 300 < p["bf16_tcgen05"] < 3000
    print("probes", p)
