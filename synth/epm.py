"""Empirical-pseudopotential band generator (setup only, not the method).

H_k[G,G'] = 1/2 |k+G|^2 delta_GG' + V(G-G'), diagonalised per k point for the
lowest `nband` states.  The plane-wave set per k is the sphere
1/2 |k+G|^2 <= E_cut^psi (the basis of the Bloch expansion, Eq. pak).  Each
eigenvector is multiplied by a seeded random phase so that no accidental
reality of the coefficients hides a conjugation error downstream.

With `symmetry=True` (shell potential only) H_k is diagonalised only at one mesh point of each
orbit of the cube's 48 rotations and the other points are filled by rotating its eigenvectors:
V depends on |G| alone and is real and even, so for a rotation R, with S the integer matrix of R
on fractional reciprocal coordinates (row vectors: (k S) B = R (k B)) and R k = k' + G_s (k' on
the mesh), the coefficients C_{k'}(G S + G_s) = C_k(G) are eigenvectors of H_{k'} with the same
energies.  The resulting sets are as valid as directly computed ones (any orthonormal basis of a
degenerate subspace is), and they cost one diagonalisation per orbit.

Two potentials are provided:
  * "shells": V constant on the first n reciprocal-lattice shells, magnitudes
    uniform in [vmin, vmax] Ha with random sign (real, inversion symmetric);
  * "atoms": V(G) = (1/N_at) sum_a A_a exp(-|G|^2 s_a^2 / 2) exp(-i G.tau_a)
    for seeded random positions tau_a (complex, no inversion symmetry).
"""
from __future__ import annotations

import os
import sys
from dataclasses import dataclass, field

import numpy as np

HARTREE_EV = 27.211386245988


@dataclass
class Cell:
    lat: np.ndarray       # [3,3] rows a1, a2, a3 (bohr)
    recip: np.ndarray     # [3,3] rows b1, b2, b3 (1/bohr), a_i . b_j = 2 pi delta_ij
    omega: float          # cell volume (bohr^3)


def _cell(lat):
    lat = np.asarray(lat, dtype=np.float64)
    omega = float(abs(np.linalg.det(lat)))
    recip = 2.0 * np.pi * np.linalg.inv(lat).T
    return Cell(lat=lat, recip=recip, omega=omega)


def fcc_cell(a):
    h = 0.5 * a
    return _cell([[0.0, h, h], [h, 0.0, h], [h, h, 0.0]])


def sc_cell(a):
    return _cell(np.eye(3) * a)


def kmesh_frac(n):
    """Gamma-centred mesh; index = (i1*n2 + i2)*n3 + i3, k = (i1/n1, i2/n2, i3/n3)."""
    n = np.asarray(n, dtype=np.int64).reshape(3)
    i1, i2, i3 = np.meshgrid(np.arange(n[0]), np.arange(n[1]), np.arange(n[2]), indexing="ij")
    idx = np.stack([i1.ravel(), i2.ravel(), i3.ravel()], axis=1)
    return idx / n[None, :]


def _miller_box(recip, radius, shift=(0.0, 0.0, 0.0)):
    # |m_i| <= radius * |a_i| / (2 pi) + |shift_i| + 1
    a_len = np.linalg.norm(2.0 * np.pi * np.linalg.inv(recip).T, axis=1)
    nmax = np.floor(radius * a_len / (2.0 * np.pi) + np.abs(np.asarray(shift)) + 1).astype(int)
    r = [np.arange(-m, m + 1) for m in nmax]
    g = np.stack(np.meshgrid(*r, indexing="ij"), axis=-1).reshape(-1, 3)
    return g


def psi_sphere(recip, k_frac, ecut):
    """Miller indices m with 1/2|(k+m) B|^2 <= ecut, in lexicographic (m1,m2,m3) order."""
    g = _miller_box(recip, np.sqrt(2.0 * ecut), k_frac)
    kin = 0.5 * np.sum(((g + np.asarray(k_frac)[None, :]) @ recip) ** 2, axis=1)
    return g[kin <= ecut]          # meshgrid 'ij' order is already lexicographic


def _shell_table(recip, nshell):
    g = _miller_box(recip, 12.0 * np.linalg.norm(recip[0]))
    g2 = np.sum((g @ recip) ** 2, axis=1)
    vals = np.unique(np.round(g2[g2 > 1e-12], 9))
    return vals[:nshell]


@dataclass
class Bands:
    cell: Cell
    kmesh: tuple
    kfrac: np.ndarray          # [nk,3]
    npw: np.ndarray            # [nk] int32
    miller: np.ndarray         # [nk, npw_max, 3] int32 (zero padded)
    coef: np.ndarray           # [nk, nband, npw_max] complex128 (zero padded)
    energy: np.ndarray         # [nk, nband] float64 (Ha)
    ecut_psi: float
    meta: dict = field(default_factory=dict)


def _potential_fn(cell, pot, rng):
    if pot["kind"] == "shells":
        shells = _shell_table(cell.recip, pot["nshell"])
        mags = rng.uniform(pot["vmin"], pot["vmax"], size=len(shells))
        signs = rng.choice([-1.0, 1.0], size=len(shells))
        v = mags * signs

        def vfun(dm):
            g2 = np.sum((dm @ cell.recip) ** 2, axis=-1)
            out = np.zeros(g2.shape, dtype=np.complex128)
            for s, val in zip(shells, v):
                out[np.abs(g2 - s) < 1e-7 * max(1.0, s)] = val
            return out
        return vfun, {"shells": shells.tolist(), "v_shell": v.tolist()}
    if pot["kind"] == "atoms":
        nat = pot["natoms"]
        tau_f = rng.uniform(0.0, 1.0, size=(nat, 3))
        tau = tau_f @ cell.lat
        amp = -rng.uniform(pot["amin"], pot["amax"], size=nat)
        wid = rng.uniform(pot["smin"], pot["smax"], size=nat)

        def vfun(dm):
            gc = dm @ cell.recip
            g2 = np.sum(gc ** 2, axis=-1)
            out = np.zeros(g2.shape, dtype=np.complex128)
            for a in range(nat):
                out += amp[a] * np.exp(-0.5 * g2 * wid[a] ** 2) * np.exp(-1j * (gc @ tau[a]))
            out /= nat
            out[g2 < 1e-12] = 0.0
            return out
        return vfun, {"natoms": nat}
    raise ValueError(pot["kind"])


def _solve_k(args):
    kf, recip, ecut, nband, vtab, vofs = args
    import scipy.linalg as sl
    m = psi_sphere(recip, kf, ecut)
    kin = 0.5 * np.sum(((m + kf[None, :]) @ recip) ** 2, axis=1)
    d = m[:, None, :] - m[None, :, :] + vofs
    h = vtab[d[..., 0], d[..., 1], d[..., 2]]
    h[np.diag_indices_from(h)] += kin
    if np.all(h.imag == 0):
        # real symmetric H (the shell potential): real eigenvectors, widened when stored
        e, v = sl.eigh(h.real, subset_by_index=[0, nband - 1], driver="evr")
    else:
        e, v = sl.eigh(h, subset_by_index=[0, nband - 1], driver="evr")
    return m.astype(np.int32), e, v.T.copy()


def _cuda_in_process():
    """True when this process may hold a CUDA context (torch initialised it, or a library such
    as the C-ABI one has the driver mapped), so a worker pool must not be forked."""
    torch = sys.modules.get("torch")
    if torch is not None and torch.cuda.is_initialized():
        return True
    try:
        with open("/proc/self/maps") as f:
            return any("libcuda.so" in line for line in f)
    except OSError:
        return False


def cubic_rotations(recip):
    """Integer matrices S of the rotations R of the cube (the 48 signed permutations of the
    Cartesian axes) that map the reciprocal lattice onto itself: (k S) B = R (k B) for fractional
    row vectors k and B the rows b1, b2, b3."""
    import itertools
    B = np.asarray(recip, dtype=np.float64)
    Binv = np.linalg.inv(B)
    out = []
    for perm in itertools.permutations(range(3)):
        for signs in itertools.product((1.0, -1.0), repeat=3):
            R = np.zeros((3, 3))
            for i in range(3):
                R[i, perm[i]] = signs[i]
            S = B @ R.T @ Binv
            Si = np.rint(S)
            if np.abs(S - Si).max() < 1e-9:
                out.append(Si.astype(np.int64))
    return out


def irreducible_mesh(kmesh, rotations):
    """For every mesh point k': (index of its orbit's representative k, S, G_s) with
    k S = k' + G_s, k' the mesh point in [0, 1)^3.  Representatives map to themselves with S = 1."""
    n = np.asarray(kmesh, dtype=np.int64)
    kf = kmesh_frac(n)
    nk = kf.shape[0]
    idx = np.rint(kf * n).astype(np.int64)
    rep = -np.ones(nk, dtype=np.int64)
    rot = [None] * nk
    shift = np.zeros((nk, 3), dtype=np.int64)
    for k in range(nk):
        if rep[k] >= 0:
            continue
        for S in rotations:
            jf = ((idx[k] / n) @ S) * n              # n * (k S), component-wise
            j = np.rint(jf).astype(np.int64)
            if np.abs(jf - j).max() > 1e-9:          # the rotation leaves the mesh
                continue
            jm = np.mod(j, n)
            kk = int((jm[0] * n[1] + jm[1]) * n[2] + jm[2])
            if rep[kk] >= 0:
                continue
            rep[kk] = k
            rot[kk] = S
            shift[kk] = (j - jm) // n
    return rep, rot, shift


def make_bands(cell, kmesh, ecut_psi, nband, pot, seed, workers=None, symmetry=False):
    """Diagonalise H_k on the whole mesh (or on one point per orbit of the cube's rotations and
    rotate, `symmetry=True`, shell potential only); returns zero-padded arrays (see Bands)."""
    rng = np.random.default_rng(seed)
    vfun, meta = _potential_fn(cell, pot, rng)
    kf = kmesh_frac(kmesh)
    nk = kf.shape[0]
    if symmetry:
        if pot["kind"] != "shells":
            raise ValueError("rotating eigenvectors needs the shell potential (V a function of |G|)")
        rots = cubic_rotations(cell.recip)
        rep, rot, gshift = irreducible_mesh(kmesh, rots)
        reps = np.unique(rep)
    else:
        reps = np.arange(nk)
    # potential table over all Miller differences that can occur
    gmax = np.sqrt(2.0 * ecut_psi) + np.linalg.norm(cell.recip, axis=1).max()
    a_len = np.linalg.norm(cell.lat, axis=1)
    L = int(np.ceil(2.0 * gmax * a_len.max() / (2.0 * np.pi))) + 2
    r = np.arange(-L, L + 1)
    grid = np.stack(np.meshgrid(r, r, r, indexing="ij"), axis=-1)
    vtab = vfun(grid.reshape(-1, 3)).reshape(grid.shape[:3])
    vofs = np.array([L, L, L])
    jobs = [(kf[i], cell.recip, ecut_psi, nband, vtab, vofs) for i in reps]
    if workers is None:
        workers = min(16, os.cpu_count() or 1)
    work = len(reps) * float(max(1, len(psi_sphere(cell.recip, kf[0], ecut_psi)))) ** 3
    if work > 2e10 and workers > 1:
        import concurrent.futures as cf
        import multiprocessing as mp
        # the cores shared out over the worker processes (one BLAS thread each when there are more
        # jobs than cores; spawned children read these at start-up)
        nthr = max(1, (os.cpu_count() or 1) // max(1, min(workers, len(jobs))))
        saved = {v: os.environ.get(v) for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")}
        for v in saved:
            os.environ[v] = str(nthr)
        # fork is safe (and needs no importable __main__) only while no CUDA context can exist in
        # this process: spawn once torch has initialised CUDA or any library has loaded the driver
        cuda_up = _cuda_in_process()
        try:
            with cf.ProcessPoolExecutor(max_workers=workers,
                                        mp_context=mp.get_context("spawn" if cuda_up else "fork")) as ex:
                res = list(ex.map(_solve_k, jobs, chunksize=max(1, len(jobs) // (4 * workers))))
        finally:
            for v, val in saved.items():
                if val is None:
                    os.environ.pop(v, None)
                else:
                    os.environ[v] = val
    else:
        res = [_solve_k(j) for j in jobs]
    if symmetry:
        by_rep = {int(r): res[i] for i, r in enumerate(reps)}
        meta.update({"irreducible_k": int(len(reps))})
    npw = np.array([by_rep[int(rep[k])][0].shape[0] for k in range(nk)] if symmetry
                   else [r_[0].shape[0] for r_ in res], dtype=np.int32)
    if np.any(npw < nband):
        raise ValueError("plane-wave set smaller than the number of bands")
    pmax = int(npw.max())
    miller = np.zeros((nk, pmax, 3), dtype=np.int32)
    coef = np.zeros((nk, nband, pmax), dtype=np.complex128)
    energy = np.zeros((nk, nband), dtype=np.float64)
    phase = np.exp(2j * np.pi * rng.uniform(size=(nk, nband)))
    for i in range(nk):
        if symmetry:
            # rotate the orbit representative's eigenvectors onto this point: C(G S + G_s) = C_rep(G)
            m, e, v = by_rep[int(rep[i])]
            if rep[i] != i:
                mk = m.astype(np.int64) @ rot[i] + gshift[i]
                order = np.lexsort((mk[:, 2], mk[:, 1], mk[:, 0]))
                m = mk[order].astype(np.int32)
                v = v[:, order]
        else:
            m, e, v = res[i]
        miller[i, : m.shape[0]] = m
        coef[i, :, : m.shape[0]] = v
        coef[i, :, : m.shape[0]] *= phase[i][:, None]
        energy[i] = e
    meta.update({"seed": seed})
    return Bands(cell=cell, kmesh=tuple(int(x) for x in kmesh), kfrac=kf, npw=npw,
                 miller=miller, coef=coef, energy=energy, ecut_psi=float(ecut_psi), meta=meta)
