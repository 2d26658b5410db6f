"""Named synthetic workloads (cell, mesh, bands, q points, frequencies).

Sizes follow the five workload descriptions of the chi0 / W benchmark plus
two small ones used by the CPU test-suite.  Cutoffs are placed in the middle
of a gap between consecutive |k+G|^2 (or |q+G|^2) values so that sphere
membership never depends on the last bit of a floating-point comparison.
"""
from __future__ import annotations

import hashlib
import os
from dataclasses import dataclass
from typing import Optional

import numpy as np

from .epm import HARTREE_EV, Bands, Cell, fcc_cell, sc_cell, make_bands, _miller_box

BASE_SEED = 200102351


def _mid_gap_cutoff(recip, shift, target, exclude_zero):
    """Cutoff E with about `target` points of 1/2|shift+G|^2 <= E, mid-gap."""
    vol_bz = abs(np.linalg.det(recip))
    radius = 2.0 * (3.0 * target * vol_bz / (4.0 * np.pi)) ** (1.0 / 3.0)
    g = _miller_box(recip, radius, shift)
    e = 0.5 * np.sum(((g + np.asarray(shift)[None, :]) @ recip) ** 2, axis=1)
    if exclude_zero:
        e = e[e > 1e-12]
    e = np.sort(e)
    n = min(max(target, 1), len(e) - 1)
    # walk upwards until the gap to the next value is clearly resolved
    while n < len(e) - 1 and (e[n] - e[n - 1]) <= 1e-6 * max(1.0, e[n]):
        n += 1
    return 0.5 * (e[n - 1] + e[n])


def _mid_gap_cutoff_mesh(recip, kmesh, target):
    """Wave-function cut-off with about `target` points at k = 0, placed in the middle of a gap of
    the values 1/2|k+G|^2 of every mesh point k, so that no sphere of the mesh has a member on
    the cut-off (a value on it would make membership depend on rounding)."""
    from .epm import kmesh_frac
    vol_bz = abs(np.linalg.det(recip))
    radius = 2.0 * (3.0 * target * vol_bz / (4.0 * np.pi)) ** (1.0 / 3.0)
    e0 = _mid_gap_cutoff(recip, (0.0, 0.0, 0.0), target, exclude_zero=False)
    g = _miller_box(recip, radius, (1.0, 1.0, 1.0))
    # every value of the mesh within 3% of e0, then the gap whose middle is nearest to e0
    near = [np.zeros(0)]
    for k in kmesh_frac(kmesh):
        e = 0.5 * np.sum(((g + k[None, :]) @ recip) ** 2, axis=1)
        near.append(e[np.abs(e - e0) <= 0.03 * e0])
    v = np.unique(np.concatenate(near))
    tol = 1e-9 * max(1.0, e0)
    gaps = np.nonzero(np.diff(v) > tol)[0]
    if gaps.size == 0:
        raise ValueError("no gap of the mesh's kinetic energies near the cut-off")
    mids = 0.5 * (v[gaps] + v[gaps + 1])
    return float(mids[np.argmin(np.abs(mids - e0))])


def log_grid(lo, hi, n):
    return lo * (hi / lo) ** (np.arange(n) / (n - 1))


CONFIGS = {
    # CPU test-suite sizes
    "micro": dict(cell=("fcc", 10.2), pot=dict(kind="shells", nshell=6, vmin=0.1, vmax=0.3),
                  npw=60, fft=(12, 12, 12), kmesh=(2, 2, 2), nocc=4, nemp=4, ng=15,
                  axis="imag", freq=log_grid(0.01, 2.0, 4), delta=0.0, q=[(0.5, 0.0, 0.0)]),
    "small": dict(cell=("fcc", 10.2), pot=dict(kind="shells", nshell=6, vmin=0.1, vmax=0.3),
                  npw=110, fft=(16, 16, 16), kmesh=(3, 3, 3), nocc=4, nemp=8, ng=27,
                  axis="real", freq=np.linspace(0.0, 1.0, 5), delta=0.02, q=[(1.0 / 3.0, 0.0, 0.0)]),
    # tiny: 4^3 mesh, 8+8 bands, NG~50, 8 imaginary frequencies 0.01..2 Ha
    "tiny": dict(cell=("fcc", 10.2), pot=dict(kind="shells", nshell=6, vmin=0.1, vmax=0.3),
                 npw=300, fft=(16, 16, 16), kmesh=(4, 4, 4), nocc=8, nemp=8, ng=50,
                 axis="imag", freq=log_grid(0.01, 2.0, 8), delta=0.0, q=[(0.25, 0.0, 0.0)]),
    # medium: 8^3 mesh, 40+160 bands, NG~400, 20 real frequencies 0..20 eV, delta 0.05 eV
    "medium": dict(cell=("fcc", 10.2), pot=dict(kind="shells", nshell=6, vmin=0.1, vmax=0.3),
                   npw=1200, fft=(32, 32, 32), kmesh=(8, 8, 8), nocc=40, nemp=160, ng=400,
                   axis="real", freq=np.linspace(0.0, 20.0, 20) / HARTREE_EV,
                   delta=0.05 / HARTREE_EV, q=[(0.125, 0.0, 0.0)]),
    # precision: 10^3 mesh, 64+448 bands, NG~1500, 30 real frequencies 0..20 eV
    "precision": dict(cell=("fcc", 10.2), pot=dict(kind="shells", nshell=6, vmin=0.1, vmax=0.3),
                      npw=4000, fft=(48, 48, 48), kmesh=(10, 10, 10), nocc=64, nemp=448, ng=1500,
                      axis="real", freq=np.linspace(0.0, 20.0, 30) / HARTREE_EV,
                      delta=0.05 / HARTREE_EV, q=[(0.1, 0.0, 0.0)], symmetry=True),
    # batched: all 216 q of a 6^3 mesh, NG 300..900 per q, 24 imaginary frequencies
    "batched": dict(cell=("fcc", 10.2), pot=dict(kind="shells", nshell=6, vmin=0.1, vmax=0.3),
                    npw=1200, fft=(32, 32, 32), kmesh=(6, 6, 6), nocc=16, nemp=64, ng=(300, 900),
                    axis="imag", freq=log_grid(0.01, 2.0, 24), delta=0.0, q="all", symmetry=True),
    # large: simple-cubic a=20 bohr, 64 Gaussian "atoms", 2^3 mesh, 256+1024 bands
    "large": dict(cell=("sc", 20.0), pot=dict(kind="atoms", natoms=64, amin=0.5, amax=1.5, smin=0.8, smax=1.6),
                  npw=9000, fft=(72, 72, 72), kmesh=(2, 2, 2), nocc=256, nemp=1024, ng=4000,
                  axis="imag", freq=log_grid(0.01, 2.0, 16), delta=0.0, q=[(0.5, 0.0, 0.0)]),
}


@dataclass
class Workload:
    name: str
    bands: Bands
    fft: tuple
    nocc: int
    nemp: int
    q: np.ndarray            # [nq,3] fractional, each a mesh vector
    ecut_eps: np.ndarray     # [nq] Ha
    axis: str                # "imag" (omega = i*nu) or "real"
    freq: np.ndarray         # [nfreq] Ha (nu on the imaginary axis)
    delta: float             # broadening (Ha)
    ordering: str = "time"   # "time" (time-ordered X) or "retarded"
    T: Optional[np.ndarray] = None   # [nk, nband] cRPA weights or None
    delta_a: float = 1e-8
    delta_r: float = 1e-8

    @property
    def cell(self) -> Cell:
        return self.bands.cell


def _cache_dir():
    d = os.environ.get("RP_CACHE_DIR", os.path.join(os.path.expanduser("~"), ".cache", "respack_gb300"))
    os.makedirs(d, exist_ok=True)
    return d


def workload_shape(name, **overrides):
    """Everything of a workload but its bands: cell, mesh, grid, cut-offs, q points, band counts and
    frequencies (cheap; used where only the sizes matter)."""
    spec = dict(CONFIGS[name])
    spec.update(overrides)
    seed = BASE_SEED + list(CONFIGS).index(name) if name in CONFIGS else BASE_SEED
    kind, a = spec["cell"]
    cell = fcc_cell(a) if kind == "fcc" else sc_cell(a)
    ecut_psi = _mid_gap_cutoff_mesh(cell.recip, spec["kmesh"], spec["npw"])
    rng = np.random.default_rng(seed + 7)
    kmesh = np.array(spec["kmesh"])
    if spec["q"] == "all":
        from .epm import kmesh_frac
        q = kmesh_frac(kmesh)
    else:
        q = np.array(spec["q"], dtype=np.float64).reshape(-1, 3)
    ng = spec["ng"]
    ecut_eps = []
    for qi in q:
        target = int(rng.integers(ng[0], ng[1] + 1)) if isinstance(ng, tuple) else int(ng)
        ecut_eps.append(_mid_gap_cutoff(cell.recip, qi, target, exclude_zero=True))
    return dict(spec=spec, seed=seed, cell=cell, kind=kind, a=a, ecut_psi=ecut_psi, q=q,
                ecut_eps=np.array(ecut_eps), rng=rng)


def make_workload(name, crpa=False, cache=True, workers=None, **overrides):
    sh = workload_shape(name, **overrides)
    spec, seed, cell, kind, a, ecut_psi = sh["spec"], sh["seed"], sh["cell"], sh["kind"], sh["a"], sh["ecut_psi"]
    nband = spec["nocc"] + spec["nemp"]
    symmetry = bool(spec.get("symmetry", False))
    key = hashlib.sha1(repr((name, seed, spec["kmesh"], ecut_psi, nband, spec["pot"], a, kind,
                             symmetry)).encode()).hexdigest()[:16]
    path = os.path.join(_cache_dir(), f"{name}_{key}.npz")
    # band sets of several GB are regenerated rather than written to and read from disk
    big = np.prod(spec["kmesh"]) * nband * spec["npw"] * 16 > (2 << 30)
    cache = cache and not big
    bands = None
    if cache and os.path.exists(path):
        z = np.load(path, allow_pickle=False)
        bands = Bands(cell=cell, kmesh=tuple(spec["kmesh"]), kfrac=z["kfrac"], npw=z["npw"],
                      miller=z["miller"], coef=z["coef"], energy=z["energy"], ecut_psi=float(ecut_psi),
                      meta={"seed": seed, "cached": True})
    if bands is None:
        bands = make_bands(cell, spec["kmesh"], ecut_psi, nband, spec["pot"], seed, workers=workers,
                           symmetry=symmetry)
        if cache:
            tmp = path + ".tmp.npz"
            np.savez(tmp, kfrac=bands.kfrac, npw=bands.npw, miller=bands.miller,
                     coef=bands.coef, energy=bands.energy)
            os.replace(tmp, path)
    T = None
    if crpa:
        T = sh["rng"].uniform(0.0, 1.0, size=bands.energy.shape)
    return Workload(name=name, bands=bands, fft=tuple(spec["fft"]), nocc=spec["nocc"], nemp=spec["nemp"],
                    q=sh["q"], ecut_eps=sh["ecut_eps"], axis=spec["axis"],
                    freq=np.asarray(spec["freq"], dtype=np.float64), delta=float(spec["delta"]), T=T)
