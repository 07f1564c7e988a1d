"""Seeded synthetic plasma loads shared by the CUDA path and the oracle.

This module only draws initial particle states (cell index, in-cell offsets, momenta) from a
seed.  It holds none of the PIC step's arithmetic; both the CUDA library and the oracle take
its arrays unchanged, so both sides start from bit-identical FP32-representable inputs.

Physics of the load (simulation section of arXiv:0808.4078): a relativistic electron beam of
density nb drifting along z through background electrons of density np = n0 - nb that carry
the return current, so the initial net current is zero; immobile ions of density n0.  Units:
density n0, momentum u = gamma v / c, length c/w_p.
"""
from __future__ import annotations

from dataclasses import dataclass, field
import math

import numpy as np

ELECTRON_Q = -1.0
ELECTRON_M = 1.0


@dataclass
class SpeciesLoad:
    """Initial state of one species.

    cell   int32 [N]      linear cell index, x fastest: (k*ny + j)*nx + i
    offset float32 [ndim, N]  in-cell offsets in [0, 1) along x, y(, z)
    u      float32 [3, N] momentum gamma*v/c
    w      density carried by one macro-particle (units n0)
    nu     Krook collision rate acting on this species' cell-mean momentum (units w_p)
    """
    name: str
    q: float
    m: float
    w: float
    nu: float
    cell: np.ndarray
    offset: np.ndarray
    u: np.ndarray

    @property
    def n(self) -> int:
        return int(self.cell.shape[0])


@dataclass
class Workload:
    name: str
    ndim: int
    nx: int
    ny: int
    nz: int
    dx: float
    dy: float
    dz: float
    dt: float
    steps: int
    species: list = field(default_factory=list)

    @property
    def ncell(self) -> int:
        return self.nx * self.ny * self.nz

    @property
    def nparticles(self) -> int:
        return sum(s.n for s in self.species)


def _cells_and_offsets(rng, ndim, nx, ny, nz, ppc, lattice=False):
    ncell = nx * ny * nz
    cell = np.repeat(np.arange(ncell, dtype=np.int32), ppc)
    n = cell.shape[0]
    if lattice:
        # quiet start: ppc = m^ndim particles per cell on a sub-lattice
        m = round(ppc ** (1.0 / ndim))
        if m ** ndim != ppc:
            raise ValueError("lattice loading needs ppc = m**ndim")
        sub = (np.arange(m, dtype=np.float64) + 0.5) / m
        grids = np.meshgrid(*([sub] * ndim), indexing="ij")
        pat = np.stack([g.reshape(-1) for g in grids])
        offset = np.tile(pat, (1, ncell)).astype(np.float32)
    else:
        offset = rng.random((ndim, n), dtype=np.float32)
    return cell, offset


def _zero_mean(a):
    return a - a.mean() if a.size else a


def _solve_drift(target_sum, duz, uperp2):
    """Drift d (FP64, Newton) with sum_p (d + duz_p) / sqrt(1 + uperp2_p + (d + duz_p)^2) = target."""
    d = 0.0
    for _ in range(60):
        uz = d + duz
        g = np.sqrt(1.0 + uperp2 + uz * uz)
        f = np.sum(uz / g) - target_sum
        fp = np.sum((1.0 + uperp2) / g ** 3)
        step = f / fp
        d -= step
        if abs(step) < 1e-15 * max(1.0, abs(d)):
            break
    return d


def weibel_load(*, ndim=2, nx, ny, nz=1, ppc, gamma_b=3.0, nb=0.1, T_perp_beam=0.0,
                T_par_beam=0.0, T_bg=0.0, nu=0.0, seed=1, dx=0.1, dt=0.05, steps=0,
                lattice=False, name=None) -> Workload:
    """Beam + return-current background electrons with zero initial net current along z.

    Beam: u_z = sqrt(gamma_b^2 - 1) (cold along z unless T_par_beam > 0), transverse
    u ~ N(0, sqrt(T_perp_beam)) per component.  Background: each component ~ N(0, sqrt(T_bg))
    around a drift along -z chosen so the sampled current sum_p w v_z vanishes (FP64 solve,
    stored in FP32).  Exactly ppc particles per cell per species; offsets U[0,1).
    """
    if ndim == 2:
        nz = 1
    dz = dx
    ss = np.random.SeedSequence(seed)
    rb, rp = [np.random.default_rng(s) for s in ss.spawn(2)]
    np_ = 1.0 - nb
    wb, wp = nb / ppc, np_ / ppc

    cb, ob = _cells_and_offsets(rb, ndim, nx, ny, nz, ppc, lattice)
    cp, op = _cells_and_offsets(rp, ndim, nx, ny, nz, ppc, lattice)
    nbp, npp = cb.shape[0], cp.shape[0]

    uz0 = math.sqrt(gamma_b * gamma_b - 1.0)
    sb = math.sqrt(T_perp_beam)
    ubx = _zero_mean(rb.standard_normal(nbp) * sb) if sb > 0 else np.zeros(nbp)
    uby = _zero_mean(rb.standard_normal(nbp) * sb) if sb > 0 else np.zeros(nbp)
    spar = math.sqrt(T_par_beam)
    ubz = uz0 + (_zero_mean(rb.standard_normal(nbp) * spar) if spar > 0 else 0.0)
    ub = np.stack([ubx, uby, np.broadcast_to(ubz, (nbp,))]).astype(np.float32)

    sp = math.sqrt(T_bg)
    upx = _zero_mean(rp.standard_normal(npp) * sp) if sp > 0 else np.zeros(npp)
    upy = _zero_mean(rp.standard_normal(npp) * sp) if sp > 0 else np.zeros(npp)
    duz = _zero_mean(rp.standard_normal(npp) * sp) if sp > 0 else np.zeros(npp)
    upx = upx.astype(np.float32).astype(np.float64)
    upy = upy.astype(np.float32).astype(np.float64)

    ub64 = ub.astype(np.float64)
    gb = np.sqrt(1.0 + (ub64 * ub64).sum(0))
    beam_current = wb * np.sum(ub64[2] / gb)
    d = _solve_drift(-beam_current / wp, duz, upx * upx + upy * upy)
    up = np.stack([upx, upy, d + duz]).astype(np.float32)

    beam = SpeciesLoad("beam", ELECTRON_Q, ELECTRON_M, wb, 0.0, cb, ob, ub)
    bg = SpeciesLoad("background", ELECTRON_Q, ELECTRON_M, wp, nu, cp, op, up)
    if name is None:
        dims = f"{nx}x{ny}" + (f"x{nz}" if ndim == 3 else "")
        name = f"weibel_{ndim}d_{dims}_ppc{ppc}"
    return Workload(name, ndim, nx, ny, nz, dx, dx, dz, dt, steps, [beam, bg])


# Named workloads (sizes in the names).  Seeds 1..3 are fixed per workload.
def cold_beam_2d_64(seed=1, steps=500):
    """64x64 2D3V, cold gamma=3 beam (nb=0.1), cold background, 16 ppc/species, collisionless."""
    return weibel_load(ndim=2, nx=64, ny=64, ppc=16, seed=seed, steps=steps,
                       name="cold_beam_2d_64x64_ppc16")


def warm_beam_krook_2d(n=1024, ppc=64, seed=2, steps=4000):
    """n x n 2D3V, beam T_perp=0.1, background T=0.001, Krook nu=0.1, 64 ppc/species."""
    return weibel_load(ndim=2, nx=n, ny=n, ppc=ppc, T_perp_beam=0.1, T_bg=0.001, nu=0.1,
                       seed=seed, steps=steps, name=f"warm_beam_krook_2d_{n}x{n}_ppc{ppc}")


def hot_beam_3d(nx=256, ny=256, nz=512, ppc=8, seed=3, steps=2000):
    """3D3V, beam along z, T_perp=0.2, cold collisionless background, 8 ppc/species."""
    return weibel_load(ndim=3, nx=nx, ny=ny, nz=nz, ppc=ppc, T_perp_beam=0.2, seed=seed,
                       steps=steps, name=f"hot_beam_3d_{nx}x{ny}x{nz}_ppc{ppc}")


SCAN_SIZES = (128, 192, 256, 384, 512)
SCAN_NU = (0.0, 0.01, 0.1, 1.0)


def scan_table(nruns=256, seed=4):
    """The run table of the temperature / collision-rate scan: per run (nx, ny, T_perp, nu),
    nx and ny drawn independently from SCAN_SIZES, T_perp ~ U[0, 1], nu from SCAN_NU."""
    rng = np.random.default_rng(seed)
    nx = rng.choice(SCAN_SIZES, nruns)
    ny = rng.choice(SCAN_SIZES, nruns)
    T = rng.random(nruns)
    nu = rng.choice(SCAN_NU, nruns)
    return [(int(nx[r]), int(ny[r]), float(T[r]), float(nu[r])) for r in range(nruns)]


def scan_runs(nruns=256, ppc=32, seed=4, steps=2000, scale=1):
    """Workloads of the scan table: 2D3V runs of 32 ppc/species, beam T_perp from the table,
    background T = 0.001 with the table's Krook rate; run r is loaded with seed 1000 + r.
    `scale` divides every grid side (small stand-ins of the same table for tests)."""
    out = []
    for r, (nx, ny, T, nu) in enumerate(scan_table(nruns, seed)):
        out.append(weibel_load(ndim=2, nx=nx // scale, ny=ny // scale, ppc=ppc, T_perp_beam=T,
                               T_bg=0.001, nu=nu, seed=1000 + r, steps=steps,
                               name=f"scan_run{r}_{nx // scale}x{ny // scale}"))
    return out


def scan_run(job):
    """Run r of the scan table at full size: job = (r, (nx, ny, T_perp, nu), ppc) -> (r, workload).
    A top-level function, so spawned process pools can generate runs in parallel."""
    r, (nx, ny, T, nu), ppc = job
    return r, weibel_load(ndim=2, nx=nx, ny=ny, ppc=ppc, T_perp_beam=T, T_bg=0.001, nu=nu,
                          seed=1000 + r, name=f"scan_run{r}_{nx}x{ny}")


# ---------------------------------------------------------------- parallel generation
# Large loads (hundreds of millions of particles) drawn by a pool of processes into shared
# memory.  Same distributions as weibel_load; the streams differ (one child seed per chunk of
# cells), so the particles are not the same as weibel_load's for the same seed.

def _chunk_fill(args):
    (shm_names, n_total, ndim, nx, ny, nz, ppc, c0, c1, seed, chunk, sb, spar, sp, uz0) = args
    from multiprocessing import shared_memory
    bufs = [shared_memory.SharedMemory(name=nm) for nm in shm_names]
    try:
        views = _views(bufs, n_total, ndim)
        rng_b, rng_p = [np.random.default_rng(s) for s in
                        np.random.SeedSequence([seed, chunk]).spawn(2)]
        p0, p1 = c0 * ppc, c1 * ppc
        n = p1 - p0
        cells = np.repeat(np.arange(c0, c1, dtype=np.int32), ppc)
        for s, rng in ((0, rng_b), (1, rng_p)):
            cell, off, u = views[s]
            cell[p0:p1] = cells
            off[:, p0:p1] = rng.random((ndim, n), dtype=np.float32)
        cell, off, u = views[0]
        u[0, p0:p1] = rng_b.standard_normal(n, dtype=np.float32) * np.float32(sb) if sb > 0 else 0.0
        u[1, p0:p1] = rng_b.standard_normal(n, dtype=np.float32) * np.float32(sb) if sb > 0 else 0.0
        u[2, p0:p1] = np.float32(uz0) + (rng_b.standard_normal(n, dtype=np.float32) * np.float32(spar)
                                         if spar > 0 else np.float32(0.0))
        cell, off, u = views[1]
        for a in range(3):       # thermal parts; the drift is added to u_z afterwards
            u[a, p0:p1] = rng_p.standard_normal(n, dtype=np.float32) * np.float32(sp) if sp > 0 else 0.0
        # partial sums for the drift solve: beam current and nothing else
        ub = views[0][2][:, p0:p1].astype(np.float64)
        beam_v = float(np.sum(ub[2] / np.sqrt(1.0 + (ub * ub).sum(0))))
        del views, ub
        return beam_v
    finally:
        for b in bufs:
            b.close()


def _views(bufs, n_total, ndim):
    out = []
    for s in range(2):
        cell = np.ndarray((n_total,), np.int32, buffer=bufs[3 * s].buf)
        off = np.ndarray((ndim, n_total), np.float32, buffer=bufs[3 * s + 1].buf)
        u = np.ndarray((3, n_total), np.float32, buffer=bufs[3 * s + 2].buf)
        out.append((cell, off, u))
    return out


class SharedLoad:
    """A Workload whose particle arrays live in shared memory; close() releases them."""

    def __init__(self, workload, bufs):
        self.workload = workload
        self._bufs = bufs

    def close(self):
        self.workload = None
        for b in self._bufs:
            b.close()
            b.unlink()
        self._bufs = []


def weibel_load_parallel(*, ndim=2, nx, ny, nz=1, ppc, gamma_b=3.0, nb=0.1, T_perp_beam=0.0,
                         T_par_beam=0.0, T_bg=0.0, nu=0.0, seed=1, dx=0.1, dt=0.05, steps=0,
                         workers=8, name=None) -> SharedLoad:
    """weibel_load's distributions drawn by `workers` processes (spawned) into shared memory.

    The background drift that zeroes the sampled current sum_p w v_z is solved in FP64 over all
    particles after the draw, as in weibel_load."""
    import multiprocessing as mp
    from multiprocessing import shared_memory
    if ndim == 2:
        nz = 1
    ncell = nx * ny * nz
    n = ncell * ppc
    bufs = []
    for _ in range(2):
        bufs.append(shared_memory.SharedMemory(create=True, size=max(4 * n, 4)))
        bufs.append(shared_memory.SharedMemory(create=True, size=max(4 * ndim * n, 4)))
        bufs.append(shared_memory.SharedMemory(create=True, size=max(12 * n, 4)))
    try:
        nchunk = max(1, min(4 * workers, ncell))
        edges = np.linspace(0, ncell, nchunk + 1).astype(np.int64)
        uz0 = math.sqrt(gamma_b * gamma_b - 1.0)
        jobs = [([b.name for b in bufs], n, ndim, nx, ny, nz, ppc, int(edges[k]), int(edges[k + 1]),
                 seed, k, math.sqrt(T_perp_beam), math.sqrt(T_par_beam), math.sqrt(T_bg), uz0)
                for k in range(nchunk)]
        with mp.get_context("spawn").Pool(workers) as pool:
            beam_v = sum(pool.map(_chunk_fill, jobs))
        views = _views(bufs, n, ndim)
        wb, wp = nb / ppc, (1.0 - nb) / ppc
        ubg = views[1][2]
        duz = ubg[2].astype(np.float64)
        uperp2 = ubg[0].astype(np.float64) ** 2 + ubg[1].astype(np.float64) ** 2
        d = _solve_drift(-wb * beam_v / wp, duz, uperp2)
        del uperp2
        ubg[2][:] = (d + duz).astype(np.float32)
        del duz
        sp = [SpeciesLoad("beam", ELECTRON_Q, ELECTRON_M, wb, 0.0, *views[0]),
              SpeciesLoad("background", ELECTRON_Q, ELECTRON_M, wp, nu, *views[1])]
        if name is None:
            dims = f"{nx}x{ny}" + (f"x{nz}" if ndim == 3 else "")
            name = f"weibel_{ndim}d_{dims}_ppc{ppc}"
        return SharedLoad(Workload(name, ndim, nx, ny, nz, dx, dx, dx, dt, steps, sp), bufs)
    except BaseException:
        for b in bufs:
            b.close()
            b.unlink()
        raise


# ---------------------------------------------------------------- hybrid-model loads
@dataclass
class HybridLoad:
    """Initial state of the quasi-neutral hybrid model: beam particles at X, Y (cell units, FP64
    holding FP32-representable offsets, so an FP32 cell + offset copy is exact), momenta (FP64
    holding FP32 values), the beam density per particle w, and the initial plasma flow beta_p0
    that carries the return current (zero net current)."""
    name: str
    nx: int
    ny: int
    dx: float
    dt: float
    nu: float
    X: np.ndarray
    Y: np.ndarray
    ux: np.ndarray
    uy: np.ndarray
    uz: np.ndarray
    w: float
    beta_p0: float

    @property
    def n(self) -> int:
        return int(self.X.shape[0])


def hybrid_beam_load(*, nx, ny, ppc, gamma_b=3.0, nb=0.1, T_perp_beam=0.1, nu=0.1, dx=0.1,
                     dt=0.05, seed=6, name=None):
    """ppc beam particles per cell in cell order (x fastest), uniform in-cell offsets, transverse
    momenta ~ N(0, sqrt(T_perp_beam)), u_z = sqrt(gamma_b^2 - 1); beta_p0 = -nb <beta_z> / (1 - nb)."""
    rng = np.random.default_rng(seed)
    ncell = nx * ny
    cell = np.repeat(np.arange(ncell, dtype=np.int64), ppc)
    off = rng.random((2, cell.shape[0]), dtype=np.float32)
    X = (cell % nx).astype(np.float64) + off[0].astype(np.float64)
    Y = (cell // nx).astype(np.float64) + off[1].astype(np.float64)
    s = np.float32(math.sqrt(T_perp_beam))
    ux = (s * rng.standard_normal(cell.shape[0], dtype=np.float32)).astype(np.float64)
    uy = (s * rng.standard_normal(cell.shape[0], dtype=np.float32)).astype(np.float64)
    uz = np.full(cell.shape[0], float(np.float32(math.sqrt(gamma_b ** 2 - 1))))
    bz = uz / np.sqrt(1.0 + ux ** 2 + uy ** 2 + uz ** 2)
    return HybridLoad(name or f"hybrid_beam_2d_{nx}x{ny}_ppc{ppc}", nx, ny, dx, dt, nu, X, Y, ux, uy,
                      uz, nb / ppc, float(-nb * bz.mean() / (1.0 - nb)))
