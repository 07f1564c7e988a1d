"""FP64 CPU oracle of the Weibel PIC step -- TEST INFRASTRUCTURE ONLY.

Only the tests, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline leg may import
this package.  It shares no code with the CUDA library (``paper_0808_4078_gb300``) and never
imports it.  The arithmetic lives in ``pic_oracle.c`` (plain C, FP64, one particle at a time);
this module only marshals numpy arrays.

Functions and the passages they follow (arXiv:0808.4078):
  Simulation.step     -- one PIC step: 2D transverse-plane geometry and species of the
                         simulation section; collisional drag of Eq. (3) on the return current
                         (Krook reading); textbook CIC/Boris/Esirkepov/Yee discretisation.
  Simulation.diag     -- field energy per component, integral of F_i^2 dx dy (simulation
                         section), kinetic energy and momentum.
  theory.*            -- cold relativistic two-fluid filamentation growth rate (closed form);
                         canonical momentum, Eq. (6); warm threshold, Eq. (11); Eq. (12)-(14).
  fit.growth_rate     -- least-squares slope of ln W_B over the exponential phase (results
                         section: linear growth rates extracted from the simulations).
Every function above is pinned by ``tests/test_oracle_pins.py``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pic_oracle.c")
_SO = os.path.join(_HERE, "liboracle.so")
_SO_OMP = os.path.join(_HERE, "liboracle_omp.so")
_lib = None
_lib_omp = None

P = ctypes.POINTER(ctypes.c_double)


def build(force: bool = False) -> str:
    """Compile pic_oracle.c into oracle/liboracle.so with the host gcc (no -march flags), and
    the all-core variant (build_threads)."""
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC",
                               "-shared", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _SO)
    build_threads(force)
    return _SO


def build_threads(force: bool = False) -> str:
    """The same C with OpenMP (-O3 -fopenmp; no -march flags, so that it gives the same results
    on every host): the particle loop on all threads, each depositing into its own current and
    moment arrays.  Used to time the oracle on every host core; the tests' oracle is the
    single-threaded build."""
    if force or not os.path.exists(_SO_OMP) or os.path.getmtime(_SO_OMP) < os.path.getmtime(_SRC):
        tmp = _SO_OMP + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O3", "-std=c11", "-ffp-contract=off", "-fopenmp", "-fPIC",
                               "-shared", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _SO_OMP)
    return _SO_OMP


class _Grid(ctypes.Structure):
    _fields_ = [("ndim", ctypes.c_int), ("nx", ctypes.c_int), ("ny", ctypes.c_int),
                ("nz", ctypes.c_int), ("dx", ctypes.c_double), ("dy", ctypes.c_double),
                ("dz", ctypes.c_double), ("dt", ctypes.c_double),
                ("Ex", P), ("Ey", P), ("Ez", P), ("Bx", P), ("By", P), ("Bz", P),
                ("Jx", P), ("Jy", P), ("Jz", P), ("step", ctypes.c_int64), ("j_filter", ctypes.c_int)]


class _Species(ctypes.Structure):
    _fields_ = [("q", ctypes.c_double), ("m", ctypes.c_double), ("w", ctypes.c_double),
                ("nu", ctypes.c_double), ("n", ctypes.c_int64),
                ("X", P), ("Y", P), ("Z", P), ("ux", P), ("uy", P), ("uz", P), ("ubar", P),
                ("nu_cell", P), ("nu_coll", ctypes.c_double), ("seed", ctypes.c_uint64),
                ("index", ctypes.c_int32)]


MAX_SPECIES = 4


class _Diag(ctypes.Structure):
    _fields_ = [("WE", ctypes.c_double * 3), ("WB", ctypes.c_double * 3),
                ("Ekin", ctypes.c_double * MAX_SPECIES), ("P", ctypes.c_double * 3)]


def lib():
    global _lib
    if _lib is None:
        _lib = _bind(ctypes.CDLL(build()))
    return _lib


def lib_threads():
    """The all-core build (see build_threads)."""
    global _lib_omp
    if _lib_omp is None:
        build()
        _lib_omp = _bind(ctypes.CDLL(build_threads()))
    return _lib_omp


def _bind(L):
    """Argument types of the oracle library's entry points."""
    L.orc_step.argtypes = [ctypes.POINTER(_Grid), ctypes.POINTER(_Species), ctypes.c_int,
                           ctypes.POINTER(_Diag)]
    L.orc_step.restype = ctypes.c_int
    L.orc_moments.argtypes = [ctypes.POINTER(_Grid), ctypes.POINTER(_Species)]
    L.orc_moments.restype = ctypes.c_int
    L.orc_yee.argtypes = [ctypes.POINTER(_Grid)]
    L.orc_yee.restype = None
    L.orc_binomial.argtypes = [ctypes.POINTER(_Grid), P]
    L.orc_binomial.restype = None
    L.orc_rho.argtypes = [ctypes.POINTER(_Grid), ctypes.POINTER(_Species), ctypes.c_int, P]
    L.orc_rho.restype = None
    L.orc_gather.argtypes = [ctypes.POINTER(_Grid), ctypes.c_double, ctypes.c_double,
                             ctypes.c_double, P]
    L.orc_gather.restype = None
    L.orc_boris.argtypes = [ctypes.c_double, ctypes.c_double, P, P]
    L.orc_boris.restype = None
    L.orc_push_particle.argtypes = [ctypes.POINTER(_Grid), ctypes.c_double, ctypes.c_double,
                                       P, P, P, P, P]
    L.orc_push_particle.restype = None
    L.orc_deposit_move.argtypes = [ctypes.POINTER(_Grid), ctypes.c_double, P, P,
                                   ctypes.c_double]
    L.orc_deposit_move.restype = None
    L.orc_gather_many.argtypes = [ctypes.POINTER(_Grid), ctypes.c_int64, P, P, P, P]
    L.orc_gather_many.restype = None
    U32 = ctypes.POINTER(ctypes.c_uint32)
    L.orc_philox4x32_10.argtypes = [U32, U32, U32]
    L.orc_philox4x32_10.restype = None
    L.orc_collide_ion.argtypes = [P, ctypes.c_double, U32]
    L.orc_collide_ion.restype = None
    return L


def _ptr(a):
    return a.ctypes.data_as(P) if a is not None else None


class Species:
    """One species' FP64 state: positions X, Y(, Z) in cell units, momenta u = gamma v / c."""

    def __init__(self, q, m, w, nu, X, Y, Z, ux, uy, uz, ncell, name=""):
        f = lambda a: np.ascontiguousarray(a, dtype=np.float64)
        self.name = name
        self.q, self.m, self.w, self.nu = float(q), float(m), float(w), float(nu)
        self.X, self.Y = f(X), f(Y)
        self.Z = f(Z) if Z is not None else np.zeros(1)
        self.ux, self.uy, self.uz = f(ux), f(uy), f(uz)
        self.ubar = np.zeros(3 * ncell) if nu > 0 else None
        self.nu_cell = None
        self.nu_coll = 0.0
        self.seed = 0
        self.index = 0

    @property
    def n(self):
        return self.X.shape[0]

    def cstruct(self):
        return _Species(self.q, self.m, self.w, self.nu, self.n, _ptr(self.X), _ptr(self.Y),
                        _ptr(self.Z), _ptr(self.ux), _ptr(self.uy), _ptr(self.uz),
                        _ptr(self.ubar), _ptr(self.nu_cell), self.nu_coll, self.seed, self.index)

    @property
    def u(self):
        return np.stack([self.ux, self.uy, self.uz])


class Simulation:
    """Grid + species, advanced by the C oracle one step at a time."""

    def __init__(self, ndim, nx, ny, nz=1, dx=0.1, dy=None, dz=None, dt=0.05, j_filter=0, threads=False):
        self.ndim, self.nx, self.ny = ndim, nx, ny
        self.threads = bool(threads)    # step with the all-core build (timing only)
        self.j_filter = int(j_filter)   # 1: binomial pass per axis on J before the field update
        self.nz = nz if ndim == 3 else 1
        self.dx = dx
        self.dy = dx if dy is None else dy
        self.dz = dx if dz is None else dz
        self.dt = dt
        shape = (self.nz, ny, nx) if ndim == 3 else (ny, nx)
        self.E = [np.zeros(shape) for _ in range(3)]
        self.B = [np.zeros(shape) for _ in range(3)]
        self.J = [np.zeros(shape) for _ in range(3)]
        self.species: list[Species] = []
        self.step_index = 0
        self.history: list[dict] = []

    @property
    def ncell(self):
        return self.nx * self.ny * self.nz

    def cgrid(self):
        E, B, J = self.E, self.B, self.J
        return _Grid(self.ndim, self.nx, self.ny, self.nz, self.dx, self.dy, self.dz, self.dt,
                     _ptr(E[0]), _ptr(E[1]), _ptr(E[2]), _ptr(B[0]), _ptr(B[1]), _ptr(B[2]),
                     _ptr(J[0]), _ptr(J[1]), _ptr(J[2]), self.step_index, self.j_filter)

    def add_species(self, q, m, w, nu, X, Y, Z, ux, uy, uz, name=""):
        s = Species(q, m, w, nu, X, Y, Z if self.ndim == 3 else None, ux, uy, uz, self.ncell, name)
        self.species.append(s)
        if s.ubar is not None:
            g = self.cgrid()
            cs = s.cstruct()
            if lib().orc_moments(ctypes.byref(g), ctypes.byref(cs)) != 0:
                raise MemoryError("orc_moments")
        return s

    def set_collisions(self, s, nu, seed):
        """Binary electron-ion collisions of species s at momentum-transfer rate nu, draws keyed
        by `seed` (64-bit), the particle index and the step (Takizuka & Abe, immobile ions)."""
        sp = self.species[s]
        sp.nu_coll = float(nu)
        sp.seed = int(seed) & 0xFFFFFFFFFFFFFFFF
        sp.index = s

    def set_nu_cell(self, s, nu_cell):
        """Per-cell Krook rates for species s (closure-driven drag; None restores the scalar
        rate).  Starts the cell-mean momentum tracking if the species had none."""
        sp = self.species[s]
        if nu_cell is None:
            sp.nu_cell = None
            return
        sp.nu_cell = np.ascontiguousarray(nu_cell, dtype=np.float64).reshape(-1)
        assert sp.nu_cell.shape[0] == self.ncell
        if sp.ubar is None:
            sp.ubar = np.zeros(3 * self.ncell)
            g = self.cgrid()
            cs = sp.cstruct()
            if lib().orc_moments(ctypes.byref(g), ctypes.byref(cs)) != 0:
                raise MemoryError("orc_moments")

    @classmethod
    def from_workload(cls, wl, j_filter=0, threads=False):
        """Build from a pic_inputs.Workload: X = cell index + FP32 offset, exactly, in FP64."""
        sim = cls(wl.ndim, wl.nx, wl.ny, wl.nz, wl.dx, wl.dy, wl.dz, wl.dt, j_filter=j_filter,
                  threads=threads)
        for s in wl.species:
            i = (s.cell % wl.nx).astype(np.float64)
            j = ((s.cell // wl.nx) % wl.ny).astype(np.float64)
            X = i + s.offset[0].astype(np.float64)
            Y = j + s.offset[1].astype(np.float64)
            Z = None
            if wl.ndim == 3:
                k = (s.cell // (wl.nx * wl.ny)).astype(np.float64)
                Z = k + s.offset[2].astype(np.float64)
            u = s.u.astype(np.float64)
            sim.add_species(s.q, s.m, s.w, s.nu, X, Y, Z, u[0], u[1], u[2], name=s.name)
        return sim

    def step(self, n=1, record=True):
        L = lib_threads() if self.threads else lib()
        g = self.cgrid()
        arr = (_Species * len(self.species))(*[s.cstruct() for s in self.species])
        for _ in range(n):
            d = _Diag()
            g.step = self.step_index          # keys this step's collision draws
            rc = L.orc_step(ctypes.byref(g), arr, len(self.species), ctypes.byref(d) if record else None)
            if rc != 0:
                raise RuntimeError(f"orc_step failed ({rc})")
            if record:
                self.history.append(dict(step=self.step_index, t=self.step_index * self.dt,
                                         WE=list(d.WE), WB=list(d.WB),
                                         Ekin=list(d.Ekin)[:len(self.species)], P=list(d.P)))
            self.step_index += 1

    def rho(self):
        out = np.zeros(self.E[0].shape)
        g = self.cgrid()
        arr = (_Species * len(self.species))(*[s.cstruct() for s in self.species])
        lib().orc_rho(ctypes.byref(g), arr, len(self.species), _ptr(out))
        return out

    def yee(self):
        g = self.cgrid()
        lib().orc_yee(ctypes.byref(g))

    def binomial(self, F):
        """One 1-2-1 pass per axis of a grid array (copy), as applied to J when j_filter is on."""
        out = np.ascontiguousarray(F, dtype=np.float64).copy()
        assert out.size == self.ncell
        lib().orc_binomial(ctypes.byref(self.cgrid()), _ptr(out))
        return out

    def gather(self, X, Y, Z=0.0):
        out = np.zeros(6)
        g = self.cgrid()
        lib().orc_gather(ctypes.byref(g), X, Y, Z, _ptr(out))
        return out

    def gather_many(self, X, Y, Z=None):
        """E and B (n x 6) at the positions X, Y(, Z) in cell units, one orc_gather each."""
        X = np.ascontiguousarray(X, dtype=np.float64)
        Y = np.ascontiguousarray(Y, dtype=np.float64)
        Zp = None
        if Z is not None and self.ndim == 3:
            Z = np.ascontiguousarray(Z, dtype=np.float64)
            Zp = _ptr(Z)
        out = np.zeros((X.shape[0], 6))
        g = self.cgrid()
        lib().orc_gather_many(ctypes.byref(g), ctypes.c_int64(X.shape[0]), _ptr(X), _ptr(Y), Zp,
                              _ptr(out))
        return out

    def deposit_move(self, qw, P0, P1, vz=0.0):
        g = self.cgrid()
        a = np.ascontiguousarray(P0, dtype=np.float64)
        b = np.ascontiguousarray(P1, dtype=np.float64)
        lib().orc_deposit_move(ctypes.byref(g), qw, _ptr(a), _ptr(b), vz)

    def push_particle(self, qm, nu, X, Y, Z, u, ubar_c=None):
        """One particle's gather/Boris/drag/move in the current fields; returns (X, Y, Z, u)."""
        x = np.array([X], dtype=np.float64)
        y = np.array([Y], dtype=np.float64)
        z = np.array([Z], dtype=np.float64)
        uu = np.ascontiguousarray(u, dtype=np.float64).copy()
        ub = None if ubar_c is None else np.ascontiguousarray(ubar_c, dtype=np.float64)
        g = self.cgrid()
        lib().orc_push_particle(ctypes.byref(g), qm, nu, _ptr(x), _ptr(y), _ptr(z), _ptr(uu),
                                _ptr(ub))
        return x[0], y[0], z[0], uu

    def history_array(self, key, comp=None):
        if comp is None:
            return np.array([h[key] for h in self.history])
        return np.array([h[key][comp] for h in self.history])


def boris(qm, dt, EB, u):
    """Single relativistic Boris update of u under the 6 field values EB."""
    e = np.ascontiguousarray(EB, dtype=np.float64)
    uu = np.ascontiguousarray(u, dtype=np.float64).copy()
    lib().orc_boris(qm, dt, _ptr(e), _ptr(uu))
    return uu


def philox4x32_10(ctr, key):
    """Philox4x32-10 of four 32-bit counter words and two key words (oracle C)."""
    c = (ctypes.c_uint32 * 4)(*[int(x) & 0xFFFFFFFF for x in ctr])
    k = (ctypes.c_uint32 * 2)(*[int(x) & 0xFFFFFFFF for x in key])
    o = (ctypes.c_uint32 * 4)()
    lib().orc_philox4x32_10(c, k, o)
    return list(o)


def collide_ion(u, sigma, r):
    """One binary electron-ion collision of momentum u (3,) with draws r (4 uint32)."""
    uu = np.ascontiguousarray(u, dtype=np.float64).copy()
    rr = (ctypes.c_uint32 * 4)(*[int(x) & 0xFFFFFFFF for x in r])
    lib().orc_collide_ion(_ptr(uu), float(sigma), rr)
    return uu
