"""Python binding of libpic (include/pic.h): argument marshalling only.

Every step of the particle-in-cell path runs in the CUDA kernels of libpic.so; PyTorch only
provides the device arena (one uint8 tensor) and the CUDA stream.  There is no CPU fallback:
if libpic.so is missing or no GPU is present, the calls raise.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
# PIC_DEBUG_BOUNDS=1 selects the bounds-checked build (build.build(debug=True))
LIB_PATH = os.path.join(_HERE, "libpic_debug.so" if os.environ.get("PIC_DEBUG_BOUNDS") == "1" else "libpic.so")
_lib = None

PIC_MAX_SPECIES = 2
PIC_FLAG_PROFILE = 1
PIC_FLAG_NO_GRAPH = 2
PIC_FLAG_KEEP_J = 4
PIC_FLAG_NVTX = 8

ERRORS = {0: "PIC_OK", -1: "PIC_EINVAL", -2: "PIC_ENOMEM", -3: "PIC_ECUDA", -4: "PIC_EOVERFLOW",
          -5: "PIC_EBADPART", -6: "PIC_ETIMEOUT", -7: "PIC_ESTATE", -8: "PIC_EBOUNDS"}


class PicError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{ERRORS.get(code, code)}: {msg}")
        self.code = code


class Config(ctypes.Structure):
    _fields_ = [("ndim", ctypes.c_int32), ("nx", ctypes.c_int32), ("ny", ctypes.c_int32),
                ("nz", ctypes.c_int32), ("dx", ctypes.c_double), ("dy", ctypes.c_double),
                ("dz", ctypes.c_double), ("dt", ctypes.c_double), ("nspecies", ctypes.c_int32),
                ("capacity", ctypes.c_int64 * PIC_MAX_SPECIES),
                ("cell_capacity", ctypes.c_int32 * PIC_MAX_SPECIES), ("sort_interval", ctypes.c_int32),
                ("diag_interval", ctypes.c_int32), ("diag_capacity", ctypes.c_int32),
                ("track_ids", ctypes.c_int32), ("flags", ctypes.c_int32),
                ("tile_x", ctypes.c_int32), ("tile_y", ctypes.c_int32), ("tile_z", ctypes.c_int32),
                ("j_filter", ctypes.c_int32), ("ctas_per_sm", ctypes.c_int32)]


class TuneEntry(ctypes.Structure):
    _fields_ = [("tile_x", ctypes.c_int32), ("tile_y", ctypes.c_int32), ("ctas_per_sm", ctypes.c_int32),
                ("ms_per_step", ctypes.c_float)]


def set_tune_cache(path):
    """Tuning-cache file of the autotuner (pic_tune_cache_set); None: memory only."""
    _check(lib().pic_tune_cache_set(None if path is None else os.fsencode(path)))


class Species(ctypes.Structure):
    _fields_ = [("q", ctypes.c_double), ("m", ctypes.c_double), ("w", ctypes.c_double),
                ("nu", ctypes.c_double)]


class DiagRec(ctypes.Structure):
    _fields_ = [("step", ctypes.c_int64), ("t", ctypes.c_double), ("WE", ctypes.c_double * 3),
                ("WB", ctypes.c_double * 3), ("Ekin", ctypes.c_double * PIC_MAX_SPECIES),
                ("P", ctypes.c_double * 3), ("flags", ctypes.c_int32), ("reserved", ctypes.c_int32)]


class Stats(ctypes.Structure):
    _fields_ = [("particles", ctypes.c_int64 * PIC_MAX_SPECIES),
                ("max_cell", ctypes.c_int32 * PIC_MAX_SPECIES),
                ("spilled", ctypes.c_int32 * PIC_MAX_SPECIES),
                ("cell_capacity", ctypes.c_int32 * PIC_MAX_SPECIES),
                ("flags", ctypes.c_int32), ("reserved", ctypes.c_int32)]


class KernelTime(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 32), ("launches", ctypes.c_int64),
                ("total_ms", ctypes.c_double)]


class HybridConfig(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("dx", ctypes.c_double),
                ("dy", ctypes.c_double), ("dt", ctypes.c_double), ("n0", ctypes.c_double),
                ("nu", ctypes.c_double), ("w", ctypes.c_double), ("capacity", ctypes.c_int64),
                ("tol", ctypes.c_double), ("max_iter", ctypes.c_int32), ("flags", ctypes.c_int32),
                ("sort_interval", ctypes.c_int32)]


class MlpNorm(ctypes.Structure):
    _fields_ = [("mu", ctypes.c_float * 9), ("sigma", ctypes.c_float * 9), ("nin", ctypes.c_int32)]


_VP = ctypes.c_void_p
_SIGNATURES = {
    "pic_required_bytes": (ctypes.c_int, [ctypes.POINTER(Config), ctypes.POINTER(ctypes.c_size_t)]),
    "pic_init": (ctypes.c_int, [ctypes.POINTER(Config), _VP, ctypes.c_size_t, _VP, ctypes.POINTER(_VP)]),
    "pic_load_species": (ctypes.c_int, [_VP, ctypes.c_int, ctypes.POINTER(Species), ctypes.c_int64,
                                        _VP, _VP, _VP]),
    "pic_required_bytes_batch": (ctypes.c_int, [ctypes.POINTER(Config), ctypes.c_int, _VP, _VP,
                                                ctypes.POINTER(ctypes.c_size_t)]),
    "pic_init_batch": (ctypes.c_int, [ctypes.POINTER(Config), ctypes.c_int, _VP, _VP, _VP, ctypes.c_size_t,
                                      _VP, ctypes.POINTER(_VP)]),
    "pic_num_runs": (ctypes.c_int, [_VP]),
    "pic_load_species_run": (ctypes.c_int, [_VP, ctypes.c_int, ctypes.c_int, ctypes.POINTER(Species),
                                            ctypes.c_int64, _VP, _VP, _VP]),
    "pic_diag_run": (ctypes.c_int, [_VP, ctypes.c_int, _VP, ctypes.c_int, ctypes.POINTER(ctypes.c_int)]),
    "pic_get_particles_run": (ctypes.c_int, [_VP, ctypes.c_int, ctypes.c_int, _VP, _VP, _VP, _VP,
                                             ctypes.c_int64]),
    "pic_get_fields_run": (ctypes.c_int, [_VP, ctypes.c_int, _VP, _VP, _VP]),
    "pic_fit_growth_run": (ctypes.c_int, [_VP, ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                          ctypes.c_double, ctypes.POINTER(ctypes.c_double),
                                          ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)]),
    "pic_step": (ctypes.c_int, [_VP, ctypes.c_int]),
    "pic_sync": (ctypes.c_int, [_VP]),
    "pic_clear_flags": (ctypes.c_int, [_VP, _VP]),
    "pic_diag": (ctypes.c_int, [_VP, _VP, ctypes.c_int, ctypes.POINTER(ctypes.c_int)]),
    "pic_get_particles": (ctypes.c_int, [_VP, ctypes.c_int, _VP, _VP, _VP, _VP, ctypes.c_int64]),
    "pic_get_fields": (ctypes.c_int, [_VP, _VP, _VP, _VP]),
    "pic_set_fields": (ctypes.c_int, [_VP, _VP, _VP]),
    "pic_fixed_point_shift": (ctypes.c_int, [_VP, ctypes.POINTER(ctypes.c_int)]),
    "pic_fit_growth": (ctypes.c_int, [_VP, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                      ctypes.c_double, ctypes.POINTER(ctypes.c_double),
                                      ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)]),
    "pic_kernel_times": (ctypes.c_int, [_VP, _VP, ctypes.c_int, ctypes.POINTER(ctypes.c_int)]),
    "pic_get_stats": (ctypes.c_int, [_VP, ctypes.POINTER(Stats)]),
    "pic_bin_cells_scratch_bytes": (ctypes.c_int, [ctypes.c_int32, ctypes.POINTER(ctypes.c_size_t)]),
    "pic_bin_cells": (ctypes.c_int, [_VP, ctypes.c_int64, ctypes.c_int32, _VP, _VP, _VP, ctypes.c_size_t, _VP]),
    "pic_record_moments_scratch_bytes": (ctypes.c_int, [_VP, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                                        ctypes.POINTER(ctypes.c_size_t)]),
    "pic_record_moments": (ctypes.c_int, [_VP, ctypes.c_int, ctypes.c_int, ctypes.c_int, _VP, ctypes.c_int64,
                                          _VP, ctypes.c_size_t, ctypes.POINTER(ctypes.c_int64)]),
    "pic_mlp_forward": (ctypes.c_int, [_VP, ctypes.POINTER(MlpNorm), _VP, ctypes.c_int64, ctypes.c_int64, _VP, _VP]),
    "pic_mlp_train_scratch_bytes": (ctypes.c_int, [ctypes.POINTER(ctypes.c_size_t)]),
    "pic_mlp_train_step": (ctypes.c_int, [_VP, _VP, _VP, ctypes.c_int32, ctypes.c_float, ctypes.POINTER(MlpNorm),
                                          _VP, ctypes.c_int64, _VP, ctypes.c_int64, _VP, _VP, ctypes.c_size_t, _VP]),
    "pic_mlp_status": (ctypes.c_int, [ctypes.c_int]),
    "pic_mlp_wait_test": (ctypes.c_int, [ctypes.c_int64, _VP]),
    "pic_autotune": (ctypes.c_int, [_VP, ctypes.c_int, _VP, ctypes.c_int, _VP]),
    "pic_tune_cache_set": (ctypes.c_int, [ctypes.c_char_p]),
    "pic_tile_config": (ctypes.c_int, [_VP, _VP]),
    "pic_mlp_fit_norm": (ctypes.c_int, [_VP, ctypes.c_int64, ctypes.c_int64, ctypes.c_int32, _VP, _VP]),
    "pic_closure_samples_scratch_bytes": (ctypes.c_int, [ctypes.c_int64, _VP]),
    "pic_closure_samples": (ctypes.c_int, [_VP, ctypes.c_int32, ctypes.c_int64, ctypes.c_int32, ctypes.c_float,
                                           ctypes.c_float, _VP, _VP, ctypes.c_int64, _VP, _VP, ctypes.c_size_t,
                                           _VP]),
    "pic_set_drag_map": (ctypes.c_int, [_VP, ctypes.c_int, ctypes.c_int, _VP, ctypes.c_int32, ctypes.c_int32]),
    "pic_set_collisions": (ctypes.c_int, [_VP, ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_uint64]),
    "pic_dispersion_growth": (ctypes.c_int, [_VP, ctypes.c_int32, ctypes.c_double, ctypes.c_double,
                                             ctypes.c_int32, _VP, _VP, _VP]),
    "pic_hybrid_required_bytes": (ctypes.c_int, [ctypes.POINTER(HybridConfig), ctypes.POINTER(ctypes.c_size_t)]),
    "pic_hybrid_init": (ctypes.c_int, [ctypes.POINTER(HybridConfig), _VP, ctypes.c_size_t, _VP, ctypes.POINTER(_VP)]),
    "pic_hybrid_load": (ctypes.c_int, [_VP, ctypes.c_int64, _VP, _VP, _VP, _VP, _VP, _VP]),
    "pic_hybrid_step": (ctypes.c_int, [_VP, ctypes.c_int]),
    "pic_hybrid_get": (ctypes.c_int, [_VP, _VP, _VP, _VP, _VP, _VP, _VP]),
    "pic_hybrid_energies": (ctypes.c_int, [_VP, _VP]),
    "pic_hybrid_stats": (ctypes.c_int, [_VP, _VP]),
    "pic_hybrid_kernel_times": (ctypes.c_int, [_VP, _VP, ctypes.c_int, ctypes.POINTER(ctypes.c_int)]),
    "pic_hybrid_launch_count": (ctypes.c_int64, [_VP]),
    "pic_hybrid_step_count": (ctypes.c_int64, [_VP]),
    "pic_hybrid_free": (None, [_VP]),
    "pic_checkpoint": (ctypes.c_int, [_VP, ctypes.c_char_p]),
    "pic_restore": (ctypes.c_int, [_VP, ctypes.c_char_p]),
    "pic_loaded_count": (ctypes.c_int64, [_VP, ctypes.c_int, ctypes.c_int]),
    "pic_launch_count": (ctypes.c_int64, [_VP]),
    "pic_step_count": (ctypes.c_int64, [_VP]),
    "pic_last_error": (ctypes.c_char_p, [_VP]),
    "pic_free": (None, [_VP]),
}


PIC_MOM_ROWS = 12
MOMENT_ROWS = ("n_b", "n_p", "uz_b", "uz_p", "Tperp_b", "Tpar_b", "Tperp_p", "Tpar_p", "W_ES",
               "Fz_p", "Fz_mean", "nu_eff")


def lib():
    """Load libpic.so (raises if it has not been built: there is no fallback)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{os.path.basename(LIB_PATH)} not built ({LIB_PATH}); run __graft_entry__.build()")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in _SIGNATURES.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(_VP)


def _check(rc, ctx=None):
    if rc != 0:
        msg = lib().pic_last_error(ctx).decode(errors="replace")
        raise PicError(rc, msg)


def required_bytes(cfg: Config) -> int:
    n = ctypes.c_size_t(0)
    _check(lib().pic_required_bytes(ctypes.byref(cfg), ctypes.byref(n)))
    return n.value


class Engine:
    """One PIC run, or a batch of independent runs (``runs=``), on one GPU.  Arena and stream
    come from PyTorch.  runs: list of (nx, ny, nz, (capacity_species0, capacity_species1))."""

    def __init__(self, ndim, nx=16, ny=16, nz=1, dx=0.1, dy=None, dz=None, dt=0.05, capacity=(0, 0),
                 nspecies=2, sort_interval=8, diag_interval=1, diag_capacity=4096,
                 track_ids=False, flags=0, device="cuda", stream=None, cell_capacity=(0, 0),
                 runs=None, j_filter=0, tile=(0, 0), ctas_per_sm=0):
        import torch
        self._torch = torch
        if not torch.cuda.is_available():
            raise RuntimeError("libpic needs a CUDA GPU")
        cap = (ctypes.c_int64 * PIC_MAX_SPECIES)(*[int(c) for c in capacity][:PIC_MAX_SPECIES])
        ccap = (ctypes.c_int32 * PIC_MAX_SPECIES)(*[int(c) for c in cell_capacity][:PIC_MAX_SPECIES])
        self.cfg = Config(ndim, nx, ny, nz if ndim == 3 else 1, dx, dx if dy is None else dy,
                          dx if dz is None else dz, dt, nspecies, cap, ccap, sort_interval,
                          diag_interval, diag_capacity, int(bool(track_ids)), flags,
                          int(tile[0]), int(tile[1]), 0, int(j_filter), int(ctas_per_sm))
        if runs is None:
            runs = [(nx, ny, nz if ndim == 3 else 1, tuple(capacity))]
        self.runs = [(int(a), int(b), int(c) if ndim == 3 else 1, tuple(int(x) for x in k))
                     for a, b, c, k in runs]
        nr = len(self.runs)
        self._dims = np.array([[a, b, c] for a, b, c, _ in self.runs], dtype=np.int32).reshape(-1)
        capa = np.zeros((nr, PIC_MAX_SPECIES), dtype=np.int64)
        for r, (_, _, _, k) in enumerate(self.runs):
            capa[r, :len(k)] = k[:PIC_MAX_SPECIES]
        self._caps = capa.reshape(-1)
        n = ctypes.c_size_t(0)
        _check(lib().pic_required_bytes_batch(ctypes.byref(self.cfg), nr, _ptr(self._dims),
                                              _ptr(self._caps), ctypes.byref(n)))
        self.nbytes = n.value
        self.device = torch.device(device)
        self.arena = torch.empty(self.nbytes, dtype=torch.uint8, device=self.device)
        self.stream = stream if stream is not None else torch.cuda.Stream(self.device)
        self._ctx = _VP()
        with torch.cuda.device(self.device):
            _check(lib().pic_init_batch(ctypes.byref(self.cfg), nr, _ptr(self._dims), _ptr(self._caps),
                                        _VP(self.arena.data_ptr()), self.nbytes,
                                        _VP(self.stream.cuda_stream), ctypes.byref(self._ctx)))
        self.loaded = [[0] * PIC_MAX_SPECIES for _ in range(nr)]
        self.ncells = [a * b * c for a, b, c, _ in self.runs]
        self.ncell = self.ncells[0]

    # -------------------------------------------------------------- lifecycle
    def close(self):
        if getattr(self, "_ctx", None) and self._ctx.value:
            lib().pic_free(self._ctx)
            self._ctx = _VP()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # -------------------------------------------------------------- calls
    def load_species(self, s, q, m, w, nu, cell, offset, u, run=0):
        cell = np.ascontiguousarray(cell, dtype=np.int32)
        offset = np.ascontiguousarray(offset, dtype=np.float32)
        u = np.ascontiguousarray(u, dtype=np.float32)
        n = cell.shape[0]
        assert offset.shape == (self.cfg.ndim, n) and u.shape == (3, n)
        sp = Species(q, m, w, nu)
        _check(lib().pic_load_species_run(self._ctx, run, s, ctypes.byref(sp), n, _ptr(cell),
                                          _ptr(offset), _ptr(u)), self._ctx)
        self.loaded[run][s] = n

    def step(self, n=1):
        _check(lib().pic_step(self._ctx, int(n)), self._ctx)

    def sync(self):
        _check(lib().pic_sync(self._ctx), self._ctx)

    def autotune(self, steps_per_variant=16):
        """Time every compiled variant of the particle kernel on the next steps of this run and
        keep the fastest (pic_autotune); returns [(tile_x, tile_y, ctas_per_sm, ms_per_step)]."""
        buf = (TuneEntry * 16)()
        n = ctypes.c_int(0)
        _check(lib().pic_autotune(self._ctx, int(steps_per_variant), ctypes.cast(buf, _VP), 16,
                                  ctypes.byref(n)), self._ctx)
        return [(e.tile_x, e.tile_y, e.ctas_per_sm, e.ms_per_step) for e in buf[:n.value]]

    def tile_config(self):
        """(tile_x, tile_y, ctas_per_sm) of the particle kernel ((tile_x, tile_y, tile_z) in 3D)."""
        out = (ctypes.c_int32 * 3)()
        _check(lib().pic_tile_config(self._ctx, ctypes.cast(out, _VP)), self._ctx)
        return tuple(out)

    def clear_flags(self):
        """Sticky device error bits (PIC_FLAG_BIT_*), cleared."""
        f = ctypes.c_int32(0)
        _check(lib().pic_clear_flags(self._ctx, ctypes.byref(f)), self._ctx)
        return f.value

    def diag(self, max_recs=None, run=0):
        cap = self.cfg.diag_capacity if max_recs is None else max_recs
        buf = (DiagRec * cap)()
        n = ctypes.c_int(0)
        _check(lib().pic_diag_run(self._ctx, run, ctypes.cast(buf, _VP), cap, ctypes.byref(n)),
               self._ctx)
        out = []
        for r in buf[:n.value]:
            out.append(dict(step=r.step, t=r.t, WE=list(r.WE), WB=list(r.WB), Ekin=list(r.Ekin),
                            P=list(r.P), flags=r.flags))
        return out

    def particles(self, s, run=0):
        n = self.loaded[run][s]
        cell = np.empty(n, np.int32)
        off = np.empty((self.cfg.ndim, n), np.float32)
        u = np.empty((3, n), np.float32)
        ids = np.empty(n, np.int32) if self.cfg.track_ids else None
        _check(lib().pic_get_particles_run(self._ctx, run, s, _ptr(cell), _ptr(off), _ptr(u),
                                           _ptr(ids), n), self._ctx)
        return cell, off, u, ids

    def fields(self, with_J=False, run=0):
        shape = (3, self.ncells[run])
        E = np.empty(shape, np.float32)
        B = np.empty(shape, np.float32)
        J = np.empty(shape, np.int64) if with_J else None
        _check(lib().pic_get_fields_run(self._ctx, run, _ptr(E), _ptr(B), _ptr(J)), self._ctx)
        return E, B, J

    def set_fields(self, E=None, B=None):
        E = None if E is None else np.ascontiguousarray(E, dtype=np.float32)
        B = None if B is None else np.ascontiguousarray(B, dtype=np.float32)
        _check(lib().pic_set_fields(self._ctx, _ptr(E), _ptr(B)), self._ctx)

    def fixed_point_shift(self):
        s = ctypes.c_int(0)
        _check(lib().pic_fixed_point_shift(self._ctx, ctypes.byref(s)), self._ctx)
        return s.value

    def fit_growth(self, width=60, t_noise=2.0, start_factor=10.0, end_factor=1.0 / 30.0, run=0):
        g, t0, t1 = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
        ef = -1.0 if end_factor is None else end_factor
        _check(lib().pic_fit_growth_run(self._ctx, run, width, t_noise, start_factor, ef,
                                        ctypes.byref(g), ctypes.byref(t0), ctypes.byref(t1)),
               self._ctx)
        return g.value, t0.value, t1.value

    def kernel_times(self):
        buf = (KernelTime * 16)()
        n = ctypes.c_int(0)
        _check(lib().pic_kernel_times(self._ctx, ctypes.cast(buf, _VP), 16, ctypes.byref(n)),
               self._ctx)
        return {b.name.decode(): (b.launches, b.total_ms) for b in buf[:n.value]}

    def stats(self):
        """pic_get_stats: particles held, the largest binning-unit count (2D: a cell; 3D: a tile of
        the 3D particle kernel), spilled particles and slots per unit, per species; sticky flags."""
        st = Stats()
        _check(lib().pic_get_stats(self._ctx, ctypes.byref(st)), self._ctx)
        n = self.cfg.nspecies
        return dict(particles=list(st.particles)[:n], max_cell=list(st.max_cell)[:n],
                    spilled=list(st.spilled)[:n], cell_capacity=list(st.cell_capacity)[:n],
                    flags=st.flags)

    def record_moments(self, bx=4, by=4, run=0, out=None):
        """Coarse-grained closure moments (pic_record_moments): a (PIC_MOM_ROWS, ncoarse) float32
        tensor on the engine's device (written into `out` if given), rows MOMENT_ROWS."""
        torch = self._torch
        nb = ctypes.c_size_t(0)
        _check(lib().pic_record_moments_scratch_bytes(self._ctx, run, bx, by, ctypes.byref(nb)), self._ctx)
        nx, ny = self.runs[run][0], self.runs[run][1]
        nc = (nx // bx) * (ny // by)
        if out is None:
            out = torch.empty((PIC_MOM_ROWS, nc), dtype=torch.float32, device=self.device)
        scratch = torch.empty(nb.value, dtype=torch.uint8, device=self.device)
        n = ctypes.c_int64(0)
        _check(lib().pic_record_moments(self._ctx, run, bx, by, _VP(out.data_ptr()), out.numel(),
                                        _VP(scratch.data_ptr()), nb.value, ctypes.byref(n)), self._ctx)
        # the scratch tensor is released when this returns: let the stream finish with it first
        self.sync()
        return out

    def set_collisions(self, s, nu, seed, run=0):
        """Binary electron-ion collisions of species s at rate nu (pic_set_collisions)."""
        _check(lib().pic_set_collisions(self._ctx, run, s, float(nu), int(seed) & 0xFFFFFFFFFFFFFFFF), self._ctx)

    def set_drag_map(self, s, nu, bx=1, by=1, run=0):
        """Per-coarse-cell Krook rates (CUDA float tensor of (nx/bx)(ny/by) values) for species s,
        or None to restore its scalar rate (pic_set_drag_map)."""
        if nu is None:
            _check(lib().pic_set_drag_map(self._ctx, run, s, None, bx, by), self._ctx)
            return
        nu = nu.contiguous()
        self._torch.cuda.current_stream(self.device).synchronize()
        _check(lib().pic_set_drag_map(self._ctx, run, s, _VP(nu.data_ptr()), bx, by), self._ctx)

    def checkpoint(self, path):
        """Write the whole run state to `path` (pic_checkpoint)."""
        _check(lib().pic_checkpoint(self._ctx, os.fsencode(path)), self._ctx)

    def restore(self, path):
        """Replace this engine's state by a checkpoint of the same configuration (pic_restore)."""
        _check(lib().pic_restore(self._ctx, os.fsencode(path)), self._ctx)
        for r in range(len(self.runs)):
            for s in range(PIC_MAX_SPECIES):
                self.loaded[r][s] = int(lib().pic_loaded_count(self._ctx, r, s))

    def launch_count(self):
        return int(lib().pic_launch_count(self._ctx))

    def step_count(self):
        return int(lib().pic_step_count(self._ctx))

    # -------------------------------------------------------------- helpers
    @classmethod
    def from_workload(cls, wl, **kw):
        """Engine sized for a pic_inputs.Workload, with its species loaded."""
        return cls.from_workloads([wl], **kw)

    @classmethod
    def from_workloads(cls, wls, **kw):
        """One batched engine holding every workload as a run (same ndim, dx, dt, species)."""
        w0 = wls[0]
        runs = []
        for wl in wls:
            assert (wl.ndim, wl.dx, wl.dt, len(wl.species)) == (w0.ndim, w0.dx, w0.dt, len(w0.species))
            cap = [s.n for s in wl.species] + [0] * (PIC_MAX_SPECIES - len(wl.species))
            runs.append((wl.nx, wl.ny, wl.nz, tuple(cap)))
        eng = cls(w0.ndim, dx=w0.dx, dy=w0.dy, dz=w0.dz, dt=w0.dt, nspecies=len(w0.species),
                  runs=runs, **kw)
        for r, wl in enumerate(wls):
            for i, s in enumerate(wl.species):
                eng.load_species(i, s.q, s.m, s.w, s.nu, s.cell, s.offset, s.u, run=r)
        return eng


def bin_cells(cell, ncell, stream=None):
    """Counting sort by cell on the GPU (pic_bin_cells): cell is an int32 CUDA tensor; returns
    (start[ncell + 1], order[n]) int32 CUDA tensors.  Scratch is a torch allocation."""
    import torch
    n = cell.numel()
    nb = ctypes.c_size_t(0)
    _check(lib().pic_bin_cells_scratch_bytes(ncell, ctypes.byref(nb)))
    scratch = torch.empty(nb.value, dtype=torch.uint8, device=cell.device)
    start = torch.empty(ncell + 1, dtype=torch.int32, device=cell.device)
    order = torch.empty(max(n, 1), dtype=torch.int32, device=cell.device)
    st = stream if stream is not None else torch.cuda.current_stream(cell.device)
    _check(lib().pic_bin_cells(_VP(cell.data_ptr()), n, ncell, _VP(start.data_ptr()),
                               _VP(order.data_ptr()), _VP(scratch.data_ptr()), nb.value,
                               _VP(st.cuda_stream)))
    st.synchronize()
    return start, order[:n]


def history_array(recs, key, comp=None):
    if comp is None:
        return np.array([r[key] for r in recs])
    return np.array([r[key][comp] for r in recs])


# ---------------------------------------------------------------- closure network
PIC_MLP_NPARAM = 4865


class ClosureNet:
    """The closure network on the GPU (pic_mlp_*): FP32 master parameters and Adam moments as
    device tensors; forward and full-batch Adam steps through the C ABI on one stream.

    x arguments are feature-major float32 CUDA tensors of shape (>= nin, n) (the moment
    recorder's rows 0..8 qualify directly)."""

    def __init__(self, params, mu, sigma, nin=9, device="cuda", stream=None):
        import torch
        self._torch = torch
        self.device = torch.device(device)
        self.params = torch.as_tensor(np.asarray(params, np.float32), device=self.device).contiguous()
        assert self.params.numel() == PIC_MLP_NPARAM
        self.m = torch.zeros_like(self.params)
        self.v = torch.zeros_like(self.params)
        self.t = 0
        self.norm = MlpNorm()
        for j in range(9):
            self.norm.mu[j] = float(mu[j]) if j < len(mu) else 0.0
            self.norm.sigma[j] = float(sigma[j]) if j < len(sigma) else 1.0
        self.norm.nin = int(nin)
        self.stream = stream if stream is not None else torch.cuda.Stream(self.device)
        nb = ctypes.c_size_t(0)
        _check(lib().pic_mlp_train_scratch_bytes(ctypes.byref(nb)))
        self._scratch = torch.empty(nb.value, dtype=torch.uint8, device=self.device)
        self._loss = torch.zeros(1, dtype=torch.float32, device=self.device)

    def _sync_inputs(self):
        # inputs made by torch on its current stream must be complete before our stream reads them
        self.stream.wait_stream(self._torch.cuda.current_stream(self.device))

    def forward(self, x, out=None):
        torch = self._torch
        n = x.shape[1]
        if out is None:
            out = torch.empty(n, dtype=torch.float32, device=self.device)
        self._sync_inputs()
        _check(lib().pic_mlp_forward(_VP(self.params.data_ptr()), ctypes.byref(self.norm), _VP(x.data_ptr()),
                                     x.stride(0), n, _VP(out.data_ptr()), _VP(self.stream.cuda_stream)))
        self.stream.synchronize()
        _check(lib().pic_mlp_status(1))
        return out

    def train_step(self, x, target, lr):
        """One Adam step on the batch; returns the loss before the update (a float)."""
        self.t += 1
        self._sync_inputs()
        _check(lib().pic_mlp_train_step(_VP(self.params.data_ptr()), _VP(self.m.data_ptr()),
                                        _VP(self.v.data_ptr()), self.t, float(lr), ctypes.byref(self.norm),
                                        _VP(x.data_ptr()), x.stride(0), _VP(target.data_ptr()), x.shape[1],
                                        _VP(self._loss.data_ptr()), _VP(self._scratch.data_ptr()),
                                        self._scratch.numel(), _VP(self.stream.cuda_stream)))
        self.stream.synchronize()
        _check(lib().pic_mlp_status(1))
        return float(self._loss.cpu()[0])


def dispersion_growth(params, kmin, kmax, nk, stream=None):
    """Max over a uniform k grid of Im w of Eq. (12) per parameter set (pic_dispersion_growth).
    params: (nsets, 4) array-like of (c_s^2, beta0, n_b, nu).  Returns (gamma, kstar) as numpy."""
    import torch
    p = torch.as_tensor(np.ascontiguousarray(params, dtype=np.float64).reshape(-1, 4), device="cuda")
    n = p.shape[0]
    g = torch.empty(n, dtype=torch.float64, device="cuda")
    k = torch.empty(n, dtype=torch.float64, device="cuda")
    st = stream if stream is not None else torch.cuda.current_stream()
    _check(lib().pic_dispersion_growth(_VP(p.data_ptr()), n, float(kmin), float(kmax), int(nk),
                                       _VP(g.data_ptr()), _VP(k.data_ptr()), _VP(st.cuda_stream)))
    st.synchronize()
    return g.cpu().numpy(), k.cpu().numpy()


# ---------------------------------------------------------------- hybrid model
class HybridEngine:
    """The quasi-neutral hybrid model (pic_hybrid_*): arena and stream from PyTorch."""

    def __init__(self, nx, ny, dx, dy, dt, n0, nu, w, capacity, tol=0.0, max_iter=0, flags=0,
                 sort_interval=0, device="cuda"):
        import torch
        self._torch = torch
        self.cfg = HybridConfig(nx, ny, dx, dy, dt, n0, nu, w, capacity, tol, max_iter, flags,
                                sort_interval)
        nb = ctypes.c_size_t(0)
        _check(lib().pic_hybrid_required_bytes(ctypes.byref(self.cfg), ctypes.byref(nb)))
        self.device = torch.device(device)
        self.arena = torch.empty(nb.value, dtype=torch.uint8, device=self.device)
        self.stream = torch.cuda.Stream(self.device)
        h = _VP()
        _check(lib().pic_hybrid_init(ctypes.byref(self.cfg), _VP(self.arena.data_ptr()), nb.value,
                                     _VP(self.stream.cuda_stream), ctypes.byref(h)))
        self._h = h
        self.n = 0

    def close(self):
        if self._h:
            lib().pic_hybrid_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def load(self, X, Y, ux, uy, uz, beta_p):
        f = lambda a: np.ascontiguousarray(a, dtype=np.float64)
        X, Y, ux, uy, uz = f(X), f(Y), f(ux), f(uy), f(uz)
        bp = np.broadcast_to(np.asarray(beta_p, np.float64), (self.cfg.ny, self.cfg.nx)).copy()
        self.n = X.shape[0]
        _check(lib().pic_hybrid_load(self._h, self.n, _ptr(X), _ptr(Y), _ptr(ux), _ptr(uy), _ptr(uz), _ptr(bp)))

    def step(self, n=1):
        _check(lib().pic_hybrid_step(self._h, int(n)))

    def sync(self):
        self.stream.synchronize()

    def state(self):
        nc = (self.cfg.ny, self.cfg.nx)
        a, bp = np.empty(nc), np.empty(nc)
        X, Y, ux, uy = (np.empty(self.n) for _ in range(4))
        _check(lib().pic_hybrid_get(self._h, _ptr(a), _ptr(bp), _ptr(X), _ptr(Y), _ptr(ux), _ptr(uy)))
        return dict(a=a, beta_p=bp, X=X, Y=Y, ux=ux, uy=uy)

    def energies(self):
        out = np.zeros(3)
        _check(lib().pic_hybrid_energies(self._h, _ptr(out)))
        return out

    def stats(self):
        out = np.zeros(4, np.int64)
        _check(lib().pic_hybrid_stats(self._h, _ptr(out)))
        return dict(steps=int(out[0]), cg_iterations=int(out[1]), unconverged_steps=int(out[2]),
                    last_iterations=int(out[3]))

    def kernel_times(self):
        recs = (KernelTime * 4)()
        n = ctypes.c_int(0)
        _check(lib().pic_hybrid_kernel_times(self._h, ctypes.cast(recs, _VP), 4, ctypes.byref(n)))
        return {recs[i].name.decode(): (int(recs[i].launches), float(recs[i].total_ms)) for i in range(n.value)}

    def launch_count(self):
        return int(lib().pic_hybrid_launch_count(self._h))
