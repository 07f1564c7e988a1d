"""Coarse-grained moments of a PIC state: the inputs and label of the learned collision
closure -- TEST INFRASTRUCTURE ONLY (see the package docstring).

The paper's conclusion conjectures that the collisional drag seen by the return current could be
expressed through a closure in the local plasma state; nothing in the paper fixes the inputs or
the label, so the definitions below are a reading, written out plainly in FP64:

Coarse cell: a block of bx x by cells of the transverse plane (x, y) and the whole z extent (3D)
or just the bx x by block (2D).  Particles belong to the cell that contains them (nearest grid
point), so to the coarse cell of that cell.  With w the weight of a macro-particle (density per
macro-particle and cell) and sums over the particles of one species in one coarse cell:

  n_s      = sum w / (cells in the coarse cell)                          (density, units n0)
  <a>_s    = sum w a / sum w                                             (weighted mean)
  uz_s     = <u_z>_s
  Tperp_s  = (Var u_x + Var u_y) / 2,   Var a = <a^2>_s - <a>_s^2        (momentum variance per
  Tpar_s   = Var u_z                                                      transverse component)
  W_ES     = mean over the coarse cell's cells of sum_c (E_c - <E_c>_z)^2, where <E_c>_z is the
             mean of the stored E_c over the column of cells sharing (x, y) (0 in 2D)
  Fz_p     = <q (E + v x B)_z>_p with E, B gathered at each background particle as in the push
             and v = u / gamma from the stored momentum
  Fz_mean  = q (Ebar_z + (vbar x Bbar)_z): Ebar, Bbar the means of the stored fields over the
             coarse cell, vbar = <v>_p
  nu_eff   = nu_p + (Fz_mean - Fz_p) / uz_p   (0 where uz_p = 0): the friction rate that the
             field fluctuations exert on the return current beyond the coarse fields' force, plus
             the imposed Krook rate; the paper's time average over 1/w_p is taken by averaging
             Fz_p, Fz_mean and uz_p over snapshots before forming the ratio (label_from_rows).

Species 0 is the beam (b), species 1 the background (p).  Rows of the result, in order:
"""
from __future__ import annotations

import numpy as np

ROWS = ("n_b", "n_p", "uz_b", "uz_p", "Tperp_b", "Tpar_b", "Tperp_p", "Tpar_p", "W_ES",
        "Fz_p", "Fz_mean", "nu_eff")
__doc__ += "  " + ", ".join(ROWS) + "\n"


def _coarse_index(sim, X, Y, bx, by):
    i = np.floor(X).astype(np.int64) % sim.nx
    j = np.floor(Y).astype(np.int64) % sim.ny
    ncx = sim.nx // bx
    return (j // by) * ncx + (i // bx)


def coarse_moments(sim, bx, by):
    """The 12 rows above for every coarse cell of an oracle Simulation (FP64, shape 12 x nc)."""
    if sim.nx % bx or sim.ny % by:
        raise ValueError("nx, ny must be multiples of bx, by")
    ncx, ncy = sim.nx // bx, sim.ny // by
    nc = ncx * ncy
    cells = bx * by * sim.nz
    out = np.zeros((len(ROWS), nc))
    means = []
    for si, s in enumerate(sim.species[:2]):
        c = _coarse_index(sim, s.X, s.Y, bx, by)
        w = np.full(s.n, s.w)
        sw = np.bincount(c, weights=w, minlength=nc)
        mean = {}
        for a, u in zip("xyz", (s.ux, s.uy, s.uz)):
            m1 = np.bincount(c, weights=w * u, minlength=nc)
            m2 = np.bincount(c, weights=w * u * u, minlength=nc)
            with np.errstate(invalid="ignore", divide="ignore"):
                mean[a] = np.where(sw > 0, m1 / sw, 0.0)
                mean[a + "2"] = np.where(sw > 0, m2 / sw, 0.0)
        var = {a: mean[a + "2"] - mean[a] ** 2 for a in "xyz"}
        out[si] = sw / cells
        out[2 + si] = mean["z"]
        out[4 + 2 * si] = 0.5 * (var["x"] + var["y"])
        out[5 + 2 * si] = var["z"]
        means.append((c, sw))
    # W_ES: deviations from the z-mean of each column
    w_es = np.zeros(sim.E[0].shape)
    for Ec in sim.E:
        zmean = Ec.mean(axis=0, keepdims=True) if sim.ndim == 3 else Ec
        w_es = w_es + (Ec - zmean) ** 2
    col = w_es.mean(axis=0) if sim.ndim == 3 else w_es          # (ny, nx) column means
    out[8] = col.reshape(ncy, by, ncx, bx).mean(axis=(1, 3)).reshape(-1)
    # forces on the background (species 1)
    if len(sim.species) > 1:
        s = sim.species[1]
        c, sw = means[1]
        EB = sim.gather_many(s.X, s.Y, s.Z if sim.ndim == 3 else None)
        g = np.sqrt(1.0 + s.ux ** 2 + s.uy ** 2 + s.uz ** 2)
        vx, vy, vz = s.ux / g, s.uy / g, s.uz / g
        fz = s.q * (EB[:, 2] + vx * EB[:, 4] - vy * EB[:, 3])
        w = np.full(s.n, s.w)
        with np.errstate(invalid="ignore", divide="ignore"):
            out[9] = np.where(sw > 0, np.bincount(c, weights=w * fz, minlength=nc) / sw, 0.0)
            vbx = np.where(sw > 0, np.bincount(c, weights=w * vx, minlength=nc) / sw, 0.0)
            vby = np.where(sw > 0, np.bincount(c, weights=w * vy, minlength=nc) / sw, 0.0)

        def block_mean(F):
            colm = F.mean(axis=0) if sim.ndim == 3 else F
            return colm.reshape(ncy, by, ncx, bx).mean(axis=(1, 3)).reshape(-1)

        Ez, Bx, By = block_mean(sim.E[2]), block_mean(sim.B[0]), block_mean(sim.B[1])
        out[10] = s.q * (Ez + vbx * By - vby * Bx)
        out[11] = label_from_rows(out[3], out[9], out[10], s.nu)
    return out


def label_from_rows(uz_p, fz_p, fz_mean, nu):
    """nu_eff = nu + (Fz_mean - Fz_p) / uz_p, 0 where uz_p = 0 (arrays, or their time means)."""
    uz_p = np.asarray(uz_p, dtype=np.float64)
    with np.errstate(invalid="ignore", divide="ignore"):
        return np.where(uz_p != 0, nu + (np.asarray(fz_mean) - np.asarray(fz_p)) / uz_p, 0.0)


def samples(rows, window, nu_p, uz_min):
    """Training samples of the closure from consecutive snapshots rows[nsnap, 12, nc] (FP64):
    windows of `window` snapshots are averaged; per (window, coarse cell), in that order, the
    features are the window means of rows 0..8 and the label is
    nu_p + (<Fz_mean> - <Fz_p>) / <uz_p> (label_from_rows of the window means: the ratio of the
    time means, not the mean of snapshot ratios); samples with |<uz_p>| < uz_min or a non-finite
    label are dropped.  Returns (features[9, n], labels[n])."""
    rows = np.asarray(rows, dtype=np.float64)
    nsnap, nrow, nc = rows.shape
    nw = nsnap // window
    feats, labs = [], []
    for w in range(nw):
        m = rows[w * window:(w + 1) * window].mean(axis=0)         # (12, nc)
        with np.errstate(invalid="ignore", divide="ignore"):
            lab = nu_p + (m[10] - m[9]) / m[3]
        keep = (np.abs(m[3]) >= uz_min) & np.isfinite(lab)
        feats.append(m[:9, keep])
        labs.append(lab[keep])
    if not feats:
        return np.zeros((9, 0)), np.zeros(0)
    return np.concatenate(feats, axis=1), np.concatenate(labs)
