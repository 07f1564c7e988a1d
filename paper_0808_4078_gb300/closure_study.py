"""The learned-closure study: a network trained on a collisionless 3D run's moments drives the
return-current drag of a cheaper 2D run, compared with the 3D run and with the 2D run without it.

The paper's conclusion conjectures that in 3D the two-stream (electrostatic) turbulence of the
beam acts on the return current like collisions, an anomalous collisionality that a 2D run,
which has no two-stream modes, lacks.  The study, all of it on the GPU through the C ABI:

  1. a collisionless 3D run (beam along z) records the coarse moments every `every` steps
     (pic_record_moments: coarse cells of bx x by transverse cells and the whole z extent);
  2. windows of `window` snapshots (about 1/w_p) become training samples: features = window means
     of the 9 moment rows, label = the friction rate nu_eff of the fluctuating fields on the
     return current (pic_closure_samples; windows whose mean return-current drift has fallen
     below uz_min are left out);
  3. two networks are trained (pic_mlp_fit_norm, pic_mlp_train_step): all 9 inputs, and 8
     without W_ES (the z-fluctuation energy, zero in 2D by construction);
  4. 2D runs of the same transverse plane and physics: without drag (nu = 0), with constant
     Krook rates, and driven by each network (every `every` steps: pic_record_moments ->
     pic_mlp_forward -> pic_set_drag_map on the background species);
  5. the transverse magnetic energy per unit volume, W_B = (B_x^2 + B_y^2) / 2 averaged over the
     box, is compared with the 3D run's: its exponential growth rate (pic_fit_growth) and its
     peak level.

Run as a script for a given size (python -m paper_0808_4078_gb300.closure_study --help); the
result is one JSON object.
"""
from __future__ import annotations

import argparse
import ctypes
import json
import math
import time

import numpy as np

from . import ClosureNet, Engine, PIC_MOM_ROWS, _VP, _check, lib

CONST_NU = (0.01, 0.03, 0.1, 0.3, 1.0)


def record(eng, steps, every, bx, by, run=0):
    """Step `steps` steps, recording the coarse moments after every `every` steps: a device
    tensor (steps // every, PIC_MOM_ROWS, ncoarse)."""
    import torch
    snaps = []
    for _ in range(steps // every):
        eng.step(every)
        snaps.append(eng.record_moments(bx, by, run=run).clone())
    return torch.stack(snaps)


def training_set(rows, window, nu_p, uz_min):
    """Samples of the closure from recorded snapshots (pic_closure_samples): features (9, n)
    and labels (n,) as device tensors."""
    import torch
    rows = rows.contiguous()
    nsnap, nrow, nc = rows.shape
    assert nrow == PIC_MOM_ROWS
    m = (nsnap // window) * nc
    nb = ctypes.c_size_t(0)
    _check(lib().pic_closure_samples_scratch_bytes(m, ctypes.byref(nb)))
    scratch = torch.empty(nb.value, dtype=torch.uint8, device=rows.device)
    feat = torch.empty((9, max(m, 1)), dtype=torch.float32, device=rows.device)
    label = torch.empty(max(m, 1), dtype=torch.float32, device=rows.device)
    n = torch.zeros(1, dtype=torch.int64, device=rows.device)
    stream = torch.cuda.current_stream(rows.device)
    _check(lib().pic_closure_samples(_VP(rows.data_ptr()), nsnap, nc, window, float(nu_p), float(uz_min),
                                     _VP(feat.data_ptr()), _VP(label.data_ptr()), m, _VP(n.data_ptr()),
                                     _VP(scratch.data_ptr()), nb.value, _VP(stream.cuda_stream)))
    k = int(n.item())
    return feat[:, :k].contiguous(), label[:k].contiguous()


def fit_norm(feat, nin):
    """Input normalisation of a network from its training features (pic_mlp_fit_norm)."""
    import torch
    ms = torch.empty(18, dtype=torch.float32, device=feat.device)
    stream = torch.cuda.current_stream(feat.device)
    _check(lib().pic_mlp_fit_norm(_VP(feat.data_ptr()), feat.stride(0), feat.shape[1], nin, _VP(ms.data_ptr()),
                                  _VP(stream.cuda_stream)))
    v = ms.cpu().numpy().astype(np.float64)
    return v[:9], v[9:]


def init_params(seed, nin):
    """Uniform(-1/sqrt(fan_in), 1/sqrt(fan_in)) weights and biases, the output bias 0, the inputs
    past nin without weight (float32 master parameters in the C ABI's order)."""
    rng = np.random.default_rng(seed)
    w1 = rng.uniform(-1, 1, (64, 9)) / math.sqrt(nin)
    w1[:, nin:] = 0.0
    b1 = rng.uniform(-1, 1, 64) / math.sqrt(nin)
    w2 = rng.uniform(-1, 1, (64, 64)) / 8.0
    b2 = rng.uniform(-1, 1, 64) / 8.0
    w3 = rng.uniform(-1, 1, 64) / 8.0
    return np.concatenate([w1.ravel(), b1, w2.ravel(), b2, w3, [0.0]]).astype(np.float32)


def train(feat, label, nin, steps=2000, lr=1e-3, seed=1):
    """A closure network trained by full-batch Adam steps on the device; returns (net, losses)."""
    mu, sd = fit_norm(feat, nin)
    net = ClosureNet(init_params(seed, nin), mu, sd, nin=nin, device=feat.device)
    losses = []
    for k in range(steps):
        loss = net.train_step(feat, label, lr)
        if k % max(1, steps // 20) == 0 or k == steps - 1:
            losses.append(loss)
    return net, losses


def drive(eng, net, steps, every, bx, by, species=1):
    """Advance a 2D engine `steps` steps with the network setting the drag of `species` every
    `every` steps from the run's own moments; returns the mean predicted rate per update
    (negative predictions act as 0 in the drag)."""
    import torch
    means = []
    for _ in range(steps // every):
        rows = eng.record_moments(bx, by)
        nu = net.forward(rows)
        means.append(float(torch.clamp(nu, min=0).mean()))
        eng.set_drag_map(species, nu, bx, by)
        eng.step(every)
    return means


def wb_perp(recs, volume):
    t = np.array([r["t"] for r in recs])
    return t, np.array([(r["WB"][0] + r["WB"][1]) / volume for r in recs])


def summary(eng, volume):
    """Growth rate of the transverse magnetic energy (0 if it has no exponential stage) and its
    peak level per unit volume."""
    recs = eng.diag()
    t, w = wb_perp(recs, volume)
    g, t0, t1 = eng.fit_growth()
    if not math.isfinite(g):
        g, t0, t1 = 0.0, float("nan"), float("nan")
    return dict(gamma=g, fit_window=[t0, t1], level=float(w.max()), t_level=float(t[w.argmax()]),
                W=[float(x) for x in w[:: max(1, len(w) // 50)]])


def errors(s, ref):
    eg = abs(s["gamma"] - ref["gamma"]) / ref["gamma"] if ref["gamma"] > 0 else float("nan")
    el = abs(math.log(max(s["level"], 1e-300) / ref["level"]))
    return dict(gamma_rel=eg, level_log=el)


def _load(big, **kw):
    """A seeded Weibel load: drawn in parallel into shared memory for large grids."""
    import pic_inputs as pi
    if big:
        L = pi.weibel_load_parallel(workers=16, **kw)
        return L.workload, L
    return pi.weibel_load(**kw), None


def run_study(nx, ny, nz, ppc, steps, every=4, window=5, bx=4, by=4, j_filter=1, train_steps=2000,
              lr=1e-3, uz_min_frac=0.25, seed3=3, seed2=5, T_perp=0.2, const_nu=CONST_NU, log=None,
              nx2=None, ny2=None, ppc2=None):
    """The whole study at one size (the 2D runs on nx2 x ny2 cells with ppc2 particles per cell
    and species, by default the 3D run's transverse grid and ppc); returns a JSON-able dict."""
    import torch
    nx2, ny2, ppc2 = nx2 or nx, ny2 or ny, ppc2 or ppc
    out = dict(config=dict(nx=nx, ny=ny, nz=nz, ppc=ppc, nx2=nx2, ny2=ny2, ppc2=ppc2, steps=steps, every=every,
                           window=window, bx=bx, by=by, j_filter=j_filter, train_steps=train_steps, lr=lr,
                           T_perp=T_perp, dx=0.1, dt=0.05))
    t0 = time.time()
    wl3, L3 = _load(nx * ny * nz * ppc > (1 << 26), ndim=3, nx=nx, ny=ny, nz=nz, ppc=ppc, T_perp_beam=T_perp,
                    seed=seed3)
    uz_p0 = float(np.mean(wl3.species[1].u[2]))
    eng3 = Engine.from_workload(wl3, diag_interval=1, diag_capacity=steps + 8, sort_interval=8, j_filter=j_filter)
    del wl3
    if L3 is not None:
        L3.close()
    t3 = time.time()
    rows = record(eng3, steps, every, bx, by)
    eng3.sync()
    vol3 = nx * ny * nz * 0.1 ** 3
    out["run3d"] = summary(eng3, vol3)
    out["run3d"]["stats"] = eng3.stats()
    out["run3d"]["wall_s"] = time.time() - t3
    eng3.close()
    del eng3
    torch.cuda.empty_cache()
    feat, label = training_set(rows, window, 0.0, uz_min_frac * abs(uz_p0))
    lab = label.double().cpu().numpy()
    out["samples"] = dict(n=int(lab.size), of=int((rows.shape[0] // window) * rows.shape[2]),
                          label_mean=float(lab.mean()), label_std=float(lab.std()),
                          label_q05_50_95=[float(v) for v in np.quantile(lab, [0.05, 0.5, 0.95])],
                          uz_min=uz_min_frac * abs(uz_p0))
    if log:
        log(f"3D done {time.time() - t0:.1f}s {out['run3d']['gamma']:.4f} {out['run3d']['level']:.3e}; "
            f"{lab.size} samples")
    nets = {}
    for nin in (9, 8):
        net, losses = train(feat, label, nin, train_steps, lr)
        pred = net.forward(feat).double().cpu().numpy()
        out[f"train{nin}"] = dict(losses=losses, r2=float(1 - np.mean((pred - lab) ** 2) / lab.var()))
        nets[nin] = net
    vol2 = nx2 * ny2 * 0.1 ** 2
    ref = out["run3d"]
    wl2, L2 = _load(nx2 * ny2 * ppc2 > (1 << 24), ndim=2, nx=nx2, ny=ny2, ppc=ppc2, T_perp_beam=T_perp, seed=seed2)

    def run2d(nu, net=None):
        eng = Engine(2, nx2, ny2, dx=wl2.dx, dt=wl2.dt, capacity=[sp.n for sp in wl2.species],
                     diag_interval=1, diag_capacity=steps + 8, sort_interval=8, j_filter=j_filter)
        for i, sp in enumerate(wl2.species):
            eng.load_species(i, sp.q, sp.m, sp.w, nu if i == 1 else sp.nu, sp.cell, sp.offset, sp.u)
        rates = None
        if net is None:
            eng.step(steps)
        else:
            rates = drive(eng, net, steps, every, bx, by)
        s = summary(eng, vol2)
        eng.close()
        del eng
        torch.cuda.empty_cache()
        s.update(errors(s, ref))
        if rates is not None:
            s["mean_rate"] = float(np.mean(rates))
        return s

    out["run2d_nu0"] = run2d(0.0)
    out["run2d_const"] = {str(nu): run2d(nu) for nu in const_nu}
    for nin in (9, 8):
        out[f"run2d_net{nin}"] = run2d(0.0, nets[nin])
    if L2 is not None:
        L2.close()
    best_l = min(out["run2d_const"].items(), key=lambda kv: kv[1]["level_log"])
    best_g = min(out["run2d_const"].items(), key=lambda kv: kv[1]["gamma_rel"])
    out["best_const_level"] = dict(nu=float(best_l[0]), **errors(best_l[1], ref))
    out["best_const_gamma"] = dict(nu=float(best_g[0]), **errors(best_g[1], ref))
    out["wall_s"] = time.time() - t0
    return out


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--nx", type=int, default=64)
    ap.add_argument("--ny", type=int, default=64)
    ap.add_argument("--nz", type=int, default=128)
    ap.add_argument("--ppc", type=int, default=8)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--bx", type=int, default=4)
    ap.add_argument("--train-steps", type=int, default=2000)
    ap.add_argument("--nx2", type=int, default=None, help="2D grid side (default: the 3D transverse grid)")
    ap.add_argument("--ppc2", type=int, default=None, help="2D particles per cell and species")
    ap.add_argument("--out", default=None)
    a = ap.parse_args()
    res = run_study(a.nx, a.ny, a.nz, a.ppc, a.steps, bx=a.bx, by=a.bx, train_steps=a.train_steps,
                    log=lambda m: print(m, flush=True), nx2=a.nx2, ny2=a.nx2, ppc2=a.ppc2)
    s = json.dumps(res)
    if a.out:
        with open(a.out, "w") as f:
            f.write(s)
    print(s)


if __name__ == "__main__":
    main()
