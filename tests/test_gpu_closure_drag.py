"""Closure-driven drag (pic_set_drag_map): per-cell Krook rates against the oracle's per-cell
rates (set_nu_cell), and the constant map against the scalar rate, bit for bit."""
import numpy as np
import pytest

import pic_inputs as pi

pytestmark = pytest.mark.gpu

NU = float(np.float32(0.2))      # a rate both sides hold exactly


@pytest.fixture(scope="module")
def pic():
    import __graft_entry__ as ge
    ge.build()
    import paper_0808_4078_gb300 as pic
    return pic


def _wl2(seed=81, nu=NU):
    return pi.weibel_load(ndim=2, nx=32, ny=32, ppc=16, T_perp_beam=0.1, T_bg=0.01, nu=nu, seed=seed)


def _dev(a):
    import torch
    return torch.as_tensor(np.ascontiguousarray(a, dtype=np.float32), device="cuda")


def _state(eng):
    E, B, _ = eng.fields()
    out = [E, B]
    for s in range(2):
        c, o, u, ids = eng.particles(s)
        k = np.argsort(ids)
        out += [c[k], o[:, k], u[:, k]]
    return out


def test_constant_map_equals_scalar_rate(pic):
    wl = _wl2()
    a = pic.Engine.from_workload(wl, track_ids=True)
    b = pic.Engine.from_workload(wl, track_ids=True)
    b.set_drag_map(1, _dev(np.full(wl.ncell, NU)))
    a.step(20)
    b.step(20)
    for x, y in zip(_state(a), _state(b)):
        assert np.array_equal(x, y)
    a.close()
    b.close()


def _check_particles(eng, sim, nsp=2, tol=1e-5):
    for s in range(nsp):
        cell, off, u, ids = eng.particles(s)
        k = np.argsort(ids)
        ug = u[:, k].astype(np.float64)
        uo = sim.species[s].u
        err = np.linalg.norm(ug - uo, axis=0) / np.maximum(np.linalg.norm(uo, axis=0), 1e-12)
        assert err.max() < tol, (s, err.max())


@pytest.mark.parametrize("ndim,bx", [(2, 1), (2, 4), (3, 4)])
def test_per_cell_rates_match_oracle(pic, ndim, bx):
    import oracle
    if ndim == 2:
        wl = _wl2(seed=83)
    else:
        wl = pi.weibel_load(ndim=3, nx=16, ny=16, nz=16, ppc=8, T_perp_beam=0.2, T_bg=0.01, nu=NU, seed=84)
    rng = np.random.default_rng(7)
    ncx, ncy = wl.nx // bx, wl.ny // bx
    nu_c = rng.uniform(0.0, 3.0, ncx * ncy).astype(np.float32)
    nu_c[::5] = -1.0                                     # acts as 0
    eng = pic.Engine.from_workload(wl, track_ids=True, sort_interval=8)
    eng.set_drag_map(1, _dev(nu_c), bx, bx)
    sim = oracle.Simulation.from_workload(wl)
    # the oracle takes the rate of each cell: expand the coarse map over x, y (and z)
    cols = np.repeat(np.repeat(nu_c.reshape(ncy, ncx), bx, axis=0), bx, axis=1).reshape(-1)
    sim.set_nu_cell(1, np.tile(cols, wl.nz).astype(np.float64))
    for chunk in (1, 4, 15):
        eng.step(chunk)
        sim.step(chunk, record=False)
        _check_particles(eng, sim)
    eng.close()


def test_map_enables_drag_and_rejects_second_species(pic):
    import oracle
    wl = _wl2(seed=85, nu=0.0)                           # no drag at load
    eng = pic.Engine.from_workload(wl, track_ids=True)
    rng = np.random.default_rng(9)
    nu_c = rng.uniform(0.5, 2.0, wl.ncell).astype(np.float32)
    eng.set_drag_map(1, _dev(nu_c))
    with pytest.raises(pic.PicError):
        eng.set_drag_map(0, _dev(nu_c))                  # the background already carries it
    sim = oracle.Simulation.from_workload(wl)
    sim.set_nu_cell(1, nu_c.astype(np.float64))
    eng.step(10)
    sim.step(10, record=False)
    _check_particles(eng, sim)
    eng.set_drag_map(1, None)                            # back to the scalar rate (0)
    sim.set_nu_cell(1, np.zeros(wl.ncell))
    eng.step(5)
    sim.step(5, record=False)
    _check_particles(eng, sim)
    eng.close()
