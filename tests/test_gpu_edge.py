"""Edge cases of the PIC engine against the oracle (2D and 3D):

  * no particles at all: the step reduces to the Yee update of seeded fields (vacuum), which
    must match the oracle's Yee step (FP32 against FP64: 1e-5 of the field scale over 10 steps);
  * one species loaded empty (capacity kept): the beam alone, with its uncompensated current,
    matches the oracle's beam-only run particle by particle over 10 steps (1e-5 relative).
"""
import numpy as np
import pytest

import pic_inputs as pi

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pic():
    import __graft_entry__ as ge
    ge.build()
    import paper_0808_4078_gb300 as pic
    return pic


def _seed(eng, sim, shape, ncell, seed=4, amp=0.05):
    rng = np.random.default_rng(seed)
    E0 = (amp * rng.standard_normal((3, ncell))).astype(np.float32)
    B0 = (amp * rng.standard_normal((3, ncell))).astype(np.float32)
    eng.set_fields(E0, B0)
    for a in range(3):
        sim.E[a][...] = E0[a].reshape(shape)
        sim.B[a][...] = B0[a].reshape(shape)


@pytest.mark.parametrize("ndim", [2, 3])
def test_no_particles_is_vacuum_yee(pic, ndim):
    import oracle
    if ndim == 2:
        nx, ny, nz, shape = 32, 48, 1, (48, 32)
    else:
        nx, ny, nz, shape = 16, 16, 8, (8, 16, 16)
    eng = pic.Engine(ndim, nx, ny, nz, dx=0.1, dt=0.05, capacity=(64, 64), diag_interval=1)
    sim = oracle.Simulation(ndim, nx, ny, nz, dx=0.1, dt=0.05)
    _seed(eng, sim, shape, nx * ny * nz)
    eng.step(10)
    sim.step(10)
    E, B = eng.fields()[:2]
    for a in range(3):
        for g, o in ((E[a], sim.E[a]), (B[a], sim.B[a])):
            o = o.reshape(-1)
            assert np.abs(g - o).max() <= 1e-5 * np.abs(o).max()
    eng.close()


@pytest.mark.parametrize("ndim", [2, 3])
def test_one_species_empty(pic, ndim):
    import oracle
    if ndim == 2:
        wl = pi.weibel_load(ndim=2, nx=32, ny=32, ppc=8, T_perp_beam=0.05, seed=15)
    else:
        wl = pi.weibel_load(ndim=3, nx=16, ny=16, nz=8, ppc=4, T_perp_beam=0.05, seed=16)
    beam, bg = wl.species
    eng = pic.Engine(wl.ndim, wl.nx, wl.ny, wl.nz, dx=wl.dx, dt=wl.dt, capacity=(beam.n, bg.n),
                     track_ids=True, diag_interval=1)
    eng.load_species(0, beam.q, beam.m, beam.w, beam.nu, beam.cell, beam.offset, beam.u)
    z = np.zeros(0)
    eng.load_species(1, bg.q, bg.m, bg.w, bg.nu, z.astype(np.int32), np.zeros((wl.ndim, 0), np.float32),
                     np.zeros((3, 0), np.float32))
    only = pi.Workload(wl.name + "_beam_only", wl.ndim, wl.nx, wl.ny, wl.nz, wl.dx, wl.dy, wl.dz,
                       wl.dt, 0, [beam])
    sim = oracle.Simulation.from_workload(only)
    eng.step(10)
    sim.step(10)
    cell, off, u, ids = eng.particles(0)
    order = np.argsort(ids)
    ug = u[:, order].astype(np.float64)
    uo = sim.species[0].u
    err = np.linalg.norm(ug - uo, axis=0) / np.maximum(np.linalg.norm(uo, axis=0), 1e-12)
    assert err.max() < 1e-5, err.max()
    assert eng.particles(1)[0].shape[0] == 0
    assert eng.stats()["flags"] == 0
    eng.close()
