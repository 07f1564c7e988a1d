"""Writes warm_krook_128_history.txt: the FP64 oracle's field-energy history of the 128 x 128
crop of the warm-beam Krook workload (64 particles per cell per species, beam T_perp = 0.1,
background T = 0.001, Krook nu = 0.1, dx = 0.1, dt = 0.05; seed 2), 4000 steps.  Every 4th step:
t, W_B (Bx^2 + By^2, the transverse magnetic energy) and W_E (all components), each summed over
the cells times dx dy.  Calls only the oracle and the seeded inputs; about half an hour on one
core.

    python tests/golden/make_warm_krook_128_history.py
"""
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import numpy as np  # noqa: E402

import oracle  # noqa: E402
import pic_inputs as pi  # noqa: E402

STEPS, EVERY = 4000, 4


def main():
    wl = pi.warm_beam_krook_2d(n=128, ppc=64)
    sim = oracle.Simulation.from_workload(wl)
    rows = []
    for n in range(STEPS):
        sim.step(1, record=True)
        if n % EVERY == 0:
            h = sim.history[-1]
            rows.append((h["t"], h["WB"][0] + h["WB"][1], sum(h["WE"])))
    out = os.path.join(HERE, "warm_krook_128_history.txt")
    with open(out, "w") as f:
        f.write("# FP64 oracle, warm_beam_krook_2d(n=128, ppc=64), 4000 steps, every 4th step\n")
        f.write("# written by tests/golden/make_warm_krook_128_history.py\n")
        f.write("# t  W_B_perp  W_E\n")
        for t, wb, we in rows:
            f.write(f"{t:.4f} {wb:.9e} {we:.9e}\n")


if __name__ == "__main__":
    main()
