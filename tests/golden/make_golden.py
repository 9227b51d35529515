"""Writes the stored expected values of tests/golden/ by running the FP64 CPU
oracle only.  Run:  python tests/golden/make_golden.py

b1_hedgehog_48_trajectory.txt: the 48^3 massless hedgehog workload (B=1 map,
f = pi exp(-r), h = 0.2, dt = 0.05 h) flowed for 1000 arrested-Newton-flow
iterations; one row per 50 iterations with the start-of-iteration energy, its
three parts, the baryon number, the residual delta and the running arrest
count.
"""
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
import workloads  # noqa: E402


def b1_hedgehog_48():
    wl = workloads.b1_hedgehog_48()
    st = oracle.new_state(oracle.seed_rational_map(wl.n, wl.h, 1, wl.seed.profile_scale))
    reps = oracle.flow(st, wl.h, wl.m, wl.dt, wl.steps, reports=True)
    path = os.path.join(HERE, "b1_hedgehog_48_trajectory.txt")
    arrests = 0
    with open(path, "w") as f:
        f.write("# FP64 oracle, 48^3 B=1 hedgehog, h=0.2, m=0, dt=0.01, 1000 ANF iterations\n")
        f.write("# written by tests/golden/make_golden.py (oracle only)\n")
        f.write("# step E E2 E4 E0 B delta arrests_so_far\n")
        for k, r in enumerate(reps):
            arrests += r["arrested"]
            if k % 50 == 0 or k == len(reps) - 1:
                f.write(f"{k} {r['E']!r} {r['E2']!r} {r['E4']!r} {r['E0']!r} {r['B']!r} "
                        f"{r['delta']!r} {arrests}\n")
    print("wrote", path)


if __name__ == "__main__":
    b1_hedgehog_48()
