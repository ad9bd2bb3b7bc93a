"""Writes gear_bath_5mm_1000.json: the FP64 oracle's clock, churning torque
about the gear axis (instantaneous and its running time average) and
lubricant heat-up after each of 1000 advection steps of the gear bath at
dx = 5 mm (the 2M workload's geometry, coarse enough for the O(N^2) oracle).

Calls only the oracle and the seeded workload generator:
    python tests/golden/make_gear_bath_5mm.py
"""
import json
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import oracle as O  # noqa: E402
from paper_2512_09904_b300 import workloads as W  # noqa: E402

DX, OMEGA, STEPS = 5e-3, 600.0, 1000
COLUMNS = ("t", "substeps", "torque", "torque_avg", "heat", "mean_T")


def main():
    threads = O.set_threads(0)
    case = W.gear_bath(dx=DX, omega=OMEGA)
    sim = O.OracleSim(case)
    cols = {k: [] for k in COLUMNS}
    t0 = time.time()
    for k in range(STEPS):
        sim.step(1)
        th, tm = sim.torque_heat(0), sim.time()
        for c, v in (("t", tm["t"]), ("substeps", tm["substeps"]), ("torque", th["torque"]),
                     ("torque_avg", th["torque_avg"]), ("heat", th["heat"]), ("mean_T", th["mean_T"])):
            cols[c].append(v)
        if (k + 1) % 50 == 0:
            print(k + 1, {c: cols[c][-1] for c in COLUMNS}, round(time.time() - t0, 1), "s", flush=True)
    out = dict(workload="gear_bath", dx=DX, omega=OMEGA, n_fluid=case.n_fluid, n_solid=case.n_solid,
               oracle_threads=threads, steps=STEPS,
               note="column k holds the state after advection step k + 1", per_step=cols)
    with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "gear_bath_5mm_1000.json"), "w") as f:
        json.dump(out, f, separators=(",", ":"))


if __name__ == "__main__":
    main()
