"""Writes gear_bath_5mm_1000.json: the FP64 oracle's clock, churning torque
(time average about the gear axis) and lubricant heat-up along 1000 advection
steps of the gear bath at dx = 5 mm (the 2M workload's geometry, coarse
enough for the O(N^2) oracle), recorded every 100 steps.

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

DX, OMEGA, STEPS, EVERY = 5e-3, 600.0, 1000, 100


def main():
    threads = O.set_threads(0)
    case = W.gear_bath(dx=DX, omega=OMEGA)
    sim = O.OracleSim(case)
    rows = []
    t0 = time.time()
    for k in range(STEPS // EVERY):
        sim.step(EVERY)
        th = sim.torque_heat(0)
        tm = sim.time()
        rows.append(dict(steps=(k + 1) * EVERY, t=tm["t"], substeps=tm["substeps"], torque_avg=th["torque_avg"],
                         heat=th["heat"], mean_T=th["mean_T"]))
        print(rows[-1], round(time.time() - t0, 1), "s", flush=True)
    out = dict(workload="gear_bath", dx=DX, omega=OMEGA, n_fluid=case.n_fluid, n_solid=case.n_solid,
               oracle_threads=threads, records=rows)
    with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "gear_bath_5mm_1000.json"), "w") as f:
        json.dump(out, f, indent=1)


if __name__ == "__main__":
    main()
