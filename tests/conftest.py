import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (B300, sm_103a)")
    config.addinivalue_line("markers", "slow: long-running oracle case")


@pytest.fixture(scope="session")
def oracle():
    from oracle import oracle as O
    O.lib()
    return O


@pytest.fixture(scope="session")
def oracle_run(oracle):
    """Oracle runs shared by the FP32 and FP64 field-parity tests (the
    oracle is FP64 either way): run(name, case, steps) steps the case one
    advection step at a time and returns, per step, the clock and the
    compared fields.  `name` must identify the case and every setting the
    oracle reads."""
    cache = {}

    def run(name, case, steps):
        if name not in cache or len(cache[name]) < steps:
            sim = oracle.OracleSim(case)
            out = []
            for _ in range(steps):
                sim.step(1)
                out.append(dict(time=sim.time(), **{k: sim.field(k).copy() for k in ("pos", "vel", "rho", "T")}))
            sim.close()
            cache[name] = out
        return cache[name][:steps]

    return run
