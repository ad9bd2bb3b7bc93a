"""Continuous-batching serving loop and batched sweep (small traces).

Each request's torque and heat-up must come out identical whether it ran in
the shared batch (admitted and retired while others ran) or alone through
the plain per-case solver.
"""
import math

import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def serving():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_2512_09904_b300 import build
    build.build()
    from paper_2512_09904_b300 import serving as S
    return S


def test_serving_results_match_plain_solver(serving):
    r = serving.serve(n_requests=6, steps=12, rate=40.0, count_scale=0.1, budget_gb=2.0, max_cases=4,
                      steps_per_poll=4)
    assert r["batched"]["unstable"] == 0
    assert r["max_abs_diff_torque_avg"] == 0.0 and r["max_abs_diff_heat"] == 0.0
    assert math.isfinite(r["batched"]["p99_latency_s"]) and r["batched"]["p99_latency_s"] > 0
    assert r["batched"]["max_resident_cases"] >= 2  # requests overlapped on the device


def test_sweep_results_match_plain_solver(serving):
    r = serving.sweep(n_cases=5, steps=6, count_scale=0.1)
    assert r["max_abs_diff_torque_avg"] == 0.0 and r["max_abs_diff_heat"] == 0.0
    assert r["batched"]["particle_substeps_per_s"] > 0
