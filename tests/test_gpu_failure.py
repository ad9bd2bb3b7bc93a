"""Failure detection through the C ABI, made on the host with ordinary inputs.

A fluid particle launched at the top of the domain box leaves it within a
few advection steps: the step reports SPH_EUNSTABLE, the case is frozen and
stays readable, and in a batch the other cases' results stay bitwise those
of their runs alone.  No GPU fault is involved: the kernels flag the particle
that left the box, and the host reads the flag.
"""
import numpy as np
import pytest

from paper_2512_09904_b300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sph():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_2512_09904_b300 import build
    build.build()
    from paper_2512_09904_b300 import sph as S
    return S


def _escaping_tank():
    """A small still tank plus one oil particle half a spacing below the top
    of the domain box, moving up at 2 m/s (0.2 c0): with the advection step
    at 0.25 h / |v|max it crosses the box's top face within 3 steps."""
    case = W.still_tank(nx=10, ny=8, nz=6, wall_h=10, seed=33)
    cfg = case.config
    top = cfg["origin"][2] + cfg["extent"][2]
    dx = cfg["dx"]
    p = np.array([[5.5 * dx, 4.5 * dx, top - 0.5 * dx]])
    case.fluids.append(dict(mat=0, pos=p, vel=np.array([[0.0, 0.0, 2.0]]), T=None, rho=None))
    return case


def test_single_context_reports_unstable_and_stays_readable(sph):
    case = _escaping_tank()
    ctx = sph.from_case(case, stream=0)
    with pytest.raises(sph.SphError) as e:
        ctx.sph_step(20)
    assert e.value.status == sph.SPH_EUNSTABLE
    info = ctx.sph_get_info()
    assert info["error_bits"] & 2  # a fluid particle left the box
    assert 1 <= info["adv_steps"] <= 4
    pos = ctx.sph_read_fields("pos")
    # the launched particle is the last fluid id (fluid blocks precede solids)
    assert pos[case.n_fluid - 1, 2] >= case.config["origin"][2] + case.config["extent"][2]
    assert np.all(np.isfinite(pos)) and np.all(np.isfinite(ctx.sph_read_fields("rho")))
    ctx.sph_read_torque_heat(0)
    # frozen: a later call reports the same error and changes nothing
    with pytest.raises(sph.SphError) as e:
        ctx.sph_step(3)
    assert e.value.status == sph.SPH_EUNSTABLE
    assert ctx.sph_get_info()["adv_steps"] == info["adv_steps"]
    assert np.array_equal(ctx.sph_read_fields("pos"), pos)
    ctx.close()


def _alone(sph, case, steps):
    ctx = sph.from_case(case, stream=0)
    ctx.sph_step(steps)
    out = {f: ctx.sph_read_fields(f) for f in ("pos", "vel", "rho", "T")}
    out["th"] = ctx.sph_read_torque_heat(0)
    ctx.close()
    return out


def test_unstable_case_in_a_batch_leaves_the_others_untouched(sph):
    healthy = {"gear": W.gear_bath(dx=7e-3, omega=300.0, depth_frac=0.5, mu=0.1, seed=31),
               "cyl": W.rotating_cylinder(omega=-40.0, seed=32)}
    bad = _escaping_tank()
    steps_a, steps_b = 8, 4
    alone = {k: _alone(sph, c, steps_a + steps_b) for k, c in healthy.items()}
    cases = [healthy["gear"], bad, healthy["cyl"]]
    n = sum(c.n_total for c in cases)
    cells = sum(sph.cells_of(c) for c in cases)
    b = sph.Batch(n, 5, cells + 10, history_steps=64, stream=0)
    slots = {"gear": b.admit(cases[0]), "bad": b.admit(cases[1]), "cyl": b.admit(cases[2])}
    b.step(steps_a)  # the batch step itself succeeds; the case's state says unstable
    done, _, state = b.poll(slots["bad"])
    assert state == sph.BATCH_UNSTABLE and done < steps_a
    for k in ("gear", "cyl"):
        assert b.poll(slots[k])[2] == sph.BATCH_RUNNING
    fl = W.flatten(bad)["kind"] == 0
    assert np.all(np.isfinite(b.fields(slots["bad"], "vel")[fl]))
    b.retire(slots["bad"])
    b.step(steps_b)
    for k in ("gear", "cyl"):
        s = slots[k]
        assert b.poll(s)[0] == steps_a + steps_b
        for f in ("pos", "vel", "rho", "T"):
            assert np.array_equal(b.fields(s, f), alone[k][f]), (k, f)
        th = b.torque_heat(s)
        for q in ("torque", "torque_avg", "heat", "mean_T"):
            assert th[q] == alone[k]["th"][q], (k, q)
    b.close()
