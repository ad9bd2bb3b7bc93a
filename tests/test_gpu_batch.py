"""Batched cases in one packed array (sweeps and serving), through the C ABI.

A case's particle dynamics must not depend on which other cases share the
batch: its particles keep their relative order, its neighbours are its own,
and every per-case sum runs in a fixed order.  So results alone and in the mix
are compared for exact equality.
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


def _cases():
    return {
        "gear": W.gear_bath(dx=7e-3, omega=300.0, depth_frac=0.5, mu=0.1, seed=31),
        "cyl": W.rotating_cylinder(omega=-40.0, seed=32),
        "tank": W.still_tank(nx=10, ny=8, nz=6, wall_h=10, seed=33),
    }


def _alone(sph, case, steps):
    ctx = sph.from_case(case, stream=0)
    ctx.sph_step(steps)
    out = {f: ctx.sph_read_fields(f) for f in ("pos", "vel", "rho", "T")}
    out["th"] = ctx.sph_read_torque_heat(0)
    out["info"] = ctx.sph_get_info()
    ctx.close()
    return out


def _batch_for(sph, cases, steps=0, max_particles=None):
    n = sum(c.n_total for c in cases)
    cells = sum(sph.cells_of(c) for c in cases)
    return sph.Batch(max_particles or n, max(len(cases), 1) + 2, cells + 10, history_steps=64, stream=0)


def _same(a, b):
    for f in ("pos", "vel", "rho", "T"):
        assert np.array_equal(a[f], b[f]), f
    for k in ("torque", "torque_avg", "heat", "mean_T"):
        assert a["th"][k] == b["th"][k], k


def test_alone_equals_mixed_bitwise(sph):
    cs = _cases()
    steps = 6
    alone = {k: _alone(sph, c, steps) for k, c in cs.items()}
    b = _batch_for(sph, list(cs.values()))
    slots = {k: b.admit(c, n_steps=0) for k, c in cs.items()}
    b.step(steps)
    for k, s in slots.items():
        got = {f: b.fields(s, f) for f in ("pos", "vel", "rho", "T")}
        got["th"] = b.torque_heat(s)
        _same(got, alone[k])
        steps_done, t, state = b.poll(s)
        assert steps_done == steps and state == sph.BATCH_RUNNING
        assert t == alone[k]["info"]["t"]
    b.close()


def test_alone_equals_mixed_bitwise_untabulated_corners(sph):
    """A case whose grid is too long for tabulated geometry-cell corners
    (snapshot offsets in their arithmetic form) next to one with them."""
    cs = {"chan": W.long_channel(), "cyl": _cases()["cyl"]}
    steps = 4
    alone = {k: _alone(sph, c, steps) for k, c in cs.items()}
    b = _batch_for(sph, list(cs.values()))
    slots = {k: b.admit(c, n_steps=0) for k, c in cs.items()}
    b.step(steps)
    for k, s in slots.items():
        got = {f: b.fields(s, f) for f in ("pos", "vel", "rho", "T")}
        got["th"] = b.torque_heat(s)
        _same(got, alone[k])
    b.close()


def test_case_constant_sources_agree_bitwise(sph):
    # the pair passes read a case's constants from one parameter-block entry
    # (a case alone), a per-slot table (batches of up to 64 slots) or the
    # global case table (more slots): all three give the same bits
    cs = _cases()
    steps = 4
    alone = _alone(sph, cs["gear"], steps)
    n = sum(c.n_total for c in cs.values())
    cells = sum(sph.cells_of(c) for c in cs.values()) + 10
    for max_cases in (4, 80):  # 80 slots > the 64-entry table
        b = sph.Batch(n, max_cases, cells, history_steps=16, stream=0)
        slots = {k: b.admit(c, n_steps=0) for k, c in cs.items()}
        b.step(steps)
        got = {f: b.fields(slots["gear"], f) for f in ("pos", "vel", "rho", "T")}
        got["th"] = b.torque_heat(slots["gear"])
        _same(got, alone)
        b.close()


def test_admit_and_retire_while_others_run(sph):
    cs = _cases()
    ref_gear = _alone(sph, cs["gear"], 5)
    ref_cyl = _alone(sph, cs["cyl"], 3)
    b = _batch_for(sph, list(cs.values()))
    s_gear = b.admit(cs["gear"])
    s_tank = b.admit(cs["tank"])
    b.step(2)
    b.retire(s_tank)            # leaves at the next step
    s_cyl = b.admit(cs["cyl"])  # joins at the next step
    b.step(3)
    assert b.info()["n_cases"] == 2
    assert b.info()["n_particles"] == cs["gear"].n_total + cs["cyl"].n_total
    g = {f: b.fields(s_gear, f) for f in ("pos", "vel", "rho", "T")}
    g["th"] = b.torque_heat(s_gear)
    _same(g, ref_gear)
    c = {f: b.fields(s_cyl, f) for f in ("pos", "vel", "rho", "T")}
    c["th"] = b.torque_heat(s_cyl)
    _same(c, ref_cyl)
    b.close()


def test_requested_steps_then_frozen(sph):
    cs = _cases()
    ref = _alone(sph, cs["cyl"], 3)
    b = _batch_for(sph, [cs["cyl"], cs["gear"]])
    s = b.admit(cs["cyl"], n_steps=3)
    s2 = b.admit(cs["gear"], n_steps=0)
    b.step(5)
    steps_done, t, state = b.poll(s)
    assert steps_done == 3 and state == sph.BATCH_DONE
    got = {f: b.fields(s, f) for f in ("pos", "vel", "rho", "T")}
    got["th"] = b.torque_heat(s)
    _same(got, ref)
    assert b.poll(s2)[0] == 5
    curve = b.curve(s, 10)
    assert curve.shape == (3, 8)
    assert np.all(np.diff(curve[:, 0]) > 0)
    assert curve[-1, 0] == t
    assert curve[-1, 2] == pytest.approx(ref["th"]["torque_avg"], rel=1e-12)
    b.close()


def test_admission_refused_when_full(sph):
    cs = _cases()
    b = _batch_for(sph, [cs["cyl"]], max_particles=cs["cyl"].n_total + 10)
    b.admit(cs["cyl"])
    with pytest.raises(sph.SphError) as e:
        b.admit(cs["tank"])
    assert e.value.status == sph.SPH_ENOMEM
    b.step(1)
    assert b.info()["n_cases"] == 1
    b.close()


def test_batch_refuses_two_fluid_materials(sph):
    # batched cases run the single-fluid-material pair path
    case = W.two_fluid_box()
    b = sph.Batch(case.n_total + 10, 2, sph.cells_of(case) + 10, history_steps=4, stream=0)
    with pytest.raises(sph.SphError) as e:
        b.admit(case)
    assert e.value.status == sph.SPH_EINVAL
    b.close()


def test_alone_equals_mixed_bitwise_two_threads_per_particle(sph):
    # the two-thread pair variant adds each list in two halves; alone (one
    # parameter-block entry) and batched (the per-slot table) still agree
    cs = _cases()
    steps = 4
    ctx = sph.from_case(cs["gear"], stream=0)
    ctx.sph_set_tuning("tpp", 2)
    ctx.sph_step(steps)
    alone = {f: ctx.sph_read_fields(f) for f in ("pos", "vel", "rho", "T")}
    alone["th"] = ctx.sph_read_torque_heat(0)
    ctx.close()
    b = _batch_for(sph, list(cs.values()))
    b.set_tuning("tpp", 2)
    slots = {k: b.admit(c, n_steps=0) for k, c in cs.items()}
    b.step(steps)
    got = {f: b.fields(slots["gear"], f) for f in ("pos", "vel", "rho", "T")}
    got["th"] = b.torque_heat(slots["gear"])
    _same(got, alone)
    b.close()
