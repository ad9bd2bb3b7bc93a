"""Degenerate cases of the method on the CUDA path (through the C ABI):

- a lone fluid particle (no partners): free fall, v = -g t and
  z = z0 - g t^2 / 2, with its density, temperature and the other axes
  untouched bit for bit;
- two fluid particles closing head on: step-by-step parity with the oracle,
  equal and opposite velocities and a fixed midpoint (to FP32 rounding);
- a perfect periodic lattice moving as a rigid whole (41^3 = 68,921 particles,
  many blocks and a ragged last one): it keeps its velocity and is carried by it
  (Galilean invariance), a property that holds at any size.

Floating-point bounds follow the field-parity norm, 1e-5 (k + 1) relative to
max(|x_ref|, s_field) after k advection steps, unless stated.
"""
import numpy as np
import pytest

from paper_2512_09904_b300 import workloads as W

pytestmark = pytest.mark.gpu

TOL = 1e-5
DX = 1e-3


@pytest.fixture(scope="module")
def sph():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_2512_09904_b300 import build
    build.build()
    from paper_2512_09904_b300 import sph as S
    return S


def _lone(g):
    cfg = W._cfg(origin=(0, 0, 0), extent=(0.1, 0.1, 0.1), dx=DX, gravity=(0, 0, -g))
    return W.Case("lone", cfg, {0: W._mat(870.0, 0.1, 0.15, 2000.0, 300.0)},
                  [dict(mat=0, pos=np.array([[0.05, 0.05, 0.05]]), vel=None, T=None, rho=None)], [])


def _head_on_pair(u, gap=DX):
    pos = np.array([[0.05 - 0.5 * gap, 0.05, 0.05], [0.05 + 0.5 * gap, 0.05, 0.05]])
    vel = np.array([[u, 0.0, 0.0], [-u, 0.0, 0.0]])
    cfg = W._cfg(origin=(0, 0, 0), extent=(0.1, 0.1, 0.1), dx=DX, c0=10.0, gravity=(0, 0, 0))
    return W.Case("head_on_pair", cfg, {0: W._mat(1000.0, 1e-3, 0.6, 4000.0, 300.0)},
                  [dict(mat=0, pos=pos, vel=vel, T=None, rho=None)], [])


def _lattice(n, v0):
    idx = W._grid((0, 0, 0), (n, n, n))
    pos = (idx + 0.5) * DX
    cfg = W._cfg(origin=(0, 0, 0), extent=(n * DX,) * 3, dx=DX, c0=10.0, gravity=(0, 0, 0), periodic_mask=0b111)
    vel = np.tile(np.asarray(v0, float), (len(pos), 1))
    return W.Case("translating_lattice", cfg, {0: W._mat(1000.0, 0.02, 0.6, 4000.0, 300.0)},
                  [dict(mat=0, pos=pos, vel=vel, T=None, rho=None)], [])


def test_lone_particle_free_fall(sph, oracle):
    g, steps = 9.81, 20
    case = _lone(g)
    ctx = sph.from_case(case, stream=0)
    ctx.sph_step(steps)
    t = ctx.sph_get_info()["t"]
    x, v = ctx.sph_read_fields("pos")[0], ctx.sph_read_fields("vel")[0]
    ref = oracle.OracleSim(case)
    ref.step(steps)
    assert t == pytest.approx(ref.time()["t"], rel=1e-6)
    # velocity: one FP32 multiply-add of dt g per sub-step (about 100 of them)
    assert v[2] == pytest.approx(-g * t, rel=TOL)
    assert v[0] == 0.0 and v[1] == 0.0
    # position: FP64 half drifts of the FP32 velocities
    fall = 0.5 * g * t * t
    assert abs(x[2] - (0.05 - fall)) <= TOL * fall
    assert x[0] == 0.05 and x[1] == 0.05
    # no partner: the density excess stays 0 (Eq. 14 keeps the larger value)
    # and no heat flows
    assert ctx.sph_read_fields("rho")[0] == 870.0
    assert ctx.sph_read_fields("T")[0] == 300.0
    ctx.close()


def test_head_on_pair_parity_and_symmetry(sph, oracle):
    u, steps = 0.1, 8
    case = _head_on_pair(u)
    ctx = sph.from_case(case, stream=0)
    ref = oracle.OracleSim(case)
    for k in range(steps):
        ctx.sph_step(1)
        ref.step(1)
        assert ctx.sph_get_info()["last_nsub"] == ref.time()["nsub"]
        x, v, rho = ctx.sph_read_fields("pos"), ctx.sph_read_fields("vel"), ctx.sph_read_fields("rho")
        xr, vr, rr = ref.field("pos"), ref.field("vel"), ref.field("rho")
        bound = TOL * (k + 1)
        assert np.abs(v - vr).max() <= bound * max(np.abs(vr).max(), case.config["u_ref"])
        assert np.abs(x - xr).max() <= bound * DX
        drho = rho - 1000.0
        assert np.abs(drho - (rr - 1000.0)).max() <= bound * max(np.abs(rr - 1000.0).max(), 1000.0 * 0.01)
        # the two particles see the pair from either side, each from its own
        # FP32 cell offsets: the mirror holds to FP32 rounding, at the norm's
        # bound relative to the pair's speed u (and the midpoint to that
        # speed times the elapsed time); across the axis the pair offsets are
        # zero up to the rounding of the pre-shifted FP32 cell offsets, so the
        # same bound holds there
        t = ctx.sph_get_info()["t"]
        dv, dyz = abs(v[0, 0] + v[1, 0]), np.abs(v[:, 1:]).max()
        print(f"MIRROR step={k + 1} dv={dv / u:.2e} v_yz={dyz / u:.2e}")
        assert dv <= bound * u and dyz <= bound * u
        assert abs(x[0, 0] + x[1, 0] - 0.1) <= bound * u * t + 1e-15
        assert np.abs(x[:, 1:] - 0.05).max() <= bound * u * t + 1e-15
    ctx.close()


def test_uniform_translation_of_a_large_lattice(sph):
    n, steps = 41, 20
    v0 = np.array([0.3, -0.2, 0.1])
    case = _lattice(n, v0)
    x0 = W.flatten(case)["pos"].copy()
    ctx = sph.from_case(case, stream=0)
    ctx.sph_step(steps)
    t = ctx.sph_get_info()["t"]
    v = ctx.sph_read_fields("vel")
    d = ctx.sph_read_fields("pos") - (x0 + v0 * t)
    d -= n * DX * np.round(d / (n * DX))
    ev = np.abs(v - v0).max() / case.config["u_ref"]
    ex = np.abs(d).max() / DX
    print(f"TRANSLATION n={n ** 3} steps={steps} vel={ev:.2e} pos={ex:.2e}")
    assert ev <= TOL * (steps + 1)
    assert ex <= TOL * (steps + 1)
    ctx.close()
