"""The 2M-oil gear bath of the bench, in the launch configuration bench.py
times (autotuned pair-pass variant): pair sets of a seeded sample of
particles checked bit-exact against the oracle's brute-force search over all
2.8M snapshot positions, plus pair symmetry on the sample; the held viscous
acceleration and dT/dt of sampled oil particles against the oracle's
brute-force passes D, V and T on the same state; the velocity kick of pass M
(one acoustic sub-step per step) against the oracle's sampled passes; and, at the same
particle count, a property that holds at any size: a periodic lattice moving
as a rigid whole keeps its velocity (Galilean invariance)."""
import numpy as np
import pytest

from paper_2512_09904_b300 import workloads as W

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


@pytest.fixture(scope="module")
def sph():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_2512_09904_b300 import build
    build.build()
    from paper_2512_09904_b300 import sph as S
    return S


def test_gear_bath_2m_sampled_pair_sets(sph, oracle):
    case = W.gear_bath(dx=1e-3, omega=600.0)
    ctx = sph.from_case(case, stream=0)
    ctx.sph_step(1)
    ctx.sph_autotune(steps_per_trial=1)
    ctx.sph_step(2)
    pos = ctx.sph_read_fields("pos")  # the snapshot of the next advection step
    ctx.sph_step(1)
    counts, lst = ctx.sph_read_neighbors()
    start = np.concatenate([[0], np.cumsum(counts)])
    n = case.n_total
    rng = np.random.default_rng(12)
    kind = W.flatten(case)["kind"]
    # oil, static walls and gear particles all represented
    idx = np.concatenate([rng.choice(np.nonzero(kind == 0)[0], 160, replace=False),
                          rng.choice(np.nonzero(kind != 0)[0], 96, replace=False)])
    R2 = case.support_radius() ** 2
    rc, rl = oracle.neighbors_of(pos, R2, idx, case.config["periodic_mask"], case.config["extent"])
    off = 0
    for q, i in enumerate(idx):
        got = lst[start[i]:start[i + 1]]
        ref = rl[off:off + rc[q]]
        off += rc[q]
        assert np.array_equal(got, ref), (int(i), len(got), len(ref))
        # symmetry: i is a partner of each of its partners
        for j in got[:8]:
            assert i in lst[start[j]:start[j + 1]]
    assert counts[idx].sum() == rc.sum() > 50 * len(idx)
    ctx.close()


def test_galilean_invariance_at_full_size(sph):
    # a perfect periodic lattice of 140^3 = 2,744,000 particles (the bench's
    # particle count) moving as a rigid whole, in the pair-pass variant the
    # autotuner picks on the bench: it keeps its velocity and is carried by
    # it, within the field-parity norm 1e-5 (k + 1) of u_ref and dx
    n, steps, dx = 140, 5, 1e-3
    v0 = np.array([0.3, -0.2, 0.1])
    idx = W._grid((0, 0, 0), (n, n, n))
    pos = (idx + 0.5) * dx
    cfg = W._cfg(origin=(0, 0, 0), extent=(n * dx,) * 3, dx=dx, c0=10.0, gravity=(0, 0, 0), periodic_mask=0b111)
    case = W.Case("translating_lattice_full", cfg, {0: W._mat(1000.0, 0.02, 0.6, 4000.0, 300.0)},
                  [dict(mat=0, pos=pos, vel=np.tile(v0, (len(pos), 1)), T=None, rho=None)], [])
    ctx = sph.from_case(case, stream=0)
    for key, val in (("list_batch", 2), ("tpp", 1), ("block", 128)):
        ctx.sph_set_tuning(key, val)
    ctx.sph_step(steps)
    t = ctx.sph_get_info()["t"]
    v = ctx.sph_read_fields("vel")
    d = ctx.sph_read_fields("pos") - (pos + v0 * t)
    d -= n * dx * np.round(d / (n * dx))
    ev, ex = np.abs(v - v0).max() / cfg["u_ref"], np.abs(d).max() / dx
    print(f"TRANSLATION n={n ** 3} steps={steps} vel={ev:.2e} pos={ex:.2e}")
    assert ev <= 1e-5 * (steps + 1) and ex <= 1e-5 * (steps + 1)
    ctx.close()


def test_gear_bath_2m_sampled_viscous_and_heat(sph, oracle):
    # passes D, V and T at full size, in the bench's launch configuration: the
    # whole state read back at the start of an advection step, then that
    # step's held viscous acceleration (Eqs. 10, 18) and dT/dt (Eq. 22) of 32
    # oil particles (16 in the bulk, 16 beside the hot rotating gear) against
    # the oracle's brute-force passes on the same state (its own kernel sums
    # for the re-initialised densities, Eq. 14), within the field-parity norm
    # 1e-5 relative to max(|x_ref|, s), s the largest sampled magnitude (and g
    # for the acceleration)
    from scipy.spatial import cKDTree
    case = W.gear_bath(dx=1e-3, omega=600.0)
    ctx = sph.from_case(case, stream=0)
    for key, val in (("list_batch", 2), ("tpp", 1), ("block", 128)):
        ctx.sph_set_tuning(key, val)
    ctx.sph_step(3)
    pos, vel, rho, T = (ctx.sph_read_fields(k) for k in ("pos", "vel", "rho", "T"))
    ctx.sph_step(1)
    av, dT = ctx.sph_read_fields("a_visc"), ctx.sph_read_fields("dTdt")
    ctx.close()
    f = W.flatten(case)
    fluid = np.flatnonzero(f["kind"] == 0)
    gear = np.flatnonzero(f["body"] >= 0)
    near = fluid[cKDTree(pos[gear]).query(pos[fluid], distance_upper_bound=2e-3)[0] < 2e-3]
    rng = np.random.default_rng(21)
    idx = np.sort(np.concatenate([rng.choice(fluid, 16, replace=False), rng.choice(near, 16, replace=False)]))
    cfg = case.config
    ref_av, ref_dT = oracle.sample_vt(pos, vel, rho, T, f["kind"], f["mat"], case.materials, cfg["dx"],
                                      cfg["h_over_dx"] * cfg["dx"], cfg["free_surface"], idx)
    s_a = max(9.81, np.abs(ref_av).max())
    s_T = np.abs(ref_dT).max()
    ea = np.abs(av[idx] - ref_av).max(1) / np.maximum(np.abs(ref_av).max(1), s_a)
    eT = np.abs(dT[idx] - ref_dT) / np.maximum(np.abs(ref_dT), s_T)
    print(f"SAMPLED_VT a_visc={ea.max():.2e} dTdt={eT.max():.2e} s_a={s_a:.3g} s_T={s_T:.3g}")
    assert s_T > 0.0
    assert ea.max() <= 1e-5 and eT.max() <= 1e-5


def test_gear_bath_2m_sampled_pressure_kick(sph, oracle):
    # pass M at full size, in the bench's launch configuration, with one
    # acoustic sub-step per advection step: the state read back at the start
    # of a step (the gear's particles at their current angle, with normals and
    # wall velocities; drho for the half kick), then the velocities after that
    # step against v + dt (a_p + a_visc + g) from the oracle's brute-force
    # passes (pressure: Eqs. 10-12, 16-19; viscous: Eqs. 10, 18) for 32 oil
    # particles, 16 of them beside the rotating gear.  Bound: 1e-5 of the
    # largest sampled velocity change, plus the FP32 rounding of the stored
    # velocity (2^-24 |v|)
    from scipy.spatial import cKDTree
    case = W.gear_bath(dx=1e-3, omega=600.0)
    case.config = dict(case.config, max_substeps=1)
    ctx = sph.from_case(case, stream=0)
    for key, val in (("list_batch", 2), ("tpp", 1), ("block", 128)):
        ctx.sph_set_tuning(key, val)
    ctx.sph_step(3)
    t0 = ctx.sph_get_info()["t"]
    pos, vel, rho, drho, T, nrm = (ctx.sph_read_fields(k) for k in ("pos", "vel", "rho", "drho", "T", "normal"))
    ctx.sph_step(1)
    dt = ctx.sph_get_info()["t"] - t0
    v2, x2 = ctx.sph_read_fields("vel"), ctx.sph_read_fields("pos")
    ctx.close()
    f = W.flatten(case)
    fluid = np.flatnonzero(f["kind"] == 0)
    gear = np.flatnonzero(f["body"] >= 0)
    near = fluid[cKDTree(pos[gear]).query(pos[fluid], distance_upper_bound=2e-3)[0] < 2e-3]
    rng = np.random.default_rng(22)
    idx = np.sort(np.concatenate([rng.choice(fluid, 16, replace=False), rng.choice(near, 16, replace=False)]))
    cfg = case.config
    h = cfg["h_over_dx"] * cfg["dx"]
    ap = oracle.sample_ap(pos, vel, rho, drho, nrm, f["kind"], f["mat"], case.materials, cfg["dx"], h,
                          cfg["free_surface"], cfg["gravity"], cfg["c0"], dt, idx)
    av, _ = oracle.sample_vt(pos, vel, rho, T, f["kind"], f["mat"], case.materials, cfg["dx"], h,
                             cfg["free_surface"], idx)
    dv = dt * (ap + av + np.asarray(cfg["gravity"]))
    v_ref = vel[idx] + dv
    x_ref = pos[idx] + 0.5 * dt * (vel[idx] + v_ref)
    bound = 1e-5 * np.abs(dv).max() + 2.0 ** -24 * np.abs(v_ref)
    ev = np.abs(v2[idx] - v_ref)
    print(f"SAMPLED_M dv_max={np.abs(dv).max():.3g} err/bound={np.max(ev / bound):.2e} "
          f"err/dv_max={ev.max() / np.abs(dv).max():.2e} x={np.abs(x2[idx] - x_ref).max() / cfg['dx']:.2e}")
    assert np.all(ev <= bound)
    assert np.abs(x2[idx] - x_ref).max() <= 1e-5 * cfg["dx"]
