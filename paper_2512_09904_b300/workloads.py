"""Seeded synthetic inputs shaped like the paper's gearbox workloads.

This module only lays particles out (lattice positions, jitter, wall normals,
initial fields) and fills parameter tables.  It holds none of the SPH method's
arithmetic, so both the CUDA path and the CPU oracle can take its output as
their common input.

Workload shapes follow the paper: a lubricant bath churned by a rigid spur
gear (Sec. 4, Table 5: shaft speeds 150-600 rad/s, fill depth, viscosity;
Table 6: lubricant and gear properties),
a still oil tank, a thermal dam break, and the two-material slab of the heat
conduction validation (Sec. 3.2, Table 3).  No CAD, dataset or measured curve
of the paper is used: every geometry here is analytic.

Units are SI; temperatures in kelvin.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

FLUID, SOLID = 0, 1


@dataclass
class Case:
    """One simulation case: config table, materials, bodies and particle blocks.

    config keys: origin[3], extent[3], dx, h_over_dx, gravity[3], c0, u_ref,
    cfl_ad, cfl_ac, cfl_T, free_surface, periodic_mask, max_substeps.
    materials: {id: dict(rho0, mu, k, cp, T_init, fixed_T)}
    fluids: list of dict(mat, pos[n,3], vel[n,3]|None, T[n]|None, rho[n]|None)
    solids: list of dict(body, mat, pos[n,3], normal[n,3], T[n]|None)
    bodies: {id: dict(center[3], axis[3], omega)}
    Particle ids are assigned in block order: all fluid blocks first, then
    all solid blocks.
    """

    name: str
    config: dict
    materials: dict
    fluids: list
    solids: list
    bodies: dict = field(default_factory=dict)
    meta: dict = field(default_factory=dict)

    @property
    def n_fluid(self) -> int:
        return int(sum(len(b["pos"]) for b in self.fluids))

    @property
    def n_solid(self) -> int:
        return int(sum(len(b["pos"]) for b in self.solids))

    @property
    def n_total(self) -> int:
        return self.n_fluid + self.n_solid

    def support_radius(self) -> float:
        return 2.0 * self.config["h_over_dx"] * self.config["dx"]


def _cfg(origin, extent, dx, *, h_over_dx=1.3, gravity=(0.0, 0.0, -9.81), c0=10.0,
         u_ref=None, free_surface=1, periodic_mask=0, max_substeps=0):
    return dict(origin=[float(v) for v in origin], extent=[float(v) for v in extent],
                dx=float(dx), h_over_dx=float(h_over_dx),
                gravity=[float(v) for v in gravity], c0=float(c0),
                u_ref=float(c0 / 10.0 if u_ref is None else u_ref),
                cfl_ad=0.25, cfl_ac=0.6, cfl_T=0.5, free_surface=int(free_surface),
                periodic_mask=int(periodic_mask), max_substeps=int(max_substeps))


def _mat(rho0, mu, k, cp, T_init, fixed_T=0):
    return dict(rho0=float(rho0), mu=float(mu), k=float(k), cp=float(cp),
                T_init=float(T_init), fixed_T=int(fixed_T))


def _grid(lo, hi):
    """Integer lattice indices lo <= idx < hi per axis, flattened x-fastest."""
    ax = [np.arange(lo[d], hi[d]) for d in range(3)]
    k, j, i = np.meshgrid(ax[2], ax[1], ax[0], indexing="ij")
    return np.stack([i.ravel(), j.ravel(), k.ravel()], axis=1)


def _jitter(rng, n, dx, amp):
    return rng.uniform(-amp, amp, size=(n, 3)) * dx


def _box_walls(nx, ny, nz_wall, layers, lid):
    """Lattice indices of a wall shell around the box [0,nx)x[0,ny)x[0,nz_wall).

    Returns (idx, inward) where inward is the unnormalised inward direction.
    """
    top = nz_wall + (layers if lid else 0)
    idx = _grid((-layers, -layers, -layers), (nx + layers, ny + layers, top))
    i, j, k = idx[:, 0], idx[:, 1], idx[:, 2]
    inside = (i >= 0) & (i < nx) & (j >= 0) & (j < ny) & (k >= 0) & (k < nz_wall)
    idx = idx[~inside]
    i, j, k = idx[:, 0], idx[:, 1], idx[:, 2]
    d = np.zeros((len(idx), 3))
    d[:, 0] = (i < 0).astype(float) - (i >= nx).astype(float)
    d[:, 1] = (j < 0).astype(float) - (j >= ny).astype(float)
    d[:, 2] = (k < 0).astype(float) - (k >= nz_wall).astype(float)
    return idx, d


def _unit(v):
    n = np.linalg.norm(v, axis=1, keepdims=True)
    n[n == 0] = 1.0
    return v / n


def _hydrostatic_rho(rho0, g, H, z, c0):
    # Initial condition only: the still column's density from p = rho0 g (H - z)
    # mapped through the linear equation of state.
    return rho0 + rho0 * g * (H - z) / (c0 * c0)


# --------------------------------------------------------------------------
# Still oil tank (plain-method FP64 case): 32x32x16 oil, 3 steel layers.
# --------------------------------------------------------------------------
def still_tank(nx=32, ny=32, nz=16, dx=1e-3, layers=3, wall_h=24, seed=1, jitter=0.01,
               rho0=870.0, mu=0.05, c0=10.0, g=9.81, T_oil=313.15, T_hot=353.15):
    rng = np.random.default_rng(seed)
    fidx = _grid((0, 0, 0), (nx, ny, nz))
    fpos = (fidx + 0.5) * dx + _jitter(rng, len(fidx), dx, jitter)
    H = nz * dx
    rho = _hydrostatic_rho(rho0, g, H, fpos[:, 2], c0)
    widx, inward = _box_walls(nx, ny, wall_h, layers, lid=False)
    wpos = (widx + 0.5) * dx
    wn = _unit(inward)
    bottom = widx[:, 2] < 0
    mats = {0: _mat(rho0, mu, 0.13, 2000.0, T_oil),
            1: _mat(7850.0, 0.0, 45.0, 460.0, T_hot, fixed_T=1),
            2: _mat(7850.0, 0.0, 0.0, 460.0, T_oil, fixed_T=1)}
    margin = 4
    cfg = _cfg(origin=(-layers * dx,) * 3,
               extent=((nx + 2 * layers) * dx, (ny + 2 * layers) * dx, (wall_h + layers + margin) * dx),
               dx=dx, c0=c0, gravity=(0, 0, -g))
    solids = [dict(body=-1, mat=1, pos=wpos[bottom], normal=wn[bottom], T=None),
              dict(body=-1, mat=2, pos=wpos[~bottom], normal=wn[~bottom], T=None)]
    fluids = [dict(mat=0, pos=fpos, vel=None, T=None, rho=rho)]
    return Case("still_tank", cfg, mats, fluids, solids, {},
                dict(H=H, rho0=rho0, g=g, seed=seed, nx=nx, ny=ny, nz=nz))


# --------------------------------------------------------------------------
# Thermal dam break: oil column 0.2x0.1x0.2 m in a closed 0.6x0.1x0.4 m tank.
# --------------------------------------------------------------------------
def dam_break(dx=2e-3, seed=2, jitter=0.01, layers=3, rho0=870.0, mu=0.05, g=9.81,
              T_oil=298.15, T_wall=333.15, tank=(0.6, 0.1, 0.4), column=(0.2, 0.1, 0.2)):
    rng = np.random.default_rng(seed)
    n_t = [int(round(t / dx)) for t in tank]
    n_c = [int(round(c / dx)) for c in column]
    H = n_c[2] * dx
    c0 = 10.0 * math.sqrt(2.0 * g * H)
    fidx = _grid((0, 0, 0), tuple(n_c))
    fpos = (fidx + 0.5) * dx + _jitter(rng, len(fidx), dx, jitter)
    rho = _hydrostatic_rho(rho0, g, H, fpos[:, 2], c0)
    widx, inward = _box_walls(n_t[0], n_t[1], n_t[2], layers, lid=True)
    mats = {0: _mat(rho0, mu, 0.13, 2000.0, T_oil),
            1: _mat(7850.0, 0.0, 45.0, 460.0, T_wall, fixed_T=1)}
    cfg = _cfg(origin=(-layers * dx,) * 3,
               extent=tuple((n + 2 * layers) * dx for n in n_t), dx=dx, c0=c0, gravity=(0, 0, -g))
    solids = [dict(body=-1, mat=1, pos=(widx + 0.5) * dx, normal=_unit(inward), T=None)]
    fluids = [dict(mat=0, pos=fpos, vel=None, T=None, rho=rho)]
    return Case("dam_break", cfg, mats, fluids, solids, {}, dict(H=H, seed=seed, c0=c0))


# --------------------------------------------------------------------------
# Rotating spur gear half-immersed in an oil sump (gear-bath family).
# --------------------------------------------------------------------------
GEAR = dict(r_pitch=0.050, teeth=24, face=0.020, pressure_angle_deg=20.0)


def _gear_inside(px, pz, r_p, z_teeth, pa, phase=0.0):
    """Inside test of a spur gear with straight-flanked (trapezoidal) teeth.

    px, pz: coordinates in the gear plane relative to the axis.  Module
    m = 2 r_p / z; tip radius r_p + m; root radius r_p - 1.25 m; the tooth
    half-thickness is pi m / 4 at the pitch circle and narrows with the
    pressure angle.  Teeth are centred at angles phase + k 2 pi / z.
    """
    m = 2.0 * r_p / z_teeth
    r_a, r_f = r_p + m, r_p - 1.25 * m
    rr = np.hypot(px, pz)
    phi = np.arctan2(pz, px) - phase
    pitch = 2.0 * math.pi / z_teeth
    dphi = np.abs((phi + 0.5 * pitch) % pitch - 0.5 * pitch)
    half = math.pi * m / 4.0 - (rr - r_p) * math.tan(math.radians(pa))
    tooth = (rr <= r_a) & (rr * np.sin(dphi) <= half) & (dphi < 0.5 * pitch)
    return (rr <= r_f) | tooth


def gear_bath(dx=1e-3, omega=600.0, depth_frac=0.5, mu=0.1, scale=1.5, seed=3, jitter=0.01,
              layers=3, gear_layers=3, rho0=968.1, k_oil=0.15, cp_oil=2000.0, T_oil=298.15,
              T_gear=318.15, g=9.81, gear=None):
    """Steel spur gear (pitch radius 50 mm, 24 teeth, face 20 mm, axis along y)
    in a closed sump 0.16x0.06x0.14 m scaled by `scale` per axis, filled to
    `depth_frac` x tip diameter above the gear's lowest point.  Lubricant and
    gear properties follow the paper's property table (Table 6).  `gear`
    overrides r_pitch / teeth / face (a geometrically similar smaller case).
    """
    rng = np.random.default_rng(seed)
    G = dict(GEAR, **(gear or {}))
    r_p, z_t, b = G["r_pitch"], G["teeth"], G["face"]
    m = 2.0 * r_p / z_t
    r_a = r_p + m
    L = np.array([0.16, 0.06, 0.14]) * scale
    n = [int(round(v / dx)) for v in L]
    Lx, Ly, Lz = (np.array(n) * dx)
    c = np.array([Lx / 2, Ly / 2, Lz / 2])
    z_fill = (c[2] - r_a) + depth_frac * 2.0 * r_a

    gpos, gnrm = _gear_shell(c, G, dx, n, gear_layers)

    # fluid: lattice points below the fill level outside the gear body
    fidx = _grid((0, 0, 0), (n[0], n[1], int(math.ceil(z_fill / dx))))
    fpos0 = (fidx + 0.5) * dx
    fpos0 = fpos0[fpos0[:, 2] < z_fill]
    rel = fpos0 - c
    in_gear = _gear_inside(rel[:, 0], rel[:, 2], r_p, z_t, G["pressure_angle_deg"]) & (np.abs(rel[:, 1]) <= b / 2)
    fpos0 = fpos0[~in_gear]
    fpos = fpos0 + _jitter(rng, len(fpos0), dx, jitter)
    u_tip = omega * r_a
    c0 = 10.0 * max(u_tip, math.sqrt(2 * g * z_fill))
    rho = _hydrostatic_rho(rho0, g, z_fill, fpos[:, 2], c0)

    widx, inward = _box_walls(n[0], n[1], n[2], layers, lid=True)
    mats = {0: _mat(rho0, mu, k_oil, cp_oil, T_oil),
            1: _mat(7850.0, 0.0, 20.0, 460.0, T_gear, fixed_T=1),
            2: _mat(7850.0, 0.0, 0.0, 460.0, T_oil, fixed_T=1)}
    cfg = _cfg(origin=(-layers * dx,) * 3, extent=tuple((v + 2 * layers) * dx for v in n),
               dx=dx, c0=c0, u_ref=c0 / 10.0, gravity=(0, 0, -g))
    solids = [dict(body=-1, mat=2, pos=(widx + 0.5) * dx, normal=_unit(inward), T=None),
              dict(body=0, mat=1, pos=gpos, normal=gnrm, T=None)]
    fluids = [dict(mat=0, pos=fpos, vel=None, T=None, rho=rho)]
    bodies = {0: dict(center=c.tolist(), axis=[0.0, 1.0, 0.0], omega=float(omega))}
    return Case("gear_bath", cfg, mats, fluids, solids, bodies,
                dict(omega=omega, depth_frac=depth_frac, mu=mu, dx=dx, z_fill=z_fill, r_tip=r_a,
                     seed=seed, scale=scale))


def _gear_shell(c, G, dx, n, gear_layers, phase=0.0):
    """Lattice particles of a gear's outer shell (gear_layers deep) and their
    normals from the gradient of the lattice signed distance."""
    from scipy import ndimage

    r_p, z_t, b = G["r_pitch"], G["teeth"], G["face"]
    r_a = r_p + 2.0 * r_p / z_t
    lo = np.floor((c - np.array([r_a, b / 2, r_a])) / dx).astype(int) - 2
    hi = np.ceil((c + np.array([r_a, b / 2, r_a])) / dx).astype(int) + 3
    lo = np.maximum(lo, 0)
    hi = np.minimum(hi, n)
    shape = tuple(hi - lo)
    gp = (_grid(tuple(lo), tuple(hi)) + 0.5) * dx
    inside = _gear_inside(gp[:, 0] - c[0], gp[:, 2] - c[2], r_p, z_t, G["pressure_angle_deg"], phase)
    inside &= np.abs(gp[:, 1] - c[1]) <= b / 2
    vol = inside.reshape(shape[2], shape[1], shape[0])  # (k, j, i)
    depth_in = ndimage.distance_transform_edt(vol)
    sdf = ndimage.distance_transform_edt(~vol) - depth_in  # >0 outside, <0 inside (lattice units)
    gz, gy, gx = np.gradient(sdf)
    keep = (vol & (depth_in <= gear_layers)).ravel()
    return gp[keep], _unit(np.stack([gx.ravel()[keep], gy.ravel()[keep], gz.ravel()[keep]], axis=1))


def gear_pair(dx=2.5e-3, omega=300.0, depth_frac=0.5, mu=0.1, seed=13, jitter=0.01, layers=3, gear_layers=3,
              rho0=968.1, k_oil=0.15, cp_oil=2000.0, T_oil=298.15, T_gear=318.15, g=9.81):
    """A meshing gear pair in one sump (a two-shaft gear train): driver of 24
    teeth (pitch radius 30 mm) and follower of 16 teeth (20 mm), module
    2.5 mm, face 12 mm, axes along y 50 mm apart at the same height; the
    follower turns at -omega 24/16 with its teeth phased into the driver's
    gaps on the line of centres.  Oil (Table 6 properties) fills the sump to
    depth_frac of the driver's tip diameter above its lowest point."""
    rng = np.random.default_rng(seed)
    G1 = dict(GEAR, r_pitch=0.030, teeth=24, face=0.012)
    G2 = dict(GEAR, r_pitch=0.020, teeth=16, face=0.012)
    ra1 = G1["r_pitch"] * (1 + 2.0 / G1["teeth"])
    ra2 = G2["r_pitch"] * (1 + 2.0 / G2["teeth"])
    L = np.array([0.15, 0.03, 0.09])
    n = [int(round(v / dx)) for v in L]
    Lx, Ly, Lz = (np.array(n) * dx)
    c1 = np.array([0.045, Ly / 2, Lz / 2])
    c2 = c1 + np.array([G1["r_pitch"] + G2["r_pitch"], 0.0, 0.0])
    pitch2 = 2.0 * math.pi / G2["teeth"]
    phase2 = math.pi - 0.5 * pitch2  # a follower gap faces the driver's tooth at angle 0
    p1, n1 = _gear_shell(c1, G1, dx, n, gear_layers)
    p2, n2 = _gear_shell(c2, G2, dx, n, gear_layers, phase2)
    z_fill = (c1[2] - ra1) + depth_frac * 2.0 * ra1
    fidx = _grid((0, 0, 0), (n[0], n[1], int(math.ceil(z_fill / dx))))
    fpos0 = (fidx + 0.5) * dx
    fpos0 = fpos0[fpos0[:, 2] < z_fill]
    in1 = _gear_inside(fpos0[:, 0] - c1[0], fpos0[:, 2] - c1[2], G1["r_pitch"], G1["teeth"],
                       G1["pressure_angle_deg"]) & (np.abs(fpos0[:, 1] - c1[1]) <= G1["face"] / 2)
    in2 = _gear_inside(fpos0[:, 0] - c2[0], fpos0[:, 2] - c2[2], G2["r_pitch"], G2["teeth"],
                       G2["pressure_angle_deg"], phase2) & (np.abs(fpos0[:, 1] - c2[1]) <= G2["face"] / 2)
    fpos0 = fpos0[~(in1 | in2)]
    fpos = fpos0 + _jitter(rng, len(fpos0), dx, jitter)
    omega2 = -omega * G1["teeth"] / G2["teeth"]
    c0 = 10.0 * max(omega * ra1, abs(omega2) * ra2, math.sqrt(2 * g * z_fill))
    rho = _hydrostatic_rho(rho0, g, z_fill, fpos[:, 2], c0)
    widx, inward = _box_walls(n[0], n[1], n[2], layers, lid=True)
    mats = {0: _mat(rho0, mu, k_oil, cp_oil, T_oil),
            1: _mat(7850.0, 0.0, 20.0, 460.0, T_gear, fixed_T=1),
            2: _mat(7850.0, 0.0, 0.0, 460.0, T_oil, fixed_T=1)}
    cfg = _cfg(origin=(-layers * dx,) * 3, extent=tuple((v + 2 * layers) * dx for v in n),
               dx=dx, c0=c0, u_ref=c0 / 10.0, gravity=(0, 0, -g))
    solids = [dict(body=-1, mat=2, pos=(widx + 0.5) * dx, normal=_unit(inward), T=None),
              dict(body=0, mat=1, pos=p1, normal=n1, T=None),
              dict(body=1, mat=1, pos=p2, normal=n2, T=None)]
    fluids = [dict(mat=0, pos=fpos, vel=None, T=None, rho=rho)]
    bodies = {0: dict(center=c1.tolist(), axis=[0.0, 1.0, 0.0], omega=float(omega)),
              1: dict(center=c2.tolist(), axis=[0.0, 1.0, 0.0], omega=float(omega2))}
    return Case("gear_pair", cfg, mats, fluids, solids, bodies,
                dict(omega=omega, omega2=omega2, dx=dx, z_fill=z_fill, seed=seed))


def perturbed(case, seed, amp=1e-9):
    """The case with every fluid position moved by a seeded normal offset of
    standard deviation amp x dx per coordinate (far below FP32 rounding of the
    pair geometry at the default): a sibling trajectory for measuring how
    fast a splashing flow forgets its initial state."""
    rng = np.random.default_rng(seed)
    sd = amp * case.config["dx"]
    for f in case.fluids:
        f["pos"] = f["pos"] + rng.normal(0.0, sd, size=f["pos"].shape)
    case.meta = dict(case.meta, perturb_seed=seed, perturb_amp=amp)
    return case


def gear_bath_dx_for(n_fluid_target, depth_frac=0.5, scale=1.5):
    """Lattice spacing that gives about n_fluid_target oil particles."""
    r_p, b = GEAR["r_pitch"], GEAR["face"]
    r_a = r_p + 2.0 * r_p / GEAR["teeth"]
    L = np.array([0.16, 0.06, 0.14]) * scale
    z_fill = (L[2] / 2 - r_a) + depth_frac * 2.0 * r_a
    v = L[0] * L[1] * z_fill - math.pi * r_p * r_p * b * min(max(depth_frac, 0.0), 1.0)
    return float((v / n_fluid_target) ** (1.0 / 3.0))


def mini_gear_bath(omega=300.0, dx=1.5e-3, depth_frac=0.5, mu=0.1, seed=9):
    """The gear bath shrunk by 5 (pitch radius 10 mm, 24 teeth of module
    0.83 mm, face 4 mm, sump 48x18x42 mm) at a coarse lattice: a case small
    enough for the O(N^2) oracle over 1000 advection steps."""
    return gear_bath(dx=dx, omega=omega, depth_frac=depth_frac, mu=mu, scale=0.3, seed=seed,
                     gear=dict(r_pitch=GEAR["r_pitch"] / 5, face=GEAR["face"] / 5))


def contact_probe(fill="full", rho_factor=1.0, dx=1e-3, n=9):
    """One rigid-body particle at the centre lattice point of an n^3 oil
    lattice block, at rest, no gravity.  fill selects the oil around it:
    'full' (every other lattice point), 'above' / 'below' (lattice points with
    z above / below the particle's), 'plane' (its own z plane), 'none'.  The
    oil density is rho_factor x rho0 everywhere."""
    idx = _grid((0, 0, 0), (n, n, n))
    c = n // 2
    sel = np.any(idx != c, axis=1)
    if fill == "above":
        sel &= idx[:, 2] > c
    elif fill == "below":
        sel &= idx[:, 2] < c
    elif fill == "plane":
        sel &= idx[:, 2] == c
    elif fill == "none":
        sel &= False
    fpos = (idx[sel] + 0.5) * dx
    rho0 = 900.0
    cfg = _cfg(origin=(-2 * dx,) * 3, extent=((n + 4) * dx,) * 3, dx=dx, gravity=(0, 0, 0), c0=10.0)
    mats = {0: _mat(rho0, 0.05, 0.15, 2000.0, 300.0), 1: _mat(7850.0, 0.0, 0.0, 460.0, 300.0, fixed_T=1)}
    center = (np.array([c, c, c]) + 0.5) * dx
    fluids = [dict(mat=0, pos=fpos, vel=None, T=None, rho=np.full(len(fpos), rho_factor * rho0))] if len(fpos) else []
    solids = [dict(body=0, mat=1, pos=center[None, :], normal=np.array([[0.0, 0.0, 1.0]]), T=None)]
    bodies = {0: dict(center=list(center + np.array([0.0, 0.0, -5 * dx])), axis=[0.0, 1.0, 0.0], omega=0.0)}
    return Case("contact_probe", cfg, mats, fluids, solids, bodies)


def flow_block(field="shear", rate=20.0, n=14, dx=1e-3, viscous_heating=1, mu=0.1, seed=None):
    """An n^3 oil lattice with a prescribed velocity field and uniform
    temperature, no gravity, no walls: 'shear' v = (rate z, 0, 0), 'rotation'
    v = rate e_z x r (rigid), 'translation' v = (rate dx, 0, 0) per unit time.
    For the viscous-dissipation term: its interior particles see a complete
    kernel support."""
    idx = _grid((0, 0, 0), (n, n, n))
    pos = (idx + 0.5) * dx
    c = 0.5 * n * dx
    vel = np.zeros_like(pos)
    if field == "shear":
        vel[:, 0] = rate * (pos[:, 2] - c)
    elif field == "rotation":
        vel[:, 0] = -rate * (pos[:, 1] - c)
        vel[:, 1] = rate * (pos[:, 0] - c)
    elif field == "translation":
        vel[:, 0] = rate * dx
    cfg = _cfg(origin=(-2 * dx,) * 3, extent=((n + 4) * dx,) * 3, dx=dx, gravity=(0, 0, 0), c0=10.0)
    cfg["viscous_heating"] = int(viscous_heating)
    mats = {0: _mat(900.0, mu, 0.0, 2000.0, 300.0)}
    fluids = [dict(mat=0, pos=pos, vel=vel, T=None, rho=None)]
    return Case("flow_block", cfg, mats, fluids, [], {}, dict(rate=rate, field=field))


def relax_body(shape="sphere", size=10e-3, dx=1e-3, h_over_dx=1.3, phi_step=None, offset=0.5):
    """A body for the particle relaxation of Sec. 2.2: its level set sampled on
    a grid (negative inside) and the lattice seeds inside it.

    shape 'sphere' (radius `size`) or 'box' (half width `size`, faces half a
    spacing beyond the outermost lattice points); the body is centred at the
    origin; lattice points at (k + offset) dx.  Returns a dict with pos[n, 3],
    phi[nz, ny, nx], phi_origin, phi_spacing, dx, h_over_dx."""
    step = phi_step or 0.5 * dx
    pad = 3.0 * h_over_dx * dx
    half = int(math.ceil((size + pad) / step))  # nodes on each side of the centre: a symmetric grid
    lo = -half * step
    m = 2 * half + 1
    ax = step * np.arange(-half, half + 1)
    Z, Y, X = np.meshgrid(ax, ax, ax, indexing="ij")
    if shape == "sphere":
        phi = np.sqrt(X ** 2 + Y ** 2 + Z ** 2) - size
    elif shape == "box":
        q = np.abs(np.stack([X, Y, Z])) - size
        outside = np.linalg.norm(np.maximum(q, 0.0), axis=0)
        phi = outside + np.minimum(np.max(q, axis=0), 0.0)
    else:
        raise ValueError(shape)
    k = int(math.ceil(size / dx)) + 1
    g = (np.arange(-k, k + 1) + offset) * dx
    P = np.stack(np.meshgrid(g, g, g, indexing="ij"), axis=-1).reshape(-1, 3)
    if shape == "sphere":
        inside = np.linalg.norm(P, axis=1) < size
    else:
        inside = np.all(np.abs(P) < size, axis=1)
    return dict(pos=P[inside], phi=phi, phi_origin=[lo, lo, lo], phi_spacing=step, dx=dx, h_over_dx=h_over_dx)


# --------------------------------------------------------------------------
# Two-material slab of the conduction validation (Sec. 3.2, Table 3):
# x in [0,1], interface x=0.5, T=0 left / 1 right; periodic in y and z.
# --------------------------------------------------------------------------
def slab(dx=0.0125, h_over_dx=1.3, n_yz=8, dt_ad=0.02):
    nx = int(round(1.0 / dx))
    idx = _grid((0, 0, 0), (nx, n_yz, n_yz))
    pos = (idx + 0.5) * dx
    left = pos[:, 0] < 0.5
    h = h_over_dx * dx
    # no fluid: the advective bound alone fixes dt_ad = 0.25 h / u_ref
    u_ref = 0.25 * h / dt_ad
    cfg = _cfg(origin=(0, 0, 0), extent=(nx * dx, n_yz * dx, n_yz * dx), dx=dx,
               h_over_dx=h_over_dx, gravity=(0, 0, 0), c0=10.0 * u_ref, u_ref=u_ref,
               periodic_mask=0b110)
    mats = {0: _mat(1000.0, 0.0, 1.0, 1.0, 0.0), 1: _mat(2000.0, 0.0, 3.0, 1.0, 1.0)}
    nrm = np.tile([0.0, 0.0, 1.0], (len(pos), 1))
    solids = [dict(body=-1, mat=0, pos=pos[left], normal=nrm[left], T=np.zeros(left.sum())),
              dict(body=-1, mat=1, pos=pos[~left], normal=nrm[~left], T=np.ones((~left).sum()))]
    return Case("slab", cfg, mats, [], solids, {}, dict(dt_ad=dt_ad))


# --------------------------------------------------------------------------
# Periodic fluid box (momentum-conservation and field-parity case, g = 0).
# --------------------------------------------------------------------------
def periodic_box(n=12, dx=1e-3, seed=7, jitter=0.05, v_amp=0.2, rho_amp=2e-3, rho0=1000.0,
                 mu=0.02, c0=10.0, periodic_mask=0b111):
    rng = np.random.default_rng(seed)
    idx = _grid((0, 0, 0), (n, n, n))
    pos = (idx + 0.5) * dx + _jitter(rng, len(idx), dx, jitter)
    vel = rng.uniform(-v_amp, v_amp, size=(len(idx), 3))
    rho = rho0 * (1.0 + rng.uniform(-rho_amp, rho_amp, size=len(idx)))
    T = 300.0 + rng.uniform(-5.0, 5.0, size=len(idx))
    cfg = _cfg(origin=(0, 0, 0), extent=(n * dx,) * 3, dx=dx, c0=c0, gravity=(0, 0, 0),
               periodic_mask=periodic_mask)
    mats = {0: _mat(rho0, mu, 0.6, 4000.0, 300.0)}
    fluids = [dict(mat=0, pos=pos, vel=vel, T=T, rho=rho)]
    return Case("periodic_box", cfg, mats, fluids, [], {}, dict(seed=seed))


# --------------------------------------------------------------------------
# Two fluids in a periodic box: water (x < L/2) beside oil, different density,
# viscosity, conductivity and temperature (the pair passes' general-material
# path: harmonic means of mu and k, per-partner masses and rest densities).
# --------------------------------------------------------------------------
def two_fluid_box(n=12, dx=1e-3, seed=19, jitter=0.05, v_amp=0.1, c0=10.0):
    rng = np.random.default_rng(seed)
    idx = _grid((0, 0, 0), (n, n, n))
    pos = (idx + 0.5) * dx + _jitter(rng, len(idx), dx, jitter)
    left = pos[:, 0] < 0.5 * n * dx
    vel = rng.uniform(-v_amp, v_amp, size=(len(idx), 3))
    cfg = _cfg(origin=(0, 0, 0), extent=(n * dx,) * 3, dx=dx, c0=c0, gravity=(0, 0, 0), periodic_mask=0b111)
    mats = {0: _mat(1000.0, 0.01, 0.6, 4180.0, 300.0), 1: _mat(870.0, 0.1, 0.15, 2000.0, 320.0)}
    fluids = [dict(mat=0, pos=pos[left], vel=vel[left], T=None, rho=None),
              dict(mat=1, pos=pos[~left], vel=vel[~left], T=None, rho=None)]
    return Case("two_fluid_box", cfg, mats, fluids, [], {}, dict(seed=seed))


# --------------------------------------------------------------------------
# Crowded periodic box: a lattice with extra particles at the cube centres of
# a central block (locally body-centred, twice the density), where a particle
# has about 147 partners, more than a 128-entry neighbour list holds; the
# rest of the box has the lattice's 80.  At rest, g = 0.
# --------------------------------------------------------------------------
def crowded_box(n=14, crowd=8, dx=1e-3, seed=17, jitter=0.02, rho0=1000.0, mu=0.02, c0=10.0):
    rng = np.random.default_rng(seed)
    idx = _grid((0, 0, 0), (n, n, n))
    lo = (n - crowd) // 2
    cidx = _grid((lo, lo, lo), (lo + crowd, lo + crowd, lo + crowd))
    pos = np.concatenate([(idx + 0.5) * dx, (cidx + 1.0) * dx])
    pos = pos + _jitter(rng, len(pos), dx, jitter)
    cfg = _cfg(origin=(0, 0, 0), extent=(n * dx,) * 3, dx=dx, c0=c0, gravity=(0, 0, 0), periodic_mask=0b111)
    mats = {0: _mat(rho0, mu, 0.6, 4000.0, 300.0)}
    fluids = [dict(mat=0, pos=pos, vel=None, T=None, rho=None)]
    return Case("crowded_box", cfg, mats, fluids, [], {}, dict(seed=seed, crowd=crowd))


# --------------------------------------------------------------------------
# Neighbour-search stress input: random points plus pairs placed within a few
# ulps of the support radius, on both sides of it.
# --------------------------------------------------------------------------
def cutoff_pairs(n_random=2000, n_pairs=400, dx=1e-3, h_over_dx=1.3, box=24, seed=11):
    rng = np.random.default_rng(seed)
    R = 2.0 * h_over_dx * dx
    L = box * dx
    pts = [rng.uniform(0.1 * L, 0.9 * L, size=(n_random, 3))]
    a = rng.uniform(0.3 * L, 0.7 * L, size=(n_pairs, 3))
    u = _unit(rng.normal(size=(n_pairs, 3)))
    ulps = rng.integers(-4, 5, size=n_pairs).astype(float)
    d = R * (1.0 + ulps * np.finfo(np.float64).eps)
    pts += [a, a + u * d[:, None]]
    pos = np.concatenate(pts)
    cfg = _cfg(origin=(0, 0, 0), extent=(L, L, L), dx=dx, h_over_dx=h_over_dx, gravity=(0, 0, 0))
    mats = {0: _mat(1000.0, 0.01, 0.6, 4000.0, 300.0)}
    return Case("cutoff_pairs", cfg, mats, [dict(mat=0, pos=pos, vel=None, T=None, rho=None)], [], {},
                dict(seed=seed))


def cell_boundaries(n_random=3000, n_edge=3000, dx=1e-3, h_over_dx=1.3, box=24,
                    origin=(-0.0123, 0.0456, 1.0), seed=12):
    """Particles on sort-cell boundaries: one coordinate at origin + k w_a
    (FP64, w_a the engine's sort-cell width along axis a, extent /
    (s_a floor(extent / 2h)) with s = 8 along x and 2 along y and z) or a
    few ulps either side, the others uniform; plus uniform particles.  The
    cell hash's FP32 estimate must hand every such particle to its FP64
    rule.  The origin is away from zero so that |o| enters the estimate's
    error."""
    rng = np.random.default_rng(seed)
    L = box * dx
    o = np.asarray(origin, np.float64)
    ng = int(np.floor(L / (2.0 * h_over_dx * dx)))
    ns = [s * ng for s in (8, 2, 2)]
    w = [L / n for n in ns]
    lo, hi = o + 1e-3 * L, o + (1.0 - 1e-3) * L
    pts = [rng.uniform(lo, hi, size=(n_random, 3))]
    e = rng.uniform(lo, hi, size=(n_edge, 3))
    axis = rng.integers(0, 3, size=n_edge)
    u = rng.random(n_edge)
    ulps = rng.integers(-2, 3, size=n_edge)
    for i in range(n_edge):
        a = axis[i]
        k = float(1 + int(u[i] * (ns[a] - 1)))  # 1 .. ns[a] - 1
        x = o[a] + k * w[a]
        for _ in range(abs(int(ulps[i]))):
            x = np.nextafter(x, np.inf if ulps[i] > 0 else -np.inf)
        e[i, a] = x
    pts.append(e)
    pos = np.concatenate(pts)
    cfg = _cfg(origin=tuple(o), extent=(L, L, L), dx=dx, h_over_dx=h_over_dx, gravity=(0, 0, 0))
    mats = {0: _mat(1000.0, 0.01, 0.6, 4000.0, 300.0)}
    return Case("cell_boundaries", cfg, mats, [dict(mat=0, pos=pos, vel=None, T=None, rho=None)], [], {},
                dict(seed=seed, sort_cell_width=w))


def long_channel(n_clumps=8, side=6, dx=0.5e-3, length=0.7, seed=14):
    """Oil clumps (side^3 jittered lattices, a temperature ramp, small random
    velocities) spread along a channel of `length` m, 12 dx wide and high, no
    gravity or walls.  At the defaults the channel has 538 geometry cells
    along x (more than the engine tabulates corners for), so the snapshot
    offsets take their arithmetic form."""
    rng = np.random.default_rng(seed)
    w = 12 * dx
    lat = _grid((0, 0, 0), (side, side, side)).astype(np.float64)
    xs = np.linspace(0.02, length - 0.01, n_clumps)
    pos, T, vel = [], [], []
    for x0 in xs:
        p = (lat - (side - 1) / 2.0) * dx + np.array([x0, w / 2, w / 2])
        pos.append(p + _jitter(rng, len(p), dx, 0.02))
        T.append(300.0 + 10.0 * lat[:, 0] / (side - 1))
        vel.append(rng.normal(scale=0.02, size=p.shape))
    cfg = _cfg(origin=(0, 0, 0), extent=(length, w, w), dx=dx, gravity=(0, 0, 0), c0=10.0, u_ref=1.0)
    mats = {0: _mat(900.0, 0.02, 0.15, 2000.0, 300.0)}
    fl = [dict(mat=0, pos=np.concatenate(pos), vel=np.concatenate(vel), T=np.concatenate(T), rho=None)]
    return Case("long_channel", cfg, mats, fl, [], {}, dict(seed=seed))


# --------------------------------------------------------------------------
# Sweep / serving request streams (parameter grid of the paper's case table).
# --------------------------------------------------------------------------
SWEEP_OMEGA = (150.0, 300.0, 450.0, 600.0)
SWEEP_DEPTH = (0.25, 0.5, 0.75)
SWEEP_MU = (0.03, 0.1, 0.3)


def sweep_cases(n_cases=64, seed=4, mu_ln=math.log(158e3), sigma_ln=0.576, lo=50e3, hi=500e3,
                count_scale=1.0):
    """Batched-sweep request list: lognormal oil counts, grid cells round-robin
    from a seeded shuffle.  count_scale shrinks every case (tests)."""
    rng = np.random.default_rng(seed)
    grid = [(w, d, m) for w in SWEEP_OMEGA for d in SWEEP_DEPTH for m in SWEEP_MU]
    order = rng.permutation(len(grid))
    counts = np.clip(rng.lognormal(mu_ln, sigma_ln, size=n_cases), lo, hi) * count_scale
    out = []
    for c in range(n_cases):
        w, d, m = grid[order[c % len(grid)]]
        out.append(dict(omega=w, depth_frac=d, mu=m, n_fluid=int(counts[c]),
                        dx=gear_bath_dx_for(counts[c], d), seed=1000 + c))
    return out


def serving_trace(n_requests=256, seed=5, rate=4.0, mu_ln=math.log(200e3), sigma_ln=1.15,
                  lo=20e3, hi=2e6, steps=2000, count_scale=1.0):
    """Poisson arrival stream of gear-bath requests (arrival time in s)."""
    rng = np.random.default_rng(seed)
    grid = [(w, d, m) for w in SWEEP_OMEGA for d in SWEEP_DEPTH for m in SWEEP_MU]
    t = np.cumsum(rng.exponential(1.0 / rate, size=n_requests))
    counts = np.clip(rng.lognormal(mu_ln, sigma_ln, size=n_requests), lo, hi) * count_scale
    cells = rng.integers(0, len(grid), size=n_requests)
    out = []
    for r in range(n_requests):
        w, d, m = grid[cells[r]]
        out.append(dict(arrival=float(t[r]), omega=w, depth_frac=d, mu=m, n_fluid=int(counts[r]),
                        dx=gear_bath_dx_for(counts[r], d), steps=int(steps), seed=5000 + r))
    return out


def flatten(case: Case):
    """Concatenate the case's blocks in id order (fluids first, then solids).

    Returns dict with kind[n], mat[n], body[n], pos[n,3], vel[n,3], T[n],
    rho[n] (NaN = material rho0), normal[n,3].
    """
    kinds, mats, bodies, pos, vel, T, rho, nrm = [], [], [], [], [], [], [], []
    for b in case.fluids:
        n = len(b["pos"])
        kinds.append(np.full(n, FLUID, np.int32))
        mats.append(np.full(n, b["mat"], np.int32))
        bodies.append(np.full(n, -1, np.int32))
        pos.append(np.asarray(b["pos"], np.float64))
        vel.append(np.zeros((n, 3)) if b.get("vel") is None else np.asarray(b["vel"], np.float64))
        T.append(np.full(n, case.materials[b["mat"]]["T_init"]) if b.get("T") is None else np.asarray(b["T"], np.float64))
        rho.append(np.full(n, np.nan) if b.get("rho") is None else np.asarray(b["rho"], np.float64))
        nrm.append(np.zeros((n, 3)))
    for b in case.solids:
        n = len(b["pos"])
        kinds.append(np.full(n, SOLID, np.int32))
        mats.append(np.full(n, b["mat"], np.int32))
        bodies.append(np.full(n, b["body"], np.int32))
        pos.append(np.asarray(b["pos"], np.float64))
        vel.append(np.zeros((n, 3)))
        T.append(np.full(n, case.materials[b["mat"]]["T_init"]) if b.get("T") is None else np.asarray(b["T"], np.float64))
        rho.append(np.full(n, np.nan))
        nrm.append(np.asarray(b["normal"], np.float64))
    cat = lambda xs, shape: np.concatenate(xs) if xs else np.zeros(shape)
    return dict(kind=cat(kinds, (0,)).astype(np.int32), mat=cat(mats, (0,)).astype(np.int32),
                body=cat(bodies, (0,)).astype(np.int32), pos=cat(pos, (0, 3)), vel=cat(vel, (0, 3)),
                T=cat(T, (0,)), rho=cat(rho, (0,)), normal=cat(nrm, (0, 3)))


# --------------------------------------------------------------------------
# Rotating rigid cylinder in a periodic fluid box (axis along z): a compact
# rigid-body coupling case (wall pressure, wall viscosity, torque).
# --------------------------------------------------------------------------
def rotating_cylinder(n=16, dx=1e-3, radius_dx=4.0, layers=3, omega=50.0, mu=0.05, rho0=900.0,
                      seed=8, jitter=0.01, T_fluid=300.0, T_solid=320.0, k_fluid=0.15):
    rng = np.random.default_rng(seed)
    idx = _grid((0, 0, 0), (n, n, n))
    pos = (idx + 0.5) * dx
    c = np.array([n * dx / 2, n * dx / 2, n * dx / 2])
    rr = np.hypot(pos[:, 0] - c[0], pos[:, 1] - c[1])
    Rc = radius_dx * dx
    solid = rr <= Rc
    shell = solid & (rr > Rc - layers * dx)
    fl = ~solid
    fpos = pos[fl] + _jitter(rng, int(fl.sum()), dx, jitter)
    nrm = np.zeros((int(shell.sum()), 3))
    nrm[:, 0] = pos[shell, 0] - c[0]
    nrm[:, 1] = pos[shell, 1] - c[1]
    nrm = _unit(nrm)
    u_tip = abs(omega) * Rc
    c0 = 10.0 * max(u_tip, 0.05)
    cfg = _cfg(origin=(0, 0, 0), extent=(n * dx,) * 3, dx=dx, c0=c0, gravity=(0, 0, 0),
               periodic_mask=0b111)
    mats = {0: _mat(rho0, mu, k_fluid, 2000.0, T_fluid), 1: _mat(7850.0, 0.0, 20.0, 460.0, T_solid, fixed_T=1)}
    fluids = [dict(mat=0, pos=fpos, vel=None, T=None, rho=None)]
    solids = [dict(body=0, mat=1, pos=pos[shell], normal=nrm, T=None)]
    bodies = {0: dict(center=c.tolist(), axis=[0.0, 0.0, 1.0], omega=float(omega))}
    return Case("rotating_cylinder", cfg, mats, fluids, solids, bodies, dict(seed=seed, radius=Rc))
