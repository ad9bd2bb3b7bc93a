"""ctypes wrapper of the FP64 CPU oracle (test infrastructure only).

Only the tests, the package smoke check and the benchmark's CPU-baseline leg
may import this module.  It loads oracle/liborc.so (built from
sph_oracle.c by oracle/build.py) and never touches the CUDA library.
"""
from __future__ import annotations

import ctypes as C
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
if HERE not in sys.path:
    sys.path.insert(0, HERE)
import build as _build  # noqa: E402

_lib = None

D = C.c_double
I64 = C.c_int64
PD = C.POINTER(C.c_double)
PI = C.POINTER(C.c_int)
PI64 = C.POINTER(C.c_int64)
PI32 = C.POINTER(C.c_int32)


class OrcConfig(C.Structure):
    _fields_ = [("origin", D * 3), ("extent", D * 3), ("dx", D), ("h_over_dx", D),
                ("gravity", D * 3), ("c0", D), ("u_ref", D), ("cfl_ad", D), ("cfl_ac", D),
                ("free_surface", C.c_int), ("periodic_mask", C.c_int), ("max_substeps", C.c_int),
                ("viscous_heating", C.c_int), ("vstar_literal", C.c_int), ("cfl_T", D),
                ("wall_pstar_printed", C.c_int)]


class OrcRelaxConfig(C.Structure):
    _fields_ = [("dx", D), ("h_over_dx", D), ("phi", C.POINTER(D)), ("nphi", C.c_int * 3),
                ("phi_origin", D * 3), ("phi_spacing", D)]


class OrcMaterial(C.Structure):
    _fields_ = [("rho0", D), ("mu", D), ("k", D), ("cp", D), ("T_init", D), ("fixed_T", C.c_int)]


def lib():
    global _lib
    if _lib is None:
        L = C.CDLL(_build.build())
        L.orc_W.restype = D; L.orc_W.argtypes = [D, D]
        L.orc_dW.restype = D; L.orc_dW.argtypes = [D, D]
        L.orc_sigma0.restype = D; L.orc_sigma0.argtypes = [D, D]
        L.orc_riemann.argtypes = [D, D, D, D, D, D, D, PD, PD]
        L.orc_wall_riemann.argtypes = [D, D, D, D, D, D, D, C.c_int, PD, PD, PD, PD, PD]
        L.orc_timesteps.argtypes = [D, D, D, D, D, D, D, PD, PD]
        L.orc_dt_thermal.restype = D; L.orc_dt_thermal.argtypes = [D, D, D, D, D]
        L.orc_neighbors.restype = I64
        L.orc_neighbors.argtypes = [I64, PD, D, C.c_int, PD, PI64, PI32, I64]
        L.orc_relax_A.restype = D; L.orc_relax_A.argtypes = [D, D]
        L.orc_relax.restype = C.c_int
        L.orc_relax.argtypes = [C.POINTER(OrcRelaxConfig), I64, PD, C.c_int, PD]
        L.orc_neighbors_of.restype = I64
        L.orc_sample_ap.restype = C.c_int
        L.orc_sample_ap.argtypes = [I64, PD, PD, PD, PD, PD, PI, PI, C.POINTER(OrcMaterial), D, D, C.c_int, PD, D,
                                    C.c_int, D, C.c_int, PD, I64, PI64, PD]
        L.orc_sample_substep.restype = C.c_int
        L.orc_sample_substep.argtypes = [I64, PD, PD, PD, PD, PD, PI, PI, C.POINTER(OrcMaterial), D, D, C.c_int, PD,
                                         D, C.c_int, D, I64, PI64, PD, PD]
        L.orc_sample_vt.restype = C.c_int
        L.orc_sample_vt.argtypes = [I64, PD, PD, PD, PD, PI, PI, C.POINTER(OrcMaterial), D, D, C.c_int, C.c_int, PD,
                                    I64, PI64, PD, PD]
        L.orc_neighbors_of.argtypes = [I64, PD, D, C.c_int, PD, I64, PI64, PI64, PI32, I64]
        L.orc_cell_order.argtypes = [I64, PD, PD, PD, PI, PI64, PI64]
        L.orc_create.restype = C.c_void_p; L.orc_create.argtypes = [C.POINTER(OrcConfig)]
        L.orc_destroy.argtypes = [C.c_void_p]
        L.orc_set_threads.restype = C.c_int; L.orc_set_threads.argtypes = [C.c_int]
        L.orc_set_material.argtypes = [C.c_void_p, C.c_int, C.POINTER(OrcMaterial)]
        L.orc_set_rotation.argtypes = [C.c_void_p, C.c_int, PD, PD, D]
        L.orc_add_particles.argtypes = [C.c_void_p, I64, PI, PI, PI, PD, PD, PD, PD, PD]
        L.orc_step.argtypes = [C.c_void_p, C.c_int]
        L.orc_get_field.argtypes = [C.c_void_p, C.c_int, PD]
        L.orc_torque_heat.argtypes = [C.c_void_p, C.c_int, PD, PD, PD, PD]
        L.orc_body_force.argtypes = [C.c_void_p, C.c_int, PD]
        L.orc_time.argtypes = [C.c_void_p, PD, PI64, PI64, PD, PI]
        L.orc_count.restype = I64; L.orc_count.argtypes = [C.c_void_p]
        _lib = L
    return _lib


def _pd(a):
    return a.ctypes.data_as(PD)


def W(r, h):
    return lib().orc_W(float(r), float(h))


def dW(r, h):
    return lib().orc_dW(float(r), float(h))


def sigma0(dx, h):
    return lib().orc_sigma0(float(dx), float(h))


def riemann(rhoL, UL, pL, rhoR, UR, pR, c0):
    us, ps = D(), D()
    lib().orc_riemann(rhoL, UL, pL, rhoR, UR, pR, c0, C.byref(us), C.byref(ps))
    return us.value, ps.value


def wall_riemann(rho_f, UL, p_f, u_w, g_dot_rfw, rho0, c0, printed=0):
    out = [D() for _ in range(5)]
    lib().orc_wall_riemann(rho_f, UL, p_f, u_w, g_dot_rfw, rho0, c0, int(printed),
                           *[C.byref(o) for o in out])
    return dict(UR=out[0].value, PR=out[1].value, rhoR=out[2].value, Ustar=out[3].value,
                pstar=out[4].value)


def timesteps(h, vmax, u_ref, nu_max, c0, cfl_ad=0.25, cfl_ac=0.6):
    a, b = D(), D()
    lib().orc_timesteps(h, vmax, u_ref, nu_max, c0, cfl_ad, cfl_ac, C.byref(a), C.byref(b))
    return a.value, b.value


def dt_thermal(rho, cp, h, k, cfl_T=0.5):
    """Eq. (26): the thermal step bound, cfl_T rho c_p h^2 / k (0.5 as printed)."""
    return lib().orc_dt_thermal(cfl_T, rho, cp, h, k)


def set_threads(n=0):
    return lib().orc_set_threads(int(n))


def neighbors(pos, R2, periodic_mask=0, extent=(0, 0, 0)):
    """Brute-force pair lists: returns (counts[n], list) with list the
    concatenation of each particle's neighbour ids in ascending order."""
    pos = np.ascontiguousarray(pos, np.float64)
    n = len(pos)
    ext = np.ascontiguousarray(extent, np.float64)
    counts = np.zeros(n, np.int64)
    total = lib().orc_neighbors(n, _pd(pos), float(R2), int(periodic_mask), _pd(ext),
                                counts.ctypes.data_as(PI64), None, 0)
    lst = np.zeros(max(total, 1), np.int32)
    got = lib().orc_neighbors(n, _pd(pos), float(R2), int(periodic_mask), _pd(ext),
                              counts.ctypes.data_as(PI64), lst.ctypes.data_as(PI32), total)
    assert got == total
    return counts, lst[:total]


def relax_A(d, h):
    return lib().orc_relax_A(float(d), float(h))


def relax(pos, dx, h_over_dx, phi, phi_origin, phi_spacing, iterations):
    """Particle relaxation (Sec. 2.2) of pos[n, 3] in the level set phi[nz, ny, nx]
    (nodes at phi_origin + (i, j, k) phi_spacing): returns (positions, max |F_p|
    per iteration)."""
    pos = np.ascontiguousarray(pos, np.float64).copy()
    phi = np.ascontiguousarray(phi, np.float64)
    c = OrcRelaxConfig()
    c.dx, c.h_over_dx = float(dx), float(h_over_dx)
    c.phi = phi.ctypes.data_as(C.POINTER(D))
    c.nphi = (C.c_int * 3)(phi.shape[2], phi.shape[1], phi.shape[0])
    c.phi_origin = (D * 3)(*[float(v) for v in phi_origin])
    c.phi_spacing = float(phi_spacing)
    amax = np.zeros(max(int(iterations), 1), np.float64)
    assert lib().orc_relax(C.byref(c), len(pos), _pd(pos), int(iterations), _pd(amax)) == 0
    return pos, amax[:iterations]


def neighbors_of(pos, R2, idx, periodic_mask=0, extent=(0, 0, 0)):
    """Brute-force neighbour sets of the particles idx only: (counts[m], list)."""
    pos = np.ascontiguousarray(pos, np.float64)
    idx = np.ascontiguousarray(idx, np.int64)
    n, m = len(pos), len(idx)
    ext = np.ascontiguousarray(extent, np.float64)
    counts = np.zeros(m, np.int64)
    total = lib().orc_neighbors_of(n, _pd(pos), float(R2), int(periodic_mask), _pd(ext), m,
                                   idx.ctypes.data_as(PI64), counts.ctypes.data_as(PI64), None, 0)
    lst = np.zeros(max(total, 1), np.int32)
    got = lib().orc_neighbors_of(n, _pd(pos), float(R2), int(periodic_mask), _pd(ext), m,
                                 idx.ctypes.data_as(PI64), counts.ctypes.data_as(PI64),
                                 lst.ctypes.data_as(PI32), total)
    assert got == total
    return counts, lst[:total]


def sample_vt(pos, vel, rho, T, kind, mat, materials, dx, h, free_surface, idx, periodic_mask=0,
              extent=(0, 0, 0)):
    """Passes D, V and T of the fluid particles idx only, from the whole state
    at the start of an advection step (brute force at any size; see
    orc_sample_vt): (a_visc[m, 3], dT/dt[m])."""
    n = len(pos)
    pos = np.ascontiguousarray(pos, np.float64)
    vel = np.ascontiguousarray(vel, np.float64)
    rho = np.ascontiguousarray(rho, np.float64)
    T = np.ascontiguousarray(T, np.float64)
    kind = np.ascontiguousarray(kind, np.int32)
    mat = np.ascontiguousarray(mat, np.int32)
    idx = np.ascontiguousarray(idx, np.int64)
    nm = max(materials) + 1
    mats = (OrcMaterial * nm)()
    for k, m in materials.items():
        mats[k] = OrcMaterial(m["rho0"], m["mu"], m["k"], m["cp"], m["T_init"], m["fixed_T"])
    ext = np.ascontiguousarray(extent, np.float64)
    av = np.zeros((len(idx), 3))
    dT = np.zeros(len(idx))
    rc = lib().orc_sample_vt(n, _pd(pos), _pd(vel), _pd(rho), _pd(T), kind.ctypes.data_as(PI),
                             mat.ctypes.data_as(PI), mats, float(dx), float(h), int(free_surface),
                             int(periodic_mask), _pd(ext), len(idx), idx.ctypes.data_as(PI64), _pd(av), _pd(dT))
    assert rc == 0, "sample_vt: an index is out of range or not a fluid particle"
    return av, dT


def sample_ap(pos, vel, rho, drho, nrm, kind, mat, materials, dx, h, free_surface, gravity, c0, dt, idx,
              wall_pstar_printed=0, periodic_mask=0, extent=(0, 0, 0)):
    """Pass M of the fluid particles idx only, for the first acoustic sub-step
    (size dt) of an advection step, from the whole state at its start (see
    orc_sample_ap): the pressure acceleration ap[m, 3]."""
    n = len(pos)
    arr = [np.ascontiguousarray(a, np.float64) for a in (pos, vel, rho, drho, nrm)]
    kind = np.ascontiguousarray(kind, np.int32)
    mat = np.ascontiguousarray(mat, np.int32)
    idx = np.ascontiguousarray(idx, np.int64)
    nm = max(materials) + 1
    mats = (OrcMaterial * nm)()
    for k, m in materials.items():
        mats[k] = OrcMaterial(m["rho0"], m["mu"], m["k"], m["cp"], m["T_init"], m["fixed_T"])
    g = np.ascontiguousarray(gravity, np.float64)
    ext = np.ascontiguousarray(extent, np.float64)
    ap = np.zeros((len(idx), 3))
    rc = lib().orc_sample_ap(n, *[_pd(a) for a in arr], kind.ctypes.data_as(PI), mat.ctypes.data_as(PI), mats,
                             float(dx), float(h), int(free_surface), _pd(g), float(c0), int(wall_pstar_printed),
                             float(dt), int(periodic_mask), _pd(ext), len(idx), idx.ctypes.data_as(PI64), _pd(ap))
    assert rc == 0, "sample_ap: an index is out of range or not a fluid particle"
    return ap


def sample_substep(pos, vel, rho, drho, nrm, kind, mat, materials, dx, h, free_surface, gravity, c0, dt, idx,
                   wall_pstar_printed=0):
    """The first acoustic sub-step (size dt) of an advection step for the
    fluid particles idx only (see orc_sample_substep; the arrays may be the
    part of the state within three support radii of every sample): the
    kicked velocities v_new[m, 3] and pass C's rates drho_new[m]."""
    n = len(pos)
    arr = [np.ascontiguousarray(a, np.float64) for a in (pos, vel, rho, drho, nrm)]
    kind = np.ascontiguousarray(kind, np.int32)
    mat = np.ascontiguousarray(mat, np.int32)
    idx = np.ascontiguousarray(idx, np.int64)
    nm = max(materials) + 1
    mats = (OrcMaterial * nm)()
    for k, m in materials.items():
        mats[k] = OrcMaterial(m["rho0"], m["mu"], m["k"], m["cp"], m["T_init"], m["fixed_T"])
    g = np.ascontiguousarray(gravity, np.float64)
    v_new = np.zeros((len(idx), 3))
    d_new = np.zeros(len(idx))
    rc = lib().orc_sample_substep(n, *[_pd(a) for a in arr], kind.ctypes.data_as(PI), mat.ctypes.data_as(PI), mats,
                                  float(dx), float(h), int(free_surface), _pd(g), float(c0), int(wall_pstar_printed),
                                  float(dt), len(idx), idx.ctypes.data_as(PI64), _pd(v_new), _pd(d_new))
    assert rc == 0, "sample_substep: an index is out of range or not a fluid particle" if rc == -1 else \
        "sample_substep: out of host memory"
    return v_new, d_new


def cell_order(pos, origin, cellw, ncell):
    pos = np.ascontiguousarray(pos, np.float64)
    n = len(pos)
    nc = int(np.prod(ncell))
    perm = np.zeros(n, np.int64)
    cs = np.zeros(nc + 1, np.int64)
    o = np.ascontiguousarray(origin, np.float64)
    w = np.ascontiguousarray(cellw, np.float64)
    g = np.ascontiguousarray(ncell, np.int32).astype(np.intc)
    lib().orc_cell_order(n, _pd(pos), _pd(o), _pd(w), g.ctypes.data_as(PI),
                         perm.ctypes.data_as(PI64), cs.ctypes.data_as(PI64))
    return perm, cs


FIELD = dict(pos=(0, 3), vel=(1, 3), rho=(2, 1), p=(3, 1), T=(4, 1), drho=(5, 1), a_visc=(6, 3),
             dTdt=(7, 1), sigma=(8, 1), normal=(9, 3), wall_vel=(10, 3), contact=(11, 1),
             rho_reinit=(12, 1))


class OracleSim:
    """One oracle simulation built from a workloads.Case."""

    def __init__(self, case, threads=0):
        L = lib()
        if threads:
            L.orc_set_threads(int(threads))
        cfg = case.config
        oc = OrcConfig()
        oc.origin = (D * 3)(*cfg["origin"]); oc.extent = (D * 3)(*cfg["extent"])
        oc.dx = cfg["dx"]; oc.h_over_dx = cfg["h_over_dx"]
        oc.gravity = (D * 3)(*cfg["gravity"]); oc.c0 = cfg["c0"]; oc.u_ref = cfg["u_ref"]
        oc.cfl_ad = cfg["cfl_ad"]; oc.cfl_ac = cfg["cfl_ac"]
        oc.free_surface = cfg["free_surface"]; oc.periodic_mask = cfg["periodic_mask"]
        oc.max_substeps = cfg.get("max_substeps", 0)
        oc.viscous_heating = cfg.get("viscous_heating", 0)
        oc.vstar_literal = cfg.get("vstar_literal", 0)
        oc.cfl_T = cfg.get("cfl_T", 0.5)
        oc.wall_pstar_printed = cfg.get("wall_pstar_printed", 0)
        self._p = L.orc_create(C.byref(oc))
        for mid, m in case.materials.items():
            om = OrcMaterial(m["rho0"], m["mu"], m["k"], m["cp"], m["T_init"], m["fixed_T"])
            assert L.orc_set_material(self._p, int(mid), C.byref(om)) == 0
        for bid, b in case.bodies.items():
            c = np.asarray(b["center"], np.float64); a = np.asarray(b["axis"], np.float64)
            L.orc_set_rotation(self._p, int(bid), _pd(c), _pd(a), float(b["omega"]))
        from paper_2512_09904_b300.workloads import flatten
        f = flatten(case)
        self.n = len(f["kind"])
        self.kind = f["kind"]
        arr = lambda x, t: np.ascontiguousarray(x, t)
        kind, mat, body = arr(f["kind"], np.intc), arr(f["mat"], np.intc), arr(f["body"], np.intc)
        pos, vel, nrm = arr(f["pos"], np.float64), arr(f["vel"], np.float64), arr(f["normal"], np.float64)
        T, rho = arr(f["T"], np.float64), arr(f["rho"], np.float64)
        rc = L.orc_add_particles(self._p, self.n, kind.ctypes.data_as(PI), mat.ctypes.data_as(PI),
                                 body.ctypes.data_as(PI), _pd(pos), _pd(vel), _pd(nrm), _pd(T), _pd(rho))
        assert rc == 0, rc

    def step(self, n=1):
        lib().orc_step(self._p, int(n))

    def field(self, name):
        fid, k = FIELD[name]
        out = np.zeros(self.n * k, np.float64)
        assert lib().orc_get_field(self._p, fid, _pd(out)) == 0
        return out.reshape(self.n, 3) if k == 3 else out

    def torque_heat(self, body=0):
        v = [D() for _ in range(4)]
        lib().orc_torque_heat(self._p, int(body), *[C.byref(x) for x in v])
        return dict(torque=v[0].value, torque_avg=v[1].value, heat=v[2].value, mean_T=v[3].value)

    def body_force(self, body=0):
        f = np.zeros(3)
        lib().orc_body_force(self._p, int(body), _pd(f))
        return f

    def time(self):
        t, dt = D(), D()
        a, s = C.c_int64(), C.c_int64()
        ns = C.c_int()
        lib().orc_time(self._p, C.byref(t), C.byref(a), C.byref(s), C.byref(dt), C.byref(ns))
        return dict(t=t.value, adv_steps=a.value, substeps=s.value, dt_ad=dt.value, nsub=ns.value)

    def close(self):
        if self._p:
            lib().orc_destroy(self._p)
            self._p = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
