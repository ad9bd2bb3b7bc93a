"""Thin ctypes binding of the C ABI in include/sph.h (same names).

Only argument marshalling lives here: every step of the SPH path runs in the
CUDA library libsph_b300.so.  Importing this module fails loudly if the
library has not been built; there is no fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libsph_b300.so")

D = C.c_double
I64 = C.c_int64
PD = C.POINTER(C.c_double)
PI64 = C.POINTER(C.c_int64)
PI32 = C.POINTER(C.c_int32)

SPH_OK, SPH_EINVAL, SPH_ENOMEM, SPH_ECUDA, SPH_EUNSTABLE, SPH_ETIMEOUT, SPH_ESTATE = 0, -1, -2, -3, -4, -5, -6
STATUS = {0: "SPH_OK", -1: "SPH_EINVAL", -2: "SPH_ENOMEM", -3: "SPH_ECUDA", -4: "SPH_EUNSTABLE",
          -5: "SPH_ETIMEOUT", -6: "SPH_ESTATE"}
TUNE = dict(list_batch=0, tpp=1, block=2)
PROF_CLASSES = ("sort", "pass_D", "pass_VT", "pass_M", "pass_C", "control", "adv_end", "idle")
FIELDS = dict(pos=(0, 3), vel=(1, 3), rho=(2, 1), p=(3, 1), T=(4, 1), drho=(5, 1), a_visc=(6, 3),
              dTdt=(7, 1), normal=(9, 3), contact=(11, 1))


class sph_config(C.Structure):
    _fields_ = [("origin", D * 3), ("extent", D * 3), ("dx", D), ("h_over_dx", D), ("gravity", D * 3),
                ("c0", D), ("u_ref", D), ("cfl_ad", D), ("cfl_ac", D), ("free_surface", C.c_int),
                ("periodic_mask", C.c_int), ("max_substeps", C.c_int), ("pair_precision", C.c_int),
                ("viscous_heating", C.c_int), ("vstar_literal", C.c_int), ("cfl_T", D),
                ("wall_pstar_printed", C.c_int)]


class sph_material(C.Structure):
    _fields_ = [("rho0", D), ("mu", D), ("k", D), ("cp", D), ("T_init", D), ("fixed_T", C.c_int)]


class sph_info(C.Structure):
    _fields_ = [("n_fluid", I64), ("n_solid", I64), ("t", D), ("adv_steps", I64), ("substeps", I64),
                ("last_dt_ad", D), ("last_nsub", C.c_int), ("kcap", C.c_int), ("ncell", C.c_int * 3),
                ("cell_width", D * 3), ("error_bits", C.c_int), ("graph_launches", C.c_int),
                ("kernels_fixed", C.c_int), ("kernels_per_substep", C.c_int), ("info_bits", C.c_int)]


class sph_relax_config(C.Structure):
    _fields_ = [("dx", D), ("h_over_dx", D), ("phi", C.POINTER(D)), ("nphi", C.c_int * 3),
                ("phi_origin", D * 3), ("phi_spacing", D)]


class sph_tune_report(C.Structure):
    _fields_ = [("list_batch", C.c_int), ("tpp", C.c_int), ("block", C.c_int), ("ms_step_start", D),
                ("ms_step_chosen", D), ("substeps_ref", D), ("trials", C.c_int), ("steps", I64)]


class sph_batch_config(C.Structure):
    _fields_ = [("max_particles", I64), ("max_cases", C.c_int), ("max_cells", I64), ("history_steps", C.c_int)]


BATCH_RUNNING, BATCH_DONE, BATCH_UNSTABLE = 0, 1, -4
CURVE_FIELDS = ("t", "torque", "torque_avg", "heat", "mean_T", "dt_ad", "nsub", "vmax")


class SphError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


_lib = None


def lib():
    """Load libsph_b300.so (raises if it is missing: no CPU fallback)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} not built; run python -m paper_2512_09904_b300.build")
        L = C.CDLL(LIB_PATH)
        vp = C.c_void_p
        L.sph_create.argtypes = [C.POINTER(sph_config), vp, C.POINTER(vp)]
        L.sph_destroy.argtypes = [vp]
        L.sph_set_material.argtypes = [vp, C.c_int, C.POINTER(sph_material)]
        L.sph_add_fluid.argtypes = [vp, C.c_int, I64, PD, PD, PD, PD, PI64]
        L.sph_add_solid.argtypes = [vp, C.c_int, C.c_int, I64, PD, PD, PD, PI64]
        L.sph_set_rotation.argtypes = [vp, C.c_int, PD, PD, D]
        L.sph_step.argtypes = [vp, C.c_int, PD]
        L.sph_read_torque_heat.argtypes = [vp, C.c_int, PD, PD, PD, PD]
        L.sph_read_fields.argtypes = [vp, C.c_int, vp, I64]
        L.sph_read_neighbors.argtypes = [vp, PI64, PI32, I64, PI64]
        L.sph_read_cell_order.argtypes = [vp, PI64, I64]
        L.sph_get_info.argtypes = [vp, C.POINTER(sph_info)]
        L.sph_last_error.argtypes = [vp]
        L.sph_last_error.restype = C.c_char_p
        L.sph_cell_sort.argtypes = [vp, I64, PD, PD, C.POINTER(C.c_int), vp, vp, vp]
        L.sph_profile.argtypes = [vp, C.c_int]
        L.sph_pair_stats.argtypes = [vp, PI64, PI64]
        L.sph_search_stats.argtypes = [vp, PI64, PI64, PI64]
        L.sph_set_tuning.argtypes = [vp, C.c_int, C.c_int]
        L.sph_batch_bytes.argtypes = [C.POINTER(sph_batch_config)]
        L.sph_batch_bytes.restype = I64
        L.sph_batch_create.argtypes = [C.POINTER(sph_batch_config), vp, C.POINTER(vp)]
        L.sph_batch_destroy.argtypes = [vp]
        L.sph_batch_last_error.argtypes = [vp]
        L.sph_batch_last_error.restype = C.c_char_p
        L.sph_batch_admit.argtypes = [vp, vp, I64, C.POINTER(C.c_int)]
        L.sph_batch_step.argtypes = [vp, C.c_int]
        L.sph_batch_poll.argtypes = [vp, C.c_int, PI64, PD, C.POINTER(C.c_int)]
        L.sph_batch_read_torque_heat.argtypes = [vp, C.c_int, C.c_int, PD, PD, PD, PD]
        L.sph_batch_read_curve.argtypes = [vp, C.c_int, PD, I64, PI64]
        L.sph_read_curve.argtypes = [vp, PD, I64, PI64]
        L.sph_batch_read_fields.argtypes = [vp, C.c_int, C.c_int, vp, I64]
        L.sph_batch_retire.argtypes = [vp, C.c_int]
        L.sph_batch_info.argtypes = [vp, PI64, C.POINTER(C.c_int), C.POINTER(C.c_int)]
        L.sph_batch_set_tuning.argtypes = [vp, C.c_int, C.c_int]
        L.sph_batch_profile.argtypes = [vp, C.c_int]
        L.sph_batch_profile_read.argtypes = [vp, PD, PI64, C.c_int]
        L.sph_get_tuning.argtypes = [vp, C.c_int, C.POINTER(C.c_int)]
        L.sph_cell_sort_noalloc.argtypes = [vp, I64, PD, PD, C.POINTER(C.c_int), vp, vp, vp]
        L.sph_profile_read.argtypes = [vp, PD, PI64, C.c_int]
        L.sph_autotune.argtypes = [vp, C.c_int, C.POINTER(sph_tune_report)]
        L.sph_relax.argtypes = [C.POINTER(sph_relax_config), I64, PD, C.c_int, vp, PD]
        L.sph_batch_autotune.argtypes = [vp, C.c_int, C.POINTER(sph_tune_report)]
        L.sph_fma_peak.argtypes = [vp, C.c_int, PD, PD]
        for name in ("sph_create", "sph_destroy", "sph_set_material", "sph_add_fluid", "sph_add_solid",
                     "sph_set_rotation", "sph_step", "sph_read_torque_heat", "sph_read_curve", "sph_read_fields",
                     "sph_read_neighbors", "sph_read_cell_order", "sph_get_info", "sph_cell_sort",
                     "sph_profile", "sph_profile_read", "sph_pair_stats", "sph_cell_sort_noalloc",
                     "sph_set_tuning", "sph_get_tuning", "sph_batch_create", "sph_batch_destroy",
                     "sph_batch_admit", "sph_batch_step", "sph_batch_poll", "sph_batch_read_torque_heat",
                     "sph_batch_read_curve", "sph_batch_read_fields", "sph_batch_retire", "sph_batch_info",
                     "sph_batch_set_tuning", "sph_batch_profile", "sph_batch_profile_read"):
            getattr(L, name).restype = C.c_int
        _lib = L
    return _lib


def _pd(a):
    return None if a is None else a.ctypes.data_as(PD)


def _f64(a, shape=None):
    if a is None:
        return None
    a = np.ascontiguousarray(a, dtype=np.float64)
    if shape is not None:
        a = a.reshape(shape)
    return a


def current_stream_handle():
    """cudaStream_t of torch's current stream (0 if torch/CUDA is unavailable)."""
    try:
        import torch
        if torch.cuda.is_available():
            return int(torch.cuda.current_stream().cuda_stream)
    except Exception:
        pass
    return 0


def config_from_dict(cfg: dict) -> sph_config:
    c = sph_config()
    c.origin = (D * 3)(*cfg["origin"])
    c.extent = (D * 3)(*cfg["extent"])
    c.dx = cfg["dx"]
    c.h_over_dx = cfg["h_over_dx"]
    c.gravity = (D * 3)(*cfg["gravity"])
    c.c0 = cfg["c0"]
    c.u_ref = cfg["u_ref"]
    c.cfl_ad = cfg["cfl_ad"]
    c.cfl_ac = cfg["cfl_ac"]
    c.free_surface = cfg["free_surface"]
    c.periodic_mask = cfg["periodic_mask"]
    c.max_substeps = cfg.get("max_substeps", 0)
    c.pair_precision = cfg.get("pair_precision", 0)
    c.viscous_heating = cfg.get("viscous_heating", 0)
    c.vstar_literal = cfg.get("vstar_literal", 0)
    c.cfl_T = cfg.get("cfl_T", 0.5)
    c.wall_pstar_printed = cfg.get("wall_pstar_printed", 0)
    return c


class Context:
    """One sph_ctx (single case)."""

    def __init__(self, cfg: dict, stream: int | None = None):
        self._L = lib()
        self._keep = []
        p = C.c_void_p()
        self.stream = current_stream_handle() if stream is None else int(stream)
        self._check(self._L.sph_create(C.byref(config_from_dict(cfg)), C.c_void_p(self.stream), C.byref(p)),
                    "sph_create")
        self._p = p
        self.n = 0

    def _check(self, rc, what):
        if rc != SPH_OK:
            msg = self._L.sph_last_error(self._p).decode() if getattr(self, "_p", None) else what
            raise SphError(rc, f"{what}: {msg}")

    def sph_set_material(self, mid, m: dict):
        sm = sph_material(m["rho0"], m["mu"], m["k"], m["cp"], m["T_init"], m["fixed_T"])
        self._check(self._L.sph_set_material(self._p, int(mid), C.byref(sm)), "sph_set_material")

    def sph_add_fluid(self, mat, pos, vel=None, T=None, rho=None):
        pos = _f64(pos, (-1, 3))
        n = len(pos)
        vel, T, rho = _f64(vel, (n, 3)), _f64(T, (n,)), _f64(rho, (n,))
        first = C.c_int64()
        self._check(self._L.sph_add_fluid(self._p, int(mat), n, _pd(pos), _pd(vel), _pd(T), _pd(rho),
                                          C.byref(first)), "sph_add_fluid")
        self.n += n
        return first.value

    def sph_add_solid(self, body, mat, pos, normal, T=None):
        pos = _f64(pos, (-1, 3))
        n = len(pos)
        normal, T = _f64(normal, (n, 3)), _f64(T, (n,))
        first = C.c_int64()
        self._check(self._L.sph_add_solid(self._p, int(body), int(mat), n, _pd(pos), _pd(normal), _pd(T),
                                          C.byref(first)), "sph_add_solid")
        self.n += n
        return first.value

    def sph_set_rotation(self, body, center, axis, omega):
        c = _f64(center, (3,))
        a = _f64(axis, (3,))
        self._check(self._L.sph_set_rotation(self._p, int(body), _pd(c), _pd(a), float(omega)),
                    "sph_set_rotation")

    def sph_step(self, n_steps=1):
        t = C.c_double()
        self._check(self._L.sph_step(self._p, int(n_steps), C.byref(t)), "sph_step")
        return t.value

    def sph_read_torque_heat(self, body=0):
        v = [C.c_double() for _ in range(4)]
        self._check(self._L.sph_read_torque_heat(self._p, int(body), *[C.byref(x) for x in v]),
                    "sph_read_torque_heat")
        return dict(torque=v[0].value, torque_avg=v[1].value, heat=v[2].value, mean_T=v[3].value)

    def sph_read_curve(self, max_steps=4096):
        """The last advection-step records, oldest first, one row of 8 each:
        time, torque of body 0, its running average, heat into fluid, mean
        fluid T, dt_ad, sub-steps, max fluid speed."""
        out = np.zeros(8 * max(int(max_steps), 1), np.float64)
        n = C.c_int64()
        self._check(self._L.sph_read_curve(self._p, _pd(out), int(max_steps), C.byref(n)), "sph_read_curve")
        return out[:8 * n.value].reshape(n.value, 8)

    def sph_read_fields(self, name, out=None):
        fid, k = FIELDS[name]
        if out is None:
            out = np.empty(self.n * k, np.float64)
        self._check(self._L.sph_read_fields(self._p, fid, out.ctypes.data_as(C.c_void_p), self.n),
                    "sph_read_fields")
        return out.reshape(self.n, 3) if k == 3 else out

    def sph_read_neighbors(self):
        counts = np.zeros(self.n, np.int64)
        total = C.c_int64()
        self._check(self._L.sph_read_neighbors(self._p, counts.ctypes.data_as(PI64), None, 0, C.byref(total)),
                    "sph_read_neighbors")
        ids = np.zeros(max(total.value, 1), np.int32)
        self._check(self._L.sph_read_neighbors(self._p, counts.ctypes.data_as(PI64), ids.ctypes.data_as(PI32),
                                               total.value, C.byref(total)), "sph_read_neighbors")
        return counts, ids[:total.value]

    def sph_read_cell_order(self):
        perm = np.zeros(self.n, np.int64)
        self._check(self._L.sph_read_cell_order(self._p, perm.ctypes.data_as(PI64), self.n), "sph_read_cell_order")
        return perm

    def sph_get_info(self):
        info = sph_info()
        self._check(self._L.sph_get_info(self._p, C.byref(info)), "sph_get_info")
        return {f: (list(getattr(info, f)) if f in ("ncell", "cell_width") else getattr(info, f))
                for f, _ in sph_info._fields_}

    def sph_pair_stats(self):
        ff, fw = C.c_int64(), C.c_int64()
        self._check(self._L.sph_pair_stats(self._p, C.byref(ff), C.byref(fw)), "sph_pair_stats")
        return ff.value, fw.value

    def sph_search_stats(self):
        a, b, c = C.c_int64(), C.c_int64(), C.c_int64()
        self._check(self._L.sph_search_stats(self._p, C.byref(a), C.byref(b), C.byref(c)), "sph_search_stats")
        return dict(searched=a.value, candidates=b.value, partners=c.value)

    def sph_set_tuning(self, key, value):
        self._check(self._L.sph_set_tuning(self._p, int(TUNE[key]), int(value)), "sph_set_tuning")

    def sph_get_tuning(self, key):
        v = C.c_int()
        self._check(self._L.sph_get_tuning(self._p, int(TUNE[key]), C.byref(v)), "sph_get_tuning")
        return v.value

    def sph_autotune(self, steps_per_trial=3):
        r = sph_tune_report()
        self._check(self._L.sph_autotune(self._p, int(steps_per_trial), C.byref(r)), "sph_autotune")
        return {f: getattr(r, f) for f, _ in sph_tune_report._fields_}

    def sph_profile(self, enable=True):
        self._check(self._L.sph_profile(self._p, int(bool(enable))), "sph_profile")

    def sph_profile_read(self, reset=False):
        ms = np.zeros(len(PROF_CLASSES), np.float64)
        cnt = np.zeros(len(PROF_CLASSES), np.int64)
        self._check(self._L.sph_profile_read(self._p, _pd(ms), cnt.ctypes.data_as(PI64), int(bool(reset))),
                    "sph_profile_read")
        return {k: (float(ms[i]), int(cnt[i])) for i, k in enumerate(PROF_CLASSES)}

    def close(self):
        if getattr(self, "_p", None):
            self._L.sph_destroy(self._p)
            self._p = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def from_case(case, stream=None) -> Context:
    """Build a Context from a workloads.Case (ids: fluid blocks, then solids)."""
    ctx = Context(case.config, 0 if stream is None else stream)
    for mid, m in case.materials.items():
        ctx.sph_set_material(mid, m)
    for bid, b in case.bodies.items():
        ctx.sph_set_rotation(bid, b["center"], b["axis"], b["omega"])
    for b in case.fluids:
        ctx.sph_add_fluid(b["mat"], b["pos"], b.get("vel"), b.get("T"), b.get("rho"))
    for b in case.solids:
        ctx.sph_add_solid(b["body"], b["mat"], b["pos"], b["normal"], b.get("T"))
    return ctx


def sph_cell_sort(pos_dev_ptr: int, n: int, origin, cellw, ncell, perm_dev_ptr: int, cell_start_dev_ptr: int,
                  stream: int = 0):
    """Stateless cell sort on device arrays (raw pointers, e.g. torch data_ptr())."""
    o, w = _f64(origin, (3,)), _f64(cellw, (3,))
    nc = (C.c_int * 3)(*[int(v) for v in ncell])
    rc = lib().sph_cell_sort(C.c_void_p(pos_dev_ptr), int(n), _pd(o), _pd(w), nc, C.c_void_p(perm_dev_ptr),
                             C.c_void_p(cell_start_dev_ptr), C.c_void_p(stream))
    if rc != SPH_OK:
        raise SphError(rc, "sph_cell_sort")


NOALLOC_MAX_N = 1 << 20
NOALLOC_MAX_CELLS = 1 << 20


def sph_cell_sort_noalloc(pos_dev_ptr: int, n: int, origin, cellw, ncell, perm_dev_ptr: int,
                          cell_start_dev_ptr: int, stream: int = 0):
    """Allocation-free cell sort: same contract as sph_cell_sort, scratch in
    the library's fixed device array (n <= NOALLOC_MAX_N, cells <=
    NOALLOC_MAX_CELLS)."""
    o, w = _f64(origin, (3,)), _f64(cellw, (3,))
    nc = (C.c_int * 3)(*[int(v) for v in ncell])
    L = lib()
    rc = L.sph_cell_sort_noalloc(C.c_void_p(pos_dev_ptr), int(n), _pd(o), _pd(w), nc, C.c_void_p(perm_dev_ptr),
                                 C.c_void_p(cell_start_dev_ptr), C.c_void_p(stream))
    if rc != SPH_OK:
        raise SphError(rc, "sph_cell_sort_noalloc: " + L.sph_last_error(None).decode())


def sph_fma_peak(reps=5, stream=None):
    """Measured FP32 FMA throughput of the current device: (TFLOP/s, ms of
    the fastest probe launch)."""
    L = lib()
    tf, ms = D(), D()
    st = L.sph_fma_peak(C.c_void_p(0 if stream is None else stream), int(reps), C.byref(tf), C.byref(ms))
    if st != SPH_OK:
        raise SphError(st, "sph_fma_peak")
    return tf.value, ms.value


class Batch:
    """A sph_batch: many cases packed in one device array, stepped together."""

    def __init__(self, max_particles, max_cases, max_cells, history_steps=2048, stream=None):
        self._L = lib()
        cfg = sph_batch_config(int(max_particles), int(max_cases), int(max_cells), int(history_steps))
        self.bytes = int(self._L.sph_batch_bytes(C.byref(cfg)))
        p = C.c_void_p()
        self.stream = current_stream_handle() if stream is None else int(stream)
        rc = self._L.sph_batch_create(C.byref(cfg), C.c_void_p(self.stream), C.byref(p))
        if rc != SPH_OK:
            raise SphError(rc, "sph_batch_create: " + self._L.sph_last_error(None).decode())
        self._p = p
        self.n_of = {}

    @staticmethod
    def bytes_for(max_particles, max_cases, max_cells, history_steps=2048):
        cfg = sph_batch_config(int(max_particles), int(max_cases), int(max_cells), int(history_steps))
        return int(lib().sph_batch_bytes(C.byref(cfg)))

    def _check(self, rc, what):
        if rc != SPH_OK:
            raise SphError(rc, f"{what}: {self._L.sph_batch_last_error(self._p).decode()}")

    def admit(self, case, n_steps=0):
        """Stage a workloads.Case and admit it; returns the slot (raises
        SphError with status SPH_ENOMEM when the batch is full)."""
        staged = from_case(case, stream=self.stream)
        slot = C.c_int()
        try:
            self._check(self._L.sph_batch_admit(self._p, staged._p, int(n_steps), C.byref(slot)), "sph_batch_admit")
        finally:
            staged.close()
        self.n_of[slot.value] = case.n_total
        return slot.value

    def step(self, n=1):
        self._check(self._L.sph_batch_step(self._p, int(n)), "sph_batch_step")

    def poll(self, slot):
        steps, t, st = C.c_int64(), C.c_double(), C.c_int()
        self._check(self._L.sph_batch_poll(self._p, int(slot), C.byref(steps), C.byref(t), C.byref(st)),
                    "sph_batch_poll")
        return steps.value, t.value, st.value

    def torque_heat(self, slot, body=0):
        v = [C.c_double() for _ in range(4)]
        self._check(self._L.sph_batch_read_torque_heat(self._p, int(slot), int(body), *[C.byref(x) for x in v]),
                    "sph_batch_read_torque_heat")
        return dict(torque=v[0].value, torque_avg=v[1].value, heat=v[2].value, mean_T=v[3].value)

    def curve(self, slot, max_steps):
        out = np.zeros(8 * max(int(max_steps), 1), np.float64)
        n = C.c_int64()
        self._check(self._L.sph_batch_read_curve(self._p, int(slot), _pd(out), int(max_steps), C.byref(n)),
                    "sph_batch_read_curve")
        return out[:8 * n.value].reshape(n.value, 8)

    def fields(self, slot, name):
        fid, k = FIELDS[name]
        n = self.n_of[slot]
        out = np.empty(n * k, np.float64)
        self._check(self._L.sph_batch_read_fields(self._p, int(slot), fid, out.ctypes.data_as(C.c_void_p), n),
                    "sph_batch_read_fields")
        return out.reshape(n, 3) if k == 3 else out

    def retire(self, slot):
        self._check(self._L.sph_batch_retire(self._p, int(slot)), "sph_batch_retire")
        self.n_of.pop(slot, None)

    def info(self):
        n, c, k = C.c_int64(), C.c_int(), C.c_int()
        self._check(self._L.sph_batch_info(self._p, C.byref(n), C.byref(c), C.byref(k)), "sph_batch_info")
        return dict(n_particles=n.value, n_cases=c.value, kernels_per_step=k.value)

    def set_tuning(self, key, value):
        self._check(self._L.sph_batch_set_tuning(self._p, int(TUNE[key]), int(value)), "sph_batch_set_tuning")

    def autotune(self, steps_per_trial=3):
        r = sph_tune_report()
        self._check(self._L.sph_batch_autotune(self._p, int(steps_per_trial), C.byref(r)), "sph_batch_autotune")
        return {f: getattr(r, f) for f, _ in sph_tune_report._fields_}

    def profile(self, enable=True):
        self._check(self._L.sph_batch_profile(self._p, int(bool(enable))), "sph_batch_profile")

    def profile_read(self, reset=False):
        ms = np.zeros(len(PROF_CLASSES), np.float64)
        cnt = np.zeros(len(PROF_CLASSES), np.int64)
        self._check(self._L.sph_batch_profile_read(self._p, _pd(ms), cnt.ctypes.data_as(PI64), int(bool(reset))),
                    "sph_batch_profile_read")
        return {k: (float(ms[i]), int(cnt[i])) for i, k in enumerate(PROF_CLASSES)}

    def close(self):
        if getattr(self, "_p", None):
            self._L.sph_batch_destroy(self._p)
            self._p = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def sph_relax(pos, dx, h_over_dx, phi, phi_origin, phi_spacing, iterations, stream=None):
    """Particle relaxation (Sec. 2.2) on the GPU: pos[n, 3] (host) relaxed in the
    level set phi[nz, ny, nx]; returns (positions, max |F_p| per iteration)."""
    L = lib()
    pos = np.ascontiguousarray(pos, np.float64).copy()
    phi = np.ascontiguousarray(phi, np.float64)
    c = sph_relax_config()
    c.dx, c.h_over_dx = float(dx), float(h_over_dx)
    c.phi = phi.ctypes.data_as(C.POINTER(D))
    c.nphi = (C.c_int * 3)(phi.shape[2], phi.shape[1], phi.shape[0])
    c.phi_origin = (D * 3)(*[float(v) for v in phi_origin])
    c.phi_spacing = float(phi_spacing)
    amax = np.zeros(max(int(iterations), 1), np.float64)
    st = L.sph_relax(C.byref(c), len(pos), pos.ctypes.data_as(PD), int(iterations),
                     C.c_void_p(0 if stream is None else stream), amax.ctypes.data_as(PD))
    if st != 0:
        raise SphError(st, "sph_relax: " + L.sph_last_error(None).decode())
    return pos, amax[:iterations]


# sort cells per geometry cell (width >= 2h) along x, y and z
SORT_SPLIT = (8, 2, 2)


def cells_of(case):
    """Sort cells of a case (SORT_SPLIT per geometry cell of width >= 2h), for batch sizing."""
    R = case.support_radius()
    n = 1
    for e, k in zip(case.config["extent"], SORT_SPLIT):
        n *= k * max(1, int(np.floor(e / R)))
    return n
