"""Host-side checks of the C-ABI library (no GPU needed).

The library must build for sm_103a, load, and export every function that
include/*.h declares; argument validation that happens before any CUDA call
is exercised here.
"""
import ctypes as C
import glob
import os
import re

import numpy as np
import pytest

from paper_2512_09904_b300 import build as B
from paper_2512_09904_b300 import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def sphlib():
    B.build()
    from paper_2512_09904_b300 import sph
    return sph


def declared_functions():
    names = []
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        txt = open(h).read()
        txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
        names += re.findall(r"^\s*(?:const\s+)?\w+\s*\*?\s*(sph_\w+)\s*\(", txt, flags=re.M)
    return sorted(set(names))


def test_library_exports_every_declared_symbol(sphlib):
    names = declared_functions()
    assert "sph_create" in names and "sph_step" in names and "sph_read_torque_heat" in names
    L = C.CDLL(sphlib.LIB_PATH)
    missing = [n for n in names if not hasattr(L, n)]
    assert not missing, missing


def test_library_is_built_for_sm103a(sphlib):
    assert "arch=compute_103a,code=sm_103a" in " ".join(B.ARCH)
    assert os.path.getsize(sphlib.LIB_PATH) > 0


def test_create_validates_config(sphlib):
    cfg = W.still_tank(nx=4, ny=4, nz=4, wall_h=6).config
    ctx = sphlib.Context(cfg, stream=0)
    info = ctx.sph_get_info()
    R = 2 * cfg["h_over_dx"] * cfg["dx"]
    for a, split in enumerate((8, 2, 2)):
        # sort cells: 8 (x) or 2 (y, z) per geometry cell of width >= 2h
        assert info["ncell"][a] == split * int(np.floor(cfg["extent"][a] / R))
        assert info["cell_width"][a] >= R / split
    # default sub-step cap: ceil(cfl_ad / cfl_ac (c0 / u_ref + 1)) + 2
    assert info["kcap"] == int(np.ceil(0.25 / 0.6 * (cfg["c0"] / cfg["u_ref"] + 1))) + 2
    ctx.close()
    bad = dict(cfg, dx=-1.0)
    with pytest.raises(sphlib.SphError) as e:
        sphlib.Context(bad, stream=0)
    assert e.value.status == sphlib.SPH_EINVAL
    # a periodic axis needs at least 3 cells
    bad = dict(cfg, periodic_mask=1, extent=[2.5 * R, cfg["extent"][1], cfg["extent"][2]])
    with pytest.raises(sphlib.SphError):
        sphlib.Context(bad, stream=0)
    # pair precision: 0 (FP32 pairs) or 1 (FP64 throughout)
    sphlib.Context(dict(cfg, pair_precision=1), stream=0).close()
    sphlib.Context(dict(cfg, viscous_heating=1), stream=0).close()
    with pytest.raises(sphlib.SphError):
        sphlib.Context(dict(cfg, viscous_heating=2), stream=0)
    with pytest.raises(sphlib.SphError) as e:
        sphlib.Context(dict(cfg, pair_precision=2), stream=0)
    assert e.value.status == sphlib.SPH_EINVAL
    # Eq. (26) coefficient: >= 0 (0 switches the thermal bound off)
    sphlib.Context(dict(cfg, cfl_T=0.0), stream=0).close()
    for bad in (-0.5, float("nan")):
        with pytest.raises(sphlib.SphError) as e:
            sphlib.Context(dict(cfg, cfl_T=bad), stream=0)
        assert e.value.status == sphlib.SPH_EINVAL
    # Eq. (13) with its printed sign: FP64 pairs only
    sphlib.Context(dict(cfg, pair_precision=1, vstar_literal=1), stream=0).close()
    for bad in (dict(vstar_literal=1), dict(pair_precision=1, vstar_literal=2)):
        with pytest.raises(sphlib.SphError) as e:
            sphlib.Context(dict(cfg, **bad), stream=0)
        assert e.value.status == sphlib.SPH_EINVAL
    # Eq. (19) as printed: FP64 pairs only
    sphlib.Context(dict(cfg, pair_precision=1, wall_pstar_printed=1), stream=0).close()
    for bad in (dict(wall_pstar_printed=1), dict(pair_precision=1, wall_pstar_printed=-1)):
        with pytest.raises(sphlib.SphError) as e:
            sphlib.Context(dict(cfg, **bad), stream=0)
        assert e.value.status == sphlib.SPH_EINVAL


def test_add_validates_arguments(sphlib):
    case = W.still_tank(nx=4, ny=4, nz=4, wall_h=6)
    ctx = sphlib.Context(case.config, stream=0)
    with pytest.raises(sphlib.SphError) as e:
        ctx.sph_add_fluid(0, case.fluids[0]["pos"])  # material 0 not set yet
    assert e.value.status == sphlib.SPH_EINVAL
    for mid, m in case.materials.items():
        ctx.sph_set_material(mid, m)
    with pytest.raises(sphlib.SphError):
        ctx.sph_set_material(16, case.materials[0])
    first = ctx.sph_add_fluid(0, case.fluids[0]["pos"], rho=case.fluids[0]["rho"])
    assert first == 0
    s = case.solids[0]
    assert ctx.sph_add_solid(-1, s["mat"], s["pos"], s["normal"]) == case.n_fluid
    with pytest.raises(sphlib.SphError):
        ctx.sph_add_solid(7, 1, s["pos"], s["normal"])  # body id out of range
    with pytest.raises(sphlib.SphError):
        ctx.sph_set_rotation(0, [0, 0, 0], [0, 0, 2.0], 1.0)  # axis not unit
    bad = case.fluids[0]["pos"].copy()
    bad[0, 0] = np.nan
    with pytest.raises(sphlib.SphError):
        ctx.sph_add_fluid(0, bad)
    ctx.close()


def test_large_blocks_are_checked_while_staged(sphlib):
    """Blocks of more than 2^20 values are copied and checked by several host
    threads: a non-finite position anywhere fails the call and stages
    nothing; non-finite densities are replaced, not refused."""
    case = W.still_tank(nx=4, ny=4, nz=4, wall_h=6)
    ctx = sphlib.Context(case.config, stream=0)
    for mid, m in case.materials.items():
        ctx.sph_set_material(mid, m)
    n = 400_000
    rng = np.random.default_rng(3)
    pos = rng.uniform(0.0, 0.01, size=(n, 3))
    for where in (0, n // 3, n - 1):
        bad = pos.copy()
        bad[where, 2] = np.inf if where % 2 else np.nan
        with pytest.raises(sphlib.SphError) as e:
            ctx.sph_add_fluid(0, bad)
        assert e.value.status == sphlib.SPH_EINVAL
        assert ctx.sph_get_info()["n_fluid"] == 0
    rho = np.full(n, 870.0)
    rho[::7] = np.nan
    assert ctx.sph_add_fluid(0, pos, rho=rho) == 0
    assert ctx.sph_add_fluid(0, pos) == n
    assert ctx.sph_get_info()["n_fluid"] == 2 * n
    ctx.close()


def test_reads_before_first_step_are_state_errors(sphlib):
    case = W.periodic_box(n=8)
    ctx = sphlib.Context(case.config, stream=0)
    with pytest.raises(sphlib.SphError) as e:
        ctx.sph_read_torque_heat(0)
    assert e.value.status == sphlib.SPH_ESTATE
    with pytest.raises(sphlib.SphError) as e:
        ctx.sph_read_curve(8)
    assert e.value.status == sphlib.SPH_ESTATE
    ctx.close()


def test_tuning_keys_are_validated(sphlib):
    case = W.still_tank(nx=4, ny=4, nz=4, wall_h=6)
    ctx = sphlib.Context(case.config, stream=0)
    for key, good, bad in (("list_batch", 4, 3), ("tpp", 2, 3), ("block", 256, 96)):
        ctx.sph_set_tuning(key, good)
        assert ctx.sph_get_tuning(key) == good
        with pytest.raises(sphlib.SphError) as e:
            ctx.sph_set_tuning(key, bad)
        assert e.value.status == sphlib.SPH_EINVAL
        assert ctx.sph_get_tuning(key) == good
    ctx.close()


def test_relax_validates_arguments(sphlib):
    b = W.relax_body("sphere", size=3e-3)
    with pytest.raises(sphlib.SphError) as e:
        sphlib.sph_relax(b["pos"], -1.0, b["h_over_dx"], b["phi"], b["phi_origin"], b["phi_spacing"], 2)
    assert e.value.status == sphlib.SPH_EINVAL
    with pytest.raises(sphlib.SphError):
        sphlib.sph_relax(b["pos"], b["dx"], b["h_over_dx"], b["phi"][:1], b["phi_origin"], b["phi_spacing"], 2)


def test_fma_peak_validates_arguments(sphlib):
    L = sphlib.lib()
    t = C.c_double()
    assert L.sph_fma_peak(None, 0, C.byref(t), None) == sphlib.SPH_EINVAL
    assert L.sph_fma_peak(None, 3, None, None) == sphlib.SPH_EINVAL


def test_empty_case_cannot_step(sphlib):
    # no particles: stepping is a state error, raised before any device work;
    # an empty add is accepted and adds nothing
    case = W.periodic_box(n=8)
    ctx = sphlib.Context(case.config, stream=0)
    for mid, m in case.materials.items():
        ctx.sph_set_material(mid, m)
    assert ctx.sph_add_fluid(0, np.zeros((0, 3))) == 0
    with pytest.raises(sphlib.SphError) as e:
        ctx.sph_step(1)
    assert e.value.status == sphlib.SPH_ESTATE
    assert ctx.sph_get_info()["n_fluid"] == 0
    ctx.close()


@pytest.mark.parametrize("fn", ["sph_cell_sort", "sph_cell_sort_noalloc"])
def test_cell_sort_rejects_grids_whose_cell_count_overflows(sphlib, fn):
    # three factors of 2^31 - 1 would overflow a 64-bit product; the count is
    # checked after each factor, so the call returns SPH_EINVAL before any
    # device work (n = 0 needs no positions; the output pointer is never used)
    L = sphlib.lib()
    f = getattr(L, fn)
    big = (C.c_int * 3)(2 ** 31 - 1, 2 ** 31 - 1, 2 ** 31 - 1)
    o = (C.c_double * 3)(0.0, 0.0, 0.0)
    w = (C.c_double * 3)(1.0, 1.0, 1.0)
    rc = f(None, 0, o, w, big, None, C.c_void_p(16), None)
    assert rc == sphlib.SPH_EINVAL
    assert "cell" in L.sph_last_error(None).decode()
