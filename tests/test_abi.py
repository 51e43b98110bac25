"""CPU checks of the boundary: libisw.so builds, loads and exports every entry point that
include/isw.h declares (no compute call: there may be no GPU here)."""
import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "isw.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+)?\w+\s*\*?\s*(\w+)\s*\(", src, flags=re.M)))


def test_header_declares_the_boundary():
    names = _declared()
    for n in ("hp_pix2vec_ring", "lightcone_intersect", "isw_map", "isw_map_adjoint", "isw_map_batched",
              "isw_create", "isw_destroy", "isw_last_error", "isw_check_status", "isw_set_param",
              "isw_get_param", "isw_get_timing", "lightcone_adjoint", "hp_vec2pix_ring", "box_place",
              "lightcone_intersect_shells", "cone_cut", "isw_map_patch", "isw_map_cl", "isw_map_f32c_noalloc",
              "isw_fma_rate"):
        assert n in names


def test_library_loads_and_exports_every_symbol():
    import paper_1204_5041_gb300 as isw

    path = isw.build()
    lib = ctypes.CDLL(path)
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_create_without_device_is_an_error_not_a_crash():
    import paper_1204_5041_gb300 as isw
    import torch

    if torch.cuda.is_available():
        return
    h = ctypes.c_void_p()
    r = isw.lib().isw_create(ctypes.byref(h), 0)
    assert r != isw.OK and not h
