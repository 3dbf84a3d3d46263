"""ctypes loader of libmkf.so.  There is no fallback: if the library is missing
or fails to load, every call raises."""
import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libmkf.so")

_lib = None

P = ctypes.c_void_p
i32 = ctypes.c_int
i64 = ctypes.c_int64
f32 = ctypes.c_float

# name -> (restype, argtypes)
SIGNATURES = {
    "mkf_create": (i32, [ctypes.POINTER(P), i32]),
    "mkf_destroy": (None, [P]),
    "mkf_last_error": (ctypes.c_char_p, [P]),
    "mkf_sync": (i32, [P, P]),
    "mkf_load_geometry": (i32, [P, P, i32, f32]),
    "mkf_bin_hits": (i32, [P, P, P, P, i64, P, i32, P]),
    "mkf_bin_hits_masked": (i32, [P, P, P, P, i64, P, i32, P, P]),
    "mkf_used_hits": (i32, [P, P, i32, P, i64, i64, P, P]),
    "mkf_get_binning": (i32, [P, P, P, ctypes.POINTER(i64), P]),
    "mkf_build_tracks": (i32, [P, P, P, P, i64, f32, i32, i32, i32, f32, P, P, P, P, P, P, P, P, P]),
    "mkf_set_debug": (i32, [P, i32]),
    "mkf_set_build_config": (i32, [P, i32, i32]),
    "mkf_set_adjoint_config": (i32, [P, i32]),
    "mkf_set_build_dedup": (i32, [P, i32]),
    "mkf_get_stats": (i32, [P, P, i32, P]),
    "mkf_set_timing": (i32, [P, i32]),
    "mkf_get_timings": (i32, [P, P, i32, P]),
    "mkf_set_strip_config": (i32, [P, i32, i32, i32]),
    "mkf_seed_tracks": (i32, [P, f32, f32, f32, f32, i64, P, P, P, P, P]),
    "mkf_get_seed_stats": (i32, [P, P, i32, P]),
    "mkf_set_seed_config": (i32, [P, i64]),
    "mkf_find_overlaps": (i32, [P, P, P, P, i64, P, i32, P, P, i64, f32, f32, f32, P, P, P]),
    "mkf_get_overlap_stats": (i32, [P, P, i32, P]),
    "mkf_set_overlap_config": (i32, [P, i32]),
    "mkf_cluster_strips": (i32, [P, P, P, P, i32, i32, i32, i32, i32, P, P, P, P, P, i64, P, P]),
    "mkf_dedup_tracks": (i32, [P, P, i32, P, P, P, i32, i64, i64, i32, f32, P, P]),
    "mkf_dedup_tracks_noalloc": (i32, [P, i32, P, P, P, i32, i64, i64, i32, f32, P, P, P]),
    "mkf_fit_tracks": (i32, [P, P, P, P, i64, P, i32, P, P, i64, P, P, P, P, P, P, P, P]),
    "mkf_fit_backward": (i32, [P, P, P, P, i64, P, i32, P, i64, P, P, P, P, P, P, P]),
    "mkf_fit_tracks_adjoint": (i32, [P, P, P, P, i64, P, i32, P, P, i64, P, P, P, P, P, P, P, P, P, P]),
}


class MkfLayer(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("pos", ctypes.c_float), ("lo", ctypes.c_float), ("hi", ctypes.c_float),
                ("x_over_x0", ctypes.c_float), ("n_phi_bins", ctypes.c_int), ("n_w_bins", ctypes.c_int)]


def load():
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError("libmkf.so is not built (%s); run __graft_entry__.build() or "
                           "python -m paper_2002_06295_gb300.build_ext" % LIB_PATH)
    lib = ctypes.CDLL(LIB_PATH)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib
