"""ctypes mirror of include/raywave.h and the loader of librw.so.

Argument marshalling only.  There is no fallback: if the compiled library
is missing, loading raises.
"""
import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "librw.so")

RW_OK, RW_EINVAL, RW_ENOMEM, RW_ECUDA, RW_ECAPACITY, RW_ETIMEOUT, RW_ENOTCONV = range(7)
STATUS_NAMES = {0: "RW_OK", 1: "RW_EINVAL", 2: "RW_ENOMEM", 3: "RW_ECUDA", 4: "RW_ECAPACITY",
                5: "RW_ETIMEOUT", 6: "RW_ENOTCONV"}
RW_PLANE, RW_SPHERE, RW_ASPHERE, RW_GAUSS = 0, 1, 2, 3
RW_GATHER_NEAREST, RW_GATHER_BILINEAR = 0, 1
RW_EMIT_EXHAUSTIVE, RW_EMIT_SAMPLED, RW_EMIT_SAMPLED_UNIFORM = 0, 1, 2
RW_PHASE_HEIGHT, RW_PHASE_FIXED = 0, 1
RW_DFT_FFT32, RW_DFT_TC = 0, 1
RW_DOE_TRACE_ALL, RW_DOE_REFLECTIVE = 1, 2
KERNEL_KINDS = ("k_forward", "k_cull", "k_bs_spectra", "k_bs_trace", "k_bs_scatter",
                "k_backward", "k_spectra")
RW_MAX_SURFACES = 16
FP = C.POINTER(C.c_float)
DP = C.POINTER(C.c_double)
IP = C.POINTER(C.c_int32)


class rw_surface(C.Structure):
    _fields_ = [("kind", C.c_int32), ("reserved", C.c_int32), ("z", C.c_double),
                ("c", C.c_double), ("k", C.c_double), ("A4", C.c_double), ("A6", C.c_double),
                ("A8", C.c_double), ("A10", C.c_double), ("n_after", C.c_double),
                ("r_ap", C.c_double), ("sellmeier", C.c_double * 6)]


class rw_doe(C.Structure):
    _fields_ = [("H", C.c_int32), ("W", C.c_int32), ("pitch", C.c_double),
                ("lambda0", C.c_double), ("phi", C.c_void_p), ("amp", C.c_void_p),
                ("D", C.c_int32), ("gather", C.c_int32), ("emit", C.c_int32),
                ("n_ssr", C.c_int32), ("phase_model", C.c_int32), ("dft", C.c_int32),
                ("seed", C.c_uint64), ("rng_offset", C.c_uint64),
                ("pad", C.c_int32), ("flags", C.c_int32), ("phi2", C.c_void_p)]


class rw_sensor(C.Structure):
    _fields_ = [("z", C.c_double), ("nx", C.c_int32), ("ny", C.c_int32),
                ("pitch", C.c_double), ("coherent", C.c_int32), ("window", C.c_int32)]


class rw_system(C.Structure):
    _fields_ = [("surfaces", C.POINTER(rw_surface)), ("nsurf", C.c_int32),
                ("doe_index", C.c_int32), ("n_object", C.c_double), ("doe", rw_doe),
                ("sensor", rw_sensor)]


class rw_job(C.Structure):
    _fields_ = [("lambda_", C.c_double), ("theta_x", C.c_double), ("theta_y", C.c_double),
                ("ray_offset", C.c_int64), ("ray_count", C.c_int64),
                ("sensor_cx", C.c_double), ("sensor_cy", C.c_double),
                ("grid_n", C.c_int64), ("spacing", C.c_double), ("x0", C.c_double),
                ("y0", C.c_double)]


class rw_rays(C.Structure):
    _fields_ = [("n", C.c_int64), ("ox", C.c_void_p), ("oy", C.c_void_p), ("oz", C.c_void_p),
                ("dx", C.c_void_p), ("dy", C.c_void_p), ("dz", C.c_void_p),
                ("a_re", C.c_void_p), ("a_im", C.c_void_p), ("opl", C.c_void_p)]


class rw_emitted(C.Structure):
    _fields_ = [("capacity", C.c_int64), ("dx", C.c_void_p), ("dy", C.c_void_p),
                ("dz", C.c_void_p), ("a_re", C.c_void_p), ("a_im", C.c_void_p),
                ("bin", C.c_void_p), ("hx", C.c_void_p), ("hy", C.c_void_p),
                ("hz", C.c_void_p), ("opl", C.c_void_p)]


EXPORTS = {
    "rw_create": (C.c_int, [C.POINTER(C.c_void_p), C.c_int, C.c_void_p]),
    "rw_destroy": (C.c_int, [C.c_void_p]),
    "rw_set_stream": (C.c_int, [C.c_void_p, C.c_void_p]),
    "rw_last_error": (C.c_char_p, [C.c_void_p]),
    "rw_device_status": (C.c_int, [C.c_void_p, C.POINTER(C.c_uint32)]),
    "rw_version": (C.c_char_p, []),
    "rw_launch_count": (C.c_int64, [C.c_void_p]),
    "rw_profile": (C.c_int, [C.c_void_p, C.c_int32]),
    "rw_cull_stats": (C.c_int, [C.c_void_p, C.POINTER(C.c_int64), C.POINTER(C.c_int64)]),
    "rw_autotune": (C.c_int, [C.c_void_p, C.POINTER(rw_system), C.POINTER(rw_job), C.c_int32,
                              C.POINTER(rw_rays), C.c_void_p, C.c_void_p, C.c_void_p, C.c_int64,
                              C.c_void_p, C.c_void_p, C.POINTER(C.c_int64)]),
    "rw_set_grids": (C.c_int, [C.c_void_p, C.POINTER(C.c_int64)]),
    "rw_probe_red": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int32, C.c_int32, C.c_int32,
                               C.c_int64]),
    "rw_profile_read": (C.c_int, [C.c_void_p, C.POINTER(C.c_int32)]),
    "rw_profile_entry": (C.c_int, [C.c_void_p, C.c_int32, C.POINTER(C.c_char_p),
                                   C.POINTER(C.c_double), C.POINTER(C.c_int64)]),
    "rw_generate_rays": (C.c_int, [C.c_void_p, C.c_double, C.c_double, C.POINTER(rw_job),
                                   C.c_int32, C.POINTER(rw_rays)]),
    "rw_doe_emit": (C.c_int, [C.c_void_p, C.POINTER(rw_system), C.POINTER(rw_job), C.c_int32,
                              C.POINTER(rw_rays), C.POINTER(rw_emitted)]),
    "rw_forward": (C.c_int, [C.c_void_p, C.POINTER(rw_system), C.POINTER(rw_job), C.c_int32,
                             C.POINTER(rw_rays), C.c_void_p]),
    "rw_loss_eq3": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p,
                              C.c_void_p]),
    "rw_backward": (C.c_int, [C.c_void_p, C.POINTER(rw_system), C.POINTER(rw_job), C.c_int32,
                              C.POINTER(rw_rays), C.c_void_p, C.c_void_p, C.c_void_p,
                              C.c_void_p]),
    "rw_forward_vis": (C.c_int, [C.c_void_p, C.POINTER(rw_system), C.POINTER(rw_job), C.c_int32,
                                 C.POINTER(rw_rays), C.c_void_p, C.c_void_p, C.c_int64]),
    "rw_backward_vis": (C.c_int, [C.c_void_p, C.POINTER(rw_system), C.POINTER(rw_job), C.c_int32,
                                  C.POINTER(rw_rays), C.c_void_p, C.c_void_p, C.c_int64,
                                  C.c_void_p, C.c_void_p, C.c_void_p]),
    "rw_patch_spectra": (C.c_int, [C.c_void_p, C.POINTER(rw_system), C.POINTER(rw_job), C.c_int32,
                                   C.POINTER(rw_rays), C.c_void_p, C.c_int64]),
    "rw_generate_rays_static": (C.c_int, [C.c_double, C.c_double, C.POINTER(rw_job), C.c_int32,
                                          C.POINTER(rw_rays), C.c_void_p]),
}

_lib = None


def load(path=LIB_PATH):
    """Load librw.so and declare its prototypes (raises if it is missing)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is not built: run paper_2605_15418_gb300.build.build() "
                           "(there is no CPU fallback)")
    lib = C.CDLL(path)
    for name, (res, args) in EXPORTS.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib
