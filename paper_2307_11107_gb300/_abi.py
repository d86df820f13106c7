"""ctypes mirror of include/apic.h and the loader of the in-tree libapic.so.

Only argument marshalling lives here; every step of the computation runs in
the CUDA kernels of libapic.so.  The library must have been built (see
``build.py``); there is no fallback.
"""
import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libapic.so")

OK = 0
ERRORS = {-1: "INVALID_ARG", -2: "GEOMETRY", -3: "CAPACITY", -4: "NOT_CONVERGED", -5: "NONFINITE",
          -6: "TIMEOUT", -7: "CUDA"}
FP64 = 0
FP32_REFINED = 1
LOAD_VOLUME, FLUX_SURFACE, EXPLICIT = 0, 1, 2
NO_INJECT, NO_FIELD, CHORD_ABSORB, FLOATING, BOLTZMANN, FE_OPERATOR = 1, 2, 4, 8, 16, 32
NT, NH = 7, 11

SYMBOLS = ("apic_create", "apic_create_batch", "apic_destroy", "apic_inject", "apic_step", "apic_tallies",
           "apic_solve_poisson", "apic_get_particles", "apic_get_field", "apic_last_error",
           "apic_num_instances", "apic_stats", "apic_step_timed", "apic_deposit_static", "apic_sensitivity",
           "apic_adjoint", "apic_adjoint_window", "apic_autotune", "apic_probe_fp32_fma", "apic_check_wait_limit",
           "apic_set_schedule", "apic_checkpoint_size", "apic_checkpoint_save", "apic_checkpoint_load")
TUNE_INTERVALS = (2, 4, 6, 8, 12, 16, 24)
NPAR, NOUT = 3, 5
PARAMS = ("alpha", "phi_g", "B")
OUTPUTS = ("drag_FZ", "electric_FZ", "current", "torque", "Q")
NPHASE = 6
PHASES = ("deposit_rho", "poisson", "fields", "push", "inject", "bookkeeping")


class Species(C.Structure):
    _fields_ = [("q", C.c_double), ("m", C.c_double), ("T", C.c_double), ("n_init", C.c_int64),
                ("capacity", C.c_int64)]


class Config(C.Structure):
    _fields_ = [("alpha", C.c_double), ("x1_outer", C.c_double), ("phi_grain", C.c_double),
                ("phi_outer", C.c_double), ("B", C.c_double), ("dt", C.c_double), ("e_bind_ion", C.c_double),
                ("n1", C.c_int32), ("n2", C.c_int32), ("n_species", C.c_int32), ("sp", Species * 2),
                ("seed", C.c_uint64), ("instance", C.c_int32), ("precision", C.c_int32), ("flags", C.c_int32),
                ("poisson_tol", C.c_double), ("poisson_max_iter", C.c_int32), ("sort_interval", C.c_int32),
                ("history_cap", C.c_int32), ("poisson_guess", C.c_int32), ("newton_iters", C.c_int32),
                ("reserved", C.c_int32 * 3)]


ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p, C.c_void_p)


class Allocator(C.Structure):
    _fields_ = [("alloc", ALLOC_FN), ("free", FREE_FN), ("ctx", C.c_void_p)]


class Tallies(C.Structure):
    _fields_ = [("bins", C.POINTER(C.c_double)), ("history", C.POINTER(C.c_double)),
                ("history_rows", C.c_int64), ("counts", (C.c_int64 * 6) * 2), ("step", C.c_int64),
                ("grain_Q", C.c_double), ("grain_FZ", C.c_double), ("poisson_res", C.c_double),
                ("poisson_iters", C.c_int32), ("pad", C.c_int32)]


class Grid(C.Structure):
    _fields_ = [("n1", C.c_int32), ("n2", C.c_int32), ("x1_outer", C.c_double)]


class Stats(C.Structure):
    _fields_ = [("steps", C.c_int64), ("poisson_loop_iters", C.c_int64), ("kernels_per_step", C.c_int32),
                ("kernels_per_iter", C.c_int32), ("timed_steps", C.c_int64), ("phase_ms", C.c_double * NPHASE),
                ("solver", C.c_int32), ("kernels_per_sort", C.c_int32), ("sorts", C.c_int64),
                ("sort_interval", C.c_int32), ("win_rows", C.c_int32), ("chunk_group", C.c_int32),
                ("chunk_items", C.c_int32), ("timed_sorts", C.c_int64), ("sort_ms", C.c_double)]


SOLVERS = ("multigrid BiCGSTAB, per-phase kernels", "multigrid BiCGSTAB, one cooperative launch",
           "FP32 block cyclic reduction in FP64 iterative refinement, one cooperative launch",
           "FP32 nested dissection in FP64 iterative refinement, one cooperative launch")


_lib = None


def load():
    """Load libapic.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError("libapic.so is not built: run paper_2307_11107_gb300/build.py (nvcc, sm_103a)")
    L = C.CDLL(LIB_PATH)
    vp, i32, i64, dp = C.c_void_p, C.c_int32, C.c_int64, C.POINTER(C.c_double)
    L.apic_create.argtypes = [C.POINTER(Config), vp, C.POINTER(Allocator), C.POINTER(vp)]
    L.apic_create_batch.argtypes = [C.POINTER(Config), i32, vp, C.POINTER(Allocator), C.POINTER(vp)]
    L.apic_destroy.argtypes = [vp]
    L.apic_inject.argtypes = [vp, i32, i32, i64, i32, dp]
    L.apic_step.argtypes = [vp, i32]
    L.apic_tallies.argtypes = [vp, i32, C.POINTER(Tallies)]
    L.apic_solve_poisson.argtypes = [vp, i32, dp, dp]
    L.apic_get_particles.argtypes = [vp, i32, i32, dp, i64, C.POINTER(i64)]
    L.apic_get_field.argtypes = [vp, i32, i32, dp]
    L.apic_last_error.argtypes = [vp]
    L.apic_last_error.restype = C.c_char_p
    L.apic_num_instances.argtypes = [vp]
    L.apic_num_instances.restype = i32
    L.apic_stats.argtypes = [vp, C.POINTER(Stats)]
    L.apic_step_timed.argtypes = [vp, i32]
    L.apic_deposit_static.argtypes = [C.POINTER(Grid), vp, vp, i64, C.c_double, vp, vp, vp]
    L.apic_sensitivity.argtypes = [vp, i32, dp, dp]
    L.apic_adjoint.argtypes = [vp, i32, dp, dp]
    L.apic_adjoint_window.argtypes = [vp, i32, dp, dp, dp]
    L.apic_autotune.argtypes = [vp, i32, C.POINTER(i32), dp]
    L.apic_probe_fp32_fma.argtypes = [vp, i32, dp]
    L.apic_check_wait_limit.argtypes = [vp, i64]
    L.apic_set_schedule.argtypes = [vp, i32, i32, i32, i32]
    L.apic_checkpoint_size.argtypes = [vp, C.POINTER(i64)]
    L.apic_checkpoint_save.argtypes = [vp, vp, i64]
    L.apic_checkpoint_load.argtypes = [vp, vp, i64]
    for name in ("apic_create", "apic_create_batch", "apic_destroy", "apic_inject", "apic_step", "apic_tallies",
                 "apic_solve_poisson", "apic_get_particles", "apic_get_field", "apic_stats", "apic_step_timed",
                 "apic_deposit_static", "apic_sensitivity", "apic_adjoint", "apic_autotune", "apic_probe_fp32_fma",
                 "apic_check_wait_limit", "apic_adjoint_window", "apic_set_schedule",
                 "apic_checkpoint_size", "apic_checkpoint_save", "apic_checkpoint_load"):
        getattr(L, name).restype = C.c_int
    _lib = L
    return L
