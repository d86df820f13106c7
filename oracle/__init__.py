"""ctypes wrapper of the FP64 CPU oracle (test infrastructure only).

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` import this package.  The product library never does.

The wrapper only marshals arguments; all arithmetic is in ``apic_oracle.c``.
"""
import ctypes as C

import numpy as np

from . import build as _build

NO_INJECT = 1
NO_FIELD = 2
CHORD = 4
FLOATING = 8
BOLTZMANN = 16
FE = 32
NT = 7
NH = 11


class _Species(C.Structure):
    _fields_ = [("q", C.c_double), ("m", C.c_double), ("T", C.c_double), ("n_init", C.c_int64)]


class _Config(C.Structure):
    _fields_ = [("alpha", C.c_double), ("x1_out", C.c_double), ("phi_g", C.c_double),
                ("phi_out", C.c_double), ("B", C.c_double), ("dt", C.c_double),
                ("e_bind_ion", C.c_double), ("n1", C.c_int32), ("n2", C.c_int32),
                ("n_species", C.c_int32), ("sp", _Species * 2), ("seed", C.c_uint64),
                ("instance", C.c_int32), ("flags", C.c_int32)]


_lib = None


def lib():
    global _lib
    if _lib is None:
        L = C.CDLL(_build.build())
        d, i32, i64, vp = C.c_double, C.c_int32, C.c_int64, C.c_void_p
        P = C.POINTER
        L.or_r_of.restype = d
        L.or_r_of.argtypes = [d, d, d]
        L.or_x1_of.restype = d
        L.or_x1_of.argtypes = [d, d, d]
        L.or_metric.argtypes = [d, d, d, P(d)]
        L.or_dA_dx2.restype = d
        L.or_dA_dx2.argtypes = [d, d, d]
        L.or_dOmega.restype = d
        L.or_dOmega.argtypes = [d, d, d]
        L.or_philox4x32.argtypes = [P(C.c_uint32), P(C.c_uint32), P(C.c_uint32)]
        L.or_gauss_legendre.argtypes = [C.c_int, P(d), P(d)]
        L.or_create.restype = vp
        L.or_create.argtypes = [P(_Config)]
        L.or_destroy.argtypes = [vp]
        L.or_load_volume.argtypes = [vp, C.c_int, i64]
        L.or_add_particles.argtypes = [vp, C.c_int, i64, P(d)]
        L.or_step.argtypes = [vp, C.c_int]
        L.or_deposit.argtypes = [vp]
        L.or_solve.argtypes = [vp, P(d), P(d)]
        L.or_solve_linear.argtypes = [vp, P(d), P(d)]
        L.or_newton_iterations.argtypes = [vp]
        L.or_apply_operator.argtypes = [vp, P(d), P(d)]
        L.or_gradients.argtypes = [vp]
        L.or_set_phi.argtypes = [vp, P(d)]
        L.or_push_only.argtypes = [vp]
        L.or_count.restype = i64
        L.or_count.argtypes = [vp, C.c_int]
        L.or_get_particles.argtypes = [vp, C.c_int, P(d), P(i64)]
        L.or_get_grid.argtypes = [vp, C.c_int, P(d)]
        L.or_get_bins.argtypes = [vp, P(d)]
        L.or_get_history.restype = i64
        L.or_get_history.argtypes = [vp, P(d)]
        L.or_get_counts.argtypes = [vp, P(i64)]
        L.or_get_scalars.argtypes = [vp, P(d)]
        L.or_surface.argtypes = [vp, P(d), P(d), P(d)]
        L.or_sample_table.restype = d
        L.or_sample_table.argtypes = [vp, C.c_int, d]
        L.or_tape_mode.argtypes = [vp, C.c_int]
        L.or_tape_get.restype = i64
        L.or_tape_get.argtypes = [vp, vp, P(i64), P(i64)]
        L.or_tape_set.argtypes = [vp, vp, i64, P(i64), i64]
        L.or_tape_status.argtypes = [vp]
        L.or_tape_ix_get.restype = i64
        L.or_tape_ix_get.argtypes = [vp, vp]
        L.or_tape_ix_set.argtypes = [vp, vp, i64]
        _lib = L
    return _lib


def _dp(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def r_of(alpha, x1, x2):
    return lib().or_r_of(alpha, x1, x2)


def x1_of(alpha, r, x2):
    return lib().or_x1_of(alpha, r, x2)


def metric(alpha, r, x2):
    out = np.zeros(4)
    lib().or_metric(alpha, r, x2, _dp(out))
    return out


def dA_dx2(alpha, x1, x2):
    return lib().or_dA_dx2(alpha, x1, x2)


def dOmega(alpha, x1, x2):
    return lib().or_dOmega(alpha, x1, x2)


def gauss_legendre(n):
    x, w = np.zeros(n), np.zeros(n)
    lib().or_gauss_legendre(n, _dp(x), _dp(w))
    return x, w


def philox(ctr, key):
    c = (C.c_uint32 * 4)(*[int(v) & 0xFFFFFFFF for v in ctr])
    k = (C.c_uint32 * 2)(*[int(v) & 0xFFFFFFFF for v in key])
    o = (C.c_uint32 * 4)()
    lib().or_philox4x32(c, k, o)
    return [int(v) for v in o]


def make_config(d):
    """dict (the workload keys shared with the product binding) -> oracle config."""
    c = _Config()
    for k in ("alpha", "x1_out", "phi_g", "phi_out", "B", "dt"):
        setattr(c, k, float(d[k]))
    c.e_bind_ion = float(d.get("e_bind_ion", 0.0))
    c.n1, c.n2 = int(d["n1"]), int(d["n2"])
    sps = d["species"]
    c.n_species = len(sps)
    for k, sp in enumerate(sps):
        c.sp[k].q, c.sp[k].m, c.sp[k].T = float(sp["q"]), float(sp["m"]), float(sp["T"])
        c.sp[k].n_init = int(sp["n_init"])
    c.seed = int(d.get("seed", 1))
    c.instance = int(d.get("instance", 0))
    flags = 0
    if d.get("no_inject"):
        flags |= NO_INJECT
    if d.get("no_field"):
        flags |= NO_FIELD
    if d.get("chord_absorb"):
        flags |= CHORD
    if d.get("floating"):
        flags |= FLOATING
    if d.get("boltzmann"):
        flags |= BOLTZMANN
    if d.get("fe_operator"):
        flags |= FE
    c.flags = flags
    return c


class Sim:
    """One oracle simulation (single instance)."""

    def __init__(self, cfg: dict):
        self.cfg = dict(cfg)
        self._c = make_config(cfg)
        self.h = lib().or_create(C.byref(self._c))
        if not self.h:
            raise ValueError("oracle rejected the configuration")
        self.n1, self.n2 = self._c.n1, self._c.n2
        self.ns = self._c.n_species

    def __del__(self):
        h = getattr(self, "h", None)
        if h:
            lib().or_destroy(h)
            self.h = None

    def load_volume(self, sp, n):
        lib().or_load_volume(self.h, sp, int(n))

    def add_particles(self, sp, state5):
        st = np.ascontiguousarray(state5, dtype=np.float64).reshape(-1, 5)
        lib().or_add_particles(self.h, sp, st.shape[0], _dp(st))

    def step(self, n=1):
        lib().or_step(self.h, int(n))

    def deposit(self):
        lib().or_deposit(self.h)

    def solve(self, rho=None):
        phi = np.zeros((self.n1 + 1) * (self.n2 + 1))
        r = None if rho is None else np.ascontiguousarray(rho, dtype=np.float64).ravel()
        rc = lib().or_solve(self.h, None if r is None else _dp(r), _dp(phi))
        if rc == -2:
            raise RuntimeError("Newton iteration did not converge")
        if rc != 0:
            raise RuntimeError("oracle has no Poisson matrix (no_field)")
        return phi.reshape(self.n1 + 1, self.n2 + 1)

    def solve_linear(self, rho):
        """Eqs. 6-7 for the charge density rho, whatever the electron model."""
        phi = np.zeros((self.n1 + 1) * (self.n2 + 1))
        r = np.ascontiguousarray(rho, dtype=np.float64).ravel()
        if lib().or_solve_linear(self.h, _dp(r), _dp(phi)) != 0:
            raise RuntimeError("oracle has no Poisson matrix (no_field)")
        return phi.reshape(self.n1 + 1, self.n2 + 1)

    def apply_operator(self, phi):
        """L phi at every node (see or_apply_operator)."""
        p = np.ascontiguousarray(phi, dtype=np.float64).ravel()
        out = np.zeros_like(p)
        lib().or_apply_operator(self.h, _dp(p), _dp(out))
        return out.reshape(self.n1 + 1, self.n2 + 1)

    def newton_iterations(self):
        return int(lib().or_newton_iterations(self.h))

    def push_only(self):
        lib().or_push_only(self.h)

    def gradients(self):
        lib().or_gradients(self.h)

    def set_phi(self, phi):
        """Replace the potential by the given node values [n1+1][n2+1]."""
        p = np.ascontiguousarray(phi, dtype=np.float64).reshape(self.n1 + 1, self.n2 + 1)
        lib().or_set_phi(self.h, _dp(p))

    def count(self, sp):
        return lib().or_count(self.h, sp)

    def particles(self, sp):
        n = self.count(sp)
        st = np.zeros((n, 5))
        ids = np.zeros(n, dtype=np.int64)
        lib().or_get_particles(self.h, sp, _dp(st), ids.ctypes.data_as(C.POINTER(C.c_int64)))
        return st, ids

    def grid(self, which):
        idx = {"rho": 0, "phi": 1, "G1": 2, "G2": 3, "V": 4}[which]
        out = np.zeros((self.n1 + 1) * (self.n2 + 1))
        lib().or_get_grid(self.h, idx, _dp(out))
        return out.reshape(self.n1 + 1, self.n2 + 1)

    def bins(self):
        out = np.zeros(self.ns * self.n2 * NT)
        lib().or_get_bins(self.h, _dp(out))
        return out.reshape(self.ns, self.n2, NT)

    def history(self):
        n = lib().or_get_history(self.h, None)
        out = np.zeros(max(n, 1) * NH)
        lib().or_get_history(self.h, _dp(out))
        return out[: n * NH].reshape(n, NH)

    def counts(self):
        out = np.zeros(12, dtype=np.int64)
        lib().or_get_counts(self.h, out.ctypes.data_as(C.POINTER(C.c_int64)))
        o = out.reshape(2, 6)
        keys = ("loaded", "injected", "absorbed", "escaped", "resident", "draws")
        return [dict(zip(keys, map(int, o[k]))) for k in range(self.ns)]

    def scalars(self):
        out = np.zeros(9)
        lib().or_get_scalars(self.h, _dp(out))
        keys = ("w0", "w1", "V_dom", "A_out", "A_grain", "lam0", "lam1", "Q", "FZ")
        return dict(zip(keys, map(float, out)))

    def surface(self):
        En = np.zeros(self.n2 + 1)
        q, fz = C.c_double(), C.c_double()
        lib().or_surface(self.h, _dp(En), C.byref(q), C.byref(fz))
        return En, q.value, fz.value

    def sample_table(self, which, u):
        return lib().or_sample_table(self.h, 0 if which == "volume" else 1, float(u))

    # ---- decision tape (frozen-decision runs) ----
    TAPE_OFF, TAPE_RECORD, TAPE_REPLAY = 0, 1, 2

    def tape_mode(self, mode):
        lib().or_tape_mode(self.h, int(mode))

    def tape(self):
        """(status bytes, injection counts, cells and table intervals) recorded so far."""
        n_nk = C.c_int64()
        n = lib().or_tape_get(self.h, None, None, C.byref(n_nk))
        st = np.zeros(max(n, 1), dtype=np.uint8)
        nk = np.zeros(max(n_nk.value, 1), dtype=np.int64)
        lib().or_tape_get(self.h, st.ctypes.data_as(C.c_void_p), nk.ctypes.data_as(C.POINTER(C.c_int64)),
                          C.byref(n_nk))
        ni = lib().or_tape_ix_get(self.h, None)
        ix = np.zeros(max(ni, 1), dtype=np.int32)
        lib().or_tape_ix_get(self.h, ix.ctypes.data_as(C.c_void_p))
        return st[:n].copy(), nk[: n_nk.value].copy(), ix[:ni].copy()

    def set_tape(self, tape):
        st, nk = (np.ascontiguousarray(a) for a in tape[:2])
        st = st.astype(np.uint8)
        nk = nk.astype(np.int64)
        lib().or_tape_set(self.h, st.ctypes.data_as(C.c_void_p), st.size,
                          nk.ctypes.data_as(C.POINTER(C.c_int64)), nk.size)
        if len(tape) > 2:
            ix = np.ascontiguousarray(tape[2], dtype=np.int32)
            lib().or_tape_ix_set(self.h, ix.ctypes.data_as(C.c_void_p), ix.size)

    def tape_ok(self):
        return lib().or_tape_status(self.h) == 0
