"""Python binding of libapic: `Sim` wraps one simulation object of the C ABI.

The binding marshals arguments only.  PyTorch provides the device memory (the
library's allocator callback is bound to torch's caching allocator) and the
stream (torch's current CUDA stream); all computation is in libapic.so.
"""
import ctypes as C

import numpy as np

from . import _abi

KEYS = ("alpha", "x1_out", "phi_g", "phi_out", "B", "dt")


class ApicError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("%s (%d): %s" % (_abi.ERRORS.get(code, "?"), code, msg))
        self.code = code


def probe_fp32_fma(stream=None, reps=4096):
    """FP32 CUDA-core throughput of the current GPU in TFLOP/s
    (apic_probe_fp32_fma)."""
    import torch
    lib = _abi.load()
    s = stream if stream is not None else torch.cuda.current_stream()
    out = C.c_double()
    rc = lib.apic_probe_fp32_fma(C.c_void_p(s.cuda_stream), int(reps), C.byref(out))
    if rc != 0:
        raise ApicError(rc, "apic_probe_fp32_fma failed")
    return out.value


def make_config(d, precision="fp32"):
    """Workload dict (the keys used by tests and bench) -> apic_config_t."""
    c = _abi.Config()
    c.alpha, c.x1_outer, c.phi_grain, c.phi_outer = (float(d[k]) for k in ("alpha", "x1_out", "phi_g", "phi_out"))
    c.B, c.dt = float(d["B"]), float(d["dt"])
    c.e_bind_ion = float(d.get("e_bind_ion", 0.0))
    c.n1, c.n2 = int(d["n1"]), int(d["n2"])
    sps = d["species"]
    c.n_species = len(sps)
    for k, sp in enumerate(sps):
        c.sp[k].q, c.sp[k].m, c.sp[k].T = float(sp["q"]), float(sp["m"]), float(sp["T"])
        c.sp[k].n_init = int(sp["n_init"])
        c.sp[k].capacity = int(sp.get("capacity", max(1024, int(1.6 * sp["n_init"]) + 4096)))
    c.seed = int(d.get("seed", 1))
    c.instance = int(d.get("instance", 0))
    prec = d.get("precision", precision)
    c.precision = _abi.FP64 if prec in ("fp64", _abi.FP64) else _abi.FP32_REFINED
    c.flags = ((_abi.NO_INJECT if d.get("no_inject") else 0) | (_abi.NO_FIELD if d.get("no_field") else 0) |
               (_abi.CHORD_ABSORB if d.get("chord_absorb") else 0) |
               (_abi.FLOATING if d.get("floating") else 0) | (_abi.BOLTZMANN if d.get("boltzmann") else 0) |
               (_abi.FE_OPERATOR if d.get("fe_operator") else 0))
    c.poisson_tol = float(d.get("poisson_tol", 0.0))
    c.poisson_max_iter = int(d.get("poisson_max_iter", 0))
    c.sort_interval = int(d.get("sort_interval", 0))
    c.history_cap = int(d.get("history_cap", 0))
    c.poisson_guess = int(d.get("poisson_guess", 0))
    c.newton_iters = int(d.get("newton_iters", 0))
    return c


class _TorchAllocator:
    """Binds the library's allocation callback to torch's caching allocator."""

    def __init__(self, device):
        import torch
        self.torch = torch
        self.device = device

        def _alloc(nbytes, stream, ctx):
            try:
                return int(torch.cuda.caching_allocator_alloc(int(nbytes), device=self.device, stream=stream))
            except Exception:
                return None

        def _free(ptr, stream, ctx):
            try:
                torch.cuda.caching_allocator_delete(ptr)
            except Exception:
                pass

        self._a = _abi.ALLOC_FN(_alloc)
        self._f = _abi.FREE_FN(_free)
        self.struct = _abi.Allocator(self._a, self._f, None)


class Sim:
    """One batch of instances on the current CUDA device and stream."""

    def __init__(self, cfg, precision="fp32", stream=None, use_torch_allocator=True):
        import torch
        self._lib = _abi.load()
        cfgs = cfg if isinstance(cfg, (list, tuple)) else [cfg]
        self.cfgs = [dict(c) for c in cfgs]
        arr = (_abi.Config * len(cfgs))(*[make_config(c, precision) for c in cfgs])
        self._cfg_arr = arr
        dev = torch.cuda.current_device()
        self.stream = stream if stream is not None else torch.cuda.current_stream(dev)
        self._alloc = _TorchAllocator(dev) if use_torch_allocator else None
        h = C.c_void_p()
        rc = self._lib.apic_create_batch(arr, len(cfgs), C.c_void_p(self.stream.cuda_stream),
                                         C.byref(self._alloc.struct) if self._alloc else None, C.byref(h))
        if rc != 0:
            raise ApicError(rc, "apic_create failed")
        self.h = h
        self.n_inst = len(cfgs)

    def _check(self, rc):
        if rc != 0:
            msg = self._lib.apic_last_error(self.h)
            raise ApicError(rc, msg.decode() if msg else "")

    def close(self):
        if getattr(self, "h", None):
            self._lib.apic_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ---- the ABI, one method per entry point ----
    def inject(self, species, n, mode=_abi.LOAD_VOLUME, state=None, instance=0):
        ptr = None
        if mode == _abi.EXPLICIT:
            st = np.ascontiguousarray(state, dtype=np.float64).reshape(-1, 5)
            n = st.shape[0]
            ptr = st.ctypes.data_as(C.POINTER(C.c_double))
        self._check(self._lib.apic_inject(self.h, instance, species, int(n), mode, ptr))

    def load_volume(self, species, n, instance=0):
        self.inject(species, n, _abi.LOAD_VOLUME, instance=instance)

    def add_particles(self, species, state, instance=0):
        self.inject(species, 0, _abi.EXPLICIT, state=state, instance=instance)

    def step(self, n=1):
        self._check(self._lib.apic_step(self.h, int(n)))

    def step_timed(self, n=1):
        self._check(self._lib.apic_step_timed(self.h, int(n)))

    def stats(self):
        st = _abi.Stats()
        self._check(self._lib.apic_stats(self.h, C.byref(st)))
        return dict(steps=int(st.steps), poisson_loop_iters=int(st.poisson_loop_iters),
                    kernels_per_step=int(st.kernels_per_step), kernels_per_iter=int(st.kernels_per_iter),
                    timed_steps=int(st.timed_steps),
                    phase_ms=dict(zip(_abi.PHASES, [float(v) for v in st.phase_ms])),
                    solver=_abi.SOLVERS[int(st.solver)], sorts=int(st.sorts),
                    kernels_per_sort=int(st.kernels_per_sort), sort_interval=int(st.sort_interval),
                    win_rows=int(st.win_rows), chunk_group=int(st.chunk_group), chunk_items=int(st.chunk_items),
                    timed_sorts=int(st.timed_sorts), sort_ms=float(st.sort_ms))

    def tallies(self, instance=0, history=True):
        c = self.cfgs[instance]
        ns, n2 = len(c["species"]), int(c["n2"])
        bins = np.zeros(ns * n2 * _abi.NT)
        cap = int(c.get("history_cap", 0) or 4096)
        hist = np.zeros(cap * _abi.NH) if history else None
        t = _abi.Tallies()
        t.bins = bins.ctypes.data_as(C.POINTER(C.c_double))
        if history:
            t.history = hist.ctypes.data_as(C.POINTER(C.c_double))
        t.history_rows = cap if history else 0
        self._check(self._lib.apic_tallies(self.h, instance, C.byref(t)))
        keys = ("loaded", "injected", "absorbed", "escaped", "resident", "dropped")
        counts = [dict(zip(keys, [int(v) for v in t.counts[s]])) for s in range(ns)]
        out = dict(bins=bins.reshape(ns, n2, _abi.NT), counts=counts, step=int(t.step), Q=t.grain_Q,
                   FZ=t.grain_FZ, poisson_res=t.poisson_res, poisson_iters=int(t.poisson_iters))
        if history:
            out["history"] = hist[: int(t.history_rows) * _abi.NH].reshape(-1, _abi.NH)
        return out

    def solve_poisson(self, rho=None, instance=0):
        c = self.cfgs[instance]
        shape = (int(c["n1"]) + 1, int(c["n2"]) + 1)
        phi = np.zeros(shape)
        r = None
        if rho is not None:
            rr = np.ascontiguousarray(rho, dtype=np.float64).reshape(shape)
            r = rr.ctypes.data_as(C.POINTER(C.c_double))
        self._check(self._lib.apic_solve_poisson(self.h, instance, r, phi.ctypes.data_as(C.POINTER(C.c_double))))
        return phi

    def particles(self, species, instance=0, capacity=None):
        c = self.cfgs[instance]
        sp = c["species"][species]
        cap = capacity or int(sp.get("capacity", max(1024, int(1.6 * sp["n_init"]) + 4096)))
        out = np.zeros((cap, 5))
        n = C.c_int64()
        self._check(self._lib.apic_get_particles(self.h, instance, species,
                                                 out.ctypes.data_as(C.POINTER(C.c_double)), cap, C.byref(n)))
        return out[: n.value]

    def field(self, which, instance=0):
        c = self.cfgs[instance]
        idx = {"rho": 0, "phi": 1, "G1": 2, "G2": 3, "V": 4}[which]
        out = np.zeros((int(c["n1"]) + 1, int(c["n2"]) + 1))
        self._check(self._lib.apic_get_field(self.h, instance, idx, out.ctypes.data_as(C.POINTER(C.c_double))))
        return out

    def sensitivity(self, n_steps):
        """Forward-mode sensitivities over a window of n_steps steps
        (apic_sensitivity): window means `values` [instances, 5] of (drag F_Z,
        electric F_Z, current, torque T_z, grain charge Q) and their
        derivatives `jacobian` [instances, 5, 3] along (alpha, phi_g, B)."""
        ni = len(self.cfgs)
        vals = np.zeros((ni, _abi.NOUT))
        jac = np.zeros((ni, _abi.NOUT, _abi.NPAR))
        dp = C.POINTER(C.c_double)
        self._check(self._lib.apic_sensitivity(self.h, int(n_steps), vals.ctypes.data_as(dp), jac.ctypes.data_as(dp)))
        return dict(values=vals, jacobian=jac)

    def adjoint(self, n_steps, dL_dout, values=False):
        """Gradient [instances, 3] of sum(dL_dout * window means) along
        (alpha, phi_g, B) by the reverse sweep (apic_adjoint_window); with
        values=True also the window means [instances, 5]."""
        ni = len(self.cfgs)
        g = np.ascontiguousarray(np.broadcast_to(np.asarray(dL_dout, dtype=np.float64), (ni, _abi.NOUT)))
        grad = np.zeros((ni, _abi.NPAR))
        vals = np.zeros((ni, _abi.NOUT))
        dp = C.POINTER(C.c_double)
        self._check(self._lib.apic_adjoint_window(self.h, int(n_steps), g.ctypes.data_as(dp), vals.ctypes.data_as(dp),
                                                  grad.ctypes.data_as(dp)))
        return (grad, vals) if values else grad

    def check_wait_limit(self, limit_ns):
        """apic_check_wait_limit: returns the status code (APIC_ERR_TIMEOUT,
        -6, is the expected one) without raising."""
        return int(self._lib.apic_check_wait_limit(self.h, int(limit_ns)))

    def checkpoint(self):
        """The state the next steps depend on, as a host byte array
        (apic_checkpoint_size / apic_checkpoint_save)."""
        n = C.c_int64()
        self._check(self._lib.apic_checkpoint_size(self.h, C.byref(n)))
        buf = np.zeros(int(n.value), dtype=np.uint8)
        self._check(self._lib.apic_checkpoint_save(self.h, buf.ctypes.data_as(C.c_void_p), int(n.value)))
        return buf

    def restore(self, buf):
        """Replace the state with a checkpoint of an object created with the
        same configurations (apic_checkpoint_load)."""
        b = np.ascontiguousarray(buf, dtype=np.uint8)
        self._check(self._lib.apic_checkpoint_load(self.h, b.ctypes.data_as(C.c_void_p), int(b.size)))

    def set_schedule(self, sort_interval=0, win_rows=0, chunk_group=0, chunk_items=0):
        """Apply a schedule chosen earlier (apic_set_schedule); 0 keeps a setting."""
        self._check(self._lib.apic_set_schedule(self.h, int(sort_interval), int(win_rows), int(chunk_group),
                                                int(chunk_items)))

    def autotune(self, steps_per_trial=16):
        """Sort-interval autotuning (apic_autotune): returns the interval kept
        and the measured ms per step of every candidate."""
        ms = np.zeros(len(_abi.TUNE_INTERVALS))
        chosen = C.c_int32()
        self._check(self._lib.apic_autotune(self.h, int(steps_per_trial), C.byref(chosen),
                                            ms.ctypes.data_as(C.POINTER(C.c_double))))
        return int(chosen.value), dict(zip(_abi.TUNE_INTERVALS, ms.tolist()))
