"""Thin ctypes binding of liblbm.so (include/lbm.h).

Argument marshalling only: every step of the lattice Boltzmann update runs in
the library's CUDA kernels.  numpy arrays are passed as host pointers
(on_device = 0), CUDA torch tensors as device pointers (on_device = 1).  If
the shared library is missing or a call fails, an exception is raised; there
is no fallback implementation.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "liblbm.so")

D2Q9, D3Q19, D3Q27 = 0, 1, 2
SPACE_POPULATIONS, SPACE_RAW, SPACE_CENTRAL, SPACE_CUMULANT, SPACE_TRT = 0, 1, 2, 3, 4
SPACE_RAW_WEIGHTED = 5
EQ_DELTA, EQ_ABSOLUTE, EQ_DISCRETE2 = 0, 1, 2
STORE_F64, STORE_F32, STORE_F16_DELTA, STORE_BF16_DELTA, STORE_F64_ABSOLUTE = 0, 1, 2, 3, 4
ARITH_DEVIATION, ARITH_AS_WRITTEN = 0, 1
STEP_AUTO, STEP_DIRECT, STEP_STAGED = 0, 1, 2
FORCE_GUO, FORCE_HE = 0, 1
PULL, AA, ESOTERIC_TWIST, ESOTERIC_PULL, ESOTERIC_PUSH = 0, 1, 2, 3, 4
STREAMING_PATTERNS = (PULL, AA, ESOTERIC_TWIST, ESOTERIC_PULL, ESOTERIC_PUSH)
PERIODIC = 0
Q_OF = {D2Q9: 9, D3Q19: 19, D3Q27: 27}
ELEM_BYTES = {STORE_F64: 8, STORE_F32: 4, STORE_F16_DELTA: 2, STORE_BF16_DELTA: 2,
              STORE_F64_ABSOLUTE: 8}

ERRORS = {0: "ok", -1: "invalid argument", -2: "unsupported", -3: "inadmissible",
          -4: "device out of memory", -5: "CUDA error", -6: "non-finite populations",
          -7: "state mismatch"}


class LBMError(RuntimeError):
    def __init__(self, code, where=""):
        self.code = code
        super().__init__(f"{where}: {ERRORS.get(code, 'error')} ({code})")


class Params(ctypes.Structure):
    _fields_ = [("stencil", ctypes.c_int), ("space", ctypes.c_int),
                ("equilibrium", ctypes.c_int), ("storage", ctypes.c_int),
                ("streaming", ctypes.c_int), ("rates", ctypes.c_double * 6),
                ("dims", ctypes.c_int64 * 3), ("boundary", ctypes.c_int),
                ("stream", ctypes.c_void_p), ("arithmetic", ctypes.c_int)]


class Tuning(ctypes.Structure):
    _fields_ = [("threads", ctypes.c_int), ("cells_per_thread", ctypes.c_int),
                ("blocks_per_sm", ctypes.c_int), ("per_instance", ctypes.c_int)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class ClosureWeights(ctypes.Structure):
    """lbm_closure_weights: input normalisation and BF16 weight bits."""
    _fields_ = [("shift", ctypes.c_float * 7), ("scale", ctypes.c_float * 7),
                ("w", ctypes.c_uint16 * 1444)]


CLOSURE_NPARAM = 1444
_lib = None


def lib():
    """Load liblbm.so (raises OSError if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise OSError(f"{LIB_PATH} is missing: build it with "
                          "`python -m paper_2211_02435_b300.build`")
        L = ctypes.CDLL(LIB_PATH)
        vp, i64, c_int = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int
        d = ctypes.POINTER(ctypes.c_double)
        L.lbm_create.argtypes = [ctypes.POINTER(vp), ctypes.POINTER(Params)]
        L.lbm_init_velocity.argtypes = [vp, vp, vp, c_int]
        L.lbm_step.argtypes = [vp, i64]
        L.lbm_macroscopic.argtypes = [vp, vp, vp, c_int]
        L.lbm_run_host.argtypes = [vp, vp, vp, i64, vp, vp, c_int]
        L.lbm_set_divergence_check.argtypes = [vp, i64]
        L.lbm_get_populations.argtypes = [vp, vp, c_int]
        L.lbm_set_populations.argtypes = [vp, vp, c_int]
        L.lbm_invariants.argtypes = [vp, d]
        L.lbm_state_bytes.argtypes = [vp]
        L.lbm_state_bytes.restype = i64
        L.lbm_get_state.argtypes = [vp, vp, ctypes.c_size_t]
        L.lbm_set_state.argtypes = [vp, vp, ctypes.c_size_t]
        L.lbm_get_time.argtypes = [vp, ctypes.POINTER(i64), ctypes.POINTER(c_int)]
        L.lbm_set_rates.argtypes = [vp, d]
        L.lbm_set_stream.argtypes = [vp, vp]
        L.lbm_set_step_kernel.argtypes = [vp, c_int]
        L.lbm_set_wait_limit.argtypes = [vp, i64]
        L.lbm_set_force.argtypes = [vp, vp]
        L.lbm_set_force_field.argtypes = [vp, vp, c_int]
        L.lbm_set_force_model.argtypes = [vp, c_int]
        L.lbm_set_shallow_water.argtypes = [vp, ctypes.c_double]
        L.lbm_destroy.argtypes = [vp]
        L.lbm_destroy.restype = None
        L.lbm_error_string.argtypes = [c_int]
        L.lbm_error_string.restype = ctypes.c_char_p
        L.lbm_batch_create.argtypes = [ctypes.POINTER(vp), ctypes.POINTER(Params), c_int,
                                       ctypes.POINTER(i64), d]
        L.lbm_batch_init_velocity.argtypes = [vp, c_int, vp, vp, c_int]
        L.lbm_batch_init_tgv.argtypes = [vp, d]
        L.lbm_batch_step.argtypes = [vp, i64]
        L.lbm_batch_get_populations.argtypes = [vp, c_int, vp, c_int]
        L.lbm_batch_macroscopic.argtypes = [vp, c_int, vp, vp, c_int]
        L.lbm_batch_cells.argtypes = [vp]
        L.lbm_batch_cells.restype = i64
        L.lbm_batch_size.argtypes = [vp]
        L.lbm_batch_set_tuning.argtypes = [vp, ctypes.POINTER(Tuning)]
        L.lbm_batch_get_tuning.argtypes = [vp, ctypes.POINTER(Tuning)]
        L.lbm_batch_autotune.argtypes = [vp, c_int, ctypes.POINTER(Tuning), d]
        L.lbm_batch_get_time.argtypes = [vp, ctypes.POINTER(i64)]
        L.lbm_invariants_noalloc.argtypes = [c_int, c_int, vp, ctypes.POINTER(i64), vp, c_int, vp]
        L.lbm_set_closure.argtypes = [vp, ctypes.POINTER(ClosureWeights)]
        f32p = ctypes.POINTER(ctypes.c_float)
        L.lbm_trainer_create.argtypes = [ctypes.POINTER(vp), ctypes.POINTER(i64), ctypes.c_double,
                                         ctypes.c_double, c_int, vp]
        L.lbm_trainer_add_restricted.argtypes = [vp, vp]
        L.lbm_trainer_add_snapshot.argtypes = [vp, vp, c_int]
        L.lbm_trainer_snapshot_count.argtypes = [vp]
        L.lbm_trainer_get_snapshot.argtypes = [vp, c_int, vp, c_int]
        L.lbm_trainer_features.argtypes = [vp, c_int, vp, c_int]
        L.lbm_trainer_set_params.argtypes = [vp, f32p, f32p, f32p]
        L.lbm_trainer_get_params.argtypes = [vp, f32p]
        L.lbm_trainer_loss_grad.argtypes = [vp, c_int, d, d]
        L.lbm_trainer_set_unroll.argtypes = [vp, c_int]
        L.lbm_trainer_adam_step.argtypes = [vp, c_int, ctypes.c_double, d]
        L.lbm_trainer_export.argtypes = [vp, ctypes.POINTER(ClosureWeights)]
        L.lbm_trainer_destroy.argtypes = [vp]
        L.lbm_trainer_destroy.restype = None
        L.lbm_batch_destroy.argtypes = [vp]
        L.lbm_batch_destroy.restype = None
        _lib = L
    return _lib


def _check(rc, where):
    if rc != 0:
        raise LBMError(rc, where)


def _ptr(a, n_expected, writable=False):
    """(pointer, on_device) for a numpy array or a CUDA torch tensor."""
    if a is None:
        return None, 0
    if isinstance(a, np.ndarray):
        if a.dtype != np.float64 or not a.flags.c_contiguous:
            raise TypeError("expected a C-contiguous float64 array")
        if a.size != n_expected:
            raise ValueError(f"expected {n_expected} elements, got {a.size}")
        if writable and not a.flags.writeable:
            raise ValueError("array is read-only")
        return a.ctypes.data, 0
    if getattr(a, "is_cuda", False):  # torch tensor, duck-typed
        if str(a.dtype) != "torch.float64" or not a.is_contiguous():
            raise TypeError("expected a contiguous float64 CUDA tensor")
        if a.numel() != n_expected:
            raise ValueError(f"expected {n_expected} elements, got {a.numel()}")
        return a.data_ptr(), 1
    raise TypeError(f"unsupported buffer type {type(a)}")


def stream_handle(stream):
    """cudaStream_t value of a torch stream, an int handle, or None."""
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def invariants_noalloc(stencil, storage, df, dims, out=None, stream=None):
    """lbm_invariants_noalloc: FP64 invariants of a caller-owned device
    population field (a CUDA tensor of the storage type, slot i of cell c at
    i*N + c) without any device allocation in the library.  ``out``: None
    (returns a dict, host result) or a CUDA float64 tensor of 8 elements
    (filled asynchronously on ``stream``)."""
    dims = list(dims) + [1] * (3 - len(dims))
    d = (ctypes.c_int64 * 3)(*[int(v) for v in dims])
    ptr = df.data_ptr() if hasattr(df, "data_ptr") else int(df)
    if out is None:
        host = (ctypes.c_double * 8)()
        rc = lib().lbm_invariants_noalloc(stencil, storage, ptr, d, ctypes.addressof(host), 0,
                                          stream_handle(stream))
        _check(rc, "lbm_invariants_noalloc")
        keys = ("mass_dev", "jx", "jy", "jz", "energy", "max_u", "nonfinite", "cells")
        return dict(zip(keys, list(host)))
    p, dev = _ptr(out, 8, True)
    _check(lib().lbm_invariants_noalloc(stencil, storage, ptr, d, p, dev, stream_handle(stream)),
           "lbm_invariants_noalloc")
    return out


class Lattice:
    """One periodic domain advanced by the fused stream + collide step."""

    def __init__(self, stencil, space, equilibrium, storage, streaming, rates, dims,
                 stream=None, arithmetic=ARITH_DEVIATION):
        self.stencil, self.space, self.storage, self.streaming = stencil, space, storage, streaming
        self.equilibrium = equilibrium
        self.q = Q_OF[stencil]
        self.d = 2 if stencil == D2Q9 else 3
        dims = list(dims) + [1] * (3 - len(dims))
        self.dims = tuple(int(x) for x in dims)
        self.N = self.dims[0] * self.dims[1] * self.dims[2]
        r = list(rates) + [1.0] * (6 - len(rates))
        p = Params(stencil, space, equilibrium, storage, streaming, (ctypes.c_double * 6)(*r),
                   (ctypes.c_int64 * 3)(*self.dims), PERIODIC, stream_handle(stream),
                   int(arithmetic))
        h = ctypes.c_void_p()
        _check(lib().lbm_create(ctypes.byref(h), ctypes.byref(p)), "lbm_create")
        self._h = h

    def close(self):
        if getattr(self, "_h", None):
            lib().lbm_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    @property
    def handle(self):
        return self._h

    def init_velocity(self, rho, u):
        pr, dr = _ptr(rho, self.N)
        pu, du = _ptr(u, self.d * self.N)
        if rho is not None and dr != du:
            raise TypeError("rho and u must both be host or both be device buffers")
        _check(lib().lbm_init_velocity(self._h, pr, pu, du), "lbm_init_velocity")

    def step(self, n=1):
        _check(lib().lbm_step(self._h, int(n)), "lbm_step")

    def macroscopic(self, rho=None, u=None):
        """Fill rho[N] / u[d*N] (numpy or CUDA tensors).  With both None,
        allocates numpy arrays and returns them shaped as fields."""
        alloc = rho is None and u is None
        if alloc:
            rho = np.empty(self.N)
            u = np.empty(self.d * self.N)
        pr, dr = _ptr(rho, self.N, True)
        pu, du = _ptr(u, self.d * self.N, True)
        on_dev = dr if rho is not None else du
        _check(lib().lbm_macroscopic(self._h, pr, pu, on_dev), "lbm_macroscopic")
        if alloc:
            nx, ny, nz = self.dims
            return rho.reshape(nz, ny, nx), u.reshape(self.d, nz, ny, nx)
        return rho, u

    def run_host(self, rho, u, n, rho_out=None, u_out=None, slabs=0):
        """lbm_run_host: host fields in, n steps, host fields out, pipelined
        by slabs of z-planes (numpy float64 arrays; rho / outputs may be None)."""
        for a in (rho, u, rho_out, u_out):
            if a is not None and not isinstance(a, np.ndarray):
                raise TypeError("lbm_run_host takes host (numpy) arrays")
        pr, _ = _ptr(rho, self.N)
        pu, _ = _ptr(u, self.d * self.N)
        po, _ = _ptr(rho_out, self.N, True)
        pv, _ = _ptr(u_out, self.d * self.N, True)
        _check(lib().lbm_run_host(self._h, pr, pu, int(n), po, pv, int(slabs)), "lbm_run_host")

    def get_populations(self, out=None):
        alloc = out is None
        if alloc:
            out = np.empty(self.q * self.N)
        p, dev = _ptr(out, self.q * self.N, True)
        _check(lib().lbm_get_populations(self._h, p, dev), "lbm_get_populations")
        if alloc:
            nx, ny, nz = self.dims
            return out.reshape(self.q, nz, ny, nx)
        return out

    def set_populations(self, df):
        if isinstance(df, np.ndarray):
            df = np.ascontiguousarray(df, dtype=np.float64).reshape(-1)
        p, dev = _ptr(df, self.q * self.N)
        _check(lib().lbm_set_populations(self._h, p, dev), "lbm_set_populations")

    def invariants(self, check=True):
        out = (ctypes.c_double * 8)()
        rc = lib().lbm_invariants(self._h, out)
        if rc != -6 or check:
            _check(rc, "lbm_invariants")
        keys = ("mass_dev", "jx", "jy", "jz", "energy", "max_u", "nonfinite", "cells")
        return dict(zip(keys, list(out)))

    def state_bytes(self):
        return int(lib().lbm_state_bytes(self._h))

    def get_state(self):
        buf = np.empty(self.state_bytes(), dtype=np.uint8)
        _check(lib().lbm_get_state(self._h, buf.ctypes.data, buf.size), "lbm_get_state")
        return buf

    def set_state(self, buf):
        buf = np.ascontiguousarray(buf, dtype=np.uint8)
        _check(lib().lbm_set_state(self._h, buf.ctypes.data, buf.size), "lbm_set_state")

    def time(self):
        t, par = ctypes.c_int64(), ctypes.c_int()
        _check(lib().lbm_get_time(self._h, ctypes.byref(t), ctypes.byref(par)), "lbm_get_time")
        return t.value, par.value

    def set_rates(self, rates):
        r = list(rates) + [1.0] * (6 - len(rates))
        _check(lib().lbm_set_rates(self._h, (ctypes.c_double * 6)(*r)), "lbm_set_rates")

    def set_stream(self, stream):
        _check(lib().lbm_set_stream(self._h, stream_handle(stream)), "lbm_set_stream")

    def set_force(self, F):
        """Uniform body force F[D] (None removes it); Guo's model, include/lbm.h."""
        if F is None:
            _check(lib().lbm_set_force(self._h, None), "lbm_set_force")
            return
        arr = (ctypes.c_double * 3)(*[float(v) for v in list(F)[:3]])
        _check(lib().lbm_set_force(self._h, ctypes.cast(arr, ctypes.c_void_p)), "lbm_set_force")

    def set_force_model(self, model):
        """FORCE_GUO (default) or FORCE_HE (include/lbm.h)."""
        _check(lib().lbm_set_force_model(self._h, int(model)), "lbm_set_force_model")

    def set_force_field(self, F):
        """Per-cell body force [D, N] (numpy FP64 or a CUDA tensor); None removes it."""
        if F is None:
            _check(lib().lbm_set_force_field(self._h, None, 0), "lbm_set_force_field")
            return
        if isinstance(F, np.ndarray):
            F = np.ascontiguousarray(F, dtype=np.float64)
        p, dev = _ptr(F, self.d * self.N)
        _check(lib().lbm_set_force_field(self._h, p, dev), "lbm_set_force_field")

    def set_shallow_water(self, g):
        """Switch a D2Q9 absolute-storage CENTRAL / CUMULANT context to the
        shallow-water method with gravity g (0 switches back); include/lbm.h."""
        _check(lib().lbm_set_shallow_water(self._h, float(g)), "lbm_set_shallow_water")

    def set_divergence_check(self, every):
        """lbm_set_divergence_check: lbm_step checks f(n) for non-finite
        populations every `every` steps (0: off) and raises DIVERGED."""
        _check(lib().lbm_set_divergence_check(self._h, int(every)), "lbm_set_divergence_check")

    def set_step_kernel(self, kernel):
        """STEP_AUTO, STEP_DIRECT or STEP_STAGED (include/lbm.h)."""
        _check(lib().lbm_set_step_kernel(self._h, int(kernel)), "lbm_set_step_kernel")

    def set_wait_limit(self, cycles):
        """Bound (SM cycles) of the context's device waits (include/lbm.h)."""
        _check(lib().lbm_set_wait_limit(self._h, int(cycles)), "lbm_set_wait_limit")

    def set_closure(self, weights):
        """Enable the learned rates (a ClosureWeights) or disable them (None)."""
        ptr = None if weights is None else ctypes.byref(weights)
        _check(lib().lbm_set_closure(self._h, ptr), "lbm_set_closure")


class Batch:
    """Ensemble of independent periodic lattices advanced by one persistent
    launch per step (include/lbm_batch.h)."""

    def __init__(self, stencil, space, equilibrium, storage, rates, dims_list,
                 shear_rates=None, stream=None):
        self.stencil, self.space, self.storage = stencil, space, storage
        self.q = Q_OF[stencil]
        self.d = 2 if stencil == D2Q9 else 3
        self.dims = [tuple(int(v) for v in (list(dm) + [1] * (3 - len(dm)))) for dm in dims_list]
        n = len(self.dims)
        flat = (ctypes.c_int64 * (3 * n))(*[v for dm in self.dims for v in dm])
        r = list(rates) + [1.0] * (6 - len(rates))
        p = Params(stencil, space, equilibrium, storage, PULL, (ctypes.c_double * 6)(*r),
                   (ctypes.c_int64 * 3)(1, 1, 1), PERIODIC, stream_handle(stream), 0)
        sr = None if shear_rates is None else (ctypes.c_double * n)(*[float(x) for x in shear_rates])
        h = ctypes.c_void_p()
        _check(lib().lbm_batch_create(ctypes.byref(h), ctypes.byref(p), n, flat, sr),
               "lbm_batch_create")
        self._h = h

    def close(self):
        if getattr(self, "_h", None):
            lib().lbm_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __len__(self):
        return len(self.dims)

    def cells(self):
        return int(lib().lbm_batch_cells(self._h))

    def _n(self, k):
        nx, ny, nz = self.dims[k]
        return nx * ny * nz

    def init_velocity(self, k, rho, u):
        N = self._n(k)
        pr, dr = _ptr(rho, N)
        pu, du = _ptr(u, self.d * N)
        _check(lib().lbm_batch_init_velocity(self._h, int(k), pr, pu, du), "lbm_batch_init_velocity")

    def init_tgv(self, u0):
        u0 = np.ascontiguousarray(u0, dtype=np.float64)
        if u0.size != len(self):
            raise ValueError("one amplitude per instance")
        _check(lib().lbm_batch_init_tgv(self._h, u0.ctypes.data_as(ctypes.POINTER(ctypes.c_double))),
               "lbm_batch_init_tgv")

    def step(self, n=1):
        _check(lib().lbm_batch_step(self._h, int(n)), "lbm_batch_step")

    def get_populations(self, k):
        nx, ny, nz = self.dims[k]
        out = np.empty(self.q * self._n(k))
        _check(lib().lbm_batch_get_populations(self._h, int(k), out.ctypes.data, 0),
               "lbm_batch_get_populations")
        return out.reshape(self.q, nz, ny, nx)

    def macroscopic(self, k):
        nx, ny, nz = self.dims[k]
        rho = np.empty(self._n(k))
        u = np.empty(self.d * self._n(k))
        _check(lib().lbm_batch_macroscopic(self._h, int(k), rho.ctypes.data, u.ctypes.data, 0),
               "lbm_batch_macroscopic")
        return rho.reshape(nz, ny, nx), u.reshape(self.d, nz, ny, nx)

    def set_tuning(self, threads=128, cells_per_thread=4, blocks_per_sm=8, per_instance=0):
        t = Tuning(threads, cells_per_thread, blocks_per_sm, per_instance)
        _check(lib().lbm_batch_set_tuning(self._h, ctypes.byref(t)), "lbm_batch_set_tuning")

    def get_tuning(self):
        t = Tuning()
        _check(lib().lbm_batch_get_tuning(self._h, ctypes.byref(t)), "lbm_batch_get_tuning")
        return t.as_dict()

    def autotune(self, trial_steps=2, cache_path=None, key=None):
        """Pick the launch shape by timing (advances the ensemble: call before
        the init_* calls).  With cache_path, a JSON file maps key -> shape and
        a cached shape is applied without timing."""
        import json
        import os
        if cache_path and key and os.path.exists(cache_path):
            with open(cache_path) as f:
                cache = json.load(f)
            if key in cache:
                self.set_tuning(**cache[key]["tuning"])
                return cache[key]["tuning"], cache[key]["mlups"]
        t = Tuning()
        mlups = ctypes.c_double()
        _check(lib().lbm_batch_autotune(self._h, int(trial_steps), ctypes.byref(t),
                                        ctypes.byref(mlups)), "lbm_batch_autotune")
        if cache_path and key:
            cache = {}
            if os.path.exists(cache_path):
                with open(cache_path) as f:
                    cache = json.load(f)
            cache[key] = {"tuning": t.as_dict(), "mlups": mlups.value}
            with open(cache_path, "w") as f:
                json.dump(cache, f, indent=1)
        return t.as_dict(), mlups.value

    def time(self):
        t = ctypes.c_int64()
        _check(lib().lbm_batch_get_time(self._h, ctypes.byref(t)), "lbm_batch_get_time")
        return t.value


def _fp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_float))


def _dptr(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


class Trainer:
    """GPU trainer of the learned closure (include/lbm_closure.h)."""

    def __init__(self, coarse_dims, omega_shear, omega_bulk=1.0, max_snapshots=64, stream=None):
        self.dims = tuple(int(v) for v in coarse_dims)
        self.N = self.dims[0] * self.dims[1] * self.dims[2]
        d = (ctypes.c_int64 * 3)(*self.dims)
        h = ctypes.c_void_p()
        _check(lib().lbm_trainer_create(ctypes.byref(h), d, float(omega_shear), float(omega_bulk),
                                        int(max_snapshots), stream_handle(stream)),
               "lbm_trainer_create")
        self._h = h

    def close(self):
        if getattr(self, "_h", None):
            lib().lbm_trainer_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def add_restricted(self, fine):
        _check(lib().lbm_trainer_add_restricted(self._h, fine.handle), "lbm_trainer_add_restricted")

    def add_snapshot(self, df):
        df = np.ascontiguousarray(df, dtype=np.float64).reshape(-1)
        p, dev = _ptr(df, 27 * self.N)
        _check(lib().lbm_trainer_add_snapshot(self._h, p, dev), "lbm_trainer_add_snapshot")

    def count(self):
        return int(lib().lbm_trainer_snapshot_count(self._h))

    def snapshot(self, s):
        out = np.empty(27 * self.N)
        _check(lib().lbm_trainer_get_snapshot(self._h, int(s), out.ctypes.data, 0),
               "lbm_trainer_get_snapshot")
        nx, ny, nz = self.dims
        return out.reshape(27, nz, ny, nx)

    def features(self, s):
        out = np.empty(7 * self.N)
        _check(lib().lbm_trainer_features(self._h, int(s), out.ctypes.data, 0),
               "lbm_trainer_features")
        return out.reshape(7, self.N)

    def set_params(self, params, shift, scale):
        p = np.ascontiguousarray(params, dtype=np.float32)
        sh = np.ascontiguousarray(shift, dtype=np.float32)
        sc = np.ascontiguousarray(scale, dtype=np.float32)
        if p.size != CLOSURE_NPARAM or sh.size != 7 or sc.size != 7:
            raise ValueError("expected 1444 parameters and 7 shifts / scales")
        _check(lib().lbm_trainer_set_params(self._h, _fp(p), _fp(sh), _fp(sc)),
               "lbm_trainer_set_params")

    def params(self):
        p = np.empty(CLOSURE_NPARAM, dtype=np.float32)
        _check(lib().lbm_trainer_get_params(self._h, _fp(p)), "lbm_trainer_get_params")
        return p

    def set_unroll(self, K):
        """Steps of the rollout loss (1: one-step teacher forcing)."""
        _check(lib().lbm_trainer_set_unroll(self._h, int(K)), "lbm_trainer_set_unroll")
        self.unroll = int(K)

    def loss_grad(self, s):
        loss = np.zeros(1)
        grad = np.zeros(CLOSURE_NPARAM)
        _check(lib().lbm_trainer_loss_grad(self._h, int(s), _dptr(loss), _dptr(grad)),
               "lbm_trainer_loss_grad")
        return float(loss[0]), grad

    def adam_step(self, s, lr):
        loss = np.zeros(1)
        _check(lib().lbm_trainer_adam_step(self._h, int(s), float(lr), _dptr(loss)),
               "lbm_trainer_adam_step")
        return float(loss[0])

    def export(self):
        w = ClosureWeights()
        _check(lib().lbm_trainer_export(self._h, ctypes.byref(w)), "lbm_trainer_export")
        return w
