"""Thin Python binding of libtepai.so (include/tepai.h), argument marshalling only.

Every step of the MPS TE-PAI path runs in the library's CUDA kernels. If the
shared library is missing, importing this module raises; there is no
fallback. Problems and parameters are duck-typed objects with the fields of
tepai_problem / tepai_params (see the header).
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libtepai.so")

TEPAI_UNBIASED, TEPAI_NO_PI, TEPAI_TROTTER, TEPAI_CONTINUOUS = 0, 1, 2, 3
TEPAI_FP64, TEPAI_MIXED = 0, 1

EXPORTED = ["tepai_create", "tepai_destroy", "tepai_run", "tepai_sample_values",
            "tepai_export_circuit", "tepai_gnorm", "tepai_dev_workspace_size",
            "tepai_dev_prepare", "tepai_dev_execute", "tepai_dev_set_sample_offset",
            "tepai_dev_stats", "tepai_dev_release", "tepai_autotune", "tepai_evolve_state",
            "tepai_sample_values_static", "tepai_measure_peaks",
            "tepai_strerror", "tepai_last_cuda_error"]


class TepaiError(RuntimeError):
    def __init__(self, code: int, what: str):
        msg = _lib.tepai_strerror(code).decode()
        cu = _lib.tepai_last_cuda_error().decode()
        super().__init__(f"{what}: {msg} (code {code})" + (f" [cuda: {cu}]" if cu else ""))
        self.code = code


class Problem(C.Structure):
    _fields_ = [("n", C.c_int), ("periodic", C.c_int),
                ("Jx", C.POINTER(C.c_double)), ("Jy", C.POINTER(C.c_double)),
                ("Jz", C.POINTER(C.c_double)), ("h", C.POINTER(C.c_double)),
                ("init_bits", C.POINTER(C.c_ubyte))]


class Params(C.Structure):
    _fields_ = [("T", C.c_double), ("n_steps", C.c_longlong), ("delta", C.c_double),
                ("n_samples", C.c_longlong), ("sample_offset", C.c_longlong),
                ("run_steps", C.c_longlong), ("chi_max", C.c_int), ("cutoff", C.c_double),
                ("n_snapshots", C.c_int), ("obs_sites", C.POINTER(C.c_int)), ("n_obs", C.c_int),
                ("seed", C.c_ulonglong), ("variant", C.c_int), ("precision", C.c_int),
                ("launch_variant", C.c_int), ("obs_strings", C.POINTER(C.c_ubyte)),
                ("tie_rel", C.c_double), ("three_site", C.c_int)]


class Mps(C.Structure):
    _fields_ = [("bond_dims", C.POINTER(C.c_int)), ("tensors", C.POINTER(C.c_double))]


class Stats(C.Structure):
    _fields_ = [("events", C.c_double), ("gate_updates", C.c_double), ("swap_updates", C.c_double),
                ("qr_moves", C.c_double), ("jacobi_sweeps", C.c_double),
                ("max_discarded_weight", C.c_double), ("alg_flops", C.c_double),
                ("max_chi", C.c_int), ("n_not_converged", C.c_int),
                ("device_status", C.c_int * 3), ("phase_cycles", C.c_double * 8),
                ("grid_ctas", C.c_int), ("jacobi_pairs", C.c_double),
                ("jacobi_rotations", C.c_double), ("subphase_cycles", C.c_double * 12),
                ("sample_order", C.c_int), ("seconds", C.c_double), ("mean_nu", C.c_double),
                ("jacobi_reorth", C.c_double), ("tc_flops", C.c_double),
                ("three_site_updates", C.c_double)]

    PHASES = ("init", "sampler", "single_site", "theta", "jacobi", "truncate", "qr", "measure")
    SUBPHASES = ("qr_panel", "qr_apply", "qr_formq", "qr_rmul", "projection", "bulk_wait",
                 "jacobi_passes", "rank", "tc_gram", "tc_assemble", "tc_rounds", "tc_update")

    def as_dict(self):
        d = {f: getattr(self, f) for f, _ in self._fields_}
        d["device_status"] = list(self.device_status)
        d["phase_cycles"] = dict(zip(self.PHASES, list(self.phase_cycles)))
        d["subphase_cycles"] = dict(zip(self.SUBPHASES, list(self.subphase_cycles)))
        return d


class Event(C.Structure):
    _fields_ = [("j", C.c_int32), ("k", C.c_int32), ("v", C.c_int32), ("pad", C.c_int32)]


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"libtepai.so not built at {LIB_PATH}: run paper_2604_13144_gb300/build.py")
    lib = C.CDLL(LIB_PATH)
    vp, i, ll = C.c_void_p, C.c_int, C.c_longlong
    pd, pP, pQ, pM, pS = (C.POINTER(C.c_double), C.POINTER(Problem), C.POINTER(Params),
                          C.POINTER(Mps), C.POINTER(Stats))
    sig = {
        "tepai_create": (i, [C.POINTER(vp), i, vp]),
        "tepai_destroy": (None, [vp]),
        "tepai_run": (i, [vp, pP, pQ, pM, pd, pd, pd, pS]),
        "tepai_sample_values": (i, [vp, pP, pQ, pM, pd, C.POINTER(C.c_byte), pS]),
        "tepai_export_circuit": (i, [vp, pP, pQ, ll, C.POINTER(Event), ll, C.POINTER(ll)]),
        "tepai_gnorm": (i, [pP, pQ, pd, pd]),
        "tepai_dev_workspace_size": (i, [pP, pQ, i, C.POINTER(C.c_size_t)]),
        "tepai_dev_prepare": (i, [pP, pQ, pM, vp, C.c_size_t, i, vp]),
        "tepai_dev_execute": (i, [vp, vp, vp, vp, vp, vp, vp]),
        "tepai_dev_set_sample_offset": (i, [vp, ll]),
        "tepai_dev_stats": (i, [vp, pS, vp]),
        "tepai_dev_release": (i, [vp]),
        "tepai_autotune": (i, [vp, pP, pQ, pM, ll, C.POINTER(i), pd]),
        "tepai_evolve_state": (i, [vp, pP, pQ, pM, C.POINTER(i), pd, ll, C.POINTER(ll)]),
        "tepai_sample_values_static": (i, [pP, pQ, vp, vp, vp]),
        "tepai_measure_peaks": (i, [i, pd, pd, pd]),
        "tepai_strerror": (C.c_char_p, [i]),
        "tepai_last_cuda_error": (C.c_char_p, []),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    return lib


_lib = _load()


def _check(rc: int, what: str):
    if rc != 0:
        raise TepaiError(rc, what)


class Marshalled:
    """Keeps the numpy buffers alive for as long as the C structs point at them."""

    def __init__(self, prob, par, init=None):
        nb = prob.n if prob.periodic else prob.n - 1
        self.Jx = np.ascontiguousarray(prob.Jx[:nb], dtype=np.float64)
        self.Jy = np.ascontiguousarray(prob.Jy[:nb], dtype=np.float64)
        self.Jz = np.ascontiguousarray(prob.Jz[:nb], dtype=np.float64)
        self.h = np.ascontiguousarray(prob.h, dtype=np.float64)
        self.bits = np.ascontiguousarray(prob.init_bits, dtype=np.uint8)
        dp = lambda a: a.ctypes.data_as(C.POINTER(C.c_double))
        self.prob = Problem(int(prob.n), int(bool(prob.periodic)), dp(self.Jx), dp(self.Jy),
                            dp(self.Jz), dp(self.h), self.bits.ctypes.data_as(C.POINTER(C.c_ubyte)))
        obs = getattr(par, "obs_sites", None)
        strings = getattr(par, "obs_strings", None)
        self.strings = None
        if strings is not None:
            self.strings = np.ascontiguousarray(np.asarray(strings).reshape(-1, int(prob.n)), dtype=np.uint8)
            self.obs = None
            obs_p, nobs = None, int(self.strings.shape[0])
        elif obs is not None:
            self.obs = np.ascontiguousarray(obs, dtype=np.int32)
            obs_p, nobs = self.obs.ctypes.data_as(C.POINTER(C.c_int)), len(self.obs)
        else:
            self.obs = None
            obs_p, nobs = None, 0
        self.par = Params(float(par.T), int(par.n_steps), float(par.delta), int(par.n_samples),
                          int(getattr(par, "sample_offset", 0)), int(getattr(par, "run_steps", 0)),
                          int(par.chi_max), float(par.cutoff), int(par.n_snapshots), obs_p, nobs,
                          int(par.seed) & (2**64 - 1), int(getattr(par, "variant", 0)),
                          int(getattr(par, "precision", 0)), int(getattr(par, "launch_variant", 0)),
                          self.strings.ctypes.data_as(C.POINTER(C.c_ubyte)) if self.strings is not None
                          else None, float(getattr(par, "tie_rel", 0.0)), int(getattr(par, "three_site", 0)))
        self.n_obs = nobs if (obs is not None or self.strings is not None) else int(prob.n)
        self.M = int(par.n_snapshots)
        self.init = None
        if init is not None:
            tensors, dims = init
            self.dims = np.ascontiguousarray(dims, dtype=np.int32)
            flat = np.concatenate([np.asarray(t, dtype=np.complex128).reshape(-1) for t in tensors])
            self.tensors = np.ascontiguousarray(flat.view(np.float64))
            self.init = Mps(self.dims.ctypes.data_as(C.POINTER(C.c_int)), dp(self.tensors))

    def init_ptr(self):
        return C.byref(self.init) if self.init is not None else None


def tepai_create(device: int = 0, stream: int | None = None) -> C.c_void_p:
    ctx = C.c_void_p()
    _check(_lib.tepai_create(C.byref(ctx), int(device), stream), "tepai_create")
    return ctx


def tepai_destroy(ctx) -> None:
    _lib.tepai_destroy(ctx)


def tepai_run(ctx, prob, par, init=None):
    m = Marshalled(prob, par, init)
    mean = np.zeros((m.M, m.n_obs))
    se = np.zeros((m.M, m.n_obs))
    part = np.zeros((m.M, m.n_obs, 3))
    st = Stats()
    dp = lambda a: a.ctypes.data_as(C.POINTER(C.c_double))
    _check(_lib.tepai_run(ctx, C.byref(m.prob), C.byref(m.par), m.init_ptr(), dp(mean), dp(se),
                          dp(part), C.byref(st)), "tepai_run")
    return {"mean": mean, "stderr": se, "partials": part, "stats": st.as_dict()}


def tepai_sample_values(ctx, prob, par, init=None):
    m = Marshalled(prob, par, init)
    v = np.zeros((int(par.n_samples), m.M, m.n_obs))
    sg = np.zeros((int(par.n_samples), m.M), dtype=np.int8)
    st = Stats()
    _check(_lib.tepai_sample_values(ctx, C.byref(m.prob), C.byref(m.par), m.init_ptr(),
                                    v.ctypes.data_as(C.POINTER(C.c_double)),
                                    sg.ctypes.data_as(C.POINTER(C.c_byte)), C.byref(st)),
           "tepai_sample_values")
    return {"v": v, "sign": sg, "stats": st.as_dict()}


def tepai_export_circuit(ctx, prob, par, sample: int, cap: int = 1 << 20) -> np.ndarray:
    m = Marshalled(prob, par)
    buf = (Event * cap)()
    cnt = C.c_longlong()
    _check(_lib.tepai_export_circuit(ctx, C.byref(m.prob), C.byref(m.par), int(sample), buf, cap,
                                     C.byref(cnt)), "tepai_export_circuit")
    if cnt.value > cap:
        return tepai_export_circuit(ctx, prob, par, sample, cap=int(cnt.value))
    arr = np.frombuffer(buf, dtype=np.int32, count=4 * cnt.value).reshape(-1, 4)
    return arr[:, :3].astype(np.int64)


def tepai_gnorm(prob, par):
    m = Marshalled(prob, par)
    g = np.zeros(m.M)
    nu = C.c_double()
    _check(_lib.tepai_gnorm(C.byref(m.prob), C.byref(m.par),
                            g.ctypes.data_as(C.POINTER(C.c_double)), C.byref(nu)), "tepai_gnorm")
    return g, nu.value


def tepai_evolve_state(ctx, prob, par, init=None):
    """Final MPS of one circuit (par.n_samples == 1) as (tensors, dims): tensors
    in chain order, each (d_p, 2, d_{p+1}) complex128, in the layout `init`
    takes (so the result can start later runs)."""
    m = Marshalled(prob, par, init)
    n, cap = int(prob.n), int(par.chi_max)
    dims = np.zeros(n + 1, dtype=np.int32)
    buf = np.zeros(n * 2 * cap * cap * 2)
    used = C.c_longlong()
    _check(_lib.tepai_evolve_state(ctx, C.byref(m.prob), C.byref(m.par), m.init_ptr(),
                                   dims.ctypes.data_as(C.POINTER(C.c_int)),
                                   buf.ctypes.data_as(C.POINTER(C.c_double)), buf.size, C.byref(used)),
           "tepai_evolve_state")
    flat = buf[:int(used.value)].view(np.complex128)
    tensors, off = [], 0
    for p in range(n):
        cnt = int(dims[p]) * 2 * int(dims[p + 1])
        tensors.append(flat[off:off + cnt].reshape(int(dims[p]), 2, int(dims[p + 1])).copy())
        off += cnt
    return tensors, dims


def tepai_autotune(ctx, prob, par, init=None, trial_steps: int = 1):
    """Fastest launch variant for this problem on this device and its rate
    (two-site updates per second of kernel time); pass the variant as
    `launch_variant` in later runs."""
    m = Marshalled(prob, par, init)
    best, rate = C.c_int(), C.c_double()
    _check(_lib.tepai_autotune(ctx, C.byref(m.prob), C.byref(m.par),
                               C.byref(m.init) if m.init is not None else None, int(trial_steps),
                               C.byref(best), C.byref(rate)), "tepai_autotune")
    return int(best.value), float(rate.value)


class DeviceRun:
    """Device-resident path: the caller's torch tensors hold the workspace and
    the outputs; tepai_dev_execute launches kernels only."""

    def __init__(self, prob, par, init=None, grid_ctas: int = 0, stream=None, device="cuda"):
        import torch
        self.m = Marshalled(prob, par, init)
        nbytes = C.c_size_t()
        _check(_lib.tepai_dev_workspace_size(C.byref(self.m.prob), C.byref(self.m.par), int(grid_ctas),
                                             C.byref(nbytes)), "tepai_dev_workspace_size")
        self.ws = torch.empty(int(nbytes.value), dtype=torch.uint8, device=device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(device)
        init_dev = None
        if init is not None:
            self.d_dims = self.m.dims.copy()
            self.d_tensors = torch.from_numpy(self.m.tensors).to(device)
            init_dev = Mps(self.d_dims.ctypes.data_as(C.POINTER(C.c_int)),
                           C.cast(C.c_void_p(self.d_tensors.data_ptr()), C.POINTER(C.c_double)))
        self._init_dev = init_dev
        _check(_lib.tepai_dev_prepare(C.byref(self.m.prob), C.byref(self.m.par),
                                      C.byref(init_dev) if init_dev is not None else None,
                                      C.c_void_p(self.ws.data_ptr()), C.c_size_t(self.ws.numel()),
                                      int(grid_ctas), C.c_void_p(self.stream.cuda_stream)),
               "tepai_dev_prepare")
        M, no = self.m.M, self.m.n_obs
        self.mean = torch.zeros((M, no), dtype=torch.float64, device=device)
        self.stderr = torch.zeros((M, no), dtype=torch.float64, device=device)
        self.partials = torch.zeros((M, no, 3), dtype=torch.float64, device=device)

    def execute(self, v=None, sign=None):
        p = lambda t: C.c_void_p(t.data_ptr()) if t is not None else None
        _check(_lib.tepai_dev_execute(C.c_void_p(self.ws.data_ptr()), p(self.mean), p(self.stderr),
                                      p(self.partials), p(v), p(sign),
                                      C.c_void_p(self.stream.cuda_stream)), "tepai_dev_execute")

    def set_sample_offset(self, offset: int):
        _check(_lib.tepai_dev_set_sample_offset(C.c_void_p(self.ws.data_ptr()), int(offset)),
               "tepai_dev_set_sample_offset")

    def stats(self):
        st = Stats()
        _check(_lib.tepai_dev_stats(C.c_void_p(self.ws.data_ptr()), C.byref(st),
                                    C.c_void_p(self.stream.cuda_stream)), "tepai_dev_stats")
        return st.as_dict()

    def release(self):
        """Drop the library's bookkeeping and captured graph of this workspace."""
        if getattr(self, "ws", None) is not None:
            _lib.tepai_dev_release(C.c_void_p(self.ws.data_ptr()))
            self.ws = None

    def __del__(self):
        try:
            self.release()
        except Exception:
            pass


def tepai_measure_peaks(device: int = 0) -> dict:
    """Measured FP32-FMA, FP64-FMA and tcgen05 TF32 throughput of this device
    (TFLOP/s), from the library's own microbenchmarks."""
    f32, f64, t32 = C.c_double(), C.c_double(), C.c_double()
    _check(_lib.tepai_measure_peaks(int(device), C.byref(f32), C.byref(f64), C.byref(t32)),
           "tepai_measure_peaks")
    return {"fp32_tflops": f32.value, "fp64_tflops": f64.value, "tf32_tflops": t32.value}


def _check_device_out(t, dtype: str, numel: int, name: str):
    """A caller-owned output the kernel writes directly: it must be a contiguous
    CUDA tensor of the right dtype and exactly the right size, or the call is
    refused before any device work."""
    ok = (getattr(t, "is_cuda", False) and str(t.dtype) == f"torch.{dtype}" and t.is_contiguous()
          and int(t.numel()) == numel)
    if not ok:
        raise TepaiError(1, f"tepai_sample_values_static: {name} must be a contiguous CUDA {dtype} "
                            f"tensor of {numel} elements")


def tepai_sample_values_static(prob, par, d_v, d_sign, stream=None):
    """Per-sample values into caller-owned device tensors d_v (float64,
    [n_samples][M][n_obs]) and d_sign (int8, [n_samples][M]); the library
    allocates no device memory for this call (its scratch is a fixed static
    device array)."""
    m = Marshalled(prob, par)
    _check_device_out(d_v, "float64", int(par.n_samples) * m.M * m.n_obs, "d_v")
    _check_device_out(d_sign, "int8", int(par.n_samples) * m.M, "d_sign")
    st = stream.cuda_stream if stream is not None else None
    _check(_lib.tepai_sample_values_static(C.byref(m.prob), C.byref(m.par),
                                           C.c_void_p(d_v.data_ptr()), C.c_void_p(d_sign.data_ptr()),
                                           C.c_void_p(st) if st is not None else None),
           "tepai_sample_values_static")
