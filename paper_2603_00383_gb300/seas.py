"""Thin Python binding of the C ABI in include/seas.h (ctypes; argument marshalling only).

Every function has the C name and returns Python values instead of out-parameters; a negative status raises
``SeasError``.  Host arrays are float64 C-contiguous NumPy arrays (``SEAS_MEM_HOST``); device arrays are float64
contiguous CUDA tensors (anything with ``data_ptr()`` and ``is_cuda``), passed as raw pointers (``SEAS_MEM_DEVICE``).
All computation happens in libseas.so; if the library is missing this module raises instead of falling back.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libseas.so")

SEAS_OK = 0
SEAS_EINVAL, SEAS_ENOMEM, SEAS_ECUDA, SEAS_ESTATE, SEAS_EBUSY, SEAS_ETIMEOUT, SEAS_EIO = -1, -2, -3, -4, -5, -6, -7
SEAS_MEM_HOST, SEAS_MEM_DEVICE = 0, 1
SEAS_FLAG_DENSE, SEAS_FLAG_NO_TRUNC, SEAS_FLAG_STATIC_TAIL, SEAS_FLAG_LAG_CAP = 1, 2, 4, 8
SEAS_FLAG_CLUSTER_TRUNC = 16
SEAS_FAULT_SURFACE_START = 1
SEAS_PREC_FP64, SEAS_PREC_BF16, SEAS_PREC_FP16S, SEAS_PREC_DF64 = 0, 1, 2, 3

EXPORTED = ["seas_create", "seas_build_network", "seas_net_get_info", "seas_net_get_elements", "seas_build_hmatrix",
            "seas_op_pair_windows", "seas_op_mode_windows", "seas_op_blocks", "seas_scenario_create",
            "seas_push_slip_rate", "seas_stress_step", "seas_scenario_step", "seas_sync", "seas_strerror",
            "seas_last_error", "seas_scenario_save", "seas_scenario_load", "seas_destroy_scn", "seas_destroy_op",
            "seas_destroy_net", "seas_destroy_ctx", "seas_plan_hmatrix", "seas_scenario_set_timing",
            "seas_scenario_get_timing", "seas_op_step_bytes", "seas_scenario_check", "seas_stress_step_static",
            "seas_measure_fp64_peak", "seas_scenario_set_wait_limit", "seas_scenario_probe_wait", "seas_scenario_admit",
            "seas_scenario_retire", "seas_scenario_member_step", "seas_ctx_get_memory", "seas_integrator_create",
            "seas_integrator_step", "seas_integrator_state", "seas_destroy_integrator", "seas_push_slip_rate_steps",
            "seas_integrator_step_gamma", "seas_integrator_step_adaptive", "seas_scenario_graph_create",
            "seas_scenario_graph_step", "seas_build_hmatrix_part", "seas_scenario_autotune"]


class SeasError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{msg} (status {status})")
        self.status = status


class seas_fault(C.Structure):
    _fields_ = [("cx", C.c_double), ("cy", C.c_double), ("strike_rad", C.c_double), ("length", C.c_double),
                ("n_elem", C.c_int32), ("flags", C.c_int32)]


class seas_medium(C.Structure):
    _fields_ = [("mu", C.c_double), ("cs", C.c_double), ("cp", C.c_double), ("beta", C.c_double)]


class seas_hparams(C.Structure):
    _fields_ = [("leaf", C.c_int32), ("q_w", C.c_int32), ("eta_h", C.c_double), ("aca_tol", C.c_double),
                ("eta_tmin", C.c_double), ("eta_tmax", C.c_double), ("eta_w", C.c_double),
                ("max_steps", C.c_int32), ("precision", C.c_int32), ("flags", C.c_int32), ("max_block", C.c_int32)]


class seas_net_info(C.Structure):
    _fields_ = [("dt", C.c_double), ("n_faults", C.c_int32), ("n_elem", C.c_int32)]


class seas_op_stats(C.Structure):
    _fields_ = [("n_blocks_near", C.c_int64), ("n_blocks_far", C.c_int64), ("n_slices_dense", C.c_int64),
                ("n_slices_lowrank", C.c_int64), ("n_slices_zero", C.c_int64), ("bytes_interaction", C.c_int64),
                ("bytes_dense_causal", C.c_int64), ("compression_ratio", C.c_double), ("bytes_self", C.c_int64),
                ("max_rank", C.c_int32), ("ring_depth", C.c_int32), ("mean_rank", C.c_double),
                ("build_seconds", C.c_double), ("n_tasks", C.c_int64)]


class seas_friction(C.Structure):
    _fields_ = [("a", C.c_double), ("b", C.c_double), ("dc", C.c_double), ("f0", C.c_double), ("v0", C.c_double),
                ("sigma_n", C.c_double)]


class seas_timing(C.Structure):
    _fields_ = [("launches", C.c_int64 * 7), ("ms", C.c_double * 7), ("interaction_bytes", C.c_int64),
                ("steps", C.c_int64)]


class seas_tune(C.Structure):
    _fields_ = [("consumer_warps", C.c_int * 2), ("candidates", (C.c_int * 2) * 2), ("ms", (C.c_double * 2) * 2),
                ("from_cache", C.c_int)]


KERNEL_CLASSES = ["push", "fft_forward", "modeconv", "interaction", "reduce", "ifft_assemble", "interaction_source"]

_lib = None
_VP, _PP = C.c_void_p, C.POINTER(C.c_void_p)
_SIGS = {
    "seas_create": ([_PP, C.c_int, C.c_size_t, _VP], C.c_int),
    "seas_build_network": ([_VP, C.POINTER(seas_fault), C.c_int, C.POINTER(seas_medium), _PP], C.c_int),
    "seas_net_get_info": ([_VP, C.POINTER(seas_net_info)], C.c_int),
    "seas_net_get_elements": ([_VP, _VP, _VP], C.c_int),
    "seas_build_hmatrix": ([_VP, C.POINTER(seas_hparams), _PP, C.POINTER(seas_op_stats)], C.c_int),
    "seas_op_pair_windows": ([_VP, _VP], C.c_int),
    "seas_op_mode_windows": ([_VP, _VP], C.c_int),
    "seas_op_blocks": ([_VP, _VP, C.c_int64, _VP], C.c_int),
    "seas_scenario_create": ([_VP, C.c_int, _PP], C.c_int),
    "seas_push_slip_rate": ([_VP, _VP, _VP, C.c_int, C.c_int], C.c_int),
    "seas_stress_step": ([_VP, _VP, _VP, _VP, C.c_int], C.c_int),
    "seas_scenario_step": ([_VP, C.POINTER(C.c_int64)], C.c_int),
    "seas_sync": ([_VP], C.c_int),
    "seas_strerror": ([C.c_int], C.c_char_p),
    "seas_last_error": ([], C.c_char_p),
    "seas_scenario_save": ([_VP, C.c_char_p], C.c_int),
    "seas_scenario_load": ([_VP, C.c_char_p, _PP], C.c_int),
    "seas_destroy_scn": ([_VP], C.c_int),
    "seas_destroy_op": ([_VP], C.c_int),
    "seas_destroy_net": ([_VP], C.c_int),
    "seas_destroy_ctx": ([_VP], C.c_int),
    "seas_plan_hmatrix": ([C.POINTER(seas_fault), C.c_int, C.POINTER(seas_medium), C.POINTER(seas_hparams), _VP,
                           C.c_int64, C.POINTER(C.c_int64), _VP, _VP, C.POINTER(C.c_double)], C.c_int),
    "seas_scenario_set_timing": ([_VP, C.c_int], C.c_int),
    "seas_scenario_get_timing": ([_VP, C.POINTER(seas_timing)], C.c_int),
    "seas_op_step_bytes": ([_VP, C.c_int64, C.POINTER(C.c_int64)], C.c_int),
    "seas_scenario_check": ([_VP], C.c_int),
    "seas_stress_step_static": ([_VP, _VP, _VP], C.c_int),
    "seas_measure_fp64_peak": ([C.c_int, C.POINTER(C.c_double)], C.c_int),
    "seas_scenario_set_wait_limit": ([_VP, C.c_double], C.c_int),
    "seas_scenario_probe_wait": ([_VP], C.c_int),
    "seas_scenario_admit": ([_VP, C.c_int], C.c_int),
    "seas_scenario_retire": ([_VP, C.c_int], C.c_int),
    "seas_scenario_member_step": ([_VP, C.c_int, C.POINTER(C.c_int64)], C.c_int),
    "seas_ctx_get_memory": ([_VP, C.POINTER(C.c_size_t), C.POINTER(C.c_size_t)], C.c_int),
    "seas_integrator_create": ([_VP, C.POINTER(seas_friction), C.c_int, C.c_double, _VP, _VP, _VP, C.c_int, _PP],
                               C.c_int),
    "seas_integrator_step": ([_VP, C.c_int], C.c_int),
    "seas_integrator_state": ([_VP, _VP, _VP, _VP, C.c_int], C.c_int),
    "seas_destroy_integrator": ([_VP], C.c_int),
    "seas_push_slip_rate_steps": ([_VP, _VP, _VP, C.c_int, C.c_int, C.c_int], C.c_int),
    "seas_integrator_step_gamma": ([_VP, C.c_int], C.c_int),
    "seas_integrator_step_adaptive": ([_VP, C.c_double, C.c_int, C.c_int, C.POINTER(C.c_int64)], C.c_int),
    "seas_scenario_graph_create": ([_VP, _VP, _VP, _VP], C.c_int),
    "seas_scenario_graph_step": ([_VP], C.c_int),
    "seas_build_hmatrix_part": ([_VP, C.POINTER(seas_hparams), _VP, C.c_int, _PP, C.POINTER(seas_op_stats)], C.c_int),
    "seas_scenario_autotune": ([_VP, C.c_char_p, C.c_int, C.POINTER(seas_tune)], C.c_int),
}


def lib(path: str = LIB_PATH) -> C.CDLL:
    """Loads libseas.so (built in-tree by ``paper_2603_00383_gb300.build``).  Raises if it is missing."""
    global _lib
    if _lib is None:
        if not os.path.exists(path):
            raise FileNotFoundError(f"{path} is missing: build it with `python -m paper_2603_00383_gb300.build`")
        L = C.CDLL(path)
        for name, (args, res) in _SIGS.items():
            fn = getattr(L, name)
            fn.argtypes = args
            fn.restype = res
        _lib = L
    return _lib


def _check(status: int):
    if status < 0:
        raise SeasError(status, f"{seas_strerror(status)}: {lib().seas_last_error().decode()}")


class Handle:
    """An opaque library handle plus the sizes the binding needs to check buffers."""

    def __init__(self, ptr, kind, **meta):
        self.ptr = ptr
        self.kind = kind
        self.__dict__.update(meta)


def _buf(x, n: int, what: str, device: int = None):
    """(pointer, mem) of a float64 buffer of n elements: NumPy -> host, CUDA tensor -> device.  ``device``: the
    handle's GPU; a tensor on another GPU is rejected (the kernels would write through a foreign pointer)."""
    if x is None:
        return None, None
    if hasattr(x, "data_ptr") and getattr(x, "is_cuda", False):
        if str(x.dtype) != "torch.float64" or not x.is_contiguous() or x.numel() != n:
            raise ValueError(f"{what}: need a contiguous float64 CUDA tensor of {n} elements")
        if device is not None and x.device.index is not None and x.device.index != device:
            raise ValueError(f"{what}: tensor on cuda:{x.device.index}, the scenario lives on cuda:{device}")
        return C.c_void_p(x.data_ptr()), SEAS_MEM_DEVICE
    if not isinstance(x, np.ndarray) or x.dtype != np.float64 or not x.flags.c_contiguous or x.size != n:
        raise ValueError(f"{what}: need a C-contiguous float64 array of {n} elements")
    return C.c_void_p(x.ctypes.data), SEAS_MEM_HOST


def _device_of(scn: Handle) -> int:
    return scn.op.net.ctx.device


def seas_strerror(status: int) -> str:
    return lib().seas_strerror(status).decode()


def seas_last_error() -> str:
    return lib().seas_last_error().decode()


CUDA_STREAM_LEGACY = 1     # cudaStreamLegacy: the legacy default stream


def stream_handle(stream) -> int:
    """A cudaStream_t value for the library from a torch stream (or raw handle); the legacy default stream, whose
    handle is 0, becomes cudaStreamLegacy."""
    h = stream if isinstance(stream, int) else int(stream.cuda_stream)
    return h if h != 0 else CUDA_STREAM_LEGACY


def seas_create(device: int = 0, hbm_budget: int = 0, stream=None) -> Handle:
    """stream: None (the library owns a stream), a raw cudaStream_t value, or a torch.cuda.Stream."""
    h = C.c_void_p()
    st = None if stream is None else stream_handle(stream)
    _check(lib().seas_create(C.byref(h), device, hbm_budget, C.c_void_p(st) if st else None))
    return Handle(h, "ctx", device=device)


def _faults(faults):
    """faults: [F, 5] (cx, cy, strike_rad, length, n_elem) or [F, 6] with SEAS_FAULT_* flags in the last column."""
    faults = np.asarray(faults, dtype=np.float64)
    arr = (seas_fault * len(faults))()
    for i, row in enumerate(faults):
        cx, cy, s, L, n = row[:5]
        arr[i] = seas_fault(cx, cy, s, L, int(n), int(row[5]) if row.shape[0] > 5 else 0)
    return faults, arr


def _network_n_elem(faults) -> list:
    """Elements per fault of the network the library builds: twice N_f for faults on a free surface (method of
    images), whose operator queries report the doubled faults."""
    flags = faults[:, 5].astype(int) if faults.shape[1] > 5 else np.zeros(len(faults), dtype=int)
    return [int(n) * (2 if f & SEAS_FAULT_SURFACE_START else 1) for n, f in zip(faults[:, 4], flags)]


def _hparams(hp: dict) -> seas_hparams:
    return seas_hparams(int(hp.get("leaf", 32)), int(hp.get("q_w", 0)), float(hp.get("eta_h", 2.0)),
                        float(hp.get("aca_tol", 1e-6)), float(hp.get("eta_tmin", 0.01)),
                        float(hp.get("eta_tmax", 0.01)), float(hp.get("eta_w", 1.5)), int(hp["max_steps"]),
                        int(hp.get("precision", SEAS_PREC_FP64)), int(hp.get("flags", 0)),
                        int(hp.get("max_block", 0)))


def seas_plan_hmatrix(faults, mu: float, cs: float, cp: float, beta: float, hp: dict) -> dict:
    """Host-only plan: blocks [n, 7] (r0, p, c0, q, far, first_lag, last_lag), pair_last [F, F], mode windows per
    fault, dt."""
    faults, arr = _faults(faults)
    med = seas_medium(mu, cs, cp, beta)
    p = _hparams(hp)
    nb = C.c_int64()
    dt = C.c_double()
    F = len(faults)
    _check(lib().seas_plan_hmatrix(arr, F, C.byref(med), C.byref(p), None, 0, C.byref(nb), None, None,
                                   C.byref(dt)))
    blocks = np.zeros((nb.value, 7), dtype=np.int32)
    last = np.zeros((F, F), dtype=np.int32)
    nel = _network_n_elem(faults)
    mw = np.zeros(sum(n + 1 for n in nel), dtype=np.int32)
    _check(lib().seas_plan_hmatrix(arr, F, C.byref(med), C.byref(p), blocks.ctypes.data, nb.value, C.byref(nb),
                                   last.ctypes.data, mw.ctypes.data, C.byref(dt)))
    windows, o = [], 0
    for n in nel:
        windows.append(mw[o:o + n + 1].copy())
        o += n + 1
    return dict(blocks=blocks, pair_last=last, mode_windows=windows, dt=dt.value)


def seas_ctx_get_memory(ctx: Handle):
    """(bytes held by the context's handles, budget)."""
    u, b = C.c_size_t(), C.c_size_t()
    _check(lib().seas_ctx_get_memory(ctx.ptr, C.byref(u), C.byref(b)))
    return u.value, b.value


def seas_build_network(ctx: Handle, faults, mu: float, cs: float, cp: float = 6000.0, beta: float = 0.5) -> Handle:
    """faults: [F, 5] array (cx, cy, strike_rad, length, n_elem), or [F, 6] with SEAS_FAULT_* flags."""
    faults, arr = _faults(faults)
    med = seas_medium(mu, cs, cp, beta)
    h = C.c_void_p()
    _check(lib().seas_build_network(ctx.ptr, arr, len(faults), C.byref(med), C.byref(h)))
    info = seas_net_info()
    _check(lib().seas_net_get_info(h, C.byref(info)))
    return Handle(h, "net", ctx=ctx, N=info.n_elem, F=info.n_faults, dt=info.dt,
                  n_elem_net=_network_n_elem(faults))


def seas_net_get_info(net: Handle) -> dict:
    info = seas_net_info()
    _check(lib().seas_net_get_info(net.ptr, C.byref(info)))
    return dict(dt=info.dt, n_faults=info.n_faults, n_elem=info.n_elem)


def seas_net_get_elements(net: Handle):
    c = np.zeros((net.N, 2))
    n = np.zeros((net.N, 2))
    _check(lib().seas_net_get_elements(net.ptr, c.ctypes.data, n.ctypes.data))
    return c, n


def seas_build_hmatrix(net: Handle, hp: dict, owned=None):
    """hp keys: leaf, q_w, eta_h, aca_tol, eta_tmin, eta_tmax, eta_w, max_steps, precision, flags, max_block.
    owned: receiver faults of a partial operator (seas_build_hmatrix_part), None for all.
    Returns (op handle, stats dict)."""
    p = _hparams(hp)
    h = C.c_void_p()
    st = seas_op_stats()
    if owned is None:
        _check(lib().seas_build_hmatrix(net.ptr, C.byref(p), C.byref(h), C.byref(st)))
    else:
        f = np.ascontiguousarray(np.asarray(owned, dtype=np.int32))
        _check(lib().seas_build_hmatrix_part(net.ptr, C.byref(p), C.c_void_p(f.ctypes.data), len(f), C.byref(h),
                                             C.byref(st)))
    stats = {name: getattr(st, name) for name, _ in seas_op_stats._fields_}
    return Handle(h, "op", net=net, N=net.N, F=net.F, max_steps=p.max_steps), stats


def seas_op_pair_windows(op: Handle) -> np.ndarray:
    out = np.zeros((op.F, op.F), dtype=np.int32)
    _check(lib().seas_op_pair_windows(op.ptr, out.ctypes.data))
    return out


def seas_op_blocks(op: Handle) -> np.ndarray:
    """The operator's blocks, [n, 7] int32 rows (r0, p, c0, q, far, first_lag, last_lag)."""
    n = C.c_int64(0)
    _check(lib().seas_op_blocks(op.ptr, None, 0, C.byref(n)))
    out = np.zeros((n.value, 7), dtype=np.int32)
    _check(lib().seas_op_blocks(op.ptr, out.ctypes.data, n.value, C.byref(n)))
    return out


def seas_op_mode_windows(op: Handle) -> list:
    n_elem = op.net.n_elem_net
    flat = np.zeros(sum(n + 1 for n in n_elem), dtype=np.int32)
    _check(lib().seas_op_mode_windows(op.ptr, flat.ctypes.data))
    out, o = [], 0
    for n in n_elem:
        out.append(flat[o:o + n + 1].copy())
        o += n + 1
    return out


def seas_scenario_create(op: Handle, batch: int = 1) -> Handle:
    h = C.c_void_p()
    _check(lib().seas_scenario_create(op.ptr, batch, C.byref(h)))
    return Handle(h, "scn", op=op, N=op.N, B=batch)


def seas_push_slip_rate(scn: Handle, V, slip=None, replace_last: bool = False):
    n = scn.B * scn.N
    dev = _device_of(scn)
    pv, mem = _buf(V, n, "V", dev)
    ps, mem_s = _buf(slip, n, "slip", dev)
    if slip is not None and mem_s != mem:
        raise ValueError("V and slip must live in the same memory")
    _check(lib().seas_push_slip_rate(scn.ptr, pv, ps, mem, 1 if replace_last else 0))


def seas_push_slip_rate_steps(scn: Handle, V, gamma: int, slip=None, replace_last: bool = False):
    """V held over `gamma` lattice steps (slip integrated, or the straight line to `slip` at the last of them)."""
    n = scn.B * scn.N
    dev = _device_of(scn)
    pv, mem = _buf(V, n, "V", dev)
    ps, mem_s = _buf(slip, n, "slip", dev)
    if slip is not None and mem_s != mem:
        raise ValueError("V and slip must live in the same memory")
    _check(lib().seas_push_slip_rate_steps(scn.ptr, pv, ps, mem, int(gamma), 1 if replace_last else 0))


def seas_stress_step(scn: Handle, tau, sigma_n=None, parts=None):
    n = scn.B * scn.N
    dev = _device_of(scn)
    pt, mem = _buf(tau, n, "tau", dev)
    pn, mn = _buf(sigma_n, n, "sigma_n", dev)
    pp, mp = _buf(parts, 3 * n, "parts", dev)
    for m in (mn, mp):
        if m is not None and m != mem:
            raise ValueError("tau, sigma_n and parts must live in the same memory")
    _check(lib().seas_stress_step(scn.ptr, pt, pn, pp, mem))


def seas_stress_step_static(scn: Handle, tau, parts=None):
    """seas_stress_step into device buffers (CUDA tensors) with its scratch in a static device array, for callers
    that must not allocate device memory while stepping; limits and sharing rules are in include/seas.h."""
    n = scn.B * scn.N
    dev = _device_of(scn)
    pt, mem = _buf(tau, n, "tau", dev)
    pp, mp = _buf(parts, 3 * n, "parts", dev)
    if mem != SEAS_MEM_DEVICE or (mp is not None and mp != SEAS_MEM_DEVICE):
        raise ValueError("seas_stress_step_static takes device buffers")
    _check(lib().seas_stress_step_static(scn.ptr, pt, pp))


def seas_scenario_graph_create(scn: Handle, V, tau, parts=None):
    """Captures one step (push of the device buffer V, stress step into the device buffers tau / parts)."""
    n = scn.B * scn.N
    dev = _device_of(scn)
    pv, m0 = _buf(V, n, "V", dev)
    pt, m1 = _buf(tau, n, "tau", dev)
    pp, m2 = _buf(parts, 3 * n, "parts", dev)
    if m0 != SEAS_MEM_DEVICE or m1 != SEAS_MEM_DEVICE or (m2 is not None and m2 != SEAS_MEM_DEVICE):
        raise ValueError("seas_scenario_graph_create takes device buffers")
    _check(lib().seas_scenario_graph_create(scn.ptr, pv, pt, pp))


def seas_scenario_graph_step(scn: Handle):
    _check(lib().seas_scenario_graph_step(scn.ptr))


def seas_scenario_step(scn: Handle) -> int:
    n = C.c_int64()
    _check(lib().seas_scenario_step(scn.ptr, C.byref(n)))
    return n.value


def seas_scenario_admit(scn: Handle, member: int):
    _check(lib().seas_scenario_admit(scn.ptr, int(member)))


def seas_scenario_retire(scn: Handle, member: int):
    _check(lib().seas_scenario_retire(scn.ptr, int(member)))


def seas_scenario_member_step(scn: Handle, member: int) -> int:
    n = C.c_int64()
    _check(lib().seas_scenario_member_step(scn.ptr, int(member), C.byref(n)))
    return n.value


def seas_integrator_create(scn: Handle, friction, eps: float, tau0, V0, theta0) -> Handle:
    """friction: one (a, b, dc, f0, v0, sigma_n) tuple for every element, or a list of N of them."""
    fr = [friction] if isinstance(friction[0], (int, float)) else list(friction)
    arr = (seas_friction * len(fr))(*[seas_friction(*map(float, f)) for f in fr])
    n = scn.B * scn.N
    dev = _device_of(scn)
    pt, mem = _buf(tau0, n, "tau0", dev)
    pv, m1 = _buf(V0, n, "V0", dev)
    pth, m2 = _buf(theta0, n, "theta0", dev)
    if m1 != mem or m2 != mem:
        raise ValueError("tau0, V0 and theta0 must live in the same memory")
    h = C.c_void_p()
    _check(lib().seas_integrator_create(scn.ptr, arr, len(fr), float(eps), pt, pv, pth, mem, C.byref(h)))
    return Handle(h, "integ", scn=scn, N=scn.N, B=scn.B)


def seas_integrator_step(it: Handle, steps: int = 1):
    _check(lib().seas_integrator_step(it.ptr, int(steps)))


def seas_integrator_step_gamma(it: Handle, gamma: int):
    _check(lib().seas_integrator_step_gamma(it.ptr, int(gamma)))


def seas_integrator_step_adaptive(it: Handle, xi: float, gamma_max: int, steps: int = 1) -> int:
    """Returns the lattice steps advanced."""
    n = C.c_int64()
    _check(lib().seas_integrator_step_adaptive(it.ptr, float(xi), int(gamma_max), int(steps), C.byref(n)))
    return n.value


def seas_integrator_state(it: Handle):
    """(V, theta, slip) as host arrays [B * N]."""
    n = it.B * it.N
    V, th, d = np.zeros(n), np.zeros(n), np.zeros(n)
    _check(lib().seas_integrator_state(it.ptr, V.ctypes.data, th.ctypes.data, d.ctypes.data, SEAS_MEM_HOST))
    return V, th, d


def seas_destroy_integrator(it: Handle):
    _destroy(lib().seas_destroy_integrator, it)


def seas_scenario_set_timing(scn: Handle, enable: bool = True):
    _check(lib().seas_scenario_set_timing(scn.ptr, 1 if enable else 0))


def seas_scenario_get_timing(scn: Handle) -> dict:
    t = seas_timing()
    _check(lib().seas_scenario_get_timing(scn.ptr, C.byref(t)))
    return dict(launches={k: t.launches[i] for i, k in enumerate(KERNEL_CLASSES)},
                ms={k: t.ms[i] for i, k in enumerate(KERNEL_CLASSES)},
                interaction_bytes=t.interaction_bytes, steps=t.steps)


def seas_op_step_bytes(op: Handle, step: int) -> int:
    b = C.c_int64()
    _check(lib().seas_op_step_bytes(op.ptr, step, C.byref(b)))
    return b.value


def seas_measure_fp64_peak(device: int = 0) -> float:
    """FP64 FMA/s of the GPU, measured by the library's probe kernel."""
    r = C.c_double()
    _check(lib().seas_measure_fp64_peak(device, C.byref(r)))
    return r.value


def seas_scenario_set_wait_limit(scn: Handle, seconds: float):
    _check(lib().seas_scenario_set_wait_limit(scn.ptr, float(seconds)))


def seas_scenario_probe_wait(scn: Handle):
    _check(lib().seas_scenario_probe_wait(scn.ptr))


def seas_scenario_autotune(scn: Handle, cache_path=None, reps: int = 5) -> dict:
    """Consumer warps per interaction pass, picked by timing (seas_scenario_autotune); returns the choice, the
    candidates and their median launch times per pass (source, receiver)."""
    t = seas_tune()
    path = None if cache_path is None else os.fsencode(cache_path)
    _check(lib().seas_scenario_autotune(scn.ptr, path, int(reps), C.byref(t)))
    passes = ("source", "receiver")
    return {"consumer_warps": {passes[p]: t.consumer_warps[p] for p in range(2)},
            "ms": {passes[p]: {int(t.candidates[p][k]): t.ms[p][k] for k in range(2) if t.candidates[p][k]}
                   for p in range(2)},
            "from_cache": bool(t.from_cache)}


def seas_scenario_check(scn: Handle):
    _check(lib().seas_scenario_check(scn.ptr))


def seas_sync(ctx: Handle):
    _check(lib().seas_sync(ctx.ptr))


def seas_scenario_save(scn: Handle, path: str):
    _check(lib().seas_scenario_save(scn.ptr, path.encode()))


def seas_scenario_load(op: Handle, path: str) -> Handle:
    h = C.c_void_p()
    _check(lib().seas_scenario_load(op.ptr, path.encode(), C.byref(h)))
    with open(path, "rb") as fh:
        hdr = fh.read(24)
    B = int(np.frombuffer(hdr[12:16], dtype=np.int32)[0])
    return Handle(h, "scn", op=op, N=op.N, B=B)


def _destroy(fn, h: Handle):
    if h is not None and h.ptr:
        _check(fn(h.ptr))
        h.ptr = None


def seas_destroy_scn(h: Handle):
    _destroy(lib().seas_destroy_scn, h)


def seas_destroy_op(h: Handle):
    _destroy(lib().seas_destroy_op, h)


def seas_destroy_net(h: Handle):
    _destroy(lib().seas_destroy_net, h)


def seas_destroy_ctx(h: Handle):
    _destroy(lib().seas_destroy_ctx, h)


class Session:
    """Convenience owner of ctx -> net -> op -> scn for one workload; frees child first.  Without an explicit
    stream the library works on torch's current stream of `device` when torch is loaded (so that tensors the
    caller passes are ordered with the library's kernels), else on a stream of its own."""

    def __init__(self, workload, batch: int = 1, device: int = 0, stream=None, hbm_budget: int = 0, owned=None,
                 **hp):
        if stream is None:
            import sys
            torch = sys.modules.get("torch")
            if torch is not None and torch.cuda.is_available():
                stream = torch.cuda.current_stream(device)
        self.ctx = self.net = self.op = self.scn = None
        try:
            self.ctx = seas_create(device, hbm_budget, stream)
            self.net = seas_build_network(self.ctx, workload.faults, workload.mu, workload.cs, workload.cp,
                                          workload.beta)
            params = dict(workload.hparams)
            params.update(hp)
            self.op, self.stats = seas_build_hmatrix(self.net, params, owned)
            self.scn = seas_scenario_create(self.op, batch)
        except BaseException:
            self.close()
            raise

    def close(self):
        for fn, h in ((seas_destroy_scn, "scn"), (seas_destroy_op, "op"), (seas_destroy_net, "net"),
                      (seas_destroy_ctx, "ctx")):
            if getattr(self, h, None) is not None:
                fn(getattr(self, h))
                setattr(self, h, None)

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
