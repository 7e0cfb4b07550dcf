"""ctypes binding of libfllf.so (include/fllf.h).

Argument marshalling only: every step of the filter runs in the library's
CUDA kernels.  The functions keep the C names; a non-OK status raises
``FllfError`` carrying the status and ``fllf_last_error()``.  If the shared
library is missing, loading fails loudly (there is no fallback).
"""

import ctypes
import os

PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(PKG, "libfllf.so")

FLLF_OK, FLLF_EINVAL, FLLF_ENOMEM, FLLF_ECUDA, FLLF_EAGAIN, FLLF_ETIMEOUT, FLLF_EBUSY = range(7)
FLLF_FP32, FLLF_FP16, FLLF_BF16 = 0, 1, 2
FLLF_COEFF_QUADRATURE, FLLF_COEFF_CLOSED_FORM = 0, 1
FLLF_METHOD_FOURIER, FLLF_METHOD_FAST = 0, 1
PRECISIONS = {"fp32": FLLF_FP32, "fp16": FLLF_FP16, "bf16": FLLF_BF16}


class FllfError(RuntimeError):
    def __init__(self, status, detail):
        super().__init__(f"{status_name(status)}: {detail}")
        self.status = status
        self.detail = detail


class fllf_params(ctypes.Structure):
    _fields_ = [("H", ctypes.c_int), ("W", ctypes.c_int), ("C", ctypes.c_int),
                ("levels", ctypes.c_int), ("K", ctypes.c_int),
                ("m", ctypes.c_double), ("sigma_r", ctypes.c_double), ("T", ctypes.c_double),
                ("precision", ctypes.c_int), ("coeff_mode", ctypes.c_int),
                ("method", ctypes.c_int), ("samples", ctypes.c_int)]


class fllf_server_stats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_uint64), ("completed", ctypes.c_uint64),
                ("rejected", ctypes.c_uint64), ("p50_ms", ctypes.c_double),
                ("p99_ms", ctypes.c_double), ("mean_ms", ctypes.c_double),
                ("max_ms", ctypes.c_double), ("mpixel_per_s", ctypes.c_double),
                ("pool_bytes", ctypes.c_size_t), ("pool_peak_bytes", ctypes.c_size_t),
                ("max_active", ctypes.c_int), ("waves", ctypes.c_int),
                ("plan_cache_hits", ctypes.c_uint64), ("plan_cache_misses", ctypes.c_uint64),
                ("admission_quadratures", ctypes.c_uint64)]

    def as_dict(self):
        return {name: getattr(self, name) for name, _ in self._fields_}


_P = ctypes.c_void_p
_SIGS = {
    "fllf_status_str": (ctypes.c_char_p, [ctypes.c_int]),
    "fllf_last_error": (ctypes.c_char_p, []),
    "fllf_params_validate": (ctypes.c_int, [ctypes.POINTER(fllf_params)]),
    "fllf_coeffs": (ctypes.c_int, [ctypes.POINTER(fllf_params), ctypes.POINTER(ctypes.c_double)]),
    "fllf_plan_scratch_bytes": (ctypes.c_size_t, [ctypes.POINTER(fllf_params)]),
    "fllf_plan_create": (ctypes.c_int, [ctypes.POINTER(fllf_params), ctypes.c_int,
                                        ctypes.POINTER(_P)]),
    "fllf_plan_destroy": (ctypes.c_int, [_P]),
    "fllf_plan_params": (ctypes.c_int, [_P, ctypes.POINTER(fllf_params)]),
    "fllf_plan_coeffs": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_double)]),
    "fllf_run": (ctypes.c_int, [_P, _P, _P, _P]),
    "fllf_run_host": (ctypes.c_int, [_P, _P, _P, _P]),
    "fllf_submit": (ctypes.c_int, [_P, _P, _P, _P, ctypes.POINTER(ctypes.c_uint64)]),
    "fllf_submit_host": (ctypes.c_int, [_P, _P, _P, _P, ctypes.POINTER(ctypes.c_uint64)]),
    "fllf_poll": (ctypes.c_int, [ctypes.c_uint64, ctypes.c_int]),
    "fllf_batch_create": (ctypes.c_int, [ctypes.POINTER(_P), ctypes.c_int, ctypes.POINTER(_P)]),
    "fllf_batch_destroy": (ctypes.c_int, [_P]),
    "fllf_batch_run": (ctypes.c_int, [_P, ctypes.POINTER(_P), ctypes.POINTER(_P), _P]),
    "fllf_batch_check": (ctypes.c_int, [_P]),
    "fllf_batch_run_plans": (ctypes.c_int, [ctypes.POINTER(_P), ctypes.POINTER(_P), ctypes.POINTER(_P),
                                            ctypes.c_int, _P]),
    "fllf_plan_set_wait_test": (ctypes.c_int, [_P, ctypes.c_longlong, ctypes.c_uint]),
    "fllf_dataflow_check": (ctypes.c_int, [ctypes.POINTER(fllf_params), ctypes.c_int, ctypes.POINTER(ctypes.c_int),
                                           ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_int),
                                           ctypes.POINTER(ctypes.c_int)]),
    "fllf_run_noalloc": (ctypes.c_int, [ctypes.POINTER(fllf_params), _P, _P, _P]),
    "fllf_server_create": (ctypes.c_int, [ctypes.c_int, ctypes.c_size_t, ctypes.c_int,
                                          ctypes.c_int, ctypes.c_int, ctypes.POINTER(_P)]),
    "fllf_server_destroy": (ctypes.c_int, [_P]),
    "fllf_server_submit": (ctypes.c_int, [_P, ctypes.POINTER(fllf_params), _P, _P,
                                          ctypes.POINTER(ctypes.c_uint64)]),
    "fllf_server_poll": (ctypes.c_int, [_P, ctypes.c_uint64, ctypes.c_int]),
    "fllf_server_stats_get": (ctypes.c_int, [_P, ctypes.POINTER(fllf_server_stats)]),
    "fllf_server_stats_reset": (ctypes.c_int, [_P]),
    "fllf_plan_enable_timing": (ctypes.c_int, [_P, ctypes.c_int]),
    "fllf_plan_stage_times": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_double),
                                             ctypes.POINTER(ctypes.c_int)]),
    "fllf_optimal_period": (ctypes.c_int, [ctypes.c_double, ctypes.c_int, ctypes.c_double,
                                           ctypes.POINTER(ctypes.c_double)]),
    "fllf_run_adaptive": (ctypes.c_int, [_P, _P, _P, _P, _P]),
    "fllf_run_luma": (ctypes.c_int, [_P, _P, _P, _P]),
    "fllf_plan_set_timing_mask": (ctypes.c_int, [_P, ctypes.c_uint]),
    "fllf_plan_get_tuning": (ctypes.c_int, [_P, _P]),
    "fllf_plan_set_tuning": (ctypes.c_int, [_P, _P]),
    "fllf_plan_autotune": (ctypes.c_int, [_P, _P, _P, ctypes.c_int, _P, ctypes.POINTER(ctypes.c_double)]),
    "fllf_batch_get_ctas": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_int)]),
    "fllf_batch_get_mode": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)]),
    "fllf_batch_set_mode": (ctypes.c_int, [_P, ctypes.c_int, ctypes.POINTER(ctypes.c_int)]),
    "fllf_batch_set_ctas": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_int)]),
    "fllf_batch_autotune": (ctypes.c_int, [_P, ctypes.POINTER(_P), ctypes.POINTER(_P), ctypes.c_int, _P,
                                           ctypes.POINTER(ctypes.c_double)]),
}

STAGES = ("up0", "up", "down", "down0", "chain", "down_s", "graph")
TASK_KINDS = ("up0", "up", "down_s", "down10", "down0")


class fllf_tuning(ctypes.Structure):
    _fields_ = [("chain_pixels", ctypes.c_longlong), ("ctas_per_sm", ctypes.c_int * len(STAGES)),
                ("reduce_reverse", ctypes.c_int), ("small_pixels", ctypes.c_longlong),
                ("dataflow", ctypes.c_int), ("task_items", ctypes.c_int * len(TASK_KINDS)),
                ("dataflow_level", ctypes.c_int), ("reduce_bands", ctypes.c_int)]

    def as_dict(self):
        return {"chain_pixels": int(self.chain_pixels), "small_pixels": int(self.small_pixels),
                "ctas_per_sm": {s: int(self.ctas_per_sm[i]) for i, s in enumerate(STAGES)},
                "reduce_reverse": int(self.reduce_reverse), "dataflow": int(self.dataflow),
                "task_items": {s: int(self.task_items[i]) for i, s in enumerate(TASK_KINDS)},
                "dataflow_level": int(self.dataflow_level), "reduce_bands": int(self.reduce_bands)}

_lib = None


def lib():
    """The loaded libfllf.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(
                f"{LIB_PATH} is missing: build it with paper_2206_04681_gb300.build.build_library() "
                "(or __graft_entry__.build()); there is no non-CUDA fallback")
        handle = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            fn = getattr(handle, name, None)
            if fn is not None:
                fn.restype = res
                fn.argtypes = args
        _lib = handle
    return _lib


def status_name(s):
    try:
        return lib().fllf_status_str(s).decode()
    except Exception:  # library not loadable: still name the code
        return f"status {s}"


def _check(status):
    if status != FLLF_OK:
        raise FllfError(status, lib().fllf_last_error().decode())
    return status


def make_params(H, W, C=1, levels=5, K=8, m=3.0, sigma_r=0.2, T=2.0, precision=FLLF_FP32,
                coeff_mode=FLLF_COEFF_QUADRATURE, method=FLLF_METHOD_FOURIER, samples=0):
    if isinstance(precision, str):
        precision = PRECISIONS[precision]
    return fllf_params(int(H), int(W), int(C), int(levels), int(K), float(m), float(sigma_r),
                       float(T), int(precision), int(coeff_mode), int(method), int(samples))


def make_fast_params(H, W, C=1, levels=5, samples=16, m=3.0, sigma_r=0.2, precision=FLLF_FP32):
    """Parameters of a fast LLF plan (Sec. II-D) with S = ``samples``."""
    return make_params(H, W, C, levels, 1, m, sigma_r, 2.0, precision, FLLF_COEFF_QUADRATURE,
                       FLLF_METHOD_FAST, samples)


def fllf_params_validate(p):
    return lib().fllf_params_validate(ctypes.byref(p))


def fllf_coeffs(p):
    out = (ctypes.c_double * p.K)()
    _check(lib().fllf_coeffs(ctypes.byref(p), out))
    return list(out)


def fllf_run_adaptive(plan, d_in, d_gain, d_out, stream=None):
    """Pixel-by-pixel enhancement with a device gain map (Sec. III-B)."""
    _check(lib().fllf_run_adaptive(plan, _P(d_in), _P(d_gain), _P(d_out), _P(stream or 0)))


def fllf_run_luma(plan, d_rgb_in, d_rgb_out, stream=None):
    """Colour by luma: LLF on Y of BT.601 YUV, U and V kept (C == 1 plan)."""
    _check(lib().fllf_run_luma(plan, _P(d_rgb_in), _P(d_rgb_out), _P(stream or 0)))


def fllf_plan_set_timing_mask(plan, stages):
    """Time only the given stage kinds (names from STAGES); empty disables."""
    mask = 0
    for st in stages:
        mask |= 1 << STAGES.index(st)
    _check(lib().fllf_plan_set_timing_mask(plan, ctypes.c_uint(mask)))


def fllf_plan_get_tuning(plan):
    t = fllf_tuning()
    _check(lib().fllf_plan_get_tuning(plan, ctypes.byref(t)))
    return t


def fllf_plan_set_tuning(plan, t):
    _check(lib().fllf_plan_set_tuning(plan, ctypes.byref(t)))


def fllf_plan_autotune(plan, d_in, d_out, reps=10, stream=None):
    """Autotunes the plan's launch shape on the given device buffers; returns
    (tuning, best ms per run)."""
    ms = ctypes.c_double()
    _check(lib().fllf_plan_autotune(plan, _P(d_in), _P(d_out), int(reps), _P(stream or 0), ctypes.byref(ms)))
    return fllf_plan_get_tuning(plan), ms.value


def fllf_batch_get_ctas(batch):
    out = (ctypes.c_int * 4)()
    _check(lib().fllf_batch_get_ctas(batch, out))
    return list(out)


def fllf_batch_get_mode(batch):
    """(mode, task_items) of a batch's launch."""
    m = ctypes.c_int()
    ti = (ctypes.c_int * 5)()
    _check(lib().fllf_batch_get_mode(batch, ctypes.byref(m), ti))
    return m.value, list(ti)


def fllf_batch_set_mode(batch, mode, task_items=None):
    ti = (ctypes.c_int * 5)(*task_items) if task_items is not None else None
    _check(lib().fllf_batch_set_mode(batch, int(mode), ti))


def fllf_batch_set_ctas(batch, ctas):
    arr = (ctypes.c_int * 4)(*ctas)
    _check(lib().fllf_batch_set_ctas(batch, arr))


def fllf_batch_autotune(batch, d_in, d_out, reps=5, stream=None):
    """Autotunes the batch's per-stage CTA caps; returns (caps, best ms per run)."""
    n = len(d_in)
    ins = (_P * n)(*[_P(p) for p in d_in])
    outs = (_P * n)(*[_P(p) for p in d_out])
    ms = ctypes.c_double()
    _check(lib().fllf_batch_autotune(batch, ins, outs, int(reps), _P(stream or 0), ctypes.byref(ms)))
    return fllf_batch_get_ctas(batch), ms.value


def fllf_optimal_period(sigma_r, K, R):
    """Eq. (12) period for an R-tone image (host only)."""
    out = ctypes.c_double()
    _check(lib().fllf_optimal_period(float(sigma_r), int(K), float(R), ctypes.byref(out)))
    return out.value


def fllf_plan_scratch_bytes(p):
    return int(lib().fllf_plan_scratch_bytes(ctypes.byref(p)))


def fllf_plan_create(p, device=0):
    h = _P()
    _check(lib().fllf_plan_create(ctypes.byref(p), int(device), ctypes.byref(h)))
    return h


def fllf_plan_destroy(plan):
    _check(lib().fllf_plan_destroy(plan))


def fllf_plan_params(plan):
    out = fllf_params()
    _check(lib().fllf_plan_params(plan, ctypes.byref(out)))
    return out


def fllf_plan_coeffs(plan):
    p = fllf_plan_params(plan)
    out = (ctypes.c_double * p.K)()
    _check(lib().fllf_plan_coeffs(plan, out))
    return list(out)


def fllf_run(plan, d_in, d_out, stream=0):
    _check(lib().fllf_run(plan, _P(d_in), _P(d_out), _P(stream)))


def fllf_run_host(plan, h_in, h_out, stream=0):
    _check(lib().fllf_run_host(plan, _P(h_in), _P(h_out), _P(stream)))


def fllf_submit(plan, d_in, d_out, stream=0):
    t = ctypes.c_uint64()
    _check(lib().fllf_submit(plan, _P(d_in), _P(d_out), _P(stream), ctypes.byref(t)))
    return t.value


def fllf_submit_host(plan, h_in, h_out, stream=0):
    t = ctypes.c_uint64()
    _check(lib().fllf_submit_host(plan, _P(h_in), _P(h_out), _P(stream), ctypes.byref(t)))
    return t.value


def fllf_batch_create(plans):
    arr = (_P * len(plans))(*[p.value if isinstance(p, _P) else p for p in plans])
    h = _P()
    _check(lib().fllf_batch_create(arr, len(plans), ctypes.byref(h)))
    return h


def fllf_batch_destroy(batch):
    _check(lib().fllf_batch_destroy(batch))


def fllf_batch_run(batch, d_in, d_out, stream=0):
    """d_in, d_out: sequences of device addresses (one per plan of the batch)."""
    ins = (_P * len(d_in))(*d_in)
    outs = (_P * len(d_out))(*d_out)
    _check(lib().fllf_batch_run(batch, ins, outs, _P(stream)))


def fllf_batch_check(batch):
    _check(lib().fllf_batch_check(batch))


def fllf_batch_run_plans(plans, d_in, d_out, stream=0):
    """One-shot batch: builds a batch of the plans, runs it on the device
    buffers, waits for the stream and frees the batch."""
    n = len(plans)
    arr = (_P * n)(*[p.value if isinstance(p, _P) else p for p in plans])
    ins = (_P * n)(*d_in)
    outs = (_P * n)(*d_out)
    _check(lib().fllf_batch_run_plans(arr, ins, outs, n, _P(stream)))


def fllf_dataflow_check(params, task_items=None, with_d10=True, first_level=0):
    """Host-only check of the dataflow task list of the parameter sets;
    returns (tasks, bands) or raises FllfError with the reason."""
    n = len(params)
    arr = (fllf_params * n)(*params)
    ti = (ctypes.c_int * 5)(*task_items) if task_items is not None else None
    nt, nb = ctypes.c_int(), ctypes.c_int()
    _check(lib().fllf_dataflow_check(arr, n, ti, int(bool(with_d10)), int(first_level), ctypes.byref(nt),
                                     ctypes.byref(nb)))
    return nt.value, nb.value


def fllf_plan_set_wait_test(plan, wait_cycles=0, extra_arrivals=0):
    """Test hook: a shorter limit for the plan's bounded device waits and
    extra arrivals its chained launch's grid barriers wait for."""
    _check(lib().fllf_plan_set_wait_test(plan, int(wait_cycles), int(extra_arrivals)))


NOALLOC_SCRATCH_BYTES = 32 << 20
POLL_MAX_US = 60_000_000   # the longest wait of fllf_poll / fllf_server_poll (negative timeouts)


def fllf_run_noalloc(p, d_in, d_out, stream=0):
    """Filter with the library's fixed device scratch array (no allocation)."""
    _check(lib().fllf_run_noalloc(ctypes.byref(p), _P(d_in), _P(d_out), _P(stream)))


def fllf_plan_enable_timing(plan, enable=True):
    _check(lib().fllf_plan_enable_timing(plan, int(bool(enable))))


def fllf_plan_stage_times(plan):
    """{stage name: (total ms, launches)} since the previous call."""
    ms = (ctypes.c_double * len(STAGES))()
    n = (ctypes.c_int * len(STAGES))()
    _check(lib().fllf_plan_stage_times(plan, ms, n))
    return {name: (ms[i], n[i]) for i, name in enumerate(STAGES)}


def fllf_poll(ticket, timeout_us=-1):
    """Returns the raw status (FLLF_OK, FLLF_EAGAIN, FLLF_ETIMEOUT) or raises."""
    s = lib().fllf_poll(ctypes.c_uint64(ticket), int(timeout_us))
    if s in (FLLF_OK, FLLF_EAGAIN, FLLF_ETIMEOUT):
        return s
    _check(s)
    return s


def fllf_server_create(hbm_budget, max_slots=64, max_queue=4096, max_waves=2, device=0):
    h = _P()
    _check(lib().fllf_server_create(int(device), int(hbm_budget), int(max_slots), int(max_queue),
                                    int(max_waves), ctypes.byref(h)))
    return h


def fllf_server_destroy(server):
    _check(lib().fllf_server_destroy(server))


def fllf_server_submit(server, p, d_in, d_out):
    """Queues one image (device buffers); returns its ticket.  Raises FllfError
    with FLLF_EBUSY when the queue is full and FLLF_ENOMEM when the request can
    never fit the server's pool."""
    t = ctypes.c_uint64()
    _check(lib().fllf_server_submit(server, ctypes.byref(p), _P(d_in), _P(d_out), ctypes.byref(t)))
    return t.value


def fllf_server_poll(server, ticket, timeout_us=-1):
    """Returns FLLF_OK (done; the ticket is consumed), FLLF_EAGAIN or FLLF_ETIMEOUT; raises on failure."""
    s = lib().fllf_server_poll(server, ctypes.c_uint64(ticket), int(timeout_us))
    if s in (FLLF_OK, FLLF_EAGAIN, FLLF_ETIMEOUT):
        return s
    _check(s)
    return s


def fllf_server_stats_get(server):
    st = fllf_server_stats()
    _check(lib().fllf_server_stats_get(server, ctypes.byref(st)))
    return st.as_dict()


def fllf_server_stats_reset(server):
    _check(lib().fllf_server_stats_reset(server))
