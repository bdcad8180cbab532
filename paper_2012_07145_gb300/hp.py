"""ctypes binding of the C ABI in include/hp.h (argument marshalling only).

Every computation runs in the CUDA kernels of libhp.so; this module only
converts Python values and torch tensors (used for device memory and streams)
into the plain pointers, sizes and structs the C ABI takes.  If the library is
missing, every call raises: there is no CPU fallback.
"""

import ctypes
import os

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "_lib", "libhp.so")

# ---- enums (mirror include/hp.h) -----------------------------------------
HP_OK, HP_ERR_INVALID_ARG, HP_ERR_UNSUPPORTED, HP_ERR_SCHEDULE, HP_ERR_OOM, HP_ERR_CUDA, HP_ERR_TIMEOUT, \
    HP_ERR_STATE = range(8)
HP_U8, HP_U16, HP_F16, HP_BF16, HP_F32, HP_U32 = range(6)
(HP_STENCIL, HP_POINTWISE, HP_DOWNSAMPLE2, HP_UPSAMPLE2, HP_HISTOGRAM, HP_CDF_LUT, HP_LUT_APPLY,
 HP_MAX_STENCIL, HP_GRID_SPLAT, HP_GRID_SLICE) = range(10)
(HP_OP_GRAY, HP_OP_MUL, HP_OP_ADD, HP_OP_SUB, HP_OP_HARRIS, HP_OP_UNSHARP, HP_OP_LL_REMAP, HP_OP_LL_INTERP,
 HP_OP_LL_COLOUR, HP_OP_SELECT, HP_OP_SCALE, HP_OP_PREMUL, HP_OP_OVER, HP_OP_UNPREMUL, HP_OP_ZBLUR) = range(15)
HP_INLINE = -1
HP_OPT_CUDA_GRAPH = 1
HP_OPT_OVERLAP = 2
HP_OPT_PROBE_ATTRS = 3
HP_IMPL_AUTO, HP_IMPL_GENERIC, HP_IMPL_WAVE, HP_IMPL_LINES = 0, 1, 2, 3
(HP_KERNEL_STENCIL_CHAIN, HP_KERNEL_UNSHARP, HP_KERNEL_HARRIS, HP_KERNEL_GENERIC, HP_KERNEL_POINTWISE,
 HP_KERNEL_DOWNSAMPLE, HP_KERNEL_UPSAMPLE, HP_KERNEL_HISTOGRAM, HP_KERNEL_CDF_LUT, HP_KERNEL_LUT_APPLY,
 HP_KERNEL_LL_LEVEL, HP_KERNEL_STENCIL_WAVE, HP_KERNEL_HARRIS_ROWS, HP_KERNEL_STENCIL_ROWS,
 HP_KERNEL_HISTEQ, HP_KERNEL_LL_REMAP_ROWS, HP_KERNEL_LL_DOWN_ROWS, HP_KERNEL_LL_LEVEL_ROWS,
 HP_KERNEL_MAX_ROWS, HP_KERNEL_INTERP_ROWS, HP_KERNEL_PW_ROWS, HP_KERNEL_GRID_SPLAT,
 HP_KERNEL_GRID_SLICE, HP_KERNEL_GRID_BLUR, HP_KERNEL_STENCIL_LINES) = range(25)
KERNEL_NAMES = ["stencil_chain", "unsharp", "harris", "generic", "pointwise", "downsample", "upsample",
                "histogram", "cdf_lut", "lut_apply", "ll_level", "stencil_wave", "harris_rows", "stencil_rows", "histeq",
                "ll_remap_rows", "ll_down_rows", "ll_level_rows", "max_rows", "interp_rows", "pw_rows", "grid_splat",
                "grid_slice", "grid_blur", "stencil_lines"]
DTYPE_BYTES = {HP_U8: 1, HP_U16: 2, HP_F16: 2, HP_BF16: 2, HP_F32: 4, HP_U32: 4}

_IP = ctypes.POINTER(ctypes.c_int)
_FP = ctypes.POINTER(ctypes.c_float)


class StageDesc(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("op", ctypes.c_int), ("n_inputs", ctypes.c_int), ("inputs", _IP),
                ("rx", ctypes.c_int), ("ry", ctypes.c_int), ("wx", _FP), ("wy", _FP), ("params", _FP),
                ("n_params", ctypes.c_int), ("storage", ctypes.c_int), ("channels", ctypes.c_int),
                ("boundary", ctypes.c_int)]


class Schedule(ctypes.Structure):
    _fields_ = [("n_stages", ctypes.c_int), ("group_of_stage", _IP), ("n_groups", ctypes.c_int),
                ("tile_w", _IP), ("tile_h", _IP), ("threads", _IP), ("serial_y", _IP), ("impl", _IP)]


class Buffer(ctypes.Structure):
    _fields_ = [("data", ctypes.c_void_p), ("dtype", ctypes.c_int), ("channels", ctypes.c_int),
                ("width", ctypes.c_int), ("height", ctypes.c_int), ("row_stride_bytes", ctypes.c_longlong),
                ("plane_stride_bytes", ctypes.c_longlong)]


class GroupInfo(ctypes.Structure):
    _fields_ = [("kernel", ctypes.c_int), ("output_stage", ctypes.c_int), ("n_members", ctypes.c_int),
                ("tile_w", ctypes.c_int), ("tile_h", ctypes.c_int), ("threads", ctypes.c_int),
                ("grid_x", ctypes.c_int), ("grid_y", ctypes.c_int), ("grid_z", ctypes.c_int),
                ("smem_bytes", ctypes.c_int)]


class ServerStats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_ulonglong), ("completed", ctypes.c_ulonglong), ("failed", ctypes.c_ulonglong),
                ("batched_launches", ctypes.c_ulonglong), ("peak_bytes", ctypes.c_ulonglong),
                ("p50_us", ctypes.c_double), ("p99_us", ctypes.c_double), ("mean_us", ctypes.c_double),
                ("max_us", ctypes.c_double), ("mpix", ctypes.c_double), ("busy_s", ctypes.c_double),
                ("graph_replays", ctypes.c_ulonglong), ("resident_bytes", ctypes.c_ulonglong),
                ("device_requests", ctypes.c_ulonglong), ("evictions", ctypes.c_ulonglong)]


EXPORTS = ["hp_pipeline_create", "hp_add_stage", "hp_set_output", "hp_schedule_set", "hp_realize",
           "hp_realize_host", "hp_group_info_get", "hp_group_count", "hp_infer_bounds", "hp_set_option", "hp_check_device_error",
           "hp_pipeline_destroy", "hp_last_error", "hp_launch_count", "hp_histeq_u8_noalloc",
           "hp_server_create", "hp_server_submit", "hp_server_wait", "hp_server_stats_get", "hp_server_destroy",
           "hp_prepare", "hp_server_prepare", "hp_measure_fp32_peak", "hp_kernel_attrs_get",
           "hp_server_submit_device", "hp_realize_host_async", "hp_realize_host_wait"]

_lib = None


def lib():
    """The loaded libhp.so; raises if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"libhp.so not found at {LIB_PATH}: build it with __graft_entry__.build()")
        L = ctypes.CDLL(LIB_PATH)
        P = ctypes.c_void_p
        L.hp_pipeline_create.argtypes = [ctypes.POINTER(P), ctypes.c_int, _IP, _IP]
        L.hp_add_stage.argtypes = [P, ctypes.POINTER(StageDesc), _IP]
        L.hp_set_output.argtypes = [P, ctypes.c_int]
        L.hp_schedule_set.argtypes = [P, ctypes.POINTER(Schedule)]
        L.hp_realize.argtypes = [P, ctypes.POINTER(Buffer), ctypes.c_int, ctypes.POINTER(Buffer), P]
        L.hp_realize_host.argtypes = [P, ctypes.POINTER(Buffer), ctypes.c_int, ctypes.POINTER(Buffer), P]
        L.hp_realize_host_async.argtypes = [P, ctypes.POINTER(Buffer), ctypes.c_int, ctypes.POINTER(Buffer), P]
        L.hp_realize_host_wait.argtypes = [P]
        L.hp_group_info_get.argtypes = [P, _IP, _IP, ctypes.c_int, ctypes.POINTER(GroupInfo)]
        L.hp_group_count.argtypes = [P, _IP]
        L.hp_infer_bounds.argtypes = [P, _IP, _IP, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                      ctypes.c_int, _IP, ctypes.c_int]
        L.hp_check_device_error.argtypes = [P, _IP]
        L.hp_set_option.argtypes = [P, ctypes.c_int, ctypes.c_longlong]
        L.hp_pipeline_destroy.argtypes = [P]
        L.hp_histeq_u8_noalloc.argtypes = [ctypes.POINTER(Buffer), ctypes.POINTER(Buffer), P]
        L.hp_server_create.argtypes = [ctypes.POINTER(P), ctypes.c_longlong, ctypes.c_int, ctypes.c_int]
        L.hp_server_submit.argtypes = [P, P, ctypes.POINTER(Buffer), ctypes.c_int, ctypes.POINTER(Buffer),
                                       ctypes.POINTER(ctypes.c_ulonglong)]
        L.hp_server_submit_device.argtypes = [P, P, ctypes.POINTER(Buffer), ctypes.c_int, ctypes.POINTER(Buffer),
                                              ctypes.POINTER(ctypes.c_ulonglong)]
        L.hp_server_wait.argtypes = [P, ctypes.c_ulonglong, ctypes.c_int, ctypes.POINTER(ctypes.c_double)]
        L.hp_server_stats_get.argtypes = [P, ctypes.POINTER(ServerStats)]
        L.hp_server_destroy.argtypes = [P]
        L.hp_prepare.argtypes = [P, _IP, _IP, ctypes.c_int, P]
        L.hp_server_prepare.argtypes = [P, P, ctypes.POINTER(Buffer), ctypes.c_int]
        L.hp_measure_fp32_peak.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, P, ctypes.POINTER(ctypes.c_double),
                                           ctypes.POINTER(ctypes.c_double), _IP]
        L.hp_kernel_attrs_get.argtypes = [P, _IP, _IP, ctypes.POINTER(ctypes.c_longlong)]
        L.hp_last_error.restype = ctypes.c_char_p
        L.hp_launch_count.restype = ctypes.c_ulonglong
        for name in EXPORTS:
            if name not in ("hp_last_error", "hp_launch_count"):
                getattr(L, name).restype = ctypes.c_int
        _lib = L
    return _lib


class HPError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"hp status {status}: {msg}")
        self.status = status


def check(status: int):
    if status != HP_OK:
        raise HPError(status, lib().hp_last_error().decode())


def _ints(v):
    return (ctypes.c_int * len(v))(*v) if v is not None else None


def _floats(v):
    return (ctypes.c_float * len(v))(*v) if v is not None and len(v) else None


def launch_count() -> int:
    return int(lib().hp_launch_count())


def buffer_from_tensor(t, dtype: int) -> Buffer:
    """hp_buffer of a torch tensor shaped [C][H][W] (or [H][W]) with unit x stride."""
    if t.dim() == 2:
        c, h, w = 1, t.shape[0], t.shape[1]
        rs, ps = t.stride(0), t.stride(0) * h
    else:
        c, h, w = t.shape
        rs, ps = t.stride(1), t.stride(0)
    es = t.element_size()
    assert t.stride(-1) == 1, "x must be the unit-stride dimension"
    b = Buffer(t.data_ptr(), dtype, c, w, h, rs * es, ps * es)
    b._tensor = t  # the descriptor keeps its memory alive (it holds only the address)
    return b


def padded_empty(c: int, h: int, w: int, torch_dtype, device="cuda"):
    """A [C][H][W] torch tensor whose row and plane strides are multiples of 16
    bytes, as the C ABI requires (a view of a row-padded allocation)."""
    import torch
    es = torch.empty((), dtype=torch_dtype).element_size()
    per = 16 // es
    wp = (w + per - 1) // per * per
    plane = wp * h
    plane = (plane + per - 1) // per * per
    base = torch.empty((c * plane,), dtype=torch_dtype, device=device)
    return base.as_strided((c, h, w), (plane, wp, 1))


def padded_copy(src, device="cuda"):
    """Copy of a [C][H][W] tensor into a padded_empty tensor on `device`."""
    c, h, w = src.shape
    dst = padded_empty(c, h, w, src.dtype, device)
    dst.copy_(src)
    return dst


def histeq_u8_noalloc(inp: Buffer, out: Buffer, stream=None):
    """Allocation-free histogram equalization (hp_histeq_u8_noalloc)."""
    check(lib().hp_histeq_u8_noalloc(ctypes.byref(inp), ctypes.byref(out), ctypes.c_void_p(stream or 0)))


def measure_fp32_peak(paired: bool, iters: int = 2048, launches: int = 100, stream=None):
    """FP32 throughput of the current GPU (hp_measure_fp32_peak): returns
    (flop/s, ms per launch, SM count)."""
    f, ms, sms = ctypes.c_double(), ctypes.c_double(), ctypes.c_int()
    check(lib().hp_measure_fp32_peak(int(paired), iters, launches, ctypes.c_void_p(stream or 0), ctypes.byref(f),
                                     ctypes.byref(ms), ctypes.byref(sms)))
    return f.value, ms.value, sms.value


class Pipeline:
    """A pipeline handle: the algorithm (stages) and its schedule."""

    def __init__(self, in_dtypes, in_channels):
        self.h = ctypes.c_void_p()
        check(lib().hp_pipeline_create(ctypes.byref(self.h), len(in_dtypes), _ints(in_dtypes), _ints(in_channels)))
        self.in_dtypes = list(in_dtypes)
        self.in_channels = list(in_channels)
        self.stages = []   # python-side record of each stage desc (for builders and tests)
        self.output = None

    def __del__(self):
        h = getattr(self, "h", None)
        if h is not None and h.value and _lib is not None:
            _lib.hp_pipeline_destroy(h)
            self.h = None

    @staticmethod
    def input(k: int) -> int:
        return -1 - k

    def add_stage(self, kind, inputs, channels, storage=HP_F32, op=0, rx=0, ry=0, wx=None, wy=None, params=None):
        ins = _ints(list(inputs))
        wxa, wya, pa = _floats(wx), _floats(wy), _floats(params)
        d = StageDesc(kind, op, len(inputs), ins, rx, ry, wxa, wya, pa, len(params) if params else 0, storage,
                      channels, 0)
        sid = ctypes.c_int()
        check(lib().hp_add_stage(self.h, ctypes.byref(d), ctypes.byref(sid)))
        self.stages.append(dict(kind=kind, op=op, inputs=list(inputs), channels=channels, storage=storage,
                                rx=rx, ry=ry, wx=wx, wy=wy, params=params))
        return sid.value

    def set_output(self, sid: int):
        check(lib().hp_set_output(self.h, sid))
        self.output = sid

    def schedule(self, group_of_stage, tile_w=None, tile_h=None, threads=None, serial_y=None, impl=None):
        ng = max(g for g in group_of_stage) + 1
        keep = [_ints(group_of_stage), _ints(tile_w), _ints(tile_h), _ints(threads), _ints(serial_y), _ints(impl)]
        s = Schedule(len(group_of_stage), keep[0], ng, keep[1], keep[2], keep[3], keep[4], keep[5])
        check(lib().hp_schedule_set(self.h, ctypes.byref(s)))

    def realize(self, inputs, output, stream=None):
        """inputs: list of Buffer (device); output: Buffer (device); stream: cudaStream_t as int or None."""
        arr = (Buffer * len(inputs))(*inputs)
        check(lib().hp_realize(self.h, arr, len(inputs), ctypes.byref(output), ctypes.c_void_p(stream or 0)))

    def prepare(self, sizes, stream=None):
        """Lowers and allocates for inputs of the given (w, h) sizes without running."""
        check(lib().hp_prepare(self.h, _ints([s[0] for s in sizes]), _ints([s[1] for s in sizes]), len(sizes),
                               ctypes.c_void_p(stream or 0)))

    def realize_host(self, inputs, output, stream=None):
        arr = (Buffer * len(inputs))(*inputs)
        check(lib().hp_realize_host(self.h, arr, len(inputs), ctypes.byref(output), ctypes.c_void_p(stream or 0)))

    def realize_host_async(self, inputs, output, stream=None):
        """Enqueues copy in, realize and copy out of host buffers (hp_realize_host_async);
        the buffers must stay alive and unchanged until realize_host_wait()."""
        arr = (Buffer * len(inputs))(*inputs)
        check(lib().hp_realize_host_async(self.h, arr, len(inputs), ctypes.byref(output), ctypes.c_void_p(stream or 0)))

    def realize_host_wait(self):
        check(lib().hp_realize_host_wait(self.h))

    def set_option(self, option: int, value: int):
        check(lib().hp_set_option(self.h, option, value))

    def use_cuda_graph(self, on: bool = True):
        self.set_option(HP_OPT_CUDA_GRAPH, 1 if on else 0)

    def overlap_launches(self, on: bool = True):
        """Programmatic dependent launch between the realize's kernels (the default)."""
        self.set_option(HP_OPT_OVERLAP, 1 if on else 0)

    def probe_kernel_attrs(self, on: bool = True):
        """Record the launched kernels' registers and local-memory bytes (HP_OPT_PROBE_ATTRS)."""
        self.set_option(HP_OPT_PROBE_ATTRS, 1 if on else 0)

    def kernel_attrs(self):
        """(kernels, max registers, max local bytes per thread) of the last probed realize."""
        n, r, loc = ctypes.c_int(), ctypes.c_int(), ctypes.c_longlong()
        check(lib().hp_kernel_attrs_get(self.h, ctypes.byref(n), ctypes.byref(r), ctypes.byref(loc)))
        return n.value, r.value, loc.value

    def device_error(self) -> int:
        """Reads and clears the device error word (0 = none); synchronises."""
        c = ctypes.c_int()
        check(lib().hp_check_device_error(self.h, ctypes.byref(c)))
        return c.value

    def group_count(self) -> int:
        n = ctypes.c_int()
        check(lib().hp_group_count(self.h, ctypes.byref(n)))
        return n.value

    def group_info(self, sizes, g: int) -> GroupInfo:
        ws = _ints([s[0] for s in sizes])
        hs = _ints([s[1] for s in sizes])
        info = GroupInfo()
        check(lib().hp_group_info_get(self.h, ws, hs, g, ctypes.byref(info)))
        return info

    def infer_bounds(self, sizes, g: int, x0: int, y0: int, w: int, h: int):
        ws = _ints([s[0] for s in sizes])
        hs = _ints([s[1] for s in sizes])
        n = len(self.stages)
        out = (ctypes.c_int * (4 * n))()
        check(lib().hp_infer_bounds(self.h, ws, hs, g, x0, y0, w, h, out, n))
        return [tuple(out[4 * i:4 * i + 4]) for i in range(n)]


class Server:
    """Continuous-batching serving loop (hp_server_*): submit host-buffer (or
    device-buffer) requests for any pipeline; they run as slots and HBM budget
    allow."""

    def __init__(self, hbm_budget_bytes: int, slots: int = 4, max_batch: int = 8):
        self.h = ctypes.c_void_p()
        check(lib().hp_server_create(ctypes.byref(self.h), hbm_budget_bytes, slots, max_batch))
        self._keep = {}

    def submit(self, pipeline: "Pipeline", inputs, output) -> int:
        arr = (Buffer * len(inputs))(*inputs)
        t = ctypes.c_ulonglong()
        check(lib().hp_server_submit(self.h, pipeline.h, arr, len(inputs), ctypes.byref(output), ctypes.byref(t)))
        return t.value

    def submit_device(self, pipeline: "Pipeline", inputs, output) -> int:
        """A request whose buffers are in device memory (no host copies)."""
        arr = (Buffer * len(inputs))(*inputs)
        t = ctypes.c_ulonglong()
        check(lib().hp_server_submit_device(self.h, pipeline.h, arr, len(inputs), ctypes.byref(output),
                                            ctypes.byref(t)))
        return t.value

    def prepare(self, pipeline: "Pipeline", inputs):
        """Makes every slot's copy of the pipeline ready for inputs shaped like these."""
        arr = (Buffer * len(inputs))(*inputs)
        check(lib().hp_server_prepare(self.h, pipeline.h, arr, len(inputs)))

    def wait(self, ticket: int, timeout_ms: int = 60000):
        """(status, latency_us); status HP_ERR_TIMEOUT if not done in time."""
        lat = ctypes.c_double()
        st = lib().hp_server_wait(self.h, ticket, timeout_ms, ctypes.byref(lat))
        return st, lat.value

    def stats(self) -> ServerStats:
        s = ServerStats()
        check(lib().hp_server_stats_get(self.h, ctypes.byref(s)))
        return s

    def close(self):
        if self.h is not None and self.h.value:
            check(lib().hp_server_destroy(self.h))
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
