"""GB300 parallel in-place random permutation: Python binding of ``libpip_gb300.so``.

This module only marshals arguments into the C ABI declared in
``include/pip.h``; every step of the shuffle runs in the library's CUDA
kernels.  There is no CPU fallback: if the library has not been built, or no
GPU is present, the calls raise.

Typical use with PyTorch device memory::

    import torch, paper_2103_01216_gb300 as pip
    A = torch.arange(1 << 20, dtype=torch.int64, device="cuda")
    pip.shuffle(A, seed=1, eps=0.5)   # queued on the current stream
    pip.check()                       # synchronize and surface device-side errors
"""
from __future__ import annotations

import ctypes
import os
import threading

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libpip_gb300.so")

U32, U64, REC128 = 0, 1, 2
DTYPES = {"u32": U32, "u64": U64, "rec128": REC128}
ELEM_BYTES = {U32: 4, U64: 8, REC128: 16}

STATUS = {
    0: "PIP_OK",
    1: "PIP_EINVAL",
    2: "PIP_ENOMEM",
    3: "PIP_ECUDA",
    4: "PIP_ETIMEOUT",
    5: "PIP_EAGAIN",
    6: "PIP_EBUSY",
    7: "PIP_EINTERNAL",
    8: "PIP_ETOOLARGE",
}
PIP_OK, PIP_EINVAL, PIP_ENOMEM, PIP_ECUDA, PIP_ETIMEOUT, PIP_EAGAIN, PIP_EBUSY, PIP_EINTERNAL, PIP_ETOOLARGE = range(9)
FLAG_TEST_SKIP_BARRIER = 1
FLAG_PREFETCH = 2
AUX_C = 128.0


class PipError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = code
        super().__init__(f"{where}: {STATUS.get(code, code)}")


class PlanInfo(ctypes.Structure):
    _fields_ = [
        ("n", ctypes.c_uint64),
        ("elem_bytes", ctypes.c_uint32),
        ("eps", ctypes.c_double),
        ("fresh_per_round", ctypes.c_uint32),
        ("max_active", ctypes.c_uint32),
        ("slots", ctypes.c_uint32),
        ("grid_blocks", ctypes.c_uint32),
        ("block_threads", ctypes.c_uint32),
        ("aux_bytes", ctypes.c_uint64),
        ("aux_bound_bytes", ctypes.c_uint64),
        ("min_rounds", ctypes.c_uint64),
        ("driver", ctypes.c_uint32),
        ("flags", ctypes.c_uint32),
        ("smem_bytes", ctypes.c_uint64),
    ]


class BatchItem(ctypes.Structure):
    _fields_ = [
        ("A_dev", ctypes.c_void_p),
        ("H_dev", ctypes.c_void_p),
        ("n", ctypes.c_uint64),
        ("seed", ctypes.c_uint64),
    ]


class BatchPlan(ctypes.Structure):
    _fields_ = [
        ("count", ctypes.c_uint32),
        ("elem_bytes", ctypes.c_uint32),
        ("fmax", ctypes.c_uint32),
        ("slot_factor", ctypes.c_uint32),
        ("block_threads", ctypes.c_uint32),
        ("max_blocks", ctypes.c_uint32),
        ("any_explicit", ctypes.c_uint32),
        ("pad", ctypes.c_uint32),
        ("jobs_bytes", ctypes.c_uint64),
        ("smem_bytes", ctypes.c_uint64),
        ("total_elems", ctypes.c_uint64),
        ("eps", ctypes.c_double),
    ]


class JobStats(ctypes.Structure):
    _fields_ = [
        ("status", ctypes.c_uint32),
        ("rounds", ctypes.c_uint32),
        ("attempts", ctypes.c_uint64),
        ("losers", ctypes.c_uint64),
        ("max_active", ctypes.c_uint32),
        ("pad", ctypes.c_uint32),
    ]


class Options(ctypes.Structure):
    _fields_ = [
        ("prefix_c", ctypes.c_double),
        ("fresh_per_round", ctypes.c_uint32),
        ("slot_factor", ctypes.c_uint32),
        ("grid_blocks", ctypes.c_uint32),
        ("block_threads", ctypes.c_uint32),
        ("wait_timeout_ns", ctypes.c_uint64),
        ("flags", ctypes.c_uint32),
    ]


class Stats(ctypes.Structure):
    _fields_ = [
        ("status", ctypes.c_uint32),
        ("rounds", ctypes.c_uint32),
        ("attempts", ctypes.c_uint64),
        ("losers", ctypes.c_uint64),
        ("max_active", ctypes.c_uint32),
        ("grid_blocks", ctypes.c_uint32),
        ("reserved", ctypes.c_uint64 * 4),
    ]


class ServeOptions(ctypes.Structure):
    _fields_ = [
        ("max_resident", ctypes.c_uint32),
        ("rounds_per_tick", ctypes.c_uint32),
        ("fresh_cap", ctypes.c_uint32),
        ("slot_factor", ctypes.c_uint32),
        ("block_threads", ctypes.c_uint32),
        ("tick_us", ctypes.c_uint32),
        ("prefix_c", ctypes.c_double),
        ("lanes", ctypes.c_uint32),
        ("lane_min_log2", ctypes.c_uint32),
        ("lane_blocks", ctypes.c_uint32),
        ("pad", ctypes.c_uint32),
    ]


class ReqStats(ctypes.Structure):
    _fields_ = [
        ("status", ctypes.c_uint32),
        ("rounds", ctypes.c_uint32),
        ("attempts", ctypes.c_uint64),
        ("losers", ctypes.c_uint64),
        ("n", ctypes.c_uint64),
        ("charged_bytes", ctypes.c_uint64),
        ("submit_ns", ctypes.c_int64),
        ("admit_ns", ctypes.c_int64),
        ("done_ns", ctypes.c_int64),
        ("ticks", ctypes.c_uint32),
        ("fresh_per_round", ctypes.c_uint32),
        ("lane_launches", ctypes.c_uint32),
        ("pad", ctypes.c_uint32),
    ]


class ServeInfo(ctypes.Structure):
    _fields_ = [
        ("budget_bytes", ctypes.c_uint64),
        ("used_bytes", ctypes.c_uint64),
        ("peak_used_bytes", ctypes.c_uint64),
        ("submitted", ctypes.c_uint64),
        ("admitted", ctypes.c_uint64),
        ("completed", ctypes.c_uint64),
        ("ticks", ctypes.c_uint64),
        ("resident", ctypes.c_uint32),
        ("waiting", ctypes.c_uint32),
        ("tick_blocks", ctypes.c_uint32),
        ("fresh_cap", ctypes.c_uint32),
        ("status", ctypes.c_uint32),
        ("lane_requests", ctypes.c_uint32),
        ("tick_kernels", ctypes.c_uint64),
        ("tick_wait_ns", ctypes.c_uint64),
        ("lane_launches", ctypes.c_uint64),
        ("lane_setup_ns", ctypes.c_uint64),
    ]


STATS_BYTES = ctypes.sizeof(Stats)
JOB_STATS_BYTES = ctypes.sizeof(JobStats)
DRIVER_GRID, DRIVER_CTA, DRIVER_CLUSTER = 0, 1, 2
SERVE_NO_LANES = 0xFFFFFFFF
FLAG_SWAP_LOADSTORE = 4
FLAG_SWAP_EXCHANGE = 8
FLAG_STORE_EVICT_NORMAL = 16
FLAG_FORCE_GRID = 32
FLAG_FORCE_CTA = 64
FLAG_FORCE_CLUSTER = 128
FLAG_SPECULATE = 256
FLAG_TWO_RES = 512
FLAG_VALIDATE_INPUT = 1024
FLAG_EARLY_RESERVE = 4096
FLAG_TEST_GATED = 8192

_lock = threading.Lock()
_lib = None


def lib() -> ctypes.CDLL:
    """Load ``libpip_gb300.so`` (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(
                f"{LIB_PATH} is missing: build it with `python -m paper_2103_01216_gb300._build` "
                "(or __graft_entry__.build()); there is no CPU fallback"
            )
        L = ctypes.CDLL(LIB_PATH)
        vp, u64, u32, i32, dbl = ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_int, ctypes.c_double
        L.pip_shuffle.argtypes = [vp, u64, i32, u64, dbl, vp]
        L.pip_shuffle.restype = i32
        L.pip_shuffle_explicit_h.argtypes = [vp, u64, i32, vp, dbl, vp]
        L.pip_shuffle_explicit_h.restype = i32
        L.pip_shuffle_ex.argtypes = [vp, u64, i32, u64, vp, dbl, ctypes.POINTER(Options), vp, u64, vp, vp]
        L.pip_shuffle_ex.restype = i32
        L.pip_plan.argtypes = [u64, i32, dbl, ctypes.POINTER(Options), ctypes.POINTER(PlanInfo)]
        L.pip_plan.restype = i32
        L.pip_aux_bytes.argtypes = [u64, i32, dbl]
        L.pip_aux_bytes.restype = u64
        L.pip_check.argtypes = [vp]
        L.pip_check.restype = i32
        L.pip_status_string.argtypes = [i32]
        L.pip_status_string.restype = ctypes.c_char_p
        L.pip_version.argtypes = []
        L.pip_version.restype = ctypes.c_char_p
        L.pip_shuffle_batch.argtypes = [ctypes.POINTER(vp), ctypes.POINTER(u64), ctypes.POINTER(u64), u32, i32, dbl,
                                        vp]
        L.pip_shuffle_batch.restype = i32
        L.pip_batch_plan_make.argtypes = [ctypes.POINTER(BatchItem), u32, i32, dbl, ctypes.POINTER(Options),
                                          ctypes.POINTER(BatchPlan)]
        L.pip_batch_plan_make.restype = i32
        L.pip_batch_prepare.argtypes = [ctypes.POINTER(BatchItem), ctypes.POINTER(BatchPlan),
                                        ctypes.POINTER(Options), vp]
        L.pip_batch_prepare.restype = i32
        L.pip_batch_run.argtypes = [ctypes.POINTER(BatchPlan), vp, vp, vp]
        L.pip_batch_run.restype = i32
        L.pip_shuffle_noalloc.argtypes = [vp, u64, i32, u64, dbl, vp]
        L.pip_shuffle_noalloc.restype = i32
        L.pip_shuffle_host_stream.argtypes = [ctypes.POINTER(vp), ctypes.POINTER(vp), ctypes.POINTER(u64),
                                              ctypes.c_uint32, u64, i32, dbl, vp, u64, vp]
        L.pip_shuffle_host_stream.restype = i32
        L.pip_calibrate_swap_floor.argtypes = [vp, u64, i32, u64, i32, vp]
        L.pip_calibrate_swap_floor.restype = i32
        L.pip_serve_create.argtypes = [ctypes.POINTER(vp), u64, i32, ctypes.POINTER(ServeOptions)]
        L.pip_serve_create.restype = i32
        L.pip_serve_submit.argtypes = [vp, vp, u64, i32, u64, dbl, ctypes.POINTER(u64)]
        L.pip_serve_submit.restype = i32
        L.pip_serve_poll.argtypes = [vp, u64, ctypes.POINTER(vp), ctypes.POINTER(ReqStats)]
        L.pip_serve_poll.restype = i32
        L.pip_serve_wait.argtypes = [vp, u64, u32, ctypes.POINTER(vp), ctypes.POINTER(ReqStats)]
        L.pip_serve_wait.restype = i32
        L.pip_serve_next_done.argtypes = [vp, u32, ctypes.POINTER(u64)]
        L.pip_serve_next_done.restype = i32
        L.pip_serve_release.argtypes = [vp, u64]
        L.pip_serve_release.restype = i32
        L.pip_serve_info_get.argtypes = [vp, ctypes.POINTER(ServeInfo)]
        L.pip_serve_info_get.restype = i32
        L.pip_serve_destroy.argtypes = [vp]
        L.pip_serve_destroy.restype = i32
        L.pip_list_contract.argtypes = [vp, u64, dbl, vp]
        L.pip_list_contract.restype = i32
        L.pip_list_contract_ex.argtypes = [vp, u64, dbl, ctypes.POINTER(Options), vp, u64, vp, vp]
        L.pip_list_contract_ex.restype = i32
        L.pip_list_rank_ex.argtypes = [vp, u64, dbl, ctypes.POINTER(Options), vp, u64, vp, vp]
        L.pip_list_rank_ex.restype = i32
        L.pip_list_rank.argtypes = [vp, u64, dbl, vp]
        L.pip_list_rank.restype = i32
        L.pip_list_plan.argtypes = [u64, dbl, ctypes.POINTER(Options), ctypes.POINTER(PlanInfo)]
        L.pip_list_plan.restype = i32
        L.pip_tree_contract.argtypes = [vp, u64, dbl, vp]
        L.pip_tree_contract.restype = i32
        L.pip_tree_contract_ex.argtypes = [vp, u64, dbl, ctypes.POINTER(Options), vp, u64, vp, vp]
        L.pip_tree_contract_ex.restype = i32
        L.pip_tree_plan.argtypes = [u64, dbl, ctypes.POINTER(Options), ctypes.POINTER(PlanInfo)]
        L.pip_tree_plan.restype = i32
        L.pip_scan.argtypes = [vp, u64, i32, vp, vp]
        L.pip_scan.restype = i32
        L.pip_scan_ex.argtypes = [vp, u64, i32, vp, vp, u64, vp]
        L.pip_scan_ex.restype = i32
        L.pip_scan_aux_bytes.argtypes = []
        L.pip_scan_aux_bytes.restype = u64
        _lib = L
        return L


def _raise(code: int, where: str):
    if code != PIP_OK:
        raise PipError(code, where)


def make_options(**kw) -> Options | None:
    if not kw:
        return None
    o = Options()
    for k, v in kw.items():
        if not hasattr(o, k):
            raise TypeError(f"unknown option {k}")
        setattr(o, k, v)
    return o


def _opt_ptr(o: Options | None):
    return ctypes.byref(o) if o is not None else None


def plan(n: int, dtype: int | str, eps: float, **options) -> dict:
    """The plan the library would use (host only)."""
    d = DTYPES[dtype] if isinstance(dtype, str) else dtype
    info = PlanInfo()
    o = make_options(**options)
    _raise(lib().pip_plan(n, d, eps, _opt_ptr(o), ctypes.byref(info)), "pip_plan")
    return {f: getattr(info, f) for f, _ in PlanInfo._fields_}


def aux_bytes(n: int, dtype: int | str, eps: float) -> int:
    d = DTYPES[dtype] if isinstance(dtype, str) else dtype
    return int(lib().pip_aux_bytes(n, d, eps))


def _stream_handle(stream):
    if stream is None:
        import torch

        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def tensor_dtype(A) -> int:
    """pip dtype code of a torch tensor: 1-D 4-byte -> u32, 1-D 8-byte -> u64,
    2-D with 16-byte rows -> rec128."""
    if A.dim() == 1 and A.element_size() in (4, 8):
        return U32 if A.element_size() == 4 else U64
    if A.dim() == 2 and A.element_size() * A.shape[1] == 16:
        return REC128
    raise ValueError("expected a 1-D tensor of 4- or 8-byte elements, or 2-D with 16-byte rows")


def shuffle_ptr(ptr: int, n: int, dtype: int, seed: int, eps: float, *, H_ptr: int | None = None,
                options: Options | None = None, aux_ptr: int | None = None, aux_bytes_: int = 0,
                stats_ptr: int | None = None, stream: int = 0) -> None:
    """Raw-pointer form of :func:`shuffle` (device pointers as integers)."""
    rc = lib().pip_shuffle_ex(ptr, n, dtype, seed, H_ptr, eps, _opt_ptr(options), aux_ptr, aux_bytes_,
                              stats_ptr, stream)
    _raise(rc, "pip_shuffle_ex")


def shuffle(A, seed: int = 0, eps: float = 0.5, *, H=None, stream=None, aux=None, stats=None, tuned: bool = False,
            **options) -> None:
    """Knuth-shuffle the CUDA tensor ``A`` in place (asynchronous on ``stream``).

    ``H``: optional CUDA uint32/int32 tensor of explicit targets (0 <= H[i] <= i).
    ``aux``: optional CUDA uint8 tensor used as scratch instead of allocating.
    ``stats``: optional CUDA uint8 tensor of at least ``STATS_BYTES`` that the
    kernel fills with a ``Stats`` record.  Other keywords are ``Options`` fields.
    """
    if not A.is_cuda or not A.is_contiguous():
        raise ValueError("A must be a contiguous CUDA tensor")
    d = tensor_dtype(A)
    n = A.shape[0]
    if tuned:  # options cached by the autotuner for this size class (explicit options win)
        from . import autotune

        options = {**autotune.options_for(n, {U32: "u32", U64: "u64", REC128: "rec128"}[d], eps), **options}
    h_ptr = None
    if H is not None:
        if not H.is_cuda or H.element_size() != 4 or H.dim() != 1 or H.shape[0] != n or not H.is_contiguous():
            raise ValueError("H must be a contiguous 1-D CUDA tensor of n 4-byte targets")
        h_ptr = H.data_ptr()
    aux_ptr, aux_n = (aux.data_ptr(), aux.numel() * aux.element_size()) if aux is not None else (None, 0)
    st_ptr = None
    if stats is not None:
        if stats.numel() * stats.element_size() < STATS_BYTES:
            raise ValueError("stats buffer too small")
        st_ptr = stats.data_ptr()
    shuffle_ptr(A.data_ptr(), n, d, seed, eps, H_ptr=h_ptr, options=make_options(**options), aux_ptr=aux_ptr,
                aux_bytes_=aux_n, stats_ptr=st_ptr, stream=_stream_handle(stream))


def shuffle_host_stream(ins, outs, seeds, eps: float = 0.5, *, dev_buf=None, stream=None) -> None:
    """Shuffle a sequence of host (CPU) tensors: ins[j] is copied to the
    device, shuffled with seeds[j] and copied back to outs[j] (which may be
    ins[j]); copies overlap the neighbouring shuffles (asynchronous on
    ``stream``; pinned tensors overlap, pageable ones serialise).  All tensors
    have the same shape and dtype (1-D 4- or 8-byte, or 2-D 16-byte rows).
    ``dev_buf``: optional CUDA uint8 tensor of at least
    min(len, 3) * round_up(bytes, 256) bytes (a fourth buffer is used when it
    has room for one)."""
    ins, outs, seeds = list(ins), list(outs), [int(x) for x in seeds]
    if not (len(ins) == len(outs) == len(seeds)):
        raise ValueError("ins, outs and seeds must have the same length")
    if not ins:
        return
    d = tensor_dtype(ins[0])
    for t in ins + outs:
        if t.is_cuda or not t.is_contiguous() or t.shape != ins[0].shape or t.dtype != ins[0].dtype:
            raise ValueError("every array must be a contiguous host tensor of one shape and dtype")
    k = len(ins)
    in_p = (ctypes.c_void_p * k)(*[t.data_ptr() for t in ins])
    out_p = (ctypes.c_void_p * k)(*[t.data_ptr() for t in outs])
    sd = (ctypes.c_uint64 * k)(*seeds)
    buf_ptr, buf_n = (dev_buf.data_ptr(), dev_buf.numel() * dev_buf.element_size()) if dev_buf is not None else (None, 0)
    rc = lib().pip_shuffle_host_stream(in_p, out_p, sd, k, ins[0].shape[0], d, eps, buf_ptr, buf_n,
                                       _stream_handle(stream))
    _raise(rc, "pip_shuffle_host_stream")


def check(stream=None) -> None:
    """Synchronize ``stream`` and raise if device-side work reported an error."""
    _raise(lib().pip_check(_stream_handle(stream)), "pip_check")


def read_stats(buf) -> Stats:
    """Decode a stats buffer filled by :func:`shuffle` (synchronizes via .cpu())."""
    raw = bytes(buf.cpu().numpy().tobytes()[:STATS_BYTES])
    return Stats.from_buffer_copy(raw)


def version() -> str:
    return lib().pip_version().decode()


# ---------------------------------------------------------------- batches
def _items(arrays, seeds, H=None):
    n = len(arrays)
    items = (BatchItem * n)()
    d = None
    for j, A in enumerate(arrays):
        if not A.is_cuda or not A.is_contiguous():
            raise ValueError("every array must be a contiguous CUDA tensor")
        dj = tensor_dtype(A)
        if d is None:
            d = dj
        elif d != dj:
            raise ValueError("all arrays of a batch share one element type")
        items[j].A_dev = A.data_ptr()
        items[j].n = A.shape[0]
        items[j].seed = int(seeds[j])
        if H is not None and H[j] is not None:
            if H[j].element_size() != 4 or H[j].shape[0] != A.shape[0]:
                raise ValueError("explicit targets must be n 4-byte entries")
            items[j].H_dev = H[j].data_ptr()
    return items, (d if d is not None else U64)


class Batch:
    """A prepared batch: plan + device job list, re-runnable and graph-capturable.

    ``run()`` queues one shuffle of every array (a memset and one kernel).
    """

    def __init__(self, arrays, seeds, eps: float = 0.5, H=None, **options):
        import torch

        self.arrays = list(arrays)
        self.items, self.dtype = _items(self.arrays, seeds, H)
        self.options = make_options(**options)
        self.plan = BatchPlan()
        _raise(lib().pip_batch_plan_make(self.items, len(self.arrays), self.dtype, eps, _opt_ptr(self.options),
                                         ctypes.byref(self.plan)), "pip_batch_plan_make")
        self.jobs = torch.empty(max(256, self.plan.jobs_bytes), dtype=torch.uint8, device="cuda")
        _raise(lib().pip_batch_prepare(self.items, ctypes.byref(self.plan), _opt_ptr(self.options),
                                       self.jobs.data_ptr()), "pip_batch_prepare")

    def run(self, stream=None, stats=None) -> None:
        st = None
        if stats is not None:
            if stats.numel() * stats.element_size() < JOB_STATS_BYTES * len(self.arrays):
                raise ValueError("stats buffer too small")
            st = stats.data_ptr()
        _raise(lib().pip_batch_run(ctypes.byref(self.plan), self.jobs.data_ptr(), st, _stream_handle(stream)),
               "pip_batch_run")

    def plan_dict(self) -> dict:
        return {f: getattr(self.plan, f) for f, _ in BatchPlan._fields_}


def shuffle_batch(arrays, seeds, eps: float = 0.5, stream=None) -> None:
    """Shuffle every CUDA tensor of ``arrays`` in place in one launch
    (``pip_shuffle_batch``); ``seeds[j]`` is array j's target seed."""
    n = len(arrays)
    if n == 0:
        return
    items, d = _items(arrays, seeds)
    ptrs = (ctypes.c_void_p * n)(*[items[j].A_dev for j in range(n)])
    ns = (ctypes.c_uint64 * n)(*[items[j].n for j in range(n)])
    sd = (ctypes.c_uint64 * n)(*[items[j].seed for j in range(n)])
    _raise(lib().pip_shuffle_batch(ptrs, ns, sd, n, d, eps, _stream_handle(stream)), "pip_shuffle_batch")


def read_job_stats(buf, count: int):
    raw = bytes(buf.cpu().numpy().tobytes()[: JOB_STATS_BYTES * count])
    return [JobStats.from_buffer_copy(raw, j * JOB_STATS_BYTES) for j in range(count)]


# ---------------------------------------------------------------- serving
_TORCH_DTYPE = {U32: "int32", U64: "int64", REC128: "int64"}


class _DeviceArray:
    """Zero-copy view of raw device memory for torch.as_tensor."""

    def __init__(self, ptr: int, n: int, dtype: int):
        shape = (n, 2) if dtype == REC128 else (n,)
        typestr = "<i4" if dtype == U32 else "<i8"
        self.__cuda_array_interface__ = {"shape": shape, "typestr": typestr, "data": (ptr, False), "version": 3,
                                         "strides": None}


def device_view(ptr: int, n: int, dtype: int | str):
    """A torch tensor aliasing n elements of device memory at ``ptr``."""
    import torch

    d = DTYPES[dtype] if isinstance(dtype, str) else dtype
    if n == 0 or not ptr:
        return torch.empty((0, 2) if d == REC128 else (0,), dtype=getattr(torch, _TORCH_DTYPE[d]), device="cuda")
    return torch.as_tensor(_DeviceArray(ptr, n, d), device="cuda")


class Server:
    """A request server (``pip_serve_*``): memory-budgeted admission and
    continuous batching of shuffle requests on one GPU."""

    def __init__(self, budget_bytes: int, device: int = 0, **options):
        o = ServeOptions()
        for k, v in options.items():
            if not hasattr(o, k):
                raise TypeError(f"unknown server option {k}")
            setattr(o, k, v)
        self._h = ctypes.c_void_p()
        _raise(lib().pip_serve_create(ctypes.byref(self._h), budget_bytes, device, ctypes.byref(o)),
               "pip_serve_create")

    def submit(self, n: int, dtype: int | str = "u64", seed: int = 0, eps: float = 0.5, A=None) -> int:
        d = DTYPES[dtype] if isinstance(dtype, str) else dtype
        t = ctypes.c_uint64()
        ptr = None
        if A is not None:
            if tensor_dtype(A) != d or A.shape[0] != n:
                raise ValueError("A does not match n / dtype")
            ptr = A.data_ptr()
        _raise(lib().pip_serve_submit(self._h, ptr, n, d, seed, eps, ctypes.byref(t)), "pip_serve_submit")
        return t.value

    def poll(self, ticket: int):
        """None while running; else (device pointer, ReqStats)."""
        p, st = ctypes.c_void_p(), ReqStats()
        rc = lib().pip_serve_poll(self._h, ticket, ctypes.byref(p), ctypes.byref(st))
        if rc == PIP_EAGAIN:
            return None
        _raise(rc, "pip_serve_poll")
        return p.value or 0, st

    def wait(self, ticket: int, timeout_ms: int = 600000):
        p, st = ctypes.c_void_p(), ReqStats()
        rc = lib().pip_serve_wait(self._h, ticket, timeout_ms, ctypes.byref(p), ctypes.byref(st))
        _raise(rc, "pip_serve_wait")
        return p.value or 0, st

    def next_done(self, timeout_ms: int = 600000):
        """Ticket of the next finished request (completion order), or None on timeout."""
        t = ctypes.c_uint64()
        rc = lib().pip_serve_next_done(self._h, timeout_ms, ctypes.byref(t))
        if rc == PIP_EAGAIN:
            return None
        _raise(rc, "pip_serve_next_done")
        return t.value

    def release(self, ticket: int) -> None:
        _raise(lib().pip_serve_release(self._h, ticket), "pip_serve_release")

    def info(self) -> ServeInfo:
        out = ServeInfo()
        _raise(lib().pip_serve_info_get(self._h, ctypes.byref(out)), "pip_serve_info_get")
        return out

    def close(self) -> None:
        if self._h:
            rc = lib().pip_serve_destroy(self._h)
            self._h = ctypes.c_void_p()
            _raise(rc, "pip_serve_destroy")

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
        return False


FLOOR_EXCHANGE, FLOOR_LOADSTORE = 0, 1


def calibrate_swap_floor(A, seed: int = 0, stream=None, mode: int = FLOOR_EXCHANGE) -> None:
    """Benchmark-only probe that destroys ``A`` (``pip_calibrate_swap_floor``):
    the bare swap traffic of a shuffle of ``A`` with no conflict resolution
    (A's content afterwards is unspecified).  ``mode``: FLOOR_EXCHANGE (the
    random side as one atomic exchange at L2) or FLOOR_LOADSTORE."""
    if not A.is_cuda or not A.is_contiguous():
        raise ValueError("A must be a contiguous CUDA tensor")
    _raise(lib().pip_calibrate_swap_floor(A.data_ptr(), A.shape[0], tensor_dtype(A), seed, int(mode),
                                          _stream_handle(stream)), "pip_calibrate_swap_floor")


# ------------------------------------------------------------------ list contraction
LIST_NIL = 0xFFFFFFFFFFFFFFFF
DRIVER_LIST = 3


def list_plan(n: int, eps: float, **options) -> dict:
    """The plan pip_list_contract_ex would use (host only)."""
    info = PlanInfo()
    o = make_options(**options)
    _raise(lib().pip_list_plan(n, eps, _opt_ptr(o), ctypes.byref(info)), "pip_list_plan")
    return {f: getattr(info, f) for f, _ in PlanInfo._fields_}


def list_contract(nodes, eps: float = 0.5, *, stream=None, aux=None, stats=None, **options) -> None:
    """Contract every node of the doubly-linked lists in ``nodes`` in place
    (asynchronous on ``stream``).

    ``nodes``: contiguous CUDA tensor of shape (n, 2) with 8-byte elements
    (int64 or uint64 bit patterns) holding (prev, next) node indices, -1 /
    2^64-1 at list ends.  On return row i holds the nearest nodes with a
    larger index before and after i in its original list.  ``aux``, ``stats``
    and the keyword options are as in :func:`shuffle`.
    """
    if not nodes.is_cuda or not nodes.is_contiguous() or nodes.dim() != 2 or nodes.shape[1] != 2 \
            or nodes.element_size() != 8:
        raise ValueError("nodes must be a contiguous (n, 2) CUDA tensor of 8-byte elements")
    aux_ptr, aux_n = (aux.data_ptr(), aux.numel() * aux.element_size()) if aux is not None else (None, 0)
    st_ptr = None
    if stats is not None:
        if stats.numel() * stats.element_size() < STATS_BYTES:
            raise ValueError("stats buffer too small")
        st_ptr = stats.data_ptr()
    rc = lib().pip_list_contract_ex(nodes.data_ptr(), nodes.shape[0], eps, _opt_ptr(make_options(**options)),
                                    aux_ptr, aux_n, st_ptr, _stream_handle(stream))
    _raise(rc, "pip_list_contract_ex")


def list_rank(nodes, eps: float = 0.5, *, stream=None, aux=None, stats=None, **options) -> None:
    """List ranking of the doubly-linked lists in ``nodes`` (``pip_list_rank_ex``;
    asynchronous on ``stream``): ``nodes`` as for :func:`list_contract`, fewer
    than 2^31 rows; on return row i holds (nodes before i, nodes after i) in
    its list.  ``aux``, ``stats`` and the keyword options as in :func:`shuffle`."""
    if not nodes.is_cuda or not nodes.is_contiguous() or nodes.dim() != 2 or nodes.shape[1] != 2 \
            or nodes.element_size() != 8:
        raise ValueError("nodes must be a contiguous (n, 2) CUDA tensor of 8-byte elements")
    aux_ptr, aux_n = (aux.data_ptr(), aux.numel() * aux.element_size()) if aux is not None else (None, 0)
    st_ptr = None
    if stats is not None:
        if stats.numel() * stats.element_size() < STATS_BYTES:
            raise ValueError("stats buffer too small")
        st_ptr = stats.data_ptr()
    rc = lib().pip_list_rank_ex(nodes.data_ptr(), nodes.shape[0], eps, _opt_ptr(make_options(**options)),
                                aux_ptr, aux_n, st_ptr, _stream_handle(stream))
    _raise(rc, "pip_list_rank_ex")


# ------------------------------------------------------------------ tree contraction
TREE_NIL = 0xFFFFFFFFFFFFFFFF
DRIVER_TREE = 4


def tree_plan(n: int, eps: float, **options) -> dict:
    """The plan pip_tree_contract_ex would use (host only); its
    fresh_per_round and max_active are the F and kmax of the round schedule."""
    info = PlanInfo()
    o = make_options(**options)
    _raise(lib().pip_tree_plan(n, eps, _opt_ptr(o), ctypes.byref(info)), "pip_tree_plan")
    return {f: getattr(info, f) for f, _ in PlanInfo._fields_}


def tree_contract(nodes, eps: float = 0.5, *, stream=None, aux=None, stats=None, **options) -> None:
    """Contract the forest in ``nodes`` in place (asynchronous on ``stream``).

    ``nodes``: contiguous CUDA tensor of shape (n, 4) with 8-byte elements
    (int64 or uint64 bit patterns) holding (parent, left, right, round), -1 /
    2^64-1 for a missing pointer, 32-byte aligned.  On return every raked leaf
    holds (parent, sibling, grandparent, round) from its rake, one leaf per
    tree is left as a root and removed internal nodes keep their last record.
    ``aux``, ``stats`` and the keyword options are as in :func:`shuffle`.
    """
    if not nodes.is_cuda or not nodes.is_contiguous() or nodes.dim() != 2 or nodes.shape[1] != 4 \
            or nodes.element_size() != 8:
        raise ValueError("nodes must be a contiguous (n, 4) CUDA tensor of 8-byte elements")
    aux_ptr, aux_n = (aux.data_ptr(), aux.numel() * aux.element_size()) if aux is not None else (None, 0)
    st_ptr = None
    if stats is not None:
        if stats.numel() * stats.element_size() < STATS_BYTES:
            raise ValueError("stats buffer too small")
        st_ptr = stats.data_ptr()
    rc = lib().pip_tree_contract_ex(nodes.data_ptr(), nodes.shape[0], eps, _opt_ptr(make_options(**options)),
                                    aux_ptr, aux_n, st_ptr, _stream_handle(stream))
    _raise(rc, "pip_tree_contract_ex")


# ------------------------------------------------------------------ scan
def scan(A, total=None, *, stream=None, aux=None) -> None:
    """In-place exclusive prefix sum of the 1-D CUDA tensor ``A`` (4- or 8-byte
    elements, added as unsigned integers modulo 2^w); ``total``: optional CUDA
    tensor of at least one element of A's size that receives the sum."""
    if not A.is_cuda or not A.is_contiguous() or A.dim() != 1 or A.element_size() not in (4, 8):
        raise ValueError("A must be a contiguous 1-D CUDA tensor of 4- or 8-byte elements")
    d = U32 if A.element_size() == 4 else U64
    t_ptr = None
    if total is not None:
        if not total.is_cuda or total.element_size() != A.element_size() or total.numel() < 1:
            raise ValueError("total must be a CUDA tensor of A's element size")
        t_ptr = total.data_ptr()
    aux_ptr, aux_n = (aux.data_ptr(), aux.numel() * aux.element_size()) if aux is not None else (None, 0)
    _raise(lib().pip_scan_ex(A.data_ptr(), A.shape[0], d, t_ptr, aux_ptr, aux_n, _stream_handle(stream)),
           "pip_scan_ex")


def scan_aux_bytes() -> int:
    return int(lib().pip_scan_aux_bytes())
