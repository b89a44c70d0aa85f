"""ctypes binding of libscl (include/scl.h): same names, argument marshalling only.

Every computation runs in the CUDA library; this module converts Python
arguments (ints, numpy arrays, torch tensors' pointers) into the C types and
turns non-zero status codes into :class:`SclError`.  There is no fallback: if
``_lib/libscl.so`` is missing the import fails loudly.

PyTorch is used only by the caller, for device memory (the arena) and streams
(``torch.cuda.current_stream().cuda_stream``).
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_lib", "libscl.so")

# status codes
SCL_OK = 0
SCL_E_INVALID = 1
SCL_E_NOMEM = 2
SCL_E_BUDGET = 3
SCL_E_KEY_RANGE = 4
SCL_E_TIMEOUT = 5
SCL_E_PENDING = 6
SCL_E_CUDA = 7
SCL_E_STATE = 8
SCL_E_UNSUPPORTED = 9

# scl_dtype
SCL_U32, SCL_I32, SCL_F32, SCL_KV_I32_F32 = 0, 1, 2, 3
# scl_map_kernel
SCL_K_IDENT, SCL_K_MIX32, SCL_K_POLY3 = 0, 1, 2
# scl_reduce
SCL_R_NONE, SCL_R_SUM, SCL_R_SUM_MIN_MAX, SCL_R_KEYED_COUNT_SUM = 0, 1, 2, 3
SCL_NOALLOC_MAX_ELEMENTS = 67_108_864
SCL_MAX_REDUCE_ARRAYS = 1024
SCL_MAX_LARGE_KEYS = 1 << 24


class scl_config(ctypes.Structure):
    _fields_ = [("device", ctypes.c_int32), ("reserved0", ctypes.c_int32),
                ("arena", ctypes.c_void_p), ("arena_bytes", ctypes.c_uint64),
                ("hbm_budget_bytes", ctypes.c_uint64), ("inflight_batches", ctypes.c_int32),
                ("reserved1", ctypes.c_int32), ("tune_cache_path", ctypes.c_char_p)]


class scl_result(ctypes.Structure):
    _fields_ = [("u64_sum", ctypes.c_uint64), ("f64_sum", ctypes.c_double),
                ("f32_sum", ctypes.c_float), ("f32_min", ctypes.c_float),
                ("f32_max", ctypes.c_float), ("status", ctypes.c_int32),
                ("n", ctypes.c_uint64), ("kind", ctypes.c_uint32),
                ("reserved", ctypes.c_uint32)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_ if not k.startswith("reserved")}


class scl_shape(ctypes.Structure):
    _fields_ = [("block", ctypes.c_int32), ("items_per_thread", ctypes.c_int32),
                ("ctas_per_sm", ctypes.c_int32), ("path", ctypes.c_int32),
                ("stages", ctypes.c_int32), ("reserved", ctypes.c_int32)]


SCL_FAMILY_U32, SCL_FAMILY_F32, SCL_FAMILY_KEYED, SCL_FAMILY_MIXED = 0, 1, 2, 3


class scl_autotune_config(ctypes.Structure):
    _fields_ = [("probe_bytes", ctypes.c_uint64), ("reps", ctypes.c_uint32),
                ("families", ctypes.c_uint32)]


class scl_autotune_report(ctypes.Structure):
    _fields_ = [("chosen", scl_shape * 4), ("best_ms", ctypes.c_double * 4),
                ("candidates", ctypes.c_uint32 * 4)]


class scl_server_config(ctypes.Structure):
    _fields_ = [("inflight_batches", ctypes.c_int32), ("max_batch_tasks", ctypes.c_uint32),
                ("hbm_budget_bytes", ctypes.c_uint64), ("reserved", ctypes.c_uint64 * 2)]


class scl_server_stats(ctypes.Structure):
    _fields_ = [(k, ctypes.c_uint64) for k in (
        "submitted", "completed", "rejected", "batches", "max_batch", "kernel_launches",
        "admission_waits", "budget_bytes", "resident_bytes", "bytes_in_use",
        "peak_bytes_in_use")]


class scl_devserver_config(ctypes.Structure):
    _fields_ = [("job_ring", ctypes.c_uint32), ("unit_ring", ctypes.c_uint32),
                ("keyed_slots", ctypes.c_uint32), ("ctas_per_sm", ctypes.c_int32),
                ("idle_stop_ns", ctypes.c_uint64), ("wait_limit_ns", ctypes.c_uint64),
                ("reserved", ctypes.c_uint64 * 2)]


class scl_devserver_stats(ctypes.Structure):
    _fields_ = [(k, ctypes.c_uint64) for k in (
        "submitted", "completed", "failed", "kernel_launches", "idle_stops", "device_errors",
        "units", "ring_waits", "max_inflight")] + [
        ("grid", ctypes.c_uint32), ("block", ctypes.c_uint32),
        ("items_per_thread", ctypes.c_uint32), ("reserved0", ctypes.c_uint32),
        ("reserved", ctypes.c_uint64 * 3)]


IDLE_STOP_NEVER = (1 << 64) - 1


class scl_task(ctypes.Structure):
    _fields_ = [("part", ctypes.c_uint64), ("kernel", ctypes.c_int32),
                ("reduce", ctypes.c_int32), ("num_keys", ctypes.c_uint32),
                ("coef", ctypes.c_float * 3), ("counts_out", ctypes.c_void_p),
                ("sums_out", ctypes.c_void_p), ("sums64_out", ctypes.c_void_p),
                ("reserved", ctypes.c_uint64)]


class scl_task_data(ctypes.Structure):
    _fields_ = [("host0", ctypes.c_void_p), ("host1", ctypes.c_void_p), ("n", ctypes.c_uint64),
                ("dtype", ctypes.c_int32), ("reserved", ctypes.c_uint32)]


assert ctypes.sizeof(scl_result) == 48 and ctypes.sizeof(scl_task) == 64
assert ctypes.sizeof(scl_task_data) == 32

# Bulk array of scl_task_data.
TASK_DATA_DTYPE = np.dtype([("host0", "<u8"), ("host1", "<u8"), ("n", "<u8"), ("dtype", "<i4"),
                            ("reserved", "<u4")])
assert TASK_DATA_DTYPE.itemsize == 32

# Result array dtype matching scl_result, for bulk reads.
RESULT_DTYPE = np.dtype([("u64_sum", "<u8"), ("f64_sum", "<f8"), ("f32_sum", "<f4"),
                         ("f32_min", "<f4"), ("f32_max", "<f4"), ("status", "<i4"),
                         ("n", "<u8"), ("kind", "<u4"), ("reserved", "<u4")])
assert RESULT_DTYPE.itemsize == 48


class SclError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__("%s (%d): %s" % (_strerror(status), status, msg))
        self.status = status


def _load() -> ctypes.CDLL:
    if not os.path.exists(_LIB_PATH):
        raise ImportError("libscl.so is not built (%s); run __graft_entry__.build() or "
                          "python paper_1505_01120_gb300/build.py" % _LIB_PATH)
    return ctypes.CDLL(_LIB_PATH)


lib = _load()

_P = ctypes.c_void_p
_u64, _u32, _i32 = ctypes.c_uint64, ctypes.c_uint32, ctypes.c_int32
_PP = ctypes.POINTER(ctypes.c_void_p)

_SIGS = {
    "scl_strerror": ([ctypes.c_int], ctypes.c_char_p),
    "scl_last_error": ([], ctypes.c_char_p),
    "scl_abi_version": ([], ctypes.c_int),
    "scl_kernel_launches_total": ([ctypes.POINTER(_u64)], ctypes.c_int),
    "scl_create": ([ctypes.POINTER(scl_config), _PP], ctypes.c_int),
    "scl_destroy": ([_P], ctypes.c_int),
    "scl_arena_stats": ([_P, ctypes.POINTER(_u64), ctypes.POINTER(_u64)], ctypes.c_int),
    "scl_load_partition": ([_P, _P, ctypes.c_int, _u64, _P, ctypes.POINTER(_u64)], ctypes.c_int),
    "scl_load_partition_kv": ([_P, _P, _P, _u64, _P, ctypes.POINTER(_u64)], ctypes.c_int),
    "scl_wrap_device": ([_P, _P, _P, ctypes.c_int, _u64, ctypes.POINTER(_u64)], ctypes.c_int),
    "scl_alloc_partition": ([_P, ctypes.c_int, _u64, ctypes.POINTER(_u64)], ctypes.c_int),
    "scl_set_large_path": ([_P, ctypes.c_int], ctypes.c_int),
    "scl_set_batch_split": ([_P, ctypes.c_int], ctypes.c_int),
    "scl_free_partition": ([_P, _u64], ctypes.c_int),
    "scl_reload_partition": ([_P, _u64, _P, _P, _P], ctypes.c_int),
    "scl_partition_info": ([_P, _u64, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(_u64),
                            _PP, _PP], ctypes.c_int),
    "scl_read_partition": ([_P, _u64, _P, _P, _P], ctypes.c_int),
    "scl_map": ([_P, _u64, ctypes.c_int, _P, _P, ctypes.POINTER(_u64)], ctypes.c_int),
    "scl_map_into": ([_P, _u64, ctypes.c_int, _P, _u64, _P], ctypes.c_int),
    "scl_map_reduce": ([_P, _u64, ctypes.c_int, _P, ctypes.c_int, _P,
                        ctypes.POINTER(scl_result)], ctypes.c_int),
    "scl_map_reduce_async": ([_P, _u64, ctypes.c_int, _P, ctypes.c_int, _P, _P], ctypes.c_int),
    "scl_keyed_reduce": ([_P, _u64, _u32, _P, _P, _P, _P, ctypes.POINTER(scl_result)],
                         ctypes.c_int),
    "scl_keyed_reduce_async": ([_P, _u64, _u32, _P, _P, _P, _P, _P], ctypes.c_int),
    "scl_keyed_reduce_large": ([_P, _u64, _u32, _P, _P, _P, _P, ctypes.POINTER(scl_result)],
                               ctypes.c_int),
    "scl_keyed_reduce_large_async": ([_P, _u64, _u32, _P, _P, _P, _P, _P], ctypes.c_int),
    "scl_keyed_reduce_hashed": ([_P, _u64, _u32, _P, _P, _P, _P, ctypes.POINTER(scl_result)],
                                ctypes.c_int),
    "scl_reduce_arrays": ([_P, _P, _u32, _P, ctypes.POINTER(_u64)], ctypes.c_int),
    "scl_reduce_arrays_into": ([_P, _P, _u32, _u64, _P], ctypes.c_int),
    "scl_vector_add": ([_P, _u64, _u64, _P, ctypes.POINTER(_u64)], ctypes.c_int),
    "scl_combine": ([_P, _u32, ctypes.POINTER(scl_result)], ctypes.c_int),
    "scl_combine_keyed": ([_P, _P, _u32, _u32, _P, _P], ctypes.c_int),
    "scl_batch_create": ([_P, _P, _u32, _PP], ctypes.c_int),
    "scl_batch_launch": ([_P, _P], ctypes.c_int),
    "scl_batch_capture": ([_P, _P], ctypes.c_int),
    "scl_batch_results": ([_P, _P, _P], ctypes.c_int),
    "scl_batch_kernel_launches": ([_P, ctypes.POINTER(_u32)], ctypes.c_int),
    "scl_batch_destroy": ([_P], ctypes.c_int),
    "scl_batch_run": ([_P, _P, _u32, _P, _P], ctypes.c_int),
    "scl_get_shape": ([_P, ctypes.c_int, ctypes.POINTER(scl_shape)], ctypes.c_int),
    "scl_set_shape": ([_P, ctypes.c_int, ctypes.POINTER(scl_shape)], ctypes.c_int),
    "scl_autotune": ([_P, ctypes.POINTER(scl_autotune_config), _P,
                      ctypes.POINTER(scl_autotune_report)], ctypes.c_int),
    "scl_server_start": ([_P, ctypes.POINTER(scl_server_config)], ctypes.c_int),
    "scl_server_submit": ([_P, _P, ctypes.POINTER(_u64)], ctypes.c_int),
    "scl_server_submit_load": ([_P, _P, _P, ctypes.c_int, _u64, _P, ctypes.POINTER(_u64)],
                               ctypes.c_int),
    "scl_server_poll": ([_P, _u64, ctypes.POINTER(scl_result)], ctypes.c_int),
    "scl_server_wait": ([_P, _u64, _u32, ctypes.POINTER(scl_result)], ctypes.c_int),
    "scl_server_get_stats": ([_P, ctypes.POINTER(scl_server_stats)], ctypes.c_int),
    "scl_server_stop": ([_P], ctypes.c_int),
    "scl_server_replay": ([_P, _P, _P, _u32, _P, _P], ctypes.c_int),
    "scl_server_replay_load": ([_P, _P, _P, _P, _u32, _P, _P], ctypes.c_int),
    "scl_devserver_start": ([_P, ctypes.POINTER(scl_devserver_config)], ctypes.c_int),
    "scl_devserver_submit": ([_P, _P, ctypes.POINTER(_u64)], ctypes.c_int),
    "scl_devserver_poll": ([_P, _u64, ctypes.POINTER(scl_result)], ctypes.c_int),
    "scl_devserver_wait": ([_P, _u64, _u32, ctypes.POINTER(scl_result)], ctypes.c_int),
    "scl_devserver_get_stats": ([_P, ctypes.POINTER(scl_devserver_stats)], ctypes.c_int),
    "scl_devserver_stop": ([_P], ctypes.c_int),
    "scl_devserver_replay": ([_P, _P, _P, _u32, _P, _P], ctypes.c_int),
    "scl_map_reduce_noalloc": ([_P, ctypes.c_int, _u64, ctypes.c_int, _P, ctypes.c_int, _P, _P],
                               ctypes.c_int),
}

for _name, (_args, _res) in _SIGS.items():
    _f = getattr(lib, _name)
    _f.argtypes = _args
    _f.restype = _res


def exported_symbols() -> list[str]:
    """Names of every entry point this binding declares."""
    return list(_SIGS)


def _strerror(status: int) -> str:
    return lib.scl_strerror(status).decode()


def _check(status: int, allow=(SCL_OK,)) -> int:
    if status not in allow:
        raise SclError(status, lib.scl_last_error().decode())
    return status


def _ptr(x) -> int | None:
    """Address of a numpy array, a torch tensor, an int address, or None."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if isinstance(x, np.ndarray):
        return x.ctypes.data
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    raise TypeError("cannot take the address of %r" % type(x))


def _coef(coef):
    if coef is None:
        return None
    c = np.ascontiguousarray(coef, dtype=np.float32)
    if c.size != 3:
        raise ValueError("coef must have 3 entries")
    return c


# ------------------------------------------------------------------ API

def scl_abi_version() -> int:
    return lib.scl_abi_version()


def scl_kernel_launches_total() -> int:
    v = _u64()
    _check(lib.scl_kernel_launches_total(ctypes.byref(v)))
    return v.value


def scl_create(device: int, arena_ptr: int, arena_bytes: int, hbm_budget_bytes: int = 0,
               inflight_batches: int = 4, tune_cache_path: str | None = None) -> int:
    cfg = scl_config(device=device, arena=arena_ptr, arena_bytes=arena_bytes,
                     hbm_budget_bytes=hbm_budget_bytes, inflight_batches=inflight_batches,
                     tune_cache_path=tune_cache_path.encode() if tune_cache_path else None)
    h = ctypes.c_void_p()
    _check(lib.scl_create(ctypes.byref(cfg), ctypes.byref(h)))
    return h.value


def scl_destroy(ctx: int) -> None:
    _check(lib.scl_destroy(ctx))


def scl_arena_stats(ctx: int) -> tuple[int, int]:
    f, l = _u64(), _u64()
    _check(lib.scl_arena_stats(ctx, ctypes.byref(f), ctypes.byref(l)))
    return f.value, l.value


def scl_load_partition(ctx: int, host, dtype: int, n: int | None = None, stream: int = 0) -> int:
    if n is None:
        n = int(host.size if isinstance(host, np.ndarray) else host.numel())
    out = _u64()
    _check(lib.scl_load_partition(ctx, _ptr(host), dtype, n, stream, ctypes.byref(out)))
    return out.value


def scl_load_partition_kv(ctx: int, keys, vals, n: int | None = None, stream: int = 0) -> int:
    if n is None:
        n = int(keys.size if isinstance(keys, np.ndarray) else keys.numel())
    out = _u64()
    _check(lib.scl_load_partition_kv(ctx, _ptr(keys), _ptr(vals), n, stream, ctypes.byref(out)))
    return out.value


SCL_LARGE_AUTO, SCL_LARGE_PACKED, SCL_LARGE_PARTITIONED, SCL_LARGE_DIRECT = 0, 1, 2, 3


def scl_set_large_path(ctx: int, path: int) -> None:
    """Path of this context's later large-key reduces (SCL_LARGE_*)."""
    _check(lib.scl_set_large_path(ctx, path))


def scl_set_batch_split(ctx: int, on: bool) -> None:
    """Whether later batches mixing families launch one kernel per family,
    concurrently (the default), or one mixed kernel."""
    _check(lib.scl_set_batch_split(ctx, int(bool(on))))


def scl_alloc_partition(ctx: int, dtype: int, n: int) -> int:
    """An arena-resident partition whose contents the caller writes on the
    device (pointers from scl_partition_info)."""
    out = _u64()
    _check(lib.scl_alloc_partition(ctx, dtype, n, ctypes.byref(out)))
    return out.value


def scl_wrap_device(ctx: int, dev0, dev1, dtype: int, n: int) -> int:
    out = _u64()
    _check(lib.scl_wrap_device(ctx, _ptr(dev0), _ptr(dev1), dtype, n, ctypes.byref(out)))
    return out.value


def scl_reload_partition(ctx: int, part: int, host0, host1=None, stream: int = 0) -> None:
    _check(lib.scl_reload_partition(ctx, part, _ptr(host0), _ptr(host1), stream))


def scl_free_partition(ctx: int, part: int) -> None:
    _check(lib.scl_free_partition(ctx, part))


def scl_partition_info(ctx: int, part: int) -> tuple[int, int, int, int | None]:
    dt, n, d0, d1 = ctypes.c_int(), _u64(), ctypes.c_void_p(), ctypes.c_void_p()
    _check(lib.scl_partition_info(ctx, part, ctypes.byref(dt), ctypes.byref(n),
                                  ctypes.byref(d0), ctypes.byref(d1)))
    return dt.value, n.value, d0.value, d1.value


def scl_read_partition(ctx: int, part: int, host0, host1=None, stream: int = 0) -> None:
    _check(lib.scl_read_partition(ctx, part, _ptr(host0), _ptr(host1), stream))


def scl_map(ctx: int, part: int, kernel: int, coef=None, stream: int = 0) -> int:
    c = _coef(coef)
    out = _u64()
    _check(lib.scl_map(ctx, part, kernel, _ptr(c), stream, ctypes.byref(out)))
    return out.value


def scl_map_into(ctx: int, part: int, kernel: int, out: int, coef=None, stream: int = 0) -> None:
    c = _coef(coef)
    _check(lib.scl_map_into(ctx, part, kernel, _ptr(c), out, stream))


def scl_map_reduce(ctx: int, part: int, kernel: int, reduce: int, coef=None,
                   stream: int = 0) -> scl_result:
    c = _coef(coef)
    r = scl_result()
    _check(lib.scl_map_reduce(ctx, part, kernel, _ptr(c), reduce, stream, ctypes.byref(r)))
    return r


def scl_map_reduce_async(ctx: int, part: int, kernel: int, reduce: int, dev_out, coef=None,
                         stream: int = 0) -> None:
    c = _coef(coef)
    _check(lib.scl_map_reduce_async(ctx, part, kernel, _ptr(c), reduce, stream, _ptr(dev_out)))


def scl_keyed_reduce(ctx: int, part: int, num_keys: int = 4096, stream: int = 0,
                     want_f64: bool = True):
    """Returns (counts uint32[num_keys], sums float32[num_keys], sums64 or None,
    scl_result).  Raises SclError(SCL_E_KEY_RANGE) after filling the tables if
    a key was out of range; the partial tables are on the exception as .tables."""
    counts = np.empty(num_keys, np.uint32)
    sums = np.empty(num_keys, np.float32)
    s64 = np.empty(num_keys, np.float64) if want_f64 else None
    r = scl_result()
    st = lib.scl_keyed_reduce(ctx, part, num_keys, stream, _ptr(counts), _ptr(sums), _ptr(s64),
                              ctypes.byref(r))
    if st == SCL_E_KEY_RANGE:
        err = SclError(st, lib.scl_last_error().decode())
        err.tables = (counts, sums, s64, r)
        raise err
    _check(st)
    return counts, sums, s64, r


def scl_keyed_reduce_hashed(ctx: int, part: int, num_keys: int = 4096, stream: int = 0,
                            want_f64: bool = True):
    """Keyed reduce with keys hashed into buckets: (counts, sums, sums64, result)."""
    counts = np.empty(num_keys, np.uint32)
    sums = np.empty(num_keys, np.float32)
    s64 = np.empty(num_keys, np.float64) if want_f64 else None
    r = scl_result()
    _check(lib.scl_keyed_reduce_hashed(ctx, part, num_keys, stream, _ptr(counts), _ptr(sums),
                                       _ptr(s64), ctypes.byref(r)))
    return counts, sums, s64, r


def scl_keyed_reduce_large(ctx: int, part: int, num_keys: int, stream: int = 0,
                           want_f64: bool = True):
    """Keyed reduce for key spaces up to 2^24: (counts, sums, sums64, result).
    Raises SclError(SCL_E_KEY_RANGE) with .tables after a skipped key."""
    counts = np.empty(num_keys, np.uint32)
    sums = np.empty(num_keys, np.float32)
    s64 = np.empty(num_keys, np.float64) if want_f64 else None
    r = scl_result()
    st = lib.scl_keyed_reduce_large(ctx, part, num_keys, stream, _ptr(counts), _ptr(sums),
                                    _ptr(s64), ctypes.byref(r))
    if st == SCL_E_KEY_RANGE:
        err = SclError(st, lib.scl_last_error().decode())
        err.tables = (counts, sums, s64, r)
        raise err
    _check(st)
    return counts, sums, s64, r


def scl_keyed_reduce_large_async(ctx: int, part: int, num_keys: int, counts_dev, sums_dev,
                                 sums64_dev, result_dev, stream: int = 0) -> None:
    _check(lib.scl_keyed_reduce_large_async(ctx, part, num_keys, stream, _ptr(counts_dev),
                                            _ptr(sums_dev), _ptr(sums64_dev), _ptr(result_dev)))


def scl_keyed_reduce_async(ctx: int, part: int, num_keys: int, counts_dev, sums_dev,
                           sums64_dev=None, result_dev=None, stream: int = 0) -> None:
    _check(lib.scl_keyed_reduce_async(ctx, part, num_keys, stream, _ptr(counts_dev),
                                      _ptr(sums_dev), _ptr(sums64_dev), _ptr(result_dev)))


def _parts(parts) -> ctypes.Array:
    return (ctypes.c_uint64 * max(1, len(parts)))(*parts)


def scl_reduce_arrays(ctx: int, parts, stream: int = 0) -> int:
    out = _u64()
    _check(lib.scl_reduce_arrays(ctx, ctypes.cast(_parts(parts), ctypes.c_void_p), len(parts),
                                 stream, ctypes.byref(out)))
    return out.value


def scl_reduce_arrays_into(ctx: int, parts, out: int, stream: int = 0) -> None:
    _check(lib.scl_reduce_arrays_into(ctx, ctypes.cast(_parts(parts), ctypes.c_void_p),
                                      len(parts), out, stream))


def scl_vector_add(ctx: int, a: int, b: int, stream: int = 0) -> int:
    out = _u64()
    _check(lib.scl_vector_add(ctx, a, b, stream, ctypes.byref(out)))
    return out.value


def scl_combine(parts) -> scl_result:
    arr = (scl_result * len(parts))(*parts)
    out = scl_result()
    _check(lib.scl_combine(ctypes.cast(arr, ctypes.c_void_p), len(parts), ctypes.byref(out)))
    return out


def scl_combine_keyed(counts: np.ndarray, sums64: np.ndarray | None):
    counts = np.ascontiguousarray(counts, np.uint32)
    k, nk = counts.shape
    co = np.empty(nk, np.uint32)
    so = None
    if sums64 is not None:
        sums64 = np.ascontiguousarray(sums64, np.float64)
        so = np.empty(nk, np.float64)
    _check(lib.scl_combine_keyed(_ptr(counts), _ptr(sums64), k, nk, _ptr(co), _ptr(so)))
    return co, so


def scl_get_shape(ctx: int, family: int) -> dict:
    s = scl_shape()
    _check(lib.scl_get_shape(ctx, family, ctypes.byref(s)))
    return {k: getattr(s, k) for k, _ in s._fields_ if k != "reserved"}


def scl_set_shape(ctx: int, family: int, block: int, items_per_thread: int,
                  ctas_per_sm: int = 0, path: int = 0, stages: int = 0) -> None:
    s = scl_shape(block=block, items_per_thread=items_per_thread, ctas_per_sm=ctas_per_sm,
                  path=path, stages=stages)
    _check(lib.scl_set_shape(ctx, family, ctypes.byref(s)))


def scl_autotune(ctx: int, stream: int = 0, probe_bytes: int = 0, reps: int = 0,
                 families: int = 0) -> list[dict]:
    """Run the autotuner; returns per family the chosen shape, its probe time
    and how many candidates were timed."""
    cfg = scl_autotune_config(probe_bytes=probe_bytes, reps=reps, families=families)
    rep = scl_autotune_report()
    _check(lib.scl_autotune(ctx, ctypes.byref(cfg), stream, ctypes.byref(rep)))
    out = []
    for f in range(4):
        s = rep.chosen[f]
        out.append({"block": s.block, "items_per_thread": s.items_per_thread,
                    "ctas_per_sm": s.ctas_per_sm, "path": s.path, "stages": s.stages,
                    "best_ms": rep.best_ms[f], "candidates": rep.candidates[f]})
    return out


def scl_server_start(ctx: int, inflight_batches: int = 4, max_batch_tasks: int = 4096,
                     hbm_budget_bytes: int = 0) -> None:
    cfg = scl_server_config(inflight_batches=inflight_batches, max_batch_tasks=max_batch_tasks,
                            hbm_budget_bytes=hbm_budget_bytes)
    _check(lib.scl_server_start(ctx, ctypes.byref(cfg)))


def scl_server_submit(ctx: int, tasks: ctypes.Array, index: int = 0) -> int:
    t = _u64()
    _check(lib.scl_server_submit(ctx, ctypes.byref(tasks[index]), ctypes.byref(t)))
    return t.value


def scl_server_submit_load(ctx: int, host0, host1, dtype: int, n: int, tasks: ctypes.Array,
                           index: int = 0) -> int:
    t = _u64()
    _check(lib.scl_server_submit_load(ctx, _ptr(host0), _ptr(host1), dtype, n,
                                      ctypes.byref(tasks[index]), ctypes.byref(t)))
    return t.value


def scl_server_poll(ctx: int, ticket: int):
    """scl_result when done, None while pending."""
    r = scl_result()
    st = lib.scl_server_poll(ctx, ticket, ctypes.byref(r))
    if st == SCL_E_PENDING:
        return None
    _check(st)
    return r


def scl_server_wait(ctx: int, ticket: int, timeout_ms: int = 60_000) -> scl_result:
    r = scl_result()
    _check(lib.scl_server_wait(ctx, ticket, timeout_ms, ctypes.byref(r)))
    return r


def scl_server_get_stats(ctx: int) -> dict:
    s = scl_server_stats()
    _check(lib.scl_server_get_stats(ctx, ctypes.byref(s)))
    return {k: getattr(s, k) for k, _ in s._fields_}


def scl_server_stop(ctx: int) -> None:
    _check(lib.scl_server_stop(ctx))


def scl_server_replay(ctx: int, tasks: ctypes.Array, arrival_s: np.ndarray, n: int,
                      allow_errors: bool = False):
    """Returns (latency_ns int64[n], results RESULT_DTYPE[n])."""
    arr = np.ascontiguousarray(arrival_s, dtype=np.float64)
    lat = np.zeros(max(1, n), dtype=np.int64)
    res = np.zeros(max(1, n), dtype=RESULT_DTYPE)
    st = lib.scl_server_replay(ctx, _tasks_ptr(tasks), arr.ctypes.data, n,
                               lat.ctypes.data, res.ctypes.data)
    if not allow_errors:
        _check(st)
    return lat[:n], res[:n]


def scl_server_replay_load(ctx: int, tasks: ctypes.Array, data: np.ndarray,
                           arrival_s: np.ndarray, n: int, allow_errors: bool = False):
    """scl_server_replay where data[i] (TASK_DATA_DTYPE; host0 = 0 for a task on
    its resident partition) gives the host arrays of tasks that bring new
    data.  Returns (latency_ns int64[n], results RESULT_DTYPE[n])."""
    arr = np.ascontiguousarray(arrival_s, dtype=np.float64)
    d = np.ascontiguousarray(data, dtype=TASK_DATA_DTYPE)
    lat = np.zeros(max(1, n), dtype=np.int64)
    res = np.zeros(max(1, n), dtype=RESULT_DTYPE)
    st = lib.scl_server_replay_load(ctx, _tasks_ptr(tasks), d.ctypes.data,
                                    arr.ctypes.data, n, lat.ctypes.data, res.ctypes.data)
    if not allow_errors:
        _check(st)
    return lat[:n], res[:n]


def scl_devserver_start(ctx: int, job_ring: int = 0, unit_ring: int = 0, keyed_slots: int = 0,
                        ctas_per_sm: int = 0, idle_stop_ns: int = 0,
                        wait_limit_ns: int = 0) -> None:
    cfg = scl_devserver_config(job_ring=job_ring, unit_ring=unit_ring, keyed_slots=keyed_slots,
                               ctas_per_sm=ctas_per_sm, idle_stop_ns=idle_stop_ns,
                               wait_limit_ns=wait_limit_ns)
    _check(lib.scl_devserver_start(ctx, ctypes.byref(cfg)))


def scl_devserver_submit(ctx: int, tasks: ctypes.Array, index: int = 0) -> int:
    t = _u64()
    _check(lib.scl_devserver_submit(ctx, ctypes.byref(tasks[index]), ctypes.byref(t)))
    return t.value


def scl_devserver_poll(ctx: int, ticket: int):
    """The result, or None while the job is pending."""
    r = scl_result()
    st = lib.scl_devserver_poll(ctx, ticket, ctypes.byref(r))
    if st == SCL_E_PENDING:
        return None
    _check(st)
    return r


def scl_devserver_wait(ctx: int, ticket: int, timeout_ms: int = 60_000) -> scl_result:
    r = scl_result()
    _check(lib.scl_devserver_wait(ctx, ticket, timeout_ms, ctypes.byref(r)))
    return r


def scl_devserver_get_stats(ctx: int) -> dict:
    s = scl_devserver_stats()
    _check(lib.scl_devserver_get_stats(ctx, ctypes.byref(s)))
    return {k: getattr(s, k) for k, _ in scl_devserver_stats._fields_
            if not k.startswith("reserved")}


def scl_devserver_stop(ctx: int) -> None:
    _check(lib.scl_devserver_stop(ctx))


def scl_devserver_replay(ctx: int, tasks: ctypes.Array, arrival_s: np.ndarray, n: int,
                         allow_errors: bool = False):
    """Returns (latency_ns int64[n], results RESULT_DTYPE[n])."""
    arr = np.ascontiguousarray(arrival_s, dtype=np.float64)
    lat = np.zeros(max(1, n), dtype=np.int64)
    res = np.zeros(max(1, n), dtype=RESULT_DTYPE)
    st = lib.scl_devserver_replay(ctx, _tasks_ptr(tasks), arr.ctypes.data, n,
                                  lat.ctypes.data, res.ctypes.data)
    if not allow_errors:
        _check(st)
    return lat[:n], res[:n]


# Bulk array of scl_task (for traces of many tasks; replay functions take it).
TASK_DTYPE = np.dtype([("part", "<u8"), ("kernel", "<i4"), ("reduce", "<i4"),
                       ("num_keys", "<u4"), ("coef", "<f4", 3), ("counts_out", "<u8"),
                       ("sums_out", "<u8"), ("sums64_out", "<u8"), ("reserved", "<u8")])
assert TASK_DTYPE.itemsize == 64 and TASK_DTYPE.fields["counts_out"][1] == 32


def _tasks_ptr(tasks):
    if isinstance(tasks, np.ndarray):
        if tasks.dtype != TASK_DTYPE or not tasks.flags.c_contiguous:
            raise ValueError("tasks must be a contiguous TASK_DTYPE array")
        return tasks.ctypes.data
    return ctypes.cast(tasks, ctypes.c_void_p)


def make_tasks(specs) -> ctypes.Array:
    """specs: iterable of dicts with keys part, kernel, reduce and optionally
    num_keys, coef, counts_out, sums_out, sums64_out (device addresses)."""
    specs = list(specs)
    arr = (scl_task * max(1, len(specs)))()
    for i, s in enumerate(specs):
        t = arr[i]
        t.part = s["part"]
        t.kernel = s["kernel"]
        t.reduce = s["reduce"]
        t.num_keys = s.get("num_keys", 0)
        cf = s.get("coef", (0.5, -1.25, 0.1))
        t.coef[0], t.coef[1], t.coef[2] = (float(np.float32(v)) for v in cf)
        t.counts_out = _ptr(s.get("counts_out"))
        t.sums_out = _ptr(s.get("sums_out"))
        t.sums64_out = _ptr(s.get("sums64_out"))
    return arr


def scl_batch_create(ctx: int, tasks: ctypes.Array, ntasks: int) -> int:
    b = ctypes.c_void_p()
    _check(lib.scl_batch_create(ctx, ctypes.cast(tasks, ctypes.c_void_p), ntasks, ctypes.byref(b)))
    return b.value


def scl_batch_launch(batch: int, stream: int = 0) -> None:
    _check(lib.scl_batch_launch(batch, stream))


def scl_batch_capture(batch: int, stream: int) -> None:
    _check(lib.scl_batch_capture(batch, stream))


def scl_batch_results(batch: int, ntasks: int, stream: int = 0, allow_key_range: bool = False):
    out = np.zeros(max(1, ntasks), dtype=RESULT_DTYPE)
    allow = (SCL_OK, SCL_E_KEY_RANGE) if allow_key_range else (SCL_OK,)
    _check(lib.scl_batch_results(batch, stream, out.ctypes.data), allow)
    return out[:ntasks]


def scl_batch_kernel_launches(batch: int) -> int:
    v = _u32()
    _check(lib.scl_batch_kernel_launches(batch, ctypes.byref(v)))
    return v.value


def scl_batch_destroy(batch: int) -> None:
    _check(lib.scl_batch_destroy(batch))


def scl_batch_run(ctx: int, tasks: ctypes.Array, ntasks: int, stream: int = 0,
                  allow_key_range: bool = False):
    out = np.zeros(max(1, ntasks), dtype=RESULT_DTYPE)
    allow = (SCL_OK, SCL_E_KEY_RANGE) if allow_key_range else (SCL_OK,)
    _check(lib.scl_batch_run(ctx, ctypes.cast(tasks, ctypes.c_void_p), ntasks, stream,
                             out.ctypes.data), allow)
    return out[:ntasks]


def scl_map_reduce_noalloc(dev_in, dtype: int, n: int, kernel: int, reduce: int, dev_out,
                           coef=None, stream: int = 0) -> None:
    """Map + reduce without any allocation (see include/scl.h): for callers
    that cannot allocate device memory when they need the result.  Inputs and
    the scl_result slot are device addresses the caller owns."""
    c = _coef(coef)
    _check(lib.scl_map_reduce_noalloc(_ptr(dev_in), dtype, n, kernel, _ptr(c), reduce, stream,
                                      _ptr(dev_out)))
