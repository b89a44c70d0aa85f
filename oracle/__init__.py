"""CPU oracle for the SparkCL per-partition map/reduce path.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference leg of ``bench.py`` may import this package.  The
product path (the CUDA library and its Python binding) never imports it, and
it never imports the product path: the two share no code.

The arithmetic lives in ``oracle.c`` (plain C, one thread, fp64 accumulation,
compiled with ``-O2 -ffp-contract=off``); this module compiles it on first use
with gcc and marshals numpy arrays through ctypes.  Every function cites the
passage of the SparkCL paper (Segal et al. 2015) it follows:

* ``mix32`` / ``map_mix32`` / ``sum_u32`` / ``mix32_sum_range`` -- the integer
  user kernel run once per element (Sec. 3.1.1.2) and ReduceCL's sum
  (Sec. 3.1.3 item 3).
* ``poly3`` / ``map_poly3`` / ``reduce_f32`` -- the fp32 user kernel
  (MapCLPartition, Sec. 3.1.3 item 2) with ReduceCL's sum/min/max.
* ``keyed_count_sum`` -- the WordCount-style reduce-by-key (Sec. 3.2.3);
  ``keyed_hashed_count_sum`` the same after hashing each key into a bucket.
* ``combine`` / ``combine_keyed`` -- ReduceCL's tree combine of per-partition
  results (Sec. 3.1.3 item 3, Sec. 3.2.2), as a plain left fold.
* ``add_arrays`` -- ReduceCL over k partition arrays with the vector-add
  kernel of Fig. 3 (Sec. 3.2.2), in the binary-counter tree order.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_CFLAGS = ["-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared"]

_lock = threading.Lock()
_lib = None

F32_DEFAULT_COEF = (0.5, -1.25, 0.1)


def build(src: str = _SRC, out: str = _LIB_PATH) -> str:
    """Compile ``src`` into the shared object ``out`` with gcc; return ``out``."""
    tmp = out + ".tmp%d" % os.getpid()
    subprocess.check_call(["gcc", *_CFLAGS, "-o", tmp, src, "-lm"])
    os.replace(tmp, out)
    return out


def _bind(lib: ctypes.CDLL) -> ctypes.CDLL:
    P = ctypes.c_void_p
    u64, u32, i32 = ctypes.c_uint64, ctypes.c_uint32, ctypes.c_int
    lib.orc_mix32.argtypes, lib.orc_mix32.restype = [u32], u32
    lib.orc_poly3.argtypes = [ctypes.c_float] * 4
    lib.orc_poly3.restype = ctypes.c_float
    lib.orc_map_mix32.argtypes, lib.orc_map_mix32.restype = [P, u64, P], None
    lib.orc_map_poly3.argtypes, lib.orc_map_poly3.restype = [P, u64, P, P], None
    lib.orc_sum_u32.argtypes, lib.orc_sum_u32.restype = [P, u64, i32], u64
    lib.orc_mix32_sum_range.argtypes = [u64, u64]
    lib.orc_mix32_sum_range.restype = u64
    lib.orc_reduce_f32.argtypes = [P, u64, i32, P, P, P, P]
    lib.orc_reduce_f32.restype = None
    lib.orc_keyed_count_sum.argtypes = [P, P, u64, u32, P, P]
    lib.orc_keyed_count_sum.restype = u64
    lib.orc_combine.argtypes = [P, P, P, P, u32, P, P, P, P]
    lib.orc_combine.restype = None
    lib.orc_combine_keyed.argtypes = [P, P, u32, u32, P, P]
    lib.orc_combine_keyed.restype = None
    lib.orc_keyed_hashed_count_sum.argtypes = [P, P, u64, u32, P, P]
    lib.orc_keyed_hashed_count_sum.restype = None
    lib.orc_add_arrays_f32.argtypes = [P, u32, u64, P]
    lib.orc_add_arrays_f32.restype = None
    lib.orc_add_arrays_u32.argtypes = [P, u32, u64, P]
    lib.orc_add_arrays_u32.restype = None
    return lib


def load(path: str | None = None) -> ctypes.CDLL:
    """Return the bound oracle library, compiling it first if needed.

    ``path`` loads another build of the oracle (the mutation tests compile
    deliberately broken copies of ``oracle.c`` to show the pins catch them).
    """
    global _lib
    if path is not None:
        return _bind(ctypes.CDLL(path))
    with _lock:
        if _lib is None:
            if (not os.path.exists(_LIB_PATH)
                    or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC)):
                build()
            _lib = _bind(ctypes.CDLL(_LIB_PATH))
    return _lib


def _ptr(a: np.ndarray) -> int:
    return a.ctypes.data


def _c(a, dtype) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=dtype)


# --------------------------------------------------------------------- maps

def mix32(x: int, lib=None) -> int:
    """mix32 of one uint32 (Sec. 3.1.1.2, run() over one element)."""
    return int((lib or load()).orc_mix32(int(x) & 0xFFFFFFFF))


def poly3(x: float, coef=F32_DEFAULT_COEF, lib=None) -> np.float32:
    """poly3 of one fp32 element (Sec. 3.1.1.2, run() over one element)."""
    a, b, c = (float(np.float32(v)) for v in coef)
    return np.float32((lib or load()).orc_poly3(float(np.float32(x)), a, b, c))


def map_mix32(a, lib=None) -> np.ndarray:
    """MapCL of mix32 with the output array materialised (Sec. 3.1.3 item 1)."""
    a = _c(a, np.uint32)
    out = np.empty_like(a)
    (lib or load()).orc_map_mix32(_ptr(a), a.size, _ptr(out))
    return out


def map_poly3(x, coef=F32_DEFAULT_COEF, lib=None) -> np.ndarray:
    """MapCL of poly3 with the output array materialised (Sec. 3.1.3 item 1)."""
    x = _c(x, np.float32)
    cf = np.asarray(coef, dtype=np.float32)
    out = np.empty_like(x)
    (lib or load()).orc_map_poly3(_ptr(x), x.size, _ptr(cf), _ptr(out))
    return out


# --------------------------------------------------------------- reductions

def sum_u32(a, mix: bool = True, lib=None) -> int:
    """ReduceCL sum of map(x) over a uint32 partition, mod 2^64 (Sec. 3.1.3)."""
    a = _c(a, np.uint32)
    return int((lib or load()).orc_sum_u32(_ptr(a), a.size, 1 if mix else 0))


def mix32_sum_range(lo: int, hi: int, lib=None) -> int:
    """ReduceCL sum of mix32 over the implicit partition lo, lo+1, ..., hi-1."""
    return int((lib or load()).orc_mix32_sum_range(lo, hi))


def reduce_f32(x, poly: bool = True, coef=F32_DEFAULT_COEF, lib=None):
    """ReduceCL over an fp32 partition: (fp64 sum, fp32 min, fp32 max) of map(x)
    (Sec. 3.1.3 items 2-3).  Empty input gives (0.0, +inf, -inf)."""
    x = _c(x, np.float32)
    cf = np.asarray(coef, dtype=np.float32)
    s = ctypes.c_double()
    mn, mx = ctypes.c_float(), ctypes.c_float()
    (lib or load()).orc_reduce_f32(_ptr(x), x.size, 2 if poly else 0, _ptr(cf),
                                   ctypes.byref(s), ctypes.byref(mn),
                                   ctypes.byref(mx))
    return s.value, np.float32(mn.value), np.float32(mx.value)


def keyed_count_sum(keys, vals, num_keys: int = 4096, lib=None):
    """Reduce-by-key (Sec. 3.2.3): (uint32 count[num_keys], fp64 sum[num_keys],
    number of pairs skipped for an out-of-range key)."""
    keys = _c(keys, np.int32)
    vals = _c(vals, np.float32)
    if keys.size != vals.size:
        raise ValueError("keys and vals differ in length")
    cnt = np.empty(num_keys, dtype=np.uint32)
    s = np.empty(num_keys, dtype=np.float64)
    bad = (lib or load()).orc_keyed_count_sum(_ptr(keys), _ptr(vals), keys.size,
                                              num_keys, _ptr(cnt), _ptr(s))
    return cnt, s, int(bad)


def keyed_hashed_count_sum(keys, vals, num_keys: int = 4096, lib=None):
    """Reduce-by-key after hashing each key into a bucket,
    (mix32(key) * num_keys) >> 32 (Sec. 3.2.3): (uint32 count, fp64 sum)."""
    keys = _c(keys, np.int32)
    vals = _c(vals, np.float32)
    if keys.size != vals.size:
        raise ValueError("keys and vals differ in length")
    cnt = np.empty(num_keys, dtype=np.uint32)
    s = np.empty(num_keys, dtype=np.float64)
    (lib or load()).orc_keyed_hashed_count_sum(_ptr(keys), _ptr(vals), keys.size, num_keys,
                                               _ptr(cnt), _ptr(s))
    return cnt, s


def combine(u64_sums, f64_sums, mins, maxs, lib=None):
    """ReduceCL combine of per-partition results (Sec. 3.1.3 item 3):
    (uint64 sum, fp64 sum, min, max)."""
    u = _c(u64_sums, np.uint64)
    f = _c(f64_sums, np.float64)
    lo = _c(mins, np.float32)
    hi = _c(maxs, np.float32)
    k = u.size
    if not (f.size == lo.size == hi.size == k):
        raise ValueError("per-partition arrays differ in length")
    uo, fo = ctypes.c_uint64(), ctypes.c_double()
    mno, mxo = ctypes.c_float(), ctypes.c_float()
    (lib or load()).orc_combine(_ptr(u), _ptr(f), _ptr(lo), _ptr(hi), k,
                                ctypes.byref(uo), ctypes.byref(fo),
                                ctypes.byref(mno), ctypes.byref(mxo))
    return int(uo.value), fo.value, np.float32(mno.value), np.float32(mxo.value)


def combine_keyed(counts, sums, lib=None):
    """Merge per-partition keyed tables, shapes [k, num_keys] (Sec. 3.2.3)."""
    c = _c(counts, np.uint32)
    s = _c(sums, np.float64)
    if c.ndim != 2 or c.shape != s.shape:
        raise ValueError("tables must be 2-D and of one shape")
    k, nk = c.shape
    co = np.empty(nk, dtype=np.uint32)
    so = np.empty(nk, dtype=np.float64)
    (lib or load()).orc_combine_keyed(_ptr(c), _ptr(s), k, nk, _ptr(co), _ptr(so))
    return co, so


def add_arrays(arrays, lib=None) -> np.ndarray:
    """ReduceCL of k equal-length fp32 or uint32 arrays with the Fig. 3 vector-add
    kernel (Sec. 3.2.2): fp32 in the binary-counter tree order, uint32 wrapping."""
    arrays = list(arrays)
    if not arrays:
        raise ValueError("need at least one array")
    if len(arrays) > 4096:
        raise ValueError("at most 4096 arrays")
    dt = np.asarray(arrays[0]).dtype
    if dt not in (np.float32, np.uint32):
        raise ValueError("fp32 or uint32 arrays")
    arrs = [np.ascontiguousarray(a, dtype=dt) for a in arrays]
    n = arrs[0].size
    if any(a.size != n for a in arrs):
        raise ValueError("arrays differ in length")
    ptrs = (ctypes.c_void_p * len(arrs))(*[a.ctypes.data for a in arrs])
    out = np.empty(n, dtype=dt)
    fn = (lib or load()).orc_add_arrays_f32 if dt == np.float32 else \
        (lib or load()).orc_add_arrays_u32
    fn(ctypes.cast(ptrs, ctypes.c_void_p), len(arrs), n, out.ctypes.data)
    return out
