"""Seeded synthetic partitions for the SparkCL per-partition workloads.

This module only draws random inputs; it holds none of the map or reduce
arithmetic, so the CUDA path and the CPU oracle can both be fed from it
without sharing any of the method's code.  All draws use
``numpy.random.default_rng(seed)`` so a (workload, seed) pair fixes every byte.

Workloads (the paper runs MapCL / MapCLPartition / ReduceCL over RDD
partitions of primitive arrays, Sec. 3.1.3; its demos are Pi, vector add and
word count, Sec. 3.2; it prints no dataset, so these synthetic shapes stand in):

* ``mix32_partition``      1 x 1,048,576 uint32 uniform          (seed 1)
* ``poly3_partitions``     64 x 4,194,304 fp32 ~ N(0, 1)          (seed 2)
* ``keyed_partitions``     16 x 16,777,216 (int32 key U[0,4096), fp32 U(0,1)) (seed 3)
* ``batch_tasks``          10,000 log-normal sizes (median 16,384, sigma 1.5,
                           clipped [256, 8,388,608]), kernel uniform over 3  (seed 4)
* ``serve_trace``          Poisson arrivals, log-normal sizes clipped
                           [1,024, 67,108,864], kernel uniform over 3        (seed 5)
"""
from __future__ import annotations

import dataclasses

import numpy as np

KIND_MIX32 = 0     # uint32 partition, mix32 map, uint64 sum
KIND_POLY3 = 1     # fp32 partition, poly3 map, sum / min / max
KIND_KEYED = 2     # (int32 key, fp32 value) partition, per-key count / sum
KIND_NAMES = ("mix32_sum", "poly3_sum_min_max", "keyed_count_sum")

NUM_KEYS = 4096


def uniform_u32(n: int, rng: np.random.Generator) -> np.ndarray:
    return rng.integers(0, 1 << 32, size=n, dtype=np.uint32)


def normal_f32(n: int, rng: np.random.Generator, out=None) -> np.ndarray:
    if out is not None:
        rng.standard_normal(size=n, dtype=np.float32, out=out)
        return out
    return rng.standard_normal(size=n, dtype=np.float32)


def keys_i32(n: int, rng: np.random.Generator, num_keys: int = NUM_KEYS) -> np.ndarray:
    return rng.integers(0, num_keys, size=n, dtype=np.int32)


def zipf_keys_i32(n: int, rng: np.random.Generator, num_keys: int, s: float = 1.2) -> np.ndarray:
    """Keys with Zipf-like frequencies: numpy's zipf(s) ranks minus one, wrapped
    into [0, num_keys), so id 0 is the most frequent (a dictionary numbered by
    frequency, as WordCount's vocabulary would be)."""
    return ((rng.zipf(s, size=n) - 1) % num_keys).astype(np.int32)


def unit_f32(n: int, rng: np.random.Generator, out=None) -> np.ndarray:
    if out is not None:
        rng.random(size=n, dtype=np.float32, out=out)
        return out
    return rng.random(size=n, dtype=np.float32)


def mix32_partition(n: int = 1 << 20, seed: int = 1) -> np.ndarray:
    """One uint32 partition drawn uniformly."""
    return uniform_u32(n, np.random.default_rng(seed))


def poly3_partitions(parts: int = 64, n: int = 1 << 22, seed: int = 2) -> np.ndarray:
    """``parts`` fp32 partitions of ``n`` N(0,1) values, shape [parts, n]."""
    return normal_f32(parts * n, np.random.default_rng(seed)).reshape(parts, n)


def keyed_partitions(parts: int = 16, n: int = 1 << 24, seed: int = 3,
                     num_keys: int = NUM_KEYS):
    """``parts`` keyed partitions, SoA: (keys [parts, n] int32, vals [parts, n] fp32)."""
    rng = np.random.default_rng(seed)
    keys = keys_i32(parts * n, rng, num_keys).reshape(parts, n)
    vals = unit_f32(parts * n, rng).reshape(parts, n)
    return keys, vals


def lognormal_sizes(count: int, median: float, sigma: float, lo: int, hi: int,
                    rng: np.random.Generator) -> np.ndarray:
    """floor(exp(N(ln median, sigma))) clipped to [lo, hi], as int64."""
    s = np.floor(np.exp(rng.normal(np.log(median), sigma, size=count)))
    return np.clip(s, lo, hi).astype(np.int64)


@dataclasses.dataclass
class TaskSpec:
    kind: int       # KIND_MIX32 / KIND_POLY3 / KIND_KEYED
    n: int          # elements (pairs for keyed)
    seed: int       # seed of this task's data


def batch_tasks(count: int = 10_000, median: int = 16_384, sigma: float = 1.5,
                lo: int = 256, hi: int = 8_388_608, seed: int = 4) -> list[TaskSpec]:
    """Uneven partitions for one batched launch; kernel uniform over the three."""
    rng = np.random.default_rng(seed)
    sizes = lognormal_sizes(count, median, sigma, lo, hi, rng)
    kinds = rng.integers(0, 3, size=count)
    seeds = rng.integers(0, 1 << 31, size=count)
    return [TaskSpec(int(k), int(n), int(s)) for k, n, s in zip(kinds, sizes, seeds)]


def task_data(spec: TaskSpec, num_keys: int = NUM_KEYS):
    """The partition arrays of one task: (array,) or (keys, vals)."""
    rng = np.random.default_rng(spec.seed)
    if spec.kind == KIND_MIX32:
        return (uniform_u32(spec.n, rng),)
    if spec.kind == KIND_POLY3:
        return (normal_f32(spec.n, rng),)
    return (keys_i32(spec.n, rng, num_keys), unit_f32(spec.n, rng))


def batch_data_packed(specs: list[TaskSpec], seed: int = 4, num_keys: int = NUM_KEYS):
    """All tasks' data of a batch in three flat arrays (u32 words, f32 values,
    keyed pairs) plus per-task offsets, drawn from one stream so large batches
    generate quickly.  Returns dict with 'u32', 'f32', 'keys', 'vals', 'offset'
    (offset of each task inside the array of its kind)."""
    rng = np.random.default_rng(seed + 1_000_003)
    tot = [0, 0, 0]
    offs = np.zeros(len(specs), dtype=np.int64)
    for i, s in enumerate(specs):
        # start every partition on a 64-element (256-byte) boundary
        offs[i] = tot[s.kind]
        tot[s.kind] += (s.n + 63) // 64 * 64
    return {
        "u32": uniform_u32(tot[KIND_MIX32], rng),
        "f32": normal_f32(tot[KIND_POLY3], rng),
        "keys": keys_i32(tot[KIND_KEYED], rng, num_keys),
        "vals": unit_f32(tot[KIND_KEYED], rng),
        "offset": offs,
    }


def poisson_arrivals(rate: float, count: int, rng: np.random.Generator) -> np.ndarray:
    """Open-loop arrival times (seconds from 0) of a Poisson process."""
    return np.cumsum(rng.exponential(1.0 / rate, size=count))


def serve_trace(rate: float, count: int, median: int = 1 << 18, sigma: float = 1.5,
                lo: int = 1024, hi: int = 1 << 26, seed: int = 5):
    """Arrival times (s), sizes and kernels for the serving workload."""
    rng = np.random.default_rng(seed)
    t = poisson_arrivals(rate, count, rng)
    sizes = lognormal_sizes(count, median, sigma, lo, hi, rng)
    kinds = rng.integers(0, 3, size=count)
    return t, sizes, kinds
