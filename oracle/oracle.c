/*
 * oracle.c -- plain, slow, single-threaded CPU definition of every map and
 * reduction on the SparkCL per-partition offload path.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link, load or
 * call this file: only the tests, the package smoke check and the benchmark's
 * CPU-baseline leg use it.  It shares no header, helper, table or constant
 * generator with the CUDA library; every constant below is written out here
 * from the workload definitions.
 *
 * What the method computes (SparkCL, Segal et al. 2015):
 *   - a user kernel's run() body executes once per element of a partition's
 *     primitive array (Sec. 3.1.1.2, Fig. 3: one work item per global id);
 *   - MapCL / MapCLPartition apply that kernel over a partition
 *     (Sec. 3.1.3 items 1-2);
 *   - ReduceCL folds per-element / per-partition results with a tree reduce
 *     (Sec. 3.1.3 item 3, Sec. 3.2.2);
 *   - the WordCount demo folds (key, value) pairs into per-key results
 *     (Sec. 3.2.3).
 * The paper does not fix the user kernels; the catalogue here is
 *   mix32  : x ^= x>>16; x *= 0x7feb352d; x ^= x>>15; x *= 0x846ca68b;
 *            x ^= x>>16  (all mod 2^32), summed into a uint64;
 *   poly3  : y = 0.5 x^3 - 1.25 x + 0.1 in fp32, read as the Horner form
 *            t = fma(a, x*x, b); y = fma(t, x, c) with x*x rounded once,
 *            coefficients {a, b, c} = {0.5f, -1.25f, 0.1f} by default;
 *   keyed  : count[key] += 1, sum[key] += value over (int32 key, fp32 value)
 *            pairs, keys in [0, num_keys);
 *   hashed keyed: the keyed reduce with each key first mixed by mix32 and
 *            mapped into [0, num_keys) as (mix32(key) * num_keys) >> 32
 *            (a WordCount-style hash into buckets, Sec. 3.2.3);
 *   add    : the vector-add kernel of Fig. 3, c[gid] = a[gid] + b[gid], used by
 *            ReduceCL to fold k equal-length partition arrays with a tree
 *            reduce (Sec. 3.2.2).  The tree is the binary-counter tree:
 *            leaves are taken left to right; whenever the two newest subtrees
 *            hold the same number of leaves they are combined (older + newer);
 *            after the last leaf the remaining subtrees are combined from the
 *            newest to the oldest, each older one on the left.  For k a power
 *            of two this is the balanced pairwise tree.
 * Accumulation is fp64 for floating point (the method's reference precision)
 * and exact uint64 (mod 2^64) for integers.  Min/max ignore NaN (a NaN never
 * replaces a number); an empty partition has sum 0, min +inf, max -inf.
 *
 * Build: gcc -O2 -ffp-contract=off -fPIC -shared oracle.c -lm
 * (-ffp-contract=off keeps x*x a separately rounded product; no fast-math).
 */
#include <math.h>
#include <stdint.h>
#include <string.h>

/* ------------------------------------------------------------------ maps */

/* mix32 bit-mix of one uint32 (the integer user kernel; Sec. 3.1.1.2 run()
 * body applied to one element). */
uint32_t orc_mix32(uint32_t x)
{
    x ^= x >> 16;
    x *= 0x7feb352du;
    x ^= x >> 15;
    x *= 0x846ca68bu;
    x ^= x >> 16;
    return x;
}

/* poly3 of one fp32 element: ((a*x^2) + b)*x + c, x^2 rounded once, then two
 * fused multiply-adds (the fp32 user kernel; Sec. 3.1.1.2). */
float orc_poly3(float x, float a, float b, float c)
{
    float x2 = x * x;
    float t = fmaf(a, x2, b);
    return fmaf(t, x, c);
}

/* MapCL with a materialised output array (Sec. 3.1.3 item 1; the
 * mapReturnValue "return an array" form of Sec. 3.1.1.3). */
void orc_map_mix32(const uint32_t *in, uint64_t n, uint32_t *out)
{
    for (uint64_t i = 0; i < n; ++i)
        out[i] = orc_mix32(in[i]);
}

void orc_map_poly3(const float *in, uint64_t n, const float coef[3], float *out)
{
    for (uint64_t i = 0; i < n; ++i)
        out[i] = orc_poly3(in[i], coef[0], coef[1], coef[2]);
}

/* ------------------------------------------------------------ reductions */

/* ReduceCL over one uint32 partition: sum of map(x) into uint64 (mod 2^64).
 * map = 0: identity, map = 1: mix32.  (Sec. 3.1.3 item 3.) */
uint64_t orc_sum_u32(const uint32_t *in, uint64_t n, int map)
{
    uint64_t s = 0;
    for (uint64_t i = 0; i < n; ++i) {
        uint32_t v = map ? orc_mix32(in[i]) : in[i];
        s += (uint64_t)v;
    }
    return s;
}

/* The same reduction over the implicit partition {lo, lo+1, ..., hi-1}
 * (an iota partition that needs no buffer; hi <= 2^32). */
uint64_t orc_mix32_sum_range(uint64_t lo, uint64_t hi)
{
    uint64_t s = 0;
    for (uint64_t i = lo; i < hi; ++i)
        s += (uint64_t)orc_mix32((uint32_t)i);
    return s;
}

/* ReduceCL over one fp32 partition: fp64 sum, fp32 min and max of map(x).
 * map = 0: identity, map = 2: poly3 with coef[3].  (Sec. 3.1.3 item 3.) */
void orc_reduce_f32(const float *in, uint64_t n, int map, const float coef[3],
                    double *sum, float *mn, float *mx)
{
    double s = 0.0;
    float lo = INFINITY, hi = -INFINITY;
    for (uint64_t i = 0; i < n; ++i) {
        float y = map ? orc_poly3(in[i], coef[0], coef[1], coef[2]) : in[i];
        s += (double)y;
        if (y == y) {             /* NaN never becomes the min or the max */
            if (y < lo) lo = y;
            if (y > hi) hi = y;
        }
    }
    *sum = s;
    *mn = lo;
    *mx = hi;
}

/* Keyed reduce of (key, value) pairs into count[num_keys] and an fp64
 * sum[num_keys] (the reduce-by-key of the WordCount demo, Sec. 3.2.3).
 * Outputs are overwritten.  Pairs whose key lies outside [0, num_keys) are
 * skipped; the return value is how many were skipped. */
uint64_t orc_keyed_count_sum(const int32_t *keys, const float *vals, uint64_t n,
                             uint32_t num_keys, uint32_t *count, double *sum)
{
    uint64_t bad = 0;
    memset(count, 0, sizeof(uint32_t) * num_keys);
    for (uint32_t k = 0; k < num_keys; ++k)
        sum[k] = 0.0;
    for (uint64_t i = 0; i < n; ++i) {
        int32_t k = keys[i];
        if (k < 0 || (uint32_t)k >= num_keys) {
            ++bad;
            continue;
        }
        count[k] += 1u;
        sum[k] += (double)vals[i];
    }
    return bad;
}

/* Keyed reduce with hashed keys: bucket = (mix32(key) * num_keys) >> 32,
 * computed in 64-bit, so every 32-bit key lands in [0, num_keys).  Outputs
 * are overwritten; num_keys >= 1. */
void orc_keyed_hashed_count_sum(const int32_t *keys, const float *vals, uint64_t n,
                                uint32_t num_keys, uint32_t *count, double *sum)
{
    memset(count, 0, sizeof(uint32_t) * num_keys);
    for (uint32_t k = 0; k < num_keys; ++k)
        sum[k] = 0.0;
    for (uint64_t i = 0; i < n; ++i) {
        uint32_t h = orc_mix32((uint32_t)keys[i]);
        uint32_t b = (uint32_t)(((uint64_t)h * num_keys) >> 32);
        count[b] += 1u;
        sum[b] += (double)vals[i];
    }
}

/* --------------------------------------- ReduceCL over partition arrays */

/* One output element of the tree reduce of k fp32 values x[0..k-1] (fp32
 * adds in the binary-counter tree order described at the top).  The stack
 * holds one subtree per set bit of the number of leaves seen so far, the
 * oldest (largest) at the bottom. */
static float tree_sum_f32(const float *x, uint32_t k)
{
    float stack[64];
    uint32_t size[64];
    uint32_t top = 0;
    for (uint32_t j = 0; j < k; ++j) {
        stack[top] = x[j];
        size[top] = 1;
        ++top;
        while (top >= 2 && size[top - 2] == size[top - 1]) {
            stack[top - 2] = stack[top - 2] + stack[top - 1];   /* older + newer */
            size[top - 2] += size[top - 1];
            --top;
        }
    }
    if (top == 0)
        return 0.0f;
    float acc = stack[top - 1];
    for (uint32_t i = top - 1; i-- > 0;)
        acc = stack[i] + acc;                                    /* older on the left */
    return acc;
}

/* ReduceCL of k fp32 partition arrays of n elements each (Sec. 3.2.2 with the
 * Fig. 3 kernel): out[i] = tree sum over j of arrays[j][i].  k >= 1. */
void orc_add_arrays_f32(const float *const *arrays, uint32_t k, uint64_t n, float *out)
{
    float col[4096];
    for (uint64_t i = 0; i < n; ++i) {
        for (uint32_t j = 0; j < k; ++j)
            col[j] = arrays[j][i];
        out[i] = tree_sum_f32(col, k);
    }
}

/* The same for uint32 arrays: wrapping addition mod 2^32 (order-free). */
void orc_add_arrays_u32(const uint32_t *const *arrays, uint32_t k, uint64_t n, uint32_t *out)
{
    for (uint64_t i = 0; i < n; ++i) {
        uint32_t s = 0;
        for (uint32_t j = 0; j < k; ++j)
            s += arrays[j][i];
        out[i] = s;
    }
}

/* ---------------------------------------------- combine across partitions */

/* ReduceCL's tree combine of per-partition results, written as the plain
 * left fold it must agree with (Sec. 3.1.3 item 3, Sec. 3.2.2): sums add,
 * min of mins, max of maxes. */
void orc_combine(const uint64_t *u64_sums, const double *f64_sums,
                 const float *mins, const float *maxs, uint32_t k,
                 uint64_t *u64_out, double *f64_out, float *min_out,
                 float *max_out)
{
    uint64_t us = 0;
    double fs = 0.0;
    float lo = INFINITY, hi = -INFINITY;
    for (uint32_t i = 0; i < k; ++i) {
        us += u64_sums[i];
        fs += f64_sums[i];
        if (mins[i] == mins[i] && mins[i] < lo) lo = mins[i];
        if (maxs[i] == maxs[i] && maxs[i] > hi) hi = maxs[i];
    }
    *u64_out = us;
    *f64_out = fs;
    *min_out = lo;
    *max_out = hi;
}

/* Merge k per-partition keyed tables (row-major [k][num_keys]) into one. */
void orc_combine_keyed(const uint32_t *counts, const double *sums, uint32_t k,
                       uint32_t num_keys, uint32_t *count_out, double *sum_out)
{
    for (uint32_t j = 0; j < num_keys; ++j) {
        uint32_t c = 0;
        double s = 0.0;
        for (uint32_t i = 0; i < k; ++i) {
            c += counts[(uint64_t)i * num_keys + j];
            s += sums[(uint64_t)i * num_keys + j];
        }
        count_out[j] = c;
        sum_out[j] = s;
    }
}
