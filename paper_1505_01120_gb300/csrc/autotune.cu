// autotune.cu -- launch-shape autotuner (block size, items per thread, CTAs
// per SM, load path, TMA ring depth) for each kernel family.
//
// For each family the tuner builds two probe batches in the arena -- a few
// large partitions (memory-bound steady state) and many 16 Ki-element
// partitions (per-segment and per-task overheads) -- fills them on the device,
// and times every compiled candidate with CUDA events over repeated launches.
// The objective is the sum of the two batch times.  The fp32 family is tuned
// first because mixed batches inherit its (block, items per thread): an fp32
// partition gives the same bits alone and inside a mixed batch.
#include <string.h>

#include <algorithm>
#include <vector>

#include "runtime.h"

namespace scl {

namespace {

__global__ void k_fill_probe(uint32_t* u, float* f, int32_t* keys, float* vals, uint64_t n) {
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n;
         i += (uint64_t)gridDim.x * blockDim.x) {
        uint32_t h = (uint32_t)i * 2654435761u + 0x9e3779b9u;
        h ^= h >> 13;
        h *= 0x5bd1e995u;
        h ^= h >> 15;
        u[i] = h;
        f[i] = ((float)(h & 0xffffu) * (1.0f / 65536.0f) - 0.5f) * 6.0f;
        keys[i] = (int32_t)(h % kMaxKeys);
        vals[i] = 0.5f;
    }
}

struct Probe {
    std::vector<scl_part> parts;
    std::vector<scl_task> big, small;
};

scl_part add_part(Ctx* c, scl_dtype dt, void* d0, void* d1, uint64_t n) {
    const scl_part h = c->next_part++;
    c->parts[h] = Partition{dt, n, d0, d1, nullptr};
    return h;
}

scl_task make_task(scl_part p, int kernel, int reduce, uint32_t* cnt, float* sums) {
    scl_task t;
    memset(&t, 0, sizeof t);
    t.part = p;
    t.kernel = kernel;
    t.reduce = reduce;
    t.num_keys = cnt ? kMaxKeys : 0;
    t.coef[0] = 0.5f;
    t.coef[1] = -1.25f;
    t.coef[2] = 0.1f;
    t.counts_out = cnt;
    t.sums_out = sums;
    return t;
}

// Mean ms per launch of `tasks` planned with the context's current shapes.
int time_tasks(Ctx* c, const std::vector<scl_task>& tasks, cudaStream_t st, uint32_t reps,
               double* ms) {
    Plan p;
    SCL_TRY(plan_tasks(c, tasks.data(), (uint32_t)tasks.size(), &p));
    PlanImage img;
    std::vector<char> host;
    KernelArgs args;
    SCL_TRY(build_image(c, p, &img, &host, &args));
    int st_ok = SCL_OK;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    do {
        if (cudaMemcpy(img.block, host.data(), img.plan_bytes, cudaMemcpyHostToDevice) !=
                cudaSuccess ||
            cudaMemset((char*)img.block + img.zero_off, 0, img.zero_bytes) != cudaSuccess ||
            cudaDeviceSynchronize() != cudaSuccess) {
            st_ok = fail(SCL_E_CUDA, "autotune: probe upload failed");
            break;
        }
        for (int w = 0; w < 2 && st_ok == SCL_OK; ++w) st_ok = launch_plan(c, p, args, st);
        if (st_ok != SCL_OK) break;
        if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
            st_ok = fail(SCL_E_CUDA, "autotune: event create failed");
            break;
        }
        cudaEventRecord(e0, st);
        for (uint32_t r = 0; r < reps && st_ok == SCL_OK; ++r) st_ok = launch_plan(c, p, args, st);
        cudaEventRecord(e1, st);
        if (cudaEventSynchronize(e1) != cudaSuccess) {
            st_ok = fail(SCL_E_CUDA, "autotune: probe launch failed");
            break;
        }
        float t = 0.f;
        cudaEventElapsedTime(&t, e0, e1);
        *ms = t / reps;
        uint32_t err = 0;
        cudaMemcpy(&err, img.hdr + H_ERROR, 4, cudaMemcpyDeviceToHost);
        if (err) st_ok = fail(SCL_E_TIMEOUT, "autotune: device error word 0x%x", err);
    } while (0);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    c->arena.release(img.block);
    return st_ok;
}

std::vector<Shape> candidates(int family, const Shape& f32) {
    static const int kLdg[][2] = {{256, 2}, {256, 4}, {256, 8}, {512, 2}, {512, 4}, {512, 8}};
    static const int kTma[][3] = {{256, 2, 12}, {256, 4, 6}, {256, 4, 4},
                                  {256, 8, 3},  {512, 2, 6}, {512, 4, 3}};
    std::vector<Shape> out;
    if (family == M_ALL) {
        for (int cps : {0, 4, 2}) out.push_back(Shape{f32.block, f32.ipt, cps, PATH_LDG, 0});
        return out;
    }
    for (auto& s : kLdg)
        for (int cps : {0, 4, 3})
            if (find_entry(family, s[0], s[1])) out.push_back(Shape{s[0], s[1], cps, PATH_LDG, 0});
    if (family == M_U32 || family == M_F32)
        for (auto& s : kTma)
            if (find_entry(family, s[0], s[1], PATH_TMA, s[2]))
                out.push_back(Shape{s[0], s[1], 0, PATH_TMA, s[2]});
    return out;
}

}  // namespace

int autotune(Ctx* c, const scl_autotune_config* cfg, cudaStream_t st, scl_autotune_report* rep) {
    uint64_t probe = cfg && cfg->probe_bytes ? cfg->probe_bytes : (256ull << 20);
    const uint32_t reps = cfg && cfg->reps ? cfg->reps : 10;
    const uint32_t fams = cfg && cfg->families ? cfg->families : 0xfu;
    const uint64_t small_n = 16384, small_parts = 512;
    // room: u32 + f32 + keys + vals regions, plus keyed output tables
    const uint64_t room = c->arena.largest_free();
    while (probe > (16ull << 20) && 4 * (probe + small_n * small_parts * 4) + (64ull << 20) > room)
        probe /= 2;
    const uint64_t nbig = probe / 4;                     // elements of the big region
    const uint64_t n = nbig + small_n * small_parts;     // elements per region
    const uint64_t region = align_up(n * 4);
    char* buf = (char*)c->arena.alloc(4 * region);
    const uint32_t nkeyed_out = 8 + (uint32_t)small_parts;
    uint32_t* kout = (uint32_t*)c->arena.alloc((size_t)nkeyed_out * kKeyedTableWords * 4);
    if (!buf || !kout) {
        c->arena.release(buf);
        c->arena.release(kout);
        return fail(SCL_E_NOMEM, "autotune: arena too small for the probe");
    }
    uint32_t* U = (uint32_t*)buf;
    float* F = (float*)(buf + region);
    int32_t* K = (int32_t*)(buf + 2 * region);
    float* V = (float*)(buf + 3 * region);
    k_fill_probe<<<c->sms * 8, 256, 0, st>>>(U, F, K, V, n);
    int status = cudaStreamSynchronize(st) == cudaSuccess
                     ? SCL_OK
                     : fail(SCL_E_CUDA, "autotune: probe fill failed");

    // probe batches per family: 4 big partitions + small_parts small ones
    std::vector<scl_part> reg;
    std::vector<scl_task> big[M_NUM], small[M_NUM];
    auto table = [&](uint32_t i) { return kout + (size_t)i * kKeyedTableWords; };
    uint32_t kt = 0;
    for (int b = 0; b < 4; ++b) {
        const uint64_t off = b * (nbig / 4), len = nbig / 4;
        scl_part pu = add_part(c, SCL_U32, U + off, nullptr, len);
        scl_part pf = add_part(c, SCL_F32, F + off, nullptr, len / 2 * 2);
        scl_part pk = add_part(c, SCL_KV_I32_F32, K + off / 2, V + off / 2, len / 2);
        reg.insert(reg.end(), {pu, pf, pk});
        big[M_U32].push_back(make_task(pu, SCL_K_MIX32, SCL_R_SUM, nullptr, nullptr));
        big[M_F32].push_back(make_task(pf, SCL_K_POLY3, SCL_R_SUM_MIN_MAX, nullptr, nullptr));
        uint32_t* tb = table(kt++);
        big[M_KEYED].push_back(make_task(pk, SCL_K_IDENT, SCL_R_KEYED_COUNT_SUM, tb,
                                         (float*)(tb + kMaxKeys)));
    }
    for (uint64_t s = 0; s < small_parts; ++s) {
        const uint64_t off = nbig + s * small_n;
        scl_part pu = add_part(c, SCL_U32, U + off, nullptr, small_n);
        scl_part pf = add_part(c, SCL_F32, F + off, nullptr, small_n);
        scl_part pk = add_part(c, SCL_KV_I32_F32, K + off, V + off, small_n);
        reg.insert(reg.end(), {pu, pf, pk});
        small[M_U32].push_back(make_task(pu, SCL_K_MIX32, SCL_R_SUM, nullptr, nullptr));
        small[M_F32].push_back(make_task(pf, SCL_K_POLY3, SCL_R_SUM_MIN_MAX, nullptr, nullptr));
        uint32_t* tb = table(kt++ % nkeyed_out);
        small[M_KEYED].push_back(make_task(pk, SCL_K_IDENT, SCL_R_KEYED_COUNT_SUM, tb,
                                           (float*)(tb + kMaxKeys)));
    }
    // mixed: a third of each
    for (int m = 0; m < 3; ++m) {
        big[M_ALL].push_back(big[m][0]);
        for (uint64_t s = m; s < small_parts; s += 3) small[M_ALL].push_back(small[m][s]);
    }

    if (rep) memset(rep, 0, sizeof *rep);
    const int order[M_NUM] = {M_F32, M_U32, M_KEYED, M_ALL};
    for (int oi = 0; oi < M_NUM && status == SCL_OK; ++oi) {
        const int fam = order[oi];
        if (!(fams & (1u << fam))) continue;
        const Shape keep = c->shape[fam];
        Shape best = keep;
        double best_ms = 1e30;
        uint32_t tried = 0;
        for (const Shape& s : candidates(fam, c->shape[M_F32])) {
            c->shape[fam] = s;
            double t_big = 0, t_small = 0;
            int r = time_tasks(c, big[fam], st, reps, &t_big);
            if (r == SCL_OK) r = time_tasks(c, small[fam], st, reps, &t_small);
            if (r == SCL_E_TIMEOUT || r == SCL_E_CUDA) {
                status = r;
                break;
            }
            if (r != SCL_OK) continue;
            ++tried;
            if (t_big + t_small < best_ms) {
                best_ms = t_big + t_small;
                best = s;
            }
        }
        c->shape[fam] = status == SCL_OK ? best : keep;
        if (rep) {
            const Shape sh = c->shape_for(fam);
            const KernelEntry* e = find_entry(fam, sh);
            rep->chosen[fam] = scl_shape{sh.block, sh.ipt, sh.ctas_per_sm, sh.path,
                                         e ? e->stages : 0, 0};
            rep->best_ms[fam] = best_ms;
            rep->candidates[fam] = tried;
        }
    }
    for (scl_part p : reg) c->parts.erase(p);
    cudaDeviceSynchronize();
    c->arena.release(buf);
    c->arena.release(kout);
    c->occ_cache.clear();
    if (status == SCL_OK && !c->tune_path.empty()) status = save_tuning(c, c->tune_path.c_str());
    return status;
}

}  // namespace scl
