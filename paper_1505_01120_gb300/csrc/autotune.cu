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
#include <cmath>
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
        // the best of three rounds of `reps` back-to-back launches
        double best = 1e30;
        for (int round = 0; round < 3 && st_ok == SCL_OK; ++round) {
            cudaEventRecord(e0, st);
            for (uint32_t r = 0; r < reps && st_ok == SCL_OK; ++r)
                st_ok = launch_plan(c, p, args, st);
            cudaEventRecord(e1, st);
            if (cudaEventSynchronize(e1) != cudaSuccess) {
                st_ok = fail(SCL_E_CUDA, "autotune: probe launch failed");
                break;
            }
            float t = 0.f;
            cudaEventElapsedTime(&t, e0, e1);
            best = std::min(best, (double)t / reps);
        }
        if (st_ok != SCL_OK) break;
        *ms = best;
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

// Deterministic log-normal partition sizes (median `med`, sigma 1.5, clipped
// to [256, 64 * med]) summing to at most `total`: the shape of a batch of
// uneven partitions.  splitmix64 + Box-Muller, so every run probes the same.
static std::vector<uint64_t> lognormal_probe_sizes(uint64_t total, uint64_t med) {
    std::vector<uint64_t> out;
    uint64_t x = 0x5eedull, used = 0;
    auto next = [&]() {
        uint64_t z = (x += 0x9e3779b97f4a7c15ull);
        z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
        z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
        return ((z ^ (z >> 31)) >> 11) * (1.0 / 9007199254740992.0);
    };
    while (out.size() < 16384) {
        const double u1 = std::max(next(), 1e-12), u2 = next();
        const double g = std::sqrt(-2.0 * std::log(u1)) * std::cos(6.283185307179586 * u2);
        uint64_t n = (uint64_t)std::floor(std::exp(std::log((double)med) + 1.5 * g));
        n = std::min<uint64_t>(std::max<uint64_t>(n, 256), 64 * med);
        n = (n + 63) / 64 * 64;   // keep every partition 256-byte aligned
        if (used + n > total) break;
        out.push_back(n);
        used += n;
    }
    return out;
}

int autotune(Ctx* c, const scl_autotune_config* cfg, cudaStream_t st, scl_autotune_report* rep) {
    uint64_t probe = cfg && cfg->probe_bytes ? cfg->probe_bytes : (512ull << 20);
    const uint32_t reps = cfg && cfg->reps ? cfg->reps : 10;
    const uint32_t fams = cfg && cfg->families ? cfg->families : 0xfu;
    // four regions (u32, f32, keys, values) of 2 * probe bytes each: a large
    // probe and a log-normal many-partition probe, each reading `probe` bytes
    const uint64_t room = c->arena.largest_free();
    while (probe > (16ull << 20) && 8 * probe + (64ull << 20) > room) probe /= 2;
    const uint64_t P = probe / 4;                 // elements per probe
    const uint64_t n = 2 * P;                     // elements per region
    const uint64_t region = align_up(n * 4);
    char* buf = (char*)c->arena.alloc(4 * region);
    const uint32_t ntables = 64;                  // keyed output tables, shared round-robin
    uint32_t* kout = (uint32_t*)c->arena.alloc((size_t)ntables * kKeyedTableWords * 4);
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

    std::vector<scl_part> reg;
    std::vector<scl_task> big[M_NUM], small[M_NUM];
    uint32_t kt = 0;
    auto table = [&]() { return kout + (size_t)(kt++ % ntables) * kKeyedTableWords; };
    auto add_set = [&](std::vector<scl_task>* dst, uint64_t off, uint64_t len) {
        scl_part pu = add_part(c, SCL_U32, U + off, nullptr, len);
        scl_part pf = add_part(c, SCL_F32, F + off, nullptr, len);
        scl_part pk = add_part(c, SCL_KV_I32_F32, K + off / 2, V + off / 2, len / 2);
        reg.insert(reg.end(), {pu, pf, pk});
        dst[M_U32].push_back(make_task(pu, SCL_K_MIX32, SCL_R_SUM, nullptr, nullptr));
        dst[M_F32].push_back(make_task(pf, SCL_K_POLY3, SCL_R_SUM_MIN_MAX, nullptr, nullptr));
        uint32_t* tb = table();
        dst[M_KEYED].push_back(make_task(pk, SCL_K_IDENT, SCL_R_KEYED_COUNT_SUM, tb,
                                         (float*)(tb + kMaxKeys)));
    };
    // large probe: 4 partitions of P/4 elements (P/8 pairs for keyed)
    for (int b = 0; b < 4; ++b) add_set(big, b * (P / 4), P / 4);
    // many-partition probe: log-normal sizes, median 16 Ki (scaled down for
    // small probes), the uneven-batch workload
    const uint64_t med = std::min<uint64_t>(16384, std::max<uint64_t>(1024, P / 2048));
    uint64_t off = P;
    for (uint64_t len : lognormal_probe_sizes(P, med)) {
        add_set(small, off, len);
        off += len;
    }
    // mixed batches: a third of each kind
    for (int m = 0; m < 3; ++m) {
        big[M_ALL].push_back(big[m][0]);
        for (size_t i = m; i < small[m].size(); i += 3) small[M_ALL].push_back(small[m][i]);
    }

    if (rep) memset(rep, 0, sizeof *rep);
    // fp32 first: mixed batches inherit its block and items per thread, so its
    // candidates are also scored on the mixed many-partition probe
    const int order[M_NUM] = {M_F32, M_U32, M_KEYED, M_ALL};
    for (int oi = 0; oi < M_NUM && status == SCL_OK; ++oi) {
        const int fam = order[oi];
        if (!(fams & (1u << fam))) continue;
        const Shape keep = c->shape[fam];
        const std::vector<Shape> cand = candidates(fam, c->shape[M_F32]);
        std::vector<std::vector<double>> t(cand.size());   // per candidate, per probe
        for (size_t ci = 0; ci < cand.size() && status == SCL_OK; ++ci) {
            c->shape[fam] = cand[ci];
            double tb = 0, ts = 0, tm = 0;
            int r = time_tasks(c, big[fam], st, reps, &tb);
            if (r == SCL_OK) r = time_tasks(c, small[fam], st, reps, &ts);
            if (r == SCL_OK && fam == M_F32) r = time_tasks(c, small[M_ALL], st, reps, &tm);
            if (r == SCL_E_TIMEOUT || r == SCL_E_CUDA) {
                status = r;
                break;
            }
            if (r != SCL_OK) continue;
            t[ci] = fam == M_F32 ? std::vector<double>{tb, ts, tm} : std::vector<double>{tb, ts};
        }
        // objective: sum over probes of time / the best time on that probe.
        // The keyed family's shape serves single keyed reduces and keyed-only
        // batches, mostly large partitions (mixed batches take the fp32
        // family's), so its large probe counts four times.
        const double wbig = fam == M_KEYED ? 4.0 : 1.0;
        size_t best = cand.size();
        double best_score = 1e30, best_ms = 0;
        uint32_t tried = 0;
        if (status == SCL_OK) {
            std::vector<double> lo(3, 1e30);
            for (auto& v : t)
                for (size_t k = 0; k < v.size(); ++k) lo[k] = std::min(lo[k], v[k]);
            for (size_t ci = 0; ci < cand.size(); ++ci) {
                if (t[ci].empty()) continue;
                ++tried;
                double score = 0, ms = 0;
                for (size_t k = 0; k < t[ci].size(); ++k) {
                    score += (k == 0 ? wbig : 1.0) * t[ci][k] / lo[k];
                    ms += t[ci][k];
                }
                if (score < best_score) {
                    best_score = score;
                    best = ci;
                    best_ms = ms;
                }
            }
        }
        c->shape[fam] = (status == SCL_OK && best < cand.size()) ? cand[best] : keep;
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
