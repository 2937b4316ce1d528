// Autotuner: times one job under every launch configuration and keeps the
// fastest, optionally caching the choice per workload key in a JSON file.
// Host code only; it drives the library through its own C ABI.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <cstring>
#include <fstream>
#include <map>
#include <sstream>
#include <string>
#include <vector>

#include "trees.h"

namespace {

struct CacheEntry {
    int bs = 0, tpt = 0, sched = 0;
    double ms = 0.0;
};

// The cache is one JSON object: {"key": {"block_size": B, "tasks_per_thread": T,
// "scheduler": S, "ms": M}, ...}.  Keys are written without quotes or
// backslashes inside them.
std::map<std::string, CacheEntry> read_cache(const char *path) {
    std::map<std::string, CacheEntry> out;
    std::ifstream f(path);
    if (!f) return out;
    std::stringstream ss;
    ss << f.rdbuf();
    const std::string s = ss.str();
    size_t pos = 0;
    while (true) {
        const size_t k0 = s.find('"', pos);
        if (k0 == std::string::npos) break;
        const size_t k1 = s.find('"', k0 + 1);
        if (k1 == std::string::npos) break;
        const size_t o0 = s.find('{', k1);
        const size_t o1 = s.find('}', o0 == std::string::npos ? k1 : o0);
        if (o0 == std::string::npos || o1 == std::string::npos) break;
        const std::string key = s.substr(k0 + 1, k1 - k0 - 1);
        const std::string body = s.substr(o0, o1 - o0);
        auto num = [&](const char *name) -> double {
            const size_t p = body.find(std::string("\"") + name + "\"");
            if (p == std::string::npos) return -1.0;
            const size_t c = body.find(':', p);
            return c == std::string::npos ? -1.0 : std::atof(body.c_str() + c + 1);
        };
        CacheEntry e;
        e.bs = (int)num("block_size");
        e.tpt = (int)num("tasks_per_thread");
        e.sched = (int)num("scheduler");
        e.ms = num("ms");
        if (e.bs > 0 && e.tpt > 0 && e.sched >= 0) out[key] = e;
        pos = o1 + 1;
    }
    return out;
}

void write_cache(const char *path, const std::map<std::string, CacheEntry> &m) {
    std::ofstream f(path);
    f << "{\n";
    size_t i = 0;
    for (const auto &kv : m) {
        f << "  \"" << kv.first << "\": {\"block_size\": " << kv.second.bs
          << ", \"tasks_per_thread\": " << kv.second.tpt << ", \"scheduler\": " << kv.second.sched
          << ", \"ms\": " << kv.second.ms << "}" << (++i < m.size() ? ",\n" : "\n");
    }
    f << "}\n";
}

bool key_ok(const char *key) {
    for (const char *p = key; *p; ++p)
        if (*p == '"' || *p == '\\' || *p == '{' || *p == '}') return false;
    return true;
}

}  // namespace

extern "C" int trees_autotune(const trees_job_t *job, size_t capacity_slots, const trees_config_t *base, int32_t reps,
                              const char *cache_path, const char *key, trees_config_t *best, double *best_ms,
                              trees_tune_entry_t *table, int32_t table_cap, int32_t *table_n) {
    if (!job || !best || !best_ms || reps < 1 || (key && !key_ok(key))) return TREES_ERR_INVALID_ARG;
    trees_config_t b0;
    if (base) b0 = *base;
    else trees_default_config(&b0);
    if (table_n) *table_n = 0;
    std::map<std::string, CacheEntry> cache;
    if (cache_path && key) {
        cache = read_cache(cache_path);
        auto it = cache.find(key);
        if (it != cache.end()) {
            *best = b0;
            best->block_size = it->second.bs;
            best->tasks_per_thread = it->second.tpt;
            best->scheduler = it->second.sched;
            *best_ms = it->second.ms;
            return TREES_OK;
        }
    }
    // a mergesort job sorts its keys in place: keep a copy to restore them
    uint32_t *backup = nullptr;
    const size_t nkeys = job->program == TREES_PROG_MERGESORT ? job->n : 0;
    if (nkeys) {
        if (cudaMalloc(&backup, nkeys * 4) != cudaSuccess) return TREES_ERR_CUDA;
        if (cudaMemcpy(backup, job->keys, nkeys * 4, cudaMemcpyDeviceToDevice) != cudaSuccess) {
            cudaFree(backup);
            return TREES_ERR_CUDA;
        }
    }
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    const int bss[4] = {128, 256, 512, 1024}, tpts[3] = {1, 2, 4};
    const int scheds[2] = {TREES_SCHED_PERSISTENT, TREES_SCHED_GRAPH};
    double bestv = -1.0;
    int first_err = TREES_OK, n = 0;
    for (int si = 0; si < 2; ++si)
        for (int bi = 0; bi < 4; ++bi)
            for (int ti = 0; ti < 3; ++ti) {
                trees_config_t cfg = b0;
                cfg.block_size = bss[bi];
                cfg.tasks_per_thread = tpts[ti];
                cfg.scheduler = scheds[si];
                cfg.trace = 0;
                trees_ctx *ctx = nullptr;
                int rc = trees_create(capacity_slots, &cfg, &ctx);
                double ms = -1.0;
                for (int r = 0; rc == TREES_OK && r <= reps; ++r) {
                    if (nkeys && cudaMemcpy(job->keys, backup, nkeys * 4, cudaMemcpyDeviceToDevice) != cudaSuccess) {
                        rc = TREES_ERR_CUDA;
                        break;
                    }
                    cudaEventRecord(e0, 0);
                    rc = trees_run(ctx, job, nullptr);
                    cudaEventRecord(e1, 0);
                    if (rc == TREES_OK) rc = trees_sync(ctx);
                    cudaEventSynchronize(e1);
                    float t = 0.f;
                    cudaEventElapsedTime(&t, e0, e1);
                    if (rc == TREES_OK && r > 0 && (ms < 0 || t < ms)) ms = t;
                }
                if (ctx) trees_destroy(ctx);
                if (table && n < table_cap) {
                    table[n].cfg = cfg;
                    table[n].ms = ms;
                    table[n].status = rc;
                    table[n].pad = 0;
                }
                ++n;
                if (rc != TREES_OK) {
                    if (first_err == TREES_OK) first_err = rc;
                    continue;
                }
                if (bestv < 0 || ms < bestv) {
                    bestv = ms;
                    *best = cfg;
                }
            }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (nkeys) {
        cudaMemcpy(job->keys, backup, nkeys * 4, cudaMemcpyDeviceToDevice);
        cudaFree(backup);
    }
    if (table_n) *table_n = std::min(n, table_cap);
    if (bestv < 0) return first_err == TREES_OK ? TREES_ERR_CUDA : first_err;
    *best_ms = bestv;
    if (cache_path && key) {
        CacheEntry e;
        e.bs = best->block_size;
        e.tpt = best->tasks_per_thread;
        e.sched = best->scheduler;
        e.ms = bestv;
        cache[key] = e;
        write_cache(cache_path, cache);
    }
    return TREES_OK;
}
