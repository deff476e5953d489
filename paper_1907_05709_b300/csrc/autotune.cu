// autotune.cu -- picks the steps-per-launch depth and tile variant of the
// forward step for one grid by timing every supported candidate on a
// snapshot of the grid's own state (restored afterwards), and remembers the
// choice in an optional JSON cache keyed by shape, precision and damage mode.
#include "rfa_internal.cuh"

#include <cstdio>
#include <fstream>
#include <map>
#include <sstream>
#include <utility>
#include <vector>

namespace rfa {

namespace {

std::string tune_key(const rfa_grid *g)
{
    char buf[96];
    std::snprintf(buf, sizeof buf, "%dx%dx%d/s%d/p%d/d%d", g->nx, g->ny, g->nz, g->sp, g->pp, g->dmg);
    return buf;
}

// cache file: {"<key>": [depth, variant], ...}
std::map<std::string, std::pair<int, int>> cache_read(const char *path)
{
    std::map<std::string, std::pair<int, int>> m;
    if (!path) return m;
    std::ifstream f(path);
    if (!f) return m;
    std::stringstream ss;
    ss << f.rdbuf();
    std::string s = ss.str();
    size_t pos = 0;
    while ((pos = s.find('"', pos)) != std::string::npos) {
        size_t end = s.find('"', pos + 1);
        if (end == std::string::npos) break;
        std::string key = s.substr(pos + 1, end - pos - 1);
        size_t lb = s.find('[', end), rb = s.find(']', end);
        if (lb == std::string::npos || rb == std::string::npos) break;
        int d = 0, v = 0;
        if (std::sscanf(s.c_str() + lb + 1, "%d , %d", &d, &v) == 2) m[key] = {d, v};
        pos = rb + 1;
    }
    return m;
}

void cache_write(const char *path, const std::map<std::string, std::pair<int, int>> &m)
{
    if (!path) return;
    std::ofstream f(path, std::ios::trunc);
    if (!f) return;
    f << "{";
    bool first = true;
    for (auto &kv : m) {
        f << (first ? "\n  " : ",\n  ") << '"' << kv.first << "\": [" << kv.second.first << ", "
          << kv.second.second << "]";
        first = false;
    }
    f << "\n}\n";
}

struct Snapshot {
    void *th = nullptr, *lo = nullptr, *om = nullptr, *oc = nullptr;
    uint8_t *latch = nullptr;
    int cur = 0;
    int64_t steps = 0;
    void release()
    {
        for (void *p : {th, lo, om, oc, (void *)latch})
            if (p) cudaFree(p);
        th = lo = om = oc = nullptr;
        latch = nullptr;
    }
};

cudaError_t snap_take(rfa_grid *g, Snapshot &s)
{
    size_t nvp = g->nvp;
    cudaError_t e = cudaMalloc(&s.th, nvp * g->state_elem());
    if (e == cudaSuccess && g->sp == RFA_STATE_F32C) e = cudaMalloc(&s.lo, nvp * 4);
    if (e == cudaSuccess) e = cudaMalloc(&s.om, nvp * 8);
    if (e == cudaSuccess) e = cudaMalloc(&s.oc, nvp * 4);
    if (e == cudaSuccess) e = cudaMalloc((void **)&s.latch, nvp);
    if (e != cudaSuccess) return e;
    s.cur = g->cur;
    s.steps = g->steps;
    cudaMemcpyAsync(s.th, g->th[g->cur], nvp * g->state_elem(), cudaMemcpyDeviceToDevice, g->stream);
    if (s.lo) cudaMemcpyAsync(s.lo, g->lo[g->cur], nvp * 4, cudaMemcpyDeviceToDevice, g->stream);
    cudaMemcpyAsync(s.om, g->omega, nvp * 8, cudaMemcpyDeviceToDevice, g->stream);
    cudaMemcpyAsync(s.oc, g->omega_c, nvp * 4, cudaMemcpyDeviceToDevice, g->stream);
    return cudaMemcpyAsync(s.latch, g->latch, nvp, cudaMemcpyDeviceToDevice, g->stream);
}

cudaError_t snap_restore(rfa_grid *g, const Snapshot &s)
{
    size_t nvp = g->nvp;
    g->cur = s.cur;
    g->steps = s.steps;
    cudaMemcpyAsync(g->th[g->cur], s.th, nvp * g->state_elem(), cudaMemcpyDeviceToDevice, g->stream);
    if (s.lo) cudaMemcpyAsync(g->lo[g->cur], s.lo, nvp * 4, cudaMemcpyDeviceToDevice, g->stream);
    cudaMemcpyAsync(g->omega, s.om, nvp * 8, cudaMemcpyDeviceToDevice, g->stream);
    cudaMemcpyAsync(g->omega_c, s.oc, nvp * 4, cudaMemcpyDeviceToDevice, g->stream);
    return cudaMemcpyAsync(g->latch, s.latch, nvp, cudaMemcpyDeviceToDevice, g->stream);
}

}  // namespace

}  // namespace rfa

using namespace rfa;

extern "C" rfa_status rfa_autotune(rfa_grid *g, const char *cache_path)
{
    if (!g) {
        set_error("null grid");
        return RFA_E_INVALID;
    }
    if (!g->have_tissue) {
        set_error("rfa_set_tissue must come first");
        return RFA_E_STATE;
    }
    const std::string key = tune_key(g);
    auto cache = cache_read(cache_path);
    auto hit = cache.find(key);
    if (hit != cache.end()) {
        int d = hit->second.first, v = hit->second.second;
        if (d == 1 || tb_supported(g, d, v)) {
            g->sched.tb_depth = d;
            g->sched.tile_variant = v;
            return RFA_OK;
        }
    }
    std::vector<std::pair<int, int>> cands = {{1, 0}};
    for (int v = 0; v <= 1; ++v)
        for (int d = 2; d <= 8; ++d)
            if (tb_supported(g, d, v)) cands.push_back({d, v});
    if (cands.size() == 1) {
        g->sched = Schedule{};
        cache[key] = {1, 0};
        cache_write(cache_path, cache);
        return RFA_OK;
    }
    Snapshot snap;
    cudaError_t e = snap_take(g, snap);
    if (e != cudaSuccess) {
        snap.release();
        cudaGetLastError();
        set_error("autotune snapshot allocation failed");
        return RFA_E_OOM;
    }
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    const Schedule saved = g->sched;
    const bool dmg = g->dmg != 0;
    // 24 steps is a whole number of blocks for every depth (2 or 3)
    const int64_t nwarm = 12, ntime = 24;
    float best = 1e30f;
    Schedule pick = saved;
    rfa_status st = RFA_OK;
    for (auto &c : cands) {
        g->sched.tb_depth = c.first;
        g->sched.tile_variant = c.second;
        st = advance(g, nwarm, dmg, true);
        if (st != RFA_OK) break;
        cudaEventRecord(e0, g->stream);
        st = advance(g, ntime, dmg, true);
        if (st != RFA_OK) break;
        cudaEventRecord(e1, g->stream);
        if ((e = cudaEventSynchronize(e1)) != cudaSuccess) {
            st = cuda_fail(e, "autotune timing");
            break;
        }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (ms < best) {
            best = ms;
            pick = g->sched;
        }
        snap_restore(g, snap);
    }
    snap_restore(g, snap);
    cudaStreamSynchronize(g->stream);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    snap.release();
    if (st != RFA_OK) {
        g->sched = saved;
        return st;
    }
    g->sched = pick;
    cache[key] = {pick.tb_depth, pick.tile_variant};
    cache_write(cache_path, cache);
    return RFA_OK;
}
