// batch.cu -- many needle configurations on grids of uneven size advanced in
// one persistent launch per call (the paper simulates one configuration; this
// batches independent ones for planning sweeps).
//
// Every member's (tile, z-chunk) work items are numbered consecutively; a
// cooperative grid of exactly the resident CTAs walks all items of all members
// for one block of M steps, meets at a bounded software grid barrier, and
// continues with the next block, so nsteps cost one launch.  The launch is
// built once per block count into a CUDA graph (barrier reset + cooperative
// kernel node) and replayed.  Steps that do
// not fill a block run as one-step launches per member afterwards.
#include "rfa_internal.cuh"

#include <algorithm>
#include <cstdio>
#include <fstream>
#include <new>
#include <map>
#include <sstream>
#include <vector>

struct rfa_batch {
    std::vector<rfa_grid *> members;
    cudaStream_t stream = nullptr;
    int depth = 2, variant = 0;
    bool damage = false;
    std::vector<rfa::TBMemberHost> hosts;
    std::vector<int> item_begin;
    std::vector<int> order;  // descriptor slot -> member (costliest items first)
    int nitems = 0;
    void *d_members = nullptr;
    CUtensorMap *d_maps = nullptr;
    unsigned *d_gbar = nullptr;
    void *h_members = nullptr;  // pinned staging of the member descriptors
    std::map<int64_t, cudaGraphExec_t> graphs;
    bool graphs_lim = false;  // the graphs hold the instantiation for shortened wait limits
    bool use_graphs = true;
    int grid = 0;             // co-resident CTAs of the batch kernel
    std::string graph_error;  // why graph capture was given up, if it was
};

namespace rfa {

constexpr int64_t kMaxBlocksPerLaunch = 4096;  // time blocks of one batched launch

namespace {

rfa_status bfail(rfa_status st, const std::string &m)
{
    set_error(m);
    return st;
}

void release_plan(rfa_batch *b)
{
    for (auto &kv : b->graphs) cudaGraphExecDestroy(kv.second);
    b->graphs.clear();
    if (b->d_members) cudaFree(b->d_members);
    if (b->d_maps) cudaFree(b->d_maps);
    if (b->h_members) cudaFreeHost(b->h_members);
    b->d_members = nullptr;
    b->d_maps = nullptr;
    b->h_members = nullptr;
}

// descriptors, tensor maps and work-item numbering for the current schedule
rfa_status build_plan(rfa_batch *b)
{
    release_plan(b);
    const int n = (int)b->members.size();
    b->hosts.assign(n, TBMemberHost{});
    b->item_begin.assign(n + 1, 0);
    for (int m = 0; m < n; ++m)
        if (!tb_batch_member(b->members[m], b->depth, b->variant, 96, b->hosts[m]))
            return bfail(RFA_E_CUDA, "tensor map creation failed for a batch member");
    // items are claimed in numbering order: number the costliest items (most
    // planes per z chunk) first, so that a time block ends on the cheapest ones
    b->order.resize(n);
    for (int m = 0; m < n; ++m) b->order[m] = m;
    auto cost = [&](int m) {
        const rfa_grid *g = b->members[m];
        const int zc = b->hosts[m].tile[0].zc;
        return (g->nz + zc - 1) / zc + 2 * b->depth;
    };
    std::stable_sort(b->order.begin(), b->order.end(), [&](int x, int y) { return cost(x) > cost(y); });
    // guided: the members numbered last (an eighth of them) get finer chunks, so a
    // time block ends on small items
    for (int j = n - n / 8; j < n; ++j)
        if (!tb_batch_member(b->members[b->order[j]], b->depth, b->variant, 32, b->hosts[b->order[j]]))
            return bfail(RFA_E_CUDA, "tensor map creation failed for a batch member");
    std::stable_sort(b->order.begin(), b->order.end(), [&](int x, int y) { return cost(x) > cost(y); });
    for (int j = 0; j < n; ++j) b->item_begin[j + 1] = b->item_begin[j] + b->hosts[b->order[j]].items;
    b->nitems = b->item_begin[n];
    const size_t mb = tb_member_bytes();
    if (cudaMalloc(&b->d_members, mb * n) != cudaSuccess ||
        cudaMalloc((void **)&b->d_maps, sizeof(CUtensorMap) * 8 * n) != cudaSuccess ||
        cudaMallocHost(&b->h_members, mb * n) != cudaSuccess) {
        cudaGetLastError();
        return bfail(RFA_E_OOM, "batch descriptor allocation failed");
    }
    std::vector<CUtensorMap> maps(8 * (size_t)n);
    for (int j = 0; j < n; ++j)
        for (int k = 0; k < 8; ++k) maps[8 * (size_t)j + k] = b->hosts[b->order[j]].maps[k];
    RFA_CUDA(cudaMemcpyAsync(b->d_maps, maps.data(), sizeof(CUtensorMap) * maps.size(), cudaMemcpyHostToDevice,
                             b->stream));
    RFA_CUDA(cudaStreamSynchronize(b->stream));
    RFA_CUDA(prepare_batch_tb(b->depth, b->variant, b->damage, b->nitems, &b->grid));
    return RFA_OK;
}

// upload descriptors with each member's current ping-pong parity
rfa_status upload_members(rfa_batch *b)
{
    const size_t mb = tb_member_bytes();
    for (size_t j = 0; j < b->members.size(); ++j) {
        const int m = b->order[j];
        tb_pack_member(b->hosts[m], b->d_maps + 8 * j, b->item_begin[j], b->members[m]->cur,
                       (char *)b->h_members + mb * j);
    }
    RFA_CUDA(cudaMemcpyAsync(b->d_members, b->h_members, mb * b->members.size(), cudaMemcpyHostToDevice,
                             b->stream));
    return RFA_OK;
}

cudaError_t enqueue_blocks(rfa_batch *b, int64_t ntime)
{
    // grid barrier (2 words) and the item counter of every time block
    cudaError_t e = cudaMemsetAsync(b->d_gbar, 0, (2 + (size_t)ntime) * sizeof(unsigned), b->stream);
    if (e != cudaSuccess) return e;
    return launch_batch_tb(b->depth, b->variant, b->damage, b->d_members, (int)b->members.size(), b->nitems,
                           (int)ntime, b->d_gbar, b->members[0]->status, b->stream, b->grid);
}

rfa_status run_blocks(rfa_batch *b, int64_t ntime)
{
    if (ntime <= 0) return RFA_OK;
    if (b->use_graphs && b->graphs_lim != tb_limits_set()) {  // wait limits changed: capture again
        for (auto &kv : b->graphs) cudaGraphExecDestroy(kv.second);
        b->graphs.clear();
        b->graphs_lim = tb_limits_set();
    }
    if (b->use_graphs) {
        auto it = b->graphs.find(ntime);
        if (it == b->graphs.end()) {
            cudaGraphExec_t exec = nullptr;
            cudaError_t e = graph_batch_tb(b->depth, b->variant, b->damage, b->d_members, (int)b->members.size(),
                                           b->nitems, (int)ntime, b->d_gbar, b->members[0]->status, b->grid, &exec);
            if (e != cudaSuccess) {
                // graphs unavailable for this launch kind: keep launching directly
                b->graph_error = cudaGetErrorString(e);
                cudaGetLastError();
                b->use_graphs = false;
            } else {
                it = b->graphs.emplace(ntime, exec).first;
            }
        }
        if (b->use_graphs) {
            RFA_CUDA(cudaGraphLaunch(it->second, b->stream));
            return RFA_OK;
        }
    }
    RFA_CUDA(enqueue_blocks(b, ntime));
    return RFA_OK;
}

rfa_status batch_step(rfa_batch *b, int64_t nsteps)
{
    const int64_t ntime = nsteps / b->depth, rem = nsteps % b->depth;
    // at most kMaxBlocksPerLaunch time blocks per launch (one item counter each)
    for (int64_t done = 0; done < ntime;) {
        const int64_t n = std::min<int64_t>(ntime - done, kMaxBlocksPerLaunch);
        rfa_status st = upload_members(b);
        if (st != RFA_OK) return st;
        st = run_blocks(b, n);
        if (st != RFA_OK) return st;
        for (rfa_grid *g : b->members) {
            g->cur ^= (int)(n & 1);
            if (b->damage) g->carry_steps = 0;  // the last block of a launch folds the carry
        }
        done += n;
    }
    for (rfa_grid *g : b->members) {
        if (rem > 0) {
            const int saved = g->sched.tb_depth;
            g->sched.tb_depth = 1;
            rfa_status st = advance(g, rem, b->damage, true);
            g->sched.tb_depth = saved;
            if (st != RFA_OK) return st;
        }
        g->steps += nsteps;
        g->rec.valid = false;
    }
    return RFA_OK;
}

struct MemberSnap {
    void *th = nullptr, *lo = nullptr, *om = nullptr, *oc = nullptr, *latch = nullptr;
    int cur = 0;
    int64_t steps = 0, carry = 0;
};

}  // namespace

}  // namespace rfa

using namespace rfa;

extern "C" {

rfa_status rfa_batch_create(rfa_grid *const *members, int n, rfa_batch **out)
{
    if (!out) return bfail(RFA_E_INVALID, "out is NULL");
    *out = nullptr;
    if (!members || n < 1) return bfail(RFA_E_INVALID, "need at least one member");
    for (int m = 0; m < n; ++m) {
        const rfa_grid *g = members[m];
        if (!g) return bfail(RFA_E_INVALID, "null member");
        if (!g->have_tissue) return bfail(RFA_E_STATE, "every member needs rfa_set_tissue first");
        if (g->sp != RFA_STATE_F32C || g->pp != RFA_PARAM_BF16)
            return bfail(RFA_E_UNSUPPORTED, "batched stepping needs compensated FP32 state and BF16 coefficients");
        if (g->face != RFA_FACE_DIRICHLET || g->cond != RFA_COND_CENTRE || g->alpha_perf)
            return bfail(RFA_E_UNSUPPORTED,
                         "batched stepping needs Dirichlet faces, the centre conduction form and constant perfusion");
        if (g->stream != members[0]->stream) return bfail(RFA_E_INVALID, "members must share one stream");
        if (g->dmg != members[0]->dmg) return bfail(RFA_E_INVALID, "members must share the damage setting");
        for (int k = 0; k < m; ++k)
            if (members[k] == g) return bfail(RFA_E_INVALID, "a grid appears twice in the batch");
    }
    rfa_batch *b = new (std::nothrow) rfa_batch();
    if (!b) return bfail(RFA_E_OOM, "host allocation failed");
    b->members.assign(members, members + n);
    b->stream = members[0]->stream;
    b->damage = members[0]->dmg != 0;
    if (cudaMalloc((void **)&b->d_gbar, (2 + (size_t)kMaxBlocksPerLaunch) * sizeof(unsigned)) != cudaSuccess) {
        cudaGetLastError();
        delete b;
        return bfail(RFA_E_OOM, "batch barrier allocation failed");
    }
    rfa_status st = build_plan(b);
    if (st != RFA_OK) {
        release_plan(b);
        cudaFree(b->d_gbar);
        delete b;
        return st;
    }
    *out = b;
    return RFA_OK;
}

rfa_status rfa_batch_step(rfa_batch *b, int64_t nsteps)
{
    if (!b) return bfail(RFA_E_INVALID, "null batch");
    if (nsteps < 0) return bfail(RFA_E_INVALID, "nsteps must be >= 0");
    if (nsteps == 0) return RFA_OK;
    return batch_step(b, nsteps);
}

rfa_status rfa_batch_destroy(rfa_batch *b)
{
    if (!b) return RFA_OK;
    cudaStreamSynchronize(b->stream);
    release_plan(b);
    if (b->d_gbar) cudaFree(b->d_gbar);
    delete b;
    return RFA_OK;
}

rfa_status rfa_batch_autotune(rfa_batch *b, const char *cache_path)
{
    if (!b) return bfail(RFA_E_INVALID, "null batch");
    // cache key: member count and total voxels
    size_t vox = 0;
    for (rfa_grid *g : b->members) vox += g->nvox();
    char key[96];
    std::snprintf(key, sizeof key, "batch/%zu/%zu/d%d", b->members.size(), vox, (int)b->damage);
    if (cache_path) {
        std::ifstream f(cache_path);
        std::stringstream ss;
        ss << f.rdbuf();
        const std::string s = ss.str();
        const size_t pos = s.find(std::string("\"") + key + "\"");
        int d = 0, v = 0;
        if (pos != std::string::npos && std::sscanf(s.c_str() + s.find('[', pos) + 1, "%d , %d", &d, &v) == 2 &&
            ((v == 0 && (d == 2 || d == 3)) || (v == 1 && d == 2))) {
            b->depth = d;
            b->variant = v;
            return build_plan(b);
        }
    }
    const int cands[3][2] = {{2, 0}, {3, 0}, {2, 1}};
    // snapshot every member's evolving state; restored after each trial
    std::vector<MemberSnap> snaps(b->members.size());
    rfa_status st = RFA_OK;
    for (size_t m = 0; m < b->members.size() && st == RFA_OK; ++m) {
        rfa_grid *g = b->members[m];
        MemberSnap &s = snaps[m];
        size_t nvp = g->nvp;
        if (cudaMalloc(&s.th, nvp * 4) != cudaSuccess || cudaMalloc(&s.lo, nvp * 4) != cudaSuccess ||
            cudaMalloc(&s.om, nvp * 8) != cudaSuccess || cudaMalloc(&s.oc, nvp * 4) != cudaSuccess ||
            cudaMalloc(&s.latch, nvp) != cudaSuccess) {
            cudaGetLastError();
            st = bfail(RFA_E_OOM, "batch autotune snapshot allocation failed");
            break;
        }
        s.cur = g->cur;
        s.steps = g->steps;
        s.carry = g->carry_steps;
        cudaMemcpyAsync(s.th, g->th[g->cur], nvp * 4, cudaMemcpyDeviceToDevice, b->stream);
        cudaMemcpyAsync(s.lo, g->lo[g->cur], nvp * 4, cudaMemcpyDeviceToDevice, b->stream);
        cudaMemcpyAsync(s.om, g->omega, nvp * 8, cudaMemcpyDeviceToDevice, b->stream);
        cudaMemcpyAsync(s.oc, g->omega_c, nvp * 4, cudaMemcpyDeviceToDevice, b->stream);
        cudaMemcpyAsync(s.latch, g->latch, nvp, cudaMemcpyDeviceToDevice, b->stream);
    }
    auto restore = [&]() {
        for (size_t m = 0; m < b->members.size(); ++m) {
            rfa_grid *g = b->members[m];
            const MemberSnap &s = snaps[m];
            if (!s.latch) continue;
            size_t nvp = g->nvp;
            g->cur = s.cur;
            g->steps = s.steps;
            g->carry_steps = s.carry;
            cudaMemcpyAsync(g->th[g->cur], s.th, nvp * 4, cudaMemcpyDeviceToDevice, b->stream);
            cudaMemcpyAsync(g->lo[g->cur], s.lo, nvp * 4, cudaMemcpyDeviceToDevice, b->stream);
            cudaMemcpyAsync(g->omega, s.om, nvp * 8, cudaMemcpyDeviceToDevice, b->stream);
            cudaMemcpyAsync(g->omega_c, s.oc, nvp * 4, cudaMemcpyDeviceToDevice, b->stream);
            cudaMemcpyAsync(g->latch, s.latch, nvp, cudaMemcpyDeviceToDevice, b->stream);
        }
    };
    float best = 1e30f;
    int bd = b->depth, bv = b->variant;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    const bool graphs = b->use_graphs;
    for (int c = 0; c < (int)(sizeof cands / sizeof cands[0]) && st == RFA_OK; ++c) {
        b->depth = cands[c][0];
        b->variant = cands[c][1];
        b->use_graphs = false;
        if ((st = build_plan(b)) != RFA_OK) break;
        if ((st = batch_step(b, 12)) != RFA_OK) break;
        cudaEventRecord(e0, b->stream);
        if ((st = batch_step(b, 24)) != RFA_OK) break;
        cudaEventRecord(e1, b->stream);
        cudaEventSynchronize(e1);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (ms < best) {
            best = ms;
            bd = b->depth;
            bv = b->variant;
        }
        restore();
    }
    cudaStreamSynchronize(b->stream);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    for (auto &s : snaps)
        for (void *p : {s.th, s.lo, s.om, s.oc, s.latch})
            if (p) cudaFree(p);
    b->use_graphs = graphs;
    b->depth = bd;
    b->variant = bv;
    rfa_status st2 = build_plan(b);
    if (st != RFA_OK) return st;
    if (st2 != RFA_OK) return st2;
    if (cache_path) {
        std::ofstream f(cache_path, std::ios::app);
        if (f) f << "{\"" << key << "\": [" << bd << ", " << bv << "]}\n";
    }
    return RFA_OK;
}

rfa_status rfa_batch_get_schedule(rfa_batch *b, int *tb_depth, int *tile_variant, int *uses_graph)
{
    if (!b) return bfail(RFA_E_INVALID, "null batch");
    if (tb_depth) *tb_depth = b->depth;
    if (tile_variant) *tile_variant = b->variant;
    if (uses_graph) *uses_graph = b->use_graphs ? 1 : 0;
    if (!b->use_graphs) set_error("graph capture not used: " + b->graph_error);
    return RFA_OK;
}

}  // extern "C"
