// Continuous-batching render server.
//
// Requests (scene, camera, options, output buffer) are queued by any host
// thread.  A worker thread owned by the server
//   1. admits queued requests in arrival order into free slots, as long as the
//      slots' workspaces fit the server's device-memory budget (a request that
//      cannot fit even alone is refused with MGS_ERR_OOM);
//   2. forms a group from the admitted requests: a view of more than
//      kSmallTiles tiles goes alone; consecutive small views (up to max_batch)
//      go together;
//   3. runs every slot's work on the slot's own stream, so the requests in
//      flight overlap on the device: a lone view runs preprocessing, the MLP,
//      binning and its rasteriser as one CUDA graph; the views of a group run
//      preprocessing and binning as graphs on their streams, and the group
//      is rasterised by one launch of the persistent batched rasteriser,
//      whose CTAs pull (view, tile) items from a shared counter (the small
//      views' tiles fill each other's tails);
//   4. polls completion events, stamps completion times, re-queues a request
//      whose tile lists overflowed its workspace (with a larger capacity),
//      and frees the slots.
// Graphs are instantiated once per (slot, scene, resolution, options) and
// relaunched with the new camera and output written into the kernel nodes
// that read them (preprocessing and rasterisation); binning reads only the
// workspace, which the key pins.  Each view's image depends only on its own
// tile lists: alone or in a mix it is the same up to FP32 rounding of the
// accumulation order.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "mgs_internal.cuh"

using namespace mgs;

namespace {

double now_s() {
    using namespace std::chrono;
    return duration_cast<duration<double>>(steady_clock::now().time_since_epoch()).count();
}

enum { kQueued = 0, kRunning = 1, kDone = 2 };

// Views up to this many tiles (e.g. 640x480: 1,200) are rasterised together
// when several are admitted at once; larger views fill the GPU alone.
constexpr int kSmallTiles = 2048;
constexpr int kGraphsPerSlot = 16;

struct Request {
    int64_t ticket = 0;
    mgs_scene scene = nullptr;
    mgs_camera cam{};
    mgs_render_opts opts{};
    float *out = nullptr;
    double t_submit = 0, t_admit = 0, t_done = 0;
    int state = kQueued;
    mgs_status result = MGS_OK;
    uint64_t pairs_hint = 0;
    int attempts = 0;
};

// A cached executable graph of one slot: preprocessing + binning (+ the
// single-view rasteriser when `raster`), with the nodes whose arguments
// depend on the camera and the output.
struct SlotGraph {
    uint64_t key = 0;
    uint64_t gen = 0;           // workspace buffer generation it was captured with
    uint64_t last_use = 0;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    std::vector<cudaGraphNode_t> arg_nodes;   // kernel nodes taking RenderArgs
};

struct Slot {
    mgs_workspace ws = nullptr;
    cudaStream_t stream = nullptr;
    cudaEvent_t prepared = nullptr;
    DevStatus *status_host = nullptr;  // pinned
    bool busy = false;
    int64_t ticket = 0;
    RenderArgs args{};
    std::vector<SlotGraph> graphs;
};

struct Group {
    bool active = false;
    std::vector<int> slots;
    cudaEvent_t done = nullptr;
    RenderArgs *args_host = nullptr;  // pinned
    int *prefix_host = nullptr;       // pinned
    RenderArgs *args_dev = nullptr;
    int *prefix_dev = nullptr;
    unsigned *counter_dev = nullptr;
};

}  // namespace

struct mgs_server_s {
    mgs_ctx ctx = nullptr;
    int device = 0;
    int sm_count = 0;
    int64_t budget = 0;
    int max_batch = 8;
    std::vector<Slot> slots;
    std::vector<Group> groups;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<int64_t> queue;
    std::unordered_map<int64_t, Request> reqs;
    int64_t next_ticket = 1;
    int64_t completed = 0;
    uint64_t clock = 0;
    bool stop = false;
    bool graphs = true;
    std::unordered_map<uint64_t, uint64_t> pairs_cache;  // (scene, size) -> pairs
    std::thread worker;

    void run();
    int64_t reserved_bytes() const {
        int64_t b = 0;
        for (const Slot &s : slots) b += mgs_workspace_bytes(s.ws);
        return b;
    }
};

namespace {

uint64_t cache_key(mgs_scene s, int w, int h) {
    return (reinterpret_cast<uint64_t>(s) * 1000003ull) ^ ((uint64_t)w << 32) ^ (uint64_t)h;
}

uint64_t graph_key(const Request &rq, bool raster) {
    uint64_t k = cache_key(rq.scene, rq.cam.width, rq.cam.height);
    k = k * 31ull + (uint64_t)rq.opts.use_mlp;
    k = k * 31ull + (uint64_t)rq.opts.mlp_rgb_residual;
    k = k * 131ull + (uint64_t)rq.opts.flags;
    return k * 2ull + (raster ? 1ull : 0ull);
}

int64_t estimate_bytes(int64_t n, int w, int h, uint64_t pairs, int sm_count) {
    const int64_t T = (int64_t)((w + kTile - 1) / kTile) * ((h + kTile - 1) / kTile);
    return n * (int64_t)(sizeof(ProjRec) + sizeof(uint2) + sizeof(uint4)) + (T + 1) * 12 +
           bin_scratch_words(n, T, sm_count) * 4 + (int64_t)pairs * 4 + 4096;
}

void drop_graphs(Slot &sl) {
    for (SlotGraph &g : sl.graphs) {
        if (g.exec) cudaGraphExecDestroy(g.exec);
        if (g.graph) cudaGraphDestroy(g.graph);
    }
    sl.graphs.clear();
}

// Kernel nodes of a captured graph whose only argument is a RenderArgs (the
// preprocessing and rasterisation kernels), found by their parameter size.
std::vector<cudaGraphNode_t> render_arg_nodes(cudaGraph_t g) {
    std::vector<cudaGraphNode_t> out;
    size_t n = 0;
    if (cudaGraphGetNodes(g, nullptr, &n) != cudaSuccess || n == 0) return out;
    std::vector<cudaGraphNode_t> nodes(n);
    if (cudaGraphGetNodes(g, nodes.data(), &n) != cudaSuccess) return out;
    for (cudaGraphNode_t nd : nodes) {
        cudaGraphNodeType t;
        if (cudaGraphNodeGetType(nd, &t) != cudaSuccess || t != cudaGraphNodeTypeKernel) continue;
        cudaKernelNodeParams p{};
        if (cudaGraphKernelNodeGetParams(nd, &p) != cudaSuccess) continue;
        size_t off = 0, sz = 0;
        // exactly one parameter of sizeof(RenderArgs)
        if (cudaFuncGetParamInfo(p.func, 0, &off, &sz) == cudaSuccess && sz == sizeof(RenderArgs) &&
            cudaFuncGetParamInfo(p.func, 1, &off, &sz) != cudaSuccess)
            out.push_back(nd);
        cudaGetLastError();
    }
    return out;
}

// The request's work on the slot's stream: preprocessing and binning, and the
// single-view rasteriser when `raster`.  Through the slot's cached graph for
// this key when graphs are usable, else by direct launches.
mgs_status launch_view(mgs_server_s *S, Slot &sl, Request &rq, bool raster) {
    // Stream-ordered preparation; sets sl.args (needed for the batched raster
    // and the status read-back) and grows the workspace if it must.
    auto direct = [&]() -> mgs_status {
        mgs_status st = prepare_view(sl.ws, rq.scene, &rq.cam, &rq.opts, rq.out, sl.stream, &sl.args);
        if (st == MGS_OK && raster && launch_raster(sl.args, sl.stream) != cudaSuccess)
            st = MGS_ERR_CUDA;
        return st;
    };
    if (!S->graphs) return direct();
    const uint64_t key = graph_key(rq, raster);
    const uint64_t gen = workspace_generation(sl.ws);
    SlotGraph *hit = nullptr;
    for (SlotGraph &g : sl.graphs)
        if (g.key == key && g.gen == gen) hit = &g;
    if (hit) {
        // same scene, size, options and workspace buffers: new camera / output
        RenderArgs a{};
        mgs_status st = prepare_view(sl.ws, rq.scene, &rq.cam, &rq.opts, rq.out, nullptr, &a, true);
        if (st != MGS_OK) return st;
        bool ok = workspace_generation(sl.ws) == gen;
        void *params[1] = {&a};
        for (cudaGraphNode_t nd : hit->arg_nodes) {
            if (!ok) break;
            cudaKernelNodeParams p{};
            ok = cudaGraphKernelNodeGetParams(nd, &p) == cudaSuccess;
            p.kernelParams = params;
            p.extra = nullptr;
            ok = ok && cudaGraphExecKernelNodeSetParams(hit->exec, nd, &p) == cudaSuccess;
        }
        if (ok && cudaGraphLaunch(hit->exec, sl.stream) == cudaSuccess) {
            sl.args = a;
            hit->last_use = ++S->clock;
            return MGS_OK;
        }
        cudaGetLastError();
        hit->key = 0;   // unusable: recapture below
    }
    // capture this key's graph (the workspace is sized first, outside capture)
    {
        RenderArgs a{};
        mgs_status st = prepare_view(sl.ws, rq.scene, &rq.cam, &rq.opts, rq.out, nullptr, &a, true);
        if (st != MGS_OK) return st;
    }
    cudaGraph_t g = nullptr;
    RenderArgs a{};
    mgs_status st = MGS_ERR_CUDA;
    cudaError_t e = cudaStreamBeginCapture(sl.stream, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        st = prepare_view(sl.ws, rq.scene, &rq.cam, &rq.opts, rq.out, sl.stream, &a);
        if (st == MGS_OK && raster && launch_raster(a, sl.stream) != cudaSuccess) st = MGS_ERR_CUDA;
        e = cudaStreamEndCapture(sl.stream, &g);
    }
    if (e == cudaSuccess && st != MGS_OK) {   // argument error, not a capture problem
        if (g) cudaGraphDestroy(g);
        return st;
    }
    cudaGraphExec_t exec = nullptr;
    // the nodes that take the camera and output must all be found, else a
    // relaunch would draw with stale arguments: then no graphs at all
    std::vector<cudaGraphNode_t> arg_nodes;
    const size_t want = (scene_size(rq.scene) > 0 ? 1u : 0u) + (raster ? 1u : 0u);
    if (e == cudaSuccess && g) arg_nodes = render_arg_nodes(g);
    if (e == cudaSuccess && g && arg_nodes.size() == want &&
        cudaGraphInstantiate(&exec, g, 0) == cudaSuccess &&
        cudaGraphLaunch(exec, sl.stream) == cudaSuccess) {
        SlotGraph sg;
        sg.key = key;
        sg.gen = workspace_generation(sl.ws);
        sg.graph = g;
        sg.exec = exec;
        sg.arg_nodes = arg_nodes;
        sg.last_use = ++S->clock;
        if ((int)sl.graphs.size() >= kGraphsPerSlot) {   // evict the least recently used
            auto lru = std::min_element(sl.graphs.begin(), sl.graphs.end(),
                                        [](const SlotGraph &x, const SlotGraph &y) {
                                            return x.last_use < y.last_use;
                                        });
            if (lru->exec) cudaGraphExecDestroy(lru->exec);
            if (lru->graph) cudaGraphDestroy(lru->graph);
            *lru = sg;
        } else {
            sl.graphs.push_back(sg);
        }
        sl.args = a;
        return MGS_OK;
    }
    if (exec) cudaGraphExecDestroy(exec);
    if (g) cudaGraphDestroy(g);
    // capture unavailable here: direct launches from now on
    cudaGetLastError();
    S->graphs = false;
    for (Slot &x : S->slots) drop_graphs(x);
    return direct();
}

}  // namespace

void mgs_server_s::run() {
    cudaSetDevice(device);
    std::vector<int> admitted;
    for (;;) {
        bool progress = false;
        // 1. retire finished groups
        for (Group &b : groups) {
            if (!b.active) continue;
            cudaError_t q = cudaEventQuery(b.done);
            if (q == cudaErrorNotReady) continue;
            const double t = now_s();
            std::lock_guard<std::mutex> lk(mu);
            for (int si : b.slots) {
                Slot &sl = slots[si];
                Request &rq = reqs[sl.ticket];
                const uint64_t need = sl.status_host->last_pairs;
                pairs_cache[cache_key(rq.scene, rq.cam.width, rq.cam.height)] = need;
                if (q != cudaSuccess || (sl.status_host->overflow & kStatusMmaTimeout)) {
                    rq.result = q != cudaSuccess ? MGS_ERR_CUDA : MGS_ERR_TIMEOUT;
                    rq.state = kDone;
                    rq.t_done = t;
                    ++completed;
                    if (q == cudaSuccess)  // clear the sticky flag for the slot's next request
                        cudaMemsetAsync(sl.args.status, 0, sizeof(unsigned int), sl.stream);
                } else if (need > sl.args.capacity && rq.attempts < 3) {
                    rq.pairs_hint = need + need / 4 + 1024;  // retry with room
                    rq.state = kQueued;
                    queue.push_front(rq.ticket);
                } else {
                    rq.result = need > sl.args.capacity ? MGS_ERR_OVERFLOW : MGS_OK;
                    rq.state = kDone;
                    rq.t_done = t;
                    ++completed;
                }
                sl.busy = false;
            }
            if (q != cudaSuccess) cudaGetLastError();
            b.active = false;
            b.slots.clear();
            progress = true;
            cv_done.notify_all();
        }
        // 2. admit one group: the queue's head, and after a small view the
        //    following small views, up to max_batch
        admitted.clear();
        int bi = -1;
        {
            std::unique_lock<std::mutex> lk(mu);
            if (stop && queue.empty()) {
                bool any = false;
                for (const Group &b : groups) any |= b.active;
                if (!any) return;
            }
            for (int k = 0; k < (int)groups.size(); ++k)
                if (!groups[k].active) {
                    bi = k;
                    break;
                }
            bool released = false;
            bool small_group = false;
            while (bi >= 0 && !queue.empty() && (int)admitted.size() < max_batch) {
                Request &rq = reqs[queue.front()];
                const int tiles = ((rq.cam.width + kTile - 1) / kTile) * ((rq.cam.height + kTile - 1) / kTile);
                const bool small = tiles <= kSmallTiles && (rq.opts.flags & MGS_FLAG_SORTED) == 0;
                if (!admitted.empty() && (!small_group || !small)) break;
                int free_slot = -1;
                for (int k = 0; k < (int)slots.size(); ++k)
                    if (!slots[k].busy &&
                        std::find(admitted.begin(), admitted.end(), k) == admitted.end() &&
                        (free_slot < 0 ||
                         mgs_workspace_bytes(slots[k].ws) > mgs_workspace_bytes(slots[free_slot].ws)))
                        free_slot = k;
                if (free_slot < 0) break;
                const int64_t n = scene_size(rq.scene);
                auto it = pairs_cache.find(cache_key(rq.scene, rq.cam.width, rq.cam.height));
                uint64_t pairs = it != pairs_cache.end() ? it->second + it->second / 8 + 1024
                                                         : (uint64_t)std::max<int64_t>(48 * n, 1 << 20);
                pairs = std::max(pairs, rq.pairs_hint);
                const int64_t need = estimate_bytes(n, rq.cam.width, rq.cam.height, pairs, sm_count);
                if (need > budget) {
                    rq.result = MGS_ERR_OOM;
                    rq.state = kDone;
                    rq.t_done = now_s();
                    ++completed;
                    queue.pop_front();
                    cv_done.notify_all();
                    continue;
                }
                const int64_t cur = mgs_workspace_bytes(slots[free_slot].ws);
                if (reserved_bytes() - cur + std::max(need, cur) > budget) {
                    // release idle slots' scratch, then retry once the GPU is idle
                    bool any_busy = false;
                    for (const Slot &s : slots) any_busy |= s.busy;
                    if (any_busy || !admitted.empty() || released) break;
                    released = true;
                    for (Slot &s : slots) {
                        drop_graphs(s);
                        mgs_workspace_destroy(s.ws);
                        mgs_workspace_create(ctx, &s.ws);
                    }
                    continue;
                }
                Slot &sl = slots[free_slot];
                mgs_status rs = mgs_workspace_reserve(sl.ws, n, rq.cam.width, rq.cam.height,
                                                      (int64_t)pairs);
                if (rs == MGS_OK && reserved_bytes() > budget) {
                    // capacities only grow: rebuild this slot's scratch at exactly
                    // this request's size so the total stays within the budget
                    drop_graphs(sl);
                    mgs_workspace_destroy(sl.ws);
                    mgs_workspace_create(ctx, &sl.ws);
                    rs = mgs_workspace_reserve(sl.ws, n, rq.cam.width, rq.cam.height, (int64_t)pairs);
                }
                if (rs != MGS_OK) {
                    rq.result = MGS_ERR_OOM;
                    rq.state = kDone;
                    rq.t_done = now_s();
                    ++completed;
                    queue.pop_front();
                    cv_done.notify_all();
                    continue;
                }
                queue.pop_front();
                rq.state = kRunning;
                rq.attempts += 1;
                rq.t_admit = now_s();
                sl.busy = true;
                sl.ticket = rq.ticket;
                admitted.push_back(free_slot);
                if (admitted.size() == 1) small_group = small;
            }
        }
        // 3. launch the admitted group
        if (!admitted.empty()) {
            Group &b = groups[bi];
            const bool alone = admitted.size() == 1;
            std::vector<int> ok;
            for (int si : admitted) {
                Slot &sl = slots[si];
                Request *rq;
                {
                    std::lock_guard<std::mutex> lk(mu);
                    rq = &reqs[sl.ticket];
                }
                mgs_status st = launch_view(this, sl, *rq, alone);
                if (st == MGS_OK && !alone &&
                    cudaEventRecord(sl.prepared, sl.stream) != cudaSuccess)
                    st = MGS_ERR_CUDA;
                if (st != MGS_OK) {
                    std::lock_guard<std::mutex> lk(mu);
                    rq->result = st;
                    rq->state = kDone;
                    rq->t_done = now_s();
                    ++completed;
                    sl.busy = false;
                    cv_done.notify_all();
                    continue;
                }
                ok.push_back(si);
            }
            if (!ok.empty()) {
                Slot &lead = slots[ok[0]];
                if (!alone) {
                    // the group's views rasterised together on the first view's stream
                    for (size_t v = 1; v < ok.size(); ++v)
                        cudaStreamWaitEvent(lead.stream, slots[ok[v]].prepared, 0);
                    b.prefix_host[0] = 0;
                    for (size_t v = 0; v < ok.size(); ++v) {
                        const RenderArgs &a = slots[ok[v]].args;
                        b.args_host[v] = a;
                        b.prefix_host[v + 1] = b.prefix_host[v] + a.cam.tiles_x * a.cam.tiles_y;
                    }
                    const int nv = (int)ok.size();
                    cudaMemcpyAsync(b.args_dev, b.args_host, sizeof(RenderArgs) * nv,
                                    cudaMemcpyHostToDevice, lead.stream);
                    cudaMemcpyAsync(b.prefix_dev, b.prefix_host, sizeof(int) * (nv + 1),
                                    cudaMemcpyHostToDevice, lead.stream);
                    launch_raster_batch(b.args_dev, b.prefix_dev, nv, b.counter_dev, sm_count,
                                        lead.stream);
                }
                for (int si : ok)
                    cudaMemcpyAsync(slots[si].status_host, slots[si].args.status, sizeof(DevStatus),
                                    cudaMemcpyDeviceToHost, lead.stream);
                cudaEventRecord(b.done, lead.stream);
                b.slots = ok;
                b.active = true;
            }
            progress = true;
        }
        if (!progress) {
            std::unique_lock<std::mutex> lk(mu);
            bool inflight = false;
            for (const Group &b : groups) inflight |= b.active;
            if (inflight)
                cv_work.wait_for(lk, std::chrono::microseconds(20));
            else
                cv_work.wait_for(lk, std::chrono::milliseconds(2),
                                 [&] { return stop || !queue.empty(); });
        }
    }
}

extern "C" {

mgs_status mgs_server_create(mgs_ctx ctx, const mgs_server_config *cfg, mgs_server *out) {
    if (!ctx || !cfg || !out) {
        set_last_error("NULL argument");
        return MGS_ERR_INVALID_ARG;
    }
    *out = nullptr;
    if (cfg->slots < 1 || cfg->slots > 64 || cfg->hbm_budget_bytes <= 0 || cfg->max_batch < 1 ||
        cfg->max_batch > 64) {
        set_last_error("server config: slots and max_batch in 1..64, positive budget");
        return MGS_ERR_INVALID_ARG;
    }
    mgs_server S = new mgs_server_s;
    S->ctx = ctx;
    S->device = ctx_device(ctx);
    S->sm_count = ctx_sm_count(ctx);
    S->budget = cfg->hbm_budget_bytes;
    S->max_batch = cfg->max_batch;
    int prev = 0;
    cudaGetDevice(&prev);
    cudaSetDevice(S->device);
    bool ok = true;
    S->slots.resize(cfg->slots);
    for (Slot &s : S->slots) {
        ok &= mgs_workspace_create(ctx, &s.ws) == MGS_OK;
        ok &= cudaStreamCreateWithFlags(&s.stream, cudaStreamNonBlocking) == cudaSuccess;
        ok &= cudaEventCreateWithFlags(&s.prepared, cudaEventDisableTiming) == cudaSuccess;
        ok &= cudaMallocHost(&s.status_host, sizeof(DevStatus)) == cudaSuccess;
    }
    S->groups.resize(cfg->slots);
    for (Group &b : S->groups) {
        ok &= cudaEventCreateWithFlags(&b.done, cudaEventDisableTiming) == cudaSuccess;
        ok &= cudaMallocHost(&b.args_host, sizeof(RenderArgs) * cfg->max_batch) == cudaSuccess;
        ok &= cudaMallocHost(&b.prefix_host, sizeof(int) * (cfg->max_batch + 1)) == cudaSuccess;
        ok &= cudaMalloc(&b.args_dev, sizeof(RenderArgs) * cfg->max_batch) == cudaSuccess;
        ok &= cudaMalloc(&b.prefix_dev, sizeof(int) * (cfg->max_batch + 1)) == cudaSuccess;
        ok &= cudaMalloc(&b.counter_dev, sizeof(unsigned)) == cudaSuccess;
    }
    cudaSetDevice(prev);
    if (!ok) {
        mgs_server_destroy(S);
        set_last_error("server resources could not be allocated");
        return MGS_ERR_OOM;
    }
    S->worker = std::thread([S] { S->run(); });
    *out = S;
    return MGS_OK;
}

mgs_status mgs_server_destroy(mgs_server S) {
    if (!S) return MGS_OK;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->stop = true;
    }
    S->cv_work.notify_all();
    if (S->worker.joinable()) S->worker.join();
    int prev = 0;
    cudaGetDevice(&prev);
    cudaSetDevice(S->device);
    for (Slot &s : S->slots) {
        if (s.stream) cudaStreamSynchronize(s.stream);
        drop_graphs(s);
        if (s.ws) mgs_workspace_destroy(s.ws);
        if (s.stream) cudaStreamDestroy(s.stream);
        if (s.prepared) cudaEventDestroy(s.prepared);
        if (s.status_host) cudaFreeHost(s.status_host);
    }
    for (Group &b : S->groups) {
        if (b.done) cudaEventDestroy(b.done);
        if (b.args_host) cudaFreeHost(b.args_host);
        if (b.prefix_host) cudaFreeHost(b.prefix_host);
        if (b.args_dev) cudaFree(b.args_dev);
        if (b.prefix_dev) cudaFree(b.prefix_dev);
        if (b.counter_dev) cudaFree(b.counter_dev);
    }
    cudaSetDevice(prev);
    delete S;
    return MGS_OK;
}

mgs_status mgs_server_submit(mgs_server S, mgs_scene scene, const mgs_camera *cam,
                             const mgs_render_opts *opts, float *out_rgb, int64_t *ticket) {
    if (!S || !scene || !cam || !opts || !out_rgb || !ticket) {
        set_last_error("NULL argument");
        return MGS_ERR_INVALID_ARG;
    }
    if (scene_ctx(scene) != S->ctx) {
        set_last_error("scene belongs to another context");
        return MGS_ERR_INVALID_ARG;
    }
    if (validate_camera(cam) != MGS_OK) return MGS_ERR_INVALID_ARG;
    Request rq;
    rq.scene = scene;
    rq.cam = *cam;
    rq.opts = *opts;
    rq.out = out_rgb;
    rq.t_submit = now_s();
    {
        std::lock_guard<std::mutex> lk(S->mu);
        rq.ticket = S->next_ticket++;
        *ticket = rq.ticket;
        S->reqs[rq.ticket] = rq;
        S->queue.push_back(rq.ticket);
    }
    S->cv_work.notify_one();
    return MGS_OK;
}

mgs_status mgs_server_wait(mgs_server S, int64_t ticket, double timeout_ms) {
    if (!S) {
        set_last_error("NULL server");
        return MGS_ERR_INVALID_ARG;
    }
    std::unique_lock<std::mutex> lk(S->mu);
    auto it = S->reqs.find(ticket);
    if (it == S->reqs.end()) {
        set_last_error("unknown ticket");
        return MGS_ERR_INVALID_ARG;
    }
    const auto deadline = std::chrono::steady_clock::now() +
                          std::chrono::microseconds((int64_t)(timeout_ms * 1000.0));
    while (S->reqs[ticket].state != kDone) {
        if (S->cv_done.wait_until(lk, deadline) == std::cv_status::timeout &&
            S->reqs[ticket].state != kDone) {
            set_last_error("timed out waiting for the ticket");
            return MGS_ERR_TIMEOUT;
        }
    }
    const mgs_status r = S->reqs[ticket].result;
    if (r != MGS_OK) set_last_error("request failed (see mgs_server_ticket)");
    return r;
}

mgs_status mgs_server_ticket(mgs_server S, int64_t ticket, int32_t *state, int32_t *result,
                             double *t_submit, double *t_admit, double *t_done) {
    if (!S) {
        set_last_error("NULL server");
        return MGS_ERR_INVALID_ARG;
    }
    std::lock_guard<std::mutex> lk(S->mu);
    auto it = S->reqs.find(ticket);
    if (it == S->reqs.end()) {
        set_last_error("unknown ticket");
        return MGS_ERR_INVALID_ARG;
    }
    const Request &r = it->second;
    if (state) *state = r.state;
    if (result) *result = r.result;
    if (t_submit) *t_submit = r.t_submit;
    if (t_admit) *t_admit = r.t_admit;
    if (t_done) *t_done = r.t_done;
    return MGS_OK;
}

mgs_status mgs_server_stats(mgs_server S, int64_t *completed, int64_t *queued,
                            int64_t *running, int64_t *workspace_bytes, int32_t *graphs) {
    if (!S) {
        set_last_error("NULL server");
        return MGS_ERR_INVALID_ARG;
    }
    std::lock_guard<std::mutex> lk(S->mu);
    int64_t run = 0;
    for (const Slot &s : S->slots) run += s.busy;
    if (completed) *completed = S->completed;
    if (queued) *queued = (int64_t)S->queue.size();
    if (running) *running = run;
    if (workspace_bytes) *workspace_bytes = S->reserved_bytes();
    if (graphs) *graphs = S->graphs ? 1 : 0;
    return MGS_OK;
}

double mgs_now(void) { return now_s(); }

}  // extern "C"
