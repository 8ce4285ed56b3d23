// Step server (include/ms_server.h).
//
// Sessions are ordinary batches (ms_create_batch_flat) whose state stays
// resident.  Clients queue step requests from any thread; one worker thread
// takes every pending request (at most one per session, in arrival order),
// stages their drive targets, and runs one launch of k_multi over the union
// of their envs: a persistent kernel whose work list names (session, env)
// pairs and which reads each env's batch view from a device table, so
// sessions of different scene types and solver parameters share a launch
// (a warp's envs always come from one session).
// The launch (queue reset + kernel) is captured once per workspace layout
// (bucketed sizes) in a CUDA graph whose kernel parameters are updated per
// launch.  Up to max_inflight launches run at once, each on its own stream
// (a "slot"); the worker polls their completion events, so a new launch can
// start while earlier ones run.  Every request is stamped with its host
// arrival and completion times.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "../../include/ms.h"
#include "../../include/ms_server.h"
#include "ms_internal.h"
#include "ms_stages.cuh"

namespace ms {

// G lanes per env, K = 32 / G envs per warp, all of one session: the work
// list is grouped by session and each session's envs are padded to a
// multiple of K with inactive items (env = -1), so the envs of a warp share
// their parameters (substeps, iterations) and the lockstep loops stay
// warp-uniform, as in the batched kernel.
template <int G>
__global__ void __launch_bounds__(256, 1) k_multi(const DevBatch* __restrict__ batches, const float* const* actions,
                                                  const int2* work, int n_work, Layout L, int* queue,
                                                  char* gscratch) {
    extern __shared__ __align__(16) char smem[];
    constexpr int K = 32 / G;
    int warp = threadIdx.x >> 5, wl = threadIdx.x & 31;
    int gi = wl / G;
    Grp g;
    g.lane = wl % G; g.size = G; g.base = gi * G;
    char* s = smem + (size_t)(warp * K + gi) * L.s_bytes;
    size_t gslot = ((size_t)blockIdx.x * (blockDim.x >> 5) + warp) * K + gi;
    char* gl = gscratch + gslot * (size_t)L.g_bytes;
    EnvView e;
    e.x = at<float4>(s, L.x); e.q = at<float4>(s, L.q); e.v = at<float4>(s, L.v); e.w = at<float4>(s, L.w);
    view_workspace(e, s, gl, L);
    e.status = at<unsigned>(s, L.status);
    e.rec_man = nullptr; e.rec_pts = nullptr; e.rec_cnt = nullptr; e.rec_col = nullptr;

    for (;;) {
        int t0 = 0;
        if (wl == 0) t0 = atomicAdd(queue, K);
        t0 = __shfl_sync(FULL_MASK, t0, 0);
        if (t0 >= n_work) break;                              // warp-uniform; n_work is a multiple of K
        int2 it = work[t0 + gi];
        const DevBatch& D = batches[it.x];                    // one session per warp
        int env = it.y;
        bool active = env >= 0;
        int b0 = 0, j0 = 0, nb = 0, nj = 0;
        if (active) {
            b0 = D.body_off[env]; j0 = D.joint_off[env];
            nb = D.body_off[env + 1] - b0; nj = D.joint_off[env + 1] - j0;
        }
        e.shape = D.shape + b0; e.inv = D.inv + b0; e.meta = D.meta + b0; e.adj = D.adj + b0;
        e.jf = D.jf + 4 * (size_t)j0; e.jp = D.jp + j0; e.jm = D.jm + j0; e.jt = D.jt + j0;
        e.rest = D.rest + b0;
        e.hulls = D.hulls;
        e.force = nullptr;
        bool wm = active && D.wc;
        e.wc = wm ? D.wc + 2 * (size_t)env * (size_t)D.P.contact_cap : nullptr;
        e.wc_n = wm ? D.wc_n + env : nullptr;
        e.wjl = wm ? D.wjl + 8 * (size_t)j0 : nullptr;
        int nbmax = g.wmax(nb);
        for (int i0 = 0; i0 < nbmax; i0 += G) {
            int i = i0 + g.lane;
            if (i < nb) { e.x[i] = D.x[b0 + i]; e.q[i] = D.q[b0 + i]; e.v[i] = D.v[b0 + i]; e.w[i] = D.w[b0 + i]; }
        }
        if (g.lane == 0) *e.status = active ? D.status[env] : 0u;
        g.sync();
        bool frozen = (*e.status & ST_NAN) != 0;
        e.nb = frozen ? 0 : nb;
        e.nj = frozen ? 0 : nj;
        DevParams P = D.P;
        const float* act = (active && actions[it.x]) ? actions[it.x] + (size_t)env * D.A : nullptr;
        stage_actions(e, g, act, D.A, nullptr);
        stage_broadphase(e, g, P);
        stage_narrowphase(e, g, P);
        begin_step_solve(e, g, P);
        for (int sub = 0; sub < P.substeps; sub++) run_substep(e, g, P, sub == 0, sub == P.substeps - 1);
        end_step_solve(e, g, P);
        stage_check(e, g);
        for (int i0 = 0; i0 < nbmax; i0 += G) {
            int i = i0 + g.lane;
            if (i < nb) { D.x[b0 + i] = e.x[i]; D.q[b0 + i] = e.q[i]; D.v[b0 + i] = e.v[i]; D.w[b0 + i] = e.w[i]; }
        }
        if (g.lane == 0 && active) D.status[env] = *e.status;
        g.sync();
    }
}

constexpr int MULTI_G = 8;                      // lanes per env of merged launches
constexpr int MULTI_K = 32 / MULTI_G;           // envs per warp

}  // namespace ms

using namespace ms;

namespace {

double now_s() {
    using namespace std::chrono;
    return duration<double>(steady_clock::now().time_since_epoch()).count();
}

struct Session {
    uint64_t id = 0;
    ms_batch* b = nullptr;
    int E = 0, A = 0, max_nb = 0, max_nj = 0;
    ms_sim_params p{};
    size_t bytes = 0;
    int inflight = 0;             // queued or running requests
    bool running = false;         // one of its requests is in a launch
};

struct Req {
    uint64_t ticket = 0, session = 0;
    double t_arrive = 0, t_done = 0;
    bool done = false;
    int status = MS_OK;
    int launch_envs = 0;
    std::vector<float> act;       // empty: no target change
};

struct GraphKey {
    int s_bytes, g_bytes, threads, grid;
    bool operator<(const GraphKey& o) const {
        return std::tie(s_bytes, g_bytes, threads, grid) < std::tie(o.s_bytes, o.g_bytes, o.threads, o.grid);
    }
};

struct GraphE {
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaGraphNode_t kernel = nullptr;
    cudaKernelNodeParams kp{};
};

// One launch in flight at a time per slot: its stream and completion event,
// the requests it serves, the device tables of a merged launch with their
// pinned host staging, and its graphs (one per workspace layout).  The
// worker is the only thread that touches a slot.
struct Slot {
    cudaStream_t stream = nullptr;
    cudaEvent_t done = nullptr;
    bool busy = false;
    int status = MS_OK;
    int envs = 0;
    double t0 = 0.0;
    std::vector<std::pair<Req*, Session*>> batch;
    DevBatch* d_batches = nullptr;
    const float** d_acts = nullptr;
    int2* d_work = nullptr;
    int* d_queue = nullptr;
    char* d_gscratch = nullptr;
    float* d_act = nullptr;
    DevBatch* h_batches = nullptr;
    const float** h_acts = nullptr;
    int2* h_work = nullptr;
    float* h_act = nullptr;
    size_t cap_batches = 0, cap_work = 0, cap_gscratch = 0, cap_act = 0;
    std::map<GraphKey, GraphE> graphs;
};

ms_status sfail(ms_status code, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    set_last_error(buf);
    return code;
}

// Smallest listed size >= v (v itself above the list): merged launches of
// similar sessions share a workspace layout, hence a graph.
int bucket(int v, std::initializer_list<int> sizes) {
    for (int s : sizes)
        if (v <= s) return s;
    return v;
}

// Requests whose sessions fall in one cost class are merged into one launch:
// the solver's sweeps per step and the bucketed env size (the same buckets
// as a merged launch's workspace layout), so the envs of a launch take
// similar time.
uint64_t cost_class(const Session* se) {
    uint64_t k = (uint64_t)se->p.substeps;
    k = k * 4099 + (uint64_t)(se->p.pos_iters + 1) * 131 + (uint64_t)se->p.vel_iters;
    k = k * 131 + (uint64_t)bucket(se->max_nb, {4, 8, 12, 16, 24, 32, 48, 64});
    k = k * 131 + (uint64_t)bucket(se->max_nj, {0, 4, 8, 12, 16, 24, 32, 48, 64});
    k = k * 2053 + (uint64_t)bucket(se->p.contact_capacity, {8, 16, 32, 64, 128, 256, 512, 1024});
    return k;
}

}  // namespace

struct ms_server {
    size_t budget = 0, used = 0;
    ms_server_options opt{1, 0, 0.0, 16};
    int device = 0, sm_count = 0, smem_optin = 0;
    std::mutex mu;
    // Serialises the worker's stream captures with the client threads'
    // batch creation, destruction and device-wide synchronisation, any of
    // which may invalidate a capture in flight.  Never taken while the
    // worker holds `mu`; a client may hold `mu` and then take it.
    std::mutex dev_mu;
    std::condition_variable cv, done_cv;
    std::thread worker;
    bool stop = false;
    uint64_t next_session = 1, next_ticket = 1;
    std::unordered_map<uint64_t, Session*> sessions;
    std::deque<uint64_t> pending;
    std::unordered_map<uint64_t, Req> reqs;     // element addresses stay valid across inserts
    std::vector<Slot> slots;
    std::vector<void*> retired_host;            // outgrown pinned staging, freed at destroy
    // statistics
    uint64_t sessions_admitted = 0, sessions_rejected = 0, requests_done = 0, launches = 0, env_steps = 0;
    std::atomic<uint64_t> graph_captures{0};     // counted by the worker outside `mu`
    int running = 0;                            // slots with a launch in flight
    double busy_since = 0.0, busy = 0.0;
    std::vector<double> lat, launch_t, queue_t, stage_t;
};

// Device tables grow stream-ordered on the slot's stream (no device-wide
// synchronisation); outgrown pinned buffers are kept until destroy.
template <class T>
static cudaError_t grow_dev(Slot& sl, T** p, size_t& cap, size_t need, size_t elem) {
    if (need <= cap) return cudaSuccess;
    size_t c = std::max(need, 2 * cap);
    if (*p) cudaFreeAsync((void*)*p, sl.stream);
    *p = nullptr;
    cudaError_t e = cudaMallocAsync((void**)p, c * elem, sl.stream);
    if (e == cudaSuccess) cap = c;
    else cap = 0;
    return e;
}

template <class T>
static cudaError_t grow_host(ms_server* s, T** p, size_t old_cap, size_t new_cap, size_t elem) {
    if (new_cap <= old_cap && *p) return cudaSuccess;
    if (*p) s->retired_host.push_back((void*)*p);
    *p = nullptr;
    return cudaMallocHost((void**)p, new_cap * elem);
}

static cudaError_t grow_slot(ms_server* s, Slot& sl, size_t nb, size_t nw, size_t gbytes, size_t nact) {
    cudaError_t e;
    if (nb > sl.cap_batches) {
        size_t old = sl.cap_batches;
        if ((e = grow_dev(sl, &sl.d_batches, sl.cap_batches, nb, sizeof(DevBatch))) != cudaSuccess) return e;
        size_t c = sl.cap_batches, c2 = old;
        if ((e = grow_dev(sl, &sl.d_acts, c2, c, sizeof(float*))) != cudaSuccess) return e;
        if ((e = grow_host(s, &sl.h_batches, old, c, sizeof(DevBatch))) != cudaSuccess) return e;
        if ((e = grow_host(s, &sl.h_acts, old, c, sizeof(float*))) != cudaSuccess) return e;
    }
    if (nw > sl.cap_work) {
        size_t old = sl.cap_work;
        if ((e = grow_dev(sl, &sl.d_work, sl.cap_work, nw, sizeof(int2))) != cudaSuccess) return e;
        if ((e = grow_host(s, &sl.h_work, old, sl.cap_work, sizeof(int2))) != cudaSuccess) return e;
    }
    if (nact > sl.cap_act) {
        size_t old = sl.cap_act;
        if ((e = grow_dev(sl, &sl.d_act, sl.cap_act, nact, sizeof(float))) != cudaSuccess) return e;
        if ((e = grow_host(s, &sl.h_act, old, sl.cap_act, sizeof(float))) != cudaSuccess) return e;
    }
    if ((e = grow_dev(sl, &sl.d_gscratch, sl.cap_gscratch, gbytes, 1)) != cudaSuccess) return e;
    if (!sl.d_queue && (e = cudaMallocAsync((void**)&sl.d_queue, 256, sl.stream)) != cudaSuccess) return e;
    return cudaSuccess;
}

static void free_slot(ms_server* s, Slot& sl) {
    cudaStreamSynchronize(sl.stream);
    for (auto& kv : sl.graphs) {
        cudaGraphExecDestroy(kv.second.exec);
        cudaGraphDestroy(kv.second.graph);
    }
    sl.graphs.clear();
    cudaFreeAsync(sl.d_batches, sl.stream); cudaFreeAsync(sl.d_acts, sl.stream); cudaFreeAsync(sl.d_work, sl.stream);
    cudaFreeAsync(sl.d_queue, sl.stream); cudaFreeAsync(sl.d_gscratch, sl.stream); cudaFreeAsync(sl.d_act, sl.stream);
    cudaStreamSynchronize(sl.stream);
    cudaFreeHost(sl.h_batches); cudaFreeHost(sl.h_acts); cudaFreeHost(sl.h_work); cudaFreeHost(sl.h_act);
    cudaEventDestroy(sl.done);
    cudaStreamDestroy(sl.stream);
    (void)s;
}

// Stages and launches one merged launch over the slot's sessions (one
// request each); does not wait for it.
static int launch_merged(ms_server* s, Slot& sl) {
    auto& batch = sl.batch;
    int mb = 1, mj = 0, pc = 1, cc = 1;
    size_t nact = 0, nenv = 0;
    for (auto& rs : batch) {
        Session* se = rs.second;
        mb = std::max(mb, se->max_nb); mj = std::max(mj, se->max_nj);
        pc = std::max(pc, se->p.pair_capacity); cc = std::max(cc, se->p.contact_capacity);
        nact += rs.first->act.size();
        nenv += (size_t)se->E;
    }
    mb = bucket(mb, {4, 8, 12, 16, 24, 32, 48, 64});
    mj = bucket(mj, {0, 4, 8, 12, 16, 24, 32, 48, 64});
    pc = bucket(pc, {8, 16, 32, 64, 128, 256, 512, 1024});
    cc = bucket(cc, {8, 16, 32, 64, 128, 256, 512, 1024});
    const int warps = 1;
    const int envs_per_cta = warps * MULTI_K;
    // contact rows on chip for as many points as leave 4 CTAs per SM (16
    // envs); every row on chip if that fits, else the joint rows, then the
    // lists and impulses move to the global part
    auto occ = [&](const Layout& Lc) {
        size_t sm = (size_t)Lc.s_bytes * envs_per_cta;
        if (sm > (size_t)s->smem_optin) return 0;
        int n = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, (const void*)k_multi<MULTI_G>, 32 * warps, sm) != cudaSuccess)
            return 0;
        return n;
    };
    Layout L{};
    bool found = false;
    for (int ps : {cc, 32, 16, 8, 0}) {
        if (ps > cc) continue;
        Layout c = make_layout(mb, mj, pc, cc, true, true, ps, true, false);
        if (occ(c) >= 4 || (ps == 0 && occ(c) >= 1)) { L = c; found = true; break; }
    }
    if (!found) {
        L = make_layout(mb, mj, pc, cc, true, false, 0, true, false);
        if (occ(L) < 1) L = make_layout(mb, mj, pc, cc, true, false, 0, false, false);
    }
    size_t smem = (size_t)L.s_bytes * envs_per_cta;
    if (smem > (size_t)s->smem_optin) return sfail(MS_ERR_INVALID_ARG, "merged layout needs %zu B of shared memory", smem);
    int per_sm = occ(L);
    if (per_sm < 1) return sfail(MS_ERR_INVALID_ARG, "merged layout does not fit on an SM");
    // a fixed grid per layout keeps one graph per layout; warps without work exit at once
    int grid = per_sm * s->sm_count;
    // the work list: sessions heaviest first, each session's envs padded to a
    // multiple of MULTI_K with inactive items
    std::vector<int> order(batch.size());
    for (size_t i = 0; i < batch.size(); i++) order[i] = (int)i;
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) {
        const Session* sx = batch[x].second;
        const Session* sy = batch[y].second;
        return sx->max_nj * 8 + sx->max_nb > sy->max_nj * 8 + sy->max_nb;
    });
    size_t npad = 0;
    for (auto& rs : batch) npad += (size_t)((rs.second->E + MULTI_K - 1) / MULTI_K * MULTI_K);
    if (grow_slot(s, sl, batch.size(), npad, (size_t)grid * envs_per_cta * L.g_bytes, nact) != cudaSuccess)
        return sfail(MS_ERR_OOM, "server tables: device or pinned allocation failed");
    size_t w = 0, a = 0;
    for (size_t i = 0; i < batch.size(); i++) {
        Session* se = batch[i].second;
        Req* r = batch[i].first;
        sl.h_batches[i] = batch_dev(se->b);
        sl.h_acts[i] = nullptr;
        if (!r->act.empty()) {
            memcpy(sl.h_act + a, r->act.data(), r->act.size() * sizeof(float));
            sl.h_acts[i] = sl.d_act + a;
            a += r->act.size();
        }
    }
    for (int i : order) {
        int E = batch[i].second->E;
        int Ep = (E + MULTI_K - 1) / MULTI_K * MULTI_K;
        for (int e = 0; e < Ep; e++) sl.h_work[w++] = make_int2(i, e < E ? e : -1);
    }
    if (a) cudaMemcpyAsync(sl.d_act, sl.h_act, a * sizeof(float), cudaMemcpyHostToDevice, sl.stream);
    cudaMemcpyAsync(sl.d_batches, sl.h_batches, batch.size() * sizeof(DevBatch), cudaMemcpyHostToDevice, sl.stream);
    cudaMemcpyAsync(sl.d_acts, sl.h_acts, batch.size() * sizeof(float*), cudaMemcpyHostToDevice, sl.stream);
    cudaMemcpyAsync(sl.d_work, sl.h_work, w * sizeof(int2), cudaMemcpyHostToDevice, sl.stream);
    GraphKey key{L.s_bytes, L.g_bytes, 32 * warps, grid};
    auto it = sl.graphs.find(key);
    const DevBatch* a0 = sl.d_batches;
    const float* const* a1 = sl.d_acts;
    const int2* a2 = sl.d_work;
    int a3 = (int)w;
    Layout a4 = L;
    int* a5 = sl.d_queue;
    char* a6 = sl.d_gscratch;
    void* args[] = {(void*)&a0, (void*)&a1, (void*)&a2, (void*)&a3, (void*)&a4, (void*)&a5, (void*)&a6};
    if (it == sl.graphs.end()) {
        GraphE ge;
        cudaGraph_t g;
        {
            std::lock_guard<std::mutex> dk(s->dev_mu);
            if (cudaStreamBeginCapture(sl.stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
                return sfail(MS_ERR_CUDA, "merged launch: begin capture failed");
            cudaMemsetAsync(sl.d_queue, 0, sizeof(int), sl.stream);
            cudaLaunchKernel((const void*)k_multi<MULTI_G>, dim3(grid), dim3(32 * warps), args, smem, sl.stream);
            cudaError_t ce = cudaStreamEndCapture(sl.stream, &g);
            if (ce != cudaSuccess) return sfail(MS_ERR_CUDA, "merged launch capture: %s", cudaGetErrorString(ce));
        }
        if (cudaGraphInstantiate(&ge.exec, g, 0) != cudaSuccess) return sfail(MS_ERR_CUDA, "graph instantiate failed");
        size_t n = 0;
        cudaGraphGetNodes(g, nullptr, &n);
        std::vector<cudaGraphNode_t> nodes(n);
        cudaGraphGetNodes(g, nodes.data(), &n);
        for (auto nd : nodes) {
            cudaGraphNodeType ty;
            cudaGraphNodeGetType(nd, &ty);
            if (ty == cudaGraphNodeTypeKernel) { ge.kernel = nd; cudaGraphKernelNodeGetParams(nd, &ge.kp); }
        }
        ge.graph = g;
        it = sl.graphs.emplace(key, ge).first;
        s->graph_captures++;
    } else {
        cudaKernelNodeParams kp = it->second.kp;
        kp.kernelParams = args;
        kp.extra = nullptr;
        if (cudaGraphExecKernelNodeSetParams(it->second.exec, it->second.kernel, &kp) != cudaSuccess)
            return sfail(MS_ERR_CUDA, "graph parameter update failed");
    }
    if (cudaGraphLaunch(it->second.exec, sl.stream) != cudaSuccess) return sfail(MS_ERR_CUDA, "graph launch failed");
    if (cudaEventRecord(sl.done, sl.stream) != cudaSuccess) return sfail(MS_ERR_CUDA, "event record failed");
    sl.envs = (int)nenv;                    // padding items are not env-steps
    return MS_OK;
}

// One request, one ms_step of its session's batch; does not wait for it.
static int launch_single(ms_server* s, Slot& sl) {
    Req* r = sl.batch[0].first;
    Session* se = sl.batch[0].second;
    const float* act = nullptr;
    if (!r->act.empty()) {
        if (grow_slot(s, sl, 1, 1, 0, r->act.size()) != cudaSuccess)
            return sfail(MS_ERR_OOM, "server tables: device or pinned allocation failed");
        memcpy(sl.h_act, r->act.data(), r->act.size() * sizeof(float));
        cudaMemcpyAsync(sl.d_act, sl.h_act, r->act.size() * sizeof(float), cudaMemcpyHostToDevice, sl.stream);
        act = sl.d_act;
    }
    // sessions are short-lived (tens of requests): launched directly, no
    // graph captured per session
    int st = batch_step_eager(se->b, act, 1, sl.stream);
    if (st) return st;
    if (cudaEventRecord(sl.done, sl.stream) != cudaSuccess) return sfail(MS_ERR_CUDA, "event record failed");
    sl.envs = se->E;
    return MS_OK;
}

// Completes the slot's requests (mu held).
static void retire(ms_server* s, Slot& sl, double t) {
    for (auto& rs : sl.batch) {
        Req* r = rs.first;
        r->done = true;
        r->status = sl.status;
        r->t_done = t;
        r->launch_envs = sl.envs;
        r->act.clear();
        r->act.shrink_to_fit();
        rs.second->inflight--;
        rs.second->running = false;
        s->lat.push_back(t - r->t_arrive);
        s->queue_t.push_back(sl.t0 - r->t_arrive);
        s->requests_done++;
    }
    if (sl.status == MS_OK) {
        s->launches++;
        s->env_steps += (uint64_t)sl.envs;
    }
    s->launch_t.push_back(t - sl.t0);
    sl.batch.clear();
    sl.busy = false;
    if (--s->running == 0) s->busy += t - s->busy_since;
}

static void worker_loop(ms_server* s) {
    cudaSetDevice(s->device);
    std::unique_lock<std::mutex> lk(s->mu);
    for (;;) {
        bool progress = false;
        // 1. retire finished launches
        for (auto& sl : s->slots) {
            if (!sl.busy) continue;
            if (sl.status == MS_OK) {
                cudaError_t q = cudaEventQuery(sl.done);
                if (q == cudaErrorNotReady) continue;
                if (q != cudaSuccess) sl.status = MS_ERR_CUDA;
            }
            retire(s, sl, now_s());
            progress = true;
        }
        if (progress) s->done_cv.notify_all();
        // 2. start launches on the free slots: pending requests in arrival
        //    order, at most one per session, none of a running session.
        //    Merged: requests of one cost class (solver settings and size
        //    bucket, see cost_class) share a launch, one launch per class --
        //    a launch lasts as long as its slowest env, so a light session
        //    never waits on a heavy one.  Unmerged: one launch per request.
        std::vector<Slot*> free_slots;
        for (auto& sl : s->slots)
            if (!sl.busy) free_slots.push_back(&sl);
        bool wait_coalesce = false;
        if (!free_slots.empty() && !s->pending.empty() && s->opt.coalesce_us > 0.0 && !s->stop) {
            const Req& first = s->reqs[s->pending.front()];
            wait_coalesce = now_s() < first.t_arrive + s->opt.coalesce_us * 1e-6;
        }
        if (!free_slots.empty() && !s->pending.empty() && !wait_coalesce) {
            std::vector<std::pair<uint64_t, std::vector<std::pair<Req*, Session*>>>> groups;
            std::deque<uint64_t> keep;
            while (!s->pending.empty()) {
                uint64_t t = s->pending.front();
                s->pending.pop_front();
                Req& r = s->reqs[t];
                auto sit = s->sessions.find(r.session);
                if (sit == s->sessions.end()) {
                    r.done = true; r.status = MS_ERR_NOT_FOUND; r.t_done = now_s();
                    progress = true;
                    continue;
                }
                Session* se = sit->second;
                if (se->running) { keep.push_back(t); continue; }
                uint64_t k = s->opt.merge ? cost_class(se) : t;
                size_t gi = 0;
                while (gi < groups.size() && groups[gi].first != k) gi++;
                bool full = gi < groups.size() ? (!s->opt.merge || (s->opt.max_requests > 0 &&
                                                                    (int)groups[gi].second.size() >= s->opt.max_requests))
                                               : groups.size() >= free_slots.size();
                if (full) { keep.push_back(t); continue; }
                if (gi == groups.size()) groups.emplace_back(k, std::vector<std::pair<Req*, Session*>>());
                se->running = true;
                groups[gi].second.emplace_back(&r, se);
            }
            s->pending = std::move(keep);
            for (size_t gi = 0; gi < groups.size(); gi++) {
                Slot& sl = *free_slots[gi];
                sl.batch = std::move(groups[gi].second);
                sl.busy = true;
                sl.status = MS_OK;
                sl.envs = 0;
                double t0 = now_s();
                sl.t0 = t0;
                if (s->running++ == 0) s->busy_since = t0;
                lk.unlock();
                int st = s->opt.merge ? launch_merged(s, sl) : launch_single(s, sl);
                double t1 = now_s();
                if (st != MS_OK)
                    fprintf(stderr, "ms_server: launch of %zu request(s) failed (%d): %s\n", sl.batch.size(), st,
                            ms_last_error());
                lk.lock();
                s->stage_t.push_back(t1 - t0);
                sl.status = st;
                progress = true;
            }
        }
        if (progress) continue;
        bool any_busy = s->running > 0;
        if (s->stop && s->pending.empty() && !any_busy) break;
        if (any_busy || wait_coalesce || !s->pending.empty())
            s->cv.wait_for(lk, std::chrono::microseconds(20));    // poll the events in flight
        else
            s->cv.wait(lk, [&] { return s->stop || !s->pending.empty(); });
    }
    s->done_cv.notify_all();
}

extern "C" double ms_server_now(void) { return now_s(); }

extern "C" ms_status ms_server_create(size_t budget, const ms_server_options* opt, ms_server** out) {
    if (!out) return sfail(MS_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (opt && (opt->max_inflight < 0 || opt->max_inflight > 64))
        return sfail(MS_ERR_INVALID_ARG, "max_inflight must be 0..64");
    ms_server* s = new ms_server();
    s->budget = budget;
    if (opt) s->opt = *opt;
    if (s->opt.max_inflight == 0) s->opt.max_inflight = 16;
    cudaGetDevice(&s->device);
    cudaDeviceGetAttribute(&s->sm_count, cudaDevAttrMultiProcessorCount, s->device);
    cudaDeviceGetAttribute(&s->smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, s->device);
    // raised to the device maximum once: graphs of every layout stay valid
    cudaFuncSetAttribute((const void*)k_multi<MULTI_G>, cudaFuncAttributeMaxDynamicSharedMemorySize, s->smem_optin);
    fused_preload();                         // no module load on the worker's first launch of a kernel
    // sessions come and go: keep freed pool memory for the next session
    // instead of returning it to the driver at every synchronisation
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, s->device) == cudaSuccess) {
        uint64_t thr = ~0ull;
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
    }
    s->slots.resize((size_t)s->opt.max_inflight);
    for (auto& sl : s->slots) {
        if (cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&sl.done, cudaEventDisableTiming) != cudaSuccess) {
            for (auto& t : s->slots) {
                if (t.done) cudaEventDestroy(t.done);
                if (t.stream) cudaStreamDestroy(t.stream);
            }
            delete s;
            return sfail(MS_ERR_CUDA, "stream or event creation failed");
        }
    }
    s->worker = std::thread(worker_loop, s);
    *out = s;
    return MS_OK;
}

extern "C" ms_status ms_server_open(ms_server* s, const ms_body_desc* bodies, const int32_t* body_off,
                                    const ms_joint_desc* joints, const int32_t* joint_off, int n_envs,
                                    const ms_sim_params* p, uint64_t* session) {
    if (!s || !session || !p || !body_off || !joint_off) return sfail(MS_ERR_INVALID_ARG, "NULL argument");
    if (n_envs < 1 || n_envs > 1024) return sfail(MS_ERR_INVALID_ARG, "a session owns 1..1024 envs");
    size_t est = 0;
    ms_status st = ms_estimate_bytes(body_off, joint_off, n_envs, p, &est);
    if (st) return st;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        if (s->used + est > s->budget) {
            s->sessions_rejected++;
            return sfail(MS_ERR_NOT_ADMITTED, "session needs ~%zu B; %zu of %zu B in use", est, s->used, s->budget);
        }
        s->used += est;                      // reserve while the batch is built
    }
    ms_batch* b = nullptr;
    {
        std::lock_guard<std::mutex> dk(s->dev_mu);
        st = ms_create_batch_flat(bodies, body_off, joints, joint_off, n_envs, p, &b);
        // choose the kernel and its placement here, on the client's thread,
        // not at the session's first step on the worker (occupancy queries,
        // its workspace allocation)
        ms_tuning t{};
        if (st == MS_OK && (st = ms_get_tuning(b, &t)) != MS_OK) {
            ms_destroy(b);
            b = nullptr;
        }
    }
    std::lock_guard<std::mutex> lk(s->mu);
    if (st != MS_OK) {
        s->used -= est;
        return st;
    }
    Session* se = new Session();
    se->b = b;
    se->p = *p;
    batch_dims(b, &se->E, &se->A, &se->max_nb, &se->max_nj);
    se->bytes = est;
    se->id = s->next_session++;
    s->sessions[se->id] = se;
    s->sessions_admitted++;
    *session = se->id;
    return MS_OK;
}

// Frees a session's device memory; the caller has removed it from the
// session table and released its bytes from the budget.
static void free_session(ms_server* s, Session* se) {
    std::lock_guard<std::mutex> dk(s->dev_mu);
    ms_destroy(se->b);
    delete se;
}

extern "C" ms_status ms_server_close(ms_server* s, uint64_t session) {
    if (!s) return sfail(MS_ERR_INVALID_ARG, "NULL server");
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->sessions.find(session);
    if (it == s->sessions.end()) return sfail(MS_ERR_NOT_FOUND, "unknown session %llu", (unsigned long long)session);
    Session* se = it->second;
    s->done_cv.wait(lk, [&] { return se->inflight == 0; });
    s->sessions.erase(it);
    s->used -= se->bytes;
    lk.unlock();                              // the worker keeps serving while the memory is freed
    free_session(s, se);
    return MS_OK;
}

extern "C" ms_status ms_server_submit(ms_server* s, uint64_t session, const float* actions, uint64_t* ticket) {
    if (!s || !ticket) return sfail(MS_ERR_INVALID_ARG, "NULL argument");
    double t = now_s();
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->sessions.find(session);
    if (it == s->sessions.end()) return sfail(MS_ERR_NOT_FOUND, "unknown session %llu", (unsigned long long)session);
    Session* se = it->second;
    uint64_t tk = s->next_ticket++;
    Req r;
    r.ticket = tk;
    r.session = session;
    r.t_arrive = t;
    if (actions && se->A > 0) r.act.assign(actions, actions + (size_t)se->E * se->A);
    s->reqs.emplace(tk, std::move(r));
    s->pending.push_back(tk);
    se->inflight++;
    *ticket = tk;
    s->cv.notify_one();
    return MS_OK;
}

extern "C" ms_status ms_server_poll(ms_server* s, uint64_t ticket, ms_request_result* out) {
    if (!s || !out) return sfail(MS_ERR_INVALID_ARG, "NULL argument");
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end()) return sfail(MS_ERR_NOT_FOUND, "unknown ticket");
    const Req& r = it->second;
    out->ticket = r.ticket; out->session = r.session; out->done = r.done; out->status = r.status;
    out->t_arrive = r.t_arrive; out->t_done = r.t_done; out->latency = r.done ? r.t_done - r.t_arrive : 0.0;
    out->launch_envs = r.launch_envs;
    if (!r.done) return MS_ERR_BUSY;
    s->reqs.erase(it);
    return MS_OK;
}

extern "C" ms_status ms_server_drain(ms_server* s) {
    if (!s) return sfail(MS_ERR_INVALID_ARG, "NULL server");
    std::unique_lock<std::mutex> lk(s->mu);
    s->done_cv.wait(lk, [&] {
        if (!s->pending.empty() || s->running > 0) return false;
        for (auto& kv : s->sessions) if (kv.second->inflight) return false;
        return true;
    });
    return MS_OK;
}

extern "C" ms_status ms_server_copy_state(ms_server* s, uint64_t session, float* dst) {
    if (!s || !dst) return sfail(MS_ERR_INVALID_ARG, "NULL argument");
    ms_batch* b = nullptr;
    {
        std::unique_lock<std::mutex> lk(s->mu);
        auto it = s->sessions.find(session);
        if (it == s->sessions.end()) return sfail(MS_ERR_NOT_FOUND, "unknown session");
        Session* se = it->second;
        s->done_cv.wait(lk, [&] { return se->inflight == 0; });
        b = se->b;
    }
    std::lock_guard<std::mutex> dk(s->dev_mu);
    ms_status st = ms_copy_state(b, dst, 0, nullptr);
    if (st) return st;
    return cudaDeviceSynchronize() == cudaSuccess ? MS_OK : sfail(MS_ERR_CUDA, "copy failed");
}

extern "C" ms_status ms_server_stats_get(ms_server* s, ms_server_stats* out) {
    if (!s || !out) return sfail(MS_ERR_INVALID_ARG, "NULL argument");
    std::lock_guard<std::mutex> lk(s->mu);
    memset(out, 0, sizeof(*out));
    out->sessions_open = s->sessions.size();
    out->sessions_admitted = s->sessions_admitted;
    out->sessions_rejected = s->sessions_rejected;
    out->requests_done = s->requests_done;
    out->launches = s->launches;
    out->env_steps = s->env_steps;
    out->hbm_used = s->used;
    out->hbm_budget = s->budget;
    out->busy_s = s->busy + (s->running > 0 ? now_s() - s->busy_since : 0.0);
    out->graph_captures = s->graph_captures;
    // nearest-rank percentile of a sorted sample
    auto pct = [](const std::vector<double>& v, double q) {
        size_t k = (size_t)std::min<double>(v.size() - 1, std::max(0.0, std::ceil(q * v.size()) - 1));
        return v[k];
    };
    if (!s->lat.empty()) {
        std::vector<double> v = s->lat;
        std::sort(v.begin(), v.end());
        out->p50 = pct(v, 0.50);
        out->p99 = pct(v, 0.99);
        double sum = 0;
        for (double x : v) sum += x;
        out->mean = sum / v.size();
    }
    if (!s->launch_t.empty()) {
        std::vector<double> v = s->launch_t;
        std::sort(v.begin(), v.end());
        out->launch_p50 = pct(v, 0.50);
        out->launch_p99 = pct(v, 0.99);
        out->launch_max = v.back();
    }
    if (!s->queue_t.empty()) {
        std::vector<double> v = s->queue_t;
        std::sort(v.begin(), v.end());
        out->queue_p50 = pct(v, 0.50);
        out->queue_p99 = pct(v, 0.99);
    }
    if (!s->stage_t.empty()) {
        std::vector<double> v = s->stage_t;
        std::sort(v.begin(), v.end());
        out->stage_p99 = pct(v, 0.99);
        out->stage_max = v.back();
    }
    return MS_OK;
}

extern "C" ms_status ms_server_reset_stats(ms_server* s) {
    if (!s) return sfail(MS_ERR_INVALID_ARG, "NULL server");
    std::lock_guard<std::mutex> lk(s->mu);
    s->lat.clear();
    s->launch_t.clear();
    s->queue_t.clear();
    s->stage_t.clear();
    s->requests_done = s->launches = s->env_steps = 0;
    s->graph_captures = 0;
    s->busy = 0.0;
    if (s->running > 0) s->busy_since = now_s();
    return MS_OK;
}

extern "C" ms_status ms_server_destroy(ms_server* s) {
    if (!s) return MS_OK;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
    }
    s->cv.notify_all();
    if (s->worker.joinable()) s->worker.join();
    // sessions first: a batch stepped by ms_step remembers the slot stream
    // of its last step and synchronises it when destroyed
    for (auto& kv : s->sessions) {
        s->used -= kv.second->bytes;
        free_session(s, kv.second);
    }
    s->sessions.clear();
    for (auto& sl : s->slots) free_slot(s, sl);
    for (void* p : s->retired_host) cudaFreeHost(p);
    delete s;
    return MS_OK;
}
