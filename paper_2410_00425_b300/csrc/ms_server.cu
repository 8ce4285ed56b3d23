// Step server (include/ms_server.h).
//
// Sessions are ordinary batches (ms_create_batch_flat) whose state stays
// resident.  Clients queue step requests from any thread; one worker thread
// takes every pending request (at most one per session, in arrival order),
// stages their drive targets, and runs one launch of k_multi over the union
// of their envs: a persistent kernel whose work list names (session, env)
// pairs and which reads each env's batch view from a device table, so
// sessions of different scene types and solver parameters share a launch.
// The launch (queue reset + kernel) is captured once per workspace layout
// in a CUDA graph whose kernel parameters are updated per launch.  Every
// request is stamped with its host arrival and completion times.
#include <cuda_runtime.h>

#include <algorithm>
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

// One env per warp (G = 32): envs of different sessions in a launch may
// have different substep and iteration counts, so no two share a warp.
__global__ void __launch_bounds__(256, 2) k_multi(const DevBatch* __restrict__ batches, const float* const* actions,
                                                  const int2* work, int n_work, Layout L, int* queue,
                                                  char* gscratch) {
    extern __shared__ __align__(16) char smem[];
    int warp = threadIdx.x >> 5, wl = threadIdx.x & 31;
    Grp g;
    g.lane = wl; g.size = 32; g.base = 0;
    char* s = smem + (size_t)warp * L.s_bytes;
    size_t gslot = (size_t)blockIdx.x * (blockDim.x >> 5) + warp;
    char* gl = gscratch + gslot * (size_t)L.g_bytes;
    auto at = [](char* base, int off) { return base + off; };

    EnvView e;
    e.x = (float4*)at(s, L.x); e.q = (float4*)at(s, L.q); e.v = (float4*)at(s, L.v); e.w = (float4*)at(s, L.w);
    float4* shp = (float4*)at(s, L.shape);
    float4* inv = (float4*)at(s, L.inv);
    int2* meta = (int2*)at(s, L.meta);
    unsigned long long* adj = (unsigned long long*)at(s, L.adj);
    float4* jf = (float4*)at(s, L.jf);
    float4* jp = (float4*)at(s, L.jp);
    int4* jm = (int4*)at(s, L.jm);
    e.shape = shp; e.inv = inv; e.meta = meta; e.adj = adj; e.jf = jf; e.jp = jp; e.jm = jm;
    e.jt = (float*)at(s, L.jt);
    e.iw = (float4*)at(s, L.iw);
    char* lb = L.lists_shared ? s : gl;
    e.cons = (int4*)at(lb, L.cons);
    e.colr = (int*)at(lb, L.colr);
    e.scons = (int4*)at(lb, L.scons);
    e.lam = (float*)at(lb, L.lam);
    e.color_off = (int*)at(s, L.color_off);
    e.used = (unsigned long long*)at(s, L.used);
    e.cnt = (int*)at(s, L.cnt);
    e.aabb = (float4*)at(gl, L.aabb);
    e.pairs = (int*)at(gl, L.pairs);
    e.man = (int4*)at(gl, L.man);
    e.pts = (float4*)at(gl, L.pts);
    e.rows = L.rows_s >= 0 ? (Row*)at(s, L.rows_s) : (Row*)at(gl, L.rows_g);
    e.status = (unsigned*)at(s, L.status);
    e.rec_man = nullptr; e.rec_pts = nullptr; e.rec_cnt = nullptr;

    for (;;) {
        int t = 0;
        if (wl == 0) t = atomicAdd(queue, 1);
        t = __shfl_sync(FULL_MASK, t, 0);
        if (t >= n_work) break;
        int2 it = work[t];
        const DevBatch& D = batches[it.x];
        int env = it.y;
        int b0 = D.body_off[env], j0 = D.joint_off[env];
        int nb = D.body_off[env + 1] - b0, nj = D.joint_off[env + 1] - j0;
        for (int i = wl; i < nb; i += 32) {
            e.x[i] = D.x[b0 + i]; e.q[i] = D.q[b0 + i]; e.v[i] = D.v[b0 + i]; e.w[i] = D.w[b0 + i];
            shp[i] = D.shape[b0 + i]; inv[i] = D.inv[b0 + i]; meta[i] = D.meta[b0 + i]; adj[i] = D.adj[b0 + i];
        }
        for (int j = wl; j < nj; j += 32) {
            const float4* src = D.jf + 4 * (size_t)(j0 + j);
            jf[4 * j] = src[0]; jf[4 * j + 1] = src[1]; jf[4 * j + 2] = src[2]; jf[4 * j + 3] = src[3];
            jp[j] = D.jp[j0 + j]; jm[j] = D.jm[j0 + j]; e.jt[j] = D.jt[j0 + j];
        }
        if (wl == 0) *e.status = D.status[env];
        g.sync();
        bool frozen = (*e.status & ST_NAN) != 0;
        e.nb = frozen ? 0 : nb;
        e.nj = frozen ? 0 : nj;
        DevParams P = D.P;
        const float* act = actions[it.x] ? actions[it.x] + (size_t)env * D.A : nullptr;
        stage_actions(e, g, act, D.A);
        stage_broadphase(e, g, P);
        stage_narrowphase(e, g, P);
        stage_color(e, g);
        for (int sub = 0; sub < P.substeps; sub++) {
            stage_prep(e, g, P);
            stage_sweep(e, g, 0);
            for (int k = 0; k < P.pos_iters; k++) stage_sweep(e, g, 1);
            stage_integrate(e, g, P);
            for (int k = 0; k < P.vel_iters; k++) stage_sweep(e, g, 2);
        }
        stage_check(e, g);
        for (int i = wl; i < nb; i += 32) {
            D.x[b0 + i] = e.x[i]; D.q[b0 + i] = e.q[i]; D.v[b0 + i] = e.v[i]; D.w[b0 + i] = e.w[i];
        }
        for (int j = wl; j < nj; j += 32) D.jt[j0 + j] = e.jt[j];
        if (wl == 0) D.status[env] = *e.status;
        g.sync();
    }
}

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
    float* d_act = nullptr;       // [E][A] drive targets of the request being served
    int inflight = 0;             // queued requests not yet completed
    bool closing = false;
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

ms_status sfail(ms_status code, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    set_last_error(buf);
    return code;
}

}  // namespace

struct ms_server {
    size_t budget = 0, used = 0;
    ms_server_options opt{1, 0, 0.0};
    int device = 0, sm_count = 0, smem_optin = 0;
    std::mutex mu;
    std::condition_variable cv, done_cv;
    std::thread worker;
    bool stop = false;
    uint64_t next_session = 1, next_ticket = 1;
    std::unordered_map<uint64_t, Session*> sessions;
    std::deque<uint64_t> pending;
    std::unordered_map<uint64_t, Req> reqs;
    cudaStream_t stream = nullptr;
    // device tables of a merged launch, grown on demand
    DevBatch* d_batches = nullptr;
    const float** d_acts = nullptr;
    int2* d_work = nullptr;
    int* d_queue = nullptr;
    char* d_gscratch = nullptr;
    size_t cap_batches = 0, cap_work = 0, cap_gscratch = 0;
    DevBatch* h_batches = nullptr;        // pinned staging
    const float** h_acts = nullptr;
    int2* h_work = nullptr;
    std::map<GraphKey, GraphE> graphs;
    // statistics
    uint64_t sessions_admitted = 0, sessions_rejected = 0, requests_done = 0, launches = 0, env_steps = 0;
    std::vector<double> lat;
    double busy = 0.0;
};

static void free_tables(ms_server* s) {
    cudaFree(s->d_batches); cudaFree(s->d_acts); cudaFree(s->d_work); cudaFree(s->d_queue); cudaFree(s->d_gscratch);
    cudaFreeHost(s->h_batches); cudaFreeHost(s->h_acts); cudaFreeHost(s->h_work);
    s->d_batches = nullptr; s->d_acts = nullptr; s->d_work = nullptr; s->d_queue = nullptr; s->d_gscratch = nullptr;
    s->h_batches = nullptr; s->h_acts = nullptr; s->h_work = nullptr;
}

static cudaError_t grow_tables(ms_server* s, size_t nb, size_t nw, size_t gbytes) {
    cudaError_t e = cudaSuccess;
    if (nb > s->cap_batches) {
        size_t c = std::max(nb, 2 * s->cap_batches);
        cudaFree(s->d_batches); cudaFree(s->d_acts); cudaFreeHost(s->h_batches); cudaFreeHost(s->h_acts);
        if ((e = cudaMalloc(&s->d_batches, c * sizeof(DevBatch))) != cudaSuccess) return e;
        if ((e = cudaMalloc((void**)&s->d_acts, c * sizeof(float*))) != cudaSuccess) return e;
        if ((e = cudaMallocHost(&s->h_batches, c * sizeof(DevBatch))) != cudaSuccess) return e;
        if ((e = cudaMallocHost((void**)&s->h_acts, c * sizeof(float*))) != cudaSuccess) return e;
        s->cap_batches = c;
    }
    if (nw > s->cap_work) {
        size_t c = std::max(nw, 2 * s->cap_work);
        cudaFree(s->d_work); cudaFreeHost(s->h_work);
        if ((e = cudaMalloc(&s->d_work, c * sizeof(int2))) != cudaSuccess) return e;
        if ((e = cudaMallocHost(&s->h_work, c * sizeof(int2))) != cudaSuccess) return e;
        s->cap_work = c;
    }
    if (gbytes > s->cap_gscratch) {
        cudaFree(s->d_gscratch);
        if ((e = cudaMalloc(&s->d_gscratch, gbytes)) != cudaSuccess) return e;
        s->cap_gscratch = gbytes;
    }
    if (!s->d_queue && (e = cudaMalloc(&s->d_queue, 256)) != cudaSuccess) return e;
    return cudaSuccess;
}

// One merged launch over the sessions of `batch` (one request each).
static int run_merged(ms_server* s, std::vector<std::pair<Req*, Session*>>& batch) {
    int mb = 1, mj = 0, pc = 1, cc = 1;
    size_t nwork = 0;
    for (auto& rs : batch) {
        Session* se = rs.second;
        mb = std::max(mb, se->max_nb); mj = std::max(mj, se->max_nj);
        pc = std::max(pc, se->p.pair_capacity); cc = std::max(cc, se->p.contact_capacity);
        nwork += (size_t)se->E;
    }
    const int warps = 2;
    Layout L = make_layout(mb, mj, pc, cc, true, true, true);
    if ((size_t)L.s_bytes * warps > (size_t)s->smem_optin) L = make_layout(mb, mj, pc, cc, true, false, true);
    if ((size_t)L.s_bytes * warps > (size_t)s->smem_optin) L = make_layout(mb, mj, pc, cc, true, false, false);
    size_t smem = (size_t)L.s_bytes * warps;
    if (smem > (size_t)s->smem_optin) return MS_ERR_INVALID_ARG;
    // raised to the device maximum: graphs of other layouts stay valid
    cudaFuncSetAttribute((const void*)k_multi, cudaFuncAttributeMaxDynamicSharedMemorySize, s->smem_optin);
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, (const void*)k_multi, 32 * warps, smem);
    if (per_sm < 1) return MS_ERR_INVALID_ARG;
    // a fixed grid per layout keeps one graph per layout; warps without work exit at once
    int grid = per_sm * s->sm_count;
    if (grow_tables(s, batch.size(), nwork, (size_t)grid * warps * L.g_bytes) != cudaSuccess) return MS_ERR_OOM;
    size_t w = 0;
    for (size_t i = 0; i < batch.size(); i++) {
        Session* se = batch[i].second;
        Req* r = batch[i].first;
        s->h_batches[i] = batch_dev(se->b);
        s->h_acts[i] = nullptr;
        if (!r->act.empty()) {
            cudaMemcpyAsync(se->d_act, r->act.data(), r->act.size() * sizeof(float), cudaMemcpyHostToDevice, s->stream);
            s->h_acts[i] = se->d_act;
        }
        for (int e = 0; e < se->E; e++) s->h_work[w++] = make_int2((int)i, e);
    }
    // heaviest envs first (the work queue is popped in order)
    std::stable_sort(s->h_work, s->h_work + w, [&](int2 a, int2 b) {
        return batch[a.x].second->max_nj * 8 + batch[a.x].second->max_nb > batch[b.x].second->max_nj * 8 + batch[b.x].second->max_nb;
    });
    cudaMemcpyAsync(s->d_batches, s->h_batches, batch.size() * sizeof(DevBatch), cudaMemcpyHostToDevice, s->stream);
    cudaMemcpyAsync(s->d_acts, s->h_acts, batch.size() * sizeof(float*), cudaMemcpyHostToDevice, s->stream);
    cudaMemcpyAsync(s->d_work, s->h_work, w * sizeof(int2), cudaMemcpyHostToDevice, s->stream);
    GraphKey key{L.s_bytes, L.g_bytes, 32 * warps, grid};
    auto it = s->graphs.find(key);
    const DevBatch* a0 = s->d_batches;
    const float* const* a1 = s->d_acts;
    const int2* a2 = s->d_work;
    int a3 = (int)w;
    Layout a4 = L;
    int* a5 = s->d_queue;
    char* a6 = s->d_gscratch;
    void* args[] = {(void*)&a0, (void*)&a1, (void*)&a2, (void*)&a3, (void*)&a4, (void*)&a5, (void*)&a6};
    if (it == s->graphs.end()) {
        GraphE ge;
        cudaGraph_t g;
        if (cudaStreamBeginCapture(s->stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return MS_ERR_CUDA;
        cudaMemsetAsync(s->d_queue, 0, sizeof(int), s->stream);
        cudaLaunchKernel((const void*)k_multi, dim3(grid), dim3(32 * warps), args, smem, s->stream);
        if (cudaStreamEndCapture(s->stream, &g) != cudaSuccess) return MS_ERR_CUDA;
        if (cudaGraphInstantiate(&ge.exec, g, 0) != cudaSuccess) return MS_ERR_CUDA;
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
        it = s->graphs.emplace(key, ge).first;
    } else {
        cudaKernelNodeParams kp = it->second.kp;
        kp.kernelParams = args;
        kp.extra = nullptr;
        if (cudaGraphExecKernelNodeSetParams(it->second.exec, it->second.kernel, &kp) != cudaSuccess) return MS_ERR_CUDA;
    }
    if (cudaGraphLaunch(it->second.exec, s->stream) != cudaSuccess) return MS_ERR_CUDA;
    if (cudaStreamSynchronize(s->stream) != cudaSuccess) return MS_ERR_CUDA;
    s->launches++;
    s->env_steps += w;
    for (auto& rs : batch) rs.first->launch_envs = (int)w;
    return MS_OK;
}

static int run_single(ms_server* s, Req* r, Session* se) {
    const float* act = nullptr;
    if (!r->act.empty()) {
        cudaMemcpyAsync(se->d_act, r->act.data(), r->act.size() * sizeof(float), cudaMemcpyHostToDevice, s->stream);
        act = se->d_act;
    }
    int st = ms_step(se->b, act, 1, s->stream);
    if (st) return st;
    if (cudaStreamSynchronize(s->stream) != cudaSuccess) return MS_ERR_CUDA;
    s->launches++;
    s->env_steps += se->E;
    r->launch_envs = se->E;
    return MS_OK;
}

static void worker_loop(ms_server* s) {
    cudaSetDevice(s->device);
    std::unique_lock<std::mutex> lk(s->mu);
    for (;;) {
        s->cv.wait(lk, [&] { return s->stop || !s->pending.empty(); });
        if (s->stop && s->pending.empty()) break;
        if (s->opt.coalesce_us > 0.0) {
            double until = now_s() + s->opt.coalesce_us * 1e-6;
            while (!s->stop && now_s() < until) {
                lk.unlock();
                std::this_thread::yield();
                lk.lock();
            }
        }
        // take pending requests in arrival order, at most one per session
        std::vector<std::pair<Req*, Session*>> batch;
        std::unordered_map<uint64_t, bool> taken;
        std::deque<uint64_t> keep;
        while (!s->pending.empty()) {
            uint64_t t = s->pending.front();
            s->pending.pop_front();
            Req& r = s->reqs[t];
            auto sit = s->sessions.find(r.session);
            bool lim = s->opt.max_requests > 0 && (int)batch.size() >= s->opt.max_requests;
            if (sit == s->sessions.end()) { r.done = true; r.status = MS_ERR_NOT_FOUND; r.t_done = now_s(); continue; }
            if (taken.count(r.session) || lim || (!s->opt.merge && !batch.empty())) { keep.push_back(t); continue; }
            taken[r.session] = true;
            batch.emplace_back(&r, sit->second);
        }
        s->pending = std::move(keep);
        if (batch.empty()) { s->done_cv.notify_all(); continue; }
        lk.unlock();
        double t0 = now_s();
        int st = s->opt.merge ? run_merged(s, batch) : run_single(s, batch[0].first, batch[0].second);
        double t1 = now_s();
        if (st != MS_OK) fprintf(stderr, "ms_server: launch of %zu request(s) failed (%d): %s\n", batch.size(), st,
                                 ms_last_error());
        lk.lock();
        s->busy += t1 - t0;
        for (auto& rs : batch) {
            Req* r = rs.first;
            r->done = true;
            r->status = st;
            r->t_done = t1;
            r->act.clear();
            r->act.shrink_to_fit();
            rs.second->inflight--;
            s->lat.push_back(r->t_done - r->t_arrive);
            s->requests_done++;
        }
        s->done_cv.notify_all();
    }
}

extern "C" double ms_server_now(void) { return now_s(); }

extern "C" ms_status ms_server_create(size_t budget, const ms_server_options* opt, ms_server** out) {
    if (!out) return sfail(MS_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    ms_server* s = new ms_server();
    s->budget = budget;
    if (opt) s->opt = *opt;
    cudaGetDevice(&s->device);
    cudaDeviceGetAttribute(&s->sm_count, cudaDevAttrMultiProcessorCount, s->device);
    cudaDeviceGetAttribute(&s->smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, s->device);
    if (cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking) != cudaSuccess) {
        delete s;
        return sfail(MS_ERR_CUDA, "cudaStreamCreate failed");
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
    int max_nj = 0;
    for (int e = 0; e < n_envs; e++) max_nj = std::max(max_nj, joint_off[e + 1] - joint_off[e]);
    est += sizeof(float) * (size_t)n_envs * (size_t)std::max(max_nj, 1);
    {
        std::lock_guard<std::mutex> lk(s->mu);
        if (s->used + est > s->budget) {
            s->sessions_rejected++;
            return sfail(MS_ERR_NOT_ADMITTED, "session needs ~%zu B; %zu of %zu B in use", est, s->used, s->budget);
        }
        s->used += est;                      // reserve while the batch is built
    }
    ms_batch* b = nullptr;
    st = ms_create_batch_flat(bodies, body_off, joints, joint_off, n_envs, p, &b);
    Session* se = nullptr;
    if (st == MS_OK) {
        se = new Session();
        se->b = b;
        se->p = *p;
        batch_dims(b, &se->E, &se->A, &se->max_nb, &se->max_nj);
        se->bytes = est;
        if (cudaMalloc(&se->d_act, sizeof(float) * (size_t)se->E * (size_t)std::max(se->A, 1)) != cudaSuccess) {
            ms_destroy(b);
            delete se;
            se = nullptr;
            st = sfail(MS_ERR_OOM, "action buffer allocation failed");
        }
    }
    std::lock_guard<std::mutex> lk(s->mu);
    if (st != MS_OK) {
        s->used -= est;
        return st;
    }
    se->id = s->next_session++;
    s->sessions[se->id] = se;
    s->sessions_admitted++;
    *session = se->id;
    return MS_OK;
}

static void destroy_session(ms_server* s, Session* se) {
    ms_destroy(se->b);
    cudaFree(se->d_act);
    s->used -= se->bytes;
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
    destroy_session(s, se);
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
        if (!s->pending.empty()) return false;
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
    out->busy_s = s->busy;
    if (!s->lat.empty()) {
        std::vector<double> v = s->lat;
        std::sort(v.begin(), v.end());
        auto pct = [&](double q) {
            size_t k = (size_t)std::min<double>(v.size() - 1, std::max(0.0, std::ceil(q * v.size()) - 1));
            return v[k];
        };
        out->p50 = pct(0.50);
        out->p99 = pct(0.99);
        double sum = 0;
        for (double x : v) sum += x;
        out->mean = sum / v.size();
    }
    return MS_OK;
}

extern "C" ms_status ms_server_reset_stats(ms_server* s) {
    if (!s) return sfail(MS_ERR_INVALID_ARG, "NULL server");
    std::lock_guard<std::mutex> lk(s->mu);
    s->lat.clear();
    s->requests_done = s->launches = s->env_steps = 0;
    s->busy = 0.0;
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
    cudaStreamSynchronize(s->stream);
    for (auto& kv : s->sessions) destroy_session(s, kv.second);
    s->sessions.clear();
    for (auto& kv : s->graphs) {
        cudaGraphExecDestroy(kv.second.exec);
        cudaGraphDestroy(kv.second.graph);
    }
    free_tables(s);
    cudaStreamDestroy(s->stream);
    delete s;
    return MS_OK;
}
