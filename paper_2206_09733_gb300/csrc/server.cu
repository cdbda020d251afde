// Continuous-batching server: many independent solves share the GPU.
//
// A host thread runs this loop:
//   1. admit queued requests (FIFO) while the device-memory budget has room:
//      build the request's mesh, allocate its state, evaluate its initial
//      condition and arm its clock (t_final or n_steps);
//   2. group the running requests by (N, physics, surface flux, volume form,
//      precision, time scheme) and advance every group by one RK step with shared
//      launches: each kernel walks a table of items (one per request), so one
//      launch covers all requests of a group.  The launches of all groups
//      (and the clock gather of step 3) are captured into one CUDA graph,
//      replayed for as long as the set of running requests stays the same
//      and re-captured (updated in place where the topology allows) when a
//      request joins or leaves;
//   3. gather the clocks of all running requests into one small array, copy
//      it to pinned host memory and wait for it with a bounded poll;
//   4. retire finished requests (copy the state out, free the slot, stamp the
//      time) and go back to 1, so new requests join as soon as memory frees.
// Every element's arithmetic depends only on its own request, and the dt
// maxima are exact, so a request's result is the same alone and in any mix.
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <thread>
#include <tuple>
#include <unordered_map>
#include <vector>

#include "api_internal.h"

namespace hs3d {

struct ClockView {
    double t;
    long long step;
    int done;
    int bad;
};

__global__ void k_gather_clocks(const Item *items, int n, ClockView *out)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const Clock *c = items[i].clk;
    out[i].t = c->t;
    out[i].step = c->step;
    out[i].done = c->done;
    out[i].bad = c->bad;
}

enum ReqState { Q_QUEUED, Q_RUNNING, Q_DONE };

struct ServerReq {
    uint64_t id = 0;
    hs3d_request req{};
    std::vector<double> xyz;   // private copy of node coordinates, if given
    ReqState state = Q_QUEUED;
    hs3d_result res{};
    hs3d_mesh *mesh = nullptr;
    double *u = nullptr, *g = nullptr;
    size_t bytes = 0;
};

static size_t request_bytes(const hs3d_request &r)
{
    long long E = (long long)r.mesh.ex * r.mesh.ey * r.mesh.ez;
    long long n3 = (long long)(r.mesh.N + 1) * (r.mesh.N + 1) * (r.mesh.N + 1);
    return mesh_bytes(r.mesh.N, E, r.mesh.nodes) + 2 * sizeof(double) * (size_t)E * 5 * n3;
}

}  // namespace hs3d

using namespace hs3d;

struct hs3d_server {
    int device = 0;
    size_t budget = 0, in_use = 0;
    int max_batch = 256;
    double wait_limit_s = 120.0;
    int fault_alloc = 0;   // host-side fault injection: fail the next admissions' allocation
    std::mutex mu;
    std::condition_variable cv;
    bool stop = false;
    uint64_t next_id = 1;
    std::deque<ServerReq *> queue;
    std::vector<ServerReq *> running;
    std::unordered_map<uint64_t, ServerReq *> all;
    int64_t finished = 0;
    std::thread th;
    cudaStream_t stream = nullptr;
    std::chrono::steady_clock::time_point t0;
    // per-group device item tables and the clock gather buffers
    Item *d_items = nullptr;
    int d_items_cap = 0;
    ClockView *d_clk = nullptr, *h_clk = nullptr;
    int clk_cap = 0;
    cudaEvent_t ev = nullptr;
    // the captured step of the current set of running requests (ids in table order)
    cudaGraphExec_t gexec = nullptr;
    std::vector<uint64_t> gkey;
    // launch design (HS3D_LAUNCH_GRID / HS3D_LAUNCH_PERSISTENT), set from any thread; the step
    // thread re-captures when it differs from the design of the current graph (gmode)
    std::atomic<int> launch_mode{HS3D_LAUNCH_GRID};
    int gmode = HS3D_LAUNCH_GRID;
    // persistent design: the work table, item of every element of every group
    int *d_elem_item = nullptr;
    long long elem_cap = 0;

    double now() const
    {
        return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    }
};

namespace hs3d {

static void release(hs3d_server *S, ServerReq *r)
{
    if (r->u) cudaFree(r->u);
    if (r->g) cudaFree(r->g);
    if (r->mesh) mesh_free(r->mesh);
    r->u = r->g = nullptr;
    r->mesh = nullptr;
    S->in_use -= r->bytes;
}

// Build the request's slot.  Returns HS3D_OK, HS3D_ERR_NOMEM (retry later) or another error (fail it).
// Build a popped request's mesh, state and clock (called without the server
// lock: it touches only r and the server's private stream, so submit and
// poll stay responsive while a large mesh is set up).
static hs3d_status admit(hs3d_server *S, ServerReq *r)
{
    hs3d_mesh_desc d = r->req.mesh;
    d.node_xyz = r->xyz.empty() ? nullptr : r->xyz.data();
    hs3d_status st = mesh_build(&d, &r->mesh);
    if (st != HS3D_OK) return st;
    size_t sz = sizeof(double) * (size_t)r->mesh->E * 5 * r->mesh->n3;
    cudaError_t e = cudaMalloc(&r->u, sz);
    if (e == cudaSuccess) e = cudaMalloc(&r->g, sz);
    if (e != cudaSuccess) {
        cudaGetLastError();
        if (r->u) cudaFree(r->u);
        r->u = nullptr;
        mesh_free(r->mesh);
        r->mesh = nullptr;
        return fail(HS3D_ERR_NOMEM, "state allocation failed");
    }
    e = launch_init_state(r->mesh->N, r->mesh->E, r->mesh->X, r->req.ic, r->mesh->lo, r->mesh->hi, r->u, S->stream);
    Clock c{};
    c.t_final = r->req.t_final > 0.0 ? r->req.t_final : 0.0;
    c.nsteps = r->req.t_final > 0.0 ? 0 : r->req.n_steps;
    if (e == cudaSuccess) e = cudaMemcpyAsync(r->mesh->clk, &c, sizeof c, cudaMemcpyHostToDevice, S->stream);
    if (e == cudaSuccess) {
        // dt maxima of the initial state, for the first batched step
        Item it = make_item(r->mesh, &r->req.cfg, r->u, r->g, nullptr);
        e = prime_lambda(r->mesh->N, &r->req.cfg, single_batch(it), nullptr, S->stream);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(S->stream);
    if (e != cudaSuccess) {
        cudaFree(r->u);
        cudaFree(r->g);
        r->u = r->g = nullptr;
        mesh_free(r->mesh);
        r->mesh = nullptr;
        return cuda_fail(e, "request set-up");
    }
    r->bytes = request_bytes(r->req);
    return HS3D_OK;
}

static void finish(hs3d_server *S, ServerReq *r, hs3d_status st, const ClockView *cv)
{
    if (st == HS3D_OK && r->req.result_host) {
        size_t sz = sizeof(double) * (size_t)r->mesh->E * 5 * r->mesh->n3;
        cudaError_t e = cudaMemcpy(r->req.result_host, r->u, sz, cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) st = HS3D_ERR_CUDA;
    }
    if (cv) {
        r->res.t_sim = cv->t;
        r->res.steps = cv->step;
    }
    r->res.status = st;
    r->res.t_done = S->now();
    release(S, r);
    r->state = Q_DONE;
    S->finished++;
}

typedef std::tuple<int, int, int, int, int, int, int> BucketKey;

static BucketKey key_of(const ServerReq *r)
{
    const hs3d_solver_cfg &c = r->req.cfg;
    return BucketKey(r->req.mesh.N, c.physics, c.surface_flux, c.volume_form, c.precision, c.time_scheme,
                     r->req.mesh.nodes);
}

static cudaError_t ensure_capacity(hs3d_server *S, int n)
{
    if (n > S->d_items_cap) {
        if (S->d_items) cudaFree(S->d_items);
        int cap = std::max(n, 2 * S->d_items_cap);
        cudaError_t e = cudaMalloc(&S->d_items, sizeof(Item) * cap);
        if (e != cudaSuccess) {
            S->d_items = nullptr;
            S->d_items_cap = 0;
            return e;
        }
        S->d_items_cap = cap;
    }
    if (n > S->clk_cap) {
        if (S->d_clk) cudaFree(S->d_clk);
        if (S->h_clk) cudaFreeHost(S->h_clk);
        int cap = std::max(n, 2 * S->clk_cap);
        cudaError_t e = cudaMalloc(&S->d_clk, sizeof(ClockView) * cap);
        if (e == cudaSuccess) e = cudaMallocHost(&S->h_clk, sizeof(ClockView) * cap);
        if (e != cudaSuccess) {
            S->clk_cap = 0;
            return e;
        }
        S->clk_cap = cap;
    }
    return cudaSuccess;
}

static cudaError_t capture_step(hs3d_server *S, std::vector<ServerReq *> &run, std::vector<Item> &items,
                                const std::vector<std::pair<int, int>> &ranges,
                                const std::vector<const hs3d_solver_cfg *> &cfgs);

// One RK step for every running request, grouped into shared launches, then
// the clocks of all running requests land in S->h_clk (in `running` order).
static cudaError_t step_all(hs3d_server *S, std::vector<ServerReq *> &run)
{
    int n = (int)run.size();
    cudaError_t e = ensure_capacity(S, n);
    if (e != cudaSuccess) return e;
    std::vector<Item> items(n);
    std::map<BucketKey, std::vector<int>> buckets;
    for (int i = 0; i < n; ++i) buckets[key_of(run[i])].push_back(i);
    // order the item table bucket by bucket so each group is a contiguous range
    std::vector<int> order;
    std::vector<std::pair<int, int>> ranges;
    std::vector<const hs3d_solver_cfg *> cfgs;
    for (auto &kv : buckets) {
        for (size_t s = 0; s < kv.second.size(); s += S->max_batch) {
            int begin = (int)order.size();
            for (size_t k = s; k < std::min(kv.second.size(), s + (size_t)S->max_batch); ++k)
                order.push_back(kv.second[k]);
            ranges.push_back({begin, (int)order.size()});
            cfgs.push_back(&run[kv.second[0]]->req.cfg);
        }
    }
    std::vector<ServerReq *> sorted(n);
    for (int k = 0; k < n; ++k) sorted[k] = run[order[k]];
    run.swap(sorted);
    std::vector<uint64_t> key(n);
    for (int k = 0; k < n; ++k) key[k] = run[k]->id;
    const int mode = S->launch_mode.load();
    if (!(S->gexec && key == S->gkey && mode == S->gmode)) {
        S->gmode = mode;
        e = capture_step(S, run, items, ranges, cfgs);
        if (e != cudaSuccess) return e;
        S->gkey.swap(key);
    }
    e = cudaGraphLaunch(S->gexec, S->stream);
    if (e == cudaSuccess) e = cudaEventRecord(S->ev, S->stream);
    if (e != cudaSuccess) return e;
    // bounded wait for the step
    double t_start = S->now();
    while (true) {
        cudaError_t q = cudaEventQuery(S->ev);
        if (q == cudaSuccess) break;
        if (q != cudaErrorNotReady) return q;
        if (S->now() - t_start > S->wait_limit_s) return cudaErrorTimeout;
        std::this_thread::sleep_for(std::chrono::microseconds(50));
    }
    return cudaSuccess;
}

// Upload the item table of a new set of running requests (sorted into
// groups), capture one step of all groups plus the clock gather into a graph
// and make S->gexec execute it (updating the previous executable graph in
// place when the topology allows, else instantiating a new one).
static cudaError_t capture_step(hs3d_server *S, std::vector<ServerReq *> &run, std::vector<Item> &items,
                                const std::vector<std::pair<int, int>> &ranges,
                                const std::vector<const hs3d_solver_cfg *> &cfgs)
{
    const int n = (int)run.size();
    cudaError_t e = cudaSuccess;
    for (size_t b = 0; b < ranges.size(); ++b) {
        long long eb = 0, fb = 0;
        for (int k = ranges[b].first; k < ranges[b].second; ++k) {
            ServerReq *r = run[k];
            Item it = make_item(r->mesh, &r->req.cfg, r->u, r->g, nullptr);
            it.elem_begin = eb;
            it.face_begin = fb;
            eb += r->mesh->E;
            fb += 3LL * r->mesh->E;
            items[k] = it;
        }
    }
    e = cudaMemcpyAsync(S->d_items, items.data(), sizeof(Item) * n, cudaMemcpyHostToDevice, S->stream);
    if (e != cudaSuccess) return e;
    // persistent design: the work table (item of every element, group by group)
    const bool persistent = S->gmode == HS3D_LAUNCH_PERSISTENT;
    std::vector<long long> table_off(ranges.size(), 0);
    std::vector<int> table;
    if (persistent) {
        for (size_t b = 0; b < ranges.size(); ++b) {
            table_off[b] = (long long)table.size();
            for (int k = ranges[b].first; k < ranges[b].second; ++k)
                table.insert(table.end(), (size_t)run[k]->mesh->E, k - ranges[b].first);
        }
        if ((long long)table.size() > S->elem_cap) {
            const long long cap = std::max((long long)table.size(), 2 * S->elem_cap);
            if (S->d_elem_item) cudaFree(S->d_elem_item);
            S->d_elem_item = nullptr;
            S->elem_cap = 0;
            e = cudaMalloc(&S->d_elem_item, sizeof(int) * cap);
            if (e != cudaSuccess) return e;
            S->elem_cap = cap;
        }
        if (!table.empty())
            e = cudaMemcpyAsync(S->d_elem_item, table.data(), sizeof(int) * table.size(), cudaMemcpyHostToDevice,
                                S->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(S->stream);   // (the host table is freed on return)
        if (e != cudaSuccess) return e;
    }
    cudaGraph_t graph = nullptr;
    e = cudaStreamBeginCapture(S->stream, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return e;
    for (size_t b = 0; b < ranges.size() && e == cudaSuccess; ++b) {
        int lo = ranges[b].first, hi = ranges[b].second;
        Batch bt{};
        bt.nitems = hi - lo;
        if (bt.nitems == 1) {
            bt.single = items[lo];
            bt.single.elem_begin = 0;
            bt.single.face_begin = 0;
        }
        bt.items = S->d_items + lo;
        bt.total_elems = 0;
        for (int k = lo; k < hi; ++k) bt.total_elems += run[k]->mesh->E;
        bt.total_faces = 3 * bt.total_elems;
        bt.gauss = items[lo].gauss;
        if (persistent) {
            bt.persistent = 1;
            if (bt.nitems > 1) bt.elem_item = S->d_elem_item + table_off[b];
        }
        e = enqueue_rk3_step(run[lo]->req.mesh.N, cfgs[b], bt, 0.0, 0, S->stream);
    }
    if (e == cudaSuccess) {
        k_gather_clocks<<<(n + 127) / 128, 128, 0, S->stream>>>(S->d_items, n, S->d_clk);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(S->h_clk, S->d_clk, sizeof(ClockView) * n, cudaMemcpyDeviceToHost, S->stream);
    cudaError_t e2 = cudaStreamEndCapture(S->stream, &graph);
    if (e == cudaSuccess) e = e2;
    if (e == cudaSuccess && S->gexec) {
        cudaGraphExecUpdateResultInfo info;
        if (cudaGraphExecUpdate(S->gexec, graph, &info) != cudaSuccess) {
            cudaGetLastError();
            cudaGraphExecDestroy(S->gexec);
            S->gexec = nullptr;
        }
    }
    if (e == cudaSuccess && !S->gexec) e = cudaGraphInstantiate(&S->gexec, graph, 0);
    if (graph) cudaGraphDestroy(graph);
    if (e != cudaSuccess) {
        if (S->gexec) cudaGraphExecDestroy(S->gexec);
        S->gexec = nullptr;
        S->gkey.clear();
    }
    return e;
}

static void server_loop(hs3d_server *S)
{
    cudaSetDevice(S->device);
    std::unique_lock<std::mutex> lk(S->mu);
    while (!S->stop) {
        // 1. admission (FIFO while the budget has room)
        while (!S->queue.empty()) {
            ServerReq *r = S->queue.front();
            size_t need = request_bytes(r->req);
            if (S->in_use + need > S->budget && !S->running.empty()) break;
            S->queue.pop_front();
            S->in_use += need;   // reserved while the request is set up without the lock
            const bool inject = S->fault_alloc > 0;
            if (inject) S->fault_alloc--;
            lk.unlock();
            hs3d_status st = inject ? fail(HS3D_ERR_NOMEM, "injected allocation failure") : admit(S, r);
            lk.lock();
            if (st != HS3D_OK) S->in_use -= need;
            if (st == HS3D_ERR_NOMEM && !S->running.empty()) {
                S->queue.push_front(r);   // wait for memory to free
                break;
            }
            if (st != HS3D_OK) {
                r->res.status = st;
                r->res.t_done = S->now();
                r->state = Q_DONE;
                S->finished++;
                continue;
            }
            r->state = Q_RUNNING;
            r->res.t_admit = S->now();
            r->res.device_bytes = r->bytes;
            S->running.push_back(r);
        }
        if (S->running.empty()) {
            S->cv.wait_for(lk, std::chrono::milliseconds(20));
            continue;
        }
        // 2-3. one batched step, without holding the lock (submit/poll stay responsive)
        std::vector<ServerReq *> run = S->running;
        lk.unlock();
        cudaError_t e = step_all(S, run);
        lk.lock();
        S->running = run;   // step_all reorders by bucket
        // 4. retire
        std::vector<ServerReq *> keep;
        for (size_t k = 0; k < run.size(); ++k) {
            ServerReq *r = run[k];
            if (e != cudaSuccess) {
                finish(S, r, e == cudaErrorTimeout ? HS3D_ERR_TIMEOUT : HS3D_ERR_CUDA, nullptr);
                continue;
            }
            const ClockView &cv = S->h_clk[k];
            bool complete = (r->req.t_final > 0.0) ? cv.t >= r->req.t_final : cv.step >= r->req.n_steps;
            if (cv.bad) finish(S, r, cv.bad == 2 ? HS3D_ERR_TIMEOUT : HS3D_ERR_NONPHYSICAL, &cv);
            else if (complete || cv.done) finish(S, r, HS3D_OK, &cv);
            else keep.push_back(r);
        }
        if (e != cudaSuccess) cudaGetLastError();
        S->running.swap(keep);
    }
}

}  // namespace hs3d

extern "C" {

hs3d_status hs3d_server_create(size_t hbm_budget_bytes, int max_batch, hs3d_server **out)
{
    if (!out) return fail(HS3D_ERR_INVALID, "out is NULL");
    *out = nullptr;
    if (max_batch < 0) return fail(HS3D_ERR_INVALID, "max_batch < 0");
    hs3d_server *S = new (std::nothrow) hs3d_server();
    if (!S) return fail(HS3D_ERR_NOMEM, "host allocation failed");
    cudaError_t e = cudaGetDevice(&S->device);
    size_t fr = 0, tot = 0;
    if (e == cudaSuccess) e = cudaMemGetInfo(&fr, &tot);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&S->stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&S->ev, cudaEventDisableTiming);
    if (e != cudaSuccess) {
        if (S->stream) cudaStreamDestroy(S->stream);
        delete S;
        return cuda_fail(e, "server set-up");
    }
    S->budget = hbm_budget_bytes ? hbm_budget_bytes : (size_t)(0.9 * (double)fr);
    S->max_batch = max_batch ? max_batch : 256;
    if (const char *w = getenv("HS3D_SERVER_WAIT_LIMIT_S")) S->wait_limit_s = atof(w);
    if (const char *f = getenv("HS3D_FAULT_ALLOC_FAILURES")) S->fault_alloc = atoi(f);
    S->t0 = std::chrono::steady_clock::now();
    S->th = std::thread(server_loop, S);
    *out = S;
    return HS3D_OK;
}

void hs3d_server_destroy(hs3d_server *S)
{
    if (!S) return;
    {
        std::lock_guard<std::mutex> g(S->mu);
        S->stop = true;
    }
    S->cv.notify_all();
    if (S->th.joinable()) S->th.join();
    cudaStreamSynchronize(S->stream);
    for (auto &kv : S->all) {
        ServerReq *r = kv.second;
        if (r->state == Q_RUNNING) release(S, r);
        delete r;
    }
    if (S->gexec) cudaGraphExecDestroy(S->gexec);
    if (S->d_items) cudaFree(S->d_items);
    if (S->d_elem_item) cudaFree(S->d_elem_item);
    if (S->d_clk) cudaFree(S->d_clk);
    if (S->h_clk) cudaFreeHost(S->h_clk);
    if (S->ev) cudaEventDestroy(S->ev);
    if (S->stream) cudaStreamDestroy(S->stream);
    delete S;
}

hs3d_status hs3d_server_set_launch_mode(hs3d_server *S, int mode)
{
    if (!S) return fail(HS3D_ERR_INVALID, "server is NULL");
    if (mode != HS3D_LAUNCH_GRID && mode != HS3D_LAUNCH_PERSISTENT) return fail(HS3D_ERR_INVALID, "bad launch mode");
    S->launch_mode.store(mode);
    return HS3D_OK;
}

hs3d_status hs3d_submit(hs3d_server *S, const hs3d_request *req, uint64_t *ticket)
{
    if (!S || !req || !ticket) return fail(HS3D_ERR_INVALID, "server, request or ticket is NULL");
    hs3d_status st = validate_desc(&req->mesh);
    if (st == HS3D_OK) st = validate_cfg(&req->cfg);
    if (st == HS3D_OK && req->mesh.nodes == HS3D_NODES_GAUSS && req->cfg.volume_form != HS3D_VOL_STANDARD)
        st = fail(HS3D_ERR_UNSUPPORTED, "split volume forms need Gauss-Lobatto nodes");
    if (st != HS3D_OK) return st;
    if (!(req->t_final > 0.0) && req->n_steps <= 0)
        return fail(HS3D_ERR_INVALID, "request needs t_final > 0 or n_steps > 0");
    if (req->ic.kind != HS3D_IC_VORTEX && req->ic.kind != HS3D_IC_TGV)
        return fail(HS3D_ERR_INVALID, "bad initial condition kind");
    size_t need = request_bytes(*req);
    ServerReq *r = new (std::nothrow) ServerReq();
    if (!r) return fail(HS3D_ERR_NOMEM, "host allocation failed");
    r->req = *req;
    if (req->mesh.node_xyz) {
        size_t cnt = (size_t)req->mesh.ex * req->mesh.ey * req->mesh.ez * 3 * (req->mesh.N + 1) * (req->mesh.N + 1) *
                     (req->mesh.N + 1);
        r->xyz.assign(req->mesh.node_xyz, req->mesh.node_xyz + cnt);
    }
    r->req.mesh.node_xyz = nullptr;
    long long E = (long long)req->mesh.ex * req->mesh.ey * req->mesh.ez;
    r->res.status = HS3D_PENDING;
    r->res.dof = E * (req->mesh.N + 1) * (req->mesh.N + 1) * (req->mesh.N + 1);
    {
        std::lock_guard<std::mutex> g(S->mu);
        if (need > S->budget) {
            delete r;
            return fail(HS3D_ERR_NOMEM, "request needs %zu bytes, budget is %zu", need, S->budget);
        }
        r->id = S->next_id++;
        r->res.t_submit = S->now();
        S->all[r->id] = r;
        S->queue.push_back(r);
        *ticket = r->id;
    }
    S->cv.notify_all();
    return HS3D_OK;
}

hs3d_status hs3d_poll(hs3d_server *S, uint64_t ticket, hs3d_result *res)
{
    if (!S) return fail(HS3D_ERR_INVALID, "server is NULL");
    std::lock_guard<std::mutex> g(S->mu);
    auto it = S->all.find(ticket);
    if (it == S->all.end()) return fail(HS3D_ERR_INVALID, "unknown ticket %llu", (unsigned long long)ticket);
    ServerReq *r = it->second;
    if (res) *res = r->res;
    if (r->state != Q_DONE) return HS3D_PENDING;
    if (r->res.status != HS3D_OK) return fail(r->res.status, "request %llu failed", (unsigned long long)ticket);
    return HS3D_OK;
}

hs3d_status hs3d_server_stats(hs3d_server *S, int64_t *queued, int64_t *running, int64_t *finished, size_t *bytes)
{
    if (!S) return fail(HS3D_ERR_INVALID, "server is NULL");
    std::lock_guard<std::mutex> g(S->mu);
    if (queued) *queued = (int64_t)S->queue.size();
    if (running) *running = (int64_t)S->running.size();
    if (finished) *finished = S->finished;
    if (bytes) *bytes = S->in_use;
    return HS3D_OK;
}

}  // extern "C"
