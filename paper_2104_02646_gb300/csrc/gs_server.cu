// Continuous-batching server for system-identification gradient queries.
//
// A query is a whole gradient request (mesh, materials, dt, horizon, target;
// the paper's parameter-estimation loop, Sec. 3, with a position loss).  One
// worker thread owns the GPU work on its own stream and advances time in
// ticks.  Every tick launches the forward step kernels once and the adjoint
// step kernels once over the patches of *all* active queries; each query is
// in its own phase (forward chunk, segment recompute, or reverse steps), which
// its device record selects through the active flags and the tick-affine
// buffer indices (in = in_a + in_b * tick, ...).  Queries are admitted from a
// FIFO as slots and the HBM budget free up, so queries that arrive while
// others run join the next tick; finished queries leave and release memory.
// Mesh construction (ordering, patches, uploads, set-up kernels) runs on
// builder threads with their own streams, so the worker keeps ticking while
// new queries are prepared.  The worker uploads the device records of the
// active meshes when a phase changes and rebuilds the launch lists only when
// the set of active meshes changes.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <string>
#include <memory>
#include <new>
#include <mutex>
#include <thread>
#include <vector>

#include "gs_runtime.h"

using namespace gs;

namespace {

double now_s() {
    using namespace std::chrono;
    return duration<double>(steady_clock::now().time_since_epoch()).count();
}

enum Phase { P_FWD, P_REC, P_ADJ, P_FINISHING, P_DONE };

struct Query {
    uint64_t id = 0;
    // deep copy of the request
    gs_mesh_desc desc{};
    std::vector<int32_t> elems, hinges;
    std::vector<double> X, v0, mu, lam, rho, kb;
    std::vector<float> target;
    float dt = 0.f;
    int S = 0, K = 1, n_ck = 1;
    size_t bytes = 0;
    // run state
    gs_mesh* mesh = nullptr;
    Phase phase = P_FWD;
    int chunk = 0;          // forward chunk or segment index
    int t0 = 0;             // tick at which the phase started
    int steps = 0;          // steps of the phase
    int seg_steps = 0;      // steps of the current reverse segment
    int done = 0;           // steps done in the phase
    bool cancelled = false;
    gs_status build_status = GS_OK;
    std::string build_error;
    // results
    Buf g_dev;              // device gradients
    double* h_stage = nullptr;  // pinned host staging
    size_t stage_bytes = 0;
    cudaEvent_t ev = nullptr;
    gs_result res{};
    bool ready = false;
    double t_submit = 0, t_admit = 0, t_done = 0;
};

// Checkpoint interval of a query: the server's fixed K, else K = 1 (every
// state kept: one forward phase and one reverse phase, no recomputation)
// when those states take at most 1/32 of the budget, else about sqrt(S).
size_t estimate_bytes(const gs_mesh_desc& d, int S, int K);
int query_K(const gs_server_opts& o, const gs_mesh_desc& d, int S) {
    if (o.K > 0) return std::min(o.K, std::max(S, 1));
    if (o.hbm_budget_bytes == 0 || estimate_bytes(d, S, 1) <= o.hbm_budget_bytes / 32) return 1;
    return std::max(1, (int)std::ceil(std::sqrt((double)std::max(S, 1))));
}

size_t estimate_bytes(const gs_mesh_desc& d, int S, int K) {
    const size_t N = d.n_nodes, E = d.n_elems, B = d.kind == GS_CLOTH ? d.n_hinges : 0;
    const int n_ck = std::max(1, (S + K - 1) / K);
    const size_t bufs = 2 + n_ck + K;
    return E * 200 + B * 80 + N * (48 * bufs + 160) + ((size_t)1 << 20);
}

}  // namespace

struct gs_server {
    gs_ctx* ctx = nullptr;
    gs_server_opts opts{};
    cudaStream_t stream = nullptr;
    std::thread worker;
    std::mutex mu;
    std::condition_variable cv;      // wakes the worker
    std::condition_variable cv_done; // wakes pollers
    bool stop = false;
    bool failed = false;             // the worker stopped on a host-side exception
    uint64_t next_id = 1;
    std::deque<Query*> pending;
    std::deque<Query*> to_build;     // admitted, waiting for a builder thread
    std::vector<Query*> built;       // mesh ready, not yet started by the worker
    int building = 0;                // queries a builder thread holds
    std::vector<std::thread> builders;
    std::condition_variable cv_build;  // wakes builder threads
    std::vector<Query*> active;      // admitted, in some phase
    std::map<uint64_t, Query*> all;  // every query not yet collected
    size_t admitted = 0;
    uint64_t submitted = 0, completed = 0, rejected = 0;
    std::vector<double> latencies;
    double busy_since = -1.0, busy_time = 0.0, elem_steps = 0.0;
    LaunchSet ls;
    bool ls_valid = false;  // ls holds exactly the meshes of `active`
    bool ls_dirty = false;  // a query left: rebuild before the next launch
    int tick = 0;
    std::deque<cudaEvent_t> tick_events;
    std::vector<cudaEvent_t> free_events;
    // worker-time breakdown (seconds) and counters
    double t_build = 0, t_start = 0, t_rebuild = 0, t_sync = 0, t_wait = 0;
    uint64_t n_ticks = 0, n_rebuilds = 0, n_syncs = 0;

    void run();
    void run_loop();
    void build_loop();
    void admit_locked();
    gs_status start_query(Query* q);
    void set_phase(Query* q, Phase ph, int chunk);
    gs_status enter_phase(Query* q);
    void finish(Query* q);
    void collect();
};

void gs_server::set_phase(Query* q, Phase ph, int chunk) {
    q->phase = ph;
    q->chunk = chunk;
    q->t0 = tick;
    q->done = 0;
}

// per-query actions at the start of a phase and its device record fields
gs_status gs_server::enter_phase(Query* q) {
    gs_mesh* m = q->mesh;
    MeshRT& r = m->rt;
    const int seg0 = 1 + q->n_ck;
    if (q->phase == P_FWD && q->K == 1) {
        // every state kept: step n reads buffer 1 + n and writes 2 + n
        q->steps = q->S;
        r.active = ACT_FWD;
        r.in_a = 1 - q->t0;
        r.in_b = 1;
        r.out_a = 2 - q->t0;
        r.out_b = 1;
        r.ck_tick = -1;
    } else if (q->phase == P_FWD) {
        q->steps = std::min(q->K, q->S - q->chunk * q->K);
        r.active = ACT_FWD;
        r.in_a = r.in_b = r.out_a = r.out_b = 0;
        r.ck_tick = (q->chunk + 1 < q->n_ck) ? q->t0 + q->steps - 1 : -1;
        r.ck_buf = 2 + q->chunk;
    } else if (q->phase == P_REC) {
        // a segment of n steps needs its states 0..n-1 and the element forces
        // at each of them, which the forward step from that state writes: n
        // forward steps
        q->seg_steps = std::min(q->K, q->S - q->chunk * q->K);
        q->steps = q->seg_steps;
        r.active = ACT_FWD;
        r.cp_src = 1 + q->chunk;
        r.cp_dst = seg0;
        GS_TRY(m->self->sync_rt(stream));
        launch_copy_state(m->self->launch, stream);
        r.in_a = seg0 - q->t0;
        r.in_b = 1;
        r.out_a = seg0 + 1 - q->t0;
        r.out_b = 1;
        r.ck_tick = -1;
    } else if (q->phase == P_ADJ) {
        r.active = ACT_ADJ;
        // reverse step of step n reads its input state: the stored state n
        // (K = 1: buffer 1 + n) or the recomputed segment
        r.adj_a = (q->K == 1 ? q->S : seg0 + q->steps - 1) + q->t0;
        r.adj_b = -1;
    }
    return GS_OK;
}

// builder thread: the mesh, its state/checkpoint/adjoint buffers and the
// target, all on the builder's stream, finished before the query is handed on
static gs_status build_query(gs_ctx* ctx, Query* q, cudaStream_t bs) {
    gs_mesh* m = nullptr;
    GS_TRY(mesh_create(ctx, &q->desc, bs, &m));
    q->mesh = m;
    q->n_ck = std::max(1, (q->S + q->K - 1) / q->K);
    GS_TRY(m->ensure_buffers(1 + q->n_ck + q->K + 1, bs));
    GS_TRY(m->ensure_adjoint(bs));
    m->rt.g_act = nullptr;  // results carry no actuation gradients
    m->rt.g_hact = nullptr;
    GS_TRY(m->target.alloc(ctx, q->target.size() * sizeof(float), bs));
    GS_CUDA(cudaMemcpyAsync(m->target.p, q->target.data(), m->target.bytes, cudaMemcpyHostToDevice, bs));
    m->rt.target = (const float*)m->target.p;
    m->rt.dt = q->dt;
    GS_CUDA(cudaStreamSynchronize(bs));
    return GS_OK;
}

void gs_server::build_loop() {
    cudaSetDevice(ctx->device);
    cudaStream_t bs = nullptr;
    const bool have_stream = cudaStreamCreateWithFlags(&bs, cudaStreamNonBlocking) == cudaSuccess;
    while (true) {
        Query* q = nullptr;
        {
            std::unique_lock<std::mutex> lk(mu);
            cv_build.wait(lk, [this] { return stop || !to_build.empty(); });
            if (stop) break;
            q = to_build.front();
            to_build.pop_front();
            building++;
        }
        const double t = now_s();
        gs_status st;
        try {  // the query then fails with the status; the builder carries on
            st = have_stream ? build_query(ctx, q, bs) : set_error(GS_ECUDA, "builder stream");
        } catch (const std::bad_alloc&) {
            st = set_error(GS_ENOMEM, "host allocation failed while building the query");
        } catch (const std::exception& x) {
            st = set_error(GS_EINTERNAL, std::string("host exception while building the query: ") + x.what());
        }
        // a failed build may leave copies in flight on the builder's stream:
        // they finish before the worker releases the query's buffers
        if (st < 0 && have_stream) cudaStreamSynchronize(bs);
        const std::string err = st < 0 ? std::string(gs_last_error()) : std::string();
        {
            std::lock_guard<std::mutex> lk(mu);
            q->build_status = st;
            q->build_error = err;
            t_build += now_s() - t;
            building--;
            built.push_back(q);
        }
        cv.notify_all();
    }
    if (have_stream) cudaStreamDestroy(bs);
}

// worker: the query's first phase on the server stream
gs_status gs_server::start_query(Query* q) {
    gs_mesh* m = q->mesh;
    // checkpoint 0 = the initial state
    m->rt.cp_src = 0;
    m->rt.cp_dst = 1;
    m->rt.active = ACT_FWD;
    GS_TRY(m->self->sync_rt(stream));
    launch_copy_state(m->self->launch, stream);
    set_phase(q, P_FWD, 0);
    return enter_phase(q);
}

// last reverse step done: gradients out, device -> pinned host, event
void gs_server::finish(Query* q) {
    gs_mesh* m = q->mesh;
    const size_t E = m->info.n_elems, B = m->info.n_hinges, N = m->info.n_nodes;
    m->rt.active = 0;
    q->stage_bytes = sizeof(double) * (3 * E + B + 1) + sizeof(float) * 6 * N;
    if (q->g_dev.alloc(ctx, q->stage_bytes, stream) < 0 || cudaMallocHost((void**)&q->h_stage, q->stage_bytes) != cudaSuccess) {
        q->res.status = GS_ENOMEM;
        q->phase = P_FINISHING;
        cudaEventCreateWithFlags(&q->ev, cudaEventDisableTiming);
        cudaEventRecord(q->ev, stream);
        return;
    }
    char* p = (char*)q->g_dev.p;
    gs_grads g{};
    g.d_mu = (double*)p;
    g.d_lambda = g.d_mu + E;
    g.d_density = g.d_lambda + E;
    g.d_kb = B ? g.d_density + E : nullptr;
    double* d_loss = g.d_density + E + B;
    g.d_x0 = (float*)(d_loss + 1);
    g.d_v0 = g.d_x0 + 3 * N;
    m->self->sync_rt(stream);
    const size_t sm = std::max(sizeof(double) * (size_t)m->max_loc, (size_t)16);
    launch_finalize_grads(m->self->launch, (double*)m->mbar.p, g, sm, stream);
    // the loss of the final state
    launch_seed_loss(m->self->launch, (double*)m->self->d_loss.p, 0, stream);
    launch_loss_finalize((const double*)m->self->d_loss.p, 0, (int)m->node_blocks.size(), d_loss, stream);
    cudaMemcpyAsync(q->h_stage, q->g_dev.p, q->stage_bytes, cudaMemcpyDeviceToHost, stream);
    cudaEventCreateWithFlags(&q->ev, cudaEventDisableTiming);
    cudaEventRecord(q->ev, stream);
    q->phase = P_FINISHING;
}

// finished queries whose copies landed: fill results, release the mesh
void gs_server::collect() {
    std::vector<Query*> keep;
    bool any = false;
    for (Query* q : active) {
        if (q->phase != P_FINISHING || cudaEventQuery(q->ev) != cudaSuccess) {
            keep.push_back(q);
            continue;
        }
        gs_mesh* m = q->mesh;
        const size_t E = m->info.n_elems, B = m->info.n_hinges, N = m->info.n_nodes;
        gs_result& r = q->res;
        if (r.status == GS_OK && q->h_stage) {
            int st = 0;
            cudaMemcpy(&st, m->status.p, sizeof(int), cudaMemcpyDeviceToHost);
            r.status = (st & 4) ? GS_EINDEX : (st & 2) ? GS_ETIMEOUT : (st & 1) ? GS_ENONFINITE : GS_OK;
            const double* d = q->h_stage;
            r.n_elems = (int)E;
            r.n_hinges = (int)B;
            r.n_nodes = (int)N;
            r.d_mu = (double*)malloc(8 * E);
            r.d_lambda = (double*)malloc(8 * E);
            r.d_density = (double*)malloc(8 * E);
            std::memcpy(r.d_mu, d, 8 * E);
            std::memcpy(r.d_lambda, d + E, 8 * E);
            std::memcpy(r.d_density, d + 2 * E, 8 * E);
            if (B) {
                r.d_kb = (double*)malloc(8 * B);
                std::memcpy(r.d_kb, d + 3 * E, 8 * B);
            }
            r.loss = d[3 * E + B];
            const float* f = (const float*)(d + 3 * E + B + 1);
            r.d_x0 = (float*)malloc(12 * N);
            r.d_v0 = (float*)malloc(12 * N);
            std::memcpy(r.d_x0, f, 12 * N);
            std::memcpy(r.d_v0, f + 3 * N, 12 * N);
        }
        q->t_done = now_s();
        r.t_submit = q->t_submit;
        r.t_admit = q->t_admit;
        r.t_done = q->t_done;
        cudaEventDestroy(q->ev);
        q->ev = nullptr;
        if (q->h_stage) cudaFreeHost(q->h_stage);
        q->h_stage = nullptr;
        q->g_dev.release(stream);
        gs_mesh_destroy(q->mesh);
        q->mesh = nullptr;
        {
            std::lock_guard<std::mutex> lk(mu);
            admitted -= q->bytes;
            completed++;
            if (r.status == GS_OK) {
                latencies.push_back(q->t_done - q->t_submit);
                elem_steps += (double)E * q->S;
            }
            q->ready = true;
            q->phase = P_DONE;
        }
        any = true;
    }
    active.swap(keep);
    if (any) {
        ls_dirty = true;
        cv_done.notify_all();
    }
}

void gs_server::admit_locked() {
    while (!pending.empty()) {
        Query* q = pending.front();
        if (q->cancelled) {
            pending.pop_front();
            q->res.status = GS_ECANCELLED;
            q->ready = true;
            completed++;
            cv_done.notify_all();
            continue;
        }
        const int n_active = (int)(active.size() + to_build.size() + built.size()) + building;
        if (opts.max_active > 0 && n_active >= opts.max_active) break;
        if (opts.hbm_budget_bytes && admitted + q->bytes > opts.hbm_budget_bytes && n_active > 0) break;
        pending.pop_front();
        admitted += q->bytes;
        q->t_admit = now_s();
        to_build.push_back(q);
        cv_build.notify_one();
    }
}

// The worker.  Should it meet a host-side exception (a failed allocation
// while staging results, say), it stops: queries not finished by then, and
// later submissions, fail with GS_EINTERNAL (their memory is released by
// gs_server_destroy), so no poller waits on a worker that is gone.
void gs_server::run() {
    try {
        run_loop();
    } catch (...) {
        std::lock_guard<std::mutex> lk(mu);
        failed = true;
        cv_done.notify_all();
    }
}

void gs_server::run_loop() {
    cudaSetDevice(ctx->device);
    while (true) {
        std::vector<Query*> fresh;
        bool waiting;  // queries admitted but still being built
        {
            std::unique_lock<std::mutex> lk(mu);
            if (stop) break;
            admit_locked();
            fresh.swap(built);
            waiting = !to_build.empty() || building > 0;
            const bool idle = active.empty() && fresh.empty() && !waiting;
            if (idle && busy_since >= 0) {
                busy_time += now_s() - busy_since;
                busy_since = -1.0;
            }
            if (!idle && busy_since < 0) busy_since = now_s();
            if (active.empty() && fresh.empty()) {
                cv.wait_for(lk, std::chrono::milliseconds(waiting ? 5 : 50));
                continue;
            }
        }
        bool members = false, rt_changed = false;
        for (Query* q : fresh) {
            bool c;
            {
                std::lock_guard<std::mutex> lk(mu);
                c = q->cancelled;
            }
            gs_status st = q->build_status;
            if (st >= 0 && c) st = GS_ECANCELLED;
            if (st >= 0) {
                const double t = now_s();
                st = start_query(q);
                t_start += now_s() - t;
            }
            if (st < 0) {
                if (q->mesh) gs_mesh_destroy(q->mesh);
                q->mesh = nullptr;
                std::lock_guard<std::mutex> lk(mu);
                admitted -= q->bytes;
                q->res.status = st;
                q->t_done = now_s();
                q->ready = true;
                completed++;
                cv_done.notify_all();
                continue;
            }
            active.push_back(q);
            members = true;
        }
        // cancellations of running queries
        for (Query* q : active) {
            bool c;
            {
                std::lock_guard<std::mutex> lk(mu);
                c = q->cancelled;
            }
            if (c && q->phase != P_FINISHING) {
                q->mesh->rt.active = 0;
                q->res.status = GS_ECANCELLED;
                q->phase = P_FINISHING;
                cudaEventCreateWithFlags(&q->ev, cudaEventDisableTiming);
                cudaEventRecord(q->ev, stream);
                rt_changed = true;
            }
        }
        // phase transitions (queries whose phase has run all its steps)
        for (Query* q : active) {
            while (q->phase != P_FINISHING && q->done >= q->steps) {
                rt_changed = true;
                if (q->phase == P_FWD) {
                    if (q->K > 1 && (q->chunk + 1) * q->K < q->S) {
                        set_phase(q, P_FWD, q->chunk + 1);
                    } else {
                        // forward done: seed dL/dx(S) from the target, zero the accumulators
                        gs_mesh* m = q->mesh;
                        if (q->K == 1) {  // the final state (buffer S + 1) becomes the current one
                            m->rt.cp_src = q->S + 1;
                            m->rt.cp_dst = 0;
                            m->rt.active = ACT_FWD;
                            m->self->sync_rt(stream);
                            launch_copy_state(m->self->launch, stream);
                        }
                        m->rt.active = ACT_FWD | ACT_ADJ;
                        m->self->sync_rt(stream);
                        launch_seed_loss(m->self->launch, (double*)m->self->d_loss.p, 1, stream);
                        launch_zero_adjoint(m->self->launch, stream);
                        launch_zero_f64((double*)m->g_ml.p, 2 * (long long)m->info.n_elems, stream);
                        launch_zero_f64((double*)m->g_act.p, m->info.n_elems, stream);
                        launch_zero_f64((double*)m->g_kb.p, m->info.n_hinges, stream);
                        launch_zero_f64((double*)m->g_hact.p, m->info.n_hinges, stream);
                        if (q->K == 1) {
                            set_phase(q, P_ADJ, 0);
                            q->steps = q->S;
                        } else {
                            set_phase(q, P_REC, q->n_ck - 1);
                        }
                    }
                } else if (q->phase == P_REC) {
                    set_phase(q, P_ADJ, q->chunk);
                    q->steps = q->seg_steps;
                } else if (q->phase == P_ADJ) {
                    if (q->chunk > 0) {
                        set_phase(q, P_REC, q->chunk - 1);
                    } else {
                        finish(q);
                        break;
                    }
                }
                if (q->phase != P_FINISHING) enter_phase(q);
            }
        }
        // device records: full launch lists when the set of meshes changed,
        // otherwise only the per-mesh records (phase fields)
        if (members || ls_dirty || !ls_valid) {
            const double t = now_s();
            std::vector<gs_mesh*> ms;
            for (Query* q : active) ms.push_back(q->mesh);
            ls_valid = !ms.empty() && ls.build(ctx, ms, stream) == GS_OK;
            ls_dirty = false;
            t_rebuild += now_s() - t;
            n_rebuilds++;
        } else if (rt_changed) {
            const double t = now_s();
            ls.sync_rt(stream);
            t_sync += now_s() - t;
            n_syncs++;
        }
        // ticks until the next phase change of any running query, back to back
        bool any_f = false, any_a = false;
        int run = 1 << 30;
        for (Query* q : active) {
            if (q->phase == P_FWD || q->phase == P_REC) any_f = true;
            if (q->phase == P_ADJ) any_a = true;
            if (q->phase == P_FWD || q->phase == P_REC || q->phase == P_ADJ) run = std::min(run, q->steps - q->done);
        }
        {
            std::lock_guard<std::mutex> lk(mu);
            // let queries that are arriving or being built join soon
            if (!pending.empty() || !to_build.empty() || building > 0 || !built.empty()) run = std::min(run, 8);
        }
        run = std::max(1, std::min(run, 64));
        if ((any_f || any_a) && ls_valid) {
            for (int r = 0; r < run; ++r) {
                if (any_f) launch_forward_step(ls.launch, tick, stream);
                if (any_a) launch_adjoint_step(ls.launch, tick, stream);
                tick++;
            }
            n_ticks += run;
            for (Query* q : active)
                if (q->phase == P_FWD || q->phase == P_REC || q->phase == P_ADJ) q->done += run;
            // bound the work in flight: wait for the batch of ticks 4 back
            if (tick_events.size() >= 4) {
                const double t = now_s();
                cudaEventSynchronize(tick_events.front());
                t_wait += now_s() - t;
                free_events.push_back(tick_events.front());
                tick_events.pop_front();
            }
            cudaEvent_t e;
            if (!free_events.empty()) {
                e = free_events.back();
                free_events.pop_back();
            } else {
                cudaEventCreateWithFlags(&e, cudaEventDisableTiming);
            }
            cudaEventRecord(e, stream);
            tick_events.push_back(e);
            // keep ticks in a range where tick-affine indices stay small
            if (tick > (1 << 28)) {
                for (Query* q : active) {
                    MeshRT& r = q->mesh->rt;
                    const int sh = tick;
                    q->t0 -= sh;
                    r.in_a += r.in_b * sh;
                    r.out_a += r.out_b * sh;
                    r.adj_a += r.adj_b * sh;
                    if (r.ck_tick >= 0) r.ck_tick -= sh;
                }
                tick = 0;
                ls.sync_rt(stream);
            }
        } else {
            const double t = now_s();
            cudaStreamSynchronize(stream);
            t_wait += now_s() - t;
        }
        collect();
    }
    cudaStreamSynchronize(stream);
    for (cudaEvent_t e : tick_events) cudaEventDestroy(e);
    for (cudaEvent_t e : free_events) cudaEventDestroy(e);
    tick_events.clear();
    free_events.clear();
}

extern "C" gs_status gs_server_create(gs_ctx* ctx, const gs_server_opts* opts, gs_server** out) try {
    clear_error();
    if (!ctx || !out) return set_error(GS_EINVAL, "null argument");
    *out = nullptr;
    GS_CUDA(cudaSetDevice(ctx->device));
    std::unique_ptr<gs_server> s(new gs_server());
    s->ctx = ctx;
    if (opts) s->opts = *opts;
    GS_CUDA(cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking));
    gs_server* raw = s.get();
    const int nb = s->opts.build_threads > 0 ? std::min(s->opts.build_threads, 64) : 4;
    try {
        s->builders.reserve(nb);
        for (int i = 0; i < nb; ++i) s->builders.emplace_back([raw] { raw->build_loop(); });
        s->worker = std::thread([raw] { raw->run(); });
    } catch (...) {  // a thread could not be started: stop and join the ones that were
        {
            std::lock_guard<std::mutex> lk(s->mu);
            s->stop = true;
        }
        s->cv.notify_all();
        s->cv_build.notify_all();
        for (std::thread& t : s->builders)
            if (t.joinable()) t.join();
        if (s->worker.joinable()) s->worker.join();
        cudaStreamDestroy(s->stream);
        s->stream = nullptr;
        return set_error(GS_ENOMEM, "could not start the server's threads");
    }
    *out = s.release();
    return GS_OK;
} GS_ABI_CATCH

extern "C" void gs_server_destroy(gs_server* s) {
    if (!s) return;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
        for (auto& kv : s->all) kv.second->cancelled = true;
    }
    s->cv.notify_all();
    s->cv_build.notify_all();
    for (std::thread& b : s->builders)
        if (b.joinable()) b.join();
    if (s->worker.joinable()) s->worker.join();
    for (Query* q : s->built)
        if (q->mesh) gs_mesh_destroy(q->mesh);
    for (Query* q : s->active) {
        if (q->mesh) gs_mesh_destroy(q->mesh);
        if (q->h_stage) cudaFreeHost(q->h_stage);
        if (q->ev) cudaEventDestroy(q->ev);
    }
    for (auto& kv : s->all) {
        gs_result_free(&kv.second->res);
        delete kv.second;
    }
    cudaStreamDestroy(s->stream);
    delete s;
}

static gs_status query_submit(gs_server* s, const gs_query* q, uint64_t* ticket) {
    if (!s || !q || !ticket) return set_error(GS_EINVAL, "null argument");
    const gs_mesh_desc& d = q->mesh;
    if (d.n_nodes <= 0 || d.n_elems <= 0 || !d.elems || !d.X || !d.mu || !d.lambda || !d.density || !q->target)
        return set_error(GS_EINVAL, "query needs a mesh, materials and a target");
    if (q->n_steps < 0 || !(q->dt > 0.f)) return set_error(GS_EINVAL, "query needs dt > 0 and n_steps >= 0");
    std::unique_ptr<Query> Q(new Query());
    const int nc = d.kind == GS_TET ? 4 : 3;
    const size_t N = d.n_nodes, E = d.n_elems, B = d.kind == GS_CLOTH ? d.n_hinges : 0;
    Q->elems.assign(d.elems, d.elems + nc * E);
    Q->X.assign(d.X, d.X + 3 * N);
    if (d.v0) Q->v0.assign(d.v0, d.v0 + 3 * N);
    Q->mu.assign(d.mu, d.mu + E);
    Q->lam.assign(d.lambda, d.lambda + E);
    Q->rho.assign(d.density, d.density + E);
    if (B) {
        if (!d.hinges || !d.kb) return set_error(GS_EINVAL, "cloth query needs hinges and kb");
        Q->hinges.assign(d.hinges, d.hinges + 4 * B);
        Q->kb.assign(d.kb, d.kb + B);
    }
    Q->target.assign(q->target, q->target + 3 * N);
    Q->desc = d;
    Q->desc.elems = Q->elems.data();
    Q->desc.X = Q->X.data();
    Q->desc.v0 = d.v0 ? Q->v0.data() : nullptr;
    Q->desc.mu = Q->mu.data();
    Q->desc.lambda = Q->lam.data();
    Q->desc.density = Q->rho.data();
    Q->desc.hinges = B ? Q->hinges.data() : nullptr;
    Q->desc.kb = B ? Q->kb.data() : nullptr;
    Q->desc.act = nullptr;
    Q->desc.hinge_act = nullptr;
    Q->desc.pinned = nullptr;
    Q->dt = q->dt;
    Q->S = q->n_steps;
    Q->K = query_K(s->opts, d, Q->S);
    Q->bytes = estimate_bytes(d, Q->S, Q->K);
    Q->t_submit = now_s();
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->failed) return set_error(GS_EINTERNAL, "the server's worker stopped on a host-side failure");
    s->submitted++;
    if (s->opts.hbm_budget_bytes && Q->bytes > s->opts.hbm_budget_bytes) {
        s->rejected++;
        return set_error(GS_ENOMEM, "query needs more than the whole server budget");
    }
    Q->id = s->next_id++;
    *ticket = Q->id;
    s->all[Q->id] = Q.get();
    s->pending.push_back(Q.release());
    s->cv.notify_all();
    return GS_OK;
}

// the query is deep-copied on the host (a failed allocation: GS_ENOMEM)
extern "C" gs_status gs_query_submit(gs_server* s, const gs_query* q, uint64_t* ticket) try {
    clear_error();
    return query_submit(s, q, ticket);
} GS_ABI_CATCH

extern "C" gs_status gs_query_poll(gs_server* s, uint64_t ticket, gs_result* out, int timeout_ms) try {
    clear_error();
    if (!s) return set_error(GS_EINVAL, "null server");
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->all.find(ticket);
    if (it == s->all.end()) return set_error(GS_ENOTFOUND, "unknown ticket");
    Query* q = it->second;
    if (!q->ready && timeout_ms > 0 && !s->failed)
        s->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), [s, q] { return q->ready || s->failed; });
    if (!q->ready) {
        if (s->failed) return set_error(GS_EINTERNAL, "the server's worker stopped on a host-side failure");
        return timeout_ms > 0 ? GS_ETIMEOUT : GS_PENDING;
    }
    const gs_status st = q->res.status;
    if (out) {
        *out = q->res;  // ownership of the host arrays passes to the caller
        std::memset(&q->res, 0, sizeof(q->res));
    }
    s->all.erase(it);
    delete q;
    if (st == GS_ECANCELLED) return set_error(GS_ECANCELLED, "query cancelled");
    if (st == GS_ENONFINITE) return set_error(GS_ENONFINITE, "query produced a non-finite state");
    if (st < 0) return set_error(st, "query failed");
    return GS_OK;
} GS_ABI_CATCH

extern "C" gs_status gs_query_cancel(gs_server* s, uint64_t ticket) try {
    clear_error();
    if (!s) return set_error(GS_EINVAL, "null server");
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->all.find(ticket);
    if (it == s->all.end()) return set_error(GS_ENOTFOUND, "unknown ticket");
    it->second->cancelled = true;
    s->cv.notify_all();
    return GS_OK;
} GS_ABI_CATCH

extern "C" gs_status gs_server_stats_get(gs_server* s, gs_server_stats* out) try {
    clear_error();
    if (!s || !out) return set_error(GS_EINVAL, "null argument");
    std::lock_guard<std::mutex> lk(s->mu);
    std::memset(out, 0, sizeof(*out));
    out->submitted = s->submitted;
    out->completed = s->completed;
    out->rejected = s->rejected;
    out->active = s->active.size();
    out->queued = s->pending.size();
    out->admitted_bytes = s->admitted;
    std::vector<double> l = s->latencies;
    if (!l.empty()) {
        std::sort(l.begin(), l.end());
        auto pct = [&](double p) { return l[std::min(l.size() - 1, (size_t)std::floor(p * (l.size() - 1) + 0.5))]; };
        out->p50_latency_s = pct(0.50);
        out->p99_latency_s = pct(0.99);
    }
    double busy = s->busy_time + (s->busy_since >= 0 ? now_s() - s->busy_since : 0.0);
    out->elem_steps_per_s = busy > 0 ? s->elem_steps / busy : 0.0;
    out->busy_s = busy;
    out->build_s = s->t_build;
    out->start_s = s->t_start;
    out->rebuild_s = s->t_rebuild;
    out->rt_sync_s = s->t_sync;
    out->gpu_wait_s = s->t_wait;
    out->ticks = s->n_ticks;
    out->rebuilds = s->n_rebuilds;
    out->rt_syncs = s->n_syncs;
    return GS_OK;
} GS_ABI_CATCH

extern "C" void gs_result_free(gs_result* r) {
    if (!r) return;
    free(r->d_mu);
    free(r->d_lambda);
    free(r->d_density);
    free(r->d_kb);
    free(r->d_x0);
    free(r->d_v0);
    r->d_mu = r->d_lambda = r->d_density = r->d_kb = nullptr;
    r->d_x0 = r->d_v0 = nullptr;
}
