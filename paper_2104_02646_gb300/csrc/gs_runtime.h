// Host-side objects of the gradsim runtime (shared by the runtime and the
// server translation units).
#pragma once

#include <atomic>
#include <map>
#include <memory>
#include <utility>
#include <vector>

#include "gs_internal.h"

namespace gs {
// per-launch CUDA-event timing of the step kernels (gs_profile); with CUDA
// graphs on, the events are external event nodes of the captured graphs
struct EventProf : Prof {
    struct Pending {
        int kind;
        cudaEvent_t a, b;
    };
    std::vector<cudaEvent_t> pool;
    std::vector<Pending> pending;
    cudaEvent_t open = nullptr;
    bool capture = false;  // recording into a stream capture: external event nodes
    double total_ms[KT_COUNT] = {0};
    unsigned long long launches[KT_COUNT] = {0};
    cudaEvent_t get();
    void begin(int kind, cudaStream_t s) override;
    void end(int kind, cudaStream_t s) override;
    void collect();  // synchronises the pending events and accumulates
    ~EventProf() override;
};
}  // namespace gs

struct gs_ctx {
    gs::EventProf* prof = nullptr;  // non-null while gs_profile is on
    int device = 0;
    size_t budget = 0;
    std::atomic<size_t> used{0};  // device bytes held (builder threads allocate concurrently)
    gs_allocator alloc{};
    bool has_alloc = false;
    bool graphs = true;
    cudaStream_t capture_stream = nullptr;
    int num_sms = 0;
    size_t smem_optin = 0;
};

namespace gs {

const char* g_last_error_cstr();

// A device allocation made through the context (budget-checked).  Move-only;
// release() frees stream-ordered, the destructor frees on the legacy stream.
struct Buf {
    gs_ctx* ctx = nullptr;
    void* p = nullptr;
    size_t bytes = 0;
    Buf() = default;
    Buf(const Buf&) = delete;
    Buf& operator=(const Buf&) = delete;
    Buf(Buf&& o) noexcept { take(o); }
    Buf& operator=(Buf&& o) noexcept {
        if (this != &o) {
            release(0);
            take(o);
        }
        return *this;
    }
    ~Buf() { release(0); }
    gs_status alloc(gs_ctx* c, size_t nbytes, cudaStream_t s);
    void release(cudaStream_t s);

   private:
    void take(Buf& o) {
        ctx = o.ctx;
        p = o.p;
        bytes = o.bytes;
        o.p = nullptr;
        o.bytes = 0;
    }
};

struct LaunchSet {
    gs_ctx* ctx = nullptr;
    std::vector<gs_mesh*> meshes;
    Buf d_tet, d_cloth, d_bnd, d_nodes, d_rt, d_loss;
    std::vector<MeshRT> host_rt;
    std::vector<int> node_block_begin;
    Launch launch;
    int stage_var[2][4] = {{0, 0, 0, 0}, {0, 0, 0, 0}};  // stage bytes per patch kernel, [extras]
    int threads = 256, threads_adj = 256;
    std::map<std::pair<int, int>, cudaGraphExec_t> graphs;

    gs_status build(gs_ctx* c, const std::vector<gs_mesh*>& ms, cudaStream_t s);
    gs_status sync_rt(cudaStream_t s);
    gs_status run(int phase, int steps, cudaStream_t s);
    gs_status step(const std::vector<float>& dts, int n, cudaStream_t s);
    gs_status rollout(const std::vector<float>& dts, int S, int K, const std::vector<const float*>& targets,
                      double* loss_dev, cudaStream_t s);
    gs_status adjoint(const std::vector<const float*>& seed_x, const std::vector<const float*>& seed_v,
                      const std::vector<gs_grads>& grads, int keep, cudaStream_t s);
    ~LaunchSet();
};

void launch_gather_elems(const MeshRT* rt_dev, const float* src_caller_order, float* dst_internal, cudaStream_t s);

}  // namespace gs

struct gs_mesh {
    gs_ctx* ctx = nullptr;
    gs_mesh_info info{};
    int n_pad = 0, threads = 256, threads_adj = 256, max_loc = 0, max_slots = 0, max_rec = 0, n_bufs = 0;
    size_t smem_fwd[2] = {0, 0}, smem_adj[2] = {0, 0};  // stage bytes [without, with] the extra regions
    std::vector<gs::PatchDesc> patches;
    std::vector<gs::NodeBlock> bnd_blocks, node_blocks;
    gs::Buf rec, hrec, Xs, Xp, v0, bnd_ids, loc_rowptr, loc_slots, bnd_rowptr, part_pos, topo, partials,
        node_perm, elem_perm, hinge_perm, w, X, rho, pinned, st, xb, vb, wbar, mbar, g_ml, g_act, g_kb,
        g_hact, status, target, scratch, act_seq, hact_seq, dact_seq, dhact_seq, partials_v;
    gs::MeshRT rt{};
    struct {
        bool valid = false;
        int S = 0, K = 0, n_ck = 0;
    } ro;
    std::unique_ptr<gs::LaunchSet> self;  // the mesh alone; self->launch.rt is its device record

    const gs::MeshRT* rt_dev() const { return self->launch.rt; }
    gs_status refresh_rt();
    gs_status ensure_buffers(int n, cudaStream_t s);
    gs_status ensure_adjoint(cudaStream_t s);
    gs_status run_setup(int geometry, cudaStream_t s);
    ~gs_mesh();
};

namespace gs {
gs_status mesh_create(gs_ctx* ctx, const gs_mesh_desc* desc, cudaStream_t s, gs_mesh** out);
}
