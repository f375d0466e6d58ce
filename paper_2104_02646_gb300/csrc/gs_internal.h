// Internal layout of the gradsim library (not part of the C ABI).
//
// Work decomposition.  Elements are Morton-ordered and cut into *patches*
// (one CTA each).  A node is *interior* to a patch when every element that
// touches it lies in that patch; otherwise it is a *boundary* node.  Interior
// nodes of a patch are numbered contiguously, so each patch CTA gathers its
// element forces for them in shared memory in a fixed order and integrates
// them in the same kernel; for boundary nodes it writes one partial sum per
// (patch, node) and a boundary kernel adds the partials in patch order.  No
// floating-point atomics anywhere: results depend only on the decomposition.
//
// Launch sets.  A launch set is a list of meshes advanced together: one
// launch per kernel per step covers the patches of all of them.  A mesh run
// alone is a launch set of one; a batch or the server's active queries form
// larger ones.  Per-mesh pointers and constants live in a device-side
// MeshRT array indexed by the patch's `mesh` field.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <map>
#include <string>
#include <utility>
#include <vector>

#include "../../include/gradsim.h"

namespace gs {

// --------------------------------------------------------------------------
// device-side tables
// --------------------------------------------------------------------------
struct PatchDesc {
    int e_begin, n_e;      // elements (tets or triangles), internal order
    int h_begin, n_h;      // hinges (cloth)
    int int_begin, n_int;  // interior nodes: internal ids [int_begin, int_begin + n_int)
    int bnd_begin, n_bnd;  // boundary local nodes: bnd_ids / partials [bnd_begin, +n_bnd)
    int lr_begin;          // local CSR row pointers: n_int + n_bnd + 1 entries
    int slot_begin;        // local CSR slot list
    int mesh;              // index into the launch set's MeshRT array
    int pad;
};

struct NodeBlock {  // a run of node indices of one mesh
    int mesh, begin, count, pad;
};

enum { ACT_FWD = 1, ACT_ADJ = 2 };

struct MeshRT {
    // static mesh data
    int kind, n_nodes, n_int, n_bnd;
    int n_elems, n_hinges, active, pad0;
    const uint2* eidx;       // [E] 4 (tets) / 3 (tris) uint16 local node ids
    float4* ea;              // tets: Dm^-1 00 01 02 10 | tris: Dm^-1 00 01 10 11
    float4* eb;              // tets: Dm^-1 11 12 20 21 | tris: A, mu, lambda, act
    float4* ec;              // tets: Dm^-1 22, V, mu, lambda | tris: rest frame r0, r1.x
    float2* ed;              // tris: rest frame r1.y, r1.z
    float* eact;             // tets: actuation [E] (nullable)
    const uint2* hidx;       // [B] 4 uint16 local ids (x1, x2, x3, x4)
    float4* hq;              // [3B] (X1-X3, kb), (X2-X3, act), (X4-X3, 0)
    const int* bnd_ids;      // per-patch boundary lists (internal node ids)
    const uint16_t* loc_rowptr;
    const uint16_t* loc_slots;
    const int* bnd_rowptr;   // [n_bnd + 1] over boundary nodes (internal id - n_int)
    const int* bnd_parts;    // partial slots, in patch order
    float4* partials;        // one per (patch, boundary local node)
    const int* node_perm;    // internal node -> caller node
    const int* elem_perm;    // internal element -> caller element
    const int* hinge_perm;   // internal hinge -> caller hinge
    float* w;                // inverse masses [N]
    const float4* Xs;        // per node: X - sphere centre, |X - c|^2 - r^2 (FP64-derived)
    const float* Xp;         // per node: plane offset h - n.X (FP64-derived)
    const double* Xd;        // rest positions (FP64, for state in/out and the loss)
    // state buffers: buffer b at st_x + b * buf_stride; the state holds the
    // displacement u = x - X (and the inverse mass in .w)
    float4* st_x;            // (ux, uy, uz, w)
    float4* st_v;            // (vx, vy, vz, 0)
    long long buf_stride;
    int in_a, in_b, out_a, out_b;   // forward: in = in_a + in_b * tick, out likewise
    int ck_tick, ck_buf;            // tick at which the output is also written to ck_buf
    int adj_a, adj_b;               // adjoint: state buffer = adj_a + adj_b * tick
    int cp_src, cp_dst;             // buffer copy
    // adjoint state and accumulators
    float4* xb;
    float4* vb;
    double* wbar;            // [N]
    double* g_mu;            // [E]
    double* g_lam;
    double* g_act;           // nullable
    double* g_kb;            // [B]
    double* g_hact;          // nullable
    // seeds / loss (caller order)
    const float* target;
    const float* seed_x;
    const float* seed_v;
    // constants
    float dt, gx, gy, gz;
    float ke, kd, kf, mu_f;
    int plane_on, sphere_on, pad1, pad2;
    float pnx, pny, pnz, ph;
    float scx, scy, scz, sr;
    int* status;             // bit 0: non-finite state
};

// Everything one kernel launch over a launch set needs.
struct Launch {
    const PatchDesc* tet_patches = nullptr;
    int n_tet_patches = 0;
    const PatchDesc* cloth_patches = nullptr;
    int n_cloth_patches = 0;
    const NodeBlock* bnd_blocks = nullptr;
    int n_bnd_blocks = 0;
    const NodeBlock* node_blocks = nullptr;
    int n_node_blocks = 0;
    MeshRT* rt = nullptr;
    int threads = 256;
    size_t smem_tet_fwd = 0, smem_tet_adj = 0, smem_cloth_fwd = 0, smem_cloth_adj = 0;
};

// --------------------------------------------------------------------------
// kernels (gs_kernels.cu)
// --------------------------------------------------------------------------
size_t smem_bytes(int kind, bool adjoint, int max_loc, int max_slots);
void set_kernel_smem_limits(size_t bytes);
// kernels whose launches can be timed one by one (gs_profile)
enum { KT_TET_FWD, KT_CLOTH_FWD, KT_FWD_BND, KT_TET_ADJ, KT_CLOTH_ADJ, KT_ADJ_BND, KT_COUNT };
const char* kernel_name(int kind);
struct Prof {
    virtual void begin(int kind, cudaStream_t s) = 0;
    virtual void end(int kind, cudaStream_t s) = 0;
    virtual ~Prof() {}
};
void launch_forward_step(const Launch& L, int tick, cudaStream_t s, Prof* prof = nullptr);
void launch_adjoint_step(const Launch& L, int tick, cudaStream_t s, Prof* prof = nullptr);
void launch_copy_state(const Launch& L, cudaStream_t s);
void launch_seed_loss(const Launch& L, double* block_partials, int write_seeds, cudaStream_t s);
void launch_loss_finalize(const double* block_partials, int begin, int count, double* out, cudaStream_t s);
void launch_zero_adjoint(const Launch& L, cudaStream_t s);
void launch_zero_f64(double* p, long long n, cudaStream_t s);
void launch_setup_mesh(const Launch& L, const double* X, const float* rho, double* mass, double* mass_part,
                       const uint8_t* pinned_internal, int* bad, int geometry, size_t smem, cudaStream_t s);
void launch_scatter_params(const MeshRT* rt_dev, const float* mu, const float* lam, const float* act,
                           const float* kb, cudaStream_t s);
void launch_set_state(const MeshRT* rt_dev, int buf, const float* x, const float* v, cudaStream_t s);
void launch_get_state(const MeshRT* rt_dev, int buf, float* x, float* v, cudaStream_t s);
void launch_reset_state(const MeshRT* rt_dev, const float* v0_caller, cudaStream_t s);
void launch_finalize_grads(const Launch& L, double* mbar, const gs_grads& g, size_t smem, cudaStream_t s);

// --------------------------------------------------------------------------
// runtime helpers shared by the runtime and the server
// --------------------------------------------------------------------------
gs_status set_error(gs_status s, const std::string& msg);
gs_status cuda_error(cudaError_t e, const char* what);
void clear_error();

#define GS_CUDA(call)                                              \
    do {                                                           \
        cudaError_t _e = (call);                                   \
        if (_e != cudaSuccess) return ::gs::cuda_error(_e, #call); \
    } while (0)
#define GS_TRY(call)           \
    do {                       \
        gs_status _s = (call); \
        if (_s < 0) return _s; \
    } while (0)

}  // namespace gs
