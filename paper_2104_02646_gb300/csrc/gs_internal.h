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

#include <exception>
#include <map>
#include <new>
#include <string>
#include <utility>
#include <vector>

#include "../../include/gradsim.h"

namespace gs {

// --------------------------------------------------------------------------
// device-side tables
// --------------------------------------------------------------------------
// Element records, 4 float4 planes (plane k of element e at rec[k * E + e]);
// a patch's slice of each plane is contiguous, so 4 bulk copies stage it:
//   tet   [0] Dm^-1 00 01 02 10  [1] Dm^-1 11 12 20 21  [2] Dm^-1 22, V, mu, lambda
//         [3] ids (0|1<<16), ids (2|3<<16) as bits, act, 0
//   tri   [0] Dm^-1 00 01 10 11  [1] A, mu, lambda, act  [2] r0.x r0.y r0.z r1.x
//         [3] ids (0|1<<16), ids (2) as bits, r1.y, r1.z       (r0, r1: rest frame R0)
//   hinge [0] X1-X3, kb  [1] X2-X3, act  [2] X4-X3, 0  [3] ids (1|2<<16), ids (3|4<<16) as bits, 0, 0
// In shared memory the planes are [4][n_rec] over the patch's records
// (triangles first, then hinges); a corner result of record r, corner c is
// written in place to plane c, row r.  CSR slot s = (record << 2) | corner.
struct PatchDesc {
    int e_begin, n_e;      // elements (tets or triangles), internal order
    int h_begin, n_h;      // hinges (cloth)
    int int_begin, n_int;  // interior nodes: internal ids [int_begin, int_begin + n_int)
    int bnd_begin, n_bnd;  // boundary local nodes: bnd_ids / part_pos [bnd_begin, +n_bnd); bnd_begin % 4 == 0
    int lr_begin;          // local CSR row pointers: n_int + n_bnd + 1 entries (16 B aligned)
    int slot_begin;        // local CSR slot list (16 B aligned)
    int mesh;              // index into the launch set's MeshRT array
    int n_slots;           // local CSR slots, every row padded to a multiple of 4
    int topo;              // the patch's topology block in MeshRT::topo (16 B units)
};

// shared-memory pipeline stages of the patch kernels
constexpr int kStages = 2;

// Element records are patch-contiguous: the patch of elements [b, b + n)
// (b = p * pe, n = min(pe, E - b)) holds its 4 planes of n float4 at 4 b, so
// one bulk copy stages the whole patch.  Index of plane k of element e:
__host__ __device__ __forceinline__ size_t rec_at(int E, int pe, int k, int e) {
    const int b = (e / pe) * pe;
    const int n = (E - b < pe) ? (E - b) : pe;
    return 4 * (size_t)b + (size_t)k * (size_t)n + (size_t)(e - b);
}

// nodes per NodeBlock (boundary kernels: 2 nodes per thread of a 128-thread CTA)
constexpr int kNodeBlock = 256;

struct NodeBlock {  // a run of node indices of one mesh
    int mesh, begin, count, pad;
};

enum { ACT_FWD = 1, ACT_ADJ = 2 };

struct alignas(16) MeshRT {  // 16 B aligned: the patch kernels bulk-copy it into shared memory
    // static mesh data
    int kind, n_nodes, n_int, n_bnd;
    int n_elems, n_hinges, active, pe;  // pe: elements per patch
    int n_part, pad_[3];                // boundary partials (bnd_rowptr[n_bnd])
    float4* rec;             // element records, patch-contiguous (rec_at), 4 float4 planes per patch
    float4* hrec;            // [4][B] hinge records
    const int* bnd_ids;      // per-patch boundary lists (internal node ids)
    const uint16_t* loc_rowptr;
    const uint16_t* loc_slots;
    const int* bnd_rowptr;   // [n_bnd + 1] over boundary nodes (internal id - n_int)
    const int* part_pos;     // per (patch, boundary local node): index of its partial
    const uint4* topo;       // per patch, 16 B aligned: CSR row pointers, CSR slots, partial positions
    float4* partials;        // node-major: node b's partials at [bnd_rowptr[b], bnd_rowptr[b+1]), patch order
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
    // buffer b of st_f: the elements' force on each node in the state of
    // buffer b, written by the forward step that starts from it (the
    // adjoint's dL/dw term needs it, and recomputing it cost the adjoint's
    // element phase a force evaluation per element)
    float4* st_f;            // (fx, fy, fz, 0)
    long long buf_stride;
    int in_a, in_b, out_a, out_b;   // forward: in = in_a + in_b * tick, out likewise
    int ck_tick, ck_buf;            // tick at which the output is also written to ck_buf
    int adj_a, adj_b;               // adjoint: state buffer = adj_a + adj_b * tick
    int cp_src, cp_dst;             // buffer copy
    // adjoint state and accumulators
    float4* xb;
    float4* vb;
    double* wbar;            // [N]
    double2* g_ml;           // [E]: (dL/dmu, dL/dlambda) per element
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
    int plane_on, sphere_on;
    int act_ld, hact_ld;     // row strides of act_seq / d_act_seq and hact_seq / d_hact_seq (multiples of 4)
    float pnx, pny, pnz, ph;
    float scx, scy, scz, sr;
    int* status;             // bit 0: non-finite state
    // time-varying actuation (nullable): during step n = st_a + st_b * tick,
    // row n < n_act of act_seq [n_act][act_ld] (hact_seq [n_act][hact_ld]),
    // internal element (hinge) order, is added to the element's (hinge's)
    // actuation; the adjoint writes dL/d(that actuation) into row n < n_dact
    // of d_act_seq [n_dact][act_ld] (d_hact_seq [n_dact][hact_ld])
    const float* act_seq;
    const float* hact_seq;
    float* d_act_seq;
    float* d_hact_seq;
    int n_act, n_dact, st_a, st_b;
    // air on the triangles (cloth, when air_on): drag / lift coefficients,
    // wind; the adjoint's boundary partials of dL/dv from it
    float k_drag, k_lift, wx, wy, wz;
    int air_on;
    float4* partials_v;
};

// Dynamic shared memory of a patch kernel: the mbarriers, kStages stages, and
// the producer warp's own copy of the current mesh record
constexpr size_t kPipeHead = 128;
constexpr size_t kProdRt = (sizeof(MeshRT) + 127) / 128 * 128;
__host__ __device__ __forceinline__ size_t patch_dyn_smem(int stage_bytes) {
    return kPipeHead + kStages * (size_t)stage_bytes + kProdRt;
}

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
    int threads = 256;      // consumer threads of the forward patch kernels
    int threads_adj = 256;  // consumer threads of the adjoint patch kernels
    // patch kernels (tet fwd, cloth fwd, tet adj, cloth adj): persistent grid
    // size and bytes of one of the two shared-memory pipeline stages
    int grid[4] = {0, 0, 0, 0};
    int stage[4] = {0, 0, 0, 0};
    int bgrid[2] = {0, 0};  // boundary kernels (fwd, adj): CTAs striding over bnd_blocks
    int air = 0;            // some cloth mesh of the set has air on: the adjoint step adds k_adj_boundary_air
    int extras = -1;        // stages hold actuation slices / boundary v (a mesh has a sequence or air); -1: unset
};

// --------------------------------------------------------------------------
// kernels (gs_kernels.cu)
// --------------------------------------------------------------------------
size_t patch_smem_bytes(int kind, int n_e, int n_h, int n_loc, int n_int, int n_slots, bool adjoint, bool extras);
int patch_grid(int which, int threads, int stage_bytes, int n_patches, int num_sms);
int boundary_grid(int adjoint, int n_blocks, int num_sms);
gs_status selftest_bounded_wait(int iterations, int* status_host, cudaStream_t s);
// rows x count floats between caller order and internal order: to_internal:
// dst[r][i] = src[r][perm[i]]; else dst[r][perm[i]] = src[r][i]
void launch_permute_rows(const float* src, float* dst, int rows, int count, int ld, const int* perm, int to_internal,
                         cudaStream_t s);
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

// Closes the function-try-block of every extern "C" entry point that returns
// a status, so that no C++ exception crosses the C ABI: a failed host
// allocation becomes GS_ENOMEM, anything else GS_EINTERNAL with its text.
#define GS_ABI_CATCH                                                                       \
    catch (const std::bad_alloc&) {                                                        \
        return ::gs::set_error(GS_ENOMEM, "host allocation failed");                       \
    }                                                                                      \
    catch (const std::exception& _x) {                                                     \
        return ::gs::set_error(GS_EINTERNAL, std::string("host exception: ") + _x.what()); \
    }                                                                                      \
    catch (...) {                                                                          \
        return ::gs::set_error(GS_EINTERNAL, "unknown host exception");                    \
    }

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
