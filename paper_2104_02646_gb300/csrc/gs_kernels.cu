// Kernels of the explicit step (forward) and of its discrete adjoint.
//
// One CTA per element patch.  At the start one elected thread moves the
// patch's element records, its local CSR and the state of its interior nodes
// (all contiguous, 16 B aligned) into shared memory with TMA bulk copies
// (cp.async.bulk) that complete on an mbarrier, while the other threads
// gather the boundary nodes with ordinary loads; the CTA then waits for both.
// The element phase computes each element from its shared record and writes
// its corner results in place over that record (each record is read and
// overwritten by one thread only).  The node phase sums the corners of every
// local node through the shared CSR in a fixed order, finishes interior nodes
// (contact + semi-implicit Euler, or the reverse of both) and writes one
// partial per boundary node, which the boundary kernel sums in patch order.
// Nothing uses floating-point atomics.
#include <cuda_runtime.h>

#include "gs_internal.h"
#include "gs_math.cuh"
#include "gs_runtime.h"

namespace gs {

namespace {

__device__ __forceinline__ int local_gid(const PatchDesc& p, const MeshRT& m, int l) {
    return l < p.n_int ? p.int_begin + l : m.bnd_ids[p.bnd_begin + (l - p.n_int)];
}

__device__ __forceinline__ float4* bufx(const MeshRT& m, int b) { return m.st_x + (size_t)b * (size_t)m.buf_stride; }
__device__ __forceinline__ float4* bufv(const MeshRT& m, int b) { return m.st_v + (size_t)b * (size_t)m.buf_stride; }

__device__ __forceinline__ ContactParams cparams(const MeshRT& m) {
    ContactParams c;
    c.ke = m.ke;
    c.kd = m.kd;
    c.kf = m.kf;
    c.mu_f = m.mu_f;
    return c;
}

__device__ __forceinline__ uint2 rec_ids(float4 w) { return make_uint2(__float_as_uint(w.x), __float_as_uint(w.y)); }

// row of the time-varying actuation applied during the current step, or -1
// (no sequence, or the step lies past its end: no extra actuation)
__device__ __forceinline__ int act_row(const MeshRT& m, const float* seq, int tick) {
    const int n = m.st_a + m.st_b * tick;
    return (seq && n >= 0 && n < m.n_act) ? n : -1;
}
// dL/d(actuation during the current step), when per-step gradients are requested
__device__ __forceinline__ void act_grad_step(const MeshRT& m, float* dseq, int ld, int tick, int i, float g) {
    if (!dseq) return;
    const int n = m.st_a + m.st_b * tick;
    if (n >= 0 && n < m.n_dact) dseq[(size_t)n * ld + i] = g;
}
// the slice [r4down(begin), r4up(begin + n)) of a sequence row that holds a
// patch's n entries from `begin`: 16 B aligned ends for one bulk copy
__host__ __device__ __forceinline__ int act_slice_lo(int begin) { return begin & ~3; }
__host__ __device__ __forceinline__ int act_slice_n(int begin, int n) { return ((begin + n + 3) & ~3) - (begin & ~3); }


// ---------------------------------------------------------------------------
// Programmatic dependent launch between the step kernels: a kernel waits
// for the previous one in its stream to complete and its memory to be
// visible before it reads anything (pdl_enter), and once a CTA has finished
// its work it lets the next kernel be scheduled (pdl_done; the next kernel
// launches when every CTA has done so or exited, and still waits for this
// one to complete).  Without the launch attribute both are no-ops.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void pdl_enter() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_done() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

// ---------------------------------------------------------------------------
// Index checks of the checked build (compiled with -DGS_CHECK): every index
// that the step kernels read from the mesh tables and then use to address
// shared or global memory (local node ids of a record, CSR row pointers and
// slots, partial positions, boundary node ids, interior node ranges, the
// stage layout) is tested against its range first.  A violation sets bit 2
// (value 4) of the mesh's status word and the access is skipped or sent to a
// harmless slot, so the kernel never leaves its buffers; the run's results
// are then invalid and gs_mesh_check reports GS_EINDEX.  Without GS_CHECK
// every test compiles away.
// ---------------------------------------------------------------------------
#ifdef GS_CHECK
constexpr bool kChecked = true;
#else
constexpr bool kChecked = false;
#endif
constexpr int kStatusIndex = 4;

__device__ __forceinline__ bool idx_ok(bool ok, int* status) {
    if (kChecked && !ok) {
        atomicOr(status, kStatusIndex);
        return false;
    }
    return true;
}
// the four (three) 16-bit local node ids of a record are below n_loc
__device__ __forceinline__ bool ids_in(uint2 id, int n_loc, int n_ids) {
    return (int)(id.x & 0xffff) < n_loc && (int)(id.x >> 16) < n_loc && (int)(id.y & 0xffff) < n_loc &&
           (n_ids < 4 || (int)(id.y >> 16) < n_loc);
}
// four CSR slots (float4 indices into the staged planes, 4 n_rec = the zero
// slot): out-of-range slots are sent to the zero slot
__device__ __forceinline__ uint2 checked_slots(uint2 q, int n_rec, int* status) {
    if (!kChecked) return q;
    const uint32_t lim = 4u * (uint32_t)n_rec;
    uint32_t a = q.x & 0xffff, b = q.x >> 16, c = q.y & 0xffff, d = q.y >> 16;
    if (a > lim || b > lim || c > lim || d > lim) {
        atomicOr(status, kStatusIndex);
        a = a > lim ? lim : a;
        b = b > lim ? lim : b;
        c = c > lim ? lim : c;
        d = d > lim ? lim : d;
    }
    return make_uint2(a | (b << 16), c | (d << 16));
}

// ---------------------------------------------------------------------------
// TMA bulk copies global -> shared completing on an mbarrier
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t saddr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// barrier completing a phase after `count` arrivals (and its expected bytes)
__device__ __forceinline__ void mbar_init(uint64_t* bar, int count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(saddr(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_init_fence() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.shared::cta.b64 st, [%0];\n\t}" ::"r"(saddr(bar)) : "memory");
}
// arrive on `bar` once all of this thread's earlier cp.async copies have landed
// (the arrival is one of the barrier's initial count)
__device__ __forceinline__ void cp_async_mbar_arrive(uint64_t* bar) {
    asm volatile("cp.async.mbarrier.arrive.noinc.shared::cta.b64 [%0];" ::"r"(saddr(bar)) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n\t}" ::"r"(saddr(bar)),
                 "r"(bytes)
                 : "memory");
}

// bytes: multiple of 16; src, dst: 16 B aligned
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     saddr(dst)),
                 "l"(src), "r"(bytes), "r"(saddr(bar))
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(saddr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait for the given phase parity of the barrier.  try_wait suspends for a
// hardware-defined interval per call, so the limit is seconds, far above
// any real transfer; on expiry the kernel reports GS error bit 2 and, after
// a second bounded wait for its own copies, the caller returns.
constexpr int kWaitLimit = 1 << 22;
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity, int* status,
                                                  int limit = kWaitLimit) {
    for (int i = 0; i < limit; ++i)
        if (mbar_try_wait(bar, parity)) return true;
    atomicOr(status, 2);
    for (int i = 0; i < limit; ++i)
        if (mbar_try_wait(bar, parity)) break;
    return false;
}

// one thread waits on a barrier that nothing arrives at, `limit` polls
__global__ void k_selftest_wait(int limit, int* status) {
    __shared__ uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        mbar_init_fence();
        mbar_wait_bounded(&bar, 0u, status, limit);
    }
}

__host__ __device__ __forceinline__ int r16(int bytes) { return (bytes + 15) & ~15; }

// Shared-memory layout of one pipeline stage (byte offsets, 16 B aligned):
// the 4 record planes and one zero float4 (the target of padded CSR slots),
// the local CSR, the partial positions of the boundary nodes, local node
// state.  The adjoint also holds the adjoint state x_bar, v_hat of every
// local node (interior ones bulk-copied, boundary ones gathered behind them).
struct Layout {
    int rec, rp, sl, pos, xs, vs, xb, xbB, vb, vbB, fs, wb, act, hact, vB, total;
};

// `extras`: the stage also holds the step's actuation slices and, for
// cloth, the boundary velocities the air needs (a launch set reserves them
// only when one of its meshes has an actuation sequence or air on)
__host__ __device__ __forceinline__ Layout patch_layout(int kind, int n_e, int n_h, int n_loc, int n_int,
                                                        int n_slots, bool adjoint, bool extras) {
    const int n_rec = n_e + n_h;
    const int n_bnd = n_loc - n_int;
    Layout L;
    L.rec = 0;
    L.rp = L.rec + 64 * n_rec + 16;
    L.sl = L.rp + r16(2 * (n_loc + 1));
    L.pos = L.sl + r16(2 * n_slots);
    L.xs = L.pos + r16(4 * n_bnd);
    L.vs = L.xs + 16 * n_loc;
    // adjoint: x_bar of the interior nodes then of the boundary nodes (one
    // array over the local nodes), then v_hat likewise
    L.xb = L.vs + 16 * n_int;
    L.xbB = L.xb + (adjoint ? 16 * n_int : 0);
    L.vb = L.xbB + (adjoint ? 16 * n_bnd : 0);
    L.vbB = L.vb + (adjoint ? 16 * n_int : 0);
    // adjoint: the element force of the interior nodes at the step's state
    L.fs = L.vbB + (adjoint ? 16 * n_bnd : 0);
    // adjoint: dL/dw of the interior nodes
    L.wb = L.fs + (adjoint ? 16 * n_int : 0);
    // the step's row slices of a time-varying actuation (elements, hinges);
    // up to 3 entries of slack on each side for the aligned slice ends
    L.act = L.wb + (adjoint ? r16(8 * n_int) : 0);
    L.hact = L.act + (extras ? r16(4 * (n_e + 6)) : 0);
    // cloth: v of the boundary nodes (the air on the triangles needs every
    // corner's velocity)
    L.vB = L.hact + (extras && n_h ? r16(4 * (n_h + 6)) : 0);
    L.total = L.vB + (extras && kind == GS_CLOTH ? 16 * (n_loc - n_int) : 0);
    return L;
}

// cp.async 16 B global -> shared (LDGSTS), groups per thread
__device__ __forceinline__ void cp16(void* dst, const void* src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(saddr(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp8(void* dst, const void* src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(saddr(dst)), "l"(src) : "memory");
}
// order earlier generic-proxy accesses of shared memory before async-proxy writes
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// Contact geometry from the displacement u of node g.  The penetrations are
// formed from FP64-derived rest offsets so that FP32 keeps their relative
// precision near contact: plane C = (h - n.X) - n.u; sphere
// C = r - |d| = -(|X - c|^2 - r^2 + 2 (X - c).u + u.u) / (|d| + r), d = X - c + u.

// total contact force on a node: plane and sphere; `ph` = h - n.X of the
// node (carried in the .w lane of its velocity)
__device__ __forceinline__ float3 contact_force(const MeshRT& m, int g, float3 u, float3 v, float ph) {
    float3 f = make_float3(0.f, 0.f, 0.f);
    const ContactParams cp = cparams(m);
    if (m.plane_on) {
        const float3 n = make_float3(m.pnx, m.pny, m.pnz);
        const float C = ph - dot3(n, u);
        if (C > 0.0f) f += contact_one(v, n, C, cp);
    }
    if (m.sphere_on) {
        const float4 xs = m.Xs[g];
        const float3 d = xyz(xs) + u;
        const float q = xs.w + 2.0f * dot3(xyz(xs), u) + dot3(u, u);
        const float dist = sqrtf(dot3(d, d));
        const float C = -q / (dist + m.sr);
        if (C > 0.0f && dist > 0.0f) f += contact_one(v, d * (1.0f / dist), C, cp);
    }
    return f;
}

// reverse mode of contact_force: adds dL/du, dL/dv for fb = dL/df and returns f
__device__ __forceinline__ float3 contact_adjoint(const MeshRT& m, int g, float3 u, float3 v, float ph, float3 fb,
                                                  float3& xb, float3& vb) {
    float3 f = make_float3(0.f, 0.f, 0.f);
    const ContactParams cp = cparams(m);
    if (m.plane_on) {
        const float3 n = make_float3(m.pnx, m.pny, m.pnz);
        const float C = ph - dot3(n, u);
        if (C > 0.0f) {
            float3 vb1, nb, f1;
            float Cb;
            contact_one_adjoint(v, n, C, cp, fb, vb1, nb, Cb, f1);
            f += f1;
            vb += vb1;
            xb -= Cb * n;  // dC/du = -n
        }
    }
    if (m.sphere_on) {
        const float4 xs = m.Xs[g];
        const float3 d = xyz(xs) + u;
        const float q = xs.w + 2.0f * dot3(xyz(xs), u) + dot3(u, u);
        const float dist = sqrtf(dot3(d, d));
        const float C = -q / (dist + m.sr);
        if (C > 0.0f && dist > 0.0f) {
            const float inv = 1.0f / dist;
            const float3 n = d * inv;
            float3 vb1, nb, f1;
            float Cb;
            contact_one_adjoint(v, n, C, cp, fb, vb1, nb, Cb, f1);
            f += f1;
            vb += vb1;
            // n = d / dist, C = r - dist, dist = |d|, d = X - c + u
            const float distb = -Cb - dot3(nb, d) * inv * inv;
            xb += nb * inv + (distb * inv) * d;
        }
    }
    return f;
}

// forward node update (App. B): v+ = v + dt (w f + g [w > 0]), x+ = x + dt v+
__device__ __forceinline__ void node_forward(const MeshRT& m, int tick, int gid, float4 x4, float4 v4, float3 fel) {
    const float3 x = xyz(x4);  // displacement u
    float3 v = xyz(v4);
    const float w = x4.w;
    const float3 f = fel + contact_force(m, gid, x, v, v4.w);
    if (w > 0.0f) {
        v.x = v.x + m.dt * (w * f.x + m.gx);
        v.y = v.y + m.dt * (w * f.y + m.gy);
        v.z = v.z + m.dt * (w * f.z + m.gz);
    }
    const float3 xn = x + m.dt * v;
    m.st_f[(size_t)(m.in_a + m.in_b * tick) * (size_t)m.buf_stride + gid] = f4(fel, 0.f);
    const int ob = m.out_a + m.out_b * tick;
    const float4 xo = f4(xn, w), vo = f4(v, v4.w);
    bufx(m, ob)[gid] = xo;
    bufv(m, ob)[gid] = vo;
    if (tick == m.ck_tick) {
        bufx(m, m.ck_buf)[gid] = xo;
        bufv(m, m.ck_buf)[gid] = vo;
    }
    if (!(isfinite(xn.x) && isfinite(xn.y) && isfinite(xn.z) && isfinite(v.x) && isfinite(v.y) && isfinite(v.z)))
        atomicOr(m.status, 1);
}

// The adjoint state kept per node between reverse steps is x_bar = dL/du(n)
// and v_hat = dL/dv(n) + dt x_bar: the total dL/dv+ that the reverse of step
// n - 1 needs (x+ = x + dt v+), which is all the element phase reads of a
// node's velocity adjoint.  dL/dv(n) itself is v_hat - dt x_bar.
__device__ __forceinline__ float3 vhat_of(const MeshRT& m, float3 xb, float3 vb) { return vb + m.dt * xb; }

// reverse of node_forward for one node.  Inputs: state (u, v) at step n, the
// adjoint (xb, vh) of step n+1, the gathered element terms xsum = sum of
// corner dL/du, the elements' force fel on the node at step n (stored by the
// forward; the sum over the node's corners of f . v_hat is fel . v_hat), and
// dL/dw so far.  Writes the adjoint (x_bar, v_hat) of step n and the
// accumulated dL/dw (FP64).
__device__ __forceinline__ void node_adjoint(const MeshRT& m, int gid, float4 x4, float4 v4, float4 xb4, float4 vh4,
                                             float3 xsum, float3 fel, double wb_old, float3 vsum) {
    const float w = x4.w;
    const float3 xbn = xyz(xb4);
    const float3 vh = xyz(vh4);                 // dL/dv+ (total)
    const float3 fb = (m.dt * w) * vh;          // dL/df
    float3 xb = xbn + xsum;
    float3 vb = vh;
    const float3 fc = contact_adjoint(m, gid, xyz(x4), xyz(v4), v4.w, fb, xb, vb);
    vb += vsum;  // the elements' velocity-dependent forces (air), added last
    m.xb[gid] = f4(xb, 0.0f);
    m.vb[gid] = f4(vhat_of(m, xb, vb), 0.0f);
    m.wbar[gid] = wb_old + (double)(m.dt * (dot3(fel, vh) + dot3(fc, vh)));
}

// A staged patch in shared memory.
struct Stage {
    int n_rec, n_e, n_h;
    float4* rec;  // planes [4][n_rec]
    uint16_t* rp;
    uint16_t* sl;
    int* pos;     // partial positions of the boundary local nodes
    float4* xs;   // local node state (u, w)
    float4* vs;   // interior v
    float4* xb;   // adjoint: x_bar of the local nodes (interior, then boundary = xbB)
    float4* vb;   // adjoint: v_hat of the local nodes (interior, then boundary = vbB)
    float4* xbB;  // adjoint: boundary x_bar (gathered)
    float4* vbB;  // adjoint: boundary v_hat (gathered)
    float4* fs;   // adjoint: element force of the interior nodes at the step's state
    double* wb;   // adjoint: dL/dw of the interior nodes
    const float* act;   // this step's actuation of the patch's elements [n_e], or null
    const float* hact;  // this step's actuation of the patch's hinges [n_h], or null
    float4* vB;         // cloth with air: boundary v
    bool extras;        // the actuation slices and boundary v regions exist
};

__device__ __forceinline__ Stage stage_at(const PatchDesc& p, int kind, unsigned char* buf, bool adjoint,
                                          bool extras) {
    const int n_loc = p.n_int + p.n_bnd;
    const int n_rec = p.n_e + p.n_h;
    const Layout L = patch_layout(kind, p.n_e, p.n_h, n_loc, p.n_int, p.n_slots, adjoint, extras);
    Stage S;
    S.n_rec = n_rec;
    S.n_e = p.n_e;
    S.n_h = p.n_h;
    S.rec = (float4*)(buf + L.rec);
    S.rp = (uint16_t*)(buf + L.rp);
    S.sl = (uint16_t*)(buf + L.sl);
    S.pos = (int*)(buf + L.pos);
    S.xs = (float4*)(buf + L.xs);
    S.vs = (float4*)(buf + L.vs);
    S.xb = (float4*)(buf + L.xb);
    S.vb = (float4*)(buf + L.vb);
    S.xbB = (float4*)(buf + L.xbB);
    S.vbB = (float4*)(buf + L.vbB);
    S.fs = (float4*)(buf + L.fs);
    S.wb = (double*)(buf + L.wb);
    S.act = (const float*)(buf + L.act) + (p.e_begin & 3);
    S.hact = (const float*)(buf + L.hact) + (p.h_begin & 3);
    S.vB = (float4*)(buf + L.vB);
    S.extras = extras;
    return S;
}

// staged actuation of the current step, if the producer copied one
__device__ __forceinline__ void bind_act(Stage& S, const PatchDesc& p, const MeshRT& m, int tick) {
    if (!S.extras || act_row(m, m.act_seq, tick) < 0 || p.n_e == 0) S.act = nullptr;
    if (!S.extras || act_row(m, m.hact_seq, tick) < 0 || p.n_h == 0) S.hact = nullptr;
}
// the air acts on this stage's triangles (cloth with air on, region present)
__device__ __forceinline__ bool stage_air(const Stage& S, const MeshRT& m) { return S.extras && m.air_on; }
__device__ __forceinline__ float act_of(const float* a, int i) { return a ? a[i] : 0.f; }

// velocity of local node l (cloth with air: interior staged in vs, boundary in vB)
__device__ __forceinline__ float3 local_v(const Stage& S, const PatchDesc& p, int l) {
    return xyz(l < p.n_int ? S.vs[l] : S.vB[l - p.n_int]);
}
// air: the triangle's velocity through the air and its deformed vector area
// N = A (F0 x F1) (A the rest area: the rest frame has det Dm > 0)
__device__ __forceinline__ float3 air_vr(const MeshRT& m, const Stage& S, const PatchDesc& p, int i0, int i1, int i2) {
    return (local_v(S, p, i0) + local_v(S, p, i1) + local_v(S, p, i2)) * (1.0f / 3.0f) -
           make_float3(m.wx, m.wy, m.wz);
}

// state buffers a patch reads
__device__ __forceinline__ int in_buffer(const MeshRT& m, int tick, bool adjoint) {
    return adjoint ? m.adj_a + m.adj_b * tick : m.in_a + m.in_b * tick;
}

// Elected thread: bulk copies of the mesh record (into `hdr_rt`, unless the
// stage holds it already) and of the patch's records (one copy: they are
// patch-contiguous; hinges plane by plane), topology block (one copy) and
// interior node data into `buf`, completing on `bar`.
__device__ __forceinline__ void issue_bulk(const PatchDesc& p, const MeshRT* rt_global, const MeshRT& m, int tick,
                                           unsigned char* buf, MeshRT* hdr_rt, bool copy_rt, uint64_t* bar,
                                           bool adjoint, bool extras) {
    const Stage S = stage_at(p, m.kind, buf, adjoint, extras);
    const int n_loc = p.n_int + p.n_bnd;
    const int n_rec = S.n_rec;
    const int n_slots = p.n_slots;
    const int ib = in_buffer(m, tick, adjoint);
    const float4* X = bufx(m, ib);
    const float4* V = bufv(m, ib);
    const uint32_t b_rp = r16(2 * (n_loc + 1)), b_sl = r16(2 * n_slots), b_int = 16 * p.n_int;
    const uint32_t b_pos = (uint32_t)r16(4 * p.n_bnd);
    // this step's actuation rows, aligned slices around the patch's entries
    const int ra = extras && p.n_e ? act_row(m, m.act_seq, tick) : -1;
    const int rh = extras && p.n_h ? act_row(m, m.hact_seq, tick) : -1;
    const uint32_t b_act = ra >= 0 ? 4u * act_slice_n(p.e_begin, p.n_e) : 0u;
    const uint32_t b_hact = rh >= 0 ? 4u * act_slice_n(p.h_begin, p.n_h) : 0u;
    const uint32_t tx = (copy_rt ? (uint32_t)sizeof(MeshRT) : 0u) + 64u * n_rec + b_rp + b_sl + b_pos +
                        (p.n_int ? (adjoint ? 5u : 2u) * b_int : 0u) + b_act + b_hact;
    fence_proxy_async();
    mbar_expect_tx(bar, tx);
    if (copy_rt) bulk_g2s(hdr_rt, rt_global, (uint32_t)sizeof(MeshRT), bar);
    if (p.n_e) bulk_g2s(S.rec, m.rec + 4 * (size_t)p.e_begin, 64u * p.n_e, bar);
    for (int k = 0; k < 4 && p.n_h; ++k)
        bulk_g2s(S.rec + 4 * p.n_e + k * p.n_h, m.hrec + (size_t)k * m.n_hinges + p.h_begin, 16u * p.n_h, bar);
    bulk_g2s(S.rp, m.topo + p.topo, b_rp + b_sl + b_pos, bar);  // S.rp, S.sl, S.pos are consecutive
    if (p.n_int) {
        bulk_g2s(S.xs, X + p.int_begin, b_int, bar);
        bulk_g2s(S.vs, V + p.int_begin, b_int, bar);
        if (adjoint) {
            bulk_g2s(S.xb, m.xb + p.int_begin, b_int, bar);
            bulk_g2s(S.vb, m.vb + p.int_begin, b_int, bar);
            bulk_g2s(S.fs, m.st_f + (size_t)ib * (size_t)m.buf_stride + p.int_begin, b_int, bar);
        }
    }
    if (b_act)
        bulk_g2s((void*)(S.act - (p.e_begin & 3)), m.act_seq + (size_t)ra * m.act_ld + act_slice_lo(p.e_begin), b_act, bar);
    if (b_hact)
        bulk_g2s((void*)(S.hact - (p.h_begin & 3)), m.hact_seq + (size_t)rh * m.hact_ld + act_slice_lo(p.h_begin), b_hact,
                 bar);
}

// producer warp: asynchronous gather of the boundary nodes' state into `buf`;
// the ids of the first 128 boundary nodes
// (`g`, lane + 32 j) and the state pointer X were loaded ahead.  The adjoint
// also stages dL/dw of the interior nodes.
constexpr int kPrefetchIds = 4;

__device__ __forceinline__ void prefetch_ids(const PatchDesc& p, const MeshRT& m, int lane, int* g) {
#pragma unroll
    for (int j = 0; j < kPrefetchIds; ++j) {
        const int k = lane + 32 * j;
        g[j] = k < p.n_bnd ? m.bnd_ids[p.bnd_begin + k] : 0;
    }
}

__device__ __forceinline__ void produce_gather(const PatchDesc& p, const MeshRT& m, const float4* X, const float4* V,
                                               const int* g, unsigned char* buf, bool adjoint, bool extras, int lane) {
    const Stage S = stage_at(p, m.kind, buf, adjoint, extras);
    const bool gv = m.kind == GS_CLOTH && stage_air(S, m);  // boundary v for the air
#pragma unroll
    for (int j = 0; j < kPrefetchIds; ++j) {
        const int k = lane + 32 * j;
        if (k < p.n_bnd && idx_ok(g[j] >= m.n_int && g[j] < m.n_nodes, m.status)) {
            cp16(S.xs + p.n_int + k, X + g[j]);
            if (gv) cp16(S.vB + k, V + g[j]);
            if (adjoint) {
                cp16(S.xbB + k, m.xb + g[j]);
                cp16(S.vbB + k, m.vb + g[j]);
            }
        }
    }
    const int* ids = m.bnd_ids + p.bnd_begin;
    for (int k0 = 32 * kPrefetchIds; k0 < p.n_bnd; k0 += 32 * kPrefetchIds) {
        int h[kPrefetchIds];
#pragma unroll
        for (int j = 0; j < kPrefetchIds; ++j) {
            const int k = k0 + lane + 32 * j;
            h[j] = k < p.n_bnd ? ids[k] : 0;
        }
#pragma unroll
        for (int j = 0; j < kPrefetchIds; ++j) {
            const int k = k0 + lane + 32 * j;
            if (k < p.n_bnd && idx_ok(h[j] >= m.n_int && h[j] < m.n_nodes, m.status)) {
                cp16(S.xs + p.n_int + k, X + h[j]);
                if (gv) cp16(S.vB + k, V + h[j]);
                if (adjoint) {
                    cp16(S.xbB + k, m.xb + h[j]);
                    cp16(S.vbB + k, m.vb + h[j]);
                }
            }
        }
    }
    if (adjoint)
        for (int l = lane; l < p.n_int; l += 32) cp8(S.wb + l, m.wbar + p.int_begin + l);
}

// Staged records: the element planes [4][n_e], then the hinge planes
// [4][n_h].  Corner c of a record is written in place into its plane c; a CSR
// slot is that float4 index, or 4 * n_rec for a padding slot.
struct RecAt {
    int base, stride;  // plane k of the record at base + k * stride
};
__device__ __forceinline__ RecAt rec_slot(const Stage& S, int lr) {
    return lr < S.n_e ? RecAt{lr, S.n_e} : RecAt{4 * S.n_e + (lr - S.n_e), S.n_h};
}
__device__ __forceinline__ void put(const Stage& S, int r, int c, float4 f) { S.rec[c * S.n_e + r] = f; }  // elements
__device__ __forceinline__ void put(const Stage& S, RecAt q, int c, float4 f) { S.rec[q.base + c * q.stride] = f; }
__device__ __forceinline__ void zero_pad_slot(const Stage& S) {
    if (threadIdx.x == 0) S.rec[4 * S.n_rec] = make_float4(0.f, 0.f, 0.f, 0.f);  // a consumer thread
}

// ---------------------------------------------------------------------------
// element phases (one thread per element record)
// ---------------------------------------------------------------------------
__device__ __forceinline__ void tet_elements_fwd(const PatchDesc& p, const MeshRT& m, int tick, const Stage& S,
                                                 int nt) {
    const int nr = S.n_rec;
    zero_pad_slot(S);
    const int n_loc = p.n_int + p.n_bnd;
    for (int le = threadIdx.x; le < p.n_e; le += nt) {
        const float4 a = S.rec[le], b = S.rec[nr + le], c = S.rec[2 * nr + le], w = S.rec[3 * nr + le];
        const uint2 id = rec_ids(w);
        if (!idx_ok(ids_in(id, n_loc, 4), m.status)) continue;
        TetState s;
        tet_state(xyz(S.xs[id.x & 0xffff]), xyz(S.xs[id.x >> 16]), xyz(S.xs[id.y & 0xffff]), xyz(S.xs[id.y >> 16]), a,
                  b, c, w.z + act_of(S.act, le), s);
        float3 f0, f1, f2, f3;
        tet_forces(s, a, b, c, f0, f1, f2, f3);
        put(S, le, 0, f4(f0, 0.f));
        put(S, le, 1, f4(f1, 0.f));
        put(S, le, 2, f4(f2, 0.f));
        put(S, le, 3, f4(f3, 0.f));
    }
}

__device__ __forceinline__ void cloth_elements_fwd(const PatchDesc& p, const MeshRT& m, int tick, const Stage& S,
                                                   int nt) {
    const int nr = S.n_rec;
    zero_pad_slot(S);
    const int n_loc = p.n_int + p.n_bnd;
    for (int lr = threadIdx.x; lr < nr; lr += nt) {
        const RecAt q = rec_slot(S, lr);
        const float4 a = S.rec[q.base], c = S.rec[q.base + 2 * q.stride], w = S.rec[q.base + 3 * q.stride];
        float4 b = S.rec[q.base + q.stride];
        const uint2 id = rec_ids(w);
        if (!idx_ok(ids_in(id, n_loc, lr < p.n_e ? 3 : 4), m.status)) continue;
        if (lr < p.n_e) {
            TriState s;
            b.w += act_of(S.act, lr);  // actuation (b.w)
            tri_state(xyz(S.xs[id.x & 0xffff]), xyz(S.xs[id.x >> 16]), xyz(S.xs[id.y & 0xffff]), a, b,
                      make_float3(c.x, c.y, c.z), make_float3(c.w, w.z, w.w), s);
            float3 f0, f1, f2;
            tri_forces(s, a, b, f0, f1, f2);
            if (stage_air(S, m)) {
                const float3 vr = air_vr(m, S, p, id.x & 0xffff, id.x >> 16, id.y & 0xffff);
                const float3 Fa = air_force(b.x * cross3(s.F0, s.F1), vr, m.k_drag, m.k_lift) * (1.0f / 3.0f);
                f0 += Fa;
                f1 += Fa;
                f2 += Fa;
            }
            put(S, q, 0, f4(f0, 0.f));
            put(S, q, 1, f4(f1, 0.f));
            put(S, q, 2, f4(f2, 0.f));
        } else {
            HingeState s;
            hinge_state(xyz(S.xs[id.x & 0xffff]), xyz(S.xs[id.x >> 16]), xyz(S.xs[id.y & 0xffff]),
                        xyz(S.xs[id.y >> 16]), xyz(a), xyz(b), xyz(c),
                        b.w + act_of(S.hact, lr - p.n_e), s);
            float3 f1, f2, f3, f4_;
            hinge_forces(s, a.w, f1, f2, f3, f4_);
            put(S, q, 0, f4(f1, 0.f));
            put(S, q, 1, f4(f2, 0.f));
            put(S, q, 2, f4(f3, 0.f));
            put(S, q, 3, f4(f4_, 0.f));
        }
    }
}

// adds one step's (dL/dmu, dL/dlambda) of an element to its FP64 accumulator
// as fire-and-forget reductions in L2: one thread owns an element per launch
// and the launches are ordered, so each entry receives its terms one per step
// in step order, each rounded once, as a load / add / store would
__device__ __forceinline__ void accumulate_ml(double2* g, float gmu, float glam) {
    atomicAdd(&g->x, (double)gmu);
    atomicAdd(&g->y, (double)glam);
}

// v_hat = v_bar + dt x_bar (dL/dv+, App. B) of local node l: the stage holds
// the adjoint state as (x_bar, v_hat)
__device__ __forceinline__ float3 vhat(const Stage& S, int l) { return xyz(S.vb[l]); }

// corner result dL/du_corner in place (the fourth lane is unused: the
// dL/dw term takes the stored element force of the node)
__device__ __forceinline__ void tet_elements_adj(const PatchDesc& p, const MeshRT& m, int tick, const Stage& S,
                                                 int nt) {
    const float dt = m.dt;
    const int nr = S.n_rec;
    zero_pad_slot(S);
    const int n_loc = p.n_int + p.n_bnd;
    for (int le = threadIdx.x; le < p.n_e; le += nt) {
        const float4 a = S.rec[le], b = S.rec[nr + le], c = S.rec[2 * nr + le], w = S.rec[3 * nr + le];
        const uint2 id = rec_ids(w);
        if (!idx_ok(ids_in(id, n_loc, 4), m.status)) continue;
        const int i0 = id.x & 0xffff, i1 = id.x >> 16, i2 = id.y & 0xffff, i3 = id.y >> 16;
        const float4 x0 = S.xs[i0], x1 = S.xs[i1], x2 = S.xs[i2], x3 = S.xs[i3];
        const float3 v0 = vhat(S, i0), v1 = vhat(S, i1), v2 = vhat(S, i2), v3 = vhat(S, i3);
        TetState s;
        tet_state(xyz(x0), xyz(x1), xyz(x2), xyz(x3), a, b, c, w.z + act_of(S.act, le), s);
        float3 xb0, xb1, xb2, xb3;
        float gmu, glam, gact;
        tet_adjoint(s, a, b, c, (dt * x0.w) * v0, (dt * x1.w) * v1, (dt * x2.w) * v2, (dt * x3.w) * v3, xb0, xb1,
                    xb2, xb3, gmu, glam, gact);
        put(S, le, 0, f4(xb0, 0.f));
        put(S, le, 1, f4(xb1, 0.f));
        put(S, le, 2, f4(xb2, 0.f));
        put(S, le, 3, f4(xb3, 0.f));
        const int e = p.e_begin + le;
        accumulate_ml(m.g_ml + e, gmu, glam);
        if (m.g_act) m.g_act[e] += (double)gact;
        act_grad_step(m, m.d_act_seq, m.act_ld, tick, e, gact);
    }
}

__device__ __forceinline__ void cloth_elements_adj(const PatchDesc& p, const MeshRT& m, int tick, const Stage& S,
                                                   int nt) {
    const float dt = m.dt;
    const int nr = S.n_rec;
    zero_pad_slot(S);
    const int n_loc = p.n_int + p.n_bnd;
    for (int lr = threadIdx.x; lr < nr; lr += nt) {
        const RecAt q = rec_slot(S, lr);
        const float4 a = S.rec[q.base], b = S.rec[q.base + q.stride], c = S.rec[q.base + 2 * q.stride],
                     w = S.rec[q.base + 3 * q.stride];
        const uint2 id = rec_ids(w);
        if (!idx_ok(ids_in(id, n_loc, lr < p.n_e ? 3 : 4), m.status)) continue;
        if (lr < p.n_e) {
            const int i0 = id.x & 0xffff, i1 = id.x >> 16, i2 = id.y & 0xffff;
            const float4 x0 = S.xs[i0], x1 = S.xs[i1], x2 = S.xs[i2];
            const float3 v0 = vhat(S, i0), v1 = vhat(S, i1), v2 = vhat(S, i2);
            TriState s;
            float4 bt = b;
            bt.w += act_of(S.act, lr);  // actuation (b.w)
            tri_state(xyz(x0), xyz(x1), xyz(x2), a, bt, make_float3(c.x, c.y, c.z), make_float3(c.w, w.z, w.w), s);
            float3 xb0, xb1, xb2;
            float gmu, glam, gact;
            const float3 y0 = (dt * x0.w) * v0, y1 = (dt * x1.w) * v1, y2 = (dt * x2.w) * v2;
            tri_adjoint(s, a, bt, y0, y1, y2, xb0, xb1, xb2, gmu, glam, gact);
            if (stage_air(S, m)) {
                // F on each corner F/3: dL/dF = (y0 + y1 + y2)/3; N = A (F0 x F1)
                const float3 vr = air_vr(m, S, p, i0, i1, i2);
                const float3 N = b.x * cross3(s.F0, s.F1);
                float3 Nb = make_float3(0.f, 0.f, 0.f), vrb = make_float3(0.f, 0.f, 0.f);
                air_adjoint(N, vr, m.k_drag, m.k_lift, (y0 + y1 + y2) * (1.0f / 3.0f), Nb, vrb);
                const float3 F0b = b.x * cross3(s.F1, Nb), F1b = b.x * cross3(Nb, s.F0);
                const float3 d1 = F0b * a.x + F1b * a.y, d2 = F0b * a.z + F1b * a.w;
                xb1 += d1;
                xb2 += d2;
                xb0 -= d1 + d2;
                // the same dL/dv for each corner, summed per node by the node phase
                put(S, q, 3, f4(vrb * (1.0f / 3.0f), 0.f));
            }
            put(S, q, 0, f4(xb0, 0.f));
            put(S, q, 1, f4(xb1, 0.f));
            put(S, q, 2, f4(xb2, 0.f));
            const int t = p.e_begin + lr;
            accumulate_ml(m.g_ml + t, gmu, glam);
            if (m.g_act) m.g_act[t] += (double)gact;
            act_grad_step(m, m.d_act_seq, m.act_ld, tick, t, gact);
        } else {
            const int i1 = id.x & 0xffff, i2 = id.x >> 16, i3 = id.y & 0xffff, i4 = id.y >> 16;
            const float4 x1 = S.xs[i1], x2 = S.xs[i2], x3 = S.xs[i3], x4 = S.xs[i4];
            const float3 v1 = vhat(S, i1), v2 = vhat(S, i2), v3 = vhat(S, i3), v4 = vhat(S, i4);
            HingeState s;
            hinge_state(xyz(x1), xyz(x2), xyz(x3), xyz(x4), xyz(a), xyz(b), xyz(c),
                        b.w + act_of(S.hact, lr - p.n_e), s);
            float3 xb1, xb2, xb3, xb4;
            float gkb, gact;
            hinge_adjoint(s, a.w, (dt * x1.w) * v1, (dt * x2.w) * v2, (dt * x3.w) * v3, (dt * x4.w) * v4, xb1, xb2,
                          xb3, xb4, gkb, gact);
            put(S, q, 0, f4(xb1, 0.f));
            put(S, q, 1, f4(xb2, 0.f));
            put(S, q, 2, f4(xb3, 0.f));
            put(S, q, 3, f4(xb4, 0.f));
            const int h = p.h_begin + (lr - p.n_e);
            m.g_kb[h] += (double)gkb;
            if (m.g_hact) m.g_hact[h] += (double)gact;
            act_grad_step(m, m.d_hact_seq, m.hact_ld, tick, h, gact);
        }
    }
}

// Fixed-order sum of the corner results of CSR row [k, k1): rows are padded
// to a multiple of 4 (padding slots read a zero float4), so four slot indices
// come in one 8 B load and all four corner loads are issued before the adds;
// the adds stay in row order.  The forward sums 3 lanes, the adjoint 4.
__device__ __forceinline__ void add4(float4& acc, float4 q) {
    acc.x += q.x;
    acc.y += q.y;
    acc.z += q.z;
    acc.w += q.w;
}
__device__ __forceinline__ void add3(float3& acc, float4 q) {
    acc.x += q.x;
    acc.y += q.y;
    acc.z += q.z;
}
// software-pipelined: the next group's slot and corner loads are issued
// before the current group's adds
#define GS_ROW_SUM(T, ADD, ZERO)                                                                            \
    T acc = ZERO;                                                                                           \
    if (k >= k1) return acc;                                                                                \
    uint2 q = checked_slots(*reinterpret_cast<const uint2*>(S.sl + k), S.n_rec, status);                   \
    float4 c0 = S.rec[q.x & 0xffff], c1 = S.rec[q.x >> 16], c2 = S.rec[q.y & 0xffff], c3 = S.rec[q.y >> 16]; \
    for (k += 4; k < k1; k += 4) {                                                                          \
        q = checked_slots(*reinterpret_cast<const uint2*>(S.sl + k), S.n_rec, status);                     \
        const float4 n0 = S.rec[q.x & 0xffff], n1 = S.rec[q.x >> 16], n2 = S.rec[q.y & 0xffff],              \
                     n3 = S.rec[q.y >> 16];                                                                 \
        ADD(acc, c0);                                                                                       \
        ADD(acc, c1);                                                                                       \
        ADD(acc, c2);                                                                                       \
        ADD(acc, c3);                                                                                       \
        c0 = n0;                                                                                            \
        c1 = n1;                                                                                            \
        c2 = n2;                                                                                            \
        c3 = n3;                                                                                            \
    }                                                                                                       \
    ADD(acc, c0);                                                                                           \
    ADD(acc, c1);                                                                                           \
    ADD(acc, c2);                                                                                           \
    ADD(acc, c3);                                                                                           \
    return acc;

__device__ __forceinline__ float4 row_sum4(const Stage& S, int k, int k1, int* status) {
    GS_ROW_SUM(float4, add4, make_float4(0.f, 0.f, 0.f, 0.f))
}
__device__ __forceinline__ float3 row_sum3(const Stage& S, int k, int k1, int* status) {
    GS_ROW_SUM(float3, add3, make_float3(0.f, 0.f, 0.f))
}
// a local CSR row [k, k1): 4-aligned (padded rows) and inside the patch's slots
__device__ __forceinline__ bool row_ok(int k, int k1, int n_slots, int* status) {
    return idx_ok(k <= k1 && k1 <= n_slots && (k & 3) == 0 && (k1 & 3) == 0, status);
}
#undef GS_ROW_SUM

// node phases: fixed-order corner sums, then interior update or partial
__device__ __forceinline__ void forward_nodes(const PatchDesc& p, const MeshRT& m, int tick, const Stage& S, int nt) {
    const int n_loc = p.n_int + p.n_bnd;
    if (!idx_ok(p.int_begin >= 0 && p.int_begin + p.n_int <= m.n_int, m.status)) return;
    for (int l = threadIdx.x; l < n_loc; l += nt) {
        const int k = S.rp[l], k1 = S.rp[l + 1];
        if (!row_ok(k, k1, p.n_slots, m.status)) continue;
        const float3 f = row_sum3(S, k, k1, m.status);
        if (l < p.n_int) {
            node_forward(m, tick, p.int_begin + l, S.xs[l], S.vs[l], f);
        } else {
            const int pp = S.pos[l - p.n_int];
            if (idx_ok(pp >= 0 && pp < m.n_part, m.status)) m.partials[pp] = f4(f, 0.f);
        }
    }
}

// cloth with air: fixed-order sum over the node's triangle corners of the
// triangles' dL/dv (plane 3 of a triangle record; slot c n_e + r with c < 3
// is corner c of triangle r, hinge and padding slots add nothing)
__device__ __forceinline__ float3 row_sum_air_v(const Stage& S, int k, int k1) {
    float3 acc = make_float3(0.f, 0.f, 0.f);
    const int ne = S.n_e;
    for (; k < k1; ++k) {
        const int s = S.sl[k];
        if (s < 3 * ne) {
            const int r = s - ne * ((s >= ne) + (s >= 2 * ne));
            add3(acc, S.rec[3 * ne + r]);
        }
    }
    return acc;
}

template <int KIND>
__device__ __forceinline__ void adjoint_nodes(const PatchDesc& p, const MeshRT& m, const Stage& S, int nt) {
    const int n_loc = p.n_int + p.n_bnd;
    const bool air = KIND == GS_CLOTH && stage_air(S, m);
    if (!idx_ok(p.int_begin >= 0 && p.int_begin + p.n_int <= m.n_int, m.status)) return;
    for (int l = threadIdx.x; l < n_loc; l += nt) {
        const int k = S.rp[l], k1 = S.rp[l + 1];
        if (!row_ok(k, k1, p.n_slots, m.status)) continue;
        const float4 acc = row_sum4(S, k, k1, m.status);
        const float3 va = air ? row_sum_air_v(S, k, k1) : make_float3(0.f, 0.f, 0.f);
        if (l < p.n_int) {
            node_adjoint(m, p.int_begin + l, S.xs[l], S.vs[l], S.xb[l], S.vb[l], xyz(acc), xyz(S.fs[l]), S.wb[l], va);
        } else {
            const int pp = S.pos[l - p.n_int];
            if (!idx_ok(pp >= 0 && pp < m.n_part, m.status)) continue;
            m.partials[pp] = acc;
            if (air) m.partials_v[pp] = f4(va, 0.f);
        }
    }
}


// ---------------------------------------------------------------------------
// The pipeline: a persistent CTA walks the live patches blockIdx.x,
// +gridDim.x, ... through kStages shared-memory stages, warp-specialised.  The
// last warp produces: it finds the next live patch, waits until the
// consumers released the stage (empty[s]), writes the patch descriptor into
// the stage header, issues the bulk copies (one elected lane, expect_tx on
// full[s]) and the boundary gathers (all lanes, each lane's cp.async copies
// counted on full[s] by a no-increment arrival).  The other warps consume:
// wait for full[s], run the element phase, sync among themselves (named
// barrier 1), run the node phase and release the stage.  After the last patch
// the producer fills one more stage with an end marker.
// full[s] completes after 33 arrivals (the elected lane's expect_tx + one per
// producer lane) and the expected bytes; empty[s] after one arrival per
// consumer warp.
// ---------------------------------------------------------------------------
// stage header: the patch descriptor at 0, the mesh record at kHdrRt
constexpr int kHdrRt = 64;
constexpr int kHdr = kHdrRt + (int)((sizeof(MeshRT) + 63) / 64 * 64);

__device__ __forceinline__ void consumer_sync(int nt) { asm volatile("bar.sync 1, %0;" ::"r"(nt) : "memory"); }

// hint: bring [p, p + bytes) into L2 (16 B aligned, a multiple of 16 B)
__device__ __forceinline__ void l2_prefetch(const void* p, uint32_t bytes) {
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"(bytes) : "memory");
}

// Run by the producer warp once its CTA has no patch left.  The next launch of
// the same kernel gives this CTA the same patches, and its first two start
// cold (nothing else overlaps the stage fill at the start of a launch), so
// their records, topology block and boundary ids are brought into L2 now,
// with this CTA's slice of the boundary row pointers that the boundary kernel
// between the two launches reads.  Hints only: the data are constant over a
// rollout and nothing depends on the prefetch.
__device__ __forceinline__ void prefetch_next_launch(const PatchDesc* __restrict__ patches, int n_patches,
                                                     const MeshRT* __restrict__ rts, const MeshRT* prt, int rt_mesh,
                                                     int lane) {
    if (lane < 2) {
        const int q = blockIdx.x + lane * gridDim.x;
        if (q < n_patches) {
            const PatchDesc pq = patches[q];
            const MeshRT& mq = pq.mesh == rt_mesh ? *prt : rts[pq.mesh];
            const uint32_t bt = r16(2 * (pq.n_int + pq.n_bnd + 1)) + r16(2 * pq.n_slots) + r16(4 * pq.n_bnd);
            if (pq.n_e) l2_prefetch(mq.rec + 4 * (size_t)pq.e_begin, 64u * pq.n_e);
            l2_prefetch(mq.topo + pq.topo, bt);
            if (pq.n_bnd >= 4) l2_prefetch(mq.bnd_ids + pq.bnd_begin, (4u * pq.n_bnd) & ~15u);
        }
    } else if (lane == 2 && rt_mesh >= 0 && prt->n_bnd > 0) {
        const int per = ((prt->n_bnd + 1 + (int)gridDim.x - 1) / (int)gridDim.x + 3) & ~3;
        const int lo = blockIdx.x * per;
        const int hi = min(lo + per, (prt->n_bnd + 1) & ~3);
        if (hi - lo >= 4) l2_prefetch(prt->bnd_rowptr + lo, 4u * (uint32_t)(hi - lo));
    }
}

// first live patch at or after `pi` in steps of gridDim.x; `cached` is the
// record of mesh `cached_mesh` in shared memory (or null)
__device__ __forceinline__ int next_live(const PatchDesc* __restrict__ patches, int n_patches,
                                         const MeshRT* __restrict__ rts, int pi, int mask,
                                         const MeshRT* cached = nullptr, int cached_mesh = -1) {
    for (; pi < n_patches; pi += gridDim.x) {
        const int pm = patches[pi].mesh;
        if ((pm == cached_mesh && cached ? cached->active : rts[pm].active) & mask) break;
    }
    return pi;
}

// the producer warp's copy of a mesh record in shared memory: every field it
// reads per patch comes from there instead of a chain of global loads
__device__ __forceinline__ void load_producer_rt(MeshRT* dst, const MeshRT* src, int lane) {
    const int* s = reinterpret_cast<const int*>(src);
    int* d = reinterpret_cast<int*>(dst);
    for (int k = lane; k < (int)(sizeof(MeshRT) / sizeof(int)); k += 32) d[k] = s[k];
    __syncwarp();
}

template <int KIND, bool ADJ>
__device__ __forceinline__ void patch_pipeline(const PatchDesc* __restrict__ patches, int n_patches,
                                               const MeshRT* __restrict__ rts, int tick, int stage_bytes,
                                               int extras) {
    extern __shared__ __align__(128) unsigned char sm[];
    uint64_t* full = (uint64_t*)sm;
    uint64_t* empty = full + kStages;
    unsigned char* const buf0 = sm + kPipeHead;
    MeshRT* const prt = reinterpret_cast<MeshRT*>(buf0 + kStages * stage_bytes);  // the producer's mesh record
    const int mask = ADJ ? ACT_ADJ : ACT_FWD;
    const int nt = (int)blockDim.x - 32;  // consumer threads
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        for (int s = 0; s < kStages; ++s) {
            mbar_init(&full[s], 33);
            mbar_init(&empty[s], nt >> 5);
            ((PatchDesc*)(buf0 + s * stage_bytes))->mesh = -1;  // no mesh record staged yet
        }
        mbar_init_fence();
    }
    __syncthreads();
    pdl_enter();
    if (n_patches <= 0) return;
    int* const status = rts[patches[blockIdx.x < n_patches ? blockIdx.x : 0].mesh].status;
    if (warp == (nt >> 5)) {
        // ---- producer warp: the next patch's descriptor, boundary ids and
        // state pointer are loaded while waiting for its stage ----
        int pi = next_live(patches, n_patches, rts, blockIdx.x, mask);
        int rt_mesh = -1;  // the mesh whose record *prt holds
        PatchDesc p;
        int g[kPrefetchIds];
        const float4* X = nullptr;
        const float4* V = nullptr;
        if (pi < n_patches) {
            p = patches[pi];
            load_producer_rt(prt, &rts[p.mesh], lane);
            rt_mesh = p.mesh;
            prefetch_ids(p, *prt, lane, g);
            X = bufx(*prt, in_buffer(*prt, tick, ADJ));
            V = bufv(*prt, in_buffer(*prt, tick, ADJ));
        }
        for (int it = 0;; ++it) {
            const int s = it % kStages;
            unsigned char* const b = buf0 + s * stage_bytes;
            if (it >= kStages && !mbar_wait_bounded(&empty[s], (it / kStages - 1) & 1u, status)) return;
            if (pi >= n_patches) {
                if (lane == 0) ((PatchDesc*)b)->n_e = -1;  // end marker
                __syncwarp();
                mbar_arrive(&full[s]);
                if (lane == 0) mbar_arrive(&full[s]);
                prefetch_next_launch(patches, n_patches, rts, prt, rt_mesh, lane);
                return;
            }
            const MeshRT& m = *prt;  // the record of p.mesh
            if (kChecked) {
                // the patch's stage fits the stage the launch reserved and its
                // local ids fit 16 bits; otherwise it is replaced by an empty patch
                const Layout Lc = patch_layout(m.kind, p.n_e, p.n_h, p.n_int + p.n_bnd, p.n_int, p.n_slots, ADJ,
                                               extras != 0);
                if (!idx_ok(kHdr + Lc.total <= stage_bytes && p.n_int + p.n_bnd < 65536 && 4 * (p.n_e + p.n_h) < 65535,
                            m.status)) {
                    p.n_e = p.n_h = p.n_int = p.n_bnd = p.n_slots = 0;
                }
            }
            if (lane == 0) {
                // the stage keeps its mesh record from the last patch it held
                const bool copy_rt = ((const PatchDesc*)b)->mesh != p.mesh;
                *(PatchDesc*)b = p;
                issue_bulk(p, &rts[p.mesh], m, tick, b + kHdr, (MeshRT*)(b + kHdrRt), copy_rt, &full[s], ADJ, extras != 0);
            }
            produce_gather(p, m, X, V, g, b + kHdr, ADJ, extras != 0, lane);
            cp_async_mbar_arrive(&full[s]);
            pi = next_live(patches, n_patches, rts, pi + gridDim.x, mask, prt, rt_mesh);
            if (pi < n_patches) {
                p = patches[pi];
                if (p.mesh != rt_mesh) {
                    load_producer_rt(prt, &rts[p.mesh], lane);
                    rt_mesh = p.mesh;
                }
                prefetch_ids(p, *prt, lane, g);
                X = bufx(*prt, in_buffer(*prt, tick, ADJ));
                V = bufv(*prt, in_buffer(*prt, tick, ADJ));
            }
        }
    }
    // ---- consumer warps: descriptor and mesh record from the stage header ----
    for (int it = 0;; ++it) {
        const int s = it % kStages;
        unsigned char* const b = buf0 + s * stage_bytes;
        if (!mbar_wait_bounded(&full[s], (it / kStages) & 1u, status)) return;
        const PatchDesc p = *(const PatchDesc*)b;
        if (p.n_e < 0) {
            pdl_done();
            return;
        }
        const MeshRT& m = *(const MeshRT*)(b + kHdrRt);
        Stage S = stage_at(p, KIND, b + kHdr, ADJ, extras != 0);
        bind_act(S, p, m, tick);
        if (KIND == GS_TET) {
            if (ADJ) tet_elements_adj(p, m, tick, S, nt);
            else tet_elements_fwd(p, m, tick, S, nt);
        } else {
            if (ADJ) cloth_elements_adj(p, m, tick, S, nt);
            else cloth_elements_fwd(p, m, tick, S, nt);
        }
        consumer_sync(nt);
        if (ADJ) adjoint_nodes<KIND>(p, m, S, nt);
        else forward_nodes(p, m, tick, S, nt);
        // this warp's generic shared accesses of the stage are ordered before the
        // async-proxy writes that will refill it
        fence_proxy_async();
        __syncwarp();
        if (lane == 0) mbar_arrive(&empty[s]);
    }
}

}  // namespace

// ===========================================================================
// patch kernels (persistent, pipelined)
// ===========================================================================
__global__ void k_tet_fwd(const PatchDesc* __restrict__ patches, int n_patches, const MeshRT* __restrict__ rts,
                          int tick, int stage_bytes, int extras) {
    patch_pipeline<GS_TET, false>(patches, n_patches, rts, tick, stage_bytes, extras);
}
__global__ void k_cloth_fwd(const PatchDesc* __restrict__ patches, int n_patches, const MeshRT* __restrict__ rts,
                            int tick, int stage_bytes, int extras) {
    patch_pipeline<GS_CLOTH, false>(patches, n_patches, rts, tick, stage_bytes, extras);
}
__global__ void k_tet_adj(const PatchDesc* __restrict__ patches, int n_patches, const MeshRT* __restrict__ rts,
                          int tick, int stage_bytes, int extras) {
    patch_pipeline<GS_TET, true>(patches, n_patches, rts, tick, stage_bytes, extras);
}
// capped at 128 registers: 144 left 2 CTAs of 5 warps per SM; at 128 (a few
// spilled values) 3 fit, and the 256^2 cloth's adjoint runs 18 % faster
__global__ void __maxnreg__(128) k_cloth_adj(const PatchDesc* __restrict__ patches, int n_patches,
                                              const MeshRT* __restrict__ rts, int tick, int stage_bytes,
                                              int extras) {
    patch_pipeline<GS_CLOTH, true>(patches, n_patches, rts, tick, stage_bytes, extras);
}

// Boundary nodes: sum the node's partials (contiguous, in patch order), then
// finish the node.  A CTA of 128 threads takes a 256-node block, two nodes
// per thread, with every independent load of both nodes issued before the
// dependent ones; CTAs stride over the blocks (grid sized to one wave).  The
// row pointers and the node's state (written by the boundary kernel of the
// previous step, which completed before the patch kernel in between could
// signal its dependents) are loaded before waiting on that patch kernel, so
// a CTA that starts during its tail has them in flight already.
constexpr int kBndThreads = kNodeBlock / 2;

// fixed-order sums of the partials [k0, k0 + n0) and [k1, k1 + n1), four
// loads of each row in flight per round (absent terms read as zero)
__device__ __forceinline__ void partial_sums2(const float4* __restrict__ P, int k0, int n0, int k1, int n1, float4& a0,
                                              float4& a1) {
    const float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
    a0 = z;
    a1 = z;
    const int n = n0 > n1 ? n0 : n1;
    for (int j = 0; j < n; j += 4) {
        float4 q0[4], q1[4];
#pragma unroll
        for (int t = 0; t < 4; ++t) {
            q0[t] = j + t < n0 ? P[k0 + j + t] : z;
            q1[t] = j + t < n1 ? P[k1 + j + t] : z;
        }
#pragma unroll
        for (int t = 0; t < 4; ++t) {
            add4(a0, q0[t]);
            add4(a1, q1[t]);
        }
    }
}

__global__ void __launch_bounds__(kBndThreads, 8)
    k_fwd_boundary(const NodeBlock* __restrict__ blocks, int n_blocks, const MeshRT* __restrict__ rts, int tick) {
    for (int bi = blockIdx.x; bi < n_blocks; bi += gridDim.x) {
        const NodeBlock nb = blocks[bi];
        const MeshRT& m = rts[nb.mesh];
        if (!(m.active & ACT_FWD)) continue;
        const int ib = m.in_a + m.in_b * tick;
        const float4* X = bufx(m, ib);
        const float4* V = bufv(m, ib);
        const int i0 = threadIdx.x, i1 = threadIdx.x + kBndThreads;
        bool h0 = i0 < nb.count, h1 = i1 < nb.count;
        const int b0 = nb.begin + i0, b1 = nb.begin + i1;
        int k0 = 0, e0 = 0, k1 = 0, e1 = 0;
        float4 x0, v0, x1, v1;
        if (kChecked) {
            h0 = h0 && idx_ok(b0 >= 0 && b0 < m.n_bnd, m.status);
            h1 = h1 && idx_ok(b1 >= 0 && b1 < m.n_bnd, m.status);
        }
        if (h0) {
            k0 = m.bnd_rowptr[b0];
            e0 = m.bnd_rowptr[b0 + 1];
            x0 = X[m.n_int + b0];
            v0 = V[m.n_int + b0];
        }
        if (h1) {
            k1 = m.bnd_rowptr[b1];
            e1 = m.bnd_rowptr[b1 + 1];
            x1 = X[m.n_int + b1];
            v1 = V[m.n_int + b1];
        }
        if (kChecked) {
            if (!idx_ok(!h0 || (b0 < m.n_bnd && 0 <= k0 && k0 <= e0 && e0 <= m.n_part), m.status)) h0 = false, k0 = e0 = 0;
            if (!idx_ok(!h1 || (b1 < m.n_bnd && 0 <= k1 && k1 <= e1 && e1 <= m.n_part), m.status)) h1 = false, k1 = e1 = 0;
        }
        // only the partials come from the patch kernel this launch follows
        pdl_enter();
        float4 f0, f1;
        partial_sums2(m.partials, k0, e0 - k0, k1, e1 - k1, f0, f1);
        if (h0) node_forward(m, tick, m.n_int + b0, x0, v0, xyz(f0));
        if (h1) node_forward(m, tick, m.n_int + b1, x1, v1, xyz(f1));
    }
    pdl_done();
}

__global__ void __launch_bounds__(kBndThreads, 6)
    k_adj_boundary(const NodeBlock* __restrict__ blocks, int n_blocks, const MeshRT* __restrict__ rts, int tick) {
    for (int bi = blockIdx.x; bi < n_blocks; bi += gridDim.x) {
        const NodeBlock nb = blocks[bi];
        const MeshRT& m = rts[nb.mesh];
        if (!(m.active & ACT_ADJ)) continue;
        const int sb = m.adj_a + m.adj_b * tick;
        const float4* X = bufx(m, sb);
        const float4* V = bufv(m, sb);
        const float4* F = m.st_f + (size_t)sb * (size_t)m.buf_stride;
        const int i0 = threadIdx.x, i1 = threadIdx.x + kBndThreads;
        bool h0 = i0 < nb.count, h1 = i1 < nb.count;
        const int b0 = nb.begin + i0, b1 = nb.begin + i1;
        const int g0 = m.n_int + b0, g1 = m.n_int + b1;
        if (kChecked) {
            h0 = h0 && idx_ok(b0 >= 0 && b0 < m.n_bnd, m.status);
            h1 = h1 && idx_ok(b1 >= 0 && b1 < m.n_bnd, m.status);
        }
        int k0 = 0, e0 = 0, k1 = 0, e1 = 0;
        float4 x0, v0, xb0, vb0, f0, x1, v1, xb1, vb1, f1;
        double w0 = 0.0, w1 = 0.0;
        if (h0) {
            k0 = m.bnd_rowptr[b0];
            e0 = m.bnd_rowptr[b0 + 1];
            x0 = X[g0];
            v0 = V[g0];
            xb0 = m.xb[g0];
            vb0 = m.vb[g0];
            f0 = F[g0];
            w0 = m.wbar[g0];
        }
        if (h1) {
            k1 = m.bnd_rowptr[b1];
            e1 = m.bnd_rowptr[b1 + 1];
            x1 = X[g1];
            v1 = V[g1];
            xb1 = m.xb[g1];
            vb1 = m.vb[g1];
            f1 = F[g1];
            w1 = m.wbar[g1];
        }
        if (kChecked) {
            if (!idx_ok(!h0 || (b0 < m.n_bnd && 0 <= k0 && k0 <= e0 && e0 <= m.n_part), m.status)) h0 = false, k0 = e0 = 0;
            if (!idx_ok(!h1 || (b1 < m.n_bnd && 0 <= k1 && k1 <= e1 && e1 <= m.n_part), m.status)) h1 = false, k1 = e1 = 0;
        }
        // only the partials come from the patch kernel this launch follows
        pdl_enter();
        float4 a0, a1;
        partial_sums2(m.partials, k0, e0 - k0, k1, e1 - k1, a0, a1);
        const float3 z = make_float3(0.f, 0.f, 0.f);
        if (h0) node_adjoint(m, g0, x0, v0, xb0, vb0, xyz(a0), xyz(f0), w0, z);
        if (h1) node_adjoint(m, g1, x1, v1, xb1, vb1, xyz(a1), xyz(f1), w1, z);
    }
    pdl_done();
}

// Cloth with air, after k_adj_boundary: each boundary node's dL/dv from the
// triangles' air forces (partials at the node's partial positions), added
// last to v_bar (so to v_hat = v_bar + dt x_bar) as node_adjoint does for
// interior nodes.
__global__ void __launch_bounds__(kBndThreads)
    k_adj_boundary_air(const NodeBlock* __restrict__ blocks, int n_blocks, const MeshRT* __restrict__ rts) {
    pdl_enter();
    for (int bi = blockIdx.x; bi < n_blocks; bi += gridDim.x) {
        const NodeBlock nb = blocks[bi];
        const MeshRT& m = rts[nb.mesh];
        if (!(m.active & ACT_ADJ) || !m.air_on) continue;
        for (int i = threadIdx.x; i < nb.count; i += kBndThreads) {
            const int b = nb.begin + i, g = m.n_int + b;
            float3 c = make_float3(0.f, 0.f, 0.f);
            for (int k = m.bnd_rowptr[b], k1 = m.bnd_rowptr[b + 1]; k < k1; ++k) add3(c, m.partials_v[k]);
            m.vb[g] = f4(xyz(m.vb[g]) + c, 0.0f);
        }
    }
    pdl_done();
}

// ===========================================================================
// buffers, seeds, loss
// ===========================================================================
__global__ void k_copy_state(const NodeBlock* __restrict__ blocks, const MeshRT* __restrict__ rts) {
    const NodeBlock nb = blocks[blockIdx.x];
    const MeshRT& m = rts[nb.mesh];
    if (!(m.active & (ACT_FWD | ACT_ADJ))) return;
    for (int i = threadIdx.x; i < nb.count; i += blockDim.x) {
        const int g = nb.begin + i;
        bufx(m, m.cp_dst)[g] = bufx(m, m.cp_src)[g];
        bufv(m, m.cp_dst)[g] = bufv(m, m.cp_src)[g];
    }
}

// seeds dL/dx(S) = 2 (x - x*) + seed_x, dL/dv(S) = seed_v (buffer 0 holds x(S)),
// and per-block FP64 partial sums of |x - x*|^2 (fixed-order tree)
__global__ void k_seed_loss(const NodeBlock* __restrict__ blocks, const MeshRT* __restrict__ rts,
                            double* __restrict__ block_partials, int write_seeds) {
    __shared__ double red[256];
    const NodeBlock nb = blocks[blockIdx.x];
    const MeshRT& m = rts[nb.mesh];
    double acc = 0.0;
    for (int i = threadIdx.x; i < nb.count; i += blockDim.x) {
        const int g = nb.begin + i;
        const int u = m.node_perm[g];
        const float4 q = m.st_x[g];
        float3 xb = make_float3(0.f, 0.f, 0.f), vb = make_float3(0.f, 0.f, 0.f);
        if (m.target) {
            // x = X + u in FP64 against the target
            const double dx = m.Xd[3 * g] + (double)q.x - (double)m.target[3 * u];
            const double dy = m.Xd[3 * g + 1] + (double)q.y - (double)m.target[3 * u + 1];
            const double dz = m.Xd[3 * g + 2] + (double)q.z - (double)m.target[3 * u + 2];
            acc += dx * dx + dy * dy + dz * dz;
            xb = make_float3((float)(2.0 * dx), (float)(2.0 * dy), (float)(2.0 * dz));
        }
        if (m.seed_x) xb += make_float3(m.seed_x[3 * u], m.seed_x[3 * u + 1], m.seed_x[3 * u + 2]);
        if (m.seed_v) vb = make_float3(m.seed_v[3 * u], m.seed_v[3 * u + 1], m.seed_v[3 * u + 2]);
        if (write_seeds) {
            m.xb[g] = f4(xb, 0.f);
            m.vb[g] = f4(vhat_of(m, xb, vb), 0.f);  // the adjoint state holds v_hat
        }
    }
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) block_partials[blockIdx.x] = red[0];
}

__global__ void k_loss_finalize(const double* __restrict__ parts, int begin, int count, double* out) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        double s = 0.0;
        for (int i = 0; i < count; ++i) s += parts[begin + i];
        *out = s;
    }
}

__global__ void k_zero_adjoint(const NodeBlock* __restrict__ blocks, const MeshRT* __restrict__ rts) {
    const NodeBlock nb = blocks[blockIdx.x];
    const MeshRT& m = rts[nb.mesh];
    for (int i = threadIdx.x; i < nb.count; i += blockDim.x) m.wbar[nb.begin + i] = 0.0;
}

__global__ void k_zero_f64(double* p, long long n) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        p[i] = 0.0;
}

// ===========================================================================
// set-up (a1): Dm^-1, rest volume / area in FP64 from the rest positions,
// lumped masses m_i = sum rho_e V_e / 4 (tets) or rho_t A_t / 3 (tris)
// ===========================================================================
struct SetupArgs {
    const double* X;      // rest positions, internal node order [3N]
    const float* rho;     // per element, internal order
    double* mass;         // [N]
    double* mass_part;    // per (patch, boundary local node)
    int* bad;             // set to 1 on an inverted / degenerate element
    int geometry;         // 1: also write Dm^-1 and V into the element data
};

__global__ void k_setup_patch(const PatchDesc* __restrict__ patches, const MeshRT* __restrict__ rts, SetupArgs a) {
    extern __shared__ double dsm[];
    const PatchDesc p = patches[blockIdx.x];
    const MeshRT& m = rts[p.mesh];
    const int n_loc = p.n_int + p.n_bnd;
    const int n_rec = p.n_e + p.n_h;
    double* xs = dsm;               // 3 per local node
    double* mc = dsm + 3 * n_loc;   // one per corner, indexed as the CSR slots, + the padding slot
    for (int l = threadIdx.x; l < n_loc; l += blockDim.x) {
        const int g = local_gid(p, m, l);
        xs[3 * l] = a.X[3 * g];
        xs[3 * l + 1] = a.X[3 * g + 1];
        xs[3 * l + 2] = a.X[3 * g + 2];
    }
    __syncthreads();
    const int nc = m.kind == GS_TET ? 4 : 3;
    for (int le = threadIdx.x; le < p.n_e; le += blockDim.x) {
        const int e = p.e_begin + le;
        float4* const R = m.rec + 4 * (size_t)p.e_begin;  // the patch's planes of p.n_e records
        const uint2 id = rec_ids(R[3 * p.n_e + le]);
        const int li[4] = {(int)(id.x & 0xffff), (int)(id.x >> 16), (int)(id.y & 0xffff), (int)(id.y >> 16)};
        double share;
        if (m.kind == GS_TET) {
            double D[3][3];
            for (int c = 0; c < 3; ++c)
                for (int r = 0; r < 3; ++r) D[r][c] = xs[3 * li[c + 1] + r] - xs[3 * li[0] + r];
            const double c00 = D[1][1] * D[2][2] - D[1][2] * D[2][1];
            const double c01 = D[1][2] * D[2][0] - D[1][0] * D[2][2];
            const double c02 = D[1][0] * D[2][1] - D[1][1] * D[2][0];
            const double det = D[0][0] * c00 + D[0][1] * c01 + D[0][2] * c02;
            if (!(det > 0.0)) atomicOr(a.bad, 1);
            const double id_ = 1.0 / det;
            // inverse = adjugate / det (adjugate = transposed cofactor matrix)
            const double i00 = c00 * id_, i10 = c01 * id_, i20 = c02 * id_;
            const double i01 = (D[0][2] * D[2][1] - D[0][1] * D[2][2]) * id_;
            const double i11 = (D[0][0] * D[2][2] - D[0][2] * D[2][0]) * id_;
            const double i21 = (D[0][1] * D[2][0] - D[0][0] * D[2][1]) * id_;
            const double i02 = (D[0][1] * D[1][2] - D[0][2] * D[1][1]) * id_;
            const double i12 = (D[0][2] * D[1][0] - D[0][0] * D[1][2]) * id_;
            const double i22 = (D[0][0] * D[1][1] - D[0][1] * D[1][0]) * id_;
            const double V = det / 6.0;
            if (a.geometry) {
                const int n = p.n_e;
                R[le] = make_float4((float)i00, (float)i01, (float)i02, (float)i10);
                R[n + le] = make_float4((float)i11, (float)i12, (float)i20, (float)i21);
                float4 c = R[2 * n + le];
                c.x = (float)i22;
                c.y = (float)V;
                R[2 * n + le] = c;
            }
            share = (double)a.rho[e] * V / 4.0;
        } else {
            double e1[3], e2[3], n[3];
            for (int r = 0; r < 3; ++r) {
                e1[r] = xs[3 * li[1] + r] - xs[3 * li[0] + r];
                e2[r] = xs[3 * li[2] + r] - xs[3 * li[0] + r];
            }
            n[0] = e1[1] * e2[2] - e1[2] * e2[1];
            n[1] = e1[2] * e2[0] - e1[0] * e2[2];
            n[2] = e1[0] * e2[1] - e1[1] * e2[0];
            const double ln = sqrt(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]);
            const double l1 = sqrt(e1[0] * e1[0] + e1[1] * e1[1] + e1[2] * e1[2]);
            if (!(ln > 0.0) || !(l1 > 0.0)) atomicOr(a.bad, 1);
            double t1[3], t2[3];
            for (int r = 0; r < 3; ++r) { t1[r] = e1[r] / l1; n[r] /= ln; }
            t2[0] = n[1] * t1[2] - n[2] * t1[1];
            t2[1] = n[2] * t1[0] - n[0] * t1[2];
            t2[2] = n[0] * t1[1] - n[1] * t1[0];
            const double A11 = e1[0] * t1[0] + e1[1] * t1[1] + e1[2] * t1[2];
            const double A12 = e2[0] * t1[0] + e2[1] * t1[1] + e2[2] * t1[2];
            const double A21 = e1[0] * t2[0] + e1[1] * t2[1] + e1[2] * t2[2];
            const double A22 = e2[0] * t2[0] + e2[1] * t2[1] + e2[2] * t2[2];
            const double det = A11 * A22 - A12 * A21;
            const double area = 0.5 * ln;
            if (a.geometry) {
                const double d00 = A22 / det, d01 = -A12 / det, d10 = -A21 / det, d11 = A11 / det;
                const int n = p.n_e;
                R[le] = make_float4((float)d00, (float)d01, (float)d10, (float)d11);
                float4 b = R[n + le];
                b.x = (float)area;
                R[n + le] = b;
                // rest frame R0 = Ds_rest Dm^-1 (orthonormal columns)
                double r0[3], r1[3];
                for (int r = 0; r < 3; ++r) {
                    r0[r] = e1[r] * d00 + e2[r] * d10;
                    r1[r] = e1[r] * d01 + e2[r] * d11;
                }
                R[2 * n + le] = make_float4((float)r0[0], (float)r0[1], (float)r0[2], (float)r1[0]);
                float4 w = R[3 * n + le];
                w.z = (float)r1[1];
                w.w = (float)r1[2];
                R[3 * n + le] = w;
            }
            share = (double)a.rho[e] * area / 3.0;
        }
        for (int c = 0; c < 4; ++c) mc[c * p.n_e + le] = c < nc ? share : 0.0;
    }
    // hinge corners carry no mass (staged after the element planes); hinge
    // rest vectors X1-X3, X2-X3, X4-X3
    for (int lh = threadIdx.x; lh < 4 * p.n_h; lh += blockDim.x) mc[4 * p.n_e + (lh & 3) * p.n_h + (lh >> 2)] = 0.0;
    if (threadIdx.x == 0) mc[4 * n_rec] = 0.0;
    if (a.geometry) {
        for (int lh = threadIdx.x; lh < p.n_h; lh += blockDim.x) {
            const int h = p.h_begin + lh;
            const size_t B = m.n_hinges;
            const uint2 id = rec_ids(m.hrec[3 * B + h]);
            const int l1 = id.x & 0xffff, l2 = id.x >> 16, l3 = id.y & 0xffff, l4 = id.y >> 16;
            float4 q0 = m.hrec[h], q1 = m.hrec[B + h], q2 = m.hrec[2 * B + h];
            q0.x = (float)(xs[3 * l1] - xs[3 * l3]);
            q0.y = (float)(xs[3 * l1 + 1] - xs[3 * l3 + 1]);
            q0.z = (float)(xs[3 * l1 + 2] - xs[3 * l3 + 2]);
            q1.x = (float)(xs[3 * l2] - xs[3 * l3]);
            q1.y = (float)(xs[3 * l2 + 1] - xs[3 * l3 + 1]);
            q1.z = (float)(xs[3 * l2 + 2] - xs[3 * l3 + 2]);
            q2.x = (float)(xs[3 * l4] - xs[3 * l3]);
            q2.y = (float)(xs[3 * l4 + 1] - xs[3 * l3 + 1]);
            q2.z = (float)(xs[3 * l4 + 2] - xs[3 * l3 + 2]);
            m.hrec[h] = q0;
            m.hrec[B + h] = q1;
            m.hrec[2 * B + h] = q2;
        }
    }
    __syncthreads();
    const uint16_t* rp = m.loc_rowptr + p.lr_begin;
    const uint16_t* sl = m.loc_slots + p.slot_begin;
    for (int l = threadIdx.x; l < n_loc; l += blockDim.x) {
        double s = 0.0;
        const int k1 = rp[l + 1];
        for (int k = rp[l]; k < k1; ++k) s += mc[sl[k]];
        if (l < p.n_int) a.mass[p.int_begin + l] = s;
        else a.mass_part[m.part_pos[p.bnd_begin + (l - p.n_int)]] = s;
    }
}

__global__ void k_mass_boundary(const NodeBlock* __restrict__ blocks, const MeshRT* __restrict__ rts, SetupArgs a) {
    const NodeBlock nb = blocks[blockIdx.x];
    const MeshRT& m = rts[nb.mesh];
    for (int i = threadIdx.x; i < nb.count; i += blockDim.x) {
        const int b = nb.begin + i;
        double s = 0.0;
        for (int k = m.bnd_rowptr[b]; k < m.bnd_rowptr[b + 1]; ++k) s += a.mass_part[k];
        a.mass[m.n_int + b] = s;
    }
}

// inverse mass: w = 1/m, 0 for pinned nodes and nodes without mass; copy to
// the .w lane of the current state
__global__ void k_mass_finalize(const MeshRT* __restrict__ rts, const double* __restrict__ mass,
                                const uint8_t* __restrict__ pinned_internal) {
    const MeshRT& m = rts[0];
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < m.n_nodes; i += gridDim.x * blockDim.x) {
        const bool pin = pinned_internal && pinned_internal[i];
        const float w = (!pin && mass[i] > 0.0) ? (float)(1.0 / mass[i]) : 0.0f;
        m.w[i] = w;
        float4 x = m.st_x[i];
        x.w = w;
        m.st_x[i] = x;
    }
}

// ===========================================================================
// caller <-> internal order
// ===========================================================================
__global__ void k_scatter_params(const MeshRT* __restrict__ rts, const float* mu, const float* lam, const float* act,
                                 const float* kb) {
    const MeshRT& m = rts[0];
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < m.n_elems; e += gridDim.x * blockDim.x) {
        const int u = m.elem_perm[e];
        const int E = m.n_elems;
        if (m.kind == GS_TET) {
            float4 c = m.rec[rec_at(E, m.pe, 2, e)];
            if (mu) c.z = mu[u];
            if (lam) c.w = lam[u];
            m.rec[rec_at(E, m.pe, 2, e)] = c;
            if (act) m.rec[rec_at(E, m.pe, 3, e)].z = act[u];
        } else {
            float4 b = m.rec[rec_at(E, m.pe, 1, e)];
            if (mu) b.y = mu[u];
            if (lam) b.z = lam[u];
            if (act) b.w = act[u];
            m.rec[rec_at(E, m.pe, 1, e)] = b;
        }
    }
    if (kb && m.kind == GS_CLOTH) {
        for (int h = blockIdx.x * blockDim.x + threadIdx.x; h < m.n_hinges; h += gridDim.x * blockDim.x)
            m.hrec[h].w = kb[m.hinge_perm[h]];
    }
}

__global__ void k_gather_elems(const MeshRT* __restrict__ rts, const float* src, float* dst) {
    const MeshRT& m = rts[0];
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < m.n_elems; e += gridDim.x * blockDim.x)
        dst[e] = src[m.elem_perm[e]];
}

__global__ void k_set_state(const MeshRT* __restrict__ rts, int buf, const float* x, const float* v) {
    const MeshRT& m = rts[0];
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < m.n_nodes; i += gridDim.x * blockDim.x) {
        const int u = m.node_perm[i];
        if (x)
            bufx(m, buf)[i] = make_float4((float)((double)x[3 * u] - m.Xd[3 * i]),
                                          (float)((double)x[3 * u + 1] - m.Xd[3 * i + 1]),
                                          (float)((double)x[3 * u + 2] - m.Xd[3 * i + 2]), m.w[i]);
        if (v) bufv(m, buf)[i] = make_float4(v[3 * u], v[3 * u + 1], v[3 * u + 2], m.Xp[i]);
    }
}

// rest state: u = 0 (x = X), inverse mass in .w, v = v0 (caller order)
__global__ void k_reset_state(const MeshRT* __restrict__ rts, const float* v0) {
    const MeshRT& m = rts[0];
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < m.n_nodes; i += gridDim.x * blockDim.x) {
        const int u = m.node_perm[i];
        m.st_x[i] = make_float4(0.f, 0.f, 0.f, m.w[i]);
        m.st_v[i] = make_float4(v0[3 * u], v0[3 * u + 1], v0[3 * u + 2], m.Xp[i]);
    }
}

__global__ void k_get_state(const MeshRT* __restrict__ rts, int buf, float* x, float* v) {
    const MeshRT& m = rts[0];
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < m.n_nodes; i += gridDim.x * blockDim.x) {
        const int u = m.node_perm[i];
        if (x) {
            const float4 q = bufx(m, buf)[i];
            x[3 * u] = (float)(m.Xd[3 * i] + (double)q.x);
            x[3 * u + 1] = (float)(m.Xd[3 * i + 1] + (double)q.y);
            x[3 * u + 2] = (float)(m.Xd[3 * i + 2] + (double)q.z);
        }
        if (v) {
            const float4 q = bufv(m, buf)[i];
            v[3 * u] = q.x; v[3 * u + 1] = q.y; v[3 * u + 2] = q.z;
        }
    }
}

// a11: dL/dm_i = -w_i^2 dL/dw_i; node outputs in caller order
__global__ void k_node_grads(const MeshRT* __restrict__ rts, double* mbar, float* d_x0, float* d_v0, double* d_mass) {
    const MeshRT& m = rts[0];
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < m.n_nodes; i += gridDim.x * blockDim.x) {
        const float w = m.w[i];
        const double mb = -(double)w * (double)w * m.wbar[i];
        mbar[i] = mb;
        const int u = m.node_perm[i];
        if (d_mass) d_mass[u] = mb;
        if (d_x0) {
            const float4 q = m.xb[i];
            d_x0[3 * u] = q.x; d_x0[3 * u + 1] = q.y; d_x0[3 * u + 2] = q.z;
        }
        if (d_v0) {
            // dL/dv(0) = v_hat - dt x_bar
            const float3 q = xyz(m.vb[i]) - m.dt * xyz(m.xb[i]);
            d_v0[3 * u] = q.x; d_v0[3 * u + 1] = q.y; d_v0[3 * u + 2] = q.z;
        }
    }
}

// dL/drho_e = (V_e / 4) sum_{i in e} dL/dm_i  (A_t / 3 for triangles), plus
// the per-element accumulators in caller order
__global__ void k_elem_grads(const PatchDesc* __restrict__ patches, const MeshRT* __restrict__ rts,
                             const double* __restrict__ mbar, double* d_mu, double* d_lam, double* d_rho,
                             double* d_act, double* d_kb, double* d_hact) {
    extern __shared__ double msm[];
    const PatchDesc p = patches[blockIdx.x];
    const MeshRT& m = rts[p.mesh];
    const int n_loc = p.n_int + p.n_bnd;
    for (int l = threadIdx.x; l < n_loc; l += blockDim.x) msm[l] = mbar[local_gid(p, m, l)];
    __syncthreads();
    for (int le = threadIdx.x; le < p.n_e; le += blockDim.x) {
        const int e = p.e_begin + le;
        const int u = m.elem_perm[e];
        const float4* R = m.rec + 4 * (size_t)p.e_begin;  // the patch's planes of p.n_e records
        const uint2 id = rec_ids(R[3 * p.n_e + le]);
        if (d_rho) {
            if (m.kind == GS_TET) {
                const double s = msm[id.x & 0xffff] + msm[id.x >> 16] + msm[id.y & 0xffff] + msm[id.y >> 16];
                d_rho[u] = s * ((double)R[2 * p.n_e + le].y / 4.0);
            } else {
                const double s = msm[id.x & 0xffff] + msm[id.x >> 16] + msm[id.y & 0xffff];
                d_rho[u] = s * ((double)R[p.n_e + le].x / 3.0);
            }
        }
        if (d_mu) d_mu[u] = m.g_ml[e].x;
        if (d_lam) d_lam[u] = m.g_ml[e].y;
        if (d_act && m.g_act) d_act[u] = m.g_act[e];
    }
    for (int lh = threadIdx.x; lh < p.n_h; lh += blockDim.x) {
        const int h = p.h_begin + lh;
        const int u = m.hinge_perm[h];
        if (d_kb) d_kb[u] = m.g_kb[h];
        if (d_hact && m.g_hact) d_hact[u] = m.g_hact[h];
    }
}

// ===========================================================================
// launchers
// ===========================================================================
size_t patch_smem_bytes(int kind, int n_e, int n_h, int n_loc, int n_int, int n_slots, bool adjoint, bool extras) {
    return (size_t)((kHdr + patch_layout(kind, n_e, n_h, n_loc, n_int, n_slots, adjoint, extras).total + 127) & ~127);
}

// persistent grid: resident CTAs per SM x SMs, at most one CTA per patch
int patch_grid(int which, int threads, int stage_bytes, int n_patches, int num_sms) {
    if (n_patches <= 0) return 0;
    const void* f = which == 0 ? (const void*)k_tet_fwd
                  : which == 1 ? (const void*)k_cloth_fwd
                  : which == 2 ? (const void*)k_tet_adj
                               : (const void*)k_cloth_adj;
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, f, threads + 32, patch_dyn_smem(stage_bytes)) !=
        cudaSuccess) {
        cudaGetLastError();
        nb = 1;
    }
    nb = nb < 1 ? 1 : nb;
    const long long g = (long long)nb * num_sms;
    return (int)(g < n_patches ? g : n_patches);
}

// boundary kernels: one wave of CTAs striding over the 256-node blocks
int boundary_grid(int adjoint, int n_blocks, int num_sms) {
    if (n_blocks <= 0) return 0;
    int nb = 0;
    const void* f = adjoint ? (const void*)k_adj_boundary : (const void*)k_fwd_boundary;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, f, kBndThreads, 0) != cudaSuccess) {
        cudaGetLastError();
        nb = 1;
    }
    nb = nb < 1 ? 1 : nb;
    const long long g = (long long)nb * num_sms;
    return (int)(g < n_blocks ? g : n_blocks);
}

void set_kernel_smem_limits(size_t bytes) {
    cudaFuncSetAttribute(k_tet_fwd, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    cudaFuncSetAttribute(k_cloth_fwd, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    cudaFuncSetAttribute(k_tet_adj, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    cudaFuncSetAttribute(k_cloth_adj, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    cudaFuncSetAttribute(k_setup_patch, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    cudaFuncSetAttribute(k_elem_grads, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

const char* kernel_name(int kind) {
    static const char* names[KT_COUNT] = {"tet_fwd_patch", "cloth_fwd_patch", "fwd_boundary",
                                          "tet_adj_patch", "cloth_adj_patch", "adj_boundary"};
    return (kind >= 0 && kind < KT_COUNT) ? names[kind] : "?";
}

#define GS_TIMED(kind, launch)       \
    do {                              \
        if (prof) prof->begin(kind, s); \
        launch;                       \
        if (prof) prof->end(kind, s);   \
    } while (0)

// step kernels are launched with programmatic stream serialisation (see pdl_enter)
template <typename... KArgs, typename... Args>
static void launch_pdl(void (*k)(KArgs...), int grid, int block, size_t smem, cudaStream_t s, Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3((unsigned)block);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    cudaLaunchKernelEx(&cfg, k, args...);
}

void launch_forward_step(const Launch& L, int tick, cudaStream_t s, Prof* prof) {
    if (L.n_tet_patches)
        GS_TIMED(KT_TET_FWD, launch_pdl(k_tet_fwd, L.grid[0], L.threads + 32, patch_dyn_smem(L.stage[0]), s,
                                        L.tet_patches, L.n_tet_patches, (const MeshRT*)L.rt, tick, L.stage[0], L.extras));
    if (L.n_cloth_patches)
        GS_TIMED(KT_CLOTH_FWD, launch_pdl(k_cloth_fwd, L.grid[1], L.threads + 32, patch_dyn_smem(L.stage[1]),
                                          s, L.cloth_patches, L.n_cloth_patches, (const MeshRT*)L.rt, tick,
                                          L.stage[1], L.extras));
    if (L.n_bnd_blocks)
        GS_TIMED(KT_FWD_BND, launch_pdl(k_fwd_boundary, L.bgrid[0], kBndThreads, 0, s, L.bnd_blocks,
                                        L.n_bnd_blocks, (const MeshRT*)L.rt, tick));
}

void launch_adjoint_step(const Launch& L, int tick, cudaStream_t s, Prof* prof) {
    if (L.n_tet_patches)
        GS_TIMED(KT_TET_ADJ, launch_pdl(k_tet_adj, L.grid[2], L.threads_adj + 32, patch_dyn_smem(L.stage[2]), s,
                                        L.tet_patches, L.n_tet_patches, (const MeshRT*)L.rt, tick, L.stage[2], L.extras));
    if (L.n_cloth_patches)
        GS_TIMED(KT_CLOTH_ADJ, launch_pdl(k_cloth_adj, L.grid[3], L.threads_adj + 32, patch_dyn_smem(L.stage[3]),
                                          s, L.cloth_patches, L.n_cloth_patches, (const MeshRT*)L.rt, tick,
                                          L.stage[3], L.extras));
    if (L.n_bnd_blocks)
        GS_TIMED(KT_ADJ_BND, launch_pdl(k_adj_boundary, L.bgrid[1], kBndThreads, 0, s, L.bnd_blocks,
                                        L.n_bnd_blocks, (const MeshRT*)L.rt, tick));
    if (L.air && L.n_bnd_blocks)
        GS_TIMED(KT_ADJ_BND, launch_pdl(k_adj_boundary_air, L.bgrid[1], kBndThreads, 0, s, L.bnd_blocks,
                                        L.n_bnd_blocks, (const MeshRT*)L.rt));
}

void launch_copy_state(const Launch& L, cudaStream_t s) {
    if (L.n_node_blocks) k_copy_state<<<L.n_node_blocks, 256, 0, s>>>(L.node_blocks, L.rt);
}

void launch_seed_loss(const Launch& L, double* block_partials, int write_seeds, cudaStream_t s) {
    if (L.n_node_blocks) k_seed_loss<<<L.n_node_blocks, 256, 0, s>>>(L.node_blocks, L.rt, block_partials, write_seeds);
}

void launch_loss_finalize(const double* block_partials, int begin, int count, double* out, cudaStream_t s) {
    k_loss_finalize<<<1, 32, 0, s>>>(block_partials, begin, count, out);
}

void launch_zero_adjoint(const Launch& L, cudaStream_t s) {
    if (L.n_node_blocks) k_zero_adjoint<<<L.n_node_blocks, 256, 0, s>>>(L.node_blocks, L.rt);
}

gs_status selftest_bounded_wait(int iterations, int* status_host, cudaStream_t s) {
    int* d = nullptr;
    GS_CUDA(cudaMallocAsync((void**)&d, sizeof(int), s));
    cudaError_t e = cudaMemsetAsync(d, 0, sizeof(int), s);
    if (e == cudaSuccess) {
        k_selftest_wait<<<1, 32, 0, s>>>(iterations, d);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(status_host, d, sizeof(int), cudaMemcpyDeviceToHost, s);
    cudaFreeAsync(d, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_error(e, "gs_selftest_bounded_wait");
    return GS_OK;
}

// rows of `count` entries between caller order (row stride count) and
// internal order (row stride ld >= count; the padding is written as 0)
__global__ void k_permute_rows(const float* __restrict__ src, float* __restrict__ dst, int rows, int count, int ld,
                               const int* __restrict__ perm, int to_internal) {
    const long long total = (long long)rows * ld;
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < total; k += (long long)gridDim.x * blockDim.x) {
        const long long r = k / ld;
        const int i = (int)(k - r * ld);
        if (to_internal) dst[k] = i < count ? src[r * count + perm[i]] : 0.f;
        else if (i < count) dst[r * count + perm[i]] = src[k];
    }
}

void launch_permute_rows(const float* src, float* dst, int rows, int count, int ld, const int* perm, int to_internal,
                         cudaStream_t s) {
    const long long total = (long long)rows * ld;
    if (total <= 0) return;
    const long long blocks = (total + 255) / 256;
    k_permute_rows<<<(int)(blocks < 8192 ? blocks : 8192), 256, 0, s>>>(src, dst, rows, count, ld, perm, to_internal);
}

void launch_zero_f64(double* p, long long n, cudaStream_t s) {
    if (n > 0 && p) k_zero_f64<<<(int)((n + 255) / 256 < 4096 ? (n + 255) / 256 : 4096), 256, 0, s>>>(p, n);
}

void launch_setup_mesh(const Launch& L, const double* X, const float* rho, double* mass, double* mass_part,
                       const uint8_t* pinned_internal, int* bad, int geometry, size_t smem, cudaStream_t s) {
    SetupArgs a{X, rho, mass, mass_part, bad, geometry};
    const PatchDesc* pd = L.n_tet_patches ? L.tet_patches : L.cloth_patches;
    const int np = L.n_tet_patches ? L.n_tet_patches : L.n_cloth_patches;
    k_setup_patch<<<np, L.threads, smem, s>>>(pd, L.rt, a);
    if (L.n_bnd_blocks) k_mass_boundary<<<L.n_bnd_blocks, 256, 0, s>>>(L.bnd_blocks, L.rt, a);
    k_mass_finalize<<<256, 256, 0, s>>>(L.rt, mass, pinned_internal);
}

void launch_scatter_params(const MeshRT* rt_dev, const float* mu, const float* lam, const float* act,
                           const float* kb, cudaStream_t s) {
    k_scatter_params<<<512, 256, 0, s>>>(rt_dev, mu, lam, act, kb);
}

void launch_gather_elems(const MeshRT* rt_dev, const float* src, float* dst, cudaStream_t s) {
    k_gather_elems<<<512, 256, 0, s>>>(rt_dev, src, dst);
}

void launch_set_state(const MeshRT* rt_dev, int buf, const float* x, const float* v, cudaStream_t s) {
    k_set_state<<<512, 256, 0, s>>>(rt_dev, buf, x, v);
}

void launch_reset_state(const MeshRT* rt_dev, const float* v0, cudaStream_t s) {
    k_reset_state<<<512, 256, 0, s>>>(rt_dev, v0);
}

void launch_get_state(const MeshRT* rt_dev, int buf, float* x, float* v, cudaStream_t s) {
    k_get_state<<<512, 256, 0, s>>>(rt_dev, buf, x, v);
}

void launch_finalize_grads(const Launch& L, double* mbar, const gs_grads& g, size_t smem, cudaStream_t s) {
    k_node_grads<<<512, 256, 0, s>>>(L.rt, mbar, g.d_x0, g.d_v0, g.d_mass);
    const PatchDesc* pd = L.n_tet_patches ? L.tet_patches : L.cloth_patches;
    const int np = L.n_tet_patches ? L.n_tet_patches : L.n_cloth_patches;
    if (g.d_mu || g.d_lambda || g.d_density || g.d_act || g.d_kb || g.d_hinge_act)
        k_elem_grads<<<np, L.threads, smem, s>>>(pd, L.rt, mbar, g.d_mu, g.d_lambda, g.d_density, g.d_act, g.d_kb,
                                                 g.d_hinge_act);
}

}  // namespace gs

extern "C" GS_API int gs_build_flags(void) { return gs::kChecked ? GS_BUILD_CHECKED : 0; }
