// Kernels of the explicit step (forward) and of its discrete adjoint.
//
// One CTA per element patch.  Shared memory holds, for the patch's local
// nodes, the gathered node data (positions with inverse mass in .w; in the
// adjoint also the total adjoint velocity v_hat), and one float4 per element
// corner.  The element phase writes corner results; the node phase sums the
// corners of every local node through the patch's CSR in a fixed order,
// finishes interior nodes (contact + semi-implicit Euler, or the reverse of
// both) and writes one partial per boundary node, which the boundary kernel
// sums in patch order.  Nothing uses floating-point atomics.
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

// Contact geometry from the displacement u of node g.  The penetrations are
// formed from FP64-derived rest offsets so that FP32 keeps their relative
// precision near contact: plane C = (h - n.X) - n.u; sphere
// C = r - |d| = -(|X - c|^2 - r^2 + 2 (X - c).u + u.u) / (|d| + r), d = X - c + u.

// total contact force on a node: plane and sphere
__device__ __forceinline__ float3 contact_force(const MeshRT& m, int g, float3 u, float3 v) {
    float3 f = make_float3(0.f, 0.f, 0.f);
    const ContactParams cp = cparams(m);
    if (m.plane_on) {
        const float3 n = make_float3(m.pnx, m.pny, m.pnz);
        const float C = m.Xp[g] - dot3(n, u);
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
__device__ __forceinline__ float3 contact_adjoint(const MeshRT& m, int g, float3 u, float3 v, float3 fb, float3& xb,
                                                  float3& vb) {
    float3 f = make_float3(0.f, 0.f, 0.f);
    const ContactParams cp = cparams(m);
    if (m.plane_on) {
        const float3 n = make_float3(m.pnx, m.pny, m.pnz);
        const float C = m.Xp[g] - dot3(n, u);
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
    const float3 f = fel + contact_force(m, gid, x, v);
    if (w > 0.0f) {
        v.x = v.x + m.dt * (w * f.x + m.gx);
        v.y = v.y + m.dt * (w * f.y + m.gy);
        v.z = v.z + m.dt * (w * f.z + m.gz);
    }
    const float3 xn = x + m.dt * v;
    const int ob = m.out_a + m.out_b * tick;
    const float4 xo = f4(xn, w), vo = f4(v, 0.0f);
    bufx(m, ob)[gid] = xo;
    bufv(m, ob)[gid] = vo;
    if (tick == m.ck_tick) {
        bufx(m, m.ck_buf)[gid] = xo;
        bufv(m, m.ck_buf)[gid] = vo;
    }
    if (!(isfinite(xn.x) && isfinite(xn.y) && isfinite(xn.z) && isfinite(v.x) && isfinite(v.y) && isfinite(v.z)))
        atomicOr(m.status, 1);
}

// reverse of node_forward for one node.  Inputs: state (x, v) at step n,
// adjoint (xb, vb) of step n+1, the gathered element terms xsum = sum of
// corner dL/dx and ssum = sum of corner f . v_hat.  Outputs the adjoint of
// step n in place and accumulates dL/dw (FP64).
__device__ __forceinline__ void node_adjoint(const MeshRT& m, int gid, float4 x4, float4 v4, float3 xsum, float ssum) {
    const float w = x4.w;
    const float4 xb4 = m.xb[gid], vb4 = m.vb[gid];
    const float3 xbn = xyz(xb4);
    const float3 vh = xyz(vb4) + m.dt * xbn;    // dL/dv+ (total)
    const float3 fb = (m.dt * w) * vh;          // dL/df
    float3 xb = xbn + xsum;
    float3 vb = vh;
    const float3 fc = contact_adjoint(m, gid, xyz(x4), xyz(v4), fb, xb, vb);
    m.xb[gid] = f4(xb, 0.0f);
    m.vb[gid] = f4(vb, 0.0f);
    m.wbar[gid] += (double)(m.dt * (ssum + dot3(fc, vh)));
}

}  // namespace

// ===========================================================================
// forward
// ===========================================================================
// dynamic shared memory: xs[max_loc] (float4) then fc[max_slots] (float4)
__global__ void k_tet_fwd(const PatchDesc* __restrict__ patches, const MeshRT* __restrict__ rts, int tick) {
    extern __shared__ float4 smem[];
    const PatchDesc p = patches[blockIdx.x];
    const MeshRT& m = rts[p.mesh];
    if (!(m.active & ACT_FWD)) return;
    const int n_loc = p.n_int + p.n_bnd;
    float4* xs = smem;
    float4* fc = smem + n_loc;
    const int ib = m.in_a + m.in_b * tick;
    const float4* __restrict__ X = bufx(m, ib);
    for (int l = threadIdx.x; l < n_loc; l += blockDim.x) xs[l] = X[local_gid(p, m, l)];
    __syncthreads();
    for (int le = threadIdx.x; le < p.n_e; le += blockDim.x) {
        const int e = p.e_begin + le;
        const uint2 id = m.eidx[e];
        const float4 a = m.ea[e], b = m.eb[e], c = m.ec[e];
        const float act = m.eact ? m.eact[e] : 0.0f;
        TetState s;
        tet_state(xyz(xs[id.x & 0xffff]), xyz(xs[id.x >> 16]), xyz(xs[id.y & 0xffff]), xyz(xs[id.y >> 16]), a, b,
                  c, act, s);
        float3 f0, f1, f2, f3;
        tet_forces(s, a, b, c, f0, f1, f2, f3);
        fc[4 * le + 0] = f4(f0, 0.f);
        fc[4 * le + 1] = f4(f1, 0.f);
        fc[4 * le + 2] = f4(f2, 0.f);
        fc[4 * le + 3] = f4(f3, 0.f);
    }
    __syncthreads();
    const uint16_t* rp = m.loc_rowptr + p.lr_begin;
    const uint16_t* sl = m.loc_slots + p.slot_begin;
    const float4* __restrict__ Vin = bufv(m, ib);
    for (int l = threadIdx.x; l < n_loc; l += blockDim.x) {
        float3 f = make_float3(0.f, 0.f, 0.f);
        const int k1 = rp[l + 1];
        for (int k = rp[l]; k < k1; ++k) f += xyz(fc[sl[k]]);
        if (l < p.n_int) {
            const int gid = p.int_begin + l;
            node_forward(m, tick, gid, xs[l], Vin[gid], f);
        } else {
            m.partials[p.bnd_begin + (l - p.n_int)] = f4(f, 0.f);
        }
    }
}

// cloth: triangles (3 corner slots each) then hinges (4 each)
__global__ void k_cloth_fwd(const PatchDesc* __restrict__ patches, const MeshRT* __restrict__ rts, int tick) {
    extern __shared__ float4 smem[];
    const PatchDesc p = patches[blockIdx.x];
    const MeshRT& m = rts[p.mesh];
    if (!(m.active & ACT_FWD)) return;
    const int n_loc = p.n_int + p.n_bnd;
    float4* xs = smem;
    float4* fc = smem + n_loc;
    const int ib = m.in_a + m.in_b * tick;
    const float4* __restrict__ X = bufx(m, ib);
    for (int l = threadIdx.x; l < n_loc; l += blockDim.x) xs[l] = X[local_gid(p, m, l)];
    __syncthreads();
    for (int lt = threadIdx.x; lt < p.n_e; lt += blockDim.x) {
        const int t = p.e_begin + lt;
        const uint2 id = m.eidx[t];
        const float4 a = m.ea[t], b = m.eb[t], r = m.ec[t];
        const float2 r2 = m.ed[t];
        TriState s;
        tri_state(xyz(xs[id.x & 0xffff]), xyz(xs[id.x >> 16]), xyz(xs[id.y & 0xffff]), a, b,
                  make_float3(r.x, r.y, r.z), make_float3(r.w, r2.x, r2.y), s);
        float3 f0, f1, f2;
        tri_forces(s, a, b, f0, f1, f2);
        fc[3 * lt + 0] = f4(f0, 0.f);
        fc[3 * lt + 1] = f4(f1, 0.f);
        fc[3 * lt + 2] = f4(f2, 0.f);
    }
    float4* fh = fc + 3 * p.n_e;
    for (int lh = threadIdx.x; lh < p.n_h; lh += blockDim.x) {
        const int h = p.h_begin + lh;
        const uint2 id = m.hidx[h];
        const float4 q0 = m.hq[3 * h], q1 = m.hq[3 * h + 1], q2 = m.hq[3 * h + 2];
        HingeState s;
        hinge_state(xyz(xs[id.x & 0xffff]), xyz(xs[id.x >> 16]), xyz(xs[id.y & 0xffff]), xyz(xs[id.y >> 16]),
                    xyz(q0), xyz(q1), xyz(q2), q1.w, s);
        float3 f1, f2, f3, f4_;
        hinge_forces(s, q0.w, f1, f2, f3, f4_);
        fh[4 * lh + 0] = f4(f1, 0.f);
        fh[4 * lh + 1] = f4(f2, 0.f);
        fh[4 * lh + 2] = f4(f3, 0.f);
        fh[4 * lh + 3] = f4(f4_, 0.f);
    }
    __syncthreads();
    const uint16_t* rp = m.loc_rowptr + p.lr_begin;
    const uint16_t* sl = m.loc_slots + p.slot_begin;
    const float4* __restrict__ Vin = bufv(m, ib);
    for (int l = threadIdx.x; l < n_loc; l += blockDim.x) {
        float3 f = make_float3(0.f, 0.f, 0.f);
        const int k1 = rp[l + 1];
        for (int k = rp[l]; k < k1; ++k) f += xyz(fc[sl[k]]);
        if (l < p.n_int) {
            const int gid = p.int_begin + l;
            node_forward(m, tick, gid, xs[l], Vin[gid], f);
        } else {
            m.partials[p.bnd_begin + (l - p.n_int)] = f4(f, 0.f);
        }
    }
}

// boundary nodes: sum the per-patch partials in patch order, then finish
__global__ void k_fwd_boundary(const NodeBlock* __restrict__ blocks, const MeshRT* __restrict__ rts, int tick) {
    const NodeBlock nb = blocks[blockIdx.x];
    const MeshRT& m = rts[nb.mesh];
    if (!(m.active & ACT_FWD)) return;
    const int ib = m.in_a + m.in_b * tick;
    for (int i = threadIdx.x; i < nb.count; i += blockDim.x) {
        const int b = nb.begin + i;
        float3 f = make_float3(0.f, 0.f, 0.f);
        const int k1 = m.bnd_rowptr[b + 1];
        for (int k = m.bnd_rowptr[b]; k < k1; ++k) f += xyz(m.partials[m.bnd_parts[k]]);
        const int gid = m.n_int + b;
        node_forward(m, tick, gid, bufx(m, ib)[gid], bufv(m, ib)[gid], f);
    }
}

// ===========================================================================
// adjoint
// ===========================================================================
// dynamic shared memory: xs[max_loc], vh[max_loc], fc[max_slots] (float4)
// corner result: (dL/dx_corner, f_corner . v_hat_node)
__global__ void k_tet_adj(const PatchDesc* __restrict__ patches, const MeshRT* __restrict__ rts, int tick) {
    extern __shared__ float4 smem[];
    const PatchDesc p = patches[blockIdx.x];
    const MeshRT& m = rts[p.mesh];
    if (!(m.active & ACT_ADJ)) return;
    const int n_loc = p.n_int + p.n_bnd;
    float4* xs = smem;
    float4* vh = smem + n_loc;
    float4* fc = vh + n_loc;
    const int sb = m.adj_a + m.adj_b * tick;
    const float4* __restrict__ X = bufx(m, sb);
    const float dt = m.dt;
    for (int l = threadIdx.x; l < n_loc; l += blockDim.x) {
        const int g = local_gid(p, m, l);
        xs[l] = X[g];
        vh[l] = f4(xyz(m.vb[g]) + dt * xyz(m.xb[g]), 0.f);
    }
    __syncthreads();
    for (int le = threadIdx.x; le < p.n_e; le += blockDim.x) {
        const int e = p.e_begin + le;
        const uint2 id = m.eidx[e];
        const int i0 = id.x & 0xffff, i1 = id.x >> 16, i2 = id.y & 0xffff, i3 = id.y >> 16;
        const float4 a = m.ea[e], b = m.eb[e], c = m.ec[e];
        const float act = m.eact ? m.eact[e] : 0.0f;
        const float4 x0 = xs[i0], x1 = xs[i1], x2 = xs[i2], x3 = xs[i3];
        const float3 v0 = xyz(vh[i0]), v1 = xyz(vh[i1]), v2 = xyz(vh[i2]), v3 = xyz(vh[i3]);
        TetState s;
        tet_state(xyz(x0), xyz(x1), xyz(x2), xyz(x3), a, b, c, act, s);
        float3 f0, f1, f2, f3;
        tet_forces(s, a, b, c, f0, f1, f2, f3);
        float3 xb0, xb1, xb2, xb3;
        float gmu, glam, gact;
        tet_adjoint(s, a, b, c, (dt * x0.w) * v0, (dt * x1.w) * v1, (dt * x2.w) * v2, (dt * x3.w) * v3, xb0, xb1,
                    xb2, xb3, gmu, glam, gact);
        fc[4 * le + 0] = f4(xb0, dot3(f0, v0));
        fc[4 * le + 1] = f4(xb1, dot3(f1, v1));
        fc[4 * le + 2] = f4(xb2, dot3(f2, v2));
        fc[4 * le + 3] = f4(xb3, dot3(f3, v3));
        m.g_mu[e] += (double)gmu;
        m.g_lam[e] += (double)glam;
        if (m.g_act) m.g_act[e] += (double)gact;
    }
    __syncthreads();
    const uint16_t* rp = m.loc_rowptr + p.lr_begin;
    const uint16_t* sl = m.loc_slots + p.slot_begin;
    const float4* __restrict__ V = bufv(m, sb);
    for (int l = threadIdx.x; l < n_loc; l += blockDim.x) {
        float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
        const int k1 = rp[l + 1];
        for (int k = rp[l]; k < k1; ++k) {
            const float4 q = fc[sl[k]];
            acc.x += q.x; acc.y += q.y; acc.z += q.z; acc.w += q.w;
        }
        if (l < p.n_int) {
            const int gid = p.int_begin + l;
            node_adjoint(m, gid, xs[l], V[gid], xyz(acc), acc.w);
        } else {
            m.partials[p.bnd_begin + (l - p.n_int)] = acc;
        }
    }
}

__global__ void k_cloth_adj(const PatchDesc* __restrict__ patches, const MeshRT* __restrict__ rts, int tick) {
    extern __shared__ float4 smem[];
    const PatchDesc p = patches[blockIdx.x];
    const MeshRT& m = rts[p.mesh];
    if (!(m.active & ACT_ADJ)) return;
    const int n_loc = p.n_int + p.n_bnd;
    float4* xs = smem;
    float4* vh = smem + n_loc;
    float4* fc = vh + n_loc;
    const int sb = m.adj_a + m.adj_b * tick;
    const float4* __restrict__ X = bufx(m, sb);
    const float dt = m.dt;
    for (int l = threadIdx.x; l < n_loc; l += blockDim.x) {
        const int g = local_gid(p, m, l);
        xs[l] = X[g];
        vh[l] = f4(xyz(m.vb[g]) + dt * xyz(m.xb[g]), 0.f);
    }
    __syncthreads();
    for (int lt = threadIdx.x; lt < p.n_e; lt += blockDim.x) {
        const int t = p.e_begin + lt;
        const uint2 id = m.eidx[t];
        const int i0 = id.x & 0xffff, i1 = id.x >> 16, i2 = id.y & 0xffff;
        const float4 a = m.ea[t], b = m.eb[t], r = m.ec[t];
        const float2 r2 = m.ed[t];
        const float4 x0 = xs[i0], x1 = xs[i1], x2 = xs[i2];
        const float3 v0 = xyz(vh[i0]), v1 = xyz(vh[i1]), v2 = xyz(vh[i2]);
        TriState s;
        tri_state(xyz(x0), xyz(x1), xyz(x2), a, b, make_float3(r.x, r.y, r.z), make_float3(r.w, r2.x, r2.y), s);
        float3 f0, f1, f2;
        tri_forces(s, a, b, f0, f1, f2);
        float3 xb0, xb1, xb2;
        float gmu, glam, gact;
        tri_adjoint(s, a, b, (dt * x0.w) * v0, (dt * x1.w) * v1, (dt * x2.w) * v2, xb0, xb1, xb2, gmu, glam, gact);
        fc[3 * lt + 0] = f4(xb0, dot3(f0, v0));
        fc[3 * lt + 1] = f4(xb1, dot3(f1, v1));
        fc[3 * lt + 2] = f4(xb2, dot3(f2, v2));
        m.g_mu[t] += (double)gmu;
        m.g_lam[t] += (double)glam;
        if (m.g_act) m.g_act[t] += (double)gact;
    }
    float4* fh = fc + 3 * p.n_e;
    for (int lh = threadIdx.x; lh < p.n_h; lh += blockDim.x) {
        const int h = p.h_begin + lh;
        const uint2 id = m.hidx[h];
        const int i1 = id.x & 0xffff, i2 = id.x >> 16, i3 = id.y & 0xffff, i4 = id.y >> 16;
        const float4 q0 = m.hq[3 * h], q1 = m.hq[3 * h + 1], q2 = m.hq[3 * h + 2];
        const float4 x1 = xs[i1], x2 = xs[i2], x3 = xs[i3], x4 = xs[i4];
        const float3 v1 = xyz(vh[i1]), v2 = xyz(vh[i2]), v3 = xyz(vh[i3]), v4 = xyz(vh[i4]);
        HingeState s;
        hinge_state(xyz(x1), xyz(x2), xyz(x3), xyz(x4), xyz(q0), xyz(q1), xyz(q2), q1.w, s);
        float3 f1, f2, f3, f4_;
        hinge_forces(s, q0.w, f1, f2, f3, f4_);
        float3 xb1, xb2, xb3, xb4;
        float gkb, gact;
        hinge_adjoint(s, q0.w, (dt * x1.w) * v1, (dt * x2.w) * v2, (dt * x3.w) * v3, (dt * x4.w) * v4, xb1, xb2, xb3,
                      xb4, gkb, gact);
        fh[4 * lh + 0] = f4(xb1, dot3(f1, v1));
        fh[4 * lh + 1] = f4(xb2, dot3(f2, v2));
        fh[4 * lh + 2] = f4(xb3, dot3(f3, v3));
        fh[4 * lh + 3] = f4(xb4, dot3(f4_, v4));
        m.g_kb[h] += (double)gkb;
        if (m.g_hact) m.g_hact[h] += (double)gact;
    }
    __syncthreads();
    const uint16_t* rp = m.loc_rowptr + p.lr_begin;
    const uint16_t* sl = m.loc_slots + p.slot_begin;
    const float4* __restrict__ V = bufv(m, sb);
    for (int l = threadIdx.x; l < n_loc; l += blockDim.x) {
        float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
        const int k1 = rp[l + 1];
        for (int k = rp[l]; k < k1; ++k) {
            const float4 q = fc[sl[k]];
            acc.x += q.x; acc.y += q.y; acc.z += q.z; acc.w += q.w;
        }
        if (l < p.n_int) {
            const int gid = p.int_begin + l;
            node_adjoint(m, gid, xs[l], V[gid], xyz(acc), acc.w);
        } else {
            m.partials[p.bnd_begin + (l - p.n_int)] = acc;
        }
    }
}

__global__ void k_adj_boundary(const NodeBlock* __restrict__ blocks, const MeshRT* __restrict__ rts, int tick) {
    const NodeBlock nb = blocks[blockIdx.x];
    const MeshRT& m = rts[nb.mesh];
    if (!(m.active & ACT_ADJ)) return;
    const int sb = m.adj_a + m.adj_b * tick;
    for (int i = threadIdx.x; i < nb.count; i += blockDim.x) {
        const int b = nb.begin + i;
        float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
        const int k1 = m.bnd_rowptr[b + 1];
        for (int k = m.bnd_rowptr[b]; k < k1; ++k) {
            const float4 q = m.partials[m.bnd_parts[k]];
            acc.x += q.x; acc.y += q.y; acc.z += q.z; acc.w += q.w;
        }
        const int gid = m.n_int + b;
        node_adjoint(m, gid, bufx(m, sb)[gid], bufv(m, sb)[gid], xyz(acc), acc.w);
    }
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
            m.vb[g] = f4(vb, 0.f);
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
    double* xs = dsm;               // 3 per local node
    double* mc = dsm + 3 * n_loc;   // one per corner slot
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
        const uint2 id = m.eidx[e];
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
                m.ea[e] = make_float4((float)i00, (float)i01, (float)i02, (float)i10);
                m.eb[e] = make_float4((float)i11, (float)i12, (float)i20, (float)i21);
                float4 c = m.ec[e];
                c.x = (float)i22;
                c.y = (float)V;
                m.ec[e] = c;
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
                m.ea[e] = make_float4((float)d00, (float)d01, (float)d10, (float)d11);
                float4 b = m.eb[e];
                b.x = (float)area;
                m.eb[e] = b;
                // rest frame R0 = Ds_rest Dm^-1 (orthonormal columns)
                double r0[3], r1[3];
                for (int r = 0; r < 3; ++r) {
                    r0[r] = e1[r] * d00 + e2[r] * d10;
                    r1[r] = e1[r] * d01 + e2[r] * d11;
                }
                m.ec[e] = make_float4((float)r0[0], (float)r0[1], (float)r0[2], (float)r1[0]);
                m.ed[e] = make_float2((float)r1[1], (float)r1[2]);
            }
            share = (double)a.rho[e] * area / 3.0;
        }
        for (int c = 0; c < nc; ++c) mc[nc * le + c] = share;
    }
    // hinge corners carry no mass; hinge rest vectors X1-X3, X2-X3, X4-X3
    for (int lh = threadIdx.x; lh < 4 * p.n_h; lh += blockDim.x) mc[3 * p.n_e + lh] = 0.0;
    if (a.geometry) {
        for (int lh = threadIdx.x; lh < p.n_h; lh += blockDim.x) {
            const int h = p.h_begin + lh;
            const uint2 id = m.hidx[h];
            const int l1 = id.x & 0xffff, l2 = id.x >> 16, l3 = id.y & 0xffff, l4 = id.y >> 16;
            float4 q0 = m.hq[3 * h], q1 = m.hq[3 * h + 1], q2 = m.hq[3 * h + 2];
            q0.x = (float)(xs[3 * l1] - xs[3 * l3]);
            q0.y = (float)(xs[3 * l1 + 1] - xs[3 * l3 + 1]);
            q0.z = (float)(xs[3 * l1 + 2] - xs[3 * l3 + 2]);
            q1.x = (float)(xs[3 * l2] - xs[3 * l3]);
            q1.y = (float)(xs[3 * l2 + 1] - xs[3 * l3 + 1]);
            q1.z = (float)(xs[3 * l2 + 2] - xs[3 * l3 + 2]);
            q2.x = (float)(xs[3 * l4] - xs[3 * l3]);
            q2.y = (float)(xs[3 * l4 + 1] - xs[3 * l3 + 1]);
            q2.z = (float)(xs[3 * l4 + 2] - xs[3 * l3 + 2]);
            m.hq[3 * h] = q0;
            m.hq[3 * h + 1] = q1;
            m.hq[3 * h + 2] = q2;
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
        else a.mass_part[p.bnd_begin + (l - p.n_int)] = s;
    }
}

__global__ void k_mass_boundary(const NodeBlock* __restrict__ blocks, const MeshRT* __restrict__ rts, SetupArgs a) {
    const NodeBlock nb = blocks[blockIdx.x];
    const MeshRT& m = rts[nb.mesh];
    for (int i = threadIdx.x; i < nb.count; i += blockDim.x) {
        const int b = nb.begin + i;
        double s = 0.0;
        for (int k = m.bnd_rowptr[b]; k < m.bnd_rowptr[b + 1]; ++k) s += a.mass_part[m.bnd_parts[k]];
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
        if (m.kind == GS_TET) {
            float4 c = m.ec[e];
            if (mu) c.z = mu[u];
            if (lam) c.w = lam[u];
            m.ec[e] = c;
            if (act && m.eact) m.eact[e] = act[u];
        } else {
            float4 b = m.eb[e];
            if (mu) b.y = mu[u];
            if (lam) b.z = lam[u];
            if (act) b.w = act[u];
            m.eb[e] = b;
        }
    }
    if (kb && m.kind == GS_CLOTH) {
        for (int h = blockIdx.x * blockDim.x + threadIdx.x; h < m.n_hinges; h += gridDim.x * blockDim.x)
            m.hq[3 * h].w = kb[m.hinge_perm[h]];
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
        if (v) bufv(m, buf)[i] = make_float4(v[3 * u], v[3 * u + 1], v[3 * u + 2], 0.f);
    }
}

// rest state: u = 0 (x = X), inverse mass in .w, v = v0 (caller order)
__global__ void k_reset_state(const MeshRT* __restrict__ rts, const float* v0) {
    const MeshRT& m = rts[0];
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < m.n_nodes; i += gridDim.x * blockDim.x) {
        const int u = m.node_perm[i];
        m.st_x[i] = make_float4(0.f, 0.f, 0.f, m.w[i]);
        m.st_v[i] = make_float4(v0[3 * u], v0[3 * u + 1], v0[3 * u + 2], 0.f);
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
            const float4 q = m.vb[i];
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
        const uint2 id = m.eidx[e];
        if (d_rho) {
            if (m.kind == GS_TET) {
                const double s = msm[id.x & 0xffff] + msm[id.x >> 16] + msm[id.y & 0xffff] + msm[id.y >> 16];
                d_rho[u] = s * ((double)m.ec[e].y / 4.0);
            } else {
                const double s = msm[id.x & 0xffff] + msm[id.x >> 16] + msm[id.y & 0xffff];
                d_rho[u] = s * ((double)m.eb[e].x / 3.0);
            }
        }
        if (d_mu) d_mu[u] = m.g_mu[e];
        if (d_lam) d_lam[u] = m.g_lam[e];
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
size_t smem_bytes(int kind, bool adjoint, int max_loc, int max_slots) {
    (void)kind;
    return sizeof(float4) * ((size_t)max_loc * (adjoint ? 2 : 1) + (size_t)max_slots);
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

void launch_forward_step(const Launch& L, int tick, cudaStream_t s, Prof* prof) {
    if (L.n_tet_patches)
        GS_TIMED(KT_TET_FWD, (k_tet_fwd<<<L.n_tet_patches, L.threads, L.smem_tet_fwd, s>>>(L.tet_patches, L.rt, tick)));
    if (L.n_cloth_patches)
        GS_TIMED(KT_CLOTH_FWD,
                 (k_cloth_fwd<<<L.n_cloth_patches, L.threads, L.smem_cloth_fwd, s>>>(L.cloth_patches, L.rt, tick)));
    if (L.n_bnd_blocks)
        GS_TIMED(KT_FWD_BND, (k_fwd_boundary<<<L.n_bnd_blocks, 256, 0, s>>>(L.bnd_blocks, L.rt, tick)));
}

void launch_adjoint_step(const Launch& L, int tick, cudaStream_t s, Prof* prof) {
    if (L.n_tet_patches)
        GS_TIMED(KT_TET_ADJ, (k_tet_adj<<<L.n_tet_patches, L.threads, L.smem_tet_adj, s>>>(L.tet_patches, L.rt, tick)));
    if (L.n_cloth_patches)
        GS_TIMED(KT_CLOTH_ADJ,
                 (k_cloth_adj<<<L.n_cloth_patches, L.threads, L.smem_cloth_adj, s>>>(L.cloth_patches, L.rt, tick)));
    if (L.n_bnd_blocks)
        GS_TIMED(KT_ADJ_BND, (k_adj_boundary<<<L.n_bnd_blocks, 256, 0, s>>>(L.bnd_blocks, L.rt, tick)));
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
