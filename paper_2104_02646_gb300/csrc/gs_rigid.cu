// Rigid bodies (App. A.1 "Rigid Bodies"): state (x, r) with r = (w, x, y, z)
// a unit quaternion (world from body) and velocities (v, omega); the
// Newton-Euler equations with the compliant contact model of the particles
// acting at the body's contact points; semi-implicit Euler (App. B):
//   v+ = v + dt (g + F/m),  omega+ = omega + dt I_w^-1 (tau - omega x I_w omega),
//   x+ = x + dt v+,         r+ = normalise(r + dt/2 (0, omega+) (x) r),
// with I_w = R I_b R^T and F, tau the sums of the point contact forces and
// their moments about the centre of mass.
//
// Bodies do not interact, so one warp runs one body through the whole
// rollout in one launch: lanes take the contact points, a fixed xor tree
// sums force and torque, and every lane integrates the (identical) body
// state.  The rollout stores every state; the adjoint runs the steps in
// reverse in one launch, recomputing each step's contacts in one pass,
// with the parameter gradients summed in FP64.  Deterministic; no atomics.

#include <cuda_runtime.h>

#include <cmath>
#include <vector>

#include "gs_runtime.h"

namespace {

using gs::Buf;

constexpr int kWarpsPerBlock = 8;
// the adjoint holds ~150 registers per thread: blocks of 2 warps let six
// blocks (12 warps) share an SM where one 8-warp block would leave 8
constexpr int kAdjWarps = 2;
constexpr int kStateStride = 16;  // floats per stored body state (13 used)

struct Scene {
    int plane_on, sphere_on;
    float pn[3], ph;
    float sc[3], sr;
    float g[3];
};

struct Body {
    int p0, p1;           // contact points [p0, p1)
    float m;
    float I[6];           // Ixx, Iyy, Izz, Ixy, Ixz, Iyz (body frame, about the centre of mass)
    float ke, kd, kf, mu;
};

__device__ __forceinline__ float dot(const float* a, const float* b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }
__device__ __forceinline__ void cross(const float* a, const float* b, float* o) {
    o[0] = a[1] * b[2] - a[2] * b[1];
    o[1] = a[2] * b[0] - a[0] * b[2];
    o[2] = a[0] * b[1] - a[1] * b[0];
}

__device__ __forceinline__ void quat_rot(const float* r, float R[9]) {
    const float w = r[0], x = r[1], y = r[2], z = r[3];
    R[0] = 1.f - 2.f * (y * y + z * z); R[1] = 2.f * (x * y - w * z); R[2] = 2.f * (x * z + w * y);
    R[3] = 2.f * (x * y + w * z); R[4] = 1.f - 2.f * (x * x + z * z); R[5] = 2.f * (y * z - w * x);
    R[6] = 2.f * (x * z - w * y); R[7] = 2.f * (y * z + w * x); R[8] = 1.f - 2.f * (x * x + y * y);
}
// dR/dr contracted with Rb (the 9 entries above, row-major)
__device__ __forceinline__ void quat_rot_adj(const float* r, const float* Rb, float* rb) {
    const float w = r[0], x = r[1], y = r[2], z = r[3];
    rb[0] += 2.f * (-z * Rb[1] + y * Rb[2] + z * Rb[3] - x * Rb[5] - y * Rb[6] + x * Rb[7]);
    rb[1] += 2.f * (y * Rb[1] + z * Rb[2] + y * Rb[3] - 2.f * x * Rb[4] - w * Rb[5] + z * Rb[6] + w * Rb[7] -
                    2.f * x * Rb[8]);
    rb[2] += 2.f * (-2.f * y * Rb[0] + x * Rb[1] + w * Rb[2] + x * Rb[3] + z * Rb[5] - w * Rb[6] + z * Rb[7] -
                    2.f * y * Rb[8]);
    rb[3] += 2.f * (-2.f * z * Rb[0] - w * Rb[1] + x * Rb[2] + w * Rb[3] - 2.f * z * Rb[4] + y * Rb[5] + x * Rb[6] +
                    y * Rb[7]);
}

__device__ __forceinline__ void matvec(const float* M, const float* a, float* o) {
    for (int i = 0; i < 3; ++i) o[i] = M[3 * i] * a[0] + M[3 * i + 1] * a[1] + M[3 * i + 2] * a[2];
}
__device__ __forceinline__ void matTvec(const float* M, const float* a, float* o) {
    for (int i = 0; i < 3; ++i) o[i] = M[i] * a[0] + M[3 + i] * a[1] + M[6 + i] * a[2];
}
__device__ __forceinline__ void sym_full(const float* I6, float* M) {
    M[0] = I6[0]; M[4] = I6[1]; M[8] = I6[2];
    M[1] = M[3] = I6[3];
    M[2] = M[6] = I6[4];
    M[5] = M[7] = I6[5];
}
__device__ __forceinline__ void inv3(const float* A, float* B) {
    const float c00 = A[4] * A[8] - A[5] * A[7], c01 = A[5] * A[6] - A[3] * A[8], c02 = A[3] * A[7] - A[4] * A[6];
    const float det = A[0] * c00 + A[1] * c01 + A[2] * c02;
    const float id = 1.0f / det;
    B[0] = c00 * id;
    B[1] = (A[2] * A[7] - A[1] * A[8]) * id;
    B[2] = (A[1] * A[5] - A[2] * A[4]) * id;
    B[3] = c01 * id;
    B[4] = (A[0] * A[8] - A[2] * A[6]) * id;
    B[5] = (A[2] * A[3] - A[0] * A[5]) * id;
    B[6] = c02 * id;
    B[7] = (A[1] * A[6] - A[0] * A[7]) * id;
    B[8] = (A[0] * A[4] - A[1] * A[3]) * id;
}

// one contact with normal n and penetration C > 0 (the particles' law)
__device__ __forceinline__ void one_contact(const float* V, const float* n, float C, const Body& B, float* f) {
    const float vn = dot(n, V);
    const float fn = B.ke * C - B.kd * vn;
    float vs[3];
    for (int i = 0; i < 3; ++i) {
        f[i] += fn * n[i];
        vs[i] = V[i] - vn * n[i];
    }
    const float vsl = sqrtf(dot(vs, vs));
    const float afn = fabsf(fn);
    if (B.kf * vsl <= B.mu * afn) {
        for (int i = 0; i < 3; ++i) f[i] -= B.kf * vs[i];
    } else {
        const float s = B.mu * afn / vsl;
        for (int i = 0; i < 3; ++i) f[i] -= s * vs[i];
    }
}

// reverse of one_contact: adds dL/dV, dL/dn, dL/dC and the parameter gradients (ke, kd, kf, mu)
__device__ __forceinline__ void one_contact_adj(const float* V, const float* n, float C, const Body& B,
                                                const float* fb, float* Vb, float* nb, float& Cb, float* pb) {
    const float vn = dot(n, V);
    const float fn = B.ke * C - B.kd * vn;
    float vs[3];
    for (int i = 0; i < 3; ++i) vs[i] = V[i] - vn * n[i];
    const float vsl = sqrtf(dot(vs, vs));
    const float afn = fabsf(fn);
    float fnb = dot(fb, n);
    for (int i = 0; i < 3; ++i) nb[i] += fn * fb[i];
    float vsb[3];
    if (B.kf * vsl <= B.mu * afn) {
        pb[2] += -dot(fb, vs);
        for (int i = 0; i < 3; ++i) vsb[i] = -B.kf * fb[i];
    } else {
        const float s = B.mu * afn / vsl;
        const float sb = -dot(fb, vs);
        for (int i = 0; i < 3; ++i) vsb[i] = -s * fb[i];
        pb[3] += sb * afn / vsl;
        fnb += (fn < 0.f ? -1.f : 1.f) * sb * B.mu / vsl;
        const float vslb = -sb * B.mu * afn / (vsl * vsl);
        for (int i = 0; i < 3; ++i) vsb[i] += vslb * vs[i] / vsl;
    }
    // vs = V - vn n
    float vnb = -dot(vsb, n);
    for (int i = 0; i < 3; ++i) {
        Vb[i] += vsb[i];
        nb[i] += -vn * vsb[i];
    }
    // fn = ke C - kd vn
    pb[0] += fnb * C;
    Cb += B.ke * fnb;
    pb[1] += -fnb * vn;
    vnb += -B.kd * fnb;
    // vn = n . V
    for (int i = 0; i < 3; ++i) {
        Vb[i] += vnb * n[i];
        nb[i] += vnb * V[i];
    }
}

__device__ __forceinline__ void contact_force(const Scene& sc, const Body& B, const float* X, const float* V, float* f) {
    f[0] = f[1] = f[2] = 0.f;
    if (sc.plane_on) {
        const float C = sc.ph - dot(sc.pn, X);
        if (C > 0.f) one_contact(V, sc.pn, C, B, f);
    }
    if (sc.sphere_on) {
        float d[3] = {X[0] - sc.sc[0], X[1] - sc.sc[1], X[2] - sc.sc[2]};
        const float dist = sqrtf(dot(d, d));
        if (sc.sr - dist > 0.f && dist > 0.f) {
            const float n[3] = {d[0] / dist, d[1] / dist, d[2] / dist};
            one_contact(V, n, sc.sr - dist, B, f);
        }
    }
}

__device__ __forceinline__ void contact_adj(const Scene& sc, const Body& B, const float* X, const float* V,
                                            const float* fb, float* Xb, float* Vb, float* pb) {
    if (sc.plane_on) {
        const float C = sc.ph - dot(sc.pn, X);
        if (C > 0.f) {
            float nb[3] = {0.f, 0.f, 0.f}, Cb = 0.f;
            one_contact_adj(V, sc.pn, C, B, fb, Vb, nb, Cb, pb);
            for (int i = 0; i < 3; ++i) Xb[i] += -Cb * sc.pn[i];
        }
    }
    if (sc.sphere_on) {
        float d[3] = {X[0] - sc.sc[0], X[1] - sc.sc[1], X[2] - sc.sc[2]};
        const float dist = sqrtf(dot(d, d));
        if (sc.sr - dist > 0.f && dist > 0.f) {
            const float n[3] = {d[0] / dist, d[1] / dist, d[2] / dist};
            float nb[3] = {0.f, 0.f, 0.f}, Cb = 0.f;
            one_contact_adj(V, n, sc.sr - dist, B, fb, Vb, nb, Cb, pb);
            const float nn = dot(nb, n);
            for (int i = 0; i < 3; ++i) Xb[i] += (nb[i] - nn * n[i]) / dist - Cb * n[i];
        }
    }
}

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ Body load_body(const int* pb, const float* params, int b) {
    Body B;
    B.p0 = pb[b];
    B.p1 = pb[b + 1];
    const float* q = params + 11 * (size_t)b;
    B.m = q[0];
    for (int i = 0; i < 6; ++i) B.I[i] = q[1 + i];
    B.ke = q[7]; B.kd = q[8]; B.kf = q[9]; B.mu = q[10];
    return B;
}

// force and torque of the contacts at state s (lanes over points, xor-tree sums)
__device__ __forceinline__ void body_wrench(const Scene& sc, const Body& B, const float* pts, const float* s,
                                            const float* R, int lane, float* F, float* tau) {
    float f6[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    for (int k = B.p0 + lane; k < B.p1; k += 32) {
        const float p[3] = {pts[3 * (size_t)k], pts[3 * (size_t)k + 1], pts[3 * (size_t)k + 2]};
        float d[3], wd[3], X[3], V[3], fc[3], td[3];
        matvec(R, p, d);
        cross(s + 10, d, wd);
        for (int i = 0; i < 3; ++i) {
            X[i] = s[i] + d[i];
            V[i] = s[7 + i] + wd[i];
        }
        contact_force(sc, B, X, V, fc);
        cross(d, fc, td);
        for (int i = 0; i < 3; ++i) {
            f6[i] += fc[i];
            f6[3 + i] += td[i];
        }
    }
    for (int i = 0; i < 3; ++i) {
        F[i] = warp_sum(f6[i]);
        tau[i] = warp_sum(f6[3 + i]);
    }
}

// intermediate values of one step (every lane holds the same)
struct StepVals {
    float R[9], Ib[9], Binv[9];
    float F[3], tau[3];
    float e[3], c[3], L[3], h[3], a[3], bb[3], alpha[3];
    float vo[3], wo[3], q[4], qn;
};

__device__ __forceinline__ void step_forward(const Scene& sc, const Body& B, const float* pts, const float* s, float dt,
                                             int lane, StepVals& V, float* o) {
    quat_rot(s + 3, V.R);
    sym_full(B.I, V.Ib);
    inv3(V.Ib, V.Binv);
    body_wrench(sc, B, pts, s, V.R, lane, V.F, V.tau);
    // L = R I_b R^T omega, h = tau - omega x L, alpha = R I_b^-1 R^T h
    const float* w = s + 10;
    matTvec(V.R, w, V.e);
    matvec(V.Ib, V.e, V.c);
    matvec(V.R, V.c, V.L);
    float wL[3];
    cross(w, V.L, wL);
    for (int i = 0; i < 3; ++i) V.h[i] = V.tau[i] - wL[i];
    matTvec(V.R, V.h, V.a);
    matvec(V.Binv, V.a, V.bb);
    matvec(V.R, V.bb, V.alpha);
    for (int i = 0; i < 3; ++i) {
        V.vo[i] = s[7 + i] + dt * (sc.g[i] + V.F[i] / B.m);
        V.wo[i] = w[i] + dt * V.alpha[i];
        o[i] = s[i] + dt * V.vo[i];
        o[7 + i] = V.vo[i];
        o[10 + i] = V.wo[i];
    }
    const float* r = s + 3;
    float ax[3];
    cross(V.wo, r + 1, ax);
    V.q[0] = r[0] - 0.5f * dt * dot(V.wo, r + 1);
    for (int i = 0; i < 3; ++i) V.q[1 + i] = r[1 + i] + 0.5f * dt * (r[0] * V.wo[i] + ax[i]);
    V.qn = sqrtf(V.q[0] * V.q[0] + V.q[1] * V.q[1] + V.q[2] * V.q[2] + V.q[3] * V.q[3]);
    for (int i = 0; i < 4; ++i) o[3 + i] = V.q[i] / V.qn;
}

__device__ __forceinline__ void load_state(const float* src, float* s) {
    const float4* p = reinterpret_cast<const float4*>(src);
    const float4 a = p[0], b = p[1], c = p[2], d = p[3];
    s[0] = a.x; s[1] = a.y; s[2] = a.z; s[3] = a.w;
    s[4] = b.x; s[5] = b.y; s[6] = b.z; s[7] = b.w;
    s[8] = c.x; s[9] = c.y; s[10] = c.z; s[11] = c.w;
    s[12] = d.x;
}
__device__ __forceinline__ void store_state(float* dst, const float* s) {
    float4* p = reinterpret_cast<float4*>(dst);
    p[0] = make_float4(s[0], s[1], s[2], s[3]);
    p[1] = make_float4(s[4], s[5], s[6], s[7]);
    p[2] = make_float4(s[8], s[9], s[10], s[11]);
    p[3] = make_float4(s[12], 0.f, 0.f, 0.f);
}

// traj [(S + 1)][n_bodies][16]; state0 / stateS [n_bodies][13]
__global__ void __launch_bounds__(32 * kWarpsPerBlock)
    k_rigid_rollout(const int* __restrict__ pbeg, const float* __restrict__ params, const float* __restrict__ pts,
                    Scene sc, int nb, const float* __restrict__ state0, float dt, int S, float* __restrict__ traj,
                    float* __restrict__ stateS, int* __restrict__ status) {
    const int b = blockIdx.x * kWarpsPerBlock + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (b >= nb) return;
    const Body B = load_body(pbeg, params, b);
    float s[13], o[13];
    for (int i = 0; i < 13; ++i) s[i] = state0[13 * (size_t)b + i];
    if (lane == 0) store_state(traj + (size_t)b * kStateStride, s);
    bool finite = true;
    for (int n = 0; n < S; ++n) {
        StepVals V;
        step_forward(sc, B, pts, s, dt, lane, V, o);
        for (int i = 0; i < 13; ++i) {
            s[i] = o[i];
            finite = finite && isfinite(o[i]);
        }
        if (lane == 0) store_state(traj + ((size_t)(n + 1) * nb + b) * kStateStride, s);
    }
    if (lane == 0) {
        if (stateS)
            for (int i = 0; i < 13; ++i) stateS[13 * (size_t)b + i] = s[i];
        if (!finite) atomicOr(status, 1);  // integer flag, order-independent
    }
}

struct RigidGradOut {
    float* d_state0;   // [nb][13]
    double* d_mass;    // [nb]
    double* d_inertia; // [nb][6]
    double* d_contact; // [nb][4]
};

// One pass over the points per reverse step: the stored next state holds
// omega+ and r+, so dL/dF and dL/dtau are known before the contacts are
// evaluated; F and tau (the same sums, in the same order, as the forward's)
// come out of the same pass and finish the terms that need them.
__global__ void __launch_bounds__(32 * kAdjWarps, 6)
    k_rigid_adjoint(const int* __restrict__ pbeg, const float* __restrict__ params, const float* __restrict__ pts,
                    Scene sc, int nb, const float* __restrict__ traj, float dt, int S, const float* __restrict__ seed,
                    RigidGradOut out) {
    const int b = blockIdx.x * kAdjWarps + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (b >= nb) return;
    const Body B = load_body(pbeg, params, b);
    float Ib[9], Binv[9];
    sym_full(B.I, Ib);
    inv3(Ib, Binv);
    float lam[13];
    for (int i = 0; i < 13; ++i) lam[i] = seed ? seed[13 * (size_t)b + i] : 0.f;
    double gm = 0.0, gI[6] = {0, 0, 0, 0, 0, 0}, gc[4] = {0, 0, 0, 0};
    for (int n = S - 1; n >= 0; --n) {
        float s[13], o[13];
        load_state(traj + ((size_t)n * nb + b) * kStateStride, s);
        load_state(traj + ((size_t)(n + 1) * nb + b) * kStateStride, o);
        const float* r = s + 3;
        const float* w = s + 10;
        const float* wo = o + 10;
        float R[9];
        quat_rot(r, R);
        // q = r + dt/2 (0, wo) (x) r, r+ = q / |q|
        float q[4];
        {
            float ax[3];
            cross(wo, r + 1, ax);
            q[0] = r[0] - 0.5f * dt * dot(wo, r + 1);
            for (int i = 0; i < 3; ++i) q[1 + i] = r[1 + i] + 0.5f * dt * (r[0] * wo[i] + ax[i]);
        }
        const float qn = sqrtf(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
        float qb[4];
        {
            float rr = 0.f;
            for (int i = 0; i < 4; ++i) rr += lam[3 + i] * o[3 + i];
            for (int i = 0; i < 4; ++i) qb[i] = (lam[3 + i] - rr * o[3 + i]) / qn;
        }
        float rb[4], wob[3], xb[3], vb[3], wb[3], Rb[9];
        for (int i = 0; i < 9; ++i) Rb[i] = 0.f;
        {
            const float h = 0.5f * dt;
            float t[3], u[3];
            cross(wo, qb + 1, t);
            rb[0] = qb[0] + h * dot(wo, qb + 1);
            for (int i = 0; i < 3; ++i) rb[1 + i] = qb[1 + i] - h * wo[i] * qb[0] - h * t[i];
            cross(r + 1, qb + 1, u);
            for (int i = 0; i < 3; ++i) wob[i] = lam[10 + i] - h * r[1 + i] * qb[0] + h * (r[0] * qb[1 + i] + u[i]);
        }
        // x+ = x + dt v+ ; v+ = v + dt (g + F/m) ; w+ = w + dt alpha
        float vob[3], Fb[3], alb[3];
        for (int i = 0; i < 3; ++i) {
            xb[i] = lam[i];
            vob[i] = lam[7 + i] + dt * lam[i];
            vb[i] = vob[i];
            Fb[i] = dt * vob[i] / B.m;
            wb[i] = wob[i];
            alb[i] = dt * wob[i];
        }
        // alpha = R Binv R^T h: dL/dh = R Binv R^T dL/dalpha = dL/dtau
        float bbb[3], ab[3], hb[3];
        matTvec(R, alb, bbb);
        matvec(Binv, bbb, ab);
        matvec(R, ab, hb);
        // L = R Ib R^T w (independent of the contacts); h = tau - w x L
        float e[3], c[3], L[3];
        matTvec(R, w, e);
        matvec(Ib, e, c);
        matvec(R, c, L);
        float IbB[9];
        {
            float Lb[3], t[3], cb[3], eb[3], t2[3];
            cross(w, hb, Lb);
            cross(L, hb, t);
            for (int i = 0; i < 3; ++i) wb[i] -= t[i];
            for (int i = 0; i < 3; ++i)
                for (int j = 0; j < 3; ++j) Rb[3 * i + j] += Lb[i] * c[j];
            matTvec(R, Lb, cb);
            for (int i = 0; i < 3; ++i)
                for (int j = 0; j < 3; ++j) IbB[3 * i + j] = cb[i] * e[j];
            matvec(Ib, cb, eb);
            for (int i = 0; i < 3; ++i)
                for (int j = 0; j < 3; ++j) Rb[3 * i + j] += w[i] * eb[j];
            matvec(R, eb, t2);
            for (int i = 0; i < 3; ++i) wb[i] += t2[i];
        }
        // the points: F, tau and the adjoint sums in one pass
        float f6[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        float acc[22];  // x(3) v(3) w(3) R(9) contact(4)
        for (int i = 0; i < 22; ++i) acc[i] = 0.f;
        for (int k = B.p0 + lane; k < B.p1; k += 32) {
            const float p[3] = {pts[3 * (size_t)k], pts[3 * (size_t)k + 1], pts[3 * (size_t)k + 2]};
            float d[3], wd[3], X[3], Vv[3], fc[3], td[3];
            matvec(R, p, d);
            cross(w, d, wd);
            for (int i = 0; i < 3; ++i) {
                X[i] = s[i] + d[i];
                Vv[i] = s[7 + i] + wd[i];
            }
            contact_force(sc, B, X, Vv, fc);
            cross(d, fc, td);
            for (int i = 0; i < 3; ++i) {
                f6[i] += fc[i];
                f6[3 + i] += td[i];
            }
            float fcb[3], db[3], t3[3];
            cross(hb, d, t3);
            for (int i = 0; i < 3; ++i) fcb[i] = Fb[i] + t3[i];
            cross(fc, hb, db);
            float Xb[3] = {0.f, 0.f, 0.f}, Vb[3] = {0.f, 0.f, 0.f};
            contact_adj(sc, B, X, Vv, fcb, Xb, Vb, acc + 18);
            float t4[3], t5[3];
            cross(d, Vb, t4);
            cross(Vb, w, t5);
            for (int i = 0; i < 3; ++i) {
                acc[i] += Xb[i];
                acc[3 + i] += Vb[i];
                acc[6 + i] += t4[i];
                db[i] += Xb[i] + t5[i];
            }
            for (int i = 0; i < 3; ++i)
                for (int j = 0; j < 3; ++j) acc[9 + 3 * i + j] += db[i] * p[j];
        }
        float F[3], tau[3];
        for (int i = 0; i < 3; ++i) {
            F[i] = warp_sum(f6[i]);
            tau[i] = warp_sum(f6[3 + i]);
        }
        for (int i = 0; i < 22; ++i) acc[i] = warp_sum(acc[i]);
        // the terms that need F and tau
        {
            float wL[3], h[3], a[3], bb[3];
            cross(w, L, wL);
            for (int i = 0; i < 3; ++i) h[i] = tau[i] - wL[i];
            matTvec(R, h, a);
            matvec(Binv, a, bb);
            for (int i = 0; i < 3; ++i)
                for (int j = 0; j < 3; ++j) {
                    Rb[3 * i + j] += alb[i] * bb[j] + h[i] * ab[j];
                    IbB[3 * i + j] += -ab[i] * bb[j];
                }
            gm += -(double)dt * (double)dot(F, vob) / ((double)B.m * (double)B.m);
        }
        for (int i = 0; i < 3; ++i) {
            xb[i] += acc[i];
            vb[i] += acc[3 + i];
            wb[i] += acc[6 + i];
        }
        for (int i = 0; i < 9; ++i) Rb[i] += acc[9 + i];
        for (int i = 0; i < 4; ++i) gc[i] += (double)acc[18 + i];
        gI[0] += IbB[0]; gI[1] += IbB[4]; gI[2] += IbB[8];
        gI[3] += (double)IbB[1] + IbB[3];
        gI[4] += (double)IbB[2] + IbB[6];
        gI[5] += (double)IbB[5] + IbB[7];
        quat_rot_adj(r, Rb, rb);
        for (int i = 0; i < 3; ++i) {
            lam[i] = xb[i];
            lam[7 + i] = vb[i];
            lam[10 + i] = wb[i];
        }
        for (int i = 0; i < 4; ++i) lam[3 + i] = rb[i];
    }
    if (lane == 0) {
        if (out.d_state0)
            for (int i = 0; i < 13; ++i) out.d_state0[13 * (size_t)b + i] = lam[i];
        if (out.d_mass) out.d_mass[b] = gm;
        if (out.d_inertia)
            for (int i = 0; i < 6; ++i) out.d_inertia[6 * (size_t)b + i] = gI[i];
        if (out.d_contact)
            for (int i = 0; i < 4; ++i) out.d_contact[4 * (size_t)b + i] = gc[i];
    }
}

// world positions of the points: X_k = x + R p_k; one thread per point
__global__ void k_rigid_points(const int* __restrict__ owner, const float* __restrict__ pts, int np,
                               const float* __restrict__ state, float* __restrict__ out) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= np) return;
    const float* s = state + 13 * (size_t)owner[k];
    float R[9], d[3];
    quat_rot(s + 3, R);
    matvec(R, pts + 3 * (size_t)k, d);
    for (int i = 0; i < 3; ++i) out[3 * (size_t)k + i] = s[i] + d[i];
}

// dL/dstate from dL/dX of the points: one warp per body, fixed-order sums
__global__ void __launch_bounds__(32 * kWarpsPerBlock)
    k_rigid_points_adj(const int* __restrict__ pbeg, const float* __restrict__ pts, int nb,
                       const float* __restrict__ state, const float* __restrict__ gX, float* __restrict__ gstate) {
    const int b = blockIdx.x * kWarpsPerBlock + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (b >= nb) return;
    const float* s = state + 13 * (size_t)b;
    float acc[12] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};  // x(3), R(9)
    for (int k = pbeg[b] + lane; k < pbeg[b + 1]; k += 32) {
        const float* g = gX + 3 * (size_t)k;
        const float* p = pts + 3 * (size_t)k;
        for (int i = 0; i < 3; ++i) {
            acc[i] += g[i];
            for (int j = 0; j < 3; ++j) acc[3 + 3 * i + j] += g[i] * p[j];
        }
    }
    for (int i = 0; i < 12; ++i) acc[i] = warp_sum(acc[i]);
    float rb[4] = {0.f, 0.f, 0.f, 0.f};
    quat_rot_adj(s + 3, acc + 3, rb);
    if (lane == 0) {
        float* o = gstate + 13 * (size_t)b;
        for (int i = 0; i < 3; ++i) o[i] = acc[i];
        for (int i = 0; i < 4; ++i) o[3 + i] = rb[i];
        for (int i = 7; i < 13; ++i) o[i] = 0.f;
    }
}

}  // namespace

struct gs_rigid {
    gs_ctx* ctx = nullptr;
    int nb = 0, np = 0;
    Scene sc{};
    Buf pbeg, owner, pts, params, traj, status;
    int S = -1;  // steps of the stored rollout (-1: none)
    float dt = 0.f;
};

static gs_status check_params(int nb, const float* mass, const float* inertia, const float* contact) {
    for (int b = 0; b < nb; ++b) {
        if (mass && !(mass[b] > 0.f && std::isfinite(mass[b]))) return gs::set_error(GS_EINVAL, "mass must be > 0");
        if (inertia) {
            const float* I = inertia + 6 * (size_t)b;
            for (int i = 0; i < 6; ++i)
                if (!std::isfinite(I[i])) return gs::set_error(GS_EINVAL, "non-finite inertia");
            // positive definite: leading minors > 0
            const double a = I[0], bb = I[1], c = I[2], d = I[3], e = I[4], f = I[5];
            const double m2 = a * bb - d * d;
            const double m3 = a * (bb * c - f * f) - d * (d * c - f * e) + e * (d * f - bb * e);
            if (!(a > 0 && m2 > 0 && m3 > 0)) return gs::set_error(GS_EINVAL, "inertia must be positive definite");
        }
        if (contact) {
            const float* k = contact + 4 * (size_t)b;
            for (int i = 0; i < 4; ++i)
                if (!(k[i] >= 0.f && std::isfinite(k[i])))
                    return gs::set_error(GS_EINVAL, "contact parameters must be finite and >= 0");
        }
    }
    return GS_OK;
}

extern "C" gs_status gs_rigid_create(gs_ctx* ctx, const gs_rigid_desc* d, gs_rigid** out) try {
    gs::clear_error();
    if (!ctx || !d || !out) return gs::set_error(GS_EINVAL, "null argument");
    *out = nullptr;
    if (d->n_bodies <= 0 || !d->point_begin || !d->points || !d->mass || !d->inertia || !d->contact)
        return gs::set_error(GS_EINVAL, "need n_bodies > 0, point_begin, points, mass, inertia, contact");
    const int nb = d->n_bodies;
    if (d->point_begin[0] != 0) return gs::set_error(GS_EINVAL, "point_begin[0] must be 0");
    for (int b = 0; b < nb; ++b)
        if (d->point_begin[b + 1] < d->point_begin[b]) return gs::set_error(GS_EINVAL, "point_begin must not decrease");
    const int np = d->point_begin[nb];
    for (size_t i = 0; i < 3 * (size_t)np; ++i)
        if (!std::isfinite(d->points[i])) return gs::set_error(GS_EINVAL, "non-finite point");
    GS_TRY(check_params(nb, d->mass, d->inertia, d->contact));
    const gs_contact& c = d->scene;
    if (c.plane_on) {
        const double nn = (double)c.plane_n[0] * c.plane_n[0] + (double)c.plane_n[1] * c.plane_n[1] +
                          (double)c.plane_n[2] * c.plane_n[2];
        if (std::fabs(nn - 1.0) > 1e-4) return gs::set_error(GS_EINVAL, "plane normal must be unit length");
    }
    if (c.sphere_on && !(c.sphere_r > 0.f)) return gs::set_error(GS_EINVAL, "sphere radius must be > 0");
    auto r = new gs_rigid;
    r->ctx = ctx;
    r->nb = nb;
    r->np = np;
    r->sc.plane_on = c.plane_on;
    r->sc.sphere_on = c.sphere_on;
    for (int i = 0; i < 3; ++i) {
        r->sc.pn[i] = c.plane_n[i];
        r->sc.sc[i] = c.sphere_c[i];
        r->sc.g[i] = d->gravity[i];
    }
    r->sc.ph = c.plane_h;
    r->sc.sr = c.sphere_r;
    std::vector<int> owner(np > 0 ? np : 1, 0);
    for (int b = 0; b < nb; ++b)
        for (int k = d->point_begin[b]; k < d->point_begin[b + 1]; ++k) owner[k] = b;
    std::vector<float> params(11 * (size_t)nb);
    for (int b = 0; b < nb; ++b) {
        params[11 * b] = d->mass[b];
        for (int i = 0; i < 6; ++i) params[11 * b + 1 + i] = d->inertia[6 * b + i];
        for (int i = 0; i < 4; ++i) params[11 * b + 7 + i] = d->contact[4 * b + i];
    }
    cudaStream_t s = nullptr;
    gs_status st = GS_OK;
    auto up = [&](Buf& buf, const void* src, size_t bytes) -> gs_status {
        GS_TRY(buf.alloc(ctx, std::max<size_t>(bytes, 16), s));
        if (bytes) GS_CUDA(cudaMemcpyAsync(buf.p, src, bytes, cudaMemcpyHostToDevice, s));
        return GS_OK;
    };
    if ((st = up(r->pbeg, d->point_begin, 4 * (size_t)(nb + 1))) < 0 || (st = up(r->owner, owner.data(), 4 * owner.size())) < 0 ||
        (st = up(r->pts, d->points, 12 * (size_t)np)) < 0 || (st = up(r->params, params.data(), 4 * params.size())) < 0 ||
        (st = r->status.alloc(ctx, 16, s)) < 0) {
        delete r;
        return st;
    }
    cudaError_t e = cudaMemsetAsync(r->status.p, 0, 16, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        delete r;
        return gs::cuda_error(e, "gs_rigid_create");
    }
    *out = r;
    return GS_OK;
} GS_ABI_CATCH

extern "C" void gs_rigid_destroy(gs_rigid* r) {
    if (!r) return;
    cudaDeviceSynchronize();
    delete r;
}

extern "C" gs_status gs_rigid_set_params(gs_rigid* r, const float* mass, const float* inertia, const float* contact,
                                         void* stream) try {
    gs::clear_error();
    if (!r) return gs::set_error(GS_EINVAL, "null body set");
    GS_TRY(check_params(r->nb, mass, inertia, contact));
    std::vector<float> params(11 * (size_t)r->nb);
    cudaStream_t s = (cudaStream_t)stream;
    GS_CUDA(cudaMemcpyAsync(params.data(), r->params.p, 4 * params.size(), cudaMemcpyDeviceToHost, s));
    GS_CUDA(cudaStreamSynchronize(s));
    for (int b = 0; b < r->nb; ++b) {
        if (mass) params[11 * b] = mass[b];
        if (inertia)
            for (int i = 0; i < 6; ++i) params[11 * b + 1 + i] = inertia[6 * b + i];
        if (contact)
            for (int i = 0; i < 4; ++i) params[11 * b + 7 + i] = contact[4 * b + i];
    }
    GS_CUDA(cudaMemcpyAsync(r->params.p, params.data(), 4 * params.size(), cudaMemcpyHostToDevice, s));
    GS_CUDA(cudaStreamSynchronize(s));
    return GS_OK;
} GS_ABI_CATCH

extern "C" gs_status gs_rigid_rollout(gs_rigid* r, float dt, int S, const float* state0, float* stateS, void* stream) try {
    gs::clear_error();
    if (!r || !state0) return gs::set_error(GS_EINVAL, "null argument");
    if (S < 0 || !(dt > 0.f) || !std::isfinite(dt)) return gs::set_error(GS_EINVAL, "need S >= 0 and dt > 0");
    cudaStream_t s = (cudaStream_t)stream;
    const size_t bytes = sizeof(float) * kStateStride * (size_t)(S + 1) * r->nb;
    if (r->traj.bytes < bytes) GS_TRY(r->traj.alloc(r->ctx, bytes, s));
    const int grid = (r->nb + kWarpsPerBlock - 1) / kWarpsPerBlock;
    k_rigid_rollout<<<grid, 32 * kWarpsPerBlock, 0, s>>>((const int*)r->pbeg.p, (const float*)r->params.p,
                                                         (const float*)r->pts.p, r->sc, r->nb, state0, dt, S,
                                                         (float*)r->traj.p, stateS, (int*)r->status.p);
    GS_CUDA(cudaGetLastError());
    r->S = S;
    r->dt = dt;
    return GS_OK;
} GS_ABI_CATCH

extern "C" gs_status gs_rigid_adjoint(gs_rigid* r, const float* dL_dstateS, gs_rigid_grads* g, void* stream) try {
    gs::clear_error();
    if (!r || !g) return gs::set_error(GS_EINVAL, "null argument");
    if (r->S < 0) return gs::set_error(GS_ESTATE, "gs_rigid_adjoint needs a gs_rigid_rollout first");
    cudaStream_t s = (cudaStream_t)stream;
    RigidGradOut o{g->d_state0, g->d_mass, g->d_inertia, g->d_contact};
    const int grid = (r->nb + kAdjWarps - 1) / kAdjWarps;
    k_rigid_adjoint<<<grid, 32 * kAdjWarps, 0, s>>>((const int*)r->pbeg.p, (const float*)r->params.p,
                                                         (const float*)r->pts.p, r->sc, r->nb,
                                                         (const float*)r->traj.p, r->dt, r->S, dL_dstateS, o);
    GS_CUDA(cudaGetLastError());
    return GS_OK;
} GS_ABI_CATCH

extern "C" gs_status gs_rigid_points(gs_rigid* r, const float* state, float* points, void* stream) try {
    gs::clear_error();
    if (!r || !state || !points) return gs::set_error(GS_EINVAL, "null argument");
    if (r->np > 0)
        k_rigid_points<<<(r->np + 255) / 256, 256, 0, (cudaStream_t)stream>>>(
            (const int*)r->owner.p, (const float*)r->pts.p, r->np, state, points);
    GS_CUDA(cudaGetLastError());
    return GS_OK;
} GS_ABI_CATCH

extern "C" gs_status gs_rigid_points_backward(gs_rigid* r, const float* state, const float* dL_dpoints,
                                              float* dL_dstate, void* stream) try {
    gs::clear_error();
    if (!r || !state || !dL_dpoints || !dL_dstate) return gs::set_error(GS_EINVAL, "null argument");
    const int grid = (r->nb + kWarpsPerBlock - 1) / kWarpsPerBlock;
    k_rigid_points_adj<<<grid, 32 * kWarpsPerBlock, 0, (cudaStream_t)stream>>>(
        (const int*)r->pbeg.p, (const float*)r->pts.p, r->nb, state, dL_dpoints, dL_dstate);
    GS_CUDA(cudaGetLastError());
    return GS_OK;
} GS_ABI_CATCH

extern "C" gs_status gs_rigid_check(gs_rigid* r, int reset, void* stream) try {
    gs::clear_error();
    if (!r) return gs::set_error(GS_EINVAL, "null body set");
    int st = 0;
    cudaStream_t s = (cudaStream_t)stream;
    GS_CUDA(cudaMemcpyAsync(&st, r->status.p, sizeof(int), cudaMemcpyDeviceToHost, s));
    GS_CUDA(cudaStreamSynchronize(s));
    if (reset) GS_CUDA(cudaMemsetAsync(r->status.p, 0, sizeof(int), s));
    return (st & 1) ? GS_ENONFINITE : GS_OK;
} GS_ABI_CATCH
