// Device math of the explicit step and its adjoint (FP32).
//
// Element physics (App. A.1 / C.1 of the paper):
//   tets   Psi = mu/2 (I_C - 3) + lambda/2 (J - alpha)^2 - mu/2 log(I_C + 1),
//          alpha = 1 + 3 mu / (4 lambda) + a_e (rest-stable target + actuation),
//          P = mu F (1 - 1/(I_C + 1)) + lambda (J - alpha) cof F,
//          corner forces: columns of -V P Dm^-T, f0 = -(f1 + f2 + f3)
//   tris   same energy with F 3x2, I_C - 2, J = |f0 x f1|,
//          alpha = 1 + 2 mu / (3 lambda) + a_t
//   hinges Bridson's bending force  k_b |E|^2/(|N1|+|N2|) sin(phi/2 + alpha) u_i
// Contact (App. A.1 "Contact", App. C.2): penalty normal force and relaxed
// Coulomb friction against a plane and a sphere.
//
// The adjoints below are hand-derived reverse mode of exactly these
// forward formulas (the paper obtains its adjoints by source transformation;
// here they are written out): for the hyperelastic elements the Hessian of
// Psi is self-adjoint, so F_bar = dP/dF[P_bar]; the hinge and the contact
// law are differentiated statement by statement in reverse order.
#pragma once

#include <cuda_runtime.h>

namespace gs {

__device__ __forceinline__ float3 operator+(float3 a, float3 b) { return make_float3(a.x + b.x, a.y + b.y, a.z + b.z); }
__device__ __forceinline__ float3 operator-(float3 a, float3 b) { return make_float3(a.x - b.x, a.y - b.y, a.z - b.z); }
__device__ __forceinline__ float3 operator-(float3 a) { return make_float3(-a.x, -a.y, -a.z); }
__device__ __forceinline__ float3 operator*(float3 a, float s) { return make_float3(a.x * s, a.y * s, a.z * s); }
__device__ __forceinline__ float3 operator*(float s, float3 a) { return make_float3(a.x * s, a.y * s, a.z * s); }
__device__ __forceinline__ float3& operator+=(float3& a, float3 b) { a.x += b.x; a.y += b.y; a.z += b.z; return a; }
__device__ __forceinline__ float3& operator-=(float3& a, float3 b) { a.x -= b.x; a.y -= b.y; a.z -= b.z; return a; }
__device__ __forceinline__ float dot3(float3 a, float3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
__device__ __forceinline__ float3 cross3(float3 a, float3 b) {
    return make_float3(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x);
}
__device__ __forceinline__ float3 xyz(float4 a) { return make_float3(a.x, a.y, a.z); }
__device__ __forceinline__ float4 f4(float3 a, float w) { return make_float4(a.x, a.y, a.z, w); }

// ---------------------------------------------------------------------------
// Displacement form.  The state holds u = x - X (X: rest positions), so the
// deformation gradient is F = I + H (tets) or F = R0 + H (triangles; R0 the
// rest frame), H = [u1-u0, u2-u0, (u3-u0)] Dm^-1.  Stress and energy
// derivatives are written in terms of H without subtracting O(1) terms, so
// FP32 keeps full relative precision at small strain and an element at rest
// carries exactly zero force:
//   det(I+H) = 1 + tr H + i2(H) + det H,  cof(I+H) = (1 + tr H) I - H^T + cof H,
//   mu F (1 - 1/(I_C+1)) - 3/4 mu cof F = mu [3/4 (H + H^T - tr H I - cof H)
//                                             + (I_C - 3)/(4 (I_C + 1)) F].
// ---------------------------------------------------------------------------

// ---------------------------------------------------------------------------
// tetrahedron
// Dm^-1 rows: D0 = (a.x a.y a.z), D1 = (a.w b.x b.y), D2 = (b.z b.w c.x);
// V = c.y, mu = c.z, lambda = c.w.
// ---------------------------------------------------------------------------
struct TetState {
    float3 F0, F1, F2;  // columns of F = I + H
    float3 C0, C1, C2;  // columns of cof F
    float3 M0, M1, M2;  // columns of dP/dmu = F (1 - 1/(I_C+1)) - 3/4 cof F
    float inv;          // 1 / (I_C + 1)
    float cm;           // J - 1 - act
    float ca, cb;       // mu (1 - inv), lambda (J - alpha)
};

__device__ __forceinline__ void tet_state(float3 u0, float3 u1, float3 u2, float3 u3, float4 a, float4 b,
                                          float4 c, float act, TetState& s) {
    const float3 d1 = u1 - u0, d2 = u2 - u0, d3 = u3 - u0;
    const float3 H0 = d1 * a.x + d2 * a.w + d3 * b.z;  // columns of H
    const float3 H1 = d1 * a.y + d2 * b.x + d3 * b.w;
    const float3 H2 = d1 * a.z + d2 * b.y + d3 * c.x;
    const float tr = H0.x + H1.y + H2.z;
    const float Ic3 = 2.0f * tr + dot3(H0, H0) + dot3(H1, H1) + dot3(H2, H2);  // I_C - 3
    const float3 K0 = cross3(H1, H2), K1 = cross3(H2, H0), K2 = cross3(H0, H1);  // cof H
    const float jm1 = tr + (K0.x + K1.y + K2.z) + dot3(H0, K0);                  // J - 1
    const float3 T0 = make_float3(H0.x, H1.x, H2.x);                             // columns of H^T
    const float3 T1 = make_float3(H0.y, H1.y, H2.y);
    const float3 T2 = make_float3(H0.z, H1.z, H2.z);
    const float t1 = 1.0f + tr;
    s.F0 = make_float3(H0.x + 1.0f, H0.y, H0.z);
    s.F1 = make_float3(H1.x, H1.y + 1.0f, H1.z);
    s.F2 = make_float3(H2.x, H2.y, H2.z + 1.0f);
    s.C0 = make_float3(t1, 0.f, 0.f) - T0 + K0;
    s.C1 = make_float3(0.f, t1, 0.f) - T1 + K1;
    s.C2 = make_float3(0.f, 0.f, t1) - T2 + K2;
    const float mu = c.z, lam = c.w;
    s.inv = 1.0f / (Ic3 + 4.0f);
    const float q = 0.25f * Ic3 * s.inv;
    s.M0 = 0.75f * (H0 + T0 - make_float3(tr, 0.f, 0.f) - K0) + q * s.F0;
    s.M1 = 0.75f * (H1 + T1 - make_float3(0.f, tr, 0.f) - K1) + q * s.F1;
    s.M2 = 0.75f * (H2 + T2 - make_float3(0.f, 0.f, tr) - K2) + q * s.F2;
    s.cm = jm1 - act;
    s.ca = mu * (Ic3 + 3.0f) * s.inv;
    s.cb = lam * s.cm - 0.75f * mu;
}

// corner forces f1..f3 = columns of -V P Dm^-T; f0 = -(f1 + f2 + f3),
// P = mu dP/dmu + lambda (J - 1 - act) cof F
__device__ __forceinline__ void tet_forces(const TetState& s, float4 a, float4 b, float4 c, float3& f0,
                                           float3& f1, float3& f2, float3& f3) {
    const float mu = c.z, lc = c.w * s.cm;
    const float3 P0 = mu * s.M0 + lc * s.C0;
    const float3 P1 = mu * s.M1 + lc * s.C1;
    const float3 P2 = mu * s.M2 + lc * s.C2;
    const float nV = -c.y;
    f1 = nV * (P0 * a.x + P1 * a.y + P2 * a.z);
    f2 = nV * (P0 * a.w + P1 * b.x + P2 * b.y);
    f3 = nV * (P0 * b.z + P1 * b.w + P2 * c.x);
    f0 = -(f1 + f2 + f3);
}

// Reverse mode of tet_forces.  Given fb_i = dL/df_i, returns dL/du_i and
// dL/d(mu, lambda, act).  P_bar = -V G Dm^-1 with G = [fb1-fb0, fb2-fb0, fb3-fb0];
// F_bar = mu (1 - 1/(I_C+1)) P_bar + 2 mu/(I_C+1)^2 (F:P_bar) F
//         + lambda (cof F : P_bar) cof F + lambda (J - alpha) dcof[P_bar];
// Ds_bar = F_bar Dm^-T.
__device__ __forceinline__ void tet_adjoint(const TetState& s, float4 a, float4 b, float4 c, float3 fb0,
                                            float3 fb1, float3 fb2, float3 fb3, float3& xb0, float3& xb1,
                                            float3& xb2, float3& xb3, float& gmu, float& glam, float& gact) {
    const float mu = c.z, lam = c.w, nV = -c.y;
    const float3 G1 = fb1 - fb0, G2 = fb2 - fb0, G3 = fb3 - fb0;
    const float3 Pb0 = nV * (G1 * a.x + G2 * a.w + G3 * b.z);
    const float3 Pb1 = nV * (G1 * a.y + G2 * b.x + G3 * b.w);
    const float3 Pb2 = nV * (G1 * a.z + G2 * b.y + G3 * c.x);
    const float FP = dot3(s.F0, Pb0) + dot3(s.F1, Pb1) + dot3(s.F2, Pb2);
    const float CP = dot3(s.C0, Pb0) + dot3(s.C1, Pb1) + dot3(s.C2, Pb2);
    const float MP = dot3(s.M0, Pb0) + dot3(s.M1, Pb1) + dot3(s.M2, Pb2);
    const float k2 = 2.0f * mu * s.inv * s.inv * FP;
    const float lc = lam * CP;
    const float3 dC0 = cross3(Pb1, s.F2) + cross3(s.F1, Pb2);
    const float3 dC1 = cross3(Pb2, s.F0) + cross3(s.F2, Pb0);
    const float3 dC2 = cross3(Pb0, s.F1) + cross3(s.F0, Pb1);
    const float3 Fb0 = s.ca * Pb0 + k2 * s.F0 + lc * s.C0 + s.cb * dC0;
    const float3 Fb1 = s.ca * Pb1 + k2 * s.F1 + lc * s.C1 + s.cb * dC1;
    const float3 Fb2 = s.ca * Pb2 + k2 * s.F2 + lc * s.C2 + s.cb * dC2;
    xb1 = Fb0 * a.x + Fb1 * a.y + Fb2 * a.z;
    xb2 = Fb0 * a.w + Fb1 * b.x + Fb2 * b.y;
    xb3 = Fb0 * b.z + Fb1 * b.w + Fb2 * c.x;
    xb0 = -(xb1 + xb2 + xb3);
    // dP/dmu = M;  dP/dlambda = (J - 1 - act) cof F;  dP/dact = -lambda cof F
    gmu = MP;
    glam = s.cm * CP;
    gact = -lam * CP;
}

// ---------------------------------------------------------------------------
// membrane triangle.  Dm^-1 = [[a.x a.y], [a.z a.w]]; b = (A, mu, lambda, act);
// R0 = rest F (3x2, orthonormal columns r0, r1).  With F = R0 + H,
// G = F^T F = I + E, E = R0^T H + H^T R0 + H^T H;  I_C = 2 + tr E,
// J = sqrt(det G) = 1 + (tr E + det E)/(J + 1),  dJ/dF = F adj(G) / J,
// P = mu F [s1 I + 2 E / (3 J)] + lambda (J - 1 - act) dJ/dF with
// s1 = (6 (J-1) + 3 (J-1) tr E - 5 tr E - 2 (tr E)^2) / (3 J (3 + tr E)).
// ---------------------------------------------------------------------------
struct TriState {
    float3 F0, F1, n, dJ0, dJ1, M0, M1;
    float inv, iJ, cm, ca, cb;
};

__device__ __forceinline__ void tri_state(float3 u0, float3 u1, float3 u2, float4 a, float4 b, float3 r0,
                                          float3 r1, TriState& s) {
    const float3 d1 = u1 - u0, d2 = u2 - u0;
    const float3 H0 = d1 * a.x + d2 * a.z;
    const float3 H1 = d1 * a.y + d2 * a.w;
    s.F0 = r0 + H0;
    s.F1 = r1 + H1;
    const float E00 = 2.0f * dot3(r0, H0) + dot3(H0, H0);
    const float E11 = 2.0f * dot3(r1, H1) + dot3(H1, H1);
    const float E01 = dot3(r0, H1) + dot3(H0, r1) + dot3(H0, H1);
    const float trE = E00 + E11, detE = E00 * E11 - E01 * E01;
    const float J = sqrtf(1.0f + trE + detE);
    const float jm1 = (trE + detE) / (J + 1.0f);
    s.iJ = 1.0f / J;
    s.inv = 1.0f / (trE + 3.0f);
    s.dJ0 = (s.F0 * (1.0f + E11) - s.F1 * E01) * s.iJ;
    s.dJ1 = (s.F1 * (1.0f + E00) - s.F0 * E01) * s.iJ;
    const float s1 = (6.0f * jm1 + 3.0f * jm1 * trE - 5.0f * trE - 2.0f * trE * trE) / (3.0f * J * (3.0f + trE));
    const float t = (2.0f / 3.0f) * s.iJ;
    s.M0 = s.F0 * (s1 + t * E00) + s.F1 * (t * E01);
    s.M1 = s.F0 * (t * E01) + s.F1 * (s1 + t * E11);
    s.n = cross3(s.F0, s.F1) * s.iJ;
    const float mu = b.y, lam = b.z;
    s.cm = jm1 - b.w;
    s.ca = mu * (trE + 2.0f) * s.inv;
    s.cb = lam * s.cm - (2.0f / 3.0f) * mu;
}

__device__ __forceinline__ void tri_forces(const TriState& s, float4 a, float4 b, float3& f0, float3& f1,
                                           float3& f2) {
    const float mu = b.y, lc = b.z * s.cm;
    const float3 P0 = mu * s.M0 + lc * s.dJ0;
    const float3 P1 = mu * s.M1 + lc * s.dJ1;
    const float nA = -b.x;
    f1 = nA * (P0 * a.x + P1 * a.y);
    f2 = nA * (P0 * a.z + P1 * a.w);
    f0 = -(f1 + f2);
}

// Reverse mode of tri_forces: P_bar = -A G Dm^-1, F_bar = dP/dF[P_bar] with
// the Hessian of J applied through dn = (I - n n^T) dc / J,
// dc = P_bar0 x f1 + f0 x P_bar1.
__device__ __forceinline__ void tri_adjoint(const TriState& s, float4 a, float4 b, float3 fb0, float3 fb1,
                                            float3 fb2, float3& xb0, float3& xb1, float3& xb2, float& gmu,
                                            float& glam, float& gact) {
    const float mu = b.y, lam = b.z, nA = -b.x;
    const float3 G1 = fb1 - fb0, G2 = fb2 - fb0;
    const float3 Pb0 = nA * (G1 * a.x + G2 * a.z);
    const float3 Pb1 = nA * (G1 * a.y + G2 * a.w);
    const float FP = dot3(s.F0, Pb0) + dot3(s.F1, Pb1);
    const float JP = dot3(s.dJ0, Pb0) + dot3(s.dJ1, Pb1);
    const float MP = dot3(s.M0, Pb0) + dot3(s.M1, Pb1);
    const float3 dc = cross3(Pb0, s.F1) + cross3(s.F0, Pb1);
    const float3 dn = (dc - s.n * dot3(s.n, dc)) * s.iJ;
    const float3 HJ0 = cross3(Pb1, s.n) + cross3(s.F1, dn);
    const float3 HJ1 = cross3(dn, s.F0) + cross3(s.n, Pb0);
    const float k2 = 2.0f * mu * s.inv * s.inv * FP;
    const float lj = lam * JP;
    const float3 Fb0 = s.ca * Pb0 + k2 * s.F0 + lj * s.dJ0 + s.cb * HJ0;
    const float3 Fb1 = s.ca * Pb1 + k2 * s.F1 + lj * s.dJ1 + s.cb * HJ1;
    xb1 = Fb0 * a.x + Fb1 * a.y;
    xb2 = Fb0 * a.z + Fb1 * a.w;
    xb0 = -(xb1 + xb2);
    gmu = MP;
    glam = s.cm * JP;
    gact = -lam * JP;
}

// ---------------------------------------------------------------------------
// hinge (x1, x2 wing tips; x3 -> x4 edge); p = (kb, act)
// ---------------------------------------------------------------------------
struct HingeState {
    float3 E, A1, B1, A2, B2, N1, N2, Eh, n1, n2, cr, g1, g2;
    float lE2, l1s, l2s, lE, l1, l2, sy, cx, phi, q, sn, cs, p14, p24, p13, p23;
    bool ok;
};

// Hinge edge vectors from the rest differences R1 = X1 - X3, R2 = X2 - X3,
// R4 = X4 - X3 (precomputed in FP64) plus displacement differences.
__device__ __forceinline__ void hinge_state(float3 u1, float3 u2, float3 u3, float3 u4, float3 R1, float3 R2,
                                            float3 R4, float act, HingeState& s) {
    s.E = R4 + (u4 - u3);
    s.A1 = R1 + (u1 - u3);
    s.B1 = (R1 - R4) + (u1 - u4);
    s.A2 = (R2 - R4) + (u2 - u4);
    s.B2 = R2 + (u2 - u3);
    s.N1 = cross3(s.A1, s.B1);
    s.N2 = cross3(s.A2, s.B2);
    s.lE2 = dot3(s.E, s.E);
    s.l1s = dot3(s.N1, s.N1);
    s.l2s = dot3(s.N2, s.N2);
    const float tiny = 1e-24f * s.lE2 * s.lE2;
    s.ok = s.lE2 > 0.0f && s.l1s > tiny && s.l2s > tiny;
    if (!s.ok) return;
    s.lE = sqrtf(s.lE2);
    s.l1 = sqrtf(s.l1s);
    s.l2 = sqrtf(s.l2s);
    s.Eh = s.E * (1.0f / s.lE);
    s.n1 = s.N1 * (1.0f / s.l1);
    s.n2 = s.N2 * (1.0f / s.l2);
    s.cr = cross3(s.n1, s.n2);
    s.sy = dot3(s.cr, s.Eh);
    s.cx = dot3(s.n1, s.n2);
    s.phi = atan2f(s.sy, s.cx);
    s.g1 = s.N1 * (1.0f / s.l1s);
    s.g2 = s.N2 * (1.0f / s.l2s);
    s.p14 = dot3(s.B1, s.Eh);
    s.p24 = dot3(s.A2, s.Eh);
    s.p13 = dot3(s.A1, s.Eh);
    s.p23 = dot3(s.B2, s.Eh);
    s.q = s.lE2 / (s.l1 + s.l2);
    const float ang = 0.5f * s.phi + act;
    s.sn = sinf(ang);
    s.cs = cosf(ang);
}

__device__ __forceinline__ void hinge_forces(const HingeState& s, float kb, float3& f1, float3& f2, float3& f3,
                                             float3& f4) {
    if (!s.ok) {
        f1 = f2 = f3 = f4 = make_float3(0.f, 0.f, 0.f);
        return;
    }
    const float sc = kb * s.q * s.sn;
    f1 = sc * (s.lE * s.g1);
    f2 = sc * (s.lE * s.g2);
    f3 = sc * (s.p14 * s.g1 + s.p24 * s.g2);
    f4 = sc * (-(s.p13 * s.g1) - s.p23 * s.g2);
}

// Reverse mode of hinge_forces, statement by statement.
__device__ __forceinline__ void hinge_adjoint(const HingeState& s, float kb, float3 fb1, float3 fb2, float3 fb3,
                                              float3 fb4, float3& xb1, float3& xb2, float3& xb3, float3& xb4,
                                              float& gkb, float& gact) {
    const float3 z = make_float3(0.f, 0.f, 0.f);
    if (!s.ok) {
        xb1 = xb2 = xb3 = xb4 = z;
        gkb = gact = 0.f;
        return;
    }
    const float sc = kb * s.q * s.sn;
    // u_i and the scale s
    const float3 u1 = s.lE * s.g1, u2 = s.lE * s.g2;
    const float3 u3 = s.p14 * s.g1 + s.p24 * s.g2;
    const float3 u4 = -(s.p13 * s.g1) - s.p23 * s.g2;
    const float scb = dot3(fb1, u1) + dot3(fb2, u2) + dot3(fb3, u3) + dot3(fb4, u4);
    const float3 ub1 = sc * fb1, ub2 = sc * fb2, ub3 = sc * fb3, ub4 = sc * fb4;
    float lEb = dot3(ub1, s.g1) + dot3(ub2, s.g2);
    float3 gb1 = s.lE * ub1 + s.p14 * ub3 - s.p13 * ub4;
    float3 gb2 = s.lE * ub2 + s.p24 * ub3 - s.p23 * ub4;
    const float p14b = dot3(ub3, s.g1), p24b = dot3(ub3, s.g2);
    const float p13b = -dot3(ub4, s.g1), p23b = -dot3(ub4, s.g2);
    // s = kb q sin(phi/2 + act)
    gkb = s.q * s.sn * scb;
    const float qb = kb * s.sn * scb;
    const float snb = kb * s.q * scb;
    const float phib = 0.5f * s.cs * snb;
    gact = s.cs * snb;
    const float l12 = s.l1 + s.l2;
    float lE2b = qb / l12;
    float l1b = -qb * s.lE2 / (l12 * l12);
    float l2b = l1b;
    // projections onto Eh
    float3 B1b = p14b * s.Eh, A2b = p24b * s.Eh, A1b = p13b * s.Eh, B2b = p23b * s.Eh;
    float3 Ehb = p14b * s.B1 + p24b * s.A2 + p13b * s.A1 + p23b * s.B2;
    // g = N / |N|^2
    float3 N1b = gb1 * (1.0f / s.l1s), N2b = gb2 * (1.0f / s.l2s);
    float l1sb = -dot3(gb1, s.N1) / (s.l1s * s.l1s);
    float l2sb = -dot3(gb2, s.N2) / (s.l2s * s.l2s);
    // phi = atan2(sy, cx)
    const float r2 = s.sy * s.sy + s.cx * s.cx;
    const float syb = phib * s.cx / r2, cxb = -phib * s.sy / r2;
    const float3 crb = syb * s.Eh;
    Ehb += syb * s.cr;
    float3 n1b = cxb * s.n2 + cross3(s.n2, crb);
    float3 n2b = cxb * s.n1 + cross3(crb, s.n1);
    // n = N / |N|
    N1b += n1b * (1.0f / s.l1);
    l1b += -dot3(n1b, s.N1) / (s.l1 * s.l1);
    N2b += n2b * (1.0f / s.l2);
    l2b += -dot3(n2b, s.N2) / (s.l2 * s.l2);
    // Eh = E / |E|
    float3 Eb = Ehb * (1.0f / s.lE);
    lEb += -dot3(Ehb, s.E) / s.lE2;
    // square roots and squared norms
    lE2b += lEb / (2.0f * s.lE);
    l1sb += l1b / (2.0f * s.l1);
    l2sb += l2b / (2.0f * s.l2);
    Eb += (2.0f * lE2b) * s.E;
    N1b += (2.0f * l1sb) * s.N1;
    N2b += (2.0f * l2sb) * s.N2;
    // N1 = A1 x B1, N2 = A2 x B2
    A1b += cross3(s.B1, N1b);
    B1b += cross3(N1b, s.A1);
    A2b += cross3(s.B2, N2b);
    B2b += cross3(N2b, s.A2);
    // A1 = x1 - x3, B1 = x1 - x4, A2 = x2 - x4, B2 = x2 - x3, E = x4 - x3
    xb1 = A1b + B1b;
    xb2 = A2b + B2b;
    xb3 = -(A1b + B2b + Eb);
    xb4 = Eb - B1b - A2b;
}

// ---------------------------------------------------------------------------
// contact
// ---------------------------------------------------------------------------
struct ContactParams {
    float ke, kd, kf, mu_f;
};

// one contact with outward normal n and penetration C > 0
__device__ __forceinline__ float3 contact_one(float3 v, float3 n, float C, const ContactParams& cp) {
    const float vn = dot3(v, n);
    const float fn = cp.ke * C - cp.kd * vn;
    float3 f = fn * n;
    const float3 vs = v - vn * n;
    const float vsl = sqrtf(dot3(vs, vs));
    const float afn = fabsf(fn);
    if (cp.kf * vsl <= cp.mu_f * afn) {
        f -= cp.kf * vs;
    } else {
        f -= (cp.mu_f * afn / vsl) * vs;
    }
    return f;
}

// Reverse mode of contact_one for a fixed normal (plane) or a normal that
// depends on x (sphere: handled by the caller through nb / Cb).
__device__ __forceinline__ void contact_one_adjoint(float3 v, float3 n, float C, const ContactParams& cp,
                                                    float3 fb, float3& vb, float3& nb, float& Cb, float3& f) {
    const float vn = dot3(v, n);
    const float fn = cp.ke * C - cp.kd * vn;
    const float3 vs = v - vn * n;
    const float vsl = sqrtf(dot3(vs, vs));
    const float afn = fabsf(fn);
    f = fn * n;
    // f = fn n
    nb = fn * fb;
    float fnb = dot3(fb, n);
    float3 vsb;
    if (cp.kf * vsl <= cp.mu_f * afn) {
        f -= cp.kf * vs;
        vsb = -cp.kf * fb;
    } else {
        const float k = cp.mu_f * afn / vsl;
        f -= k * vs;
        const float kb = -dot3(fb, vs);
        vsb = -k * fb - (kb * k / (vsl * vsl)) * vs;
        const float afnb = kb * cp.mu_f / vsl;
        fnb += fn > 0.0f ? afnb : (fn < 0.0f ? -afnb : 0.0f);
    }
    // vs = v - vn n
    vb = vsb;
    float vnb = -dot3(vsb, n);
    nb -= vn * vsb;
    // fn = ke C - kd vn
    Cb = cp.ke * fnb;
    vnb -= cp.kd * fnb;
    // vn = v . n
    vb += vnb * n;
    nb += vnb * v;
}

// ---------------------------------------------------------------------------
// Air on a triangle (App. A.1: a lift/drag model of the surrounding air on
// the cloth surface; no formula is given).  Flat-plate reading, with N the
// deformed vector area (|N| = A) and v_r the triangle's mean velocity minus
// the wind, s = N . v_r:
//   drag  F_D = -k_D |s| v_r
//   lift  F_L = -k_L s / (A |v_r|) (|v_r|^2 N - s v_r)   (0 when v_r = 0 or A = 0)
// F is the whole triangle's force; each corner takes F/3.
// ---------------------------------------------------------------------------
__device__ __forceinline__ float3 air_force(float3 N, float3 vr, float kd, float kl) {
    const float s = dot3(N, vr);
    float3 F = (-kd * fabsf(s)) * vr;
    const float q = dot3(vr, vr), A2 = dot3(N, N);
    if (kl != 0.0f && q > 0.0f && A2 > 0.0f) {
        const float c = kl * s / (sqrtf(A2) * sqrtf(q));
        F -= c * (q * N - s * vr);
    }
    return F;
}

// reverse of air_force: yb = dL/dF; adds dL/dN and dL/dv_r
__device__ __forceinline__ void air_adjoint(float3 N, float3 vr, float kd, float kl, float3 yb, float3& Nb,
                                            float3& vrb) {
    const float s = dot3(N, vr);
    const float yv = dot3(yb, vr);
    // drag: yb . F_D = -k_D |s| (yb . v_r)
    const float sg = s < 0.0f ? -1.0f : 1.0f;
    vrb += (-kd) * ((sg * yv) * N + fabsf(s) * yb);
    Nb += (-kd * sg * yv) * vr;
    const float q = dot3(vr, vr), A2 = dot3(N, N);
    if (kl != 0.0f && q > 0.0f && A2 > 0.0f) {
        // yb . F_L = -phi psi,  phi = k_L s / (A r),  psi = q (yb . N) - s (yb . v_r)
        const float A = sqrtf(A2), r = sqrtf(q);
        const float iAr = 1.0f / (A * r);
        const float phi = kl * s * iAr;
        const float yN = dot3(yb, N);
        const float psi = q * yN - s * yv;
        const float3 dphi_dv = (kl * iAr) * (N - (s / q) * vr);
        const float3 dphi_dN = (kl * iAr) * (vr - (s / A2) * N);
        const float3 dpsi_dv = (2.0f * yN) * vr - yv * N - s * yb;
        const float3 dpsi_dN = q * yb - yv * vr;
        vrb -= psi * dphi_dv + phi * dpsi_dv;
        Nb -= psi * dphi_dN + phi * dpsi_dN;
    }
}

}  // namespace gs
