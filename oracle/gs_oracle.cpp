// FP64 CPU oracle of the gradSim explicit step and its discrete adjoint.
//
// TEST INFRASTRUCTURE ONLY (see gs_oracle.h): used by tests, by the package
// smoke check and by the benchmark's CPU-baseline leg; never by the library.
//
// Layout of this file, in the order the method is described:
//   1. dual numbers (exact forward-mode derivatives; no hand derivation)
//   2. rest-state set-up: Dm^-1, volume / area, lumped masses
//   3. element physics: neo-Hookean tet, membrane triangle, air on a triangle,
//      dihedral bending
//   4. contact and friction
//   5. the semi-implicit Euler step and the rollout
//   6. the discrete adjoint of App. B and the loss
//   7. forward-mode rollout (for checking the adjoint)

#include "gs_oracle.h"

#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#ifdef _OPENMP
#include <omp.h>
#endif

namespace {

// ---------------------------------------------------------------------------
// 1. dual numbers: value + K directional derivatives
// ---------------------------------------------------------------------------
template <int K>
struct Dual {
    double v;
    double d[K];
    Dual() : v(0.0) { for (int i = 0; i < K; ++i) d[i] = 0.0; }
    Dual(double x) : v(x) { for (int i = 0; i < K; ++i) d[i] = 0.0; }  // NOLINT: implicit on purpose
};

template <int K> Dual<K> operator+(const Dual<K>& a, const Dual<K>& b) {
    Dual<K> r; r.v = a.v + b.v; for (int i = 0; i < K; ++i) r.d[i] = a.d[i] + b.d[i]; return r;
}
template <int K> Dual<K> operator-(const Dual<K>& a, const Dual<K>& b) {
    Dual<K> r; r.v = a.v - b.v; for (int i = 0; i < K; ++i) r.d[i] = a.d[i] - b.d[i]; return r;
}
template <int K> Dual<K> operator-(const Dual<K>& a) {
    Dual<K> r; r.v = -a.v; for (int i = 0; i < K; ++i) r.d[i] = -a.d[i]; return r;
}
template <int K> Dual<K> operator*(const Dual<K>& a, const Dual<K>& b) {
    Dual<K> r; r.v = a.v * b.v; for (int i = 0; i < K; ++i) r.d[i] = a.d[i] * b.v + a.v * b.d[i]; return r;
}
template <int K> Dual<K> operator/(const Dual<K>& a, const Dual<K>& b) {
    Dual<K> r; r.v = a.v / b.v;
    for (int i = 0; i < K; ++i) r.d[i] = (a.d[i] * b.v - a.v * b.d[i]) / (b.v * b.v);
    return r;
}
template <int K> Dual<K> operator+(const Dual<K>& a, double b) { return a + Dual<K>(b); }
template <int K> Dual<K> operator+(double a, const Dual<K>& b) { return Dual<K>(a) + b; }
template <int K> Dual<K> operator-(const Dual<K>& a, double b) { return a - Dual<K>(b); }
template <int K> Dual<K> operator-(double a, const Dual<K>& b) { return Dual<K>(a) - b; }
template <int K> Dual<K> operator*(const Dual<K>& a, double b) { return a * Dual<K>(b); }
template <int K> Dual<K> operator*(double a, const Dual<K>& b) { return Dual<K>(a) * b; }
template <int K> Dual<K> operator/(const Dual<K>& a, double b) { return a / Dual<K>(b); }
template <int K> Dual<K> operator/(double a, const Dual<K>& b) { return Dual<K>(a) / b; }
template <int K> Dual<K>& operator+=(Dual<K>& a, const Dual<K>& b) { a = a + b; return a; }
template <int K> Dual<K>& operator-=(Dual<K>& a, const Dual<K>& b) { a = a - b; return a; }

inline double val(double x) { return x; }
template <int K> double val(const Dual<K>& x) { return x.v; }

inline double fsqrt(double x) { return std::sqrt(x); }
inline double flog(double x) { return std::log(x); }
inline double fsin(double x) { return std::sin(x); }
inline double fcos(double x) { return std::cos(x); }
inline double fabs_(double x) { return std::fabs(x); }
inline double fatan2(double y, double x) { return std::atan2(y, x); }

template <int K> Dual<K> fsqrt(const Dual<K>& a) {
    Dual<K> r; r.v = std::sqrt(a.v); for (int i = 0; i < K; ++i) r.d[i] = a.d[i] / (2.0 * r.v); return r;
}
template <int K> Dual<K> flog(const Dual<K>& a) {
    Dual<K> r; r.v = std::log(a.v); for (int i = 0; i < K; ++i) r.d[i] = a.d[i] / a.v; return r;
}
template <int K> Dual<K> fsin(const Dual<K>& a) {
    Dual<K> r; r.v = std::sin(a.v); const double c = std::cos(a.v);
    for (int i = 0; i < K; ++i) r.d[i] = c * a.d[i];
    return r;
}
template <int K> Dual<K> fcos(const Dual<K>& a) {
    Dual<K> r; r.v = std::cos(a.v); const double s = -std::sin(a.v);
    for (int i = 0; i < K; ++i) r.d[i] = s * a.d[i];
    return r;
}
template <int K> Dual<K> fabs_(const Dual<K>& a) { return a.v < 0.0 ? -a : a; }
template <int K> Dual<K> fatan2(const Dual<K>& y, const Dual<K>& x) {
    Dual<K> r; r.v = std::atan2(y.v, x.v); const double q = x.v * x.v + y.v * y.v;
    for (int i = 0; i < K; ++i) r.d[i] = (x.v * y.d[i] - y.v * x.d[i]) / q;
    return r;
}

// small vector helpers on T[3]
template <class T> void vsub(const T* a, const T* b, T* r) { for (int i = 0; i < 3; ++i) r[i] = a[i] - b[i]; }
template <class T> T vdot(const T* a, const T* b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }
template <class T> void vcross(const T* a, const T* b, T* r) {
    r[0] = a[1] * b[2] - a[2] * b[1];
    r[1] = a[2] * b[0] - a[0] * b[2];
    r[2] = a[0] * b[1] - a[1] * b[0];
}

// ---------------------------------------------------------------------------
// 2. rest state
// ---------------------------------------------------------------------------
// Constant-strain tet (App. A.1, App. C.1): Dm = [X1-X0, X2-X0, X3-X0],
// V = det(Dm)/6, Dm^-1 = adj(Dm)/det(Dm).  Row-major 3x3.
void tet_rest(const double* X, double* Dminv, double* V) {
    double Dm[3][3];
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) Dm[r][c] = X[3 * (c + 1) + r] - X[r];
    double cof[3][3];
    cof[0][0] = Dm[1][1] * Dm[2][2] - Dm[1][2] * Dm[2][1];
    cof[0][1] = Dm[1][2] * Dm[2][0] - Dm[1][0] * Dm[2][2];
    cof[0][2] = Dm[1][0] * Dm[2][1] - Dm[1][1] * Dm[2][0];
    cof[1][0] = Dm[0][2] * Dm[2][1] - Dm[0][1] * Dm[2][2];
    cof[1][1] = Dm[0][0] * Dm[2][2] - Dm[0][2] * Dm[2][0];
    cof[1][2] = Dm[0][1] * Dm[2][0] - Dm[0][0] * Dm[2][1];
    cof[2][0] = Dm[0][1] * Dm[1][2] - Dm[0][2] * Dm[1][1];
    cof[2][1] = Dm[0][2] * Dm[1][0] - Dm[0][0] * Dm[1][2];
    cof[2][2] = Dm[0][0] * Dm[1][1] - Dm[0][1] * Dm[1][0];
    const double det = Dm[0][0] * cof[0][0] + Dm[0][1] * cof[0][1] + Dm[0][2] * cof[0][2];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) Dminv[3 * i + j] = cof[j][i] / det;
    *V = det / 6.0;
}

// Constant-strain triangle embedded in 3D: rest edges in an orthonormal
// in-plane frame (t1 along X1-X0), Dm 2x2, area A = |(X1-X0) x (X2-X0)|/2.
void tri_rest(const double* X, double* Dminv, double* A) {
    double e1[3], e2[3], nrm[3], t1[3], t2[3];
    vsub(X + 3, X, e1);
    vsub(X + 6, X, e2);
    vcross(e1, e2, nrm);
    const double ln = std::sqrt(vdot(nrm, nrm));
    const double l1 = std::sqrt(vdot(e1, e1));
    for (int i = 0; i < 3; ++i) { t1[i] = e1[i] / l1; nrm[i] /= ln; }
    vcross(nrm, t1, t2);
    const double a = vdot(e1, t1), b = vdot(e2, t1), c = vdot(e1, t2), d = vdot(e2, t2);
    const double det = a * d - b * c;
    Dminv[0] = d / det;  Dminv[1] = -b / det;
    Dminv[2] = -c / det; Dminv[3] = a / det;
    *A = 0.5 * ln;
}

struct Rest {
    std::vector<double> tet_Dminv, tet_V, tri_Dminv, tri_A;
};

Rest make_rest(const orc_model* m) {
    Rest r;
    r.tet_Dminv.resize(9 * (size_t)m->n_tets);
    r.tet_V.resize(m->n_tets);
    for (int e = 0; e < m->n_tets; ++e) {
        double X[12];
        for (int c = 0; c < 4; ++c)
            for (int k = 0; k < 3; ++k) X[3 * c + k] = m->X[3 * m->tets[4 * e + c] + k];
        tet_rest(X, &r.tet_Dminv[9 * (size_t)e], &r.tet_V[e]);
    }
    r.tri_Dminv.resize(4 * (size_t)m->n_tris);
    r.tri_A.resize(m->n_tris);
    for (int t = 0; t < m->n_tris; ++t) {
        double X[9];
        for (int c = 0; c < 3; ++c)
            for (int k = 0; k < 3; ++k) X[3 * c + k] = m->X[3 * m->tris[3 * t + c] + k];
        tri_rest(X, &r.tri_Dminv[4 * (size_t)t], &r.tri_A[t]);
    }
    return r;
}

// Lumped mass (equal split of each element's mass among its corners):
// m_i = sum_tets rho_e V_e / 4 + sum_tris rho_t A_t / 3.
template <class T>
void node_masses(const orc_model* m, const Rest& r, const T* tet_rho, const T* tri_rho, T* mass) {
    for (int i = 0; i < m->n_nodes; ++i) mass[i] = T(0.0);
    for (int e = 0; e < m->n_tets; ++e)
        for (int c = 0; c < 4; ++c) mass[m->tets[4 * e + c]] += tet_rho[e] * (r.tet_V[e] / 4.0);
    for (int t = 0; t < m->n_tris; ++t)
        for (int c = 0; c < 3; ++c) mass[m->tris[3 * t + c]] += tri_rho[t] * (r.tri_A[t] / 3.0);
}

// ---------------------------------------------------------------------------
// 3. element physics
// ---------------------------------------------------------------------------
// Stable neo-Hookean tet, App. A.1 / C.1.  Reading: the energy's alpha is the
// rest-stable target 1 + 3 mu / (4 lambda) plus the element's actuation, so
// that the element carries no force at F = I when act = 0.
//   F = Ds Dm^-1, I_C = |F|_F^2, J = det F,
//   P = dPsi/dF = mu F (1 - 1/(I_C + 1)) + lambda (J - alpha) cof F,
//   f_{1,2,3} = columns of -V P Dm^-T, f_0 = -(f_1 + f_2 + f_3).
template <class T>
void tet_F(const T* x, const double* Dminv, T F[3][3]) {
    T Ds[3][3];
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) Ds[r][c] = x[3 * (c + 1) + r] - x[r];
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c)
            F[r][c] = Ds[r][0] * Dminv[c] + Ds[r][1] * Dminv[3 + c] + Ds[r][2] * Dminv[6 + c];
}

template <class T>
void cofactor(const T F[3][3], T cof[3][3]) {
    cof[0][0] = F[1][1] * F[2][2] - F[1][2] * F[2][1];
    cof[0][1] = F[1][2] * F[2][0] - F[1][0] * F[2][2];
    cof[0][2] = F[1][0] * F[2][1] - F[1][1] * F[2][0];
    cof[1][0] = F[0][2] * F[2][1] - F[0][1] * F[2][2];
    cof[1][1] = F[0][0] * F[2][2] - F[0][2] * F[2][0];
    cof[1][2] = F[0][1] * F[2][0] - F[0][0] * F[2][1];
    cof[2][0] = F[0][1] * F[1][2] - F[0][2] * F[1][1];
    cof[2][1] = F[0][2] * F[1][0] - F[0][0] * F[1][2];
    cof[2][2] = F[0][0] * F[1][1] - F[0][1] * F[1][0];
}

template <class T>
void tet_forces_t(const T* x, const double* Dminv, double V, T mu, T lam, T act, T* f) {
    T F[3][3], cof[3][3];
    tet_F(x, Dminv, F);
    cofactor(F, cof);
    T Ic(0.0);
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) Ic += F[r][c] * F[r][c];
    const T J = F[0][0] * cof[0][0] + F[0][1] * cof[0][1] + F[0][2] * cof[0][2];
    const T alpha = 1.0 + 0.75 * mu / lam + act;
    const T a = mu * (1.0 - 1.0 / (Ic + 1.0));
    const T b = lam * (J - alpha);
    T P[3][3];
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) P[r][c] = a * F[r][c] + b * cof[r][c];
    for (int k = 0; k < 3; ++k) f[k] = T(0.0);
    for (int c = 0; c < 3; ++c)
        for (int r = 0; r < 3; ++r) {
            const T h = -V * (P[r][0] * Dminv[3 * c] + P[r][1] * Dminv[3 * c + 1] + P[r][2] * Dminv[3 * c + 2]);
            f[3 * (c + 1) + r] = h;
            f[r] -= h;
        }
}

template <class T>
T tet_energy_t(const T* x, const double* Dminv, double V, T mu, T lam, T act) {
    T F[3][3], cof[3][3];
    tet_F(x, Dminv, F);
    cofactor(F, cof);
    T Ic(0.0);
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) Ic += F[r][c] * F[r][c];
    const T J = F[0][0] * cof[0][0] + F[0][1] * cof[0][1] + F[0][2] * cof[0][2];
    const T alpha = 1.0 + 0.75 * mu / lam + act;
    return V * (0.5 * mu * (Ic - 3.0) + 0.5 * lam * (J - alpha) * (J - alpha) - 0.5 * mu * flog(Ic + 1.0));
}

// Membrane triangle: same energy in the plane, F is 3x2, I_C = |F|^2 (= 2 at
// rest), J = |f_0 x f_1| (area ratio); rest-stable alpha = 1 + 2 mu / (3 lambda)
// plus actuation.  dJ/df_0 = f_1 x n, dJ/df_1 = n x f_0 with n = (f_0 x f_1)/J.
template <class T>
void tri_F(const T* x, const double* Dminv, T F[3][2]) {
    for (int r = 0; r < 3; ++r) {
        const T d0 = x[3 + r] - x[r], d1 = x[6 + r] - x[r];
        F[r][0] = d0 * Dminv[0] + d1 * Dminv[2];
        F[r][1] = d0 * Dminv[1] + d1 * Dminv[3];
    }
}

template <class T>
void tri_forces_t(const T* x, const double* Dminv, double A, T mu, T lam, T act, T* f) {
    T F[3][2];
    tri_F(x, Dminv, F);
    T f0[3] = {F[0][0], F[1][0], F[2][0]};
    T f1[3] = {F[0][1], F[1][1], F[2][1]};
    const T Ic = vdot(f0, f0) + vdot(f1, f1);
    T c[3];
    vcross(f0, f1, c);
    const T J = fsqrt(vdot(c, c));
    T n[3] = {c[0] / J, c[1] / J, c[2] / J};
    T dJ0[3], dJ1[3];
    vcross(f1, n, dJ0);
    vcross(n, f0, dJ1);
    const T alpha = 1.0 + (2.0 / 3.0) * mu / lam + act;
    const T a = mu * (1.0 - 1.0 / (Ic + 1.0));
    const T b = lam * (J - alpha);
    T P[3][2];
    for (int r = 0; r < 3; ++r) {
        P[r][0] = a * f0[r] + b * dJ0[r];
        P[r][1] = a * f1[r] + b * dJ1[r];
    }
    for (int k = 0; k < 3; ++k) f[k] = T(0.0);
    for (int cc = 0; cc < 2; ++cc)
        for (int r = 0; r < 3; ++r) {
            const T h = -A * (P[r][0] * Dminv[2 * cc] + P[r][1] * Dminv[2 * cc + 1]);
            f[3 * (cc + 1) + r] = h;
            f[r] -= h;
        }
}

template <class T>
T tri_energy_t(const T* x, const double* Dminv, double A, T mu, T lam, T act) {
    T F[3][2];
    tri_F(x, Dminv, F);
    T f0[3] = {F[0][0], F[1][0], F[2][0]};
    T f1[3] = {F[0][1], F[1][1], F[2][1]};
    const T Ic = vdot(f0, f0) + vdot(f1, f1);
    T c[3];
    vcross(f0, f1, c);
    const T J = fsqrt(vdot(c, c));
    const T alpha = 1.0 + (2.0 / 3.0) * mu / lam + act;
    return A * (0.5 * mu * (Ic - 2.0) + 0.5 * lam * (J - alpha) * (J - alpha) - 0.5 * mu * flog(Ic + 1.0));
}

// Air on a triangle (App. A.1 "Deformable Thin-Shells" adds lift and drag
// forces from the air around the cloth but prints no formula).  Reading, a
// flat plate in a uniform wind:
//   v_r = (v_0 + v_1 + v_2)/3 - wind        velocity of the plate through the air
//   N   = (x_1 - x_0) x (x_2 - x_0) / 2     vector area, |N| = A, N/A = n
//   s   = N . v_r = A |v_r| cos(theta)
//   drag  F_D = -k_drag |s| v_r              along -v_r, size k_drag A |cos theta| |v_r|^2
//   lift  F_L = -k_lift s/(A |v_r|) (|v_r|^2 N - s v_r)
//             = -k_lift A |v_r|^2 cos(theta) (n - cos(theta) v_r/|v_r|)
//                                            perpendicular to v_r, size k_lift A |v_r|^2 |sin 2 theta|/2
// and each corner takes F/3.  Both terms are unchanged when the winding (the
// sign of n) flips; the lift does no work, the drag only removes energy
// (zero wind).  The lift is taken as 0 when v_r = 0 or A = 0.
template <class T>
void air_forces_t(const T* x, const T* v, double k_drag, double k_lift, const double* wind, T* f) {
    T e1[3], e2[3], N[3], vr[3];
    for (int k = 0; k < 3; ++k) {
        e1[k] = x[3 + k] - x[k];
        e2[k] = x[6 + k] - x[k];
        vr[k] = (v[k] + v[3 + k] + v[6 + k]) / 3.0 - wind[k];
    }
    vcross(e1, e2, N);
    for (int k = 0; k < 3; ++k) N[k] = 0.5 * N[k];
    const T s = vdot(N, vr);
    const T abs_s = val(s) < 0.0 ? -s : s;
    T F[3];
    for (int k = 0; k < 3; ++k) F[k] = -k_drag * abs_s * vr[k];
    const T q = vdot(vr, vr), A2 = vdot(N, N);
    if (k_lift != 0.0 && val(q) > 0.0 && val(A2) > 0.0) {
        const T c = k_lift * s / (fsqrt(A2) * fsqrt(q));
        for (int k = 0; k < 3; ++k) F[k] = F[k] - c * (q * N[k] - s * vr[k]);
    }
    for (int c = 0; c < 3; ++c)
        for (int k = 0; k < 3; ++k) f[3 * c + k] = F[k] / 3.0;
}

// Dihedral angle of a hinge (x1, x2 wing tips; edge x3 -> x4):
// N1 = (x1 - x3) x (x1 - x4), N2 = (x2 - x4) x (x2 - x3), E = x4 - x3,
// phi = atan2((n1 x n2) . E/|E|, n1 . n2)   (0 when flat).
template <class T>
T hinge_angle_t(const T* x) {
    const T *x1 = x, *x2 = x + 3, *x3 = x + 6, *x4 = x + 9;
    T E[3], a[3], b[3], N1[3], N2[3], c[3];
    vsub(x4, x3, E);
    vsub(x1, x3, a); vsub(x1, x4, b); vcross(a, b, N1);
    vsub(x2, x4, a); vsub(x2, x3, b); vcross(a, b, N2);
    const T lE = fsqrt(vdot(E, E)), l1 = fsqrt(vdot(N1, N1)), l2 = fsqrt(vdot(N2, N2));
    T n1[3] = {N1[0] / l1, N1[1] / l1, N1[2] / l1};
    T n2[3] = {N2[0] / l2, N2[1] / l2, N2[2] / l2};
    vcross(n1, n2, c);
    return fatan2(vdot(c, E) / lE, vdot(n1, n2));
}

// Bending (App. A.1): f_b = k_b sin(phi/2 + alpha) d with d from Bridson et
// al.  Reading: Bridson's force in full,
//   f_i = k_b |E|^2 / (|N1| + |N2|) sin(phi/2 + alpha) u_i,
//   u1 = |E| N1/|N1|^2, u2 = |E| N2/|N2|^2,
//   u3 = ((x1-x4).E^) N1/|N1|^2 + ((x2-x4).E^) N2/|N2|^2,
//   u4 = -((x1-x3).E^) N1/|N1|^2 - ((x2-x3).E^) N2/|N2|^2,
// with the u_i equal to -d(phi)/dx_i for the angle above, so the force is
// restoring.  A degenerate hinge (zero edge or zero-area wing) exerts none.
template <class T>
void hinge_forces_t(const T* x, T kb, T act, T* f) {
    const T *x1 = x, *x2 = x + 3, *x3 = x + 6, *x4 = x + 9;
    T E[3], a[3], b[3], N1[3], N2[3], c[3];
    vsub(x4, x3, E);
    vsub(x1, x3, a); vsub(x1, x4, b); vcross(a, b, N1);
    vsub(x2, x4, a); vsub(x2, x3, b); vcross(a, b, N2);
    const T lE2 = vdot(E, E), l1s = vdot(N1, N1), l2s = vdot(N2, N2);
    for (int k = 0; k < 12; ++k) f[k] = T(0.0);
    const double tiny = 1e-24 * val(lE2) * val(lE2);
    if (val(lE2) <= 0.0 || val(l1s) <= tiny || val(l2s) <= tiny) return;
    const T lE = fsqrt(lE2), l1 = fsqrt(l1s), l2 = fsqrt(l2s);
    T Eh[3] = {E[0] / lE, E[1] / lE, E[2] / lE};
    T n1[3] = {N1[0] / l1, N1[1] / l1, N1[2] / l1};
    T n2[3] = {N2[0] / l2, N2[1] / l2, N2[2] / l2};
    vcross(n1, n2, c);
    const T phi = fatan2(vdot(c, Eh), vdot(n1, n2));
    T g1[3], g2[3];
    for (int k = 0; k < 3; ++k) { g1[k] = N1[k] / l1s; g2[k] = N2[k] / l2s; }
    T d14[3], d24[3], d13[3], d23[3];
    vsub(x1, x4, d14); vsub(x2, x4, d24); vsub(x1, x3, d13); vsub(x2, x3, d23);
    const T p14 = vdot(d14, Eh), p24 = vdot(d24, Eh), p13 = vdot(d13, Eh), p23 = vdot(d23, Eh);
    const T s = kb * lE2 / (l1 + l2) * fsin(0.5 * phi + act);
    for (int k = 0; k < 3; ++k) {
        f[k] = s * (lE * g1[k]);
        f[3 + k] = s * (lE * g2[k]);
        f[6 + k] = s * (p14 * g1[k] + p24 * g2[k]);
        f[9 + k] = s * (-(p13 * g1[k]) - p23 * g2[k]);
    }
}

// ---------------------------------------------------------------------------
// 4. contact (App. A.1 "Contact", App. C.2)
// ---------------------------------------------------------------------------
// Readings: C = penetration depth (>= 0) along the outward normal n; the
// normal force restores along n, f_n = n (k_e C + k_d dC/dt) with
// dC/dt = -v.n, applied only while C > 0 (contact distance threshold 0).
// Relaxed Coulomb friction on the sliding velocity v_s = v - (v.n) n:
// f_f = -k_f v_s when k_f |v_s| <= mu |f_n| (stick), else
// f_f = -mu |f_n| v_s / |v_s| (slip); zero when v_s = 0.  The shapes are a
// plane {y : n.y = h} (n unit) and a sphere (centre c, radius r).
template <class T>
void contact_one(const T* v, const double* n, const T& C, const T* nrm_t, bool use_t,
                 T ke, T kd, T kf, T muf, T* f) {
    T nn[3];
    for (int k = 0; k < 3; ++k) nn[k] = use_t ? nrm_t[k] : T(n[k]);
    const T vn = vdot(v, nn);
    const T fn = ke * C - kd * vn;
    T vs[3];
    for (int k = 0; k < 3; ++k) { f[k] += fn * nn[k]; vs[k] = v[k] - vn * nn[k]; }
    const double vsl_val = std::sqrt(val(vs[0]) * val(vs[0]) + val(vs[1]) * val(vs[1]) + val(vs[2]) * val(vs[2]));
    const T afn = fabs_(fn);
    if (val(kf) * vsl_val <= val(muf) * val(afn)) {
        for (int k = 0; k < 3; ++k) f[k] -= kf * vs[k];
    } else {
        const T vsl = fsqrt(vdot(vs, vs));
        const T scale = muf * afn / vsl;
        for (int k = 0; k < 3; ++k) f[k] -= scale * vs[k];
    }
}

template <class T>
void contact_t(const orc_model* m, const T* x, const T* v, T ke, T kd, T kf, T muf, T* f) {
    for (int k = 0; k < 3; ++k) f[k] = T(0.0);
    if (m->plane_on) {
        const T C = m->plane_h - (m->plane_n[0] * x[0] + m->plane_n[1] * x[1] + m->plane_n[2] * x[2]);
        if (val(C) > 0.0) contact_one(v, m->plane_n, C, (const T*)nullptr, false, ke, kd, kf, muf, f);
    }
    if (m->sphere_on) {
        T d[3];
        for (int k = 0; k < 3; ++k) d[k] = x[k] - m->sphere_c[k];
        const double dist_val = std::sqrt(val(d[0]) * val(d[0]) + val(d[1]) * val(d[1]) + val(d[2]) * val(d[2]));
        if (m->sphere_r - dist_val > 0.0 && dist_val > 0.0) {
            const T dist = fsqrt(vdot(d, d));
            const T C = m->sphere_r - dist;
            T nn[3] = {d[0] / dist, d[1] / dist, d[2] / dist};
            contact_one(v, m->sphere_c, C, nn, true, ke, kd, kf, muf, f);
        }
    }
}

// ---------------------------------------------------------------------------
// 5. the step
// ---------------------------------------------------------------------------
// Total force on every node at state (x, v): elements, hinges, then contact
// (each element adds its corner forces to its nodes in element order).
//
// Threads (OpenMP, when the oracle is built with it) only ever split loops
// whose iterations are independent: each element's corner forces go to its
// own rows of a scratch array, and the node sums then run on one thread in
// element order.  The arithmetic and its order are those of the plain
// serial loop, so every result is bitwise the same for any thread count.
template <class T>
std::vector<T>& corner_scratch(size_t n) {
    thread_local std::vector<T> buf;
    if (buf.size() < n) buf.resize(n);
    return buf;
}

template <class T>
void total_force(const orc_model* m, const Rest& r, const T* x, const T* v,
                 const T* tmu, const T* tlam, const T* tact,
                 const T* rmu, const T* rlam, const T* ract,
                 const T* kb, const T* hact, const T* cp, T* f) {
    const size_t N = (size_t)m->n_nodes;
    for (size_t i = 0; i < 3 * N; ++i) f[i] = T(0.0);
    {
        std::vector<T>& fe = corner_scratch<T>(12 * (size_t)m->n_tets);
#pragma omp parallel for schedule(static)
        for (int e = 0; e < m->n_tets; ++e) {
            T xe[12];
            for (int c = 0; c < 4; ++c)
                for (int k = 0; k < 3; ++k) xe[3 * c + k] = x[3 * (size_t)m->tets[4 * e + c] + k];
            tet_forces_t(xe, &r.tet_Dminv[9 * (size_t)e], r.tet_V[e], tmu[e], tlam[e], tact[e], &fe[12 * (size_t)e]);
        }
        for (int e = 0; e < m->n_tets; ++e)
            for (int c = 0; c < 4; ++c)
                for (int k = 0; k < 3; ++k) f[3 * (size_t)m->tets[4 * e + c] + k] += fe[12 * (size_t)e + 3 * c + k];
    }
    {
        std::vector<T>& fe = corner_scratch<T>(9 * (size_t)m->n_tris);
#pragma omp parallel for schedule(static)
        for (int t = 0; t < m->n_tris; ++t) {
            T xe[9];
            for (int c = 0; c < 3; ++c)
                for (int k = 0; k < 3; ++k) xe[3 * c + k] = x[3 * (size_t)m->tris[3 * t + c] + k];
            tri_forces_t(xe, &r.tri_Dminv[4 * (size_t)t], r.tri_A[t], rmu[t], rlam[t], ract[t], &fe[9 * (size_t)t]);
        }
        for (int t = 0; t < m->n_tris; ++t)
            for (int c = 0; c < 3; ++c)
                for (int k = 0; k < 3; ++k) f[3 * (size_t)m->tris[3 * t + c] + k] += fe[9 * (size_t)t + 3 * c + k];
    }
    if (m->air_on) {
        std::vector<T>& fe = corner_scratch<T>(9 * (size_t)m->n_tris);
#pragma omp parallel for schedule(static)
        for (int t = 0; t < m->n_tris; ++t) {
            T xe[9], ve[9];
            for (int c = 0; c < 3; ++c)
                for (int k = 0; k < 3; ++k) {
                    xe[3 * c + k] = x[3 * (size_t)m->tris[3 * t + c] + k];
                    ve[3 * c + k] = v[3 * (size_t)m->tris[3 * t + c] + k];
                }
            air_forces_t(xe, ve, m->k_drag, m->k_lift, m->wind, &fe[9 * (size_t)t]);
        }
        for (int t = 0; t < m->n_tris; ++t)
            for (int c = 0; c < 3; ++c)
                for (int k = 0; k < 3; ++k) f[3 * (size_t)m->tris[3 * t + c] + k] += fe[9 * (size_t)t + 3 * c + k];
    }
    {
        std::vector<T>& fe = corner_scratch<T>(12 * (size_t)m->n_hinges);
#pragma omp parallel for schedule(static)
        for (int h = 0; h < m->n_hinges; ++h) {
            T xe[12];
            for (int c = 0; c < 4; ++c)
                for (int k = 0; k < 3; ++k) xe[3 * c + k] = x[3 * (size_t)m->hinges[4 * h + c] + k];
            hinge_forces_t(xe, kb[h], hact[h], &fe[12 * (size_t)h]);
        }
        for (int h = 0; h < m->n_hinges; ++h)
            for (int c = 0; c < 4; ++c)
                for (int k = 0; k < 3; ++k) f[3 * (size_t)m->hinges[4 * h + c] + k] += fe[12 * (size_t)h + 3 * c + k];
    }
    if (m->plane_on || m->sphere_on) {
        // one node per iteration, adding to that node's own rows only
#pragma omp parallel for schedule(static)
        for (long long i = 0; i < (long long)N; ++i) {
            T fc[3];
            contact_t(m, x + 3 * i, v + 3 * i, cp[0], cp[1], cp[2], cp[3], fc);
            for (int k = 0; k < 3; ++k) f[3 * i + k] += fc[k];
        }
    }
}

// All inputs of the step in scalar type T (double, or dual numbers for the
// forward-mode check).
template <class T>
struct Inputs {
    std::vector<T> tmu, tlam, tact, trho, rmu, rlam, ract, rrho, kb, hact, cp;
    std::vector<T> tseq, rseq, hseq;  // per-step actuation rows (empty if none)
    int n_seq = 0;
    void load(const orc_model* m, const orc_dirs* d);
    // actuation in effect during step n: static value + row n of the sequence
    void step_act(const orc_model* m, int n, std::vector<T>& ta, std::vector<T>& ra, std::vector<T>& ha) const;
};

template <class T> void seed(T& t, double v, const double* dir, int i) { (void)dir; (void)i; t = T(v); }
template <> void seed<Dual<1>>(Dual<1>& t, double v, const double* dir, int i) {
    t = Dual<1>(v);
    if (dir) t.d[0] = dir[i];
}

template <class T>
void Inputs<T>::load(const orc_model* m, const orc_dirs* d) {
    auto fill = [&](std::vector<T>& out, int n, const double* src, double dflt, const double* dir) {
        out.resize(n);
        for (int i = 0; i < n; ++i) seed<T>(out[i], src ? src[i] : dflt, dir, i);
    };
    fill(tmu, m->n_tets, m->tet_mu, 0.0, d ? d->tet_mu : nullptr);
    fill(tlam, m->n_tets, m->tet_lam, 0.0, d ? d->tet_lam : nullptr);
    fill(tact, m->n_tets, m->tet_act, 0.0, d ? d->tet_act : nullptr);
    fill(trho, m->n_tets, m->tet_rho, 0.0, d ? d->tet_rho : nullptr);
    fill(rmu, m->n_tris, m->tri_mu, 0.0, d ? d->tri_mu : nullptr);
    fill(rlam, m->n_tris, m->tri_lam, 0.0, d ? d->tri_lam : nullptr);
    fill(ract, m->n_tris, m->tri_act, 0.0, d ? d->tri_act : nullptr);
    fill(rrho, m->n_tris, m->tri_rho, 0.0, d ? d->tri_rho : nullptr);
    fill(kb, m->n_hinges, m->hinge_kb, 0.0, d ? d->hinge_kb : nullptr);
    fill(hact, m->n_hinges, m->hinge_act, 0.0, d ? d->hinge_act : nullptr);
    const double c4[4] = {m->ke, m->kd, m->kf, m->mu_f};
    fill(cp, 4, c4, 0.0, d ? d->contact : nullptr);
    n_seq = m->n_act_steps > 0 ? m->n_act_steps : 0;
    if (n_seq && m->tet_act_seq) fill(tseq, n_seq * m->n_tets, m->tet_act_seq, 0.0, d ? d->tet_act_seq : nullptr);
    if (n_seq && m->tri_act_seq) fill(rseq, n_seq * m->n_tris, m->tri_act_seq, 0.0, d ? d->tri_act_seq : nullptr);
    if (n_seq && m->hinge_act_seq)
        fill(hseq, n_seq * m->n_hinges, m->hinge_act_seq, 0.0, d ? d->hinge_act_seq : nullptr);
}

template <class T>
void Inputs<T>::step_act(const orc_model* m, int n, std::vector<T>& ta, std::vector<T>& ra,
                         std::vector<T>& ha) const {
    ta = tact;
    ra = ract;
    ha = hact;
    if (n >= n_seq) return;
    if (!tseq.empty()) for (int e = 0; e < m->n_tets; ++e) ta[e] += tseq[(size_t)n * m->n_tets + e];
    if (!rseq.empty()) for (int t = 0; t < m->n_tris; ++t) ra[t] += rseq[(size_t)n * m->n_tris + t];
    if (!hseq.empty()) for (int h = 0; h < m->n_hinges; ++h) ha[h] += hseq[(size_t)n * m->n_hinges + h];
}

// Inverse masses w_i = 1/m_i; pinned nodes (and nodes without mass) are
// kinematic with w_i = 0.
template <class T>
void inverse_masses(const orc_model* m, const Rest& r, const Inputs<T>& in, std::vector<T>& w,
                    std::vector<T>& mass) {
    mass.assign(m->n_nodes, T(0.0));
    node_masses(m, r, in.trho.data(), in.rrho.data(), mass.data());
    w.assign(m->n_nodes, T(0.0));
    for (int i = 0; i < m->n_nodes; ++i) {
        const bool pin = m->pinned && m->pinned[i];
        if (!pin && val(mass[i]) > 0.0) w[i] = 1.0 / mass[i];
    }
}

// Semi-implicit Euler (App. B):  v+ = v + dt (w f + g [w > 0]),  x+ = x + dt v+.
// Reading of the listing's gravity term: gravity accelerates every node with
// w > 0 and leaves kinematic nodes alone; forces are all taken at s-.
template <class T>
void step(const orc_model* m, const Rest& r, const Inputs<T>& in, const std::vector<T>& w,
          double dt, int n, std::vector<T>& x, std::vector<T>& v, std::vector<T>& f) {
    std::vector<T> ta, ra, ha;
    in.step_act(m, n, ta, ra, ha);
    total_force(m, r, x.data(), v.data(), in.tmu.data(), in.tlam.data(), ta.data(),
                in.rmu.data(), in.rlam.data(), ra.data(), in.kb.data(), ha.data(),
                in.cp.data(), f.data());
    for (int i = 0; i < m->n_nodes; ++i) {
        const bool dyn = val(w[i]) > 0.0;
        for (int k = 0; k < 3; ++k) {
            v[3 * (size_t)i + k] = v[3 * (size_t)i + k] + dt * (w[i] * f[3 * (size_t)i + k] + (dyn ? m->gravity[k] : 0.0));
            x[3 * (size_t)i + k] = x[3 * (size_t)i + k] + dt * v[3 * (size_t)i + k];
        }
    }
}

// ---------------------------------------------------------------------------
// 6. discrete adjoint (App. B)
// ---------------------------------------------------------------------------
// Accumulate J^T y for one element whose force routine takes NX corner
// coordinates and NP parameters, with J the exact Jacobian from Dual<NX+NP>.
template <int NX, int NP, class Fn>
void element_vjp(const double* xe, const double* pe, const double* y, double* xbar, double* pbar, Fn fn) {
    constexpr int K = NX + NP;
    Dual<K> xd[NX], pd[NP > 0 ? NP : 1], fd[NX];
    for (int i = 0; i < NX; ++i) { xd[i] = Dual<K>(xe[i]); xd[i].d[i] = 1.0; }
    for (int j = 0; j < NP; ++j) { pd[j] = Dual<K>(pe[j]); pd[j].d[NX + j] = 1.0; }
    fn(xd, pd, fd);
    for (int k = 0; k < K; ++k) {
        double s = 0.0;
        for (int i = 0; i < NX; ++i) s += y[i] * fd[i].d[k];
        if (k < NX) xbar[k] += s; else pbar[k - NX] += s;
    }
}

int loss_grad(const orc_model* m, const double* x0, const double* v0, double dt, int S,
              const double* target, const double* xbar_extra, const double* vbar_extra,
              double* loss, orc_grads* g) {
    const size_t N = (size_t)m->n_nodes;
    const Rest r = make_rest(m);
    Inputs<double> in;
    in.load(m, nullptr);
    std::vector<double> w, mass;
    inverse_masses(m, r, in, w, mass);

    // forward, storing the input state of every step (App. B: reverse mode
    // of an explicit method keeps every step's input)
    std::vector<double> X((size_t)(S + 1) * 3 * N), V((size_t)(S + 1) * 3 * N);
    std::vector<double> x(x0, x0 + 3 * N), v(v0, v0 + 3 * N), f(3 * N);
    std::memcpy(&X[0], x.data(), 3 * N * sizeof(double));
    std::memcpy(&V[0], v.data(), 3 * N * sizeof(double));
    for (int n = 0; n < S; ++n) {
        step(m, r, in, w, dt, n, x, v, f);
        std::memcpy(&X[(size_t)(n + 1) * 3 * N], x.data(), 3 * N * sizeof(double));
        std::memcpy(&V[(size_t)(n + 1) * 3 * N], v.data(), 3 * N * sizeof(double));
    }

    // loss L = sum_i |x_i(S) - x*_i|^2 and its seed dl/ds(S)
    std::vector<double> lq(3 * N, 0.0), lu(3 * N, 0.0);
    double L = 0.0;
    if (target) {
        for (size_t i = 0; i < 3 * N; ++i) {
            const double d = x[i] - target[i];
            L += d * d;
            lq[i] = 2.0 * d;
        }
    }
    if (xbar_extra) for (size_t i = 0; i < 3 * N; ++i) lq[i] += xbar_extra[i];
    if (vbar_extra) for (size_t i = 0; i < 3 * N; ++i) lu[i] += vbar_extra[i];
    if (loss) *loss = L;

    std::vector<double> tmu_b(m->n_tets, 0.0), tlam_b(m->n_tets, 0.0), tact_b(m->n_tets, 0.0);
    // per-step actuation gradients, written when requested
    double* tseq_b = g ? g->tet_act_seq : nullptr;
    double* rseq_b = g ? g->tri_act_seq : nullptr;
    double* hseq_b = g ? g->hinge_act_seq : nullptr;
    std::vector<double> rmu_b(m->n_tris, 0.0), rlam_b(m->n_tris, 0.0), ract_b(m->n_tris, 0.0);
    std::vector<double> kb_b(m->n_hinges, 0.0), hact_b(m->n_hinges, 0.0);
    double cp_b[4] = {0, 0, 0, 0};
    std::vector<double> w_b(N, 0.0);
    std::vector<double> cq(3 * N), cu(3 * N), y(3 * N), lq_new(3 * N), lu_new(3 * N);
    // per-element (per-node) scratch of the parallel VJP loops
    const size_t n_rows = std::max({(size_t)12 * m->n_tets, (size_t)9 * m->n_tris, (size_t)12 * m->n_hinges,
                                    m->air_on ? (size_t)18 * m->n_tris : (size_t)0});
    std::vector<double> xb_e(n_rows), cpb_n(4 * N);

    std::vector<double> ta, ra, ha;
    for (int n = S - 1; n >= 0; --n) {
        const double* xn = &X[(size_t)n * 3 * N];
        const double* vn = &V[(size_t)n * 3 * N];
        in.step_act(m, n, ta, ra, ha);  // the actuation in effect during step n
        // (dg/ds+)^T c = -(dl/ds+)^T with dg/ds+ = [[0, I], [I, -dt I]] over
        // s+ = (q+, u+) and g = (g_u, g_q):  c_q = -dl/dq+,  c_u = -dl/du+ - dt dl/dq+
        for (size_t i = 0; i < 3 * N; ++i) {
            cq[i] = -lq[i];
            cu[i] = -lu[i] - dt * lq[i];
        }
        // dl/ds- = c^T dg/ds- with dg/ds- = [[-dt W df/dq, -I - dt W df/du], [-I, 0]]:
        //   dl/dq- = -c_q + (-dt W c_u)^T df/dq,  dl/du- = -c_u + (-dt W c_u)^T df/du
        // and dl/dtheta += (-dt W c_u)^T df/dtheta, dl/dw_i += -dt c_u,i . f_i.
        for (size_t i = 0; i < N; ++i)
            for (int k = 0; k < 3; ++k) y[3 * i + k] = -dt * w[i] * cu[3 * i + k];
        for (size_t i = 0; i < 3 * N; ++i) { lq_new[i] = -cq[i]; lu_new[i] = -cu[i]; }

        // element VJPs in parallel, each into its own rows of xb_e; the node
        // sums follow on one thread in element order (bitwise the serial loop)
#pragma omp parallel for schedule(static)
        for (int e = 0; e < m->n_tets; ++e) {
            double xe[12], ye[12], pb[3] = {0, 0, 0};
            double* xb = &xb_e[12 * (size_t)e];
            for (int k = 0; k < 12; ++k) xb[k] = 0.0;
            const int* t = &m->tets[4 * e];
            for (int c = 0; c < 4; ++c)
                for (int k = 0; k < 3; ++k) { xe[3 * c + k] = xn[3 * (size_t)t[c] + k]; ye[3 * c + k] = y[3 * (size_t)t[c] + k]; }
            const double pe[3] = {in.tmu[e], in.tlam[e], ta[e]};
            const double* Dmi = &r.tet_Dminv[9 * (size_t)e];
            const double Ve = r.tet_V[e];
            element_vjp<12, 3>(xe, pe, ye, xb, pb, [&](auto* xd, auto* pd, auto* fd) {
                tet_forces_t(xd, Dmi, Ve, pd[0], pd[1], pd[2], fd);
            });
            tmu_b[e] += pb[0]; tlam_b[e] += pb[1]; tact_b[e] += pb[2];
            if (tseq_b) tseq_b[(size_t)n * m->n_tets + e] = pb[2];
        }
        for (int e = 0; e < m->n_tets; ++e)
            for (int c = 0; c < 4; ++c)
                for (int k = 0; k < 3; ++k) lq_new[3 * (size_t)m->tets[4 * e + c] + k] += xb_e[12 * (size_t)e + 3 * c + k];
#pragma omp parallel for schedule(static)
        for (int e = 0; e < m->n_tris; ++e) {
            double xe[9], ye[9], pb[3] = {0, 0, 0};
            double* xb = &xb_e[9 * (size_t)e];
            for (int k = 0; k < 9; ++k) xb[k] = 0.0;
            const int* t = &m->tris[3 * e];
            for (int c = 0; c < 3; ++c)
                for (int k = 0; k < 3; ++k) { xe[3 * c + k] = xn[3 * (size_t)t[c] + k]; ye[3 * c + k] = y[3 * (size_t)t[c] + k]; }
            const double pe[3] = {in.rmu[e], in.rlam[e], ra[e]};
            const double* Dmi = &r.tri_Dminv[4 * (size_t)e];
            const double Ae = r.tri_A[e];
            element_vjp<9, 3>(xe, pe, ye, xb, pb, [&](auto* xd, auto* pd, auto* fd) {
                tri_forces_t(xd, Dmi, Ae, pd[0], pd[1], pd[2], fd);
            });
            rmu_b[e] += pb[0]; rlam_b[e] += pb[1]; ract_b[e] += pb[2];
            if (rseq_b) rseq_b[(size_t)n * m->n_tris + e] = pb[2];
        }
        for (int e = 0; e < m->n_tris; ++e)
            for (int c = 0; c < 3; ++c)
                for (int k = 0; k < 3; ++k) lq_new[3 * (size_t)m->tris[3 * e + c] + k] += xb_e[9 * (size_t)e + 3 * c + k];
#pragma omp parallel for schedule(static)
        for (int h = 0; h < m->n_hinges; ++h) {
            double xe[12], ye[12], pb[2] = {0, 0};
            double* xb = &xb_e[12 * (size_t)h];
            for (int k = 0; k < 12; ++k) xb[k] = 0.0;
            const int* t = &m->hinges[4 * h];
            for (int c = 0; c < 4; ++c)
                for (int k = 0; k < 3; ++k) { xe[3 * c + k] = xn[3 * (size_t)t[c] + k]; ye[3 * c + k] = y[3 * (size_t)t[c] + k]; }
            const double pe[2] = {in.kb[h], ha[h]};
            element_vjp<12, 2>(xe, pe, ye, xb, pb, [&](auto* xd, auto* pd, auto* fd) {
                hinge_forces_t(xd, pd[0], pd[1], fd);
            });
            kb_b[h] += pb[0]; hact_b[h] += pb[1];
            if (hseq_b) hseq_b[(size_t)n * m->n_hinges + h] = pb[1];
        }
        for (int h = 0; h < m->n_hinges; ++h)
            for (int c = 0; c < 4; ++c)
                for (int k = 0; k < 3; ++k) lq_new[3 * (size_t)m->hinges[4 * h + c] + k] += xb_e[12 * (size_t)h + 3 * c + k];
        if (m->air_on) {
            // air force of a triangle as a function of its corners' (x, v):
            // 18 inputs, 9 force outputs (y padded with zeros)
#pragma omp parallel for schedule(static)
            for (int e = 0; e < m->n_tris; ++e) {
                double xv[18], ye[18] = {0}, pb[1] = {0};
                double* xb = &xb_e[18 * (size_t)e];
                for (int k = 0; k < 18; ++k) xb[k] = 0.0;
                const int* t = &m->tris[3 * e];
                for (int c = 0; c < 3; ++c)
                    for (int k = 0; k < 3; ++k) {
                        xv[3 * c + k] = xn[3 * (size_t)t[c] + k];
                        xv[9 + 3 * c + k] = vn[3 * (size_t)t[c] + k];
                        ye[3 * c + k] = y[3 * (size_t)t[c] + k];
                    }
                element_vjp<18, 0>(xv, nullptr, ye, xb, pb, [&](auto* xd, auto* pd, auto* fd) {
                    (void)pd;
                    air_forces_t(xd, xd + 9, m->k_drag, m->k_lift, m->wind, fd);
                });
            }
            for (int e = 0; e < m->n_tris; ++e)
                for (int c = 0; c < 3; ++c)
                    for (int k = 0; k < 3; ++k) {
                        lq_new[3 * (size_t)m->tris[3 * e + c] + k] += xb_e[18 * (size_t)e + 3 * c + k];
                        lu_new[3 * (size_t)m->tris[3 * e + c] + k] += xb_e[18 * (size_t)e + 9 + 3 * c + k];
                    }
        }
        if (m->plane_on || m->sphere_on) {
            // one node per iteration (its own rows of lq_new, lu_new and of
            // the contact-parameter scratch); the parameter sums follow in node order
#pragma omp parallel for schedule(static)
            for (long long i = 0; i < (long long)N; ++i) {
                double xv[6], yi[6] = {0}, xb[6] = {0, 0, 0, 0, 0, 0};
                double* pb = &cpb_n[4 * (size_t)i];
                for (int k = 0; k < 4; ++k) pb[k] = 0.0;
                for (int k = 0; k < 3; ++k) { xv[k] = xn[3 * i + k]; xv[3 + k] = vn[3 * i + k]; yi[k] = y[3 * i + k]; }
                const double pe[4] = {m->ke, m->kd, m->kf, m->mu_f};
                // contact force as a function of the 6-vector (x, v): only its
                // first three outputs are forces, so pad y with zeros
                element_vjp<6, 4>(xv, pe, yi, xb, pb, [&](auto* xd, auto* pd, auto* fd) {
                    contact_t(m, xd, xd + 3, pd[0], pd[1], pd[2], pd[3], fd);
                });
                for (int k = 0; k < 3; ++k) { lq_new[3 * i + k] += xb[k]; lu_new[3 * i + k] += xb[3 + k]; }
            }
            for (size_t i = 0; i < N; ++i)
                for (int k = 0; k < 4; ++k) cp_b[k] += cpb_n[4 * i + k];
        }
        // dl/dw_i: the step uses w_i f_i(s-) (gravity does not depend on w)
        {
            std::vector<double> f_n(3 * N), xx(xn, xn + 3 * N), vv(vn, vn + 3 * N);
            total_force(m, r, xx.data(), vv.data(), in.tmu.data(), in.tlam.data(), ta.data(),
                        in.rmu.data(), in.rlam.data(), ra.data(), in.kb.data(), ha.data(),
                        in.cp.data(), f_n.data());
            for (size_t i = 0; i < N; ++i)
                for (int k = 0; k < 3; ++k) w_b[i] += -dt * cu[3 * i + k] * f_n[3 * i + k];
        }
        lq.swap(lq_new);
        lu.swap(lu_new);
    }

    // masses: w_i = 1/m_i  =>  dl/dm_i = -w_i^2 dl/dw_i (kinematic nodes: none);
    // m_i = sum rho_e V_e/4 (+ rho_t A_t/3)  =>  dl/drho_e = V_e/4 sum_{i in e} dl/dm_i
    std::vector<double> m_b(N, 0.0);
    for (size_t i = 0; i < N; ++i)
        if (w[i] > 0.0) m_b[i] = -w[i] * w[i] * w_b[i];
    if (g) {
        if (g->x0) std::memcpy(g->x0, lq.data(), 3 * N * sizeof(double));
        if (g->v0) std::memcpy(g->v0, lu.data(), 3 * N * sizeof(double));
        if (g->tet_mu) std::memcpy(g->tet_mu, tmu_b.data(), tmu_b.size() * sizeof(double));
        if (g->tet_lam) std::memcpy(g->tet_lam, tlam_b.data(), tlam_b.size() * sizeof(double));
        if (g->tet_act) std::memcpy(g->tet_act, tact_b.data(), tact_b.size() * sizeof(double));
        if (g->tri_mu) std::memcpy(g->tri_mu, rmu_b.data(), rmu_b.size() * sizeof(double));
        if (g->tri_lam) std::memcpy(g->tri_lam, rlam_b.data(), rlam_b.size() * sizeof(double));
        if (g->tri_act) std::memcpy(g->tri_act, ract_b.data(), ract_b.size() * sizeof(double));
        if (g->hinge_kb) std::memcpy(g->hinge_kb, kb_b.data(), kb_b.size() * sizeof(double));
        if (g->hinge_act) std::memcpy(g->hinge_act, hact_b.data(), hact_b.size() * sizeof(double));
        if (g->contact) std::memcpy(g->contact, cp_b, 4 * sizeof(double));
        if (g->node_mass) std::memcpy(g->node_mass, m_b.data(), N * sizeof(double));
        if (g->tet_rho) {
            for (int e = 0; e < m->n_tets; ++e) {
                double s = 0.0;
                for (int c = 0; c < 4; ++c) s += m_b[m->tets[4 * e + c]];
                g->tet_rho[e] = s * (r.tet_V[e] / 4.0);
            }
        }
        if (g->tri_rho) {
            for (int t = 0; t < m->n_tris; ++t) {
                double s = 0.0;
                for (int c = 0; c < 3; ++c) s += m_b[m->tris[3 * t + c]];
                g->tri_rho[t] = s * (r.tri_A[t] / 3.0);
            }
        }
    }
    return 0;
}

// ---------------------------------------------------------------------------
// 8. rigid bodies (App. A.1 "Rigid Bodies"): Newton-Euler with the contact
// model at the body's contact points, semi-implicit Euler (App. B)
// ---------------------------------------------------------------------------
// Readings: the quaternion r = (w, x, y, z) maps body to world; the contact
// law is the particles' (section 4) at X_k = x + R p_k with velocity
// V_k = v + omega x (R p_k); the world inertia is R I_b R^T; the step is
//   v+ = v + dt (g + F/m),  omega+ = omega + dt I_w^-1 (tau - omega x I_w omega),
// with I_w^-1 applied as R I_b^-1 R^T (equal for a unit quaternion; the
// same function for any r, so the gradient in r is unambiguous),
//   x+ = x + dt v+,  r+ = normalise(r + dt/2 (0, omega+) (x) r)
// (velocities first, then positions with the new velocities, as App. B's
// g(s-, s+, theta); the quaternion derivative is 1/2 omega (x) r).
template <class T>
void quat_rot(const T* r, T R[3][3]) {
    const T w = r[0], x = r[1], y = r[2], z = r[3];
    R[0][0] = 1.0 - 2.0 * (y * y + z * z); R[0][1] = 2.0 * (x * y - w * z); R[0][2] = 2.0 * (x * z + w * y);
    R[1][0] = 2.0 * (x * y + w * z); R[1][1] = 1.0 - 2.0 * (x * x + z * z); R[1][2] = 2.0 * (y * z - w * x);
    R[2][0] = 2.0 * (x * z - w * y); R[2][1] = 2.0 * (y * z + w * x); R[2][2] = 1.0 - 2.0 * (x * x + y * y);
}

template <class T>
void mat3_solve(const T A[3][3], const T* b, T* out) {  // Cramer's rule
    T c[3][3];
    c[0][0] = A[1][1] * A[2][2] - A[1][2] * A[2][1];
    c[0][1] = A[1][2] * A[2][0] - A[1][0] * A[2][2];
    c[0][2] = A[1][0] * A[2][1] - A[1][1] * A[2][0];
    c[1][0] = A[0][2] * A[2][1] - A[0][1] * A[2][2];
    c[1][1] = A[0][0] * A[2][2] - A[0][2] * A[2][0];
    c[1][2] = A[0][1] * A[2][0] - A[0][0] * A[2][1];
    c[2][0] = A[0][1] * A[1][2] - A[0][2] * A[1][1];
    c[2][1] = A[0][2] * A[1][0] - A[0][0] * A[1][2];
    c[2][2] = A[0][0] * A[1][1] - A[0][1] * A[1][0];
    const T det = A[0][0] * c[0][0] + A[0][1] * c[0][1] + A[0][2] * c[0][2];
    for (int i = 0; i < 3; ++i) out[i] = (c[0][i] * b[0] + c[1][i] * b[1] + c[2][i] * b[2]) / det;
}

// one step of one body; s [13] -> o [13]; p = (m, I6, ke, kd, kf, mu)
template <class T>
void rigid_step_t(const orc_rigid* b, const T* s, const T* p, double dt, T* o) {
    const orc_model* sc = b->scene;
    const T* x = s; const T* r = s + 3; const T* v = s + 7; const T* w = s + 10;
    const T m = p[0];
    T Ib[3][3] = {{p[1], p[4], p[5]}, {p[4], p[2], p[6]}, {p[5], p[6], p[3]}};
    T R[3][3];
    quat_rot(r, R);
    T F[3] = {T(0.0), T(0.0), T(0.0)}, tau[3] = {T(0.0), T(0.0), T(0.0)};
    for (int k = 0; k < b->n_points; ++k) {
        const double* pk = b->points + 3 * k;
        T d[3], X[3], V[3], wd[3], fc[3], td[3];
        for (int i = 0; i < 3; ++i) d[i] = R[i][0] * pk[0] + R[i][1] * pk[1] + R[i][2] * pk[2];
        vcross(w, d, wd);
        for (int i = 0; i < 3; ++i) { X[i] = x[i] + d[i]; V[i] = v[i] + wd[i]; }
        contact_t(sc, X, V, p[7], p[8], p[9], p[10], fc);
        vcross(d, fc, td);
        for (int i = 0; i < 3; ++i) { F[i] += fc[i]; tau[i] += td[i]; }
    }
    // I_w = R I_b R^T and I_w^-1 = R I_b^-1 R^T (a rotation R):
    // alpha = R I_b^-1 R^T (tau - omega x R I_b R^T omega)
    T Iw[3][3];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            T acc(0.0);
            for (int a = 0; a < 3; ++a)
                for (int c = 0; c < 3; ++c) acc += R[i][a] * Ib[a][c] * R[j][c];
            Iw[i][j] = acc;
        }
    T L[3], wL[3], h[3], alpha[3], hb[3], ab[3];
    for (int i = 0; i < 3; ++i) L[i] = Iw[i][0] * w[0] + Iw[i][1] * w[1] + Iw[i][2] * w[2];
    vcross(w, L, wL);
    for (int i = 0; i < 3; ++i) h[i] = tau[i] - wL[i];
    for (int i = 0; i < 3; ++i) hb[i] = R[0][i] * h[0] + R[1][i] * h[1] + R[2][i] * h[2];
    mat3_solve(Ib, hb, ab);
    for (int i = 0; i < 3; ++i) alpha[i] = R[i][0] * ab[0] + R[i][1] * ab[1] + R[i][2] * ab[2];
    T* xo = o; T* ro = o + 3; T* vo = o + 7; T* wo = o + 10;
    for (int i = 0; i < 3; ++i) {
        vo[i] = v[i] + dt * (sc->gravity[i] + F[i] / m);
        wo[i] = w[i] + dt * alpha[i];
        xo[i] = x[i] + dt * vo[i];
    }
    // r + dt/2 (0, omega+) (x) r:  (0, a) (x) (rw, rv) = (-a.rv, rw a + a x rv)
    T ax[3];
    vcross(wo, r + 1, ax);
    T q[4];
    q[0] = r[0] - 0.5 * dt * vdot(wo, r + 1);
    for (int i = 0; i < 3; ++i) q[1 + i] = r[1 + i] + 0.5 * dt * (r[0] * wo[i] + ax[i]);
    const T qn = fsqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
    for (int i = 0; i < 4; ++i) ro[i] = q[i] / qn;
}

template <class T>
T rigid_points_loss(const orc_rigid* b, const T* s, const double* target, const double* seed) {
    T R[3][3];
    quat_rot(s + 3, R);
    T L(0.0);
    if (target) {
        for (int k = 0; k < b->n_points; ++k) {
            const double* pk = b->points + 3 * k;
            for (int i = 0; i < 3; ++i) {
                const T X = s[i] + R[i][0] * pk[0] + R[i][1] * pk[1] + R[i][2] * pk[2];
                const T d = X - target[3 * k + i];
                L += d * d;
            }
        }
    }
    if (seed)
        for (int i = 0; i < 13; ++i) L += seed[i] * s[i];
    return L;
}

void rigid_params(const orc_rigid* b, double* p) {
    p[0] = b->mass;
    for (int i = 0; i < 6; ++i) p[1 + i] = b->inertia[i];
    for (int i = 0; i < 4; ++i) p[7 + i] = b->contact[i];
}

}  // namespace

// ---------------------------------------------------------------------------
// C API
// ---------------------------------------------------------------------------
extern "C" {

void orc_tet_rest(const double X[12], double Dminv[9], double* V) { tet_rest(X, Dminv, V); }
void orc_tri_rest(const double X[9], double Dminv[4], double* A) { tri_rest(X, Dminv, A); }

int orc_node_masses(const orc_model* m, double* mass) {
    const Rest r = make_rest(m);
    Inputs<double> in;
    in.load(m, nullptr);
    node_masses(m, r, in.trho.data(), in.rrho.data(), mass);
    return 0;
}

void orc_tet_forces(const double x[12], const double Dminv[9], double V, double mu, double lam,
                    double act, double f[12]) {
    tet_forces_t<double>(x, Dminv, V, mu, lam, act, f);
}
double orc_tet_energy(const double x[12], const double Dminv[9], double V, double mu, double lam, double act) {
    return tet_energy_t<double>(x, Dminv, V, mu, lam, act);
}
void orc_tri_forces(const double x[9], const double Dminv[4], double A, double mu, double lam,
                    double act, double f[9]) {
    tri_forces_t<double>(x, Dminv, A, mu, lam, act, f);
}
double orc_tri_energy(const double x[9], const double Dminv[4], double A, double mu, double lam, double act) {
    return tri_energy_t<double>(x, Dminv, A, mu, lam, act);
}
void orc_hinge_forces(const double x[12], double kb, double act, double f[12]) {
    hinge_forces_t<double>(x, kb, act, f);
}
double orc_hinge_angle(const double x[12]) { return hinge_angle_t<double>(x); }
void orc_hinge_angle_grad(const double x[12], double g[12]) {
    Dual<12> xd[12];
    for (int i = 0; i < 12; ++i) { xd[i] = Dual<12>(x[i]); xd[i].d[i] = 1.0; }
    const Dual<12> phi = hinge_angle_t(xd);
    for (int i = 0; i < 12; ++i) g[i] = phi.d[i];
}
void orc_air_forces(const double x[9], const double v[9], double k_drag, double k_lift, const double wind[3],
                    double f[9]) {
    air_forces_t<double>(x, v, k_drag, k_lift, wind, f);
}
void orc_contact_force(const orc_model* m, const double x[3], const double v[3], double f[3]) {
    contact_t<double>(m, x, v, m->ke, m->kd, m->kf, m->mu_f, f);
}

int orc_rigid_rollout(const orc_rigid* b, const double* state0, double dt, int S, double* stateS, double* traj) {
    double p[11], s[13], o[13];
    rigid_params(b, p);
    std::memcpy(s, state0, sizeof s);
    if (traj) std::memcpy(traj, s, sizeof s);
    for (int n = 0; n < S; ++n) {
        rigid_step_t<double>(b, s, p, dt, o);
        std::memcpy(s, o, sizeof s);
        if (traj) std::memcpy(traj + 13 * (size_t)(n + 1), s, sizeof s);
    }
    if (stateS) std::memcpy(stateS, s, sizeof s);
    return 0;
}

// Reverse mode through the stored trajectory: each step's exact Jacobian
// with respect to (state, parameters) from Dual<24>, applied transposed.
int orc_rigid_loss_grad(const orc_rigid* b, const double* state0, double dt, int S, const double* target,
                        const double* seed, double* loss, double* d_state0, double* d_mass, double* d_inertia,
                        double* d_contact) {
    double p[11];
    rigid_params(b, p);
    std::vector<double> traj(13 * (size_t)(S + 1));
    orc_rigid_rollout(b, state0, dt, S, nullptr, traj.data());
    const double* sS = &traj[13 * (size_t)S];
    // seed: dL/ds(S)
    typedef Dual<13> D13;
    D13 sd[13];
    for (int i = 0; i < 13; ++i) { sd[i] = D13(sS[i]); sd[i].d[i] = 1.0; }
    const D13 Ld = rigid_points_loss(b, sd, target, seed);
    if (loss) *loss = Ld.v;
    double lam[13], pb[11] = {0};
    for (int i = 0; i < 13; ++i) lam[i] = Ld.d[i];
    typedef Dual<24> D;
    for (int n = S - 1; n >= 0; --n) {
        const double* sn = &traj[13 * (size_t)n];
        D si[13], pi[11], so[13];
        for (int i = 0; i < 13; ++i) { si[i] = D(sn[i]); si[i].d[i] = 1.0; }
        for (int j = 0; j < 11; ++j) { pi[j] = D(p[j]); pi[j].d[13 + j] = 1.0; }
        rigid_step_t(b, si, pi, dt, so);
        double nl[13] = {0};
        for (int k = 0; k < 24; ++k) {
            double acc = 0.0;
            for (int i = 0; i < 13; ++i) acc += lam[i] * so[i].d[k];
            if (k < 13) nl[k] = acc; else pb[k - 13] += acc;
        }
        std::memcpy(lam, nl, sizeof lam);
    }
    if (d_state0) std::memcpy(d_state0, lam, sizeof lam);
    if (d_mass) *d_mass = pb[0];
    if (d_inertia) for (int i = 0; i < 6; ++i) d_inertia[i] = pb[1 + i];
    if (d_contact) for (int i = 0; i < 4; ++i) d_contact[i] = pb[7 + i];
    return 0;
}

int orc_rigid_loss_dir(const orc_rigid* b, const double* state0, double dt, int S, const double* target,
                       const double* seed, const double* dir_state0, double dir_mass, const double* dir_inertia,
                       const double* dir_contact, double* loss, double* dloss) {
    typedef Dual<1> D;
    double p[11];
    rigid_params(b, p);
    D s[13], pp[11], o[13];
    for (int i = 0; i < 13; ++i) { s[i] = D(state0[i]); s[i].d[0] = dir_state0 ? dir_state0[i] : 0.0; }
    for (int j = 0; j < 11; ++j) pp[j] = D(p[j]);
    pp[0].d[0] = dir_mass;
    for (int j = 0; j < 6; ++j) pp[1 + j].d[0] = dir_inertia ? dir_inertia[j] : 0.0;
    for (int j = 0; j < 4; ++j) pp[7 + j].d[0] = dir_contact ? dir_contact[j] : 0.0;
    for (int n = 0; n < S; ++n) {
        rigid_step_t(b, s, pp, dt, o);
        for (int i = 0; i < 13; ++i) s[i] = o[i];
    }
    const D L = rigid_points_loss(b, s, target, seed);
    if (loss) *loss = L.v;
    if (dloss) *dloss = L.d[0];
    return 0;
}

int orc_forces(const orc_model* m, const double* x, const double* v, double* f) {
    const Rest r = make_rest(m);
    Inputs<double> in;
    in.load(m, nullptr);
    total_force(m, r, x, v, in.tmu.data(), in.tlam.data(), in.tact.data(), in.rmu.data(),
                in.rlam.data(), in.ract.data(), in.kb.data(), in.hact.data(), in.cp.data(), f);
    return 0;
}

int orc_rollout(const orc_model* m, const double* x0, const double* v0, double dt, int S,
                double* xS, double* vS, double* traj) {
    const size_t N = (size_t)m->n_nodes;
    const Rest r = make_rest(m);
    Inputs<double> in;
    in.load(m, nullptr);
    std::vector<double> w, mass;
    inverse_masses(m, r, in, w, mass);
    std::vector<double> x(x0, x0 + 3 * N), v(v0, v0 + 3 * N), f(3 * N);
    if (traj) std::memcpy(traj, x.data(), 3 * N * sizeof(double));
    for (int n = 0; n < S; ++n) {
        step(m, r, in, w, dt, n, x, v, f);
        if (traj) std::memcpy(traj + (size_t)(n + 1) * 3 * N, x.data(), 3 * N * sizeof(double));
    }
    if (xS) std::memcpy(xS, x.data(), 3 * N * sizeof(double));
    if (vS) std::memcpy(vS, v.data(), 3 * N * sizeof(double));
    return 0;
}

int orc_loss_grad(const orc_model* m, const double* x0, const double* v0, double dt, int S,
                  const double* target, const double* xbar_extra, const double* vbar_extra,
                  double* loss, orc_grads* g) {
    return loss_grad(m, x0, v0, dt, S, target, xbar_extra, vbar_extra, loss, g);
}

// 7. forward mode: every input carries its direction through the set-up
// (masses) and every step; L and dL/d(direction) come out of the loss.
int orc_loss_dir(const orc_model* m, const double* x0, const double* v0, double dt, int S,
                 const double* target, const orc_dirs* d, double* loss, double* dloss) {
    typedef Dual<1> T;
    const size_t N = (size_t)m->n_nodes;
    const Rest r = make_rest(m);
    Inputs<T> in;
    in.load(m, d);
    std::vector<T> w, mass;
    inverse_masses(m, r, in, w, mass);
    std::vector<T> x(3 * N), v(3 * N), f(3 * N);
    for (size_t i = 0; i < 3 * N; ++i) {
        seed<T>(x[i], x0[i], d ? d->x0 : nullptr, (int)i);
        seed<T>(v[i], v0[i], d ? d->v0 : nullptr, (int)i);
    }
    for (int n = 0; n < S; ++n) step(m, r, in, w, dt, n, x, v, f);
    T L(0.0);
    for (size_t i = 0; i < 3 * N; ++i) {
        const T dd = x[i] - target[i];
        L += dd * dd;
    }
    if (loss) *loss = L.v;
    if (dloss) *dloss = L.d[0];
    return 0;
}

int orc_set_threads(int n) {
#ifdef _OPENMP
    static const int all = omp_get_max_threads();
    omp_set_num_threads(n > 0 ? n : all);
    return omp_get_max_threads();
#else
    (void)n;
    return 1;
#endif
}

int orc_max_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

}  // extern "C"
