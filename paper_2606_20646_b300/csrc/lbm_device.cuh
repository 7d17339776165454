// Device-side building blocks of the sm_103a total-Lagrangian vectorial LBM:
// descriptors, level-set primitives (FP64), boundary data, the neo-Hookean
// stress and small dense algebra.  Used by the kernels in lbm_kernels.cuh.
#pragma once

#include <cmath>
#include <cstdint>
#include <cuda_runtime.h>

namespace tlv {

constexpr int kMaxShapes = LBM_MAX_SHAPES;
constexpr int kMaxGroups = LBM_MAX_GROUPS;
constexpr int kMaxBCs = 16;
constexpr int kLsqCap = 160;      // LSQ stencil capacity per link (active nodes within 3 dx)
constexpr double kLsqRho2 = 9.0;  // squared stencil radius in lattice units

// flags byte per box node
constexpr uint8_t kActive = 1u << 6;   // phi(X) <= 0
constexpr uint8_t kNeedU = 1u << 7;    // u^n is read by some Neumann LSQ stencil
constexpr uint8_t kCutMask = 0x3f;     // bit q: link (m, q) is cut (neighbour m + e_q inactive)

// device status bits (mirrors lbm_device_status of the C ABI)
constexpr int kStNonfinite = 1, kStJacobian = 2, kStNewton = 4, kStLsq = 8, kStCapacity = 16, kStDomain = 32,
              kStNoBC = 64, kStBounds = 256;

struct ShapeD {
    int kind, complement, bid, pad;
    double c[3], a[3], Q[9], p;
    // kind 5 (node samples): the samples (box order, caller memory) and the lattice they sit on
    const double *phi;
    int n[3], per;  // nodes per axis; bit a: axis a periodic
    double org[3], dx;
};

struct BCD {
    int bid, kind, profile, ramp;
    double t_ramp, center[3], A[9], vec[3], amp;
};

// ---------------------------------------------------------------------------------------------
// level set: phi = max over shapes (Sec. 3.1, Eq. level-set-domain)
// ---------------------------------------------------------------------------------------------

// Sampled level set: phi between nodes is the multilinear interpolant of the node samples (linear
// along every lattice link), constant beyond the outermost node of a non-periodic axis (so a body
// reaching a non-periodic face is refused by the box-face rule) and periodic on periodic axes; its
// gradient, for the normal of Eq. (level-set-normal), is the same interpolant of the nodes'
// central differences (one-sided at non-periodic ends).  A coordinate within 1e-9 spacings of a node
// is that node, so node and link evaluations read the samples exactly.
__device__ inline double sample_at(const ShapeD &s, int D, const int j[3]) {
    long long idx = 0, stride = 1;
    for (int a = 0; a < D; ++a) {
        const int n = s.n[a];
        int k = j[a];
        if ((s.per >> a) & 1) k = ((k % n) + n) % n;
        else k = k < 0 ? 0 : (k >= n ? n - 1 : k);
        idx += stride * k;
        stride *= n;
    }
    return s.phi[idx];
}

__device__ inline double sampled_phi(const ShapeD &s, int D, const double X[3], double g[3]) {
    int i0[3] = {0, 0, 0};
    double f[3] = {0.0, 0.0, 0.0};
    for (int a = 0; a < D; ++a) {
        const double xi = (X[a] - s.org[a]) / s.dx - 0.5;
        double fl = floor(xi), fr = xi - fl;
        if (fr < 1e-9) fr = 0.0;
        else if (fr > 1.0 - 1e-9) { fl += 1.0; fr = 0.0; }
        i0[a] = (int)fl;
        f[a] = fr;
    }
    double v = 0.0, gr[3] = {0.0, 0.0, 0.0};
    for (int c = 0; c < (1 << D); ++c) {
        double w = 1.0;
        int j[3] = {0, 0, 0};
        for (int a = 0; a < D; ++a) {
            const int bit = (c >> a) & 1;
            w *= bit ? f[a] : 1.0 - f[a];
            j[a] = i0[a] + bit;
        }
        if (w == 0.0) continue;
        v += w * sample_at(s, D, j);
        if (g)
            for (int a = 0; a < D; ++a) {
                int jp[3] = {j[0], j[1], j[2]}, jm[3] = {j[0], j[1], j[2]};
                jp[a] += 1;
                jm[a] -= 1;
                double ga;
                if (s.n[a] == 1) ga = 0.0;
                else if (((s.per >> a) & 1) || (j[a] > 0 && j[a] < s.n[a] - 1))
                    ga = (sample_at(s, D, jp) - sample_at(s, D, jm)) / (2.0 * s.dx);
                else if (j[a] <= 0)
                    ga = (sample_at(s, D, jp) - sample_at(s, D, j)) / s.dx;
                else
                    ga = (sample_at(s, D, j) - sample_at(s, D, jm)) / s.dx;
                gr[a] += w * ga;
            }
    }
    if (g) { g[0] = gr[0]; g[1] = gr[1]; g[2] = gr[2]; }
    return v;
}

__device__ inline double shape_phi(const ShapeD &s, int D, const double X[3], double g[3]) {
    if (s.kind == 5) {
        double gs[3];
        double v = sampled_phi(s, D, X, g ? gs : nullptr);
        if (s.complement) { v = -v; gs[0] = -gs[0]; gs[1] = -gs[1]; gs[2] = -gs[2]; }
        if (g) { g[0] = gs[0]; g[1] = gs[1]; g[2] = (D == 3) ? gs[2] : 0.0; }
        return v;
    }
    const double d0 = X[0] - s.c[0], d1 = X[1] - s.c[1], d2 = (D == 3) ? X[2] - s.c[2] : 0.0;
    double v;
    double gx = 0.0, gy = 0.0, gz = 0.0;
    switch (s.kind) {
    case 0: {  // sphere / circle
        double r = sqrt(d0 * d0 + d1 * d1 + d2 * d2);
        v = r - s.a[0];
        if (r > 0.0) { gx = d0 / r; gy = d1 / r; gz = d2 / r; }
        break;
    }
    case 1: {  // ellipsoid, xi = Q^T d
        double xi[3], gl[3] = {0.0, 0.0, 0.0};
        for (int a = 0; a < 3; ++a) xi[a] = s.Q[0 * 3 + a] * d0 + s.Q[1 * 3 + a] * d1 + s.Q[2 * 3 + a] * d2;
        v = -1.0;
        for (int a = 0; a < D; ++a) {
            double r = xi[a] / s.a[a];
            v += r * r;
            gl[a] = 2.0 * xi[a] / (s.a[a] * s.a[a]);
        }
        gx = s.Q[0] * gl[0] + s.Q[1] * gl[1] + s.Q[2] * gl[2];
        gy = s.Q[3] * gl[0] + s.Q[4] * gl[1] + s.Q[5] * gl[2];
        gz = s.Q[6] * gl[0] + s.Q[7] * gl[1] + s.Q[8] * gl[2];
        break;
    }
    case 2: {  // superellipse (2D)
        double xi0 = s.Q[0] * d0 + s.Q[3] * d1, xi1 = s.Q[1] * d0 + s.Q[4] * d1;
        double r0 = fabs(xi0 / s.a[0]), r1 = fabs(xi1 / s.a[1]);
        v = pow(r0, s.p) + pow(r1, s.p) - 1.0;
        double s0 = xi0 > 0.0 ? 1.0 : (xi0 < 0.0 ? -1.0 : 0.0);
        double s1 = xi1 > 0.0 ? 1.0 : (xi1 < 0.0 ? -1.0 : 0.0);
        double g0 = s.p * pow(r0, s.p - 1.0) * s0 / s.a[0], g1 = s.p * pow(r1, s.p - 1.0) * s1 / s.a[1];
        gx = s.Q[0] * g0 + s.Q[1] * g1;
        gy = s.Q[3] * g0 + s.Q[4] * g1;
        break;
    }
    case 3: {  // cylinder about X_3
        double r = sqrt(d0 * d0 + d1 * d1);
        v = r - s.a[0];
        if (r > 0.0) { gx = d0 / r; gy = d1 / r; }
        break;
    }
    case 4:  // half-space with outward normal a
        v = s.a[0] * d0 + s.a[1] * d1 + ((D == 3) ? s.a[2] * d2 : 0.0);
        gx = s.a[0]; gy = s.a[1]; gz = s.a[2];
        break;
    default:
        v = 1.0;
    }
    if (D == 2) gz = 0.0;
    if (s.complement) { v = -v; gx = -gx; gy = -gy; gz = -gz; }
    if (g) { g[0] = gx; g[1] = gy; g[2] = gz; }
    return v;
}

__device__ inline double levelset(const ShapeD *__restrict__ shapes, int ns, int D, const double X[3], int *which) {
    if (ns == 0) { if (which) *which = -1; return -1.0; }
    double best = 0.0;
    int w = -1;
    for (int s = 0; s < ns; ++s) {
        double v = shape_phi(shapes[s], D, X, nullptr);
        if (w < 0 || v > best) { best = v; w = s; }
    }
    if (which) *which = w;
    return best;
}

// a specimen of a multi-specimen body: its shapes and a box containing it
struct GroupD {
    int first, count;
    double lo[3], hi[3];
};

// the level set a kernel sees: one body (ngroups == 0), or the union of disjoint groups
struct LevelSetD {
    const ShapeD *shapes;
    int nshapes;
    const GroupD *groups;
    int ngroups;
};

// phi(X) and, optionally, the shape defining it and its group: max over the shapes of one body, or
// min over the groups whose box contains X of the group's max (+1 outside every box)
__device__ inline double levelset(const LevelSetD &L, int D, const double X[3], int *which, int *group = nullptr) {
    if (L.ngroups == 0) {
        if (group) *group = 0;
        return levelset(L.shapes, L.nshapes, D, X, which);
    }
    double best = 1.0;
    int w = -1, gb = -1;
    for (int g = 0; g < L.ngroups; ++g) {
        const GroupD &G = L.groups[g];
        bool in = true;
        for (int a = 0; a < D; ++a) in = in && X[a] >= G.lo[a] && X[a] <= G.hi[a];
        if (!in) continue;
        int wg;
        const double v = levelset(L.shapes + G.first, G.count, D, X, &wg);
        if (gb < 0 || v < best) { best = v; w = G.first + wg; gb = g; }
    }
    if (which) *which = w;
    if (group) *group = gb < 0 ? 0 : gb;
    return gb < 0 ? 1.0 : best;
}

// ---------------------------------------------------------------------------------------------
// boundary data: ramps s(t), Dirichlet displacement/velocity, nominal traction
// ---------------------------------------------------------------------------------------------

__host__ __device__ inline void ramp_eval(int kind, double T, double t, double &s, double &sd) {
    const double pi = 3.14159265358979323846;
    switch (kind) {
    case 1: if (t < T) { s = t / T; sd = 1.0 / T; } else { s = 1.0; sd = 0.0; } return;
    case 2: if (t < T) { double a = sin(pi * t / (2.0 * T)); s = a * a; sd = pi / (2.0 * T) * sin(pi * t / T); }
            else { s = 1.0; sd = 0.0; } return;
    case 3: if (t < T) { s = 0.5 * (1.0 - cos(pi * t / T)); sd = pi / (2.0 * T) * sin(pi * t / T); }
            else { s = 1.0; sd = 0.0; } return;
    case 4: s = t; sd = 1.0; return;
    default: s = 1.0; sd = 0.0;
    }
}

// velocity (want_u = false) or displacement (want_u = true) of a Dirichlet profile at X, t
__device__ inline void dirichlet_eval(const BCD &bc, int D, const double X[3], double t, bool want_u, double out[3]) {
    double s, sd;
    ramp_eval(bc.ramp, bc.t_ramp, t, s, sd);
    const double a = want_u ? s : sd;
    out[0] = out[1] = out[2] = 0.0;
    const double d[3] = {X[0] - bc.center[0], X[1] - bc.center[1], (D == 3) ? X[2] - bc.center[2] : 0.0};
    switch (bc.profile) {
    case 1:
        for (int i = 0; i < D; ++i)
            for (int j = 0; j < D; ++j) out[i] += a * bc.A[i * 3 + j] * d[j];
        break;
    case 2: {
        double r = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
        for (int i = 0; i < D; ++i) out[i] = bc.amp * a * d[i] / r;
        break;
    }
    case 3: {
        double al = s * bc.amp;
        if (want_u) {
            out[0] = (cos(al) - 1.0) * d[0] - sin(al) * d[1];
            out[1] = sin(al) * d[0] + (cos(al) - 1.0) * d[1];
            if (D == 3) out[2] = s * bc.vec[2];
        } else {
            double ald = sd * bc.amp;
            out[0] = ald * (-sin(al) * d[0] - cos(al) * d[1]);
            out[1] = ald * (cos(al) * d[0] - sin(al) * d[1]);
            if (D == 3) out[2] = sd * bc.vec[2];
        }
        break;
    }
    case 4:  // translation u_D = s(t) vec
        for (int i = 0; i < D; ++i) out[i] = a * bc.vec[i];
        break;
    default:
        break;
    }
}

__device__ inline void traction_eval(const BCD &bc, int D, const double X[3], double t, double T[3]) {
    double s, sd;
    ramp_eval(bc.ramp, bc.t_ramp, t, s, sd);
    T[0] = T[1] = T[2] = 0.0;
    if (bc.profile == 2) {
        const double d[3] = {X[0] - bc.center[0], X[1] - bc.center[1], (D == 3) ? X[2] - bc.center[2] : 0.0};
        double r = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
        for (int i = 0; i < D; ++i) T[i] = bc.amp * s * d[i] / r;
    } else if (bc.profile == 4) {
        for (int i = 0; i < D; ++i) T[i] = s * bc.vec[i];
    }
}

// The geometric vector g_l of a cut link for its boundary profile, in which the FP32 forms write the
// boundary value as M(t) g_l + k(t): X_b - center (affine, twist-stretch), e_R (radial), 0 (others)
__device__ inline void link_gvec(const BCD &bc, int D, const double Xb[3], double out[3]) {
    out[0] = out[1] = out[2] = 0.0;
    const double d[3] = {Xb[0] - bc.center[0], Xb[1] - bc.center[1], (D == 3) ? Xb[2] - bc.center[2] : 0.0};
    if (bc.profile == 1 || bc.profile == 3) {
        for (int i = 0; i < 3; ++i) out[i] = d[i];
    } else if (bc.profile == 2) {
        const double r = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
        for (int i = 0; i < D; ++i) out[i] = d[i] / r;
    }
}

// ---------------------------------------------------------------------------------------------
// constitutive law: compressible neo-Hookean (Sec. 4.1, Eq. validation-nh-energy)
//   P = mu F + (lam/2 (J^2 - 1) - mu) F^{-T}
// ---------------------------------------------------------------------------------------------

template <typename real, int D> __device__ __forceinline__ real det(const real F[D * D]) {
    if constexpr (D == 2) {
        return F[0] * F[3] - F[1] * F[2];
    } else {
        return F[0] * (F[4] * F[8] - F[5] * F[7]) - F[1] * (F[3] * F[8] - F[5] * F[6]) +
               F[2] * (F[3] * F[7] - F[4] * F[6]);
    }
}

// cofactor matrix cof(F) = J F^{-T}
template <typename real, int D> __device__ __forceinline__ void cofactor(const real F[D * D], real C[D * D]) {
    if constexpr (D == 2) {
        C[0] = F[3]; C[1] = -F[2]; C[2] = -F[1]; C[3] = F[0];
    } else {
        C[0] = F[4] * F[8] - F[5] * F[7];
        C[1] = F[5] * F[6] - F[3] * F[8];
        C[2] = F[3] * F[7] - F[4] * F[6];
        C[3] = F[2] * F[7] - F[1] * F[8];
        C[4] = F[0] * F[8] - F[2] * F[6];
        C[5] = F[1] * F[6] - F[0] * F[7];
        C[6] = F[1] * F[5] - F[2] * F[4];
        C[7] = F[2] * F[3] - F[0] * F[5];
        C[8] = F[0] * F[4] - F[1] * F[3];
    }
}

// first Piola stress; returns J
template <typename real, int D>
__device__ __forceinline__ real piola(const real F[D * D], real mu, real lam, real P[D * D]) {
    real C[D * D];
    cofactor<real, D>(F, C);
    const real J = det<real, D>(F);
    const real s = real(0.5) * lam * (J * J - real(1)) - mu;
    #pragma unroll
    for (int k = 0; k < D * D; ++k) P[k] = mu * F[k] + s * (C[k] / J);  // F^{-T} = cof(F) / J
    return J;
}

// J - 1 = det(I + G) - 1 from the displacement gradient G = F - I, without forming F: the sum of
// the invariants tr G + I_2(G) + det G (3D), tr G + det G (2D), accurate to the relative precision
// of G instead of the absolute precision of F
template <typename real, int D> __device__ __forceinline__ real det_m1(const real G[D * D]) {
    if constexpr (D == 2) {
        return (G[0] + G[3]) + (G[0] * G[3] - G[1] * G[2]);
    } else {
        const real i2 = (G[0] * G[4] - G[1] * G[3]) + (G[0] * G[8] - G[2] * G[6]) + (G[4] * G[8] - G[5] * G[7]);
        return ((G[0] + G[4]) + G[8]) + i2 + det<real, D>(G);
    }
}

// First Piola stress of the neo-Hookean law from G = F - I (FP32 forms).  The same function as
// piola(), P = mu F + (lam/2 (J^2 - 1) - mu) F^{-T}, rearranged with I - F^{-T} = F^{-T} G^T into
//   P = mu (G + F^{-T} G^T) + (lam/2) (J - 1)(J + 1) F^{-T}
// so that the terms cancelling near F = I (mu F - mu F^{-T}, J^2 - 1) are never formed: every term
// is a product of small quantities, and P keeps the relative precision of G.  Returns J; Fit
// receives F^{-T}.
template <typename real, int D>
__device__ __forceinline__ real piola_g(const real G[D * D], real mu, real lam, real P[D * D], real Fit[D * D]) {
    real F[D * D], C[D * D];
    #pragma unroll
    for (int k = 0; k < D * D; ++k) F[k] = G[k] + ((k / D == k % D) ? real(1) : real(0));
    cofactor<real, D>(F, C);
    const real jm1 = det_m1<real, D>(G);
    const real J = real(1) + jm1;
    const real iJ = real(1) / J;
    #pragma unroll
    for (int k = 0; k < D * D; ++k) Fit[k] = C[k] * iJ;
    const real vol = real(0.5) * lam * jm1 * (J + real(1));
    #pragma unroll
    for (int i = 0; i < D; ++i)
        #pragma unroll
        for (int A = 0; A < D; ++A) {
            real fg = real(0);
            #pragma unroll
            for (int k = 0; k < D; ++k) fg += Fit[i * D + k] * G[A * D + k];
            P[i * D + A] = mu * (G[i * D + A] + fg) + vol * Fit[i * D + A];
        }
    return J;
}

// smallest eigenvalue of a symmetric D x D matrix (row-major): closed form in 2D, the trigonometric
// form of the cubic's roots in 3D
template <int D> __host__ __device__ inline double sym_min_eig(const double C[D * D]) {
    if constexpr (D == 2) {
        const double h = 0.5 * (C[0] + C[3]), d = 0.5 * (C[0] - C[3]);
        return h - sqrt(d * d + C[1] * C[1]);
    } else {
        const double p1 = C[1] * C[1] + C[2] * C[2] + C[5] * C[5];
        const double q = (C[0] + C[4] + C[8]) / 3.0;
        if (!(p1 > 0.0)) return fmin(C[0], fmin(C[4], C[8]));
        const double a = C[0] - q, b = C[4] - q, c = C[8] - q;
        const double p = sqrt((a * a + b * b + c * c + 2.0 * p1) / 6.0);
        const double B[9] = {a / p, C[1] / p, C[2] / p, C[3] / p, b / p, C[5] / p, C[6] / p, C[7] / p, c / p};
        double r = 0.5 * (B[0] * (B[4] * B[8] - B[5] * B[7]) - B[1] * (B[3] * B[8] - B[5] * B[6]) +
                          B[2] * (B[3] * B[7] - B[4] * B[6]));
        r = r < -1.0 ? -1.0 : (r > 1.0 ? 1.0 : r);
        const double phi = acos(r) / 3.0;
        return q + 2.0 * p * cos(phi + 2.0943951023931954923);  // + 2 pi / 3: the smallest root
    }
}

// Squared largest tangent wave speed of the neo-Hookean law at F (rho0 = 1): the largest eigenvalue
// of the acoustic tensor Q(n; F) = n_A C_iAkB n_B (Eq. acoustic-tensor-general-d) over unit
// directions n.  Here Q(n) = mu I + kappa a a^T with a = F^{-T} n and kappa = mu + lam (J^2 + 1)/2,
// so its eigenvalues are mu and mu + kappa |a|^2, and max_n |F^{-T} n|^2 = 1 / sigma_min(F)^2, the
// reciprocal of the smallest eigenvalue of F^T F.  At F = I: lam + 2 mu.
template <int D> __host__ __device__ inline double tangent_speed2(const double F[D * D], double mu, double lam) {
    double C[D * D], J;
    if constexpr (D == 2) J = F[0] * F[3] - F[1] * F[2];
    else J = F[0] * (F[4] * F[8] - F[5] * F[7]) - F[1] * (F[3] * F[8] - F[5] * F[6]) + F[2] * (F[3] * F[7] - F[4] * F[6]);
    for (int i = 0; i < D; ++i)
        for (int j = 0; j < D; ++j) {
            double v = 0.0;
            for (int k = 0; k < D; ++k) v += F[k * D + i] * F[k * D + j];
            C[i * D + j] = v;
        }
    const double smin = sym_min_eig<D>(C);
    const double kappa = mu + 0.5 * lam * (J * J + 1.0);
    const double top = smin > 0.0 ? mu + kappa / smin : INFINITY;
    return kappa > 0.0 ? top : mu;
}

// dense D x D solve by Cramer's rule (D = 2, 3); returns false if singular
template <typename real, int D> __device__ __forceinline__ bool solve_small(const real A[D * D], const real b[D], real x[D]) {
    const real J = det<real, D>(A);
    if (!(J != real(0)) || !isfinite(J)) return false;
    real C[D * D];
    cofactor<real, D>(A, C);  // A^{-1} = C^T / J
    #pragma unroll
    for (int i = 0; i < D; ++i) {
        real acc = 0;
        #pragma unroll
        for (int j = 0; j < D; ++j) acc += C[j * D + i] * b[j];
        x[i] = acc / J;
    }
    return true;
}

}  // namespace tlv
