// Reverse mode of the step for bodies with velocity-Dirichlet cut links only: the discrete adjoint
// of gather + interpolated bounce-back closure + recovery + neo-Hookean stress + BGK collision with
// source + displacement quadrature, accumulating dL/dmu per node and dL/db.  No counterpart in the
// paper; the forward it differentiates is Algorithm 1 without the projection (no Neumann links).
//
// Notation of one forward step n at node m (pull scheme, stored state S = f*^{n-1}):
//   g_q(m)  = S_q(m - e_q) across interior links, else the closure R of the cut link c = q^1:
//             eta >= 1/2: R = (D_k S_c(m) + S_b)/(2 eta) + (1 - 1/(2 eta)) S_q(m)
//             eta <  1/2: R = D_k (2 eta S_c(m) + (1 - 2 eta) S_c(m + e_q)) + S_b   (m + e_q active)
//                         R = D_k S_c(m) + S_b                                     (otherwise)
//   v = (sum_q g_v + dt/2 b)/(1 + gamma dt/2),  X = sum_q g_F  (X = F, or F - I when shifted)
//   f*_q = (1 - omega) g_q + omega f^eq_q(v, X, P(F; mu)) + src_q(v)
//   u*^{n+1} = u*^n + dt v
// Given lambda* = dL/df*^n and lambda_u = dL/du*^{n+1} (constant over the sweep, since u* enters
// additively), the reverse step forms gbar = dL/dg^n at every node, and dL/dS = dL/df*^{n-1} is
// the transpose of the gather: a pull of gbar over the same links, which the next reverse step
// (n-1) evaluates at its own node before its local product.  The stress derivative uses the
// tangent's major symmetry: the product with C^T equals the directional derivative along Pbar.
#pragma once

#include "lbm_kernels.cuh"

namespace tlv {

template <typename real> struct AdjArgs {
    const real *g_in;    // gbar of the step after this one (Q*K planes)
    real *g_out;         // gbar of this step
    double *mubar;       // dL/dmu per node
    double *bbar;        // dL/db (3)
    const double *lu;    // dL/du* (D planes, box order over npad)
    const double *grad_u;  // seed: dL/du(t_N), D * nbox values
    long long nbox;
    double th;           // time of the closure data used by this step's gather
    LinkGeom<real> L;
    const BCD *bcs;
};

// d P(F; Z) for the neo-Hookean law (Eq. tangent of P-C-general): mu Z + lam J^2 tr(F^-1 Z) F^-T
// - (lam/2 (J^2 - 1) - mu) F^-T Z^T F^-T
template <typename real, int D>
__device__ __forceinline__ void dpiola_t(const real *F, const real *Z, real mu, real lam, real *dP) {
    real C[D * D];
    cofactor<real, D>(F, C);
    const real J = det<real, D>(F);
    real Fit[D * D];
    #pragma unroll
    for (int k = 0; k < D * D; ++k) Fit[k] = C[k] / J;
    real tr = 0;
    #pragma unroll
    for (int k = 0; k < D * D; ++k) tr += Fit[k] * Z[k];
    const real s = real(0.5) * lam * (J * J - real(1)) - mu;
    #pragma unroll
    for (int i = 0; i < D; ++i)
        #pragma unroll
        for (int A = 0; A < D; ++A) {
            real m = 0;
            #pragma unroll
            for (int B = 0; B < D; ++B)
                #pragma unroll
                for (int j = 0; j < D; ++j) m += Fit[i * D + B] * Z[j * D + B] * Fit[j * D + A];
            dP[i * D + A] = mu * Z[i * D + A] + lam * J * J * tr * Fit[i * D + A] - s * m;
        }
}

// derivatives of the closure value R with respect to S_c(m) (alpha, per row kind), S_q(m) (beta)
// and the upstream S_c(m + e_q) (gamma, per row kind)
template <typename real>
__device__ __forceinline__ void bfl_coeffs(real eta, bool neu, bool up, real &al_v, real &al_F, real &be, real &ga_v,
                                           real &ga_F) {
    const real Dv = neu ? real(1) : real(-1), DF = -Dv;
    if (eta >= real(0.5)) {
        al_v = Dv / (real(2) * eta);
        al_F = DF / (real(2) * eta);
        be = real(1) - real(1) / (real(2) * eta);
        ga_v = ga_F = real(0);
    } else if (up) {
        al_v = real(2) * eta * Dv;
        al_F = real(2) * eta * DF;
        be = real(0);
        ga_v = (real(1) - real(2) * eta) * Dv;
        ga_F = (real(1) - real(2) * eta) * DF;
    } else {
        al_v = Dv;
        al_F = DF;
        be = ga_v = ga_F = real(0);
    }
}

template <typename real>
__device__ __forceinline__ void link_coeffs(const StepArgs<real> &a, const AdjArgs<real> &j, long long node,
                                            unsigned cut, int c, real &al_v, real &al_F, real &be, real &ga_v, real &ga_F) {
    const long long l = link_of(__ldg(a.lstart + node), cut, c);
    const real eta = (real)j.L.eta[l];
    const bool neu = j.bcs[j.L.bc[l]].kind != 0;
    const bool up = !((cut >> (c ^ 1)) & 1);
    bfl_coeffs<real>(eta, neu, up, al_v, al_F, be, ga_v, ga_F);
}

// dL/dS at node m (all Q*K values): the transpose of the gather applied to gbar (j.g_in)
template <typename real, int D>
__device__ __forceinline__ void adjoint_pull(const StepArgs<real> &a, const AdjArgs<real> &j, int node, int x, int y,
                                             int z, unsigned cut, real (&lam)[2 * D * (D + D * D)]) {
    constexpr int K = D + D * D, Q = 2 * D;
    const long long P = a.b.npad;
    const real *__restrict__ g = j.g_in;
    #pragma unroll
    for (int q = 0; q < Q; ++q) {
        #pragma unroll
        for (int k = 0; k < K; ++k) lam[q * K + k] = real(0);
        if (!((cut >> q) & 1)) {
            // streamed into m + e_q; and, if that node's link q is cut with eta < 1/2, its
            // reconstruction of direction q^1 reads S_q(m) as the upstream value
            const int mt = nbr(a.b, node, x, y, z, q);
            #pragma unroll
            for (int k = 0; k < K; ++k) lam[q * K + k] = g[(long long)(q * K + k) * P + mt];
            const unsigned cutt = __ldg(a.flags + mt) & kCutMask;
            if ((cutt >> q) & 1) {
                real al_v, al_F, be, ga_v, ga_F;
                link_coeffs<real>(a, j, mt, cutt, q, al_v, al_F, be, ga_v, ga_F);
                if (ga_v != real(0) || ga_F != real(0))
                    #pragma unroll
                    for (int k = 0; k < K; ++k)
                        lam[q * K + k] += (k < D ? ga_v : ga_F) * g[(long long)((q ^ 1) * K + k) * P + mt];
            }
        } else {
            // this node's reconstruction of q^1 reads S_q(m) as the outgoing value
            real al_v, al_F, be, ga_v, ga_F;
            link_coeffs<real>(a, j, node, cut, q, al_v, al_F, be, ga_v, ga_F);
            #pragma unroll
            for (int k = 0; k < K; ++k) lam[q * K + k] += (k < D ? al_v : al_F) * g[(long long)((q ^ 1) * K + k) * P + node];
        }
        if ((cut >> (q ^ 1)) & 1) {
            // this node's reconstruction of q reads S_q(m) as the incoming value
            real al_v, al_F, be, ga_v, ga_F;
            link_coeffs<real>(a, j, node, cut, q ^ 1, al_v, al_F, be, ga_v, ga_F);
            if (be != real(0))
                #pragma unroll
                for (int k = 0; k < K; ++k) lam[q * K + k] += be * g[(long long)(q * K + k) * P + node];
        }
    }
}

// forward gather of step n recomputed from the saved state (a.fsrc), with the Dirichlet closure
// data at time j.th (the values the link kernel formed after step n-1)
template <typename real, int D, int MODE>
__device__ __forceinline__ void gather_recompute(const StepArgs<real> &a, const AdjArgs<real> &j, int node, int x,
                                                 int y, int z, unsigned cut, real (&f)[2 * D * (D + D * D)]) {
    constexpr int K = D + D * D, Q = 2 * D;
    const long long P = a.b.npad;
    const real *__restrict__ fs = a.fsrc;
    if constexpr (MODE == 0) {
        #pragma unroll
        for (int q = 0; q < Q; ++q)
            #pragma unroll
            for (int k = 0; k < K; ++k) f[q * K + k] = fs[(long long)(q * K + k) * P + node];
        return;
    } else {
        const real c = a.c;
        #pragma unroll
        for (int q = 0; q < Q; ++q) {
            const int co = q ^ 1;  // cut direction whose closure supplies g_q
            if (!((cut >> co) & 1)) {
                const int src = nbr(a.b, node, x, y, z, co);
                #pragma unroll
                for (int k = 0; k < K; ++k) f[q * K + k] = fs[(long long)(q * K + k) * P + src];
            } else {
                const long long l = link_of(__ldg(a.lstart + node), cut, co);
                const BCD &bc = j.bcs[j.L.bc[l]];
                const int A = co >> 1;
                const real s = (co & 1) ? real(-1) : real(1);
                const double Xb[3] = {j.L.Xb[3 * l], j.L.Xb[3 * l + 1], j.L.Xb[3 * l + 2]};
                double vb[3];
                dirichlet_eval(bc, D, Xb, j.th, false, vb);
                real S[K];
                #pragma unroll
                for (int i = 0; i < D; ++i) {
                    S[i] = (real)vb[i] / real(D);
                    #pragma unroll
                    for (int B = 0; B < D; ++B) S[D + i * D + B] = (B == A) ? s * (real)vb[i] / c : real(0);
                }
                const real eta = (real)j.L.eta[l];
                const bool up = !((cut >> q) & 1);
                const int mu_ = up ? nbr(a.b, node, x, y, z, q) : node;
                #pragma unroll
                for (int k = 0; k < K; ++k) {
                    const real Dk = (k < D) ? real(-1) : real(1);  // D_D = diag(-I, I)
                    const real fo = fs[(long long)(co * K + k) * P + node];
                    const real fi = fs[(long long)(q * K + k) * P + node];
                    if (eta >= real(0.5)) {
                        f[q * K + k] = (Dk * fo + S[k]) / (real(2) * eta) + (real(1) - real(1) / (real(2) * eta)) * fi;
                    } else {
                        const real fu = up ? fs[(long long)(co * K + k) * P + mu_] : fo;
                        f[q * K + k] = Dk * (real(2) * eta * fo + (real(1) - real(2) * eta) * fu) + S[k];
                    }
                }
            }
        }
    }
}

// block sum of a per-thread 3-vector into bbar (one atomic per warp and component)
__device__ __forceinline__ void add_bbar(double *bbar, double b0, double b1, double b2) {
    #pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        b0 += __shfl_down_sync(0xffffffffu, b0, o);
        b1 += __shfl_down_sync(0xffffffffu, b1, o);
        b2 += __shfl_down_sync(0xffffffffu, b2, o);
    }
    if ((threadIdx.x & 31) == 0) {
        if (b0 != 0.0) atomicAdd(bbar, b0);
        if (b1 != 0.0) atomicAdd(bbar + 1, b1);
        if (b2 != 0.0) atomicAdd(bbar + 2, b2);
    }
}

// Seed of the sweep at the current state (after N steps): u(t_N) = u*^N + dt/2 v^N with v^N from
// the gather of the stored state, so dL/dv = dt/2 dL/du and gbar carries dL/dv through the
// recovery; dL/du* = dL/du for every earlier step.
template <typename real, int D>
__global__ void __launch_bounds__(128) k_adj_seed(const StepArgs<real> a, const AdjArgs<real> j, double *lu) {
    constexpr int K = D + D * D, Q = 2 * D;
    const int sgi = blockIdx.x * 4 + (threadIdx.x >> 5);
    double bb[3] = {0.0, 0.0, 0.0};
    if (sgi < a.nseg) {
        const int2 sg = __ldg(&a.seg[sgi]);
        const int lane = threadIdx.x & 31;
        const int x = sg.x - sg.y * a.b.nx + lane;
        const int node = sg.x + lane;
        const uint8_t fl = x < a.b.nx ? __ldg(a.flags + node) : (uint8_t)0;
        if (fl & kActive) {
            const long long P = a.b.npad;
            const double hdt = 0.5 * (double)a.dt;
            const double inv_damp = 1.0 / (1.0 + hdt * (double)a.gamma);
            #pragma unroll
            for (int i = 0; i < D; ++i) {
                const double gu = j.grad_u[i * j.nbox + node];
                lu[i * P + node] = gu;
                const double vbar = hdt * gu;
                bb[i] = vbar * hdt * inv_damp;
                #pragma unroll
                for (int q = 0; q < Q; ++q) j.g_out[(long long)(q * K + i) * P + node] = (real)(vbar * inv_damp);
            }
            #pragma unroll
            for (int q = 0; q < Q; ++q)
                #pragma unroll
                for (int k = D; k < K; ++k) j.g_out[(long long)(q * K + k) * P + node] = real(0);
        }
    }
    add_bbar(j.bbar, bb[0], bb[1], D == 3 ? bb[2] : 0.0);
}

// Reverse of step n: lambda* = pull of gbar(n+1) (the adjoint of step n+1's gather), the forward
// quantities of step n recomputed from the saved state before it, then gbar(n) (MODE 1 only: the
// first step has no gather to reverse) and the mu and b gradients.
template <typename real, int D, int MODE>
__global__ void __launch_bounds__(128) k_adj_step(const StepArgs<real> a, const AdjArgs<real> j) {
    constexpr int K = D + D * D, Q = 2 * D;
    const int sgi = blockIdx.x * 4 + (threadIdx.x >> 5);
    double bb[3] = {0.0, 0.0, 0.0};
    if (sgi < a.nseg) {
        const int2 sg = __ldg(&a.seg[sgi]);
        const int lane = threadIdx.x & 31;
        const int x = sg.x - sg.y * a.b.nx + lane;
        const int node = sg.x + lane;
        const uint8_t fl = x < a.b.nx ? __ldg(a.flags + node) : (uint8_t)0;
        if (fl & kActive) {
            const int y = sg.y % a.b.ny, z = sg.y / a.b.ny;
            const unsigned cut = fl & kCutMask;
            const long long P = a.b.npad;
            real lam[Q * K], f[Q * K];
            adjoint_pull<real, D>(a, j, node, x, y, z, cut, lam);
            gather_recompute<real, D, MODE>(a, j, node, x, y, z, cut, f);
            // forward recovery and stress
            const real hdt = real(0.5) * a.dt;
            const real inv_damp = real(1) / (real(1) + hdt * a.gamma);
            real v[D], X[D * D], F[D * D], Pk[D * D];
            #pragma unroll
            for (int k = 0; k < K; ++k) {
                real s = f[k];
                #pragma unroll
                for (int q = 1; q < Q; ++q) s += f[q * K + k];
                if (k < D) v[k] = (s + hdt * a.bf[k]) * inv_damp;
                else X[k - D] = s;
            }
            #pragma unroll
            for (int k = 0; k < D * D; ++k) F[k] = X[k] + ((kShifted<real> && (k / D == k % D)) ? real(1) : real(0));
            real mu, lm;
            node_material(a, node, mu, lm);
            piola<real, D>(F, mu, lm, Pk);
            // reverse of collision, equilibrium and quadrature
            const real Dc = real(D) / a.c;
            const real w = a.omega / real(2 * D);
            const real src = a.dt * (real(2) - a.omega) / real(4 * D);
            real vbar[D], Pbar[D * D], Xbar[D * D];
            #pragma unroll
            for (int i = 0; i < D; ++i) {
                real sv = 0, sF = 0;
                #pragma unroll
                for (int q = 0; q < Q; ++q) {
                    const real sq = (q & 1) ? real(-1) : real(1);
                    sv += lam[q * K + i];
                    sF += sq * lam[q * K + D + i * D + (q >> 1)];
                }
                vbar[i] = (real)(a.dt * j.lu[i * P + node]) + (w - src * a.gamma) * sv - w * Dc * sF;
                bb[i] = (double)(src * sv + vbar[i] * hdt * inv_damp);
                #pragma unroll
                for (int A = 0; A < D; ++A)
                    Pbar[i * D + A] = -w * Dc * (lam[(2 * A) * K + i] - lam[(2 * A + 1) * K + i]);
            }
            dpiola_t<real, D>(F, Pbar, mu, lm, Xbar);
            real C[D * D];
            cofactor<real, D>(F, C);
            const real J = det<real, D>(F);
            real dmu = 0;
            #pragma unroll
            for (int k = 0; k < D * D; ++k) {
                real s = 0;
                #pragma unroll
                for (int q = 0; q < Q; ++q) s += lam[q * K + D + k];
                Xbar[k] += w * s;
                dmu += Pbar[k] * (F[k] - C[k] / J);  // dP/dmu = F - F^-T
            }
            j.mubar[node] += (double)dmu;
            if constexpr (MODE == 1) {
                const real om1 = real(1) - a.omega;
                #pragma unroll
                for (int q = 0; q < Q; ++q)
                    #pragma unroll
                    for (int k = 0; k < K; ++k)
                        j.g_out[(long long)(q * K + k) * P + node] =
                            om1 * lam[q * K + k] + (k < D ? vbar[k] * inv_damp : Xbar[k - D]);
            }
        }
    }
    add_bbar(j.bbar, bb[0], bb[1], D == 3 ? bb[2] : 0.0);
}

}  // namespace tlv
