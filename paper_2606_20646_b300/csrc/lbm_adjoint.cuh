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
// (n-1) evaluates at its own node before its local product.  f*_q is linear in g, v and X except
// through P(F), so the local product needs only F of step n: the recomputation of the forward
// records it (lbm_step_moments) and the reverse step reads it instead of gathering the state.  The
// stress derivative uses the tangent's major symmetry: the product with C^T equals the directional
// derivative along Pbar.
#pragma once

#include "lbm_kernels.cuh"
#include "lbm_tma.cuh"

namespace tlv {

template <typename real> struct AdjArgs {
    const real *mom;     // X = F (or F - I when shifted) of the step being reversed (D*D planes)
    const real *g_in;    // gbar of the step after this one (Q*K planes)
    real *g_out;         // gbar of this step
    double *mubar;       // dL/dmu per node
    double *bbar;        // dL/db (3)
    const double *lu;    // dL/du* (D planes, box order over npad)
    const double *grad_u;  // seed: dL/du(t_N), D * nbox values
    long long nbox;
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

// the local product of the reverse step at one node: lambda* through the accessor L(q, k), F of
// the step; writes gbar of the step to gout and accumulates the mu and b gradients
template <typename real, int D, typename Lam>
__device__ __forceinline__ void adjoint_local(const StepArgs<real> &a, const AdjArgs<real> &j, long long node, Lam L,
                                              const real F[D * D], real mu, real lm, const double lu[D], double bb[3],
                                              real *gout) {
    constexpr int K = D + D * D, Q = 2 * D;
    const real hdt = real(0.5) * a.dt;
    const real inv_damp = real(1) / (real(1) + hdt * a.gamma);
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
            sv += L(q, i);
            sF += sq * L(q, D + i * D + (q >> 1));
        }
        vbar[i] = (real)(a.dt * lu[i]) + (w - src * a.gamma) * sv - w * Dc * sF;
        bb[i] = (double)(src * sv + vbar[i] * hdt * inv_damp);
        #pragma unroll
        for (int A = 0; A < D; ++A) Pbar[i * D + A] = -w * Dc * (L(2 * A, i) - L(2 * A + 1, i));
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
        for (int q = 0; q < Q; ++q) s += L(q, D + k);
        Xbar[k] += w * s;
        dmu += Pbar[k] * (F[k] - C[k] / J);  // dP/dmu = F - F^-T
    }
    j.mubar[node] += (double)dmu;
    const real om1 = real(1) - a.omega;
    const long long P = a.b.npad;
    #pragma unroll
    for (int q = 0; q < Q; ++q)
        #pragma unroll
        for (int k = 0; k < K; ++k)
            gout[(long long)(q * K + k) * P + node] = om1 * L(q, k) + (k < D ? vbar[k] * inv_damp : Xbar[k - D]);
}

// Reverse of step n: lambda* = pull of gbar(n+1) (the adjoint of step n+1's gather), then gbar(n)
// and the mu and b gradients from the recorded F of step n
template <typename real, int D>
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
            const long long P = a.b.npad;
            real lam[Q * K], F[D * D];
            adjoint_pull<real, D>(a, j, node, x, y, z, fl & kCutMask, lam);
            #pragma unroll
            for (int k = 0; k < D * D; ++k)
                F[k] = j.mom[(long long)k * P + node] + ((kShifted<real> && (k / D == k % D)) ? real(1) : real(0));
            real mu, lm;
            node_material(a, node, mu, lm);
            double lu[D];
            #pragma unroll
            for (int i = 0; i < D; ++i) lu[i] = j.lu[i * P + node];
            adjoint_local<real, D>(a, j, node, [&](int q, int k) { return lam[q * K + k]; }, F, mu, lm, lu, bb,
                                   j.g_out);
        }
    }
    add_bbar(j.bbar, bb[0], bb[1], D == 3 ? bb[2] : 0.0);
}

// ---------------------------------------------------------------------------------------------
// FP32 reverse step with bulk-copy staging (rows a multiple of 16): per warp one 32-node window;
// the stage holds the pulled gbar of the next step, g(q, m + e_q) (the forward's boxes one link the
// other way), and the flag bytes.  Cut links are applied from global memory by the lanes that
// have them, as in the plain kernel.
// ---------------------------------------------------------------------------------------------

template <int D> struct AdjLayout {
    using L = TmaLayout<D>;
    static constexpr int fl_off = L::warp_bytes;
    static constexpr int bytes = fl_off + 128;
    static constexpr int tx = L::tx_bytes + 32;
    // element of lane 0 inside the pulled boxes of +-x: g(q, m + e_q)
    __device__ static constexpr int g_lane0(int q) { return q == 0 ? 5 : (q == 1 ? 3 : 0); }
};

template <int D> __device__ __forceinline__ float &stG(char *w, int q, int k, int lane) {
    using L = TmaLayout<D>;
    return reinterpret_cast<float *>(w + L::slot(q))[k * L::width(q) + AdjLayout<D>::g_lane0(q) + lane];
}

template <int D>
__global__ void __launch_bounds__(32, 16) k_adj_step_tma(const StepArgs<float> a, const AdjArgs<float> j,
                                                        const __grid_constant__ TmaMaps maps) {
    using L = TmaLayout<D>;
    using AL = AdjLayout<D>;
    constexpr int K = D + D * D, Q = 2 * D;
    extern __shared__ __align__(128) char smem[];
    const int lane = threadIdx.x;
    const int sgi = blockIdx.x;
    if (sgi >= a.nseg) return;
    uint64_t *const bar = reinterpret_cast<uint64_t *>(smem + AL::bytes);
    const int2 sg = __ldg(&a.seg[sgi]);
    const int y = sg.y % a.b.ny, z = sg.y / a.b.ny, x0 = sg.x - sg.y * a.b.nx;
    if (lane == 0) {
        mbar_init(bar, 1);
        mbar_fence_init();
        mbar_arrive_expect_tx(bar, AL::tx);
        tma_load_2d(smem + AL::fl_off, &maps.flags, bar, x0, sg.y);
        #pragma unroll
        for (int q = 0; q < Q; ++q) {
            const int A = q >> 1, s = (q & 1) ? -1 : 1;
            int st;  // the window of gbar at m + s e_A
            if (A == 0) {
                st = sg.x - 4;
            } else {
                const int n = A == 1 ? a.b.ny : a.b.nz;
                int cg = (A == 1 ? y : z) + s;
                if (a.b.per[A]) cg = cg < 0 ? cg + n : (cg >= n ? cg - n : cg);
                st = A == 1 ? (z * a.b.ny + cg) * a.b.nx + x0 : (cg * a.b.ny + y) * a.b.nx + x0;
            }
            tma_load_2d(smem + L::slot(q), A == 0 ? &maps.wide : &maps.narrow, bar, st, q * K);
        }
    }
    const int x = x0 + lane;
    const int node = sg.x + lane;
    const long long P = a.b.npad;
    const bool inrow = x < a.b.nx;
    // per-node inputs fetched while the copies are in flight (planes hold a spare window past the
    // box, so every lane's index is in range)
    double lu[D];
    float F[D * D];
    #pragma unroll
    for (int i = 0; i < D; ++i) lu[i] = inrow ? j.lu[i * P + node] : 0.0;
    #pragma unroll
    for (int k = 0; k < D * D; ++k) F[k] = j.mom[(long long)k * P + node] + ((k / D == k % D) ? 1.0f : 0.0f);
    float mu = a.mu, lm = a.lam;
    if (inrow) node_material(a, node, mu, lm);
    const bool per_ = a.b.per[0] | a.b.per[1] | a.b.per[2];
    const int yy = per_ ? y : 0, zz = per_ ? z : 0;
    unsigned ncut[Q];  // cut masks of the axis neighbours
    #pragma unroll
    for (int q = 0; q < Q; ++q) {
        long long mt = nbr(a.b, node, x, yy, zz, q);
        mt = mt < 0 ? 0 : (mt >= P ? P - 1 : mt);
        ncut[q] = inrow ? (__ldg(a.flags + mt) & kCutMask) : 0u;
    }
    __syncwarp();
    if (!__all_sync(0xffffffffu, mbar_wait_bounded(bar, 0))) {
        if (lane == 0) set_status(a.status, kStTimeout);
        mbar_wait_bounded(bar, 0);  // let the copies in flight land before the warp exits
        return;
    }
    // lanes past the row end belong to the next row: they only join the warp's sum at the end
    const uint8_t fl = inrow ? reinterpret_cast<const uint8_t *>(smem + AL::fl_off)[lane] : (uint8_t)0;
    double bb[3] = {0.0, 0.0, 0.0};
    if (fl & kActive) {
        const unsigned cut = fl & kCutMask;
        const float *__restrict__ gin = j.g_in;
        if (a.b.per[0]) {  // periodic x ends: the aligned boxes do not wrap
            if (x == a.b.nx - 1 && !(cut & 1))
                for (int k = 0; k < K; ++k) stG<D>(smem, 0, k, lane) = gin[(long long)(0 * K + k) * P + node - (a.b.nx - 1)];
            if (x == 0 && !((cut >> 1) & 1))
                for (int k = 0; k < K; ++k) stG<D>(smem, 1, k, lane) = gin[(long long)(1 * K + k) * P + node + a.b.nx - 1];
        }
        // transposed gather: the staged g(q, m + e_q) is right across interior links; fix the rest
        #pragma unroll 1
        for (int q = 0; q < Q; ++q) {
            float al_v, al_F, be, ga_v, ga_F;
            if ((cut >> q) & 1) {
                link_coeffs<float>(a, j, node, cut, q, al_v, al_F, be, ga_v, ga_F);
                for (int k = 0; k < K; ++k)
                    stG<D>(smem, q, k, lane) = (k < D ? al_v : al_F) * gin[(long long)((q ^ 1) * K + k) * P + node];
            } else if ((ncut[q] >> q) & 1) {
                const int mt = nbr(a.b, node, x, yy, zz, q);
                link_coeffs<float>(a, j, mt, ncut[q], q, al_v, al_F, be, ga_v, ga_F);
                if (ga_v != 0.0f || ga_F != 0.0f)
                    for (int k = 0; k < K; ++k)
                        stG<D>(smem, q, k, lane) += (k < D ? ga_v : ga_F) * gin[(long long)((q ^ 1) * K + k) * P + mt];
            }
            if ((cut >> (q ^ 1)) & 1) {
                link_coeffs<float>(a, j, node, cut, q ^ 1, al_v, al_F, be, ga_v, ga_F);
                if (be != 0.0f)
                    for (int k = 0; k < K; ++k) stG<D>(smem, q, k, lane) += be * gin[(long long)(q * K + k) * P + node];
            }
        }
        adjoint_local<float, D>(a, j, node, [&](int q, int k) { return stG<D>(smem, q, k, lane); }, F, mu, lm, lu, bb,
                                j.g_out);
    } else if (inrow) {  // whole sectors: inactive nodes of the window get zeros
        #pragma unroll
        for (int q = 0; q < Q; ++q)
            #pragma unroll
            for (int k = 0; k < K; ++k) j.g_out[(long long)(q * K + k) * P + node] = 0.0f;
    }
    add_bbar(j.bbar, bb[0], bb[1], D == 3 ? bb[2] : 0.0);
}

}  // namespace tlv
