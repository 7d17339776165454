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

// windows add their share of dL/db into one of kAdjSlots slots (window index modulo kAdjSlots), so
// that the atomics of a step spread over distinct addresses; the slots are summed at the end
constexpr int kAdjSlots = 4096;

template <typename real> struct AdjArgs {
    const real *mom;     // X = F (or F - I when shifted) of the step being reversed (D*D planes)
    const real *g_in;    // gbar of the step after this one (Q*K planes)
    real *g_out;         // gbar of this step
    double *mubar;       // dL/dmu per node
    double *bslot;       // dL/db: kAdjSlots slots of 4 values
    const real *lu;      // dL/du* (D planes, box order over npad)
    const double *grad_u;  // seed: dL/du(t_N), D * nbox values
    const real *coef;    // per cut link: alpha_v, beta, gamma_v, 0 (k_adj_coef)
    real *side;          // per cut link (m, c): gbar_{c^1}(m) of the last reversed step (K values)
    long long nbox;
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


// derivatives of the closure value R of a cut link with respect to S_c(m) (alpha), S_q(m) (beta)
// and the upstream S_c(m + e_q) (gamma), for the velocity rows; the F rows carry -alpha and -gamma
// (the sign D_k of the reflected population is opposite in the two row kinds)
template <typename real>
__device__ __forceinline__ void bfl_coeffs(real eta, bool neu, bool up, real &al, real &be, real &ga) {
    const real Dv = neu ? real(1) : real(-1);
    if (eta >= real(0.5)) {
        al = Dv / (real(2) * eta);
        be = real(1) - real(1) / (real(2) * eta);
        ga = real(0);
    } else if (up) {
        al = real(2) * eta * Dv;
        be = real(0);
        ga = (real(1) - real(2) * eta) * Dv;
    } else {
        al = Dv;
        be = ga = real(0);
    }
}

// per cut link l = (node m, cut direction c): (alpha, beta, gamma, 0) of its closure.  Geometry
// only; built at the start of a sweep.
template <typename real>
__global__ void __launch_bounds__(256) k_adj_coef(const uint8_t *__restrict__ flags, const int *__restrict__ lnode,
                                                  const int *__restrict__ lq, const int *__restrict__ lbc,
                                                  const double *__restrict__ leta, const BCD *__restrict__ bcs,
                                                  long long ncut, real *__restrict__ coef) {
    for (long long l = blockIdx.x * (long long)blockDim.x + threadIdx.x; l < ncut; l += (long long)gridDim.x * blockDim.x) {
        const int c = lq[l];
        const unsigned cut = flags[lnode[l]] & kCutMask;
        real al, be, ga;
        bfl_coeffs<real>((real)leta[l], bcs[lbc[l]].kind != 0, !((cut >> (c ^ 1)) & 1), al, be, ga);
        coef[4 * l] = al;
        coef[4 * l + 1] = be;
        coef[4 * l + 2] = ga;
        coef[4 * l + 3] = real(0);
    }
}

// warp sum of a per-lane 3-vector, added by lane 0 into the window's dL/db slot
template <typename acc>
__device__ __forceinline__ void add_bslot(double *bslot, int sgi, acc b0, acc b1, acc b2) {
    #pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        b0 += __shfl_down_sync(0xffffffffu, b0, o);
        b1 += __shfl_down_sync(0xffffffffu, b1, o);
        b2 += __shfl_down_sync(0xffffffffu, b2, o);
    }
    if ((threadIdx.x & 31) == 0) {
        double *s = bslot + 4 * (sgi & (kAdjSlots - 1));
        if (b0 != acc(0)) atomicAdd(s, (double)b0);
        if (b1 != acc(0)) atomicAdd(s + 1, (double)b1);
        if (b2 != acc(0)) atomicAdd(s + 2, (double)b2);
    }
}

// Stores gbar of the step at node m: om1 lambda*_q + T, where T (dL/dv / (1 + gamma dt/2) in the
// velocity rows, dL/dX in the F rows) is the same for every q.  Where the cut link (m, c) reads the
// upstream population S_c(m - e_c) (gamma != 0), plane c at m also carries gamma gbar_{c^1}(m):
// the pull of m - e_c is the plane's only reader, and that is where the term belongs.  The side
// buffer keeps gbar_{c^1}(m) of every cut link for the closure terms of the next reverse step
// (plane c^1 of such a node is never folded: a link with gamma != 0 has no cut link opposite it).
template <typename real, int D, typename Lam>
__device__ __forceinline__ void adjoint_store(const AdjArgs<real> &j, long long P, long long node, unsigned cut,
                                              long long l0, Lam L, real om1, const real (&T)[D + D * D]) {
    constexpr int K = D + D * D, Q = 2 * D;
    #pragma unroll
    for (int q = 0; q < Q; ++q) {
        real ga = real(0);
        if ((cut >> q) & 1) ga = j.coef[4 * link_of(l0, cut, q) + 2];
        if (ga == real(0)) {
            #pragma unroll
            for (int k = 0; k < K; ++k) j.g_out[(long long)(q * K + k) * P + node] = om1 * L(q, k) + T[k];
        } else {
            #pragma unroll
            for (int k = 0; k < K; ++k)
                j.g_out[(long long)(q * K + k) * P + node] =
                    om1 * L(q, k) + T[k] + (k < D ? ga : -ga) * (om1 * L(q ^ 1, k) + T[k]);
        }
        if ((cut >> (q ^ 1)) & 1) {
            real s[K];
            #pragma unroll
            for (int k = 0; k < K; ++k) s[k] = om1 * L(q, k) + T[k];
            vstore<K>(j.side + link_of(l0, cut, q ^ 1) * K, s);
        }
    }
}

// Seed of the sweep at the current state (after N steps): u(t_N) = u*^N + dt/2 v^N with v^N from
// the gather of the stored state, so dL/dv = dt/2 dL/du and gbar carries dL/dv through the
// recovery; dL/du* = dL/du for every earlier step.
template <typename real, int D>
__global__ void __launch_bounds__(128) k_adj_seed(const StepArgs<real> a, const AdjArgs<real> j, real *lu) {
    constexpr int K = D + D * D;
    const int sgi = blockIdx.x * 4 + (threadIdx.x >> 5);
    real bb[3] = {real(0), real(0), real(0)};
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
            real T[K];
            #pragma unroll
            for (int i = 0; i < D; ++i) {
                const double gu = j.grad_u[i * j.nbox + node];
                lu[i * P + node] = (real)gu;
                const double vbar = hdt * gu;
                bb[i] = (real)(vbar * hdt * inv_damp);
                T[i] = (real)(vbar * inv_damp);
            }
            #pragma unroll
            for (int k = D; k < K; ++k) T[k] = real(0);
            const unsigned cut = fl & kCutMask;
            const long long l0 = cut ? (long long)__ldg(a.lstart + node) : 0;
            adjoint_store<real, D>(j, P, node, cut, l0, [](int, int) { return real(0); }, real(0), T);
        }
    }
    add_bslot<real>(j.bslot, sgi, bb[0], bb[1], bb[2]);
}

// dL/dS at node m (all Q*K values): the transpose of the gather applied to gbar (j.g_in).  Interior
// links pull the next step's gbar from m + e_q (the upstream closure terms are folded into those
// planes); a cut link's own closure reads S_c(m) (alpha) and S_{c^1}(m) (beta) against gbar_{c^1}(m),
// which the side buffer holds.
template <typename real, int D>
__device__ __forceinline__ void adjoint_pull(const StepArgs<real> &a, const AdjArgs<real> &j, int node, int x, int y,
                                             int z, unsigned cut, long long l0, real (&lam)[2 * D * (D + D * D)]) {
    constexpr int K = D + D * D, Q = 2 * D;
    const long long P = a.b.npad;
    #pragma unroll
    for (int q = 0; q < Q; ++q) {
        if (!((cut >> q) & 1)) {
            const int mt = nbr(a.b, node, x, y, z, q);
            #pragma unroll
            for (int k = 0; k < K; ++k) lam[q * K + k] = j.g_in[(long long)(q * K + k) * P + mt];
        } else {
            const long long l = link_of(l0, cut, q);
            const real al = j.coef[4 * l];
            real s[K];
            vload<K>(j.side + l * K, s);
            #pragma unroll
            for (int k = 0; k < K; ++k) lam[q * K + k] = (k < D ? al : -al) * s[k];
        }
        if ((cut >> (q ^ 1)) & 1) {
            const long long l = link_of(l0, cut, q ^ 1);
            const real be = j.coef[4 * l + 1];
            if (be != real(0)) {
                real s[K];
                vload<K>(j.side + l * K, s);
                #pragma unroll
                for (int k = 0; k < K; ++k) lam[q * K + k] += be * s[k];
            }
        }
    }
}

// the local product of the reverse step at one node: lambda* through the accessor L(q, k), F of
// the step; stores gbar of the step and accumulates the mu and b gradients
template <typename real, int D, typename Lam>
__device__ __forceinline__ void adjoint_local(const StepArgs<real> &a, const AdjArgs<real> &j, long long node,
                                              unsigned cut, long long l0, Lam L, const real F[D * D], real mu, real lm,
                                              const real lu[D], real bb[3]) {
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
        vbar[i] = a.dt * lu[i] + (w - src * a.gamma) * sv - w * Dc * sF;
        bb[i] = src * sv + vbar[i] * hdt * inv_damp;
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
    atomicAdd(j.mubar + node, (double)dmu);  // one writer per node and step: no contention
    real T[K];
    #pragma unroll
    for (int i = 0; i < D; ++i) T[i] = vbar[i] * inv_damp;
    #pragma unroll
    for (int k = 0; k < D * D; ++k) T[D + k] = Xbar[k];
    adjoint_store<real, D>(j, a.b.npad, node, cut, l0, L, real(1) - a.omega, T);
}

// Reverse of step n: lambda* = pull of gbar(n+1) (the adjoint of step n+1's gather), then gbar(n)
// and the mu and b gradients from the recorded F of step n
template <typename real, int D>
__global__ void __launch_bounds__(128) k_adj_step(const StepArgs<real> a, const AdjArgs<real> j) {
    constexpr int K = D + D * D, Q = 2 * D;
    const int sgi = blockIdx.x * 4 + (threadIdx.x >> 5);
    real bb[3] = {real(0), real(0), real(0)};
    if (sgi < a.nseg) {
        const int2 sg = __ldg(&a.seg[sgi]);
        const int lane = threadIdx.x & 31;
        const int x = sg.x - sg.y * a.b.nx + lane;
        const int node = sg.x + lane;
        const uint8_t fl = x < a.b.nx ? __ldg(a.flags + node) : (uint8_t)0;
        if (fl & kActive) {
            const int y = sg.y % a.b.ny, z = sg.y / a.b.ny;
            const long long P = a.b.npad;
            const unsigned cut = fl & kCutMask;
            const long long l0 = cut ? (long long)__ldg(a.lstart + node) : 0;
            real lam[Q * K], F[D * D];
            adjoint_pull<real, D>(a, j, node, x, y, z, cut, l0, lam);
            #pragma unroll
            for (int k = 0; k < D * D; ++k)
                F[k] = j.mom[(long long)k * P + node] + ((kShifted<real> && (k / D == k % D)) ? real(1) : real(0));
            real mu, lm;
            node_material(a, node, mu, lm);
            real lu[D];
            #pragma unroll
            for (int i = 0; i < D; ++i) lu[i] = j.lu[i * P + node];
            adjoint_local<real, D>(a, j, node, cut, l0, [&](int q, int k) { return lam[q * K + k]; }, F, mu, lm, lu, bb);
        }
    }
    add_bslot<real>(j.bslot, sgi, bb[0], bb[1], bb[2]);
}

// ---------------------------------------------------------------------------------------------
// FP32 reverse step with bulk-copy staging (rows a multiple of 16): per warp one 32-node window;
// the stage holds the pulled gbar of the next step, g(q, m + e_q) (the forward's boxes one link the
// other way).  Everything else a lane reads (flags, link offset, F, dL/du*, the material, and for
// cut links their coefficients and side rows) is fetched while the copies are in flight, so no
// lane waits on global memory after the stage lands.
// ---------------------------------------------------------------------------------------------

template <int D> struct AdjLayout {
    using L = TmaLayout<D>;
    static constexpr int bytes = L::warp_bytes;
    static constexpr int tx = L::tx_bytes;
    // element of lane 0 inside the pulled boxes of +-x: g(q, m + e_q)
    __device__ static constexpr int g_lane0(int q) { return q == 0 ? 5 : (q == 1 ? 3 : 0); }
};

template <int D> __device__ __forceinline__ float &stG(char *w, int q, int k, int lane) {
    using L = TmaLayout<D>;
    return reinterpret_cast<float *>(w + L::slot(q))[k * L::width(q) + AdjLayout<D>::g_lane0(q) + lane];
}

__device__ __forceinline__ void prefetch_l1(const void *p) { asm volatile("prefetch.global.L1 [%0];" ::"l"(p)); }

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
    const uint8_t fl = inrow ? __ldg(a.flags + node) : (uint8_t)0;
    const unsigned cut = fl & kCutMask;
    const long long l0 = cut ? (long long)__ldg(a.lstart + node) : 0;
    float lu[D], F[D * D];
    #pragma unroll
    for (int i = 0; i < D; ++i) lu[i] = j.lu[i * P + node];
    #pragma unroll
    for (int k = 0; k < D * D; ++k) F[k] = j.mom[(long long)k * P + node] + ((k / D == k % D) ? 1.0f : 0.0f);
    float mu = a.mu, lm = a.lam;
    if (inrow) node_material(a, node, mu, lm);
    if (cut) {
        #pragma unroll
        for (int q = 0; q < Q; ++q)
            if ((cut >> q) & 1) {
                const long long l = link_of(l0, cut, q);
                prefetch_l1(j.coef + 4 * l);
                prefetch_l1(j.side + l * K);
                prefetch_l1(j.side + l * K + K - 1);
            }
    }
    __syncwarp();
    if (!__all_sync(0xffffffffu, mbar_wait_bounded(bar, 0, a.spin))) {
        if (lane == 0) set_status(a.status, kStTimeout);
        mbar_wait_bounded(bar, 0);  // let the copies in flight land before the warp exits
        return;
    }
    // lanes past the row end belong to the next row: they only join the warp's sum at the end
    float bb[3] = {0.0f, 0.0f, 0.0f};
    if (fl & kActive) {
        if (a.b.per[0]) {  // periodic x ends: the aligned boxes do not wrap
            const float *__restrict__ gin = j.g_in;
            if (x == a.b.nx - 1 && !(cut & 1))
                for (int k = 0; k < K; ++k) stG<D>(smem, 0, k, lane) = gin[(long long)(0 * K + k) * P + node - (a.b.nx - 1)];
            if (x == 0 && !((cut >> 1) & 1))
                for (int k = 0; k < K; ++k) stG<D>(smem, 1, k, lane) = gin[(long long)(1 * K + k) * P + node + a.b.nx - 1];
        }
        // transposed gather: the staged g(q, m + e_q) is right across interior links; a cut link's
        // own closure terms come from its side row
        if (cut) {
            #pragma unroll 1
            for (int q = 0; q < Q; ++q) {
                float s[K];
                if ((cut >> q) & 1) {
                    const long long l = link_of(l0, cut, q);
                    const float al = j.coef[4 * l];
                    vload<K>(j.side + l * K, s);
                    #pragma unroll
                    for (int k = 0; k < K; ++k) stG<D>(smem, q, k, lane) = (k < D ? al : -al) * s[k];
                }
                if ((cut >> (q ^ 1)) & 1) {
                    const long long l = link_of(l0, cut, q ^ 1);
                    const float be = j.coef[4 * l + 1];
                    if (be != 0.0f) {
                        vload<K>(j.side + l * K, s);
                        #pragma unroll
                        for (int k = 0; k < K; ++k) stG<D>(smem, q, k, lane) += be * s[k];
                    }
                }
            }
        }
        adjoint_local<float, D>(a, j, node, cut, l0, [&](int q, int k) { return stG<D>(smem, q, k, lane); }, F, mu,
                                lm, lu, bb);
    } else if (inrow) {  // whole sectors: inactive nodes of the window get zeros
        #pragma unroll
        for (int q = 0; q < Q; ++q)
            #pragma unroll
            for (int k = 0; k < K; ++k) j.g_out[(long long)(q * K + k) * P + node] = 0.0f;
    }
    add_bslot<float>(j.bslot, sgi, bb[0], bb[1], bb[2]);
}

}  // namespace tlv
