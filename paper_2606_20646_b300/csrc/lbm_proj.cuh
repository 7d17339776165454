// Compatibility projection of the displacement accumulators (Sec. 3.5): normal-equation residual,
// damped-Jacobi sweeps, gauge reduction, the repair of the projection step's collision and the
// final reset.  The node and link arithmetic it calls is in lbm_kernels.cuh.
#pragma once

#include "lbm_kernels.cuh"

namespace tlv {

// =============================================================================================
// compatibility projection (Sec. 3.5), FP64 accumulation
// =============================================================================================

template <typename real> struct ProjArgs {
    Box b;
    const int2 *seg;
    int nseg;
    const uint8_t *flags;
    const uint8_t *dmask;
    const int *lstart;
    LinkGeom<real> L;
    const BCD *bcs;
    const real *Gst;
    const real *u0;    // warm start (displacement-accumulator layout: FP64 planes or FP32 pairs)
    // per node (r_1..r_D, w) with w = beta/deg, 4 values: residual at the warm start.  The FP32
    // forms use spare slots for the node's cut-direction bits (bit pattern of an unsigned): in 2D
    // the residual's fourth value, in 3D the fourth value of the correction d
    real *resid;
    double t, beta;
    int *status;
};

template <int N, typename real> struct VecT;
template <> struct VecT<4, float> { using T = float4; };
template <> struct VecT<2, float> { using T = float2; };

template <int N, typename real> __device__ __forceinline__ void ld_vec(const real *p, real *d) {
    if constexpr (sizeof(real) == 4) {
        const auto t = __ldg(reinterpret_cast<const typename VecT<N, float>::T *>(p));
        d[0] = t.x; d[1] = t.y;
        if constexpr (N == 4) { d[2] = t.z; d[3] = t.w; }
    } else {
        #pragma unroll
        for (int i = 0; i < N / 2; ++i) {
            const double2 t = __ldg(reinterpret_cast<const double2 *>(p) + i);
            d[2 * i] = t.x; d[2 * i + 1] = t.y;
        }
    }
}

template <int N, typename real> __device__ __forceinline__ void st_vec(real *p, const real *d) {
    if constexpr (sizeof(real) == 4) {
        if constexpr (N == 4) *reinterpret_cast<float4 *>(p) = make_float4(d[0], d[1], d[2], d[3]);
        else *reinterpret_cast<float2 *>(p) = make_float2(d[0], d[1]);
    } else {
        #pragma unroll
        for (int i = 0; i < N / 2; ++i) reinterpret_cast<double2 *>(p)[i] = make_double2(d[2 * i], d[2 * i + 1]);
    }
}

// node weight of the normal equations: active axis neighbours plus Dirichlet boundary edges
__device__ __forceinline__ int proj_degree(int D, unsigned cut, uint8_t dm) {
    return (2 * D - __popc(cut & ((1u << (2 * D)) - 1u))) + __popc((unsigned)dm);
}

#define TLV_NODE_PROLOGUE(a)                                      \
    const int sgi = blockIdx.x * 4 + (threadIdx.x >> 5);          \
    if (sgi >= (a).nseg) return;                                  \
    const int2 sg = __ldg(&(a).seg[sgi]);                         \
    const int lane = threadIdx.x & 31;                            \
    const int x = sg.x - sg.y * (a).b.nx + lane;                  \
    if (x >= (a).b.nx) return;                                    \
    const int node = sg.x + lane;                                 \
    const uint8_t fl = __ldg((a).flags + node);                   \
    if (!(fl & kActive)) return;                                  \
    const bool per_ = (a).b.per[0] | (a).b.per[1] | (a).b.per[2]; \
    const int y = per_ ? sg.y % (a).b.ny : 0;                     \
    const int z = per_ ? sg.y / (a).b.ny : 0;                     \
    (void)y;                                                      \
    (void)z;

// Residual of the normal equations of Eq. (projection-edge-relation) at the warm start u0,
//   r_m = b_m + sum_l u0_l - deg_m u0_m,   b_m = sum_l g_ml + sum_b (u_D(X_b, t^n) + G_m (X_m - X_b)),
// accumulated in FP64 (interior edges plus boundary edges to the prescribed displacement).
// Damped Jacobi on u from u0 equals damped Jacobi on the correction d = u - u0 from 0 with this
// right-hand side, so the sweeps can run on d in the population precision.
template <typename real, int D>
__global__ void __launch_bounds__(128, 6) k_proj_residual(const ProjArgs<real> a) {
    TLV_NODE_PROLOGUE(a)
    const long long P = a.b.npad;
    const unsigned cut = fl & kCutMask;
    const uint8_t dm = a.dmask[node];
    double r[D];
    #pragma unroll
    for (int i = 0; i < D; ++i) r[i] = 0.0;
    if (dm) {
        int l = a.lstart[node];
        for (int q = 0; q < 2 * D; ++q) {
            if (!((cut >> q) & 1)) continue;
            if ((dm >> q) & 1) {
                const int A = q >> 1;
                const double s = (q & 1) ? -1.0 : 1.0;
                const double Xb[3] = {a.L.Xb[3 * l], a.L.Xb[3 * l + 1], a.L.Xb[3 * l + 2]};
                double uD[3];
                dirichlet_eval(a.bcs[a.L.bc[l]], D, Xb, a.t, true, uD);
                for (int i = 0; i < D; ++i)
                    r[i] += uD[i] + (double)a.Gst[(i * D + A) * P + node] * (-s * a.L.eta[l] * a.b.dx) -
                            disp_get<real>(a.u0, P, D, i, node);
            }
            ++l;
        }
    }
    // warm start at the node and its neighbours (FP32 form: hi and lo planes, differenced part by
    // part); neighbour values of all 2D directions are loaded before use (a cut direction reads the
    // node itself and is skipped below), so the loads do not wait on one another
    constexpr int NP = kDispPair<real> ? 2 : 1;
    real um[NP][D], ul[2 * D][NP][D];
    real rf[D];
    real Gl_[2 * D][D], Gm_[D][D];
    #pragma unroll
    for (int i = 0; i < D; ++i) {
        rf[i] = real(0);
        #pragma unroll
        for (int h = 0; h < NP; ++h) um[h][i] = a.u0[(h * D + i) * P + node];
    }
    #pragma unroll
    for (int q = 0; q < 2 * D; ++q) {
        int ln = ((cut >> q) & 1) ? node : nbr(a.b, node, x, y, z, q);
        TLV_BOUND(ln, P, a.status);
        #pragma unroll
        for (int i = 0; i < D; ++i) {
            #pragma unroll
            for (int h = 0; h < NP; ++h) ul[q][h][i] = a.u0[(h * D + i) * P + ln];
            Gl_[q][i] = a.Gst[(i * D + (q >> 1)) * P + ln];
        }
    }
    #pragma unroll
    for (int i = 0; i < D; ++i)
        #pragma unroll
        for (int A = 0; A < D; ++A) Gm_[i][A] = a.Gst[(i * D + A) * P + node];
    #pragma unroll
    for (int q = 0; q < 2 * D; ++q) {
        if ((cut >> q) & 1) continue;
        const int A = q >> 1;
        #pragma unroll
        for (int i = 0; i < D; ++i) {
            const real Gm = Gm_[i][A], Gl = Gl_[q][i];
            if constexpr (kShifted<real>) {
                // FP32 edge term: FP64 difference of the nearby displacements, then FP32
                const real sdx = (q & 1) ? (real)a.b.dx : -(real)a.b.dx;
                rf[i] += ((ul[q][0][i] - um[0][i]) + (ul[q][NP - 1][i] - um[NP - 1][i])) + real(0.5) * (Gm + Gl) * sdx;
            } else {
                const double s = (q & 1) ? -1.0 : 1.0;
                r[i] += ul[q][0][i] - um[0][i] + 0.5 * ((double)Gm + (double)Gl) * (-s * a.b.dx);
            }
        }
    }
    const int deg = proj_degree(D, cut, dm);
    real out[4] = {real(0), real(0), real(0), real(0)};
    #pragma unroll
    for (int i = 0; i < D; ++i) out[i] = (real)r[i] + rf[i];
    out[D] = deg > 0 ? (real)a.beta / (real)deg : real(0);
    // FP32 2D: the record's spare fourth value carries the node's cut-direction bits, so the
    // two-sweep kernel has them with the staged residual row and loads no flag bytes
    if constexpr (D == 2 && sizeof(real) == 4) out[3] = __uint_as_float(cut);
    st_vec<4, real>(a.resid + 4 * (long long)node, out);
}

constexpr int kJacobiSegs = 1;  // segments per warp in a Jacobi sweep (default; lbm_autotune may pick 2 or 4)

// One damped-Jacobi sweep on the correction d (d = 0 before the first sweep: din == nullptr),
//   d'_m = (1 - beta) d_m + beta / deg_m (r_m + sum over active axis neighbours l of d_l),
// for segments s0 .. s0 + S - 1 of the calling warp.  A node is its flag
// byte, one residual vector, its own d vector and 2D neighbour d vectors, all loaded before any is
// used (the x neighbours, when rows do not wrap, taken from the neighbouring lanes by shuffles); a
// neighbour across a cut link (inactive, or outside a non-periodic box, where the index is clamped
// into range) is dropped by selection, as a skipped term; nodes with w = 0 keep their d and are not
// written.  (Packing the 2D residual to (r_1, r_2) and recomputing w from a Dirichlet-mask byte
// moved 26 instead of 33 B per node but ran slower, as did D planes of d and r: the sweep is bound
// by its loads in flight, not by its bytes.)
template <typename real, int D, int S, bool shx>
__device__ __forceinline__ void jacobi_segments(const ProjArgs<real> &a, const real *__restrict__ din,
                                                real *__restrict__ dout, int s0, const int2 (&sgs)[S]) {
    constexpr int Q = 2 * D, V = kDV<D>;
    const int lane = threadIdx.x & 31;
    const long long P = a.b.npad;
    const real beta = (real)a.beta;
    const bool per = a.b.per[0] | a.b.per[1] | a.b.per[2];
    int node[S], ln[S][Q];  // node indices fit 32 bits (boxes below 2^31 nodes)
    bool in[S];
    #pragma unroll
    for (int j = 0; j < S; ++j) {
        const bool seg_ok = s0 + j < a.nseg;
        const int2 sg = sgs[j];
        const int x = sg.x - sg.y * a.b.nx + lane;
        in[j] = seg_ok && x < a.b.nx;
        const int nd = in[j] ? sg.x + lane : 0;  // lanes outside the row read node 0, unused
        node[j] = nd;
        const int y = per ? sg.y % a.b.ny : 0, z = per ? sg.y / a.b.ny : 0;
        #pragma unroll
        for (int q = 0; q < Q; ++q) {
            const int l = nbr(a.b, nd, x, y, z, q);
            ln[j][q] = l < 0 ? 0 : (l >= P ? (int)(P - 1) : l);  // only inactive nodes can point outside
        }
    }
    // FP32 3D: the node's cut-direction bits travel in d's spare fourth value, written by the first
    // sweep of a solve (from the flag byte) and copied by every later one, so only the first sweep
    // loads flag bytes
    constexpr bool kCutInD = sizeof(real) == 4 && D == 3;
    real r[S][4], dold[S][V], nb[S][Q][V];
    unsigned cut[S];
    #pragma unroll
    for (int j = 0; j < S; ++j) {
        if (!kCutInD || !din) cut[j] = __ldg(a.flags + node[j]) & kCutMask;
        ld_vec<4, real>(a.resid + 4LL * node[j], r[j]);
        if (din) {
            ld_vec<V, real>(din + (long long)V * node[j], dold[j]);
            #pragma unroll
            for (int q = 0; q < Q; ++q)
                if (q >= 2 || !shx) ld_vec<V, real>(din + (long long)V * ln[j][q], nb[j][q]);
            if constexpr (shx) {
                // the x neighbours are the neighbouring lanes' own vectors; lane 31 loads node + 1 and
                // lane 0 node - 1
                real e[V];
                #pragma unroll
                for (int i = 0; i < V; ++i) e[i] = real(0);
                const int ie = lane == 31 ? node[j] + 1 : (node[j] > 0 ? node[j] - 1 : 0);
                if (lane == 0 || lane == 31) ld_vec<V, real>(din + (long long)V * ie, e);
                #pragma unroll
                for (int i = 0; i < V; ++i) {
                    const real dn = __shfl_down_sync(0xffffffffu, dold[j][i], 1);
                    const real up = __shfl_up_sync(0xffffffffu, dold[j][i], 1);
                    nb[j][0][i] = lane == 31 ? e[i] : dn;  // +x: node + 1
                    nb[j][1][i] = lane == 0 ? e[i] : up;   // -x: node - 1
                }
            }
        } else {
            #pragma unroll
            for (int i = 0; i < V; ++i) {
                dold[j][i] = real(0);
                #pragma unroll
                for (int q = 0; q < Q; ++q) nb[j][q][i] = real(0);
            }
        }
    }
    if constexpr (kCutInD) {
        if (din) {
            #pragma unroll
            for (int j = 0; j < S; ++j) cut[j] = __float_as_uint(dold[j][3]) & kCutMask;
        }
    }
    #pragma unroll
    for (int j = 0; j < S; ++j) {
        const real w = r[j][D];
        if (!in[j] || !(w > real(0))) continue;
        real out[V];
        #pragma unroll
        for (int i = 0; i < V; ++i) out[i] = real(0);
        #pragma unroll
        for (int i = 0; i < D; ++i) {
            real acc = r[j][i];
            #pragma unroll
            for (int q = 0; q < Q; ++q) acc += ((cut[j] >> q) & 1) ? real(0) : nb[j][q][i];
            // FP32: the rounding of fma(w, acc, (1 - beta) d) spelled out, which the two-sweep kernel
            // repeats; FP64: separate products, as the oracle
            if constexpr (sizeof(real) == 4) out[i] = __fmaf_rn(w, acc, __fmul_rn(real(1) - beta, dold[j][i]));
            else out[i] = (real(1) - beta) * dold[j][i] + w * acc;
        }
        if constexpr (kCutInD) out[3] = __uint_as_float(cut[j]);
        st_vec<V, real>(dout + (long long)V * node[j], out);
    }
}

// The grid is sized to the blocks that fit on the GPU at once and every warp strides over the
// segment list (S segments at a time), so no time goes to retiring and launching short blocks.
// shx: rows do not wrap (x not periodic), so a segment's x neighbours are its own lanes' vectors.
template <typename real, int D, int S = kJacobiSegs, bool shx = true>
__global__ void __launch_bounds__(128) k_jacobi(const ProjArgs<real> a, const real *__restrict__ din,
                                                real *__restrict__ dout) {
    const int stride = gridDim.x * 4 * S;
    int s0 = (blockIdx.x * 4 + (threadIdx.x >> 5)) * S;
    // the segment descriptors of the next iteration are loaded while this one's nodes are swept
    int2 nxt[S];
    #pragma unroll
    for (int j = 0; j < S; ++j) nxt[j] = s0 + j < a.nseg ? __ldg(&a.seg[s0 + j]) : make_int2(0, 0);
    for (; s0 < a.nseg; s0 += stride) {
        int2 cur[S];
        #pragma unroll
        for (int j = 0; j < S; ++j) {
            cur[j] = nxt[j];
            const int sn = s0 + stride + j;
            nxt[j] = sn < a.nseg ? __ldg(&a.seg[sn]) : make_int2(0, 0);
        }
        jacobi_segments<real, D, S, shx>(a, din, dout, s0, cur);
    }
}


// block partial sums of the correction (u^c - u^0) per component: warp shuffles, then shared memory
template <typename real, int D>
__global__ void __launch_bounds__(128) k_reduce_partial(const ProjArgs<real> a, const real *__restrict__ dc,
                                                        double *partial) {
    __shared__ double sm[4][D];
    real dl[D];
    #pragma unroll
    for (int i = 0; i < D; ++i) dl[i] = real(0);
    const int lane = threadIdx.x & 31;
    // fixed grid, segments strided over it, so the partial count (and the summation order) is fixed;
    // each thread pre-sums its own few values in the correction's precision, the rest is FP64
    const int stride = gridDim.x * 4;
    for (int s0 = blockIdx.x * 4 + (threadIdx.x >> 5); s0 < a.nseg; s0 += 4 * stride) {
        // four segments per pass: their loads are independent
        int node[4];
        bool ok[4];
        #pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int sgi = s0 + j * stride;
            const int2 sg = sgi < a.nseg ? __ldg(&a.seg[sgi]) : make_int2(0, 0);
            node[j] = sg.x + lane;
            ok[j] = sgi < a.nseg && sg.x - sg.y * a.b.nx + lane < a.b.nx;
        }
        #pragma unroll
        for (int j = 0; j < 4; ++j) ok[j] = ok[j] && (__ldg(a.flags + node[j]) & kActive);
        #pragma unroll
        for (int j = 0; j < 4; ++j)
            if (ok[j])
                #pragma unroll
                for (int i = 0; i < D; ++i) dl[i] += dc[(long long)kDV<D> * node[j] + i];
    }
    double d[D];
    #pragma unroll
    for (int i = 0; i < D; ++i) d[i] = (double)dl[i];
    #pragma unroll
    for (int i = 0; i < D; ++i)
        #pragma unroll
        for (int o = 16; o > 0; o >>= 1) d[i] += __shfl_down_sync(0xffffffffu, d[i], o);
    if (lane == 0)
        #pragma unroll
        for (int i = 0; i < D; ++i) sm[threadIdx.x >> 5][i] = d[i];
    __syncthreads();
    if (threadIdx.x < D) partial[blockIdx.x * D + threadIdx.x] = sm[0][threadIdx.x] + sm[1][threadIdx.x] + sm[2][threadIdx.x] + sm[3][threadIdx.x];
}

// deterministic final reduction (one block of 256): mean[i] = sum / n_active
template <int D>
__global__ void __launch_bounds__(256) k_reduce_final(const double *__restrict__ partial, int nblocks, double inv_n, double *mean) {
    __shared__ double sm[8][D];
    double s[D];
    #pragma unroll
    for (int i = 0; i < D; ++i) s[i] = 0.0;
    for (int j = threadIdx.x; j < nblocks; j += 256)
        #pragma unroll
        for (int i = 0; i < D; ++i) s[i] += partial[j * D + i];
    #pragma unroll
    for (int i = 0; i < D; ++i)
        #pragma unroll
        for (int o = 16; o > 0; o >>= 1) s[i] += __shfl_down_sync(0xffffffffu, s[i], o);
    if ((threadIdx.x & 31) == 0)
        #pragma unroll
        for (int i = 0; i < D; ++i) sm[threadIdx.x >> 5][i] = s[i];
    __syncthreads();
    if (threadIdx.x < D) {
        double t = 0.0;
        for (int w = 0; w < 8; ++w) t += sm[w][threadIdx.x];
        mean[threadIdx.x] = t * inv_n;
    }
}

// after the first solve: u^n = u0 + d - mean (written to u1), F^c (Eq. projection-compatible-F), F^r
// (Eq. projection-F-repair-weight), population repair (Eq. projection-population-repair),
// collision and u*^{n+1}.  f^n is read from fsrc and f*^n written to fdst, two different buffers,
// so each direction's loads can be issued ahead of the other directions' stores.
template <typename real, int D, typename pop = real>
__global__ void __launch_bounds__(128) k_repair_collide(const StepArgs<real> a, const real *__restrict__ u0,
                                                        const real *__restrict__ dc, const double *__restrict__ mean,
                                                        double theta, real *u1) {
    constexpr int K = D + D * D, Q = 2 * D;
    constexpr long long DV = kDV<D>;
    TLV_NODE_PROLOGUE(a)
    const long long P = a.b.npad;
    const unsigned cut = fl & kCutMask;
    const real *__restrict__ fsrc = a.fsrc;
    real *__restrict__ fdst = a.fdst;
    real fpre[K];
    real v[D], G[D * D], F[D * D], Pold[D * D], Fr[D * D], Gr[D * D], Pk[D * D];
    #pragma unroll
    for (int i = 0; i < D; ++i) v[i] = a.vst[i * P + node];
    #pragma unroll
    for (int k = 0; k < D * D; ++k) G[k] = a.Gst[k * P + node];
    #pragma unroll
    for (int A = 0; A < D; ++A) {
        const bool ap = !((cut >> (2 * A)) & 1), am = !((cut >> (2 * A + 1)) & 1);
        int lp = ap ? nbr(a.b, node, x, y, z, 2 * A) : node;
        int lm = am ? nbr(a.b, node, x, y, z, 2 * A + 1) : node;
        TLV_BOUND(lp, P, a.status);
        TLV_BOUND(lm, P, a.status);
        #pragma unroll
        for (int i = 0; i < D; ++i) {
            real Gc;
            if constexpr (kShifted<real>) {
                // FP32 form: u^c differences from the (hi, lo) pairs, hi parts first (u carries the large
                // offset; nearby hi parts subtract exactly), then the corrections
                const real ho = u0[i * P + node], lo_ = u0[(D + i) * P + node];
                const real dp = ((u0[i * P + lp] - ho) + (u0[(D + i) * P + lp] - lo_)) + (dc[DV * lp + i] - dc[DV * node + i]);
                const real dm = ((ho - u0[i * P + lm]) + (lo_ - u0[(D + i) * P + lm])) + (dc[DV * node + i] - dc[DV * lm + i]);
                const real inv = real(1) / (real)a.b.dx;
                if (ap && am) Gc = real(0.5) * (dp + dm) * inv;
                else if (ap) Gc = dp * inv;
                else if (am) Gc = dm * inv;
                else Gc = G[i * D + A];
                Gr[i * D + A] = (real(1) - (real)theta) * G[i * D + A] + (real)theta * Gc;
            } else {
                double gc;
                bool keep = false;
                const double up = u0[i * P + lp] + (double)dc[DV * lp + i];
                const double um = u0[i * P + lm] + (double)dc[DV * lm + i];
                const double uo = u0[i * P + node] + (double)dc[DV * node + i];
                if (ap && am) gc = (up - um) / (2.0 * a.b.dx);
                else if (ap) gc = (up - uo) / a.b.dx;
                else if (am) gc = (uo - um) / a.b.dx;
                else { gc = 0.0; keep = true; }
                Gc = keep ? G[i * D + A] : (real)gc;
                Gr[i * D + A] = (real)((1.0 - theta) * (double)G[i * D + A] + theta * (double)Gc);
            }
        }
    }
    #pragma unroll
    for (int i = 0; i < D; ++i)
        #pragma unroll
        for (int B = 0; B < D; ++B) {
            const real one = (i == B) ? real(1) : real(0);
            F[i * D + B] = G[i * D + B] + one;
            Fr[i * D + B] = Gr[i * D + B] + one;
        }
    real mu, lam;
    node_material(a, node, mu, lam);
    real J;
    if constexpr (kShifted<real>) {
        real Fit[D * D];
        piola_g<real, D>(G, mu, lam, Pold, Fit);
        J = piola_g<real, D>(Gr, mu, lam, Pk, Fit);
    } else {
        piola<real, D>(F, mu, lam, Pold);
        J = piola<real, D>(Fr, mu, lam, Pk);
    }
    const int st = check_state<real, D>(v, Fr, J);
    if (st) set_status(a.status, st);
    const real Dc = real(D) / a.c;
    const real src = a.dt * (real(2) - a.omega) * (real(1) / real(4 * D));
    real B[D];
    #pragma unroll
    for (int i = 0; i < D; ++i) B[i] = a.bf[i] - a.gamma * v[i];
    const long long l0 = cut ? __ldg(a.lstart + node) : 0;
    #pragma unroll
    for (int q = 0; q < Q; ++q) {
        const int A = q >> 1;
        const real s = (q & 1) ? real(-1) : real(1);
        real out[K];
        #pragma unroll
        for (int k = 0; k < K; ++k) fpre[k] = pop_ld<real, pop>(fsrc, (long long)(q * K + k) * P + node);
        #pragma unroll
        for (int k = 0; k < K; ++k) {
            real fv = fpre[k];
            real feq;  // equilibrium at the repaired state (Eq. feq-general-d)
            if (k < D) {
                const int i = k;
                feq = div2D<real, D>(v[i] - s * Dc * Pk[i * D + A]);
                // repair: f += f^eq(v, F^r) - f^eq(v, F) (Eq. projection-population-repair)
                if constexpr (kShifted<real>) fv = fv - div2D<real, D>(s * Dc * (Pk[i * D + A] - Pold[i * D + A]));
                else fv = fv + (feq - div2D<real, D>(v[i] - s * Dc * Pold[i * D + A]));
            } else {
                const int i = (k - D) / D, Bc = (k - D) % D;
                const real Xr = kShifted<real> ? Gr[i * D + Bc] : Fr[i * D + Bc];
                const real Xo = kShifted<real> ? G[i * D + Bc] : F[i * D + Bc];
                const real vs = (A == Bc) ? s * Dc * v[i] : real(0);
                feq = (A == Bc) ? div2D<real, D>(Xr - vs) : div2D<real, D>(Xr);
                if constexpr (kShifted<real>) fv = fv + div2D<real, D>(Gr[i * D + Bc] - G[i * D + Bc]);
                else fv = fv + (feq - ((A == Bc) ? div2D<real, D>(Xo - vs) : div2D<real, D>(Xo)));
            }
            // BGK collision with source (Eq. collision-general-d)
            out[k] = fv + a.omega * (feq - fv) + ((k < D) ? src * B[k] : real(0));
        }
        #pragma unroll
        for (int k = 0; k < K; ++k) pop_st<real, pop>(fdst, (long long)(q * K + k) * P + node, out[k]);
        if (cut) keep_link_values<real, K>(a.lfo, l0, cut, q, out, a.ncut, a.status);
    }
    #pragma unroll
    for (int i = 0; i < D; ++i) {
        if constexpr (kDispPair<real>) {
            float hi = u0[i * P + node], lo = u0[(D + i) * P + node];
            df_add(hi, lo, dc[DV * node + i] - (real)mean[i]);  // u^n after the first projection
            u1[i * P + node] = hi;
            u1[(D + i) * P + node] = lo;
            df_add(hi, lo, real(0.5) * a.dt * v[i]);           // u*^{n+1}
            a.ustar[i * P + node] = hi;
            a.ustar[(D + i) * P + node] = lo;
        } else {
            const double un = u0[i * P + node] + (double)(dc[DV * node + i] - (real)mean[i]);
            u1[i * P + node] = un;
            a.ustar[i * P + node] = (real)un + real(0.5) * a.dt * v[i];
        }
    }
    #pragma unroll
    for (int k = 0; k < D * D; ++k) a.Gst[k * P + node] = Gr[k];
}

// after the second solve: u^n = u0 + d - mean and u*^{n+1} = u^n + dt/2 v^n
template <typename real, int D>
__global__ void __launch_bounds__(128) k_proj_reset(const StepArgs<real> a, const real *__restrict__ u0,
                                                    const real *__restrict__ dc, const double *__restrict__ mean) {
    constexpr long long DV = kDV<D>;
    TLV_NODE_PROLOGUE(a)
    const long long P = a.b.npad;
    real unh[D], unl[D];
    #pragma unroll
    for (int i = 0; i < D; ++i) {
        if constexpr (kDispPair<real>) {
            float hi = u0[i * P + node], lo = u0[(D + i) * P + node];
            df_add(hi, lo, dc[DV * node + i] - (real)mean[i]);  // u^n after the second projection
            unh[i] = hi;
            unl[i] = lo;
            df_add(hi, lo, real(0.5) * a.dt * a.vst[i * P + node]);  // u*^{n+1}
            a.ustar[i * P + node] = hi;
            a.ustar[(D + i) * P + node] = lo;
        } else {
            const real un = (real)(u0[i * P + node] + (double)(dc[DV * node + i] - (real)mean[i]));
            unh[i] = un;
            unl[i] = real(0);
            a.ustar[i * P + node] = un + real(0.5) * a.dt * a.vst[i * P + node];
        }
    }
    un_store<real, D>(a.un, node, unh, unl);
}

}  // namespace tlv
