// TMA-staged gather for the fused collide-stream kernel with FP32 arithmetic (sm_103a), for
// populations stored in FP32 or in BF16.
//
// The pull gather of one 32-node x-segment reads, for every direction q, the K component
// planes of f* at the segment shifted by -e_q.  Population planes are consecutive in a
// 2D tensor (dim 0: node index, npad; dim 1: plane q*K + k), so the K planes of one
// direction are one box of (width, K).  One elected lane per warp issues Q bulk tensor
// copies into the warp's shared-memory slots, completed on a per-warp mbarrier:
//   +-x: box (40, K) starting 4 nodes before the segment for FP32, (48, K) starting 8 nodes
//        before it for BF16 (a TMA start coordinate must fall on a 16-byte boundary, so the
//        +-1 shifted windows are read from an aligned wider box)
//   +-y, +-z: box (32, K) at the source row (periodic rows wrapped).
// The wait is bounded; on timeout the kernel latches a status bit, waits once more (bounded)
// for its copies in flight and returns without writing.
#pragma once

#include <cuda.h>

#include "lbm_kernels.cuh"

namespace tlv {

constexpr int kStTimeout = 128;        // device status bit: a TMA wait ran out
constexpr int kTmaSpin = 1 << 20;      // try_wait polls before giving up
constexpr int kTmaNarrow = 32;

// stage layout of one warp for population elements of E bytes (4: FP32, 2: BF16).  The +-x boxes
// start `halo` elements before the segment, since a bulk copy's start coordinate must fall on a
// 16-byte boundary: 4 floats or 8 BF16 values, so the +-x boxes are 40 or 48 elements wide.
template <int D, int E = 4> struct TmaLayout {
    static constexpr int K = D + D * D, Q = 2 * D;
    static constexpr int halo = 16 / E;
    static constexpr int wide = 32 + 2 * halo;
    static constexpr int wide_bytes = ((wide * K * E + 127) / 128) * 128;
    static constexpr int narrow_bytes = ((kTmaNarrow * K * E + 127) / 128) * 128;
    static constexpr int warp_bytes = 2 * wide_bytes + (Q - 2) * narrow_bytes;
    static constexpr int tx_bytes = 2 * wide * K * E + (Q - 2) * kTmaNarrow * K * E;
    // byte offset of direction q's slot in a warp region
    __device__ static constexpr int slot(int q) { return q < 2 ? q * wide_bytes : 2 * wide_bytes + (q - 2) * narrow_bytes; }
    __device__ static constexpr int width(int q) { return q < 2 ? wide : kTmaNarrow; }
    // element offset of lane 0's source inside the box row: m - e_x for q = 0, m + e_x for q = 1
    __device__ static constexpr int lane0(int q) { return q == 0 ? halo - 1 : (q == 1 ? halo + 1 : 0); }
    static constexpr int block_bytes(int warps) { return warps * warp_bytes + warps * 8; }
    // fused-kernel stage: population slots, then u* (hi and lo planes: 2D x 32 floats), flags (32 bytes)
    static constexpr int us_off = warp_bytes;
    static constexpr int fl_off = us_off + ((2 * D * 32 * 4 + 127) / 128) * 128;
    static constexpr int stage_bytes = fl_off + 128;
    static constexpr int stage_tx = tx_bytes + 2 * D * 32 * 4 + 32;
};

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_fence_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ void tma_load_2d(void *dst, const CUtensorMap *map, uint64_t *bar, int x, int y) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::
            "r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_u32(bar))
        : "memory");
}

// at most `limit` polls (the first wait of a window takes StepArgs::spin, kTmaSpin unless a test
// shortens it; the drain after a timeout always takes kTmaSpin)
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity, int limit = kTmaSpin) {
    for (int it = 0; it < limit; ++it)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}

// Issue the Q bulk copies of segment sg into the warp's slots and wait for them.  Returns false
// (status latched) if the wait ran out.  Every lane of the warp must call it.
template <int D, typename pop = float>
__device__ __forceinline__ bool tma_gather_segment(const Box &b, const CUtensorMap *wide, const CUtensorMap *narrow,
                                                   char *wsm, uint64_t *bar, int2 sg, int lane, int *status, int spin) {
    using L = TmaLayout<D, sizeof(pop)>;
    constexpr int K = L::K, Q = L::Q;
    if (lane == 0) {
        mbar_init(bar, 1);
        mbar_fence_init();
    }
    __syncwarp();
    if (lane == 0) {
        const int y = sg.y % b.ny, z = sg.y / b.ny, x0 = sg.x - sg.y * b.nx;
        mbar_arrive_expect_tx(bar, L::tx_bytes);
        #pragma unroll
        for (int q = 0; q < Q; ++q) {
            const int A = q >> 1, s = (q & 1) ? -1 : 1;  // pull source of direction q is m - s e_A
            int start;
            if (A == 0) {
                start = sg.x - L::halo;
            } else if (A == 1) {
                int yy = y - s;
                if (b.per[1]) yy = yy < 0 ? yy + b.ny : (yy >= b.ny ? yy - b.ny : yy);
                start = (z * b.ny + yy) * b.nx + x0;
            } else {
                int zz = z - s;
                if (b.per[2]) zz = zz < 0 ? zz + b.nz : (zz >= b.nz ? zz - b.nz : zz);
                start = (zz * b.ny + y) * b.nx + x0;
            }
            tma_load_2d(wsm + L::slot(q), A == 0 ? wide : narrow, bar, start, q * K);
        }
    }
    bool ok = mbar_wait_bounded(bar, 0, spin);
    if (!ok) {
        if (lane == 0) set_status(status, kStTimeout);
        mbar_wait_bounded(bar, 0);  // let the copies in flight land before the block can exit
    }
    return __all_sync(0xffffffffu, ok);
}

// value of direction q, component k for this lane in the staged slots (as FP32), and its update
template <int D, typename pop = float> __device__ __forceinline__ float staged(const char *wsm, int q, int k, int lane) {
    using L = TmaLayout<D, sizeof(pop)>;
    const pop v = reinterpret_cast<const pop *>(wsm + L::slot(q))[k * L::width(q) + L::lane0(q) + lane];
    return (float)v;
}
template <int D, typename pop = float>
__device__ __forceinline__ void stage_put(char *wsm, int q, int k, int lane, float v) {
    using L = TmaLayout<D, sizeof(pop)>;
    reinterpret_cast<pop *>(wsm + L::slot(q))[k * L::width(q) + L::lane0(q) + lane] = (pop)v;
}

// closure with TMA staging: the populations that cut links leave unknown arrive reconstructed by the
// link kernel (first link of the node l0); the gathered values stay in shared memory
template <int D, typename pop = float>
__device__ __forceinline__ void tma_closure(const StepArgs<float> &a, char *wsm, int node, int x, int lane,
                                            unsigned cut, long long l0) {
    constexpr int K = D + D * D, Q = 2 * D;
    const long long P = a.b.npad;
    const float *__restrict__ fs = a.fsrc;
    if (a.b.per[0]) {  // the aligned x windows do not wrap: patch the periodic ends
        if (x == 0 && !((cut >> 1) & 1))
            #pragma unroll
            for (int k = 0; k < K; ++k)
                stage_put<D, pop>(wsm, 0, k, lane, pop_ld<float, pop>(fs, (long long)(0 * K + k) * P + node + a.b.nx - 1));
        if (x == a.b.nx - 1 && !(cut & 1))
            #pragma unroll
            for (int k = 0; k < K; ++k)
                stage_put<D, pop>(wsm, 1, k, lane, pop_ld<float, pop>(fs, (long long)(1 * K + k) * P + node - (a.b.nx - 1)));
    }
    if (!cut) return;
    // boundary nodes only: a rolled loop over the directions keeps the kernel's code small
    #pragma unroll 1
    for (int q = 0; q < Q; ++q) {
        if ((cut >> (q ^ 1)) & 1) {
            float r[K];
            long long l = link_of(l0, cut, q ^ 1);
            TLV_BOUND(l, a.ncut, a.status);
            vload<K>(a.lrec + l * K, r);
            // an eta < 1/2 link with an active upstream node: its term D_b (1 - 2 eta) f*_c(m - e_c), with
            // f*_c(m - e_c) the value staged for direction c = q^1 (pulled: link (m, q) is not cut)
            const float cv = __ldg(a.lcu + l);
            if (cv != 0.0f)
                #pragma unroll
                for (int k = 0; k < K; ++k) r[k] += (k < D ? cv : -cv) * staged<D, pop>(wsm, q ^ 1, k, lane);
            #pragma unroll
            for (int k = 0; k < K; ++k) stage_put<D, pop>(wsm, q, k, lane, r[k]);
        }
    }
}

struct TmaMaps {
    CUtensorMap wide, narrow;  // population planes of the source buffer: (40 or 48, K) and (32, K) boxes
    CUtensorMap ustar;         // u* planes: (32, D) boxes
    CUtensorMap flags;         // flag bytes as (nx, ny*nz): (32, 1) boxes
};

// recovery, collision and u quadrature of one node from its staged populations (FP32 form).
// Arithmetic is arranged to avoid divisions in the per-node path:
//   v = (sum f_v + dt/2 b) * 1/(1 + gamma dt/2),  F^{-T} = cof(F) * (1/J),
//   f*_q = (1 - omega) f_q + omega f^eq_q + src_q with omega f^eq_q = base_k +- (omega D/(2Dc)) Phi_A,k
template <int D, typename pop = float>
__device__ __forceinline__ void collide_staged(const StepArgs<float> &a, char *wsm, int node, int lane, uint8_t fl,
                                               const float us[2 * D], long long l0, bool act, float mu, float lam) {
    constexpr int K = D + D * D, Q = 2 * D;
    float S[K];
    #pragma unroll
    for (int k = 0; k < K; ++k) {
        float s = staged<D, pop>(wsm, 0, k, lane);
        #pragma unroll
        for (int q = 1; q < Q; ++q) s += staged<D, pop>(wsm, q, k, lane);
        S[k] = s;
    }
    const float hdt = 0.5f * a.dt;
    const float inv_damp = 1.0f / (1.0f + hdt * a.gamma);
    float v[D], P[D * D], Fit[D * D];
    #pragma unroll
    for (int i = 0; i < D; ++i) v[i] = (S[i] + hdt * a.bf[i]) * inv_damp;
    if (a.mom_out && act)
        #pragma unroll
        for (int k = 0; k < D * D; ++k) a.mom_out[(long long)k * a.b.npad + node] = S[D + k];
    // P(F) from G = F - I = S[D..], free of the cancellations near F = I
    const float J = piola_g<float, D>(S + D, mu, lam, P, Fit);
    float chk = J;
    #pragma unroll
    for (int i = 0; i < D; ++i) chk += v[i];
    #pragma unroll
    for (int k = 0; k < D * D; ++k) chk += P[k];
    if (act && (!(J > 0.0f) || !isfinite(chk)))
        set_status(a.status, (J > 0.0f ? 0 : kStJacobian) | (isfinite(chk) ? 0 : kStNonfinite));
    const long long Pn = a.b.npad;
    float unh[D], unl[D];
    #pragma unroll
    for (int i = 0; i < D; ++i) {
        float hi = us[i], lo = us[D + i];  // u*^n as a (hi, lo) pair
        const float d = hdt * v[i];
        df_add(hi, lo, d);  // u^n
        unh[i] = hi;
        unl[i] = lo;
        df_add(hi, lo, d);  // u*^{n+1}
        a.ustar[i * Pn + node] = act ? hi : 0.0f;
        a.ustar[(D + i) * Pn + node] = act ? lo : 0.0f;
    }
    if (fl & kNeedU) un_store<float, D>(a.un, node, unh, unl);
    const float om1 = 1.0f - a.omega;
    const float wf = a.omega * (1.0f / float(2 * D));  // omega/(2D)
    const float wc = wf * (float(D) / a.c);             // omega/(2D) * D/c
    const float src = a.dt * (2.0f - a.omega) * (1.0f / float(4 * D));
    float base[K];
    #pragma unroll
    for (int i = 0; i < D; ++i) base[i] = wf * v[i] + src * (a.bf[i] - a.gamma * v[i]);
    #pragma unroll
    for (int k = 0; k < D * D; ++k) base[D + k] = wf * S[D + k];
    float wv[D];
    #pragma unroll
    for (int i = 0; i < D; ++i) wv[i] = wc * v[i];
    const unsigned cut = fl & kCutMask;
    #pragma unroll
    for (int q = 0; q < Q; ++q) {
        const int A = q >> 1;
        const bool neg = q & 1;
        float o[K];
        #pragma unroll
        for (int k = 0; k < K; ++k) {
            float t;
            if (k < D) {
                const float fl_ = wc * P[k * D + A];   // omega/(2D) (D/c) P_kA
                t = neg ? base[k] + fl_ : base[k] - fl_;
            } else if (((k - D) % D) == A) {
                const int i = (k - D) / D;
                t = neg ? base[k] + wv[i] : base[k] - wv[i];
            } else {
                t = base[k];
            }
            o[k] = act ? fmaf(om1, staged<D, pop>(wsm, q, k, lane), t) : 0.0f;
            pop_st<float, pop>(a.fdst, (long long)(q * K + k) * Pn + node, o[k]);
        }
        if (cut) keep_link_values<float, K>(a.lfo, l0, cut, q, o, a.ncut, a.status);
    }
}

// Operands of the population repair on a projection step (Eqs. projection-compatible-F,
// projection-F-repair-weight, projection-population-repair): u^n and the first solve's correction.
struct RepairArgs {
    const float *u0;      // u^n as (hi, lo) plane pairs
    const float *dc;      // correction d of the first solve, node-major (kDV values per node)
    const double *mean;   // its gauge shift
    float theta;          // repair weight theta_F
    float *u1;            // out: u^n after the first projection, (hi, lo) pairs
};

// The repair step of a projection step with the populations re-gathered by the bulk copies (FP32):
// from the staged f^n, the recovery (as collide_staged), F^c from u^n + d (central differences, one
// sided where a neighbour is inactive), F^r, the populations translated by f^eq(v, F^r) - f^eq(v, F),
// the collision, u*^{n+1}; F^r - I stored for the second solve.  The same arithmetic as the
// plain-load k_repair_collide, from the same staged values.
// Corrected gradient of u^c = u^0 + d (central differences, one-sided next to a cut link) for the
// repair, from the node's and its axis neighbours' u^0 pairs and corrections; computed before the
// warp waits for its bulk copies, so these scattered loads overlap the copies.  own[A] marks an axis
// with no neighbour on either side, where the repair keeps the gathered gradient.
template <int D>
__device__ __forceinline__ void repair_gradient(const StepArgs<float> &a, const RepairArgs &rp, int node, int x, int y,
                                                int z, uint8_t fl, float Gc[D * D], bool own[D]) {
    constexpr long long DV = kDV<D>;
    const long long Pn = a.b.npad;
    const unsigned cut = fl & kCutMask;
    const float inv = 1.0f / (float)a.b.dx;
    #pragma unroll
    for (int A = 0; A < D; ++A) {
        const bool ap = !((cut >> (2 * A)) & 1), am = !((cut >> (2 * A + 1)) & 1);
        int lp = ap ? nbr(a.b, node, x, y, z, 2 * A) : node;
        int lm = am ? nbr(a.b, node, x, y, z, 2 * A + 1) : node;
        TLV_BOUND(lp, Pn, a.status);
        TLV_BOUND(lm, Pn, a.status);
        own[A] = !ap && !am;
        #pragma unroll
        for (int i = 0; i < D; ++i) {
            const float ho = rp.u0[i * Pn + node], lo_ = rp.u0[(D + i) * Pn + node];
            const float dp = ((rp.u0[i * Pn + lp] - ho) + (rp.u0[(D + i) * Pn + lp] - lo_)) +
                             (rp.dc[DV * lp + i] - rp.dc[DV * node + i]);
            const float dm = ((ho - rp.u0[i * Pn + lm]) + (lo_ - rp.u0[(D + i) * Pn + lm])) +
                             (rp.dc[DV * node + i] - rp.dc[DV * lm + i]);
            float g = 0.0f;
            if (ap && am) g = 0.5f * (dp + dm) * inv;
            else if (ap) g = dp * inv;
            else if (am) g = dm * inv;
            Gc[i * D + A] = g;
        }
    }
}

template <int D, typename pop = float>
__device__ __forceinline__ void repair_staged(const StepArgs<float> &a, const RepairArgs &rp, char *wsm, int node,
                                              int lane, uint8_t fl, long long l0, bool act, float mu, float lam,
                                              const float Gc[D * D], const bool own[D]) {
    constexpr int K = D + D * D, Q = 2 * D;
    constexpr long long DV = kDV<D>;
    const long long Pn = a.b.npad;
    if (!act) {  // whole sectors: zeros for an inactive node's slots
        #pragma unroll
        for (int j = 0; j < Q * K; ++j) pop_st<float, pop>(a.fdst, (long long)j * Pn + node, 0.0f);
        return;
    }
    float S[K];
    #pragma unroll
    for (int k = 0; k < K; ++k) {
        float s = staged<D, pop>(wsm, 0, k, lane);
        #pragma unroll
        for (int q = 1; q < Q; ++q) s += staged<D, pop>(wsm, q, k, lane);
        S[k] = s;
    }
    const float hdt = 0.5f * a.dt;
    const float inv_damp = 1.0f / (1.0f + hdt * a.gamma);
    float v[D], G[D * D], Gr[D * D];
    #pragma unroll
    for (int i = 0; i < D; ++i) v[i] = (S[i] + hdt * a.bf[i]) * inv_damp;
    #pragma unroll
    for (int k = 0; k < D * D; ++k) G[k] = S[D + k];
    const unsigned cut = fl & kCutMask;
    #pragma unroll
    for (int A = 0; A < D; ++A)
        #pragma unroll
        for (int i = 0; i < D; ++i)
            Gr[i * D + A] = (1.0f - rp.theta) * G[i * D + A] + rp.theta * (own[A] ? G[i * D + A] : Gc[i * D + A]);
    float Pold[D * D], Pk[D * D], Fit[D * D];
    piola_g<float, D>(G, mu, lam, Pold, Fit);
    const float J = piola_g<float, D>(Gr, mu, lam, Pk, Fit);
    float chk = J;
    #pragma unroll
    for (int i = 0; i < D; ++i) chk += v[i];
    #pragma unroll
    for (int k = 0; k < D * D; ++k) chk += Pk[k];
    if (!(J > 0.0f) || !isfinite(chk))
        set_status(a.status, (J > 0.0f ? 0 : kStJacobian) | (isfinite(chk) ? 0 : kStNonfinite));
    const float Dc = float(D) / a.c;
    const float src = a.dt * (2.0f - a.omega) * (1.0f / float(4 * D));
    float B[D];
    #pragma unroll
    for (int i = 0; i < D; ++i) B[i] = a.bf[i] - a.gamma * v[i];
    #pragma unroll
    for (int q = 0; q < Q; ++q) {
        const int A = q >> 1;
        const float s = (q & 1) ? -1.0f : 1.0f;
        float out[K];
        #pragma unroll
        for (int k = 0; k < K; ++k) {
            float fv = staged<D, pop>(wsm, q, k, lane);
            float feq;
            if (k < D) {
                const int i = k;
                feq = div2D<float, D>(v[i] - s * Dc * Pk[i * D + A]);
                fv = fv - div2D<float, D>(s * Dc * (Pk[i * D + A] - Pold[i * D + A]));
            } else {
                const int i = (k - D) / D, Bc = (k - D) % D;
                const float vs = (A == Bc) ? s * Dc * v[i] : 0.0f;
                feq = (A == Bc) ? div2D<float, D>(Gr[i * D + Bc] - vs) : div2D<float, D>(Gr[i * D + Bc]);
                fv = fv + div2D<float, D>(Gr[i * D + Bc] - G[i * D + Bc]);
            }
            out[k] = fv + a.omega * (feq - fv) + ((k < D) ? src * B[k] : 0.0f);
        }
        #pragma unroll
        for (int k = 0; k < K; ++k) pop_st<float, pop>(a.fdst, (long long)(q * K + k) * Pn + node, out[k]);
        if (cut) keep_link_values<float, K>(a.lfo, l0, cut, q, out, a.ncut, a.status);
    }
    #pragma unroll
    for (int i = 0; i < D; ++i) {
        float hi = rp.u0[i * Pn + node], lo = rp.u0[(D + i) * Pn + node];
        df_add(hi, lo, rp.dc[DV * node + i] - (float)rp.mean[i]);  // u^n after the first projection
        rp.u1[i * Pn + node] = hi;
        rp.u1[(D + i) * Pn + node] = lo;
        df_add(hi, lo, hdt * v[i]);  // u*^{n+1}
        a.ustar[i * Pn + node] = hi;
        a.ustar[(D + i) * Pn + node] = lo;
    }
    #pragma unroll
    for (int k = 0; k < D * D; ++k) a.Gst[k * Pn + node] = Gr[k];
}

// TMA start coordinates of a segment: element x of every population box, then the flag box
struct SegStarts {
    int2 sg;
    int x0, pad;
    int start[6];
};

template <int D, int halo> __device__ __forceinline__ SegStarts seg_starts(const Box &b, int2 sg) {
    SegStarts r;
    r.sg = sg;
    const int y = sg.y % b.ny, z = sg.y / b.ny;
    r.x0 = sg.x - sg.y * b.nx;
    r.pad = 0;
    #pragma unroll
    for (int q = 0; q < 6; ++q) {
        const int A = q >> 1, s = (q & 1) ? -1 : 1;  // pull source of direction q is m - s e_A
        int start = 0;
        if (q < 2 * D) {
            if (A == 0) {
                start = sg.x - halo;
            } else if (A == 1) {
                int yy = y - s;
                if (b.per[1]) yy = yy < 0 ? yy + b.ny : (yy >= b.ny ? yy - b.ny : yy);
                start = (z * b.ny + yy) * b.nx + r.x0;
            } else {
                int zz = z - s;
                if (b.per[2]) zz = zz < 0 ? zz + b.nz : (zz >= b.nz ? zz - b.nz : zz);
                start = (zz * b.ny + y) * b.nx + r.x0;
            }
        }
        r.start[q] = start;
    }
    return r;
}

// Windows (segments) per warp of the fused kernel: the tile a warp stages at once, each window on its
// own single-use barrier, computed in turn.  A warp waits for its copies before it computes, so the
// bytes an SM has in flight are its resident warps times one warp's staged bytes.  An FP32 stage
// (10 KB in 3D) keeps HBM busy with one window per warp; a BF16 stage is half that, so the BF16
// default stages two.  lbm_autotune times 1, 2 and 4 on the caller's workload.
template <typename pop> constexpr int kTmaWindows = sizeof(pop) == 2 ? 2 : 1;

// lane 0: issue the bulk copies of one window (population boxes, u* box, flag bytes) on `bar`
template <int D, typename pop>
__device__ __forceinline__ void issue_window(const StepArgs<float> &a, const TmaMaps &maps, char *cur, uint64_t *bar,
                                             int2 sg) {
    using L = TmaLayout<D, sizeof(pop)>;
    constexpr int K = L::K, Q = L::Q;
    mbar_init(bar, 1);
    mbar_fence_init();
    const SegStarts st = seg_starts<D, L::halo>(a.b, sg);
    mbar_arrive_expect_tx(bar, L::stage_tx);
    tma_load_2d(cur + L::us_off, &maps.ustar, bar, st.sg.x, 0);
    tma_load_2d(cur + L::fl_off, &maps.flags, bar, st.x0, st.sg.y);
    #pragma unroll
    for (int q = 0; q < Q; ++q)
        tma_load_2d(cur + L::slot(q), (q >> 1) == 0 ? &maps.wide : &maps.narrow, bar, st.start[q], q * K);
}

// one staged window: closure, recovery, collision, stores.  Every lane inside the row stores:
// inactive nodes receive zeros, so each warp writes whole 32-byte sectors of every plane (a partly
// written sector costs the memory system a read of the rest).  Nothing reads an inactive node's
// populations or u*: pulls across cut links are replaced by the closure.  Lanes past the row end
// belong to the next row and store nothing.
template <int D, typename pop, bool REPAIR>
__device__ __forceinline__ void collide_window(const StepArgs<float> &a, const RepairArgs &rp, char *cur, int2 sg,
                                               int lane, long long l0pre, int gpre, const float *Gc,
                                               const bool *own) {
    using L = TmaLayout<D, sizeof(pop)>;
    const int x = sg.x - sg.y * a.b.nx + lane;
    if (x >= a.b.nx) return;
    const int node = sg.x + lane;
    const uint8_t fl = reinterpret_cast<const uint8_t *>(cur + L::fl_off)[lane];
    const bool act = fl & kActive;
    float us[2 * D];
    #pragma unroll
    for (int d = 0; d < 2 * D; ++d) us[d] = reinterpret_cast<const float *>(cur + L::us_off)[d * 32 + lane];
    const long long l0 = (fl & kCutMask) ? l0pre : 0;
    if (act) tma_closure<D, pop>(a, cur, node, x, lane, fl & kCutMask, l0);
    float mu = a.mtab ? a.mtab[2 * gpre] : a.mu;
    const float lam = a.mtab ? a.mtab[2 * gpre + 1] : a.lam;
    if (a.mu_field) mu = a.mu_field[node];
    if constexpr (REPAIR) repair_staged<D, pop>(a, rp, cur, node, lane, fl, l0, act, mu, lam, Gc, own);
    else collide_staged<D, pop>(a, cur, node, lane, fl, us, l0, act, mu, lam);
}

// K3 with TMA staging (FP32 arithmetic): one warp per block, NW 32-node windows per warp.  Lane 0 issues the bulk copies of the warp's windows; every lane waits on each window's
// barrier (bounded) before computing it, so no warp can leave while one of its copies is in flight.
// REPAIR: the repair step of a projection step (repair_staged) instead of the plain collision.
template <int D, typename pop = float, int NW = kTmaWindows<pop>, bool REPAIR = false>
__global__ void __launch_bounds__(32, 16) k_stream_collide_tma(const StepArgs<float> a,
                                                              const __grid_constant__ TmaMaps maps,
                                                              const RepairArgs rp) {
    using L = TmaLayout<D, sizeof(pop)>;
    extern __shared__ __align__(128) char smem[];
    const int lane = threadIdx.x & 31;
    const int sg0 = blockIdx.x * NW;
    if (sg0 >= a.nseg) return;
    const int nw = min(NW, a.nseg - sg0);
    uint64_t *const bars = reinterpret_cast<uint64_t *>(smem + NW * L::stage_bytes);
    int2 sg[NW];
    #pragma unroll
    for (int w = 0; w < NW; ++w) sg[w] = w < nw ? __ldg(&a.seg[sg0 + w]) : make_int2(0, 0);
    if (lane == 0)
        #pragma unroll
        for (int w = 0; w < NW; ++w)
            if (w < nw) issue_window<D, pop>(a, maps, smem + w * L::stage_bytes, bars + w, sg[w]);
    // first cut link and group of each node (used by boundary nodes and multi-specimen bodies),
    // fetched while the copies are in flight; lanes past the end of the last row read a clamped
    // index and never use it
    long long l0pre[NW];
    int gpre[NW];
    #pragma unroll
    for (int w = 0; w < NW; ++w) {
        const int node = sg[w].x + lane;
        const int nc = node < a.b.npad ? node : a.b.npad - 1;
        l0pre[w] = __ldg(a.lstart + nc);
        gpre[w] = a.mtab ? __ldg(a.mat + nc) : 0;
    }
    // the repair's corrected gradient (one window per warp), also while the copies are in flight
    float Gc[REPAIR ? D * D : 1];
    bool own[REPAIR ? D : 1];
    if constexpr (REPAIR) {
        static_assert(!REPAIR || NW == 1, "the repair runs one window per warp");
        const int x = sg[0].x - sg[0].y * a.b.nx + lane;
        const int node = sg[0].x + lane;
        const uint8_t fl = x < a.b.nx ? __ldg(a.flags + node) : 0;
        if (fl & kActive) repair_gradient<D>(a, rp, node, x, sg[0].y % a.b.ny, sg[0].y / a.b.ny, fl, Gc, own);
    }
    __syncwarp();
    #pragma unroll
    for (int w = 0; w < NW; ++w) {
        if (w >= nw) break;
        if (!__all_sync(0xffffffffu, mbar_wait_bounded(bars + w, 0, a.spin))) {
            if (lane == 0) set_status(a.status, kStTimeout);
            for (int v = w; v < nw; ++v) mbar_wait_bounded(bars + v, 0);  // copies in flight land first
            return;
        }
        collide_window<D, pop, REPAIR>(a, rp, smem + w * L::stage_bytes, sg[w], lane, l0pre[w], gpre[w], Gc, own);
    }
}

// projection steps, part 1, with TMA staging (FP32)
// WRITE_F: also store the gathered f^n (for the plain-load repair); the staged repair re-gathers it
template <int D, typename pop = float, bool WRITE_F = true>
__global__ void __launch_bounds__(128) k_gather_moments_tma(const StepArgs<float> a, const __grid_constant__ TmaMaps maps) {
    constexpr int K = D + D * D, Q = 2 * D;
    using L = TmaLayout<D, sizeof(pop)>;
    extern __shared__ __align__(128) char smem[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int sgi = blockIdx.x * 4 + warp;
    if (sgi >= a.nseg) return;
    char *wsm = smem + warp * L::warp_bytes;
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem + 4 * L::warp_bytes) + warp;
    const int2 sg = __ldg(&a.seg[sgi]);
    const long long P = a.b.npad;
    // the node's flags, first cut link and u* pair are loaded before the warp waits for its copies
    // (lanes past the end of the row read their in-range slot and never use it)
    const int x = sg.x - sg.y * a.b.nx + lane;
    const int node = sg.x + lane;
    const uint8_t fl = __ldg(a.flags + node);
    const long long l0 = __ldg(a.lstart + node);
    float ush[D], usl[D];
    #pragma unroll
    for (int i = 0; i < D; ++i) {
        ush[i] = a.ustar[i * P + node];
        usl[i] = a.ustar[(D + i) * P + node];
    }
    if (!tma_gather_segment<D, pop>(a.b, &maps.wide, &maps.narrow, wsm, bar, sg, lane, a.status, a.spin)) return;
    if (x >= a.b.nx) return;
    if (!(fl & kActive)) return;
    tma_closure<D, pop>(a, wsm, node, x, lane, fl & kCutMask, (fl & kCutMask) ? l0 : 0);
    float v[D];
    const float hdt = 0.5f * a.dt;
    const float inv_damp = 1.0f / (1.0f + hdt * a.gamma);
    #pragma unroll
    for (int k = 0; k < K; ++k) {
        float s = staged<D, pop>(wsm, 0, k, lane);
        if (WRITE_F) pop_st<float, pop>(a.fdst, (long long)(0 * K + k) * P + node, s);
        #pragma unroll
        for (int q = 1; q < Q; ++q) {
            const float fq = staged<D, pop>(wsm, q, k, lane);
            if (WRITE_F) pop_st<float, pop>(a.fdst, (long long)(q * K + k) * P + node, fq);
            s += fq;
        }
        if (k < D) v[k] = (s + hdt * a.bf[k]) * inv_damp;  // as collide_staged and repair_staged
        else a.Gst[(k - D) * P + node] = s;
    }
    #pragma unroll
    for (int i = 0; i < D; ++i) {
        a.vst[i * P + node] = v[i];
        float hi = ush[i], lo = usl[i];
        df_add(hi, lo, 0.5f * a.dt * v[i]);
        a.u0[i * P + node] = hi;
        a.u0[(D + i) * P + node] = lo;
    }
}

}  // namespace tlv
