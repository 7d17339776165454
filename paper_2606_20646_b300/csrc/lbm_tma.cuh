// TMA-staged gather for the FP32 fused collide-stream kernel (sm_103a).
//
// The pull gather of one 32-node x-segment reads, for every direction q, the K component
// planes of f* at the segment shifted by -e_q.  Population planes are consecutive in a
// 2D tensor (dim 0: node index, npad; dim 1: plane q*K + k), so the K planes of one
// direction are one box of (width, K).  One elected lane per warp issues Q bulk tensor
// copies into the warp's shared-memory slots, completed on a per-warp mbarrier:
//   +-x: box (40, K) starting 4 nodes before the segment (a TMA start coordinate must be a
//        multiple of 4 floats, so the +-1 shifted windows are read from an aligned wider box)
//   +-y, +-z: box (32, K) at the source row (periodic rows wrapped).
// The wait is bounded; on timeout the kernel latches a status bit, waits once more (bounded)
// for its copies in flight and returns without writing.
#pragma once

#include <cuda.h>

#include "lbm_kernels.cuh"

namespace tlv {

constexpr int kStTimeout = 128;        // device status bit: a TMA wait ran out
constexpr int kTmaSpin = 1 << 20;      // try_wait polls before giving up
constexpr int kTmaWide = 40, kTmaNarrow = 32;

template <int D> struct TmaLayout {
    static constexpr int K = D + D * D, Q = 2 * D;
    static constexpr int wide_bytes = ((kTmaWide * K * 4 + 127) / 128) * 128;
    static constexpr int narrow_bytes = ((kTmaNarrow * K * 4 + 127) / 128) * 128;
    static constexpr int warp_bytes = 2 * wide_bytes + (Q - 2) * narrow_bytes;
    static constexpr int tx_bytes = 2 * kTmaWide * K * 4 + (Q - 2) * kTmaNarrow * K * 4;
    // byte offset of direction q's slot in a warp region
    __device__ static constexpr int slot(int q) { return q < 2 ? q * wide_bytes : 2 * wide_bytes + (q - 2) * narrow_bytes; }
    __device__ static constexpr int width(int q) { return q < 2 ? kTmaWide : kTmaNarrow; }
    // element offset of lane 0's source inside the box row
    __device__ static constexpr int lane0(int q) { return q == 0 ? 3 : (q == 1 ? 5 : 0); }
    static constexpr int block_bytes(int warps) { return warps * warp_bytes + warps * 8; }
    // pipeline stage: population slots, then u* (D x 32 floats), flags (32 bytes), header (segment)
    static constexpr int us_off = warp_bytes;
    static constexpr int fl_off = us_off + ((D * 32 * 4 + 127) / 128) * 128;
    static constexpr int hdr_off = fl_off + 128;
    static constexpr int stage_bytes = hdr_off + 128;
    static constexpr int stage_tx = tx_bytes + D * 32 * 4 + 32;
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

__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity) {
    for (int it = 0; it < kTmaSpin; ++it)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}

// Issue the Q bulk copies of segment sg into the warp's slots and wait for them.  Returns false
// (status latched) if the wait ran out.  Every lane of the warp must call it.
template <int D>
__device__ __forceinline__ bool tma_gather_segment(const Box &b, const CUtensorMap *wide, const CUtensorMap *narrow,
                                                   char *wsm, uint64_t *bar, int2 sg, int lane, int *status) {
    using L = TmaLayout<D>;
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
                start = sg.x - 4;
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
    bool ok = mbar_wait_bounded(bar, 0);
    if (!ok) {
        if (lane == 0) set_status(status, kStTimeout);
        mbar_wait_bounded(bar, 0);  // let the copies in flight land before the block can exit
    }
    return __all_sync(0xffffffffu, ok);
}

// value of direction q, component k for this lane from the staged slots
template <int D> __device__ __forceinline__ float &staged(char *wsm, int q, int k, int lane) {
    using L = TmaLayout<D>;
    return reinterpret_cast<float *>(wsm + L::slot(q))[k * L::width(q) + L::lane0(q) + lane];
}

// gather + closure with TMA staging; the gathered (and reconstructed) values stay in shared memory
template <int D>
__device__ __forceinline__ void tma_closure(const StepArgs<float> &a, char *wsm, int node, int x, int lane,
                                            unsigned cut) {
    constexpr int K = D + D * D, Q = 2 * D, LREC = K + 2;
    const long long P = a.b.npad;
    const float *__restrict__ fs = a.fsrc;
    if (a.b.per[0]) {  // the aligned x windows do not wrap: patch the periodic ends
        if (x == 0 && !((cut >> 1) & 1))
            #pragma unroll
            for (int k = 0; k < K; ++k) staged<D>(wsm, 0, k, lane) = __ldg(fs + (long long)(0 * K + k) * P + node + a.b.nx - 1);
        if (x == a.b.nx - 1 && !(cut & 1))
            #pragma unroll
            for (int k = 0; k < K; ++k) staged<D>(wsm, 1, k, lane) = __ldg(fs + (long long)(1 * K + k) * P + node - (a.b.nx - 1));
    }
    if (!cut) return;
    const float *rec0 = a.lrec + (long long)__ldg(a.lstart + node) * LREC;
    #pragma unroll 1
    for (int q = 0; q < Q; ++q) {
        const int qo = q ^ 1;
        if ((cut >> qo) & 1) {
            const float *rec = rec0 + __popc(cut & ((1u << qo) - 1u)) * LREC;
            const float eta = rec[0];
            const bool neu = rec[1] != 0.0f;
            const bool up = !((cut >> q) & 1);
            #pragma unroll 4
            for (int k = 0; k < K; ++k) {
                const float Dk = ((k < D) == neu) ? 1.0f : -1.0f;
                const float S = rec[2 + k];
                const float fo = __ldg(fs + (long long)(qo * K + k) * P + node);
                const float fi = __ldg(fs + (long long)(q * K + k) * P + node);
                float r;
                if (eta >= 0.5f) {
                    r = (Dk * fo + S) / (2.0f * eta) + (1.0f - 1.0f / (2.0f * eta)) * fi;
                } else {
                    const float fu = up ? staged<D>(wsm, qo, k, lane) : fo;
                    r = Dk * (2.0f * eta * fo + (1.0f - 2.0f * eta) * fu) + S;
                }
                staged<D>(wsm, q, k, lane) = r;
            }
        }
    }
}

struct TmaMaps {
    CUtensorMap wide, narrow;  // population planes of the source buffer: (40, K) and (32, K) boxes
    CUtensorMap ustar;         // u* planes: (32, D) boxes
    CUtensorMap flags;         // flag bytes as (nx, ny*nz): (32, 1) boxes
};

__device__ __forceinline__ void fence_proxy_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// issue the bulk copies of segment sg into stage wsm (lane 0 only): Q population boxes, and with
// `with_meta` the segment's u* box and flag bytes plus a header holding sg
template <int D, bool with_meta = false>
__device__ __forceinline__ void tma_issue(const Box &b, const TmaMaps &maps, char *wsm, uint64_t *bar, int2 sg) {
    using L = TmaLayout<D>;
    constexpr int K = L::K, Q = L::Q;
    const int y = sg.y % b.ny, z = sg.y / b.ny, x0 = sg.x - sg.y * b.nx;
    // in the pipeline the consumer that released this stage fenced its generic-proxy writes before
    // arriving on the empty barrier; the warp-local double-buffered path fences here
    if constexpr (!with_meta) fence_proxy_async_smem();
    if constexpr (with_meta) {
        *reinterpret_cast<int2 *>(wsm + L::hdr_off) = sg;  // published by the arrive's release
        mbar_arrive_expect_tx(bar, L::stage_tx);
        tma_load_2d(wsm + L::us_off, &maps.ustar, bar, sg.x, 0);
        tma_load_2d(wsm + L::fl_off, &maps.flags, bar, x0, sg.y);
    } else {
        mbar_arrive_expect_tx(bar, L::tx_bytes);
    }
    #pragma unroll
    for (int q = 0; q < Q; ++q) {
        const int A = q >> 1, s = (q & 1) ? -1 : 1;  // pull source of direction q is m - s e_A
        int start;
        if (A == 0) {
            start = sg.x - 4;
        } else if (A == 1) {
            int yy = y - s;
            if (b.per[1]) yy = yy < 0 ? yy + b.ny : (yy >= b.ny ? yy - b.ny : yy);
            start = (z * b.ny + yy) * b.nx + x0;
        } else {
            int zz = z - s;
            if (b.per[2]) zz = zz < 0 ? zz + b.nz : (zz >= b.nz ? zz - b.nz : zz);
            start = (zz * b.ny + y) * b.nx + x0;
        }
        tma_load_2d(wsm + L::slot(q), A == 0 ? &maps.wide : &maps.narrow, bar, start, q * K);
    }
}

// recovery, collision and u quadrature of one node from its staged populations (FP32 form).
// Arithmetic is arranged to avoid divisions in the per-node path:
//   v = (sum f_v + dt/2 b) * 1/(1 + gamma dt/2),  F^{-T} = cof(F) * (1/J),
//   f*_q = (1 - omega) f_q + omega f^eq_q + src_q with omega f^eq_q = base_k +- (omega D/(2Dc)) Phi_A,k
template <int D>
__device__ __forceinline__ void collide_staged(const StepArgs<float> &a, char *wsm, int node, int lane, uint8_t fl,
                                               const float us[D]) {
    constexpr int K = D + D * D, Q = 2 * D;
    float S[K];
    #pragma unroll
    for (int k = 0; k < K; ++k) {
        float s = staged<D>(wsm, 0, k, lane);
        #pragma unroll
        for (int q = 1; q < Q; ++q) s += staged<D>(wsm, q, k, lane);
        S[k] = s;
    }
    const float hdt = 0.5f * a.dt;
    const float inv_damp = 1.0f / (1.0f + hdt * a.gamma);
    float v[D], F[D * D], C[D * D], P[D * D];
    #pragma unroll
    for (int i = 0; i < D; ++i) v[i] = (S[i] + hdt * a.bf[i]) * inv_damp;
    #pragma unroll
    for (int k = 0; k < D * D; ++k) F[k] = S[D + k] + ((k / D == k % D) ? 1.0f : 0.0f);
    cofactor<float, D>(F, C);
    const float J = det<float, D>(F);
    const float sJ = (0.5f * a.lam * (J * J - 1.0f) - a.mu) * (1.0f / J);
    #pragma unroll
    for (int k = 0; k < D * D; ++k) P[k] = a.mu * F[k] + sJ * C[k];
    float chk = J;
    #pragma unroll
    for (int i = 0; i < D; ++i) chk += v[i];
    #pragma unroll
    for (int k = 0; k < D * D; ++k) chk += P[k];
    if (!(J > 0.0f) || !isfinite(chk)) set_status(a.status, (J > 0.0f ? 0 : kStJacobian) | (isfinite(chk) ? 0 : kStNonfinite));
    const long long Pn = a.b.npad;
    #pragma unroll
    for (int i = 0; i < D; ++i) {
        const float un = us[i] + hdt * v[i];
        if (fl & kNeedU) a.un[i * Pn + node] = un;
        a.ustar[i * Pn + node] = un + hdt * v[i];
    }
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
    float *out = a.fdst + node;
    #pragma unroll
    for (int q = 0; q < Q; ++q) {
        const int A = q >> 1;
        const bool neg = q & 1;
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
            out[(long long)(q * K + k) * Pn] = fmaf(om1, staged<D>(wsm, q, k, lane), t);
        }
    }
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

constexpr int kPipeProducers = 2;                     // producer warps per CTA
constexpr int kPipeConsumers = 13;                    // consumer warps per CTA
constexpr int kPipeThreads = 32 * (kPipeProducers + kPipeConsumers);

// TMA start coordinates of a segment: element x of every population box, then the flag box
struct SegStarts {
    int2 sg;
    int x0, pad;
    int start[6];
};

template <int D> __device__ __forceinline__ SegStarts seg_starts(const Box &b, int2 sg) {
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
                start = sg.x - 4;
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

// K3 with TMA staging (FP32), warp-specialised and persistent: one CTA per SM.  Warps
// 0..kPipeProducers-1 are producers that stream the bulk copies of the CTA's segments
// (b, b + G, b + 2G, ...; producer p takes local segments t = p mod kPipeProducers) into a ring of
// `stages` shared-memory stages; consumer warp c computes local segments c, c + C, ... .  Stage
// t % stages has a full barrier (completed by the copies' bytes) and an empty barrier (arrived by
// the consumer when done with the stage).  Each producer batch of 32 segments has its start
// coordinates computed by all lanes into a shared table; lane 0 alone waits and issues.
template <int D>
__global__ void __launch_bounds__(kPipeThreads, 1) k_stream_collide_tma(const StepArgs<float> a,
                                                                     const __grid_constant__ TmaMaps maps, int stages) {
    using L = TmaLayout<D>;
    constexpr int K = L::K, Q = L::Q;
    extern __shared__ __align__(128) char smem[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int G = gridDim.x, b = blockIdx.x;
    uint64_t *full = reinterpret_cast<uint64_t *>(smem + (size_t)stages * L::stage_bytes);
    uint64_t *empty = full + stages;
    SegStarts *table = reinterpret_cast<SegStarts *>(empty + stages);  // [kPipeProducers][32]
    if (threadIdx.x == 0) {
        for (int s = 0; s < stages; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        mbar_fence_init();
    }
    __syncthreads();
    const int nlocal = a.nseg > b ? (a.nseg - b + G - 1) / G : 0;  // segments of this CTA
    if (warp < kPipeProducers) {
        // ---- producer p: local segments p, p + P, p + 2P, ... in batches of 32 ----
        SegStarts *tab = table + warp * 32;
        bool ok = true;
        for (int k0 = 0; ok; k0 += 32) {
            const int tfirst = warp + kPipeProducers * k0;
            if (tfirst >= nlocal) break;
            const int t = tfirst + kPipeProducers * lane;
            if (t < nlocal) tab[lane] = seg_starts<D>(a.b, __ldg(&a.seg[b + (long long)G * t]));
            __syncwarp();
            if (lane == 0) {
                for (int k = 0; k < 32; ++k) {
                    const int tk = tfirst + kPipeProducers * k;
                    if (tk >= nlocal) break;
                    const int s = tk % stages, use = tk / stages;
                    if (use > 0 && !mbar_wait_bounded(&empty[s], (use - 1) & 1)) { ok = false; break; }
                    const SegStarts st = tab[k];
                    char *wsm = smem + (size_t)s * L::stage_bytes;
                    *reinterpret_cast<int2 *>(wsm + L::hdr_off) = st.sg;  // published by the arrive's release
                    mbar_arrive_expect_tx(&full[s], L::stage_tx);
                    tma_load_2d(wsm + L::us_off, &maps.ustar, &full[s], st.sg.x, 0);
                    tma_load_2d(wsm + L::fl_off, &maps.flags, &full[s], st.x0, st.sg.y);
                    #pragma unroll
                    for (int q = 0; q < Q; ++q)
                        tma_load_2d(wsm + L::slot(q), (q >> 1) == 0 ? &maps.wide : &maps.narrow, &full[s], st.start[q],
                                    q * K);
                }
            }
            ok = __shfl_sync(0xffffffffu, ok, 0);
            __syncwarp();  // the table is rewritten by the next batch
        }
        if (!ok && lane == 0) set_status(a.status, kStTimeout);
        // before the CTA can retire, every copy this producer issued must have landed
        if (lane == 0)
            for (int t = warp; t < nlocal; t += kPipeProducers)
                if (t >= nlocal - stages) mbar_wait_bounded(&full[t % stages], (t / stages) & 1);
        return;
    }
    // ---- consumers ----
    for (int t = warp - kPipeProducers; t < nlocal; t += kPipeConsumers) {
        const int s = t % stages, use = t / stages;
        char *const cur = smem + (size_t)s * L::stage_bytes;
        if (!__all_sync(0xffffffffu, mbar_wait_bounded(&full[s], use & 1))) {
            if (lane == 0) set_status(a.status, kStTimeout);
            return;
        }
        // segment, flags and u* come with the stage: no global load on the interior path
        const int2 sg = *reinterpret_cast<const int2 *>(cur + L::hdr_off);
        const int x = sg.x - sg.y * a.b.nx + lane;
        const int node = sg.x + lane;
        const uint8_t fl = x < a.b.nx ? reinterpret_cast<const uint8_t *>(cur + L::fl_off)[lane] : (uint8_t)0;
        const bool act = fl & kActive;
        float us[D];
        #pragma unroll
        for (int d = 0; d < D; ++d) us[d] = reinterpret_cast<const float *>(cur + L::us_off)[d * 32 + lane];
        if (act) {
            tma_closure<D>(a, cur, node, x, lane, fl & kCutMask);
            collide_staged<D>(a, cur, node, lane, fl, us);
        }
        __syncwarp();
        if (lane == 0) {
            fence_proxy_async_smem();  // this stage's shared-memory writes precede its next refill
            mbar_arrive(&empty[s]);
        }
    }
}

// projection steps, part 1, with TMA staging (FP32)
template <int D>
__global__ void __launch_bounds__(128) k_gather_moments_tma(const StepArgs<float> a, const __grid_constant__ TmaMaps maps) {
    constexpr int K = D + D * D, Q = 2 * D;
    using L = TmaLayout<D>;
    extern __shared__ __align__(128) char smem[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int sgi = blockIdx.x * 4 + warp;
    if (sgi >= a.nseg) return;
    char *wsm = smem + warp * L::warp_bytes;
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem + 4 * L::warp_bytes) + warp;
    const int2 sg = __ldg(&a.seg[sgi]);
    if (!tma_gather_segment<D>(a.b, &maps.wide, &maps.narrow, wsm, bar, sg, lane, a.status)) return;
    const int x = sg.x - sg.y * a.b.nx + lane;
    if (x >= a.b.nx) return;
    const int node = sg.x + lane;
    const uint8_t fl = __ldg(a.flags + node);
    if (!(fl & kActive)) return;
    tma_closure<D>(a, wsm, node, x, lane, fl & kCutMask);
    const long long P = a.b.npad;
    float v[D];
    #pragma unroll
    for (int k = 0; k < K; ++k) {
        float s = staged<D>(wsm, 0, k, lane);
        a.fdst[(long long)(0 * K + k) * P + node] = s;
        #pragma unroll
        for (int q = 1; q < Q; ++q) {
            const float fq = staged<D>(wsm, q, k, lane);
            a.fdst[(long long)(q * K + k) * P + node] = fq;
            s += fq;
        }
        if (k < D) v[k] = (s + 0.5f * a.dt * a.bf[k]) / (1.0f + 0.5f * a.dt * a.gamma);
        else a.Gst[(k - D) * P + node] = s;
    }
    #pragma unroll
    for (int i = 0; i < D; ++i) {
        a.vst[i * P + node] = v[i];
        a.u0[i * P + node] = (double)a.ustar[i * P + node] + 0.5 * (double)a.dt * (double)v[i];
    }
}

}  // namespace tlv
