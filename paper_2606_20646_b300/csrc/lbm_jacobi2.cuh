// Two damped-Jacobi sweeps of the compatibility projection (Sec. 3.5) per launch, FP32 forms,
// boxes with no periodic axis.
//
// A block owns a tile of the box and marches along its last axis (z in 3D, y in 2D), one plane per
// step.  Each plane of the correction d and of the residual (r, w) is copied into a ring of shared
// stages by one bulk tensor copy (a single-use mbarrier phase per plane, bounded waits); the first
// sweep's values d' of the plane are computed from the staged d into a ring of four d' planes, and
// the second sweep's values d'' of the plane behind it from those d' planes, then stored.  Halos of
// two nodes (d) and one node (d') in the tile's other directions are recomputed by the block, so
// blocks need nothing from one another; a plane of d and r comes from DRAM once per two sweeps.
//
// Every node update is the one-sweep kernel's, term for term and in the same order (the residual,
// then the neighbours q = 0 .. 2D-1 with the terms across cut links dropped, then
// fma(w, acc, (1 - beta) d)), so two sweeps here are bit-identical to two launches of k_jacobi.
#pragma once

#include "lbm_proj.cuh"
#include "lbm_tma.cuh"

namespace tlv {

// Tile constants (compile-time; the values below are the measured best: ring depth 4 in 3D and 5 in
// 2D, 3D tiles of 8 rows and 32 planes, 2D tiles of 32 rows).
#ifndef TLV_JP_STAGES3
#define TLV_JP_STAGES3 4
#endif
#ifndef TLV_JP_STAGES2
#define TLV_JP_STAGES2 5
#endif
#ifndef TLV_JP_CHUNK3
#define TLV_JP_CHUNK3 32
#endif
#ifndef TLV_JP_CHUNK2
#define TLV_JP_CHUNK2 32
#endif
// staged planes: p-1 .. p+1 in use around the plane p whose d' is computed, the rest in flight
template <int D> constexpr int kJPStages = D == 3 ? TLV_JP_STAGES3 : TLV_JP_STAGES2;
static_assert(kJPStages<3> >= 4 && kJPStages<2> >= 4, "a stage is refilled two planes behind the plane in use");
constexpr int kJPDp = 4;      // d' planes kept: p-2 .. p and the next
#ifndef TLV_JP_TY
#define TLV_JP_TY 8
#endif
constexpr int kJPTy = TLV_JP_TY;  // 3D: output rows (y) of a tile; 28 output columns (x); kJPChunk3 planes (z)
constexpr int kJPChunk3 = TLV_JP_CHUNK3;
constexpr int kJPW2 = 8;      // 2D: warps of a tile, 28 output columns each; kJPChunk2 rows (y)
constexpr int kJPChunk2 = TLV_JP_CHUNK2;

// orders this thread's earlier shared-memory accesses (after a block barrier: every thread's) before
// the bulk copies it issues next into the same bytes
__device__ __forceinline__ void fence_proxy_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ void tma_load_3d(void *dst, const CUtensorMap *map, uint64_t *bar, int c0, int c1, int c2) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];" ::
            "r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(smem_u32(bar))
        : "memory");
}

// the sweep's blend (1 - beta) d + w acc, rounded as in k_jacobi
__device__ __forceinline__ float jp_blend(float beta1, float dold, float w, float acc) {
    return __fmaf_rn(w, acc, __fmul_rn(beta1, dold));
}

// tensor maps of the sweep: the two correction buffers and the residual (2D: r for the first 768
// floats of a staged row, rt for its tail)
struct JPairMaps {
    CUtensorMap d[2];
    CUtensorMap r, rt;
};

template <int D> struct JPairLayout;
template <> struct JPairLayout<3> {
    static constexpr int RD = kJPTy + 4, RR = kJPTy + 2;  // staged rows of d and of r / d'
    static constexpr int d_bytes = RD * 32 * 16;           // box (128, RD, 1) floats
    static constexpr int r_bytes = RR * 32 * 16;           // box (128, RR, 1)
    static constexpr int stage_bytes = d_bytes + r_bytes;
    static constexpr int dp_bytes = RR * 32 * 16;
    static constexpr int threads = RR * 32;
    static constexpr int smem_bytes = kJPStages<3> * stage_bytes + kJPDp * dp_bytes + kJPStages<3> * 8;
};
template <> struct JPairLayout<2> {
    static constexpr int NP = 28 * kJPW2 + 4;                        // staged positions of a row
    static constexpr int d_bytes = ((NP * 8 + 127) / 128) * 128;     // box (NP, 1) of 8-byte pairs
    static constexpr int r_bytes = ((NP * 16 + 127) / 128) * 128;    // boxes (256, 1) x 3 and (r_tail, 1) floats
    static constexpr int r_tail = 4 * NP - 768;
    static constexpr int stage_bytes = d_bytes + r_bytes;
    static constexpr int dp_bytes = ((NP * 8 + 127) / 128) * 128;
    static constexpr int threads = kJPW2 * 32;
    static constexpr int smem_bytes = kJPStages<2> * stage_bytes + kJPDp * dp_bytes + kJPStages<2> * 8;
};
static_assert(JPairLayout<2>::r_tail > 0 && JPairLayout<2>::r_tail <= 256 && JPairLayout<2>::r_tail % 4 == 0 &&
                  3072 + 4 * JPairLayout<2>::r_tail <= JPairLayout<2>::r_bytes,
              "a staged residual row is three 256-float boxes and a tail box");

// tiles of the box: (ntx, nty, ntz) in 3D, (ntx, nty) in 2D; t = tx + ntx (ty + nty tz)
__host__ __device__ inline void jp_tile_grid(int D, int nx, int ny, int nz, int &ntx, int &nty, int &ntz) {
    if (D == 3) {
        ntx = (nx + 27) / 28;
        nty = (ny + kJPTy - 1) / kJPTy;
        ntz = (nz + kJPChunk3 - 1) / kJPChunk3;
    } else {
        ntx = (nx + 28 * kJPW2 - 1) / (28 * kJPW2);
        nty = (ny + kJPChunk2 - 1) / kJPChunk2;
        ntz = 1;
    }
}

// tiles whose output nodes include an active node: one thread per node, flag[tile] = 1
static __global__ void k_jp_mark(Box b, const uint8_t *__restrict__ flags, int *tflag) {
    const long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (n >= b.nbox || !(flags[n] & kActive)) return;
    int ntx, nty, ntz;
    jp_tile_grid(b.D, b.nx, b.ny, b.nz, ntx, nty, ntz);
    const int x = (int)(n % b.nx), r = (int)(n / b.nx), y = r % b.ny, z = r / b.ny;
    const int t = b.D == 3 ? x / 28 + ntx * (y / kJPTy + nty * (z / kJPChunk3)) : x / (28 * kJPW2) + ntx * (y / kJPChunk2);
    tflag[t] = 1;
}

static __global__ void k_jp_compact(const int *__restrict__ tflag, const int *__restrict__ pos, int nt, int *tiles) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < nt && tflag[t]) tiles[pos[t]] = t;
}

// one update of a node, the plain sweep's arithmetic: r, then the neighbours in direction order
template <int Q>
__device__ __forceinline__ float3 jp_update(float beta1, float4 own, float4 rw, unsigned cut, const float4 (&nb)[Q]) {
    float acc[3] = {rw.x, rw.y, rw.z};
    #pragma unroll
    for (int q = 0; q < Q; ++q) {
        const bool c = (cut >> q) & 1;
        acc[0] += c ? 0.0f : nb[q].x;
        acc[1] += c ? 0.0f : nb[q].y;
        acc[2] += c ? 0.0f : nb[q].z;
    }
    return make_float3(jp_blend(beta1, own.x, rw.w, acc[0]), jp_blend(beta1, own.y, rw.w, acc[1]),
                       jp_blend(beta1, own.z, rw.w, acc[2]));
}

// 3D: a tile is 28 columns (x0 .. x0+27) x kJPTy rows (y0 ..) x up to kJPChunk3 planes (z0 .. z1-1).
// Warp w holds row y0-1+w (d' rows y0-1 .. y0+kJPTy), lane l column x0-2+l.  d is staged for rows
// y0-2 .. y0+kJPTy+1 (row w+1 of the stage is warp w's), r for rows y0-1 .. y0+kJPTy.
static __global__ void __launch_bounds__(JPairLayout<3>::threads, 2)
    k_jacobi_pair3(const ProjArgs<float> a, const __grid_constant__ CUtensorMap dmap,
                   const __grid_constant__ CUtensorMap rmap, int dzero, float *__restrict__ dout,
                   const int *__restrict__ tiles, int spin) {
    using L = JPairLayout<3>;
    extern __shared__ __align__(128) char smem[];
    uint64_t *const bars = reinterpret_cast<uint64_t *>(smem + kJPStages<3> * L::stage_bytes + kJPDp * L::dp_bytes);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nx = a.b.nx, ny = a.b.ny, nz = a.b.nz;
    int ntx, nty, ntz;
    jp_tile_grid(3, nx, ny, nz, ntx, nty, ntz);
    const int t = tiles[blockIdx.x];
    const int x0 = 28 * (t % ntx), y0 = kJPTy * ((t / ntx) % nty), z0 = kJPChunk3 * (t / (ntx * nty));
    const int z1 = min(z0 + kJPChunk3, nz);
    const int x = x0 - 2 + lane, y = y0 - 1 + warp;
    const bool col_in = x >= 0 && x < nx && y >= 0 && y < ny;
    const float beta1 = 1.0f - (float)a.beta;
    const uint32_t tx = (dzero ? 0 : L::d_bytes) + L::r_bytes;
    const int p0 = z0 - 2, plast = z1 + 1;  // staged planes p0 .. plast, local index p - p0
    if (threadIdx.x == 0) {
        for (int s = 0; s < kJPStages<3>; ++s) mbar_init(bars + s, 1);
        mbar_fence_init();
    }
    __syncthreads();
    auto issue = [&](int p) {
        const int j = p - p0, s = j % kJPStages<3>;
        char *st = smem + s * L::stage_bytes;
        fence_proxy_async_smem();
        mbar_arrive_expect_tx(bars + s, tx);
        // float coordinate 4 (x0 - 2): a multiple of 4 floats, as the copies need
        if (!dzero) tma_load_3d(st, &dmap, bars + s, 4 * (x0 - 2), y0 - 2, p);
        tma_load_3d(st + L::d_bytes, &rmap, bars + s, 4 * (x0 - 2), y0 - 1, p);
    };
    auto wait = [&](int p, int lim) {
        const int j = p - p0;
        return mbar_wait_bounded(bars + j % kJPStages<3>, (j / kJPStages<3>) & 1, lim);
    };
    auto dst = [&](int p) { return reinterpret_cast<const float4 *>(smem + ((p - p0) % kJPStages<3>) * L::stage_bytes); };
    auto rst = [&](int p) {
        return reinterpret_cast<const float4 *>(smem + ((p - p0) % kJPStages<3>) * L::stage_bytes + L::d_bytes);
    };
    auto dps = [&](int p) {
        return reinterpret_cast<float4 *>(smem + kJPStages<3> * L::stage_bytes + ((p - p0) & (kJPDp - 1)) * L::dp_bytes);
    };
    auto flag_at = [&](int p) -> uint8_t {
        return (col_in && p >= 0 && p < nz) ? __ldg(a.flags + (x + nx * (y + ny * p))) : uint8_t(0);
    };
    if (threadIdx.x == 0)
        for (int p = p0; p <= min(p0 + kJPStages<3> - 2, plast); ++p) issue(p);
    int issued = min(p0 + kJPStages<3> - 2, plast), done = p0 - 1;  // planes issued, planes known complete
    bool ok = true;
    for (int p = p0; p <= p0 + 1 && ok; ++p)
        if ((ok = wait(p, spin))) done = p;
    uint8_t f_prev = 0, f_cur = flag_at(z0 - 1), f_next = flag_at(z0);
    const float4 zero4 = make_float4(0.f, 0.f, 0.f, 0.f);
    for (int z = z0 - 1; z <= z1; ++z) {
        if (ok && (ok = wait(z + 1, spin))) done = z + 1;
        // first sweep: d'(z) of this thread's node (rows y0-1 .. y0+kJPTy, columns x0-1 .. x0+28)
        {
            const float4 *D0 = dst(z), *Dm = dst(z - 1), *Dp = dst(z + 1);
            const int rw = (warp + 1) * 32 + lane;  // own slot in the d stage
            const float4 own = dzero ? zero4 : D0[rw];
            float4 out = own;
            if (lane >= 1 && lane <= 30 && (f_cur & kActive)) {
                const float4 r = rst(z)[warp * 32 + lane];
                if (r.w > 0.0f) {
                    float4 nb[6];
                    if (dzero) {
                        #pragma unroll
                        for (int q = 0; q < 6; ++q) nb[q] = zero4;
                    } else {
                        nb[0] = D0[rw + 1];
                        nb[1] = D0[rw - 1];
                        nb[2] = D0[rw + 32];
                        nb[3] = D0[rw - 32];
                        nb[4] = Dp[rw];
                        nb[5] = Dm[rw];
                    }
                    const float3 o = jp_update<6>(beta1, own, r, f_cur & kCutMask, nb);
                    out = make_float4(o.x, o.y, o.z, 0.0f);
                }
            }
            dps(z)[warp * 32 + lane] = out;
        }
        // every warp has its d'(z) in place (and every wait of this step succeeded)
        if (__syncthreads_or(!ok)) {
            ok = false;
            break;
        }
        // second sweep: d''(z-1) of the tile's own nodes (rows y0 .. y0+kJPTy-1, columns x0 .. x0+27)
        if (z - 1 >= z0 && warp >= 1 && warp <= kJPTy && lane >= 2 && lane <= 29 && (f_prev & kActive)) {
            const float4 r = rst(z - 1)[warp * 32 + lane];
            if (r.w > 0.0f) {
                const float4 *P0 = dps(z - 1), *Pm = dps(z - 2), *Pp = dps(z);
                const int o = warp * 32 + lane;
                const float4 nb[6] = {P0[o + 1], P0[o - 1], P0[o + 32], P0[o - 32], Pp[o], Pm[o]};
                const float3 v = jp_update<6>(beta1, P0[o], r, f_prev & kCutMask, nb);
                // the fourth value: the node's cut bits, which a one-sweep launch after this one reads
                *reinterpret_cast<float4 *>(dout + 4LL * (x + nx * (y + ny * (z - 1)))) =
                    make_float4(v.x, v.y, v.z, __uint_as_float(f_prev & kCutMask));
            }
        }
        // the stage of plane z-2 is free (its d fed d'(z-1), its r d''(z-2)): refill it with the plane
        // kJPStages - 2 ahead
        if (threadIdx.x == 0 && z + kJPStages<3> - 2 <= plast) {
            issue(z + kJPStages<3> - 2);
            issued = z + kJPStages<3> - 2;
        }
        f_prev = f_cur;
        f_cur = f_next;
        f_next = flag_at(z + 2);
    }
    if (!ok && threadIdx.x == 0) {
        // a wait ran out: latch the status and wait for every copy still in flight before the
        // block's shared memory is released
        set_status(a.status, kStTimeout);
        for (int p = done + 1; p <= issued; ++p) wait(p, kTmaSpin);
    }
}

// 2D: a tile is 28 kJPW2 columns (x0 ..) x up to kJPChunk2 rows (y0 .. y1-1), marching along y.
// Staged row positions i = 0 .. NP-1 are columns x0-2+i; warp k, lane l holds position 28k+l.  The
// correction's map has 8-byte elements (one (d_1, d_2) pair per node), so that the staged row is a
// whole number of 16-byte units; x0 - 2 is even, as the 8-byte elements need.
static __global__ void __launch_bounds__(JPairLayout<2>::threads, 4)
    k_jacobi_pair2(const ProjArgs<float> a, const __grid_constant__ CUtensorMap dmap,
                   const __grid_constant__ CUtensorMap rmap, const __grid_constant__ CUtensorMap rtmap, int dzero,
                   float *__restrict__ dout,
                   const int *__restrict__ tiles, int spin) {
    using L = JPairLayout<2>;
    extern __shared__ __align__(128) char smem[];
    uint64_t *const bars = reinterpret_cast<uint64_t *>(smem + kJPStages<2> * L::stage_bytes + kJPDp * L::dp_bytes);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nx = a.b.nx, ny = a.b.ny;
    int ntx, nty, ntz;
    jp_tile_grid(2, nx, ny, 1, ntx, nty, ntz);
    const int t = tiles[blockIdx.x];
    const int x0 = 28 * kJPW2 * (t % ntx), y0 = kJPChunk2 * (t / ntx);
    const int y1 = min(y0 + kJPChunk2, ny);
    const int i = 28 * warp + lane;  // staged position
    const int x = x0 - 2 + i;
    // d' positions 1 .. NP-2 split between the warps without overlap; d'' positions 2 .. NP-3
    const bool dp_mine = (lane >= 2 && lane <= 29) || (warp == 0 && lane == 1) || (warp == kJPW2 - 1 && lane == 30);
    const bool out_mine = lane >= 2 && lane <= 29;
    const float beta1 = 1.0f - (float)a.beta;
    const uint32_t tx = (dzero ? 0 : L::NP * 8) + L::NP * 16;
    const int p0 = y0 - 2, plast = y1 + 1;
    if (threadIdx.x == 0) {
        for (int s = 0; s < kJPStages<2>; ++s) mbar_init(bars + s, 1);
        mbar_fence_init();
    }
    __syncthreads();
    auto issue = [&](int p) {
        const int j = p - p0, s = j % kJPStages<2>;
        char *st = smem + s * L::stage_bytes;
        fence_proxy_async_smem();
        mbar_arrive_expect_tx(bars + s, tx);
        if (!dzero) tma_load_2d(st, &dmap, bars + s, x0 - 2, p);
        // the residual row in four pieces at 1 KB-aligned offsets (a box holds at most 256 floats)
        #pragma unroll
        for (int k = 0; k < 3; ++k) tma_load_2d(st + L::d_bytes + 1024 * k, &rmap, bars + s, 4 * (x0 - 2) + 256 * k, p);
        tma_load_2d(st + L::d_bytes + 3072, &rtmap, bars + s, 4 * (x0 - 2) + 768, p);
    };
    auto wait = [&](int p, int lim) {
        const int j = p - p0;
        return mbar_wait_bounded(bars + j % kJPStages<2>, (j / kJPStages<2>) & 1, lim);
    };
    auto dst = [&](int p) { return reinterpret_cast<const float2 *>(smem + ((p - p0) % kJPStages<2>) * L::stage_bytes); };
    auto rst = [&](int p) {
        return reinterpret_cast<const float4 *>(smem + ((p - p0) % kJPStages<2>) * L::stage_bytes + L::d_bytes);
    };
    auto dps = [&](int p) {
        return reinterpret_cast<float2 *>(smem + kJPStages<2> * L::stage_bytes + ((p - p0) & (kJPDp - 1)) * L::dp_bytes);
    };
    auto f4 = [](float2 v) { return make_float4(v.x, v.y, 0.0f, 0.0f); };
    if (threadIdx.x == 0)
        for (int p = p0; p <= min(p0 + kJPStages<2> - 2, plast); ++p) issue(p);
    int issued = min(p0 + kJPStages<2> - 2, plast), done = p0 - 1;
    bool ok = true;
    for (int p = p0; p <= p0 + 1 && ok; ++p)
        if ((ok = wait(p, spin))) done = p;
    const float2 zero2 = make_float2(0.f, 0.f);
    for (int y = y0 - 1; y <= y1; ++y) {
        if (ok && (ok = wait(y + 1, spin))) done = y + 1;
        if (dp_mine) {
            const float2 *D0 = dst(y), *Dm = dst(y - 1), *Dp = dst(y + 1);
            const float2 own = dzero ? zero2 : D0[i];
            float2 out = own;
            {
                // 2D residual record (r_1, r_2, w, cut bits); w = 0 at inactive and out-of-box positions
                const float4 r2 = rst(y)[i];
                const float4 r = make_float4(r2.x, r2.y, 0.0f, r2.z);
                if (r.w > 0.0f) {
                    float4 nb[4];
                    if (dzero) {
                        #pragma unroll
                        for (int q = 0; q < 4; ++q) nb[q] = make_float4(0.f, 0.f, 0.f, 0.f);
                    } else {
                        nb[0] = f4(D0[i + 1]);
                        nb[1] = f4(D0[i - 1]);
                        nb[2] = f4(Dp[i]);
                        nb[3] = f4(Dm[i]);
                    }
                    const float3 o = jp_update<4>(beta1, f4(own), r, __float_as_uint(r2.w) & kCutMask, nb);
                    out = make_float2(o.x, o.y);
                }
            }
            dps(y)[i] = out;
        }
        if (__syncthreads_or(!ok)) {
            ok = false;
            break;
        }
        if (y - 1 >= y0 && out_mine) {
            const float4 r2 = rst(y - 1)[i];
            const float4 r = make_float4(r2.x, r2.y, 0.0f, r2.z);
            if (r.w > 0.0f) {
                const float2 *P0 = dps(y - 1), *Pm = dps(y - 2), *Pp = dps(y);
                const float4 nb[4] = {f4(P0[i + 1]), f4(P0[i - 1]), f4(Pp[i]), f4(Pm[i])};
                const float3 v = jp_update<4>(beta1, f4(P0[i]), r, __float_as_uint(r2.w) & kCutMask, nb);
                *reinterpret_cast<float2 *>(dout + 2LL * (x + nx * (y - 1))) = make_float2(v.x, v.y);
            }
        }
        if (threadIdx.x == 0 && y + kJPStages<2> - 2 <= plast) {
            issue(y + kJPStages<2> - 2);
            issued = y + kJPStages<2> - 2;
        }
    }
    if (!ok && threadIdx.x == 0) {
        set_status(a.status, kStTimeout);
        for (int p = done + 1; p <= issued; ++p) wait(p, kTmaSpin);
    }
}

}  // namespace tlv
