// sm_103a kernels of the total-Lagrangian vectorial LBM on embedded curved domains.
//
// Storage (device, caller-owned):
//   populations  f~ = f - f^eq(0, I): one plane per (q, k), plane (q*K + k) of npad
//                entries, node index x + nx*(y + ny*z).  Only the F-diagonal rows are
//                shifted (by 1/(2D)), so F - I is summed without cancellation.
//   flags        one byte per node: bit q = link (m, q) cut, kActive, kNeedU.
//   links        cut links sorted by (node, q); record = [eta, kind, S~_0..S~_{K-1}].
// The stored population state between steps is post-collision f*^{n-1}; the next
// step's pull gather performs the streaming (Eq. streaming-general-d) and the cut-link
// reconstruction (Eqs. bfl-eta-ge-half, bfl-eta-lt-half) before recovering U^num.
#pragma once

#include <cuda_bf16.h>

#include "lbm_device.cuh"

namespace tlv {

// FP32 populations are stored shifted by f^eq(0, I); FP64 populations are stored raw and their
// arithmetic follows the FP64 oracle operation for operation (its translation unit is built
// without FMA contraction), so the FP64 form reproduces the oracle to rounding.
template <typename real> constexpr bool kShifted = sizeof(real) == 4;

// Population storage.  The planes hold the arithmetic type itself, or BF16 with FP32 arithmetic
// (rounded to nearest even on store, widened exactly on load).  StepArgs carries the population
// pointers typed by the arithmetic type; kernels instantiated for BF16 storage reinterpret them.
// pop_ld reads through the read-only path (arrays the kernel does not write); pop_ld_rw reads an
// array the kernel updates in place.
template <typename pop> struct PopIO {
    static __device__ __forceinline__ pop ld(const pop *p) { return __ldg(p); }
    static __device__ __forceinline__ pop ld_rw(const pop *p) { return *p; }
    static __device__ __forceinline__ void st(pop *p, pop v) { *p = v; }
};
template <> struct PopIO<__nv_bfloat16> {
    static __device__ __forceinline__ float ld(const __nv_bfloat16 *p) { return __bfloat162float(__ldg(p)); }
    static __device__ __forceinline__ float ld_rw(const __nv_bfloat16 *p) { return __bfloat162float(*p); }
    static __device__ __forceinline__ void st(__nv_bfloat16 *p, float v) { *p = __float2bfloat16_rn(v); }
};
template <typename real, typename pop>
__device__ __forceinline__ real pop_ld(const real *base, long long i) {
    return (real)PopIO<pop>::ld(reinterpret_cast<const pop *>(base) + i);
}
template <typename real, typename pop>
__device__ __forceinline__ real pop_ld_rw(const real *base, long long i) {
    return (real)PopIO<pop>::ld_rw(reinterpret_cast<const pop *>(base) + i);
}
template <typename real, typename pop>
__device__ __forceinline__ void pop_st(real *base, long long i, real v) {
    PopIO<pop>::st(reinterpret_cast<pop *>(base) + i, v);
}

template <typename real, int D> __device__ __forceinline__ real div2D(real x) {
    if constexpr (kShifted<real>) return x * (real(1) / real(2 * D));
    else return x / real(2 * D);
}

// Displacement accumulators u* and u^n.  The FP64 form keeps one FP64 plane per component.  The
// FP32 form keeps each component as an unevaluated pair of FP32 planes, hi (planes 0..D-1) and lo
// (planes D..2D-1) with |lo| <= ulp(hi)/2, so that u* = hi + lo carries about 48 significant bits:
// u* gains dt v every step, and the projection and the LSQ tangent images difference u across one
// lattice spacing, so one FP32 plane would drop the increments' low bits and, at fine spacings, most
// of those differences.  Both forms use D * npad * 8 bytes per accumulator.
template <typename real> constexpr bool kDispPair = sizeof(real) == 4;

// (hi, lo) + d, renormalised: Knuth's TwoSum of hi and d, then Dekker's Fast2Sum of that sum and
// the gathered low parts (the sum dominates).  Round-to-nearest intrinsics keep the compiler from
// contracting or reordering the error-free steps.
__device__ __forceinline__ void df_add(float &hi, float &lo, float d) {
    const float s = __fadd_rn(hi, d);
    const float bv = __fsub_rn(s, hi);
    const float e = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bv)), __fsub_rn(d, bv));
    const float t = __fadd_rn(e, lo);
    hi = __fadd_rn(s, t);
    lo = __fsub_rn(t, __fsub_rn(hi, s));
}

template <typename real>
__device__ __forceinline__ double disp_get(const real *p, long long P, int D, int i, long long node) {
    if constexpr (kDispPair<real>) return (double)p[i * P + node] + (double)p[(D + i) * P + node];
    else return p[i * P + node];
}

template <typename real>
__device__ __forceinline__ void disp_set(real *p, long long P, int D, int i, long long node, double u) {
    if constexpr (kDispPair<real>) {
        const float hi = (float)u;
        p[i * P + node] = hi;
        p[(D + i) * P + node] = (float)(u - (double)hi);
    } else {
        p[i * P + node] = u;
    }
}

// u^n of the nodes that Neumann LSQ stencils read, node-major so that one node is one or two
// vector accesses: FP32 form [hi_1..hi_D, (pad), lo_1..lo_D, (pad)], FP64 form [u_1..u_D, (pad)];
// 32 bytes per node in 3D, 16 in 2D.
template <typename real, int D> constexpr int kUnStride = (D == 3 ? 32 : 16) / (int)sizeof(real);

template <typename real, int D>
__device__ __forceinline__ void un_store(real *un, long long node, const real *hi, const real *lo) {
    real *p = un + (long long)kUnStride<real, D> * node;
    if constexpr (kDispPair<real>) {
        if constexpr (D == 3) {
            reinterpret_cast<float4 *>(p)[0] = make_float4(hi[0], hi[1], hi[2], 0.0f);
            reinterpret_cast<float4 *>(p)[1] = make_float4(lo[0], lo[1], lo[2], 0.0f);
        } else {
            reinterpret_cast<float4 *>(p)[0] = make_float4(hi[0], hi[1], lo[0], lo[1]);
        }
    } else {
        reinterpret_cast<double2 *>(p)[0] = make_double2(hi[0], hi[1]);
        if constexpr (D == 3) reinterpret_cast<double2 *>(p)[1] = make_double2(hi[2], 0.0);
    }
}

template <typename real, int D>
__device__ __forceinline__ void un_load(const real *un, long long node, real *hi, real *lo) {
    const real *p = un + (long long)kUnStride<real, D> * node;
    if constexpr (kDispPair<real>) {
        if constexpr (D == 3) {
            // the whole 32-byte record in one 256-bit load (records are 32-byte aligned; read-only here)
            float w[8];
            asm("ld.global.nc.v8.f32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                : "=f"(w[0]), "=f"(w[1]), "=f"(w[2]), "=f"(w[3]), "=f"(w[4]), "=f"(w[5]), "=f"(w[6]), "=f"(w[7])
                : "l"(p));
            hi[0] = w[0]; hi[1] = w[1]; hi[2] = w[2];
            lo[0] = w[4]; lo[1] = w[5]; lo[2] = w[6];
            return;
        }
        const float4 a = __ldg(reinterpret_cast<const float4 *>(p));
        hi[0] = a.x; hi[1] = a.y; lo[0] = a.z; lo[1] = a.w;
    } else {
        const double2 a = __ldg(reinterpret_cast<const double2 *>(p));
        hi[0] = a.x; hi[1] = a.y;
        if constexpr (D == 3) hi[2] = __ldg(reinterpret_cast<const double2 *>(p) + 1).x;
        #pragma unroll
        for (int i = 0; i < D; ++i) lo[i] = 0.0;
    }
}

struct Box {
    int D, nx, ny, nz;
    int per[3];
    int pad;
    long long nbox, npad;
    double dx, origin[3];
};

__device__ __forceinline__ void node_xyz(const Box &b, int node, int &x, int &y, int &z) {
    x = node % b.nx;
    int r = node / b.nx;
    y = r % b.ny;
    z = r / b.ny;
}

// neighbour m + e_q with periodic wrap (callers only use it for in-box or periodic neighbours);
// without periodic axes it is a plain offset and the coordinates are not needed
__device__ __forceinline__ int nbr(const Box &b, int node, int x, int y, int z, int q) {
    const int A = q >> 1, s = (q & 1) ? -1 : 1;
    if (!(b.per[0] | b.per[1] | b.per[2])) return node + s * (A == 0 ? 1 : (A == 1 ? b.nx : b.nx * b.ny));
    if (A == 0) {
        int xn = x + s;
        xn = xn < 0 ? xn + b.nx : (xn >= b.nx ? xn - b.nx : xn);
        return node + (xn - x);
    } else if (A == 1) {
        int yn = y + s;
        yn = yn < 0 ? yn + b.ny : (yn >= b.ny ? yn - b.ny : yn);
        return node + (yn - y) * b.nx;
    } else {
        int zn = z + s;
        zn = zn < 0 ? zn + b.nz : (zn >= b.nz ? zn - b.nz : zn);
        return node + (zn - z) * b.nx * b.ny;
    }
}

__device__ __forceinline__ void node_X(const Box &b, int x, int y, int z, double X[3]) {
    X[0] = b.origin[0] + (x + 0.5) * b.dx;
    X[1] = b.origin[1] + (y + 0.5) * b.dx;
    X[2] = (b.D == 3) ? b.origin[2] + (z + 0.5) * b.dx : 0.0;
}

__device__ __forceinline__ void set_status(int *st, int bits) {
    if (bits) atomicOr(st, bits);
}

// Bounds-checked build (-DLBM_CHECK, liblbm_b300_check.so): a data-dependent index outside its array
// latches kStBounds in the status word and is replaced by 0, so the access stays inside the array.
// Compiled out of the normal build.
#ifdef LBM_CHECK
#define TLV_BOUND(idx, n, st)                                                        \
    do {                                                                             \
        if ((unsigned long long)(long long)(idx) >= (unsigned long long)(n)) {       \
            set_status((st), kStBounds);                                             \
            (idx) = 0;                                                               \
        }                                                                            \
    } while (0)
#else
#define TLV_BOUND(idx, n, st) \
    do {                      \
    } while (0)
#endif

// =============================================================================================
// geometry pass (FP64)
// =============================================================================================

// active mask, and the group (specimen) of each active node: its material index
static __global__ void k_mask(Box b, const LevelSetD ls, uint8_t *flags, uint8_t *mat) {
    long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= b.nbox) return;
    int x, y, z;
    node_xyz(b, (int)i, x, y, z);
    double X[3];
    node_X(b, x, y, z, X);
    int g;
    const bool act = levelset(ls, b.D, X, nullptr, &g) <= 0.0;
    flags[i] = act ? kActive : 0;
    mat[i] = act ? (uint8_t)g : 0;
}

// cut bits (link (m,q) cut iff m + e_q is outside the body or outside a non-periodic box)
static __global__ void k_cutbits(Box b, const LevelSetD ls, uint8_t *flags, int *cnt,
                          unsigned long long *n_active, int *status) {
    long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    bool act = false;
    if (i < b.nbox) {
        int node = (int)i;
        uint8_t fl = flags[node];
        act = fl & kActive;
        int c = 0;
        if (act) {
            int x, y, z;
            node_xyz(b, node, x, y, z);
            uint8_t bits = 0;
            for (int q = 0; q < 2 * b.D; ++q) {
                const int A = q >> 1, s = (q & 1) ? -1 : 1;
                const int co = (A == 0 ? x : (A == 1 ? y : z)) + s;
                const int n = (A == 0 ? b.nx : (A == 1 ? b.ny : b.nz));
                if ((co < 0 || co >= n) && !b.per[A]) {
                    double X[3];
                    node_X(b, x, y, z, X);
                    X[A] += s * b.dx;
                    if (!(levelset(ls, b.D, X, nullptr) > 0.0)) set_status(status, kStDomain);
                    bits |= (1u << q);
                } else if (!(flags[nbr(b, node, x, y, z, q)] & kActive)) {
                    bits |= (1u << q);
                }
            }
            // only this thread writes this byte; neighbours read bit 6, which is unchanged
            flags[node] = fl | bits;
            c = __popc(bits);
        }
        cnt[node] = c;
    }
    unsigned mask = __ballot_sync(0xffffffffu, act);
    if ((threadIdx.x & 31) == 0 && mask) atomicAdd(n_active, (unsigned long long)__popc(mask));
}

// exclusive scan, 1024 elements per block; block totals to bsum
static __global__ void k_scan_block(const int *__restrict__ in, int *out, int *bsum, long long n) {
    __shared__ int wsum[32];
    long long i = blockIdx.x * 1024LL + threadIdx.x;
    int v = (i < n) ? in[i] : 0;
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int incl = v;
    #pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int t = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += t;
    }
    if (lane == 31) wsum[w] = incl;
    __syncthreads();
    if (w == 0) {
        int s = wsum[lane];
        int si = s;
        #pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int t = __shfl_up_sync(0xffffffffu, si, o);
            if (lane >= o) si += t;
        }
        wsum[lane] = si - s;
        if (lane == 31) bsum[blockIdx.x] = si;
    }
    __syncthreads();
    if (i < n) out[i] = incl - v + wsum[w];
}

static __global__ void k_scan_add(int *out, const int *__restrict__ boff, long long n) {
    long long i = blockIdx.x * 1024LL + threadIdx.x;
    if (i < n) out[i] += boff[blockIdx.x];
}

// one flag per 32-node x-segment of a row: does it hold an active node?
// Segments: 32-node x-windows starting at multiples of kSegAlign that cover every node of a row
// carrying `bit`, chosen left to right: a window starts at the first kSegAlign-node block holding
// such a node that the previous window does not cover, and spans that block and the next one.
// Starting windows at the runs rather than at multiples of 32 raises the share of active slots
// (the 256^3 shell: 86.9 % instead of 78.7 %); kSegAlign = 16 keeps every window start 16-byte
// aligned for bulk tensor copies of byte and float planes.  f(j) is called with the block index
// of each window start.
constexpr int kSegAlign = 16;

template <typename Fn>
__device__ __forceinline__ void for_each_window(const uint8_t *r, int nx, uint8_t bit, Fn &&f) {
    int covered = 0;  // first x not covered by the previous window
    for (int j = 0; j * kSegAlign < nx; ++j) {
        const int x0 = kSegAlign * j;
        if (x0 < covered) continue;
        bool any = false;
        for (int x = x0; x < min(x0 + kSegAlign, nx); ++x) any |= (r[x] & bit) != 0;
        if (any) {
            f(j);
            covered = x0 + 32;
        }
    }
}

// one thread per row: segflag[row * slots + j] = 1 where a window starts at block j (0 elsewhere,
// from the zeroed geometry storage)
static __global__ void k_seg_flags(Box b, const uint8_t *__restrict__ flags, int slots, long long rows, int *segflag) {
    const long long row = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (row >= rows) return;
    int *sf = segflag + row * slots;
    for_each_window(flags + row * b.nx, b.nx, kActive, [&](int j) { sf[j] = 1; });
}

static __global__ void k_seg_write(Box b, const int *__restrict__ segflag, const int *__restrict__ segidx, int slots,
                                   long long nsegmax, int2 *seg) {
    long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (s >= nsegmax || !segflag[s]) return;
    int row = (int)(s / slots), j = (int)(s % slots);
    seg[segidx[s]] = make_int2(row * b.nx + kSegAlign * j, row);
}

// ---------------------------------------------------------------------------------------------
// per-link geometry (bind): eta, X_b, N_b, boundary id / BC, tangents, LSQ weights
// ---------------------------------------------------------------------------------------------

template <typename real> struct LinkGeom {
    int *node;          // [ncut]
    int *q;             // [ncut] outgoing direction
    int *bc;            // [ncut]
    double *eta;        // [ncut]
    double *Xb;         // [3*ncut]
    double *Nb;         // [3*ncut]
    double *tan;        // [6*ncut] t_1, t_2
    real *h;            // [3*ncut] Newton state (normal image)
    int *ns;            // [ncut]
    int *sidx;          // [kLsqCap*ncut], entry j of link l at j*ncut + l
    real *w;            // [2*kLsqCap*ncut]; FP64: tangent a, entry j at (a*kLsqCap + j)*ncut + l;
                        // FP32: at (l*kLsqCap + j)*(D-1) + a, and sidx at l*kLsqCap + j
    real *rec;          // [ncut*K] reconstructed incoming populations for the next gather (link-major)
    real *fo;           // [ncut*2K] f*_c(m) then f*_{c^1}(m) of the link's node after the last collision
    float4 *bvec;       // [ncut] FP32 forms: the link's geometric vector for its boundary profile
    float *cu;          // [ncut] FP32 forms: D_b,v (1 - 2 eta) of an eta < 1/2 link with an active upstream
                        // node, else 0; the next gather adds its term D_b (1 - 2 eta) f*_c(m - e_c)
    long long ncut;
};

__device__ inline int lsq_basis(int D, bool linear, const double *xi, double *ph) {
    int nb = 0;
    ph[nb++] = 1.0;
    for (int a = 0; a < D; ++a) ph[nb++] = xi[a];
    if (linear) return nb;
    if (D == 2) {
        ph[nb++] = 0.5 * xi[0] * xi[0];
        ph[nb++] = xi[0] * xi[1];
        ph[nb++] = 0.5 * xi[1] * xi[1];
    } else {
        ph[nb++] = 0.5 * xi[0] * xi[0];
        ph[nb++] = 0.5 * xi[1] * xi[1];
        ph[nb++] = 0.5 * xi[2] * xi[2];
        ph[nb++] = xi[0] * xi[1];
        ph[nb++] = xi[0] * xi[2];
        ph[nb++] = xi[1] * xi[2];
    }
    return nb;
}

// visit the active nodes within 3 dx of X_b in (z, y, x) offset order; fn(k, xi)
template <typename Fn>
__device__ inline void for_stencil(const Box &b, const uint8_t *__restrict__ flags, int x, int y, int z,
                                   const double Xb[3], Fn fn) {
    const int R = 4;
    const int zlo = (b.D == 3) ? -R : 0, zhi = (b.D == 3) ? R : 0;
    for (int dz = zlo; dz <= zhi; ++dz)
        for (int dy = -R; dy <= R; ++dy)
            for (int dxo = -R; dxo <= R; ++dxo) {
                int cx = x + dxo, cy = y + dy, cz = z + dz;
                if (cx < 0 || cx >= b.nx || cy < 0 || cy >= b.ny) continue;
                if (b.D == 3 && (cz < 0 || cz >= b.nz)) continue;
                int k = cx + b.nx * (cy + b.ny * cz);
                if (!(flags[k] & kActive)) continue;
                double Xk[3], xi[3], r2 = 0.0;
                node_X(b, cx, cy, cz, Xk);
                for (int a = 0; a < b.D; ++a) {
                    xi[a] = (Xk[a] - Xb[a]) / b.dx;
                    r2 += xi[a] * xi[a];
                }
                if (r2 > kLsqRho2 + 1e-9) continue;
                fn(k, xi, r2);
            }
}

template <typename real, int D>
__global__ void k_link_build(Box b, const int2 *__restrict__ seg, int nseg, uint8_t *flags, uint8_t *dmask,
                             const int *__restrict__ lstart, const LevelSetD ls,
                             const BCD *__restrict__ bcs, int nbc, LinkGeom<real> L, int *status) {
    int sgi = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (sgi >= nseg) return;
    int2 sg = seg[sgi];
    int x0 = sg.x - sg.y * b.nx, x = x0 + (threadIdx.x & 31);
    if (x >= b.nx) return;
    int node = sg.x + (threadIdx.x & 31);
    uint8_t fl = flags[node];
    if (!(fl & kActive)) return;
    unsigned cut = fl & kCutMask;
    if (!cut) return;
    int y = sg.y % b.ny, z = sg.y / b.ny;
    double Xm[3];
    node_X(b, x, y, z, Xm);
    int l = lstart[node];
    uint8_t dm = 0;
    for (int q = 0; q < 2 * D; ++q) {
        if (!((cut >> q) & 1)) continue;
        const int A = q >> 1;
        const double s = (q & 1) ? -1.0 : 1.0;
        // eta by bisection of phi on the link (Eq. cut-link-point)
        double lo = 0.0, hi = 1.0;
        for (int it = 0; it < 60; ++it) {
            double mid = 0.5 * (lo + hi), Xt[3] = {Xm[0], Xm[1], Xm[2]};
            Xt[A] = Xm[A] + mid * b.dx * s;
            if (levelset(ls, D, Xt, nullptr) <= 0.0) lo = mid; else hi = mid;
        }
        const double eta = 0.5 * (lo + hi);
        double Xb[3] = {Xm[0], Xm[1], Xm[2]};
        Xb[A] = Xm[A] + eta * b.dx * s;
        int which;
        levelset(ls, D, Xb, &which);
        double g[3];
        shape_phi(ls.shapes[which], D, Xb, g);
        double gn = sqrt(g[0] * g[0] + g[1] * g[1] + g[2] * g[2]);
        double N[3] = {g[0] / gn, g[1] / gn, g[2] / gn};  // Eq. (level-set-normal)
        int bid = ls.shapes[which].bid, bci = -1;
        for (int j = 0; j < nbc; ++j)
            if (bcs[j].bid == bid) { bci = j; break; }
        int kind = 0;
        if (bci < 0) {
            set_status(status, kStNoBC);  // reported by lbm_bind_storage; treated as Dirichlet here
            bci = 0;
        } else {
            kind = bcs[bci].kind;
        }
        if (kind == 1 && L.sidx == nullptr) {  // Neumann link but no LSQ tables (cannot happen by construction)
            set_status(status, kStNoBC);
            kind = 0;
        }
        // tangent frame
        double t[2][3] = {{0, 0, 0}, {0, 0, 0}};
        if (D == 2) {
            t[0][0] = -N[1]; t[0][1] = N[0];
        } else {
            int a = 0;
            for (int k = 1; k < 3; ++k)
                if (fabs(N[k]) < fabs(N[a])) a = k;
            double e[3] = {0, 0, 0};
            e[a] = 1.0;
            double c[3] = {e[1] * N[2] - e[2] * N[1], e[2] * N[0] - e[0] * N[2], e[0] * N[1] - e[1] * N[0]};
            double nc = sqrt(c[0] * c[0] + c[1] * c[1] + c[2] * c[2]);
            for (int k = 0; k < 3; ++k) t[0][k] = c[k] / nc;
            t[1][0] = N[1] * t[0][2] - N[2] * t[0][1];
            t[1][1] = N[2] * t[0][0] - N[0] * t[0][2];
            t[1][2] = N[0] * t[0][1] - N[1] * t[0][0];
        }
        L.node[l] = node;
        L.q[l] = q;
        L.bc[l] = bci;
        L.eta[l] = eta;
        for (int a = 0; a < 3; ++a) {
            L.Xb[3 * l + a] = Xb[a];
            L.Nb[3 * l + a] = N[a];
            L.tan[6 * l + a] = t[0][a];
            L.tan[6 * l + 3 + a] = t[1][a];
            L.h[3 * l + a] = sizeof(real) == 4 ? real(0) : (real)N[a];  // FP32 forms keep h - N
        }
        if constexpr (sizeof(real) == 4) {
            double gv[3];
            link_gvec(bcs[bci], D, Xb, gv);
            L.bvec[l] = make_float4((float)gv[0], (float)gv[1], (float)gv[2], 0.0f);
        }
        int ns = 0;
        if (kind == 0) {
            dm |= (uint8_t)(1u << q);
        } else {
            // weighted quadratic LSQ (Eqs. quadratic-lsq-2d, tangent-derivative-2d); linear fallback
            int mode = -1;
            double zs[2][10];
            for (int linear = 0; linear <= 1 && mode < 0; ++linear) {
                double M[55];  // packed lower triangle
                for (int r = 0; r < 55; ++r) M[r] = 0.0;
                int nb = 0, cntn = 0;
                for_stencil(b, flags, x, y, z, Xb, [&](int k, const double *xi, double r2) {
                    double ph[10];
                    nb = lsq_basis(D, linear, xi, ph);
                    double wt = exp(-r2);
                    for (int r = 0; r < nb; ++r)
                        for (int c = 0; c <= r; ++c) M[r * (r + 1) / 2 + c] += wt * ph[r] * ph[c];
                    ++cntn;
                });
                double ph0[10], xi0[3] = {0, 0, 0};
                nb = lsq_basis(D, linear, xi0, ph0);
                if (cntn < nb) continue;
                double maxd = 0.0;
                for (int r = 0; r < nb; ++r) maxd = fmax(maxd, M[r * (r + 1) / 2 + r]);
                double Lc[55];
                bool ok = true;
                for (int c = 0; c < nb && ok; ++c) {
                    double d = M[c * (c + 1) / 2 + c];
                    for (int k = 0; k < c; ++k) d -= Lc[c * (c + 1) / 2 + k] * Lc[c * (c + 1) / 2 + k];
                    if (!(d > 1e-10 * maxd)) { ok = false; break; }
                    Lc[c * (c + 1) / 2 + c] = sqrt(d);
                    for (int r = c + 1; r < nb; ++r) {
                        double v = M[r * (r + 1) / 2 + c];
                        for (int k = 0; k < c; ++k) v -= Lc[r * (r + 1) / 2 + k] * Lc[c * (c + 1) / 2 + k];
                        Lc[r * (r + 1) / 2 + c] = v / Lc[c * (c + 1) / 2 + c];
                    }
                }
                if (!ok) continue;
                for (int al = 0; al < D - 1; ++al) {
                    double yv[10];
                    double *zz = zs[al];
                    for (int r = 0; r < nb; ++r) zz[r] = 0.0;
                    for (int a = 0; a < D; ++a) zz[1 + a] = t[al][a];
                    for (int r = 0; r < nb; ++r) {
                        double v = zz[r];
                        for (int k = 0; k < r; ++k) v -= Lc[r * (r + 1) / 2 + k] * yv[k];
                        yv[r] = v / Lc[r * (r + 1) / 2 + r];
                    }
                    for (int r = nb - 1; r >= 0; --r) {
                        double v = yv[r];
                        for (int k = r + 1; k < nb; ++k) v -= Lc[k * (k + 1) / 2 + r] * zz[k];
                        zz[r] = v / Lc[r * (r + 1) / 2 + r];
                    }
                }
                mode = linear;
            }
            if (mode < 0) {
                set_status(status, kStLsq);
            } else {
                const bool linear = mode == 1;
                for_stencil(b, flags, x, y, z, Xb, [&](int k, const double *xi, double r2) {
                    if (ns < kLsqCap) {
                        double ph[10];
                        int nb = lsq_basis(D, linear, xi, ph);
                        // FP64 tables entry-major (entry j of all links contiguous: one thread per link);
                        // FP32 tables link-major (a link's entries contiguous: one lane group per link)
                        if constexpr (sizeof(real) == 4) L.sidx[(long long)l * kLsqCap + ns] = k;
                        else L.sidx[(long long)ns * L.ncut + l] = k;
                        for (int al = 0; al < D - 1; ++al) {
                            double sacc = 0.0;
                            for (int r = 0; r < nb; ++r) sacc += ph[r] * zs[al][r];
                            const real wv = (real)(exp(-r2) * sacc / b.dx);
                            if constexpr (sizeof(real) == 4) L.w[((long long)l * kLsqCap + ns) * (D - 1) + al] = wv;
                            else L.w[((long long)al * kLsqCap + ns) * L.ncut + l] = wv;
                        }
                        unsigned *word = reinterpret_cast<unsigned *>(flags + (k & ~3));
                        atomicOr(word, (unsigned)kNeedU << (8 * (k & 3)));
                    }
                    ++ns;
                });
                if (ns > kLsqCap) { set_status(status, kStCapacity); ns = kLsqCap; }
            }
        }
        L.ns[l] = ns;
        ++l;
    }
    dmask[node] = dm;
}

// =============================================================================================
// initial state (Eqs. init-general-d, Ut-general-init; u* from Eq. u-recovery-general)
// =============================================================================================

// C_{iAkB} Z_{kB} for the neo-Hookean law, FP64
template <int D> __device__ inline void dpiola64(const double *F, const double *Z, double mu, double lam, double *dP) {
    double C[D * D];
    cofactor<double, D>(F, C);
    const double J = det<double, D>(F);
    double Fit[D * D];
    for (int k = 0; k < D * D; ++k) Fit[k] = C[k] / J;
    double tr = 0.0;
    for (int k = 0; k < D * D; ++k) tr += Fit[k] * Z[k];
    const double s = 0.5 * lam * (J * J - 1.0) - mu;
    for (int i = 0; i < D; ++i)
        for (int A = 0; A < D; ++A) {
            double m = 0.0;
            for (int B = 0; B < D; ++B)
                for (int j = 0; j < D; ++j) m += Fit[i * D + B] * Z[j * D + B] * Fit[j * D + A];
            dP[i * D + A] = mu * Z[i * D + A] + lam * J * J * tr * Fit[i * D + A] - s * m;
        }
}

template <typename real, int D, typename pop = real>
__global__ void k_init(Box b, const int2 *__restrict__ seg, int nseg, const uint8_t *__restrict__ flags,
                       const double *__restrict__ v0, const double *__restrict__ F0, const double *__restrict__ u0,
                       const double *__restrict__ dU0, int characteristic, double c, double dt, double mu_, double lam_,
                       const uint8_t *__restrict__ mat, const double *__restrict__ mtab,
                       const real *__restrict__ mu_field, double gamma, double b0, double b1, double b2, real *f,
                       real *ustar) {
    constexpr int K = D + D * D, Q = 2 * D;
    int sgi = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (sgi >= nseg) return;
    int2 sg = seg[sgi];
    int x = sg.x - sg.y * b.nx + (threadIdx.x & 31);
    if (x >= b.nx) return;
    int node = sg.x + (threadIdx.x & 31);
    uint8_t fl = flags[node];
    if (!(fl & kActive)) return;
    const long long N = b.nbox, P = b.npad;
    int y = sg.y % b.ny, z = sg.y / b.ny;
    double U0[K];
    for (int i = 0; i < D; ++i) U0[i] = v0[i * N + node];
    for (int k = 0; k < D * D; ++k) U0[D + k] = F0[k * N + node];
    const double mu = mu_field ? (double)mu_field[node] : (mtab ? mtab[2 * mat[node]] : mu_);
    const double lam = mtab ? mtab[2 * mat[node] + 1] : lam_;
    double Pm[D * D];
    piola<double, D>(U0 + D, mu, lam, Pm);
    const double shift = (sizeof(real) == 4) ? 1.0 : 0.0;  // FP32 stores f - f^eq(0, I)
    const double bf[3] = {b0, b1, b2};
    double dU[D * K], Ut[K];
    if (characteristic) {
        const unsigned cut = fl & kCutMask;
        for (int A = 0; A < D; ++A) {
            const bool ap = !((cut >> (2 * A)) & 1), am = !((cut >> (2 * A + 1)) & 1);
            const int lp = ap ? nbr(b, node, x, y, z, 2 * A) : node, lm = am ? nbr(b, node, x, y, z, 2 * A + 1) : node;
            for (int k = 0; k < K; ++k) {
                if (dU0) { dU[A * K + k] = dU0[(A * K + k) * N + node]; continue; }
                const double *src = (k < D) ? v0 + k * N : F0 + (k - D) * N;
                double vm = src[node], vp = src[lp], vn = src[lm];
                if (ap && am) dU[A * K + k] = (vp - vn) / (2.0 * b.dx);
                else if (ap) dU[A * K + k] = (vp - vm) / b.dx;
                else if (am) dU[A * K + k] = (vm - vn) / b.dx;
                else dU[A * K + k] = 0.0;
            }
        }
        // d_t U0 = B0 - Phi_A'(U0) d_A U0, with (Phi_A' Z)^{v_i} = -C_iAkB Z_F,kB, (Phi_A' Z)^{F_iB} = -d_AB Z_v_i
        for (int k = 0; k < K; ++k) Ut[k] = 0.0;
        for (int i = 0; i < D; ++i) Ut[i] = bf[i] - gamma * U0[i];
        for (int A = 0; A < D; ++A) {
            double dP[D * D];
            dpiola64<D>(U0 + D, dU + A * K + D, mu, lam, dP);
            for (int i = 0; i < D; ++i) Ut[i] += dP[i * D + A];
            for (int i = 0; i < D; ++i) Ut[D + i * D + A] += dU[A * K + i];
        }
    }
    for (int q = 0; q < Q; ++q) {
        const int A = q >> 1;
        const double s = (q & 1) ? -1.0 : 1.0;
        double fq[K];
        for (int i = 0; i < D; ++i) fq[i] = (U0[i] - s * (D / c) * Pm[i * D + A]) / (2.0 * D);
        for (int i = 0; i < D; ++i)
            for (int B = 0; B < D; ++B)
                fq[D + i * D + B] = (A == B) ? ((U0[D + i * D + B] - (i == B ? shift : 0.0)) - s * (D / c) * U0[i]) / (2.0 * D)
                                             : (U0[D + i * D + B] - (i == B ? shift : 0.0)) / (2.0 * D);
        if (characteristic) {
            double Zq[K];
            for (int k = 0; k < K; ++k) Zq[k] = Ut[k] + c * s * dU[A * K + k];
            double dP[D * D];
            dpiola64<D>(U0 + D, Zq + D, mu, lam, dP);
            for (int i = 0; i < D; ++i) fq[i] -= 0.5 * dt * (Zq[i] - s * (D / c) * dP[i * D + A]) / (2.0 * D);
            for (int i = 0; i < D; ++i)
                for (int B = 0; B < D; ++B)
                    fq[D + i * D + B] -= 0.5 * dt * (Zq[D + i * D + B] - s * (D / c) * (A == B ? Zq[i] : 0.0)) / (2.0 * D);
        }
        for (int k = 0; k < K; ++k) pop_st<real, pop>(f, (long long)(q * K + k) * P + node, (real)fq[k]);
    }
    for (int i = 0; i < D; ++i) disp_set<real>(ustar, P, D, i, node, u0[i * N + node] - 0.5 * dt * v0[i * N + node]);
}

// =============================================================================================
// gather: pull streaming + cut-link reconstruction
// =============================================================================================

template <typename real> struct StepArgs {
    Box b;
    const int2 *seg;
    int nseg;
    const uint8_t *flags;
    const int *lstart;
    const real *fsrc;
    real *fdst;
    real *ustar;
    real *un;
    const real *lrec;  // per cut link: reconstructed incoming populations (K), read by the gather
    const float *lcu;  // per cut link, FP32 forms: coefficient of the upstream term the gather adds
                       // (LinkGeom::cu), null in the FP64 form
    real *lfo;         // per cut link: f*_c(m), f*_{c^1}(m) (2K), written by the collision kernels
    real *vst, *Gst;   // projection steps: v^n and G^n = F^n - I (D and D*D planes)
    real *u0;          // projection steps: u^n (displacement-accumulator layout)
    real dt, c, omega, gamma, mu, lam, bf[3];
    const uint8_t *mat;  // per-node group of a multi-specimen body (with mtab), else null
    const real *mtab;    // (mu, lambda) per group, or null: mu and lam above for every node
    const real *mu_field;  // per-node shear modulus replacing mu, or null
    real *mom_out;         // the step's recovered F (or F - I when shifted): D*D planes, or null
    int *status;
    int spin;              // polls of a bulk-copy kernel's first wait for its copies
    long long ncut;        // cut links (bounds of the per-link arrays)
};

// material of a node: its group's (mu, lambda) for multi-specimen bodies, else the global one;
// a per-node shear-modulus field replaces mu
template <typename real>
__device__ __forceinline__ void node_material(const StepArgs<real> &a, long long node, real &mu, real &lam) {
    if (a.mtab) {
        const int g = a.mat[node];
        mu = a.mtab[2 * g];
        lam = a.mtab[2 * g + 1];
    } else {
        mu = a.mu;
        lam = a.lam;
    }
    if (a.mu_field) mu = a.mu_field[node];
}

// N consecutive values at p (aligned to 16 bytes when N*sizeof(real) is a multiple of 16, else to
// 8 bytes) as 16- or 8-byte vector loads and stores
template <int N> __device__ __forceinline__ void vload(const float *p, float *d) {
    if constexpr (N % 4 == 0) {
        #pragma unroll
        for (int i = 0; i < N / 4; ++i) {
            const float4 t = __ldg(reinterpret_cast<const float4 *>(p) + i);
            d[4 * i] = t.x; d[4 * i + 1] = t.y; d[4 * i + 2] = t.z; d[4 * i + 3] = t.w;
        }
    } else {
        static_assert(N % 2 == 0, "even count");
        #pragma unroll
        for (int i = 0; i < N / 2; ++i) {
            const float2 t = __ldg(reinterpret_cast<const float2 *>(p) + i);
            d[2 * i] = t.x; d[2 * i + 1] = t.y;
        }
    }
}
template <int N> __device__ __forceinline__ void vload(const double *p, double *d) {
    static_assert(N % 2 == 0, "even count");
    #pragma unroll
    for (int i = 0; i < N / 2; ++i) {
        const double2 t = __ldg(reinterpret_cast<const double2 *>(p) + i);
        d[2 * i] = t.x; d[2 * i + 1] = t.y;
    }
}
template <int N> __device__ __forceinline__ void vstore(float *p, const float *d) {
    if constexpr (N % 4 == 0) {
        #pragma unroll
        for (int i = 0; i < N / 4; ++i)
            reinterpret_cast<float4 *>(p)[i] = make_float4(d[4 * i], d[4 * i + 1], d[4 * i + 2], d[4 * i + 3]);
    } else {
        static_assert(N % 2 == 0, "even count");
        #pragma unroll
        for (int i = 0; i < N / 2; ++i) reinterpret_cast<float2 *>(p)[i] = make_float2(d[2 * i], d[2 * i + 1]);
    }
}
template <int N> __device__ __forceinline__ void vstore(double *p, const double *d) {
    static_assert(N % 2 == 0, "even count");
    #pragma unroll
    for (int i = 0; i < N / 2; ++i) reinterpret_cast<double2 *>(p)[i] = make_double2(d[2 * i], d[2 * i + 1]);
}

// link of node m (first link l0 = lstart[m]) whose cut bit is c: links are sorted by node, then bit
__device__ __forceinline__ long long link_of(long long l0, unsigned cut, int c) {
    return l0 + __popc(cut & ((1u << c) - 1u));
}

// After computing the post-collision values out[0..K) of direction q at a node with cut bits `cut`,
// keep the ones its cut links need: f*_c(m) for a cut direction c = q, f*_{c^1}(m) for c = q^1.
template <typename real, int K>
__device__ __forceinline__ void keep_link_values(real *lfo, long long l0, unsigned cut, int q, const real *out,
                                                 long long ncut, int *status) {
    if ((cut >> q) & 1) {
        long long l = link_of(l0, cut, q);
        TLV_BOUND(l, ncut, status);
        vstore<K>(lfo + l * (2 * K), out);
    }
    if ((cut >> (q ^ 1)) & 1) {
        long long l = link_of(l0, cut, q ^ 1);
        TLV_BOUND(l, ncut, status);
        vstore<K>(lfo + l * (2 * K) + K, out);
    }
    (void)ncut;
    (void)status;
}

// MODE 0: state is pre-collision f^0 (first step, no streaming); MODE 1: state is f*^{n-1}
template <typename real, int D, int MODE, typename pop = real>
__device__ __forceinline__ void gather(const StepArgs<real> &a, int node, int x, int y, int z, unsigned cut,
                                       real (&f)[2 * D * (D + D * D)]) {
    constexpr int K = D + D * D, Q = 2 * D;
    const long long P = a.b.npad;
    const real *__restrict__ fs = a.fsrc;
    if constexpr (MODE == 0) {
        #pragma unroll
        for (int q = 0; q < Q; ++q)
            #pragma unroll
            for (int k = 0; k < K; ++k) f[q * K + k] = pop_ld<real, pop>(fs, (long long)(q * K + k) * P + node);
        return;
    } else {
    #pragma unroll
    for (int q = 0; q < Q; ++q) {
        if (!((cut >> (q ^ 1)) & 1)) {  // source m - e_q = m + e_{q^1} is active
            int src = nbr(a.b, node, x, y, z, q ^ 1);
            TLV_BOUND(src, a.b.npad, a.status);
            #pragma unroll
            for (int k = 0; k < K; ++k) f[q * K + k] = pop_ld<real, pop>(fs, (long long)(q * K + k) * P + src);
        }
    }
    if (cut) {
        // the populations a cut link leaves unknown arrive reconstructed by the link kernel; an eta < 1/2
        // link with an active upstream node m - e_c gets its upstream term here, from the value that
        // direction c pulls from that node (slot c = q^1, pulled: link (m, q) is not cut)
        const long long l0 = __ldg(a.lstart + node);
        #pragma unroll
        for (int q = 0; q < Q; ++q)
            if ((cut >> (q ^ 1)) & 1) {
                long long l = link_of(l0, cut, q ^ 1);
                TLV_BOUND(l, a.ncut, a.status);
                real r[K];
                vload<K>(a.lrec + l * K, r);
                if constexpr (sizeof(real) == 4) {
                    const float cv = a.lcu ? __ldg(a.lcu + l) : 0.0f;
                    if (cv != 0.0f)
                        #pragma unroll
                        for (int k = 0; k < K; ++k) r[k] += (k < D ? cv : -cv) * f[(q ^ 1) * K + k];
                }
                #pragma unroll
                for (int k = 0; k < K; ++k) f[q * K + k] = r[k];
            }
    }
    }
}

// moments with half-step source and implicit damping (Eq. state-recovery-general, B = (b - gamma v, 0))
template <typename real, int D>
__device__ __forceinline__ void recover(const StepArgs<real> &a, const real (&f)[2 * D * (D + D * D)], real v[D],
                                        real G[D * D], real F[D * D]) {
    constexpr int K = D + D * D, Q = 2 * D;
    #pragma unroll
    for (int k = 0; k < K; ++k) {
        real s = f[k];
        #pragma unroll
        for (int q = 1; q < Q; ++q) s += f[q * K + k];
        if (k < D) {
            v[k] = (s + real(0.5) * a.dt * a.bf[k]) / (real(1) + real(0.5) * a.dt * a.gamma);
        } else {
            const real one = (((k - D) / D) == ((k - D) % D)) ? real(1) : real(0);
            if constexpr (kShifted<real>) { G[k - D] = s; F[k - D] = s + one; }
            else { F[k - D] = s; G[k - D] = s - one; }
        }
    }
}

// BGK collision with source (Eq. collision-general-d) in shifted variables; writes f*
// equilibrium f^eq_q (Eq. feq-general-d) in the storage variables: v rows (v - s (D/c) P_iA)/(2D),
// F rows (X_iB - s (D/c) delta_AB v_i)/(2D), X = F - I (shifted storage) or F (raw storage)
template <typename real, int D>
__device__ __forceinline__ void equilibrium(const real v[D], const real X[D * D], const real Pk[D * D], real Dc,
                                            real (&feq)[2 * D * (D + D * D)]) {
    constexpr int K = D + D * D, Q = 2 * D;
    #pragma unroll
    for (int q = 0; q < Q; ++q) {
        const int A = q >> 1;
        const real s = (q & 1) ? real(-1) : real(1);
        #pragma unroll
        for (int i = 0; i < D; ++i) feq[q * K + i] = div2D<real, D>(v[i] - s * Dc * Pk[i * D + A]);
        #pragma unroll
        for (int i = 0; i < D; ++i)
            #pragma unroll
            for (int Bc = 0; Bc < D; ++Bc)
                feq[q * K + D + i * D + Bc] =
                    (A == Bc) ? div2D<real, D>(X[i * D + Bc] - s * Dc * v[i]) : div2D<real, D>(X[i * D + Bc]);
    }
}

template <typename real, int D, typename pop = real>
__device__ __forceinline__ void collide_store(const StepArgs<real> &a, int node, unsigned cut,
                                              real (&f)[2 * D * (D + D * D)], const real v[D], const real G[D * D],
                                              const real F[D * D], const real Pk[D * D]) {
    constexpr int K = D + D * D, Q = 2 * D;
    const long long P = a.b.npad;
    const real Dc = real(D) / a.c;
    const real wq = real(1) / real(4 * D);
    const real src = a.dt * (real(2) - a.omega) * wq;
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
        for (int i = 0; i < D; ++i) {
            const real feq = div2D<real, D>(v[i] - s * Dc * Pk[i * D + A]);
            const real fv = f[q * K + i];
            out[i] = fv + a.omega * (feq - fv) + src * B[i];
        }
        #pragma unroll
        for (int i = 0; i < D; ++i)
            #pragma unroll
            for (int Bc = 0; Bc < D; ++Bc) {
                const int k = D + i * D + Bc;
                const real X = kShifted<real> ? G[i * D + Bc] : F[i * D + Bc];
                const real feq = (A == Bc) ? div2D<real, D>(X - s * Dc * v[i]) : div2D<real, D>(X);
                const real fv = f[q * K + k];
                out[k] = fv + a.omega * (feq - fv);
            }
        #pragma unroll
        for (int k = 0; k < K; ++k) pop_st<real, pop>(a.fdst, (long long)(q * K + k) * P + node, out[k]);
        if (cut) keep_link_values<real, K>(a.lfo, l0, cut, q, out, a.ncut, a.status);
    }
}

template <typename real, int D>
__device__ __forceinline__ int check_state(const real v[D], const real F[D * D], real J) {
    int st = 0;
    if (!(J > real(0))) st |= kStJacobian;
    bool fin = isfinite(J);
    #pragma unroll
    for (int i = 0; i < D; ++i) fin = fin && isfinite(v[i]);
    #pragma unroll
    for (int k = 0; k < D * D; ++k) fin = fin && isfinite(F[k]);
    if (!fin) st |= kStNonfinite;
    return st;
}

// ---------------------------------------------------------------------------------------------
// K3: fused gather + closure + recovery + collision (+ u quadrature), one thread per node
// ---------------------------------------------------------------------------------------------
template <typename real, int D, int MODE, typename pop = real>
__global__ void __launch_bounds__(128) k_stream_collide(const StepArgs<real> a) {
    constexpr int K = D + D * D, Q = 2 * D;
    const int sgi = blockIdx.x * 4 + (threadIdx.x >> 5);
    if (sgi >= a.nseg) return;
    const int2 sg = __ldg(&a.seg[sgi]);
    const int lane = threadIdx.x & 31;
    const int x = sg.x - sg.y * a.b.nx + lane;
    if (x >= a.b.nx) return;
    const int node = sg.x + lane;
    const uint8_t fl = __ldg(a.flags + node);
    if (!(fl & kActive)) return;
    const int y = sg.y % a.b.ny, z = sg.y / a.b.ny;
    const unsigned cut = fl & kCutMask;
    real f[Q * K];
    gather<real, D, MODE, pop>(a, node, x, y, z, cut, f);
    real v[D], G[D * D], F[D * D], Pk[D * D];
    recover<real, D>(a, f, v, G, F);
    real mu, lam;
    node_material(a, node, mu, lam);
    if (a.mom_out)
        #pragma unroll
        for (int k = 0; k < D * D; ++k) a.mom_out[(long long)k * a.b.npad + node] = kShifted<real> ? G[k] : F[k];
    real J;
    if constexpr (kShifted<real>) {
        real Fit[D * D];
        J = piola_g<real, D>(G, mu, lam, Pk, Fit);  // FP32: from G = F - I, no cancellation near F = I
    } else {
        J = piola<real, D>(F, mu, lam, Pk);
    }
    const int st = check_state<real, D>(v, F, J);
    if (st) set_status(a.status, st);
    const long long P = a.b.npad;
    real unh[D], unl[D];
    #pragma unroll
    for (int i = 0; i < D; ++i) {
        if constexpr (kDispPair<real>) {
            float hi = a.ustar[i * P + node], lo = a.ustar[(D + i) * P + node];
            const float d = real(0.5) * a.dt * v[i];
            df_add(hi, lo, d);  // u^n (Eq. u-recovery-general)
            unh[i] = hi;
            unl[i] = lo;
            df_add(hi, lo, d);  // u*^{n+1}
            a.ustar[i * P + node] = hi;
            a.ustar[(D + i) * P + node] = lo;
        } else {
            const real un = a.ustar[i * P + node] + real(0.5) * a.dt * v[i];  // u^n (Eq. u-recovery-general)
            unh[i] = un;
            unl[i] = real(0);
            a.ustar[i * P + node] = un + real(0.5) * a.dt * v[i];              // u*^{n+1}
        }
    }
    if (fl & kNeedU) un_store<real, D>(a.un, node, unh, unl);
    collide_store<real, D, pop>(a, node, cut, f, v, G, F, Pk);
}

// projection steps, part 1: gather + recovery; stores f^n (pre-collision), v^n, G^n, u^n (FP64)
template <typename real, int D, int MODE, typename pop = real>
__global__ void __launch_bounds__(128) k_gather_moments(const StepArgs<real> a) {
    constexpr int K = D + D * D, Q = 2 * D;
    const int sgi = blockIdx.x * 4 + (threadIdx.x >> 5);
    if (sgi >= a.nseg) return;
    const int2 sg = __ldg(&a.seg[sgi]);
    const int lane = threadIdx.x & 31;
    const int x = sg.x - sg.y * a.b.nx + lane;
    if (x >= a.b.nx) return;
    const int node = sg.x + lane;
    const uint8_t fl = __ldg(a.flags + node);
    if (!(fl & kActive)) return;
    const int y = sg.y % a.b.ny, z = sg.y / a.b.ny;
    real f[Q * K];
    gather<real, D, MODE, pop>(a, node, x, y, z, fl & kCutMask, f);
    real v[D], G[D * D], F[D * D];
    recover<real, D>(a, f, v, G, F);
    const long long P = a.b.npad;
    #pragma unroll
    for (int j = 0; j < Q * K; ++j) pop_st<real, pop>(a.fdst, (long long)j * P + node, f[j]);
    #pragma unroll
    for (int i = 0; i < D; ++i) {
        a.vst[i * P + node] = v[i];
        if constexpr (kDispPair<real>) {
            float hi = a.ustar[i * P + node], lo = a.ustar[(D + i) * P + node];
            df_add(hi, lo, real(0.5) * a.dt * v[i]);
            a.u0[i * P + node] = hi;
            a.u0[(D + i) * P + node] = lo;
        } else {
            a.u0[i * P + node] = a.ustar[i * P + node] + 0.5 * a.dt * v[i];
        }
    }
    #pragma unroll
    for (int k = 0; k < D * D; ++k) a.Gst[k * P + node] = G[k];
}

// Output of a field call: any pointer may be null.  layout 0: component c of node n at c*nbox + n;
// 1: at n*ncomp + c.
struct FieldOut {
    double *v, *F, *u, *sigma, *J;
    int layout;
};

__device__ __forceinline__ void field_put(double *p, int layout, long long nbox, long long node, int ncomp, int c,
                                          double val) {
    if (layout) p[node * ncomp + c] = val;
    else p[c * nbox + node] = val;
}

// field output: v, F, u at the current time, and the Cauchy stress sigma = J^-1 P F^T
// (Eq. cauchy-recovery-general) and J = det F in FP64 from the recovered F
template <typename real, int D, int MODE, typename pop = real>
__global__ void __launch_bounds__(128) k_fields(const StepArgs<real> a, const FieldOut o) {
    constexpr int K = D + D * D, Q = 2 * D;
    const int sgi = blockIdx.x * 4 + (threadIdx.x >> 5);
    if (sgi >= a.nseg) return;
    const int2 sg = __ldg(&a.seg[sgi]);
    const int lane = threadIdx.x & 31;
    const int x = sg.x - sg.y * a.b.nx + lane;
    if (x >= a.b.nx) return;
    const int node = sg.x + lane;
    const uint8_t fl = __ldg(a.flags + node);
    if (!(fl & kActive)) return;
    const int y = sg.y % a.b.ny, z = sg.y / a.b.ny;
    real f[Q * K];
    gather<real, D, MODE, pop>(a, node, x, y, z, fl & kCutMask, f);
    real v[D], G[D * D], F[D * D];
    recover<real, D>(a, f, v, G, F);
    const long long N = a.b.nbox, P = a.b.npad;
    for (int i = 0; i < D; ++i) {
        if (o.v) field_put(o.v, o.layout, N, node, D, i, (double)v[i]);
        if (o.u) field_put(o.u, o.layout, N, node, D, i, disp_get<real>(a.ustar, P, D, i, node) + 0.5 * (double)a.dt * (double)v[i]);
    }
    double Fd[D * D];
    for (int i = 0; i < D; ++i)
        for (int B = 0; B < D; ++B)
            Fd[i * D + B] = kShifted<real> ? (double)G[i * D + B] + (i == B ? 1.0 : 0.0) : (double)F[i * D + B];
    if (o.F)
        for (int k = 0; k < D * D; ++k) field_put(o.F, o.layout, N, node, D * D, k, Fd[k]);
    if (o.sigma || o.J) {
        real mu, lam;
        node_material(a, node, mu, lam);
        double Pd[D * D];
        const double J = piola<double, D>(Fd, (double)mu, (double)lam, Pd);
        if (o.J) field_put(o.J, o.layout, N, node, 1, 0, J);
        if (o.sigma)
            for (int i = 0; i < D; ++i)
                for (int B = 0; B < D; ++B) {
                    double sacc = 0.0;
                    for (int A = 0; A < D; ++A) sacc += Pd[i * D + A] * Fd[B * D + A];
                    field_put(o.sigma, o.layout, N, node, D * D, i * D + B, sacc / J);
                }
    }
}

// ---------------------------------------------------------------------------------------------
// whole-body diagnostics: per-block partial records over a fixed grid, then one final block
// ---------------------------------------------------------------------------------------------

// partial record: sum |v|^2, max |v|^2, min J, max J, max c_T^2, sum of squared edge residuals, edges
constexpr int kDiagRec = 8;

__device__ __forceinline__ void diag_warp_reduce(double r[kDiagRec]) {
    #pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        r[0] += __shfl_down_sync(0xffffffffu, r[0], o);
        r[1] = fmax(r[1], __shfl_down_sync(0xffffffffu, r[1], o));
        r[2] = fmin(r[2], __shfl_down_sync(0xffffffffu, r[2], o));
        r[3] = fmax(r[3], __shfl_down_sync(0xffffffffu, r[3], o));
        r[4] = fmax(r[4], __shfl_down_sync(0xffffffffu, r[4], o));
        r[5] += __shfl_down_sync(0xffffffffu, r[5], o);
        r[6] += __shfl_down_sync(0xffffffffu, r[6], o);
    }
}

__device__ __forceinline__ void diag_init(double r[kDiagRec]) {
    r[0] = 0.0; r[1] = 0.0; r[2] = INFINITY; r[3] = -INFINITY; r[4] = 0.0; r[5] = 0.0; r[6] = 0.0; r[7] = 0.0;
}

// the state of node `node` as the diagnostics use it: v, G = F - I (FP64 from the form's values), u
template <typename real, int D, int MODE, typename pop>
__device__ __forceinline__ void diag_state(const StepArgs<real> &a, int node, double v[D], double G[D * D],
                                           double u[D]) {
    constexpr int K = D + D * D, Q = 2 * D;
    int x, y, z;
    node_xyz(a.b, node, x, y, z);
    const uint8_t fl = __ldg(a.flags + node);
    real f[Q * K];
    gather<real, D, MODE, pop>(a, node, x, y, z, fl & kCutMask, f);
    real vr[D], Gr[D * D], Fr[D * D];
    recover<real, D>(a, f, vr, Gr, Fr);
    const long long P = a.b.npad;
    for (int i = 0; i < D; ++i) {
        v[i] = (double)vr[i];
        u[i] = disp_get<real>(a.ustar, P, D, i, node) + 0.5 * (double)a.dt * v[i];
    }
    for (int k = 0; k < D * D; ++k)
        G[k] = kShifted<real> ? (double)Gr[k] : (double)Fr[k] - ((k / D == k % D) ? 1.0 : 0.0);
}

// one thread per active node, segments strided over a fixed grid; the node's state and, for the
// compatibility residual, the states of its active forward axis neighbours (interior links)
template <typename real, int D, int MODE, typename pop = real>
__global__ void __launch_bounds__(128) k_diag(const StepArgs<real> a, double *partial) {
    __shared__ double sm[4][kDiagRec];
    double r[kDiagRec];
    diag_init(r);
    const int lane = threadIdx.x & 31;
    for (int sgi = blockIdx.x * 4 + (threadIdx.x >> 5); sgi < a.nseg; sgi += gridDim.x * 4) {
        const int2 sg = __ldg(&a.seg[sgi]);
        const int x = sg.x - sg.y * a.b.nx + lane;
        const int node = sg.x + lane;
        if (x >= a.b.nx || !(__ldg(a.flags + node) & kActive)) continue;
        const unsigned cut = __ldg(a.flags + node) & kCutMask;
        double v[D], G[D * D], u[D];
        diag_state<real, D, MODE, pop>(a, node, v, G, u);
        double F[D * D];
        for (int k = 0; k < D * D; ++k) F[k] = G[k] + ((k / D == k % D) ? 1.0 : 0.0);
        real mu, lam;
        node_material(a, node, mu, lam);
        double v2 = 0.0;
        for (int i = 0; i < D; ++i) v2 += v[i] * v[i];
        const double J = 1.0 + det_m1<double, D>(G);
        r[0] += v2;
        r[1] = fmax(r[1], v2);
        r[2] = fmin(r[2], J);
        r[3] = fmax(r[3], J);
        r[4] = fmax(r[4], tangent_speed2<D>(F, (double)mu, (double)lam));
        int y, z, xx;
        node_xyz(a.b, node, xx, y, z);
        for (int A = 0; A < D; ++A) {
            if ((cut >> (2 * A)) & 1) continue;  // +e_A neighbour inactive or outside the box
            const int l = nbr(a.b, node, xx, y, z, 2 * A);
            double vl[D], Gl[D * D], ul[D];
            diag_state<real, D, MODE, pop>(a, l, vl, Gl, ul);
            for (int i = 0; i < D; ++i) {
                // u_m - u_l - (G_m + G_l)(X_m - X_l)/2 with X_m - X_l = -dx e_A
                const double e = (u[i] - ul[i]) + 0.5 * (G[i * D + A] + Gl[i * D + A]) * a.b.dx;
                r[5] += e * e;
            }
            r[6] += 1.0;
        }
    }
    diag_warp_reduce(r);
    if (lane == 0)
        for (int k = 0; k < kDiagRec; ++k) sm[threadIdx.x >> 5][k] = r[k];
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < 4; ++w) {
            sm[0][0] += sm[w][0];
            sm[0][1] = fmax(sm[0][1], sm[w][1]);
            sm[0][2] = fmin(sm[0][2], sm[w][2]);
            sm[0][3] = fmax(sm[0][3], sm[w][3]);
            sm[0][4] = fmax(sm[0][4], sm[w][4]);
            sm[0][5] += sm[w][5];
            sm[0][6] += sm[w][6];
        }
        for (int k = 0; k < kDiagRec; ++k) partial[blockIdx.x * kDiagRec + k] = sm[0][k];
    }
}

// one block of 256: combines n partial diagnostic records in a fixed order into out[0..kDiagRec)
static __global__ void __launch_bounds__(256) k_diag_final(const double *__restrict__ partial, int n, double *out) {
    __shared__ double sm[8][kDiagRec];
    double r[kDiagRec];
    diag_init(r);
    for (int j = threadIdx.x; j < n; j += 256) {
        const double *p = partial + (long long)j * kDiagRec;
        r[0] += p[0];
        r[1] = fmax(r[1], p[1]);
        r[2] = fmin(r[2], p[2]);
        r[3] = fmax(r[3], p[3]);
        r[4] = fmax(r[4], p[4]);
        r[5] += p[5];
        r[6] += p[6];
    }
    diag_warp_reduce(r);
    if ((threadIdx.x & 31) == 0)
        for (int k = 0; k < kDiagRec; ++k) sm[threadIdx.x >> 5][k] = r[k];
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < 8; ++w) {
            sm[0][0] += sm[w][0];
            sm[0][1] = fmax(sm[0][1], sm[w][1]);
            sm[0][2] = fmin(sm[0][2], sm[w][2]);
            sm[0][3] = fmax(sm[0][3], sm[w][3]);
            sm[0][4] = fmax(sm[0][4], sm[w][4]);
            sm[0][5] += sm[w][5];
            sm[0][6] += sm[w][6];
        }
        for (int k = 0; k < kDiagRec; ++k) out[k] = sm[0][k];
    }
}

// squared largest tangent wave speed of the initial F0 (FP64 box planes) over the active nodes, per
// block of a fixed grid (partial[block]), for the wave-speed audit
template <int D, typename MT>
__global__ void __launch_bounds__(128) k_audit_f0(Box b, const int2 *__restrict__ seg, int nseg,
                                                  const uint8_t *__restrict__ flags, const double *__restrict__ F0,
                                                  double mu_, double lam_, const uint8_t *__restrict__ mat,
                                                  const double *__restrict__ mtab, const MT *__restrict__ mu_node,
                                                  double *partial) {
    __shared__ double sm[4];
    double c2 = 0.0;
    const int lane = threadIdx.x & 31;
    for (int sgi = blockIdx.x * 4 + (threadIdx.x >> 5); sgi < nseg; sgi += gridDim.x * 4) {
        const int2 sg = __ldg(&seg[sgi]);
        const int x = sg.x - sg.y * b.nx + lane;
        const int node = sg.x + lane;
        if (x >= b.nx || !(__ldg(flags + node) & kActive)) continue;
        double F[D * D];
        for (int k = 0; k < D * D; ++k) F[k] = F0[k * b.nbox + node];
        const double mu = mu_node ? (double)mu_node[node] : (mtab ? mtab[2 * mat[node]] : mu_);
        const double lam = mtab ? mtab[2 * mat[node] + 1] : lam_;
        c2 = fmax(c2, tangent_speed2<D>(F, mu, lam));
    }
    #pragma unroll
    for (int o = 16; o > 0; o >>= 1) c2 = fmax(c2, __shfl_down_sync(0xffffffffu, c2, o));
    if (lane == 0) sm[threadIdx.x >> 5] = c2;
    __syncthreads();
    if (threadIdx.x == 0) partial[blockIdx.x] = fmax(fmax(sm[0], sm[1]), fmax(sm[2], sm[3]));
}

// =============================================================================================
// K4: boundary sources S~_b per cut link (Secs. 3.3-3.4)
// =============================================================================================

template <typename real> struct CutArgs {
    LinkGeom<real> L;
    Box b;
    const uint8_t *flags;
    const real *fstar;  // f* after the collision of the step just taken
    const BCD *bcs;
    const real *un;
    long long npad;
    double t, dt, c, mu, lam;
    const uint8_t *mat;  // per-node group and (mu, lambda) per group of a multi-specimen body, or null
    const real *mtab;
    const real *mu_field;  // per-node shear modulus, or null
    int D;
    int *status;
};

template <typename real, int D>
__device__ __forceinline__ bool traction_residual(const real h[D], const real N[D], const real g[D - 1][D],
                                                  const real t[D - 1][D], const real T[D], real mu, real lam, real R[D]) {
    real F[D * D], P[D * D];
    #pragma unroll
    for (int i = 0; i < D; ++i)
        #pragma unroll
        for (int A = 0; A < D; ++A) {
            real v = h[i] * N[A];
            #pragma unroll
            for (int al = 0; al < D - 1; ++al) v += g[al][i] * t[al][A];
            F[i * D + A] = v;
        }
    const real J = det<real, D>(F);
    if (!(J > real(0))) return false;
    piola<real, D>(F, mu, lam, P);
    #pragma unroll
    for (int i = 0; i < D; ++i) {
        real s = 0;
        #pragma unroll
        for (int A = 0; A < D; ++A) s += P[i * D + A] * N[A];
        R[i] = s - T[i];
    }
    return true;
}

// FP64 form: one thread per cut link, the oracle's arithmetic and iteration (the FP32 forms use
// k_links_f32).
template <typename real, int D>
__global__ void __launch_bounds__(256) k_cutlinks(const CutArgs<real> a) {
    static_assert(sizeof(real) == 8, "FP64 form only");
    using pop = real;
    constexpr int K = D + D * D;
    const long long l = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (l >= a.L.ncut) return;
    const int q = a.L.q[l], A = q >> 1;
    const real s = (q & 1) ? real(-1) : real(1);  // e = s e_A, d = -e
    const BCD &bc = a.bcs[a.L.bc[l]];
    // operands of the reconstruction at the end, loaded first so that they arrive during the
    // source computation: the node's kept pair f*_c(m), f*_{c^1}(m) and, for eta < 1/2 with an
    // active upstream node m + e_{c^1}, that node's f*_c
    const int mnode = a.L.node[l];
    const real eta_r = (real)a.L.eta[l];
    const bool up = !((__ldg(a.flags + mnode) >> (q ^ 1)) & 1);
    real fo[K], fi[K], fu[K];
    vload<K>(a.L.fo + l * (2 * K), fo);
    vload<K>(a.L.fo + l * (2 * K) + K, fi);
    if (up && !(eta_r >= real(0.5))) {
        int x, y, z;
        node_xyz(a.b, mnode, x, y, z);
        int mup = nbr(a.b, mnode, x, y, z, q ^ 1);
        TLV_BOUND(mup, a.b.npad, a.status);
        #pragma unroll
        for (int k = 0; k < K; ++k) fu[k] = pop_ld<real, pop>(a.fstar, (long long)(q * K + k) * a.b.npad + mup);
    } else {
        #pragma unroll
        for (int k = 0; k < K; ++k) fu[k] = fo[k];
    }
    const double Xb[3] = {a.L.Xb[3 * l], a.L.Xb[3 * l + 1], a.L.Xb[3 * l + 2]};
    const double th = a.t + 0.5 * a.dt;  // boundary data at t^n + dt/2
    const real c = (real)a.c;
    real S[K];
    if (bc.kind == 0) {
        // velocity Dirichlet rows (Eqs. dirichlet-rows-curved, dirichlet-compact-curved)
        double vb[3];
        dirichlet_eval(bc, D, Xb, th, false, vb);
        #pragma unroll
        for (int i = 0; i < D; ++i) {
            S[i] = (real)vb[i] / real(D);
            #pragma unroll
            for (int B = 0; B < D; ++B) S[D + i * D + B] = (B == A) ? s * (real)vb[i] / c : real(0);
        }
    } else {
        // nominal-traction Neumann rows (Eqs. neumann-rows-curved, neumann-compact-curved)
        const real mu = a.mu_field ? a.mu_field[mnode] : (a.mtab ? a.mtab[2 * a.mat[mnode]] : (real)a.mu);
        const real lam = a.mtab ? a.mtab[2 * a.mat[mnode] + 1] : (real)a.lam;
        real N[D], t[D - 1][D], g[D - 1][D];
        #pragma unroll
        for (int i = 0; i < D; ++i) N[i] = (real)a.L.Nb[3 * l + i];
        #pragma unroll
        for (int al = 0; al < D - 1; ++al)
            #pragma unroll
            for (int i = 0; i < D; ++i) { t[al][i] = (real)a.L.tan[6 * l + 3 * al + i]; g[al][i] = real(0); }
        // tangent images g_a = t_a + sum_j w_aj (u_j - u_m)  (Eqs. tangent-derivative-2d, tangent-image-3d-lsq)
        const int ns = a.L.ns[l];
        // g = t + sum_j w_j u_j in stencil order, as the oracle sums it
        #pragma unroll
        for (int al = 0; al < D - 1; ++al)
            #pragma unroll
            for (int i = 0; i < D; ++i) g[al][i] = t[al][i];
        // stencil entries in groups of 4: all index loads, then all displacement loads, then the sums,
        // so each thread keeps several independent loads in flight
        constexpr int U = 4;
        for (int j0 = 0; j0 < ns; j0 += U) {
            int kk[U];
            real w[U][D - 1], uu[U][D], uul[U][D];
            #pragma unroll
            for (int jj = 0; jj < U; ++jj) {
                const int j = j0 + jj < ns ? j0 + jj : ns - 1;
                kk[jj] = __ldg(a.L.sidx + (long long)j * a.L.ncut + l);
                TLV_BOUND(kk[jj], a.npad, a.status);
                #pragma unroll
                for (int al = 0; al < D - 1; ++al) w[jj][al] = __ldg(a.L.w + ((long long)al * kLsqCap + j) * a.L.ncut + l);
            }
            #pragma unroll
            for (int jj = 0; jj < U; ++jj) un_load<real, D>(a.un, kk[jj], uu[jj], uul[jj]);
            #pragma unroll
            for (int jj = 0; jj < U; ++jj) {
                if (j0 + jj >= ns) break;
                #pragma unroll
                for (int i = 0; i < D; ++i) {
                    const real du = uu[jj][i];
                    #pragma unroll
                    for (int al = 0; al < D - 1; ++al) g[al][i] += w[jj][al] * du;
                }
            }
        }
        double Td[3];
        traction_eval(bc, D, Xb, th, Td);
        real T[D];
        real tinf = 0;
        #pragma unroll
        for (int i = 0; i < D; ++i) { T[i] = (real)Td[i]; tinf = fmax(tinf, fabs(T[i])); }
        // Newton for the normal image h (Eqs. Fb-decomp-2d/3d, neumann-newton-2d/3d): central
        // finite-difference Jacobian, halving line search that rejects det F_b <= 0, stop at
        // |R| <= 1e-13 (mu + lambda + |T|)
        const real tol = real(1e-13) * (mu + lam + tinf);
        const real fd = real(1e-6);
        real h[D], R[D];
        #pragma unroll
        for (int i = 0; i < D; ++i) h[i] = a.L.h[3 * l + i];
        bool ok = traction_residual<real, D>(h, N, g, t, T, mu, lam, R);
        if (!ok) {
            #pragma unroll
            for (int i = 0; i < D; ++i) h[i] = N[i];
            ok = traction_residual<real, D>(h, N, g, t, T, mu, lam, R);
        }
        bool conv = false;
        for (int it = 0; ok && it < 30; ++it) {
            real rinf = 0, r2 = 0;
            #pragma unroll
            for (int i = 0; i < D; ++i) { rinf = fmax(rinf, fabs(R[i])); r2 += R[i] * R[i]; }
            if (!isfinite(r2)) { ok = false; break; }  // fmax drops NaN; r2 does not
            if (rinf <= tol) { conv = true; break; }
            real hinf = 0;
            #pragma unroll
            for (int i = 0; i < D; ++i) hinf = fmax(hinf, fabs(h[i]));
            const real del = fd * fmax(real(1), hinf);
            real Jm[D * D];
            #pragma unroll
            for (int j = 0; j < D; ++j) {
                real hp[D], hm[D], Rp[D], Rm[D];
                #pragma unroll
                for (int i = 0; i < D; ++i) { hp[i] = h[i]; hm[i] = h[i]; }
                hp[j] += del;
                hm[j] -= del;
                ok = traction_residual<real, D>(hp, N, g, t, T, mu, lam, Rp) &&
                     traction_residual<real, D>(hm, N, g, t, T, mu, lam, Rm);
                if (!ok) break;
                #pragma unroll
                for (int i = 0; i < D; ++i) Jm[i * D + j] = (Rp[i] - Rm[i]) / (real(2) * del);
            }
            if (!ok) break;
            real mR[D], dh[D];
            #pragma unroll
            for (int i = 0; i < D; ++i) mR[i] = -R[i];
            if (!solve_small<real, D>(Jm, mR, dh)) { ok = false; break; }
            real al = 1;
            bool acc = false;
            real ht[D], Rt[D];
            for (int ls = 0; ls < 20; ++ls) {
                #pragma unroll
                for (int i = 0; i < D; ++i) ht[i] = h[i] + al * dh[i];
                if (traction_residual<real, D>(ht, N, g, t, T, mu, lam, Rt)) {
                    real rt2 = 0;
                    #pragma unroll
                    for (int i = 0; i < D; ++i) rt2 += Rt[i] * Rt[i];
                    if (rt2 < r2) { acc = true; break; }
                }
                al *= real(0.5);
            }
            if (!acc) { conv = rinf <= real(1e3) * tol; break; }
            #pragma unroll
            for (int i = 0; i < D; ++i) { h[i] = ht[i]; R[i] = Rt[i]; }
        }
        if (!(ok && conv)) {
            set_status(a.status, kStNewton);
            #pragma unroll
            for (int i = 0; i < D; ++i) h[i] = a.L.h[3 * l + i];
        } else {
            #pragma unroll
            for (int i = 0; i < D; ++i) a.L.h[3 * l + i] = h[i];
        }
        real Fb[D * D], Pb[D * D];
        #pragma unroll
        for (int i = 0; i < D; ++i)
            #pragma unroll
            for (int B = 0; B < D; ++B) {
                real v = h[i] * N[B];
                #pragma unroll
                for (int al = 0; al < D - 1; ++al) v += g[al][i] * t[al][B];
                Fb[i * D + B] = v;
            }
        piola<real, D>(Fb, mu, lam, Pb);
        #pragma unroll
        for (int i = 0; i < D; ++i) {
            S[i] = s * Pb[i * D + A] / c;  // -d_A P_iA / c with d = -s e_A
            #pragma unroll
            for (int B = 0; B < D; ++B)
                S[D + i * D + B] = Fb[i * D + B] / real(D);
        }
    }
    // Interpolated bounce-back of the incoming population f_{c^1}(m) for the next gather
    // (Eqs. bfl-curved-far, bfl-curved-near), from the node's post-collision values f*_c(m),
    // f*_{c^1}(m) and, for eta < 1/2, f*_c of the upstream node m + e_{c^1} (m itself when that
    // node is inactive); D_b = diag(-I, I) for Dirichlet, diag(I, -I) for Neumann links.
    {
        const real eta = eta_r;
        const bool neu = bc.kind != 0;
        real R[K];
        #pragma unroll
        for (int k = 0; k < K; ++k) {
            const real Dk = ((k < D) == neu) ? real(1) : real(-1);
            if (eta >= real(0.5))
                R[k] = (Dk * fo[k] + S[k]) / (real(2) * eta) + (real(1) - real(1) / (real(2) * eta)) * fi[k];
            else
                R[k] = Dk * (real(2) * eta * fo[k] + (real(1) - real(2) * eta) * fu[k]) + S[k];
        }
        vstore<K>(a.L.rec + l * K, R);
    }
}

// Projection correction d and residual, node-major so that a neighbour is one vector load:
// d holds kDV values per node (D components, padded to 2 or 4), the residual 4 values per node,
// (r_1..r_D, w) padded, with the sweep weight w = beta/deg (0 where a node is inactive or has no
// edge).  Inactive nodes keep d = 0 in both buffers (the storage is zeroed and sweeps write active
// nodes only).
template <int D> constexpr int kDV = D == 3 ? 4 : 2;

}  // namespace tlv
