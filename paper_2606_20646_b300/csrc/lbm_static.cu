// Geometry census without any device allocation (lbm_census_static in include/lbm.h).
//
// Some callers cannot allocate device memory at the point where they need to size a
// simulation: an embedding runtime (a serving process, a solver framework) whose device memory
// is one arena planned ahead and handed out by its own allocator, so that a library call must
// not take memory behind its back; or a process already running at its memory limit, which has
// to learn how much storage a body needs before it can free or plan that much.
// lbm_census_static gives them the counts that size lbm_create's and lbm_bind_storage's
// storage (active nodes, cut links, active 32-node x-segments) with all of its scratch in one
// file-scope device array of fixed size: the active mask of the box (one byte per node) and
// four counters.  Every GPU that loads this library holds the array until the process exits.
// It applies lbm_create's domain rules: no active node, or a body that extends past a
// non-periodic box face, is LBM_ERR_DOMAIN.
//
// Host code never dereferences the array's name (on the host it is only a stand-in): the first
// call on a device, with that device current, asks the runtime for the array's device address
// with cudaGetSymbolAddress and keeps it for that device.  That first call therefore makes a
// runtime query and should come before any stream capture.  All calls on a device share the
// array: calls that overlap on the GPU race with each other.  Each call clears the counters and
// rewrites the mask before using them.  The call synchronises the stream it is given before it
// returns the counts.
#include <cuda_runtime.h>

#include <cstdint>
#include <mutex>

#include "lbm.h"
#include "lbm_kernels.cuh"

using namespace tlv;

namespace {

constexpr long long kCensusMaxNodes = LBM_CENSUS_MAX_NODES;
constexpr int kMaxDevices = 64;
constexpr int kMaskOffset = 256;  // bytes [0, 32): counters (active, cut, segments, box-face violations)

__device__ __align__(256) unsigned char g_census_scratch[kMaskOffset + kCensusMaxNodes];

unsigned char *g_scratch_addr[kMaxDevices] = {};
std::mutex g_scratch_mu;

struct ShapeTable {
    ShapeD s[LBM_CENSUS_MAX_SHAPES];
};

__global__ void k_census_mask(Box b, const __grid_constant__ ShapeTable shapes, int nshapes, unsigned char *scratch) {
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= b.nbox) return;
    int x, y, z;
    node_xyz(b, (int)i, x, y, z);
    double X[3];
    node_X(b, x, y, z, X);
    scratch[kMaskOffset + i] = (levelset(shapes.s, nshapes, b.D, X, nullptr) <= 0.0) ? 1 : 0;
}

// counting variant of the cut-bit pass: the same link rule (neighbour inactive or outside a
// non-periodic box), summed with warp shuffles and one atomic per warp instead of scanned.  A link
// that leaves the box must cross the surface within one spacing (the point one spacing beyond the
// face lies outside the body), the rule lbm_create applies; links that break it are counted in
// cnt[3] and make the call return LBM_ERR_DOMAIN.
__global__ void k_census_count(Box b, const __grid_constant__ ShapeTable shapes, int nshapes, unsigned char *scratch) {
    unsigned long long *cnt = reinterpret_cast<unsigned long long *>(scratch);
    const unsigned char *mask = scratch + kMaskOffset;
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    unsigned long long act = 0, cut = 0, bad = 0;
    if (i < b.nbox && mask[i]) {
        int x, y, z;
        node_xyz(b, (int)i, x, y, z);
        act = 1;
        for (int q = 0; q < 2 * b.D; ++q) {
            const int A = q >> 1, s = (q & 1) ? -1 : 1;
            const int co = (A == 0 ? x : (A == 1 ? y : z)) + s;
            const int n = (A == 0 ? b.nx : (A == 1 ? b.ny : b.nz));
            if ((co < 0 || co >= n) && !b.per[A]) {
                cut += 1;
                double X[3];
                node_X(b, x, y, z, X);
                X[A] += s * b.dx;
                if (!(levelset(shapes.s, nshapes, b.D, X, nullptr) > 0.0)) bad += 1;
            } else if (!mask[nbr(b, (int)i, x, y, z, q)]) {
                cut += 1;
            }
        }
    }
    #pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        act += __shfl_down_sync(0xffffffffu, act, o);
        cut += __shfl_down_sync(0xffffffffu, cut, o);
        bad += __shfl_down_sync(0xffffffffu, bad, o);
    }
    if ((threadIdx.x & 31) == 0) {
        if (act) atomicAdd(&cnt[0], act);
        if (cut) atomicAdd(&cnt[1], cut);
        if (bad) atomicAdd(&cnt[3], bad);
    }
}

// segments: the solver's window rule applied to each row of the mask, one thread per row
__global__ void k_census_rows(Box b, unsigned char *scratch) {
    unsigned long long *cnt = reinterpret_cast<unsigned long long *>(scratch);
    const long long row = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    unsigned long long seg = 0;
    if (row < (long long)b.ny * b.nz)
        for_each_window(scratch + kMaskOffset + row * b.nx, b.nx, 1, [&](int) { seg += 1; });
    #pragma unroll
    for (int o = 16; o > 0; o >>= 1) seg += __shfl_down_sync(0xffffffffu, seg, o);
    if ((threadIdx.x & 31) == 0 && seg) atomicAdd(&cnt[2], seg);
}

// device address of the scratch array on the current device, looked up once per device
int scratch_address(unsigned char **out) {
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return LBM_ERR_CUDA;
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    if (!g_scratch_addr[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_census_scratch) != cudaSuccess || !p) {
            cudaGetLastError();
            return LBM_ERR_CUDA;
        }
        g_scratch_addr[dev] = static_cast<unsigned char *>(p);
    }
    *out = g_scratch_addr[dev];
    return LBM_OK;
}

}  // namespace

extern "C" int lbm_census_static(const lbm_grid *grid, const lbm_levelset *ls, void *cuda_stream, long long *n_active,
                                 long long *n_cut, long long *n_segments) {
    if (!grid || !ls || !n_active || !n_cut || !n_segments) return LBM_ERR_ARG;
    if ((grid->dim != 2 && grid->dim != 3) || !(grid->dx > 0.0)) return LBM_ERR_ARG;
    if (ls->nshapes < 0 || ls->nshapes > LBM_CENSUS_MAX_SHAPES || (ls->nshapes > 0 && !ls->shapes) || ls->ngroups != 0)
        return LBM_ERR_ARG;
    Box b{};
    b.D = grid->dim;
    b.nx = grid->n[0];
    b.ny = grid->n[1];
    b.nz = grid->dim == 3 ? grid->n[2] : 1;
    if (b.nx < 1 || b.ny < 1 || b.nz < 1) return LBM_ERR_ARG;
    for (int a = 0; a < 3; ++a) {
        b.per[a] = (a < grid->dim) ? (grid->periodic[a] != 0) : 1;
        b.origin[a] = (a < grid->dim) ? grid->origin[a] : 0.0;
    }
    b.dx = grid->dx;
    b.nbox = (long long)b.nx * b.ny * b.nz;
    b.npad = b.nbox;
    if (b.nbox > kCensusMaxNodes) return LBM_ERR_CAPACITY;
    ShapeTable table{};
    for (int s = 0; s < ls->nshapes; ++s) {
        const lbm_shape &sh = ls->shapes[s];
        if (sh.kind < 0 || sh.kind > LBM_SHAPE_SAMPLED || (sh.kind == LBM_SHAPE_SAMPLED && !sh.phi)) return LBM_ERR_ARG;
        if (sh.kind == LBM_SHAPE_SUPERELLIPSE && (grid->dim != 2 || !(sh.p >= 1.0))) return LBM_ERR_ARG;
        ShapeD &d = table.s[s];
        d.kind = sh.kind;
        d.complement = sh.complement != 0;
        d.bid = sh.boundary_id;
        for (int a = 0; a < 3; ++a) {
            d.c[a] = sh.center[a];
            d.a[a] = sh.axes[a];
        }
        for (int a = 0; a < 9; ++a) d.Q[a] = sh.rot[a];
        d.p = sh.p;
        d.phi = sh.kind == LBM_SHAPE_SAMPLED ? sh.phi : nullptr;
        d.per = 0;
        for (int a = 0; a < 3; ++a) {
            d.n[a] = a < grid->dim ? grid->n[a] : 1;
            d.org[a] = a < grid->dim ? grid->origin[a] : 0.0;
            if (a < grid->dim && grid->periodic[a]) d.per |= 1 << a;
        }
        d.dx = grid->dx;
    }
    unsigned char *scratch = nullptr;
    int rc = scratch_address(&scratch);
    if (rc) return rc;
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    if (cudaMemsetAsync(scratch, 0, 4 * sizeof(unsigned long long), st) != cudaSuccess) return LBM_ERR_CUDA;
    const unsigned grid_n = (unsigned)((b.nbox + 255) / 256);
    k_census_mask<<<grid_n, 256, 0, st>>>(b, table, ls->nshapes, scratch);
    k_census_count<<<grid_n, 256, 0, st>>>(b, table, ls->nshapes, scratch);
    k_census_rows<<<(unsigned)(((long long)b.ny * b.nz + 127) / 128), 128, 0, st>>>(b, scratch);
    if (cudaGetLastError() != cudaSuccess) return LBM_ERR_CUDA;
    unsigned long long host[4] = {0, 0, 0, 0};
    if (cudaMemcpyAsync(host, scratch, sizeof(host), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return LBM_ERR_CUDA;
    *n_active = (long long)host[0];
    *n_cut = (long long)host[1];
    *n_segments = (long long)host[2];
    if (host[0] == 0 || host[3] != 0) return LBM_ERR_DOMAIN;
    return LBM_OK;
}
