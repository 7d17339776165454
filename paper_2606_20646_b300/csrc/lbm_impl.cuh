// Host-side orchestration shared by the precision-specific translation units: the handle,
// storage carving helpers, and Impl<real, D, pop> which launches the kernels of one update (real:
// arithmetic type; pop: population storage type, real itself or BF16 with FP32 arithmetic).
#pragma once

#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <new>
#include <type_traits>
#include <vector>

#include <cudaTypedefs.h>
#include <cstdlib>
#include <nvtx3/nvToolsExt.h>

#include "lbm.h"
#include "lbm_kernels.cuh"
#include "lbm_proj.cuh"
#include "lbm_jacobi2.cuh"
#include "lbm_tma.cuh"
#include "lbm_links.cuh"
#include "lbm_adjoint.cuh"

using namespace tlv;

constexpr size_t kAlign = 256;
constexpr unsigned kReduceBlocks = 16 * 148;  // fixed grid of the gauge reduction (16 blocks per SM)

inline size_t align_up(size_t v) { return (v + kAlign - 1) / kAlign * kAlign; }

struct Carver {
    char *base;
    size_t off = 0;
    template <typename T> T *take(size_t count) {
        T *p = base ? reinterpret_cast<T *>(base + off) : nullptr;
        off = align_up(off + count * sizeof(T));
        return p;
    }
};

struct EventPair {
    cudaEvent_t a, b;
    int cls;
    int launches;  // kernels between the two events
};

struct lbm_handle {
    lbm_grid grid{};
    lbm_options opt{};
    lbm_material mat{};
    int nshapes = 0, nbc = 0, ngroups = 0;
    ShapeD shapes[kMaxShapes]{};
    GroupD groups[kMaxGroups]{};
    double gmat[2 * kMaxGroups]{};  // (mu, lambda) per group
    float gmat_f[2 * kMaxGroups]{};
    BCD bcs[kMaxBCs]{};
    bool has_neumann_bc = false;
    cudaStream_t stream = nullptr;
    int D = 0, K = 0, Q = 0;
    int real_size = 8;  // bytes of the arithmetic type
    int pop_size = 8;   // bytes of a stored population value (2 for BF16 storage)
    Box box{};
    int segs_per_row = 0;
    long long nsegmax = 0;
    // geometry storage
    char *geo = nullptr;
    size_t geo_bytes = 0;
    uint8_t *flags = nullptr;
    int *lstart = nullptr, *cnt = nullptr, *scan_scratch = nullptr, *segflag = nullptr, *segidx = nullptr;
    int2 *seg = nullptr;
    unsigned long long *counters = nullptr;
    ShapeD *dshapes = nullptr;
    GroupD *dgroups = nullptr;
    uint8_t *gidx = nullptr;         // per-node group index
    double *mtab_d = nullptr;        // (mu, lambda) per group, FP64 and FP32 copies
    float *mtab_f = nullptr;
    BCD *dbcs = nullptr;
    int *status = nullptr;
    long long n_active = 0, n_cut = 0, nseg = 0;
    cudaGraphExec_t graph_exec = nullptr;  // the last lbm_step_graph graph
    // reverse mode (options.adjoint)
    void *mu_field = nullptr;       // per-node shear modulus (population precision)
    bool mu_field_on = false;
    void *adj_g[2] = {nullptr, nullptr};  // gbar of consecutive steps (Q*K planes each)
    double *adj_mubar = nullptr, *adj_bslot = nullptr;  // dL/dmu per node; dL/db slots (kAdjSlots x 4)
    void *adj_lu = nullptr;         // dL/du* (D planes, population precision)
    void *adj_coef = nullptr, *adj_side = nullptr;  // per cut link: closure derivatives; side rows
    int adj_cur = 0;                // adj_g[adj_cur] holds gbar of the last reversed step
    long long adj_next = -1;        // step the next lbm_adjoint_step reverses (-1: no sweep)
    TmaMaps adj_maps[2];            // bulk-copy maps of adj_g[0], adj_g[1] (FP32)
    bool adj_maps_ok = false;
    void *mom_out = nullptr;        // lbm_step_moments: where this step records F
    cudaStream_t capture_stream = nullptr; // private stream that lbm_step_graph records on
    // solver storage
    char *sto = nullptr;
    size_t sto_bytes = 0;
    bool bound = false;
    void *fA = nullptr, *fB = nullptr, *ustar = nullptr, *un = nullptr, *vst = nullptr, *Gst = nullptr;
    uint8_t *dmask = nullptr;
    int *l_node = nullptr, *l_q = nullptr, *l_bc = nullptr, *l_ns = nullptr, *l_sidx = nullptr;
    double *l_eta = nullptr, *l_Xb = nullptr, *l_Nb = nullptr, *l_tan = nullptr;
    void *l_h = nullptr, *l_w = nullptr, *l_rec = nullptr, *l_fo = nullptr;
    float4 *l_bvec = nullptr;  // FP32 forms: per-link geometric vector of the boundary profile
    float *l_cu = nullptr;     // FP32 forms: per-link coefficient of the upstream term added by the gather
    float *l_gsum = nullptr;   // FP32 forms with Neumann links: per-link tangent-image sums (8 floats)
    void *u0 = nullptr, *u1 = nullptr;  // projection warm starts (displacement-accumulator layout)
    double *partial = nullptr, *mean = nullptr, *staging = nullptr;
    double *diag = nullptr;  // diagnostics and audit reductions: kReduceBlocks partial records + the result
    void *dA = nullptr, *dB = nullptr, *resid = nullptr;  // projection correction buffers and residual
    long long n_neu = 0, n_dir = 0, lsq_entries = 0;
    // two Jacobi sweeps per launch (FP32 forms, no periodic axis): maps of dA, dB and the residual,
    // the tiles holding an active node
    bool jp_ok = false;
    JPairMaps jp_maps;
    int *jp_tiles = nullptr;
    int jp_ntiles = 0;
    // state
    bool initialized = false;
    int phase = 0;  // 0: fA holds pre-collision f^0; 1: fA holds post-collision f*^{n-1}
    long long step = 0;
    long long launches = 0;
    // TMA staging of the FP32 gather: tensor maps of both population buffers
    bool tma_ok = false;
    void *tma_buf[2] = {nullptr, nullptr};
    TmaMaps tma_maps[2];
    // tile shapes (0: the form's default): 32-node windows per warp of the fused kernel, segments
    // per warp of a Jacobi sweep, threads per block of the link kernel
    int tune_nw = 0, tune_jseg = 0, tune_lblock = 0, tune_jsweeps = 0;
    int wait_limit = -1;  // polls of the bulk-copy kernels' first wait (< 0: kTmaSpin)
    // timing
    bool timing = false;
    std::vector<EventPair> events;
    double acc_ms[4] = {0, 0, 0, 0};  // stream-collide, cut links, projection, Jacobi sweeps
    long long acc_n[4] = {0, 0, 0, 0};
};

// =============================================================================================
// helpers
// =============================================================================================

// NVTX range over a host scope (header-only NVTX 3: inert unless a profiler is attached)
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};

#define CK(call)                                           \
    do {                                                   \
        cudaError_t e_ = (call);                           \
        if (e_ != cudaSuccess) return LBM_ERR_CUDA;        \
    } while (0)

#define CKL()                                              \
    do {                                                   \
        cudaError_t e_ = cudaGetLastError();               \
        if (e_ != cudaSuccess) return LBM_ERR_CUDA;        \
    } while (0)

static __global__ void k_convert_field(const double *__restrict__ in, void *out, long long n, int rs) {
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= n) return;
    if (rs == 8) static_cast<double *>(out)[i] = in[i];
    else static_cast<float *>(out)[i] = (float)in[i];
}

// a box-ordered FP64 field into a field of the population precision (same node indices)
inline cudaError_t convert_field(const double *in, void *out, long long n, int rs, cudaStream_t st) {
    k_convert_field<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(in, out, n, rs);
    return cudaGetLastError();
}

// the first n values of a node-indexed FP64 array to caller memory (device or host)
inline cudaError_t gather_box(const double *in, double *out, long long n, cudaStream_t st);

inline bool is_device_ptr(const void *p) {
    if (!p) return false;
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

inline cudaError_t gather_box(const double *in, double *out, long long n, cudaStream_t st) {
    return cudaMemcpyAsync(out, in, (size_t)n * sizeof(double),
                           is_device_ptr(out) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, st);
}

inline unsigned grid_for(long long n, int per_block) { return (unsigned)((n + per_block - 1) / per_block); }

inline size_t scan_scratch_ints(long long n) {
    size_t s = 0;
    while (n > 1) {
        long long nb = (n + 1023) / 1024;
        s += 2 * (size_t)nb + 32;
        n = nb;
    }
    return s + 64;
}

// exclusive scan of n ints (in -> out) using scratch; returns LBM_OK or LBM_ERR_CUDA
inline int scan(const int *in, int *out, long long n, int *scratch, cudaStream_t st) {
    long long nb = (n + 1023) / 1024;
    int *bsum = scratch, *boff = scratch + nb + 16;
    k_scan_block<<<(unsigned)nb, 1024, 0, st>>>(in, out, bsum, n);
    CKL();
    if (nb > 1) {
        int rc = scan(bsum, boff, nb, boff + nb + 16, st);
        if (rc) return rc;
        k_scan_add<<<(unsigned)nb, 1024, 0, st>>>(out, boff, n);
        CKL();
    }
    return LBM_OK;
}

inline void timing_begin(lbm_handle *h, EventPair &ep, int cls, int launches = 1) {
    ep.cls = cls;
    ep.launches = launches;
    cudaEventCreate(&ep.a);
    cudaEventCreate(&ep.b);
    cudaEventRecord(ep.a, h->stream);
}

inline void timing_end(lbm_handle *h, EventPair &ep) {
    cudaEventRecord(ep.b, h->stream);
    h->events.push_back(ep);
}

inline void timing_fold(lbm_handle *h) {
    for (auto &ep : h->events) {
        cudaEventSynchronize(ep.b);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, ep.a, ep.b);
        h->acc_ms[ep.cls] += ms;
        h->acc_n[ep.cls] += ep.launches;
        cudaEventDestroy(ep.a);
        cudaEventDestroy(ep.b);
    }
    h->events.clear();
}

// Tensor maps of a population buffer viewed as a 2D tensor (node index, plane); cuTensorMapEncodeTiled
// is fetched through the runtime's driver entry point so the library does not link libcuda.
inline PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
    static PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
    if (!encode) {
        void *fn = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) !=
                cudaSuccess ||
            q != cudaDriverEntryPointSuccess || !fn) {
            cudaGetLastError();
            return nullptr;
        }
        encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
    }
    return encode;
}

// u* planes (npad, 2D: hi then lo) with (32, 2D) boxes, and the flag bytes viewed as (nx, ny*nz) with
// (32, 1) boxes
inline bool encode_meta_maps(void *ustar, long long npad, int D, void *flags, int nx, long long rows, TmaMaps *out) {
    PFN_cuTensorMapEncodeTiled_v12000 encode = tensor_map_encoder();
    if (!encode) return false;
    const cuuint32_t es[2] = {1, 1};
    const cuuint64_t udims[2] = {(cuuint64_t)npad, (cuuint64_t)(2 * D)};
    const cuuint64_t ustr[1] = {(cuuint64_t)npad * 4};
    const cuuint32_t ubox[2] = {32, (cuuint32_t)(2 * D)};
    const cuuint64_t fdims[2] = {(cuuint64_t)nx, (cuuint64_t)rows};
    const cuuint64_t fstr[1] = {(cuuint64_t)nx};
    const cuuint32_t fbox[2] = {32, 1};
    CUresult r1 = encode(&out->ustar, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, ustar, udims, ustr, ubox, es,
                         CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                         CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    CUresult r2 = encode(&out->flags, CU_TENSOR_MAP_DATA_TYPE_UINT8, 2, flags, fdims, fstr, fbox, es,
                         CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                         CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r1 == CUDA_SUCCESS && r2 == CUDA_SUCCESS;
}

// population planes as a 2D tensor (node index, plane) of E-byte elements (4: FP32, 2: BF16): boxes of
// (32 + 2*16/E, K) for the +-x pulls and (32, K) otherwise
inline bool encode_population_maps(void *base, long long npad, int planes, int K, TmaMaps *out, int E = 4) {
    static PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
    if (!encode) {
        void *fn = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) !=
                cudaSuccess ||
            q != cudaDriverEntryPointSuccess || !fn) {
            cudaGetLastError();
            return false;
        }
        encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
    }
    const cuuint64_t dims[2] = {(cuuint64_t)npad, (cuuint64_t)planes};
    if (E != 4 && E != 2) return false;
    const CUtensorMapDataType ty = E == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16;
    const cuuint64_t strides[1] = {(cuuint64_t)npad * E};
    const cuuint32_t es[2] = {1, 1};
    const cuuint32_t wide[2] = {(cuuint32_t)(32 + 2 * (16 / E)), (cuuint32_t)K};
    const cuuint32_t narrow[2] = {(cuuint32_t)kTmaNarrow, (cuuint32_t)K};
    CUresult r1 = encode(&out->wide, ty, 2, base, dims, strides, wide, es,
                         CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                         CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    CUresult r2 = encode(&out->narrow, ty, 2, base, dims, strides, narrow, es,
                         CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                         CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r1 == CUDA_SUCCESS && r2 == CUDA_SUCCESS;
}

// Maps of the two-sweep Jacobi kernel.  A row's 4-float node records are one float axis of 4 nx
// values, so a box row is one contiguous run of bytes (boxes whose innermost extent was a single
// 16-byte record copied as many small pieces: the 3D two-sweep kernel took 87 instead of 74.5 us per
// sweep at 256^3).  3D: d and the residual as (4 nx floats, y, z) with boxes (128, rows, 1).  2D: d
// as (x, y) of 8-byte elements (a (d_1, d_2) pair) with box (NP, 1), the residual as (4 nx floats,
// y) with boxes (256, 1) (three per row) and (4 NP - 768, 1) (the row's tail).
inline bool encode_jpair_maps(int D, void *dA, void *dB, void *resid, int nx, int ny, int nz, JPairMaps *out) {
    PFN_cuTensorMapEncodeTiled_v12000 encode = tensor_map_encoder();
    if (!encode) return false;
    bool ok = true;
    auto enc = [&](CUtensorMap *m, CUtensorMapDataType ty, int rank, void *base, const cuuint64_t *dims,
                   const cuuint64_t *strides, const cuuint32_t *box) {
        const cuuint32_t es[4] = {1, 1, 1, 1};
        ok = ok && encode(m, ty, rank, base, dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                          CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
    };
    if (D == 3) {
        const cuuint64_t dims[3] = {4ull * nx, (cuuint64_t)ny, (cuuint64_t)nz};
        const cuuint64_t str[2] = {16ull * nx, 16ull * nx * ny};
        const cuuint32_t bd[3] = {128, (cuuint32_t)JPairLayout<3>::RD, 1};
        const cuuint32_t br[3] = {128, (cuuint32_t)JPairLayout<3>::RR, 1};
        enc(&out->d[0], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, dA, dims, str, bd);
        enc(&out->d[1], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, dB, dims, str, bd);
        enc(&out->r, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, resid, dims, str, br);
    } else {
        if (nx % 2) return false;  // rows of 8-byte pairs must be 16-byte multiples
        const cuuint64_t dd[2] = {(cuuint64_t)nx, (cuuint64_t)ny};
        const cuuint64_t sd[1] = {8ull * nx};
        const cuuint32_t bd[2] = {(cuuint32_t)JPairLayout<2>::NP, 1};
        const cuuint64_t dr[2] = {4ull * nx, (cuuint64_t)ny};
        const cuuint64_t sr[1] = {16ull * nx};
        const cuuint32_t br[2] = {256, 1}, brt[2] = {(cuuint32_t)JPairLayout<2>::r_tail, 1};
        enc(&out->d[0], CU_TENSOR_MAP_DATA_TYPE_UINT64, 2, dA, dd, sd, bd);
        enc(&out->d[1], CU_TENSOR_MAP_DATA_TYPE_UINT64, 2, dB, dd, sd, bd);
        enc(&out->r, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, resid, dr, sr, br);
        enc(&out->rt, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, resid, dr, sr, brt);
    }
    return ok;
}

inline LevelSetD levelset_view(const lbm_handle *h) {
    LevelSetD L;
    L.shapes = h->dshapes;
    L.nshapes = h->nshapes;
    L.groups = h->dgroups;
    L.ngroups = h->ngroups;
    return L;
}

// =============================================================================================
// precision- and dimension-specialised operations
// =============================================================================================

template <typename real, int D, typename pop = real> struct Impl {
    static constexpr bool kPlainPop = std::is_same<real, pop>::value;
    static constexpr int K = D + D * D, Q = 2 * D;

    static const real *mtab(lbm_handle *h) {
        if constexpr (sizeof(real) == 8) return h->mtab_d;
        else return h->mtab_f;
    }

    static LinkGeom<real> links(lbm_handle *h) {
        LinkGeom<real> L;
        L.node = h->l_node;
        L.q = h->l_q;
        L.bc = h->l_bc;
        L.eta = h->l_eta;
        L.Xb = h->l_Xb;
        L.Nb = h->l_Nb;
        L.tan = h->l_tan;
        L.h = static_cast<real *>(h->l_h);
        L.ns = h->l_ns;
        L.sidx = h->l_sidx;
        L.w = static_cast<real *>(h->l_w);
        L.rec = static_cast<real *>(h->l_rec);
        L.fo = static_cast<real *>(h->l_fo);
        L.cu = h->l_cu;
        L.bvec = h->l_bvec;
        L.ncut = h->n_cut;
        return L;
    }

    static StepArgs<real> step_args(lbm_handle *h) {
        StepArgs<real> a;
        a.b = h->box;
        a.seg = h->seg;
        a.nseg = (int)h->nseg;
        a.flags = h->flags;
        a.lstart = h->lstart;
        a.fsrc = static_cast<const real *>(h->fA);
        a.fdst = static_cast<real *>(h->fB);
        a.ustar = static_cast<real *>(h->ustar);
        a.un = static_cast<real *>(h->un);
        a.lrec = static_cast<const real *>(h->l_rec);
        a.lcu = h->l_cu;
        a.lfo = static_cast<real *>(h->l_fo);
        a.vst = static_cast<real *>(h->vst);
        a.Gst = static_cast<real *>(h->Gst);
        a.u0 = static_cast<real *>(h->u0);
        const double dt = h->grid.dx / h->opt.c;
        a.dt = (real)dt;
        a.c = (real)h->opt.c;
        a.omega = (real)h->opt.omega;
        a.gamma = (real)h->opt.gamma;
        a.mu = (real)h->mat.mu;
        a.lam = (real)h->mat.lambda;
        for (int i = 0; i < 3; ++i) a.bf[i] = (real)h->opt.body_force[i];
        a.mat = h->ngroups > 0 ? h->gidx : nullptr;
        a.mtab = h->ngroups > 0 ? mtab(h) : nullptr;
        a.mu_field = h->mu_field_on ? static_cast<const real *>(h->mu_field) : nullptr;
        a.mom_out = static_cast<real *>(h->mom_out);
        a.status = h->status;
        a.spin = h->wait_limit >= 0 ? h->wait_limit : kTmaSpin;
        a.ncut = std::max<long long>(h->n_cut, 1);
        return a;
    }

    static ProjArgs<real> proj_args(lbm_handle *h, double t, const real *warm) {
        ProjArgs<real> p;
        p.b = h->box;
        p.seg = h->seg;
        p.nseg = (int)h->nseg;
        p.flags = h->flags;
        p.dmask = h->dmask;
        p.lstart = h->lstart;
        p.L = links(h);
        p.bcs = h->dbcs;
        p.Gst = static_cast<const real *>(h->Gst);
        p.u0 = warm;
        p.resid = static_cast<real *>(h->resid);
        p.t = t;
        p.beta = h->opt.proj_beta;
        p.status = h->status;
        return p;
    }

    // FP32 arithmetic only (FP32 or BF16 storage): tensor maps for the TMA-staged gather (rows of a
    // multiple of 16 nodes, so that window starts and the flag box fall on 16-byte boundaries)
    static void setup_tma(lbm_handle *h) {
        h->tma_ok = false;
        h->adj_maps_ok = false;
        if constexpr (sizeof(real) == 4) {
            const char *off = std::getenv("LBM_B300_NO_TMA");
            // population boxes need rows aligned to 4 floats; the flag box needs rows of 16 bytes
            if ((off && off[0] == '1') || (h->box.nx % 16) != 0) return;
            bool ok = true;
            for (int j = 0; j < 2; ++j) {
                h->tma_buf[j] = j == 0 ? h->fA : h->fB;
                ok = ok && encode_population_maps(h->tma_buf[j], h->box.npad, Q * K, K, &h->tma_maps[j], (int)sizeof(pop)) &&
                     encode_meta_maps(h->ustar, h->box.npad, D, h->flags, h->box.nx,
                                      (long long)h->box.ny * h->box.nz, &h->tma_maps[j]);
            }
            if (ok)
                ok = fused_attr<1>() && fused_attr<2>() && fused_attr<4>() && fused_attr<1, true>() &&
                     cudaFuncSetAttribute(k_gather_moments_tma<D, pop>, cudaFuncAttributePreferredSharedMemoryCarveout, 100) ==
                         cudaSuccess &&
                     cudaFuncSetAttribute(k_gather_moments_tma<D, pop, false>, cudaFuncAttributePreferredSharedMemoryCarveout,
                                          100) == cudaSuccess;
            if (ok && h->opt.adjoint && kPlainPop) {
                h->adj_maps_ok = true;
                for (int j = 0; j < 2; ++j) {
                    h->adj_maps[j] = h->tma_maps[0];  // flags and u* maps; population maps replaced
                    h->adj_maps_ok = h->adj_maps_ok &&
                                     encode_population_maps(h->adj_g[j], h->box.npad, Q * K, K, &h->adj_maps[j]);
                }
                h->adj_maps_ok = h->adj_maps_ok &&
                                 cudaFuncSetAttribute(k_adj_step_tma<D>, cudaFuncAttributePreferredSharedMemoryCarveout,
                                                      100) == cudaSuccess;
            }
            cudaGetLastError();
            h->tma_ok = ok;
        }
    }

    template <int NW> static int fused_smem() { return NW * (TmaLayout<D, sizeof(pop)>::stage_bytes + 8); }
    template <int NW, bool REPAIR = false> static bool fused_attr() {
        return cudaFuncSetAttribute(k_stream_collide_tma<D, pop, NW, REPAIR>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    fused_smem<NW>()) == cudaSuccess &&
               cudaFuncSetAttribute(k_stream_collide_tma<D, pop, NW, REPAIR>,
                                    cudaFuncAttributePreferredSharedMemoryCarveout, 100) == cudaSuccess;
    }
    // the fused kernel with the handle's windows per warp
    template <int NW> static void launch_fused_nw(lbm_handle *h, const StepArgs<float> &a) {
        k_stream_collide_tma<D, pop, NW><<<grid_for(h->nseg, NW), 32, fused_smem<NW>(), h->stream>>>(a, *maps_of(h, h->fA),
                                                                                                  RepairArgs{});
    }
    static void launch_fused(lbm_handle *h, const StepArgs<float> &a) {
        const int nw = h->tune_nw ? h->tune_nw : kTmaWindows<pop>;
        if (nw == 4) launch_fused_nw<4>(h, a);
        else if (nw == 2) launch_fused_nw<2>(h, a);
        else launch_fused_nw<1>(h, a);
    }
    // a grid of the blocks resident at once (occupancy query, once per instantiation), at most one
    // block per 4 S segments
    template <int S> static void launch_jacobi_s(lbm_handle *h, const ProjArgs<real> &p, const real *src, real *dst) {
        if (h->box.per[0]) launch_jacobi_sx<S, false>(h, p, src, dst);
        else launch_jacobi_sx<S, true>(h, p, src, dst);
    }
    template <int S, bool SHX>
    static void launch_jacobi_sx(lbm_handle *h, const ProjArgs<real> &p, const real *src, real *dst) {
        static int resident = 0;
        if (resident == 0) {
            int per_sm = 0, dev = 0, sms = 0;
            if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_jacobi<real, D, S, SHX>, 128, 0) != cudaSuccess ||
                cudaGetDevice(&dev) != cudaSuccess ||
                cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || per_sm < 1) {
                cudaGetLastError();
                per_sm = 8;
                sms = 148;
            }
            resident = per_sm * sms;
        }
        const unsigned g = std::min<unsigned>(grid_for(h->nseg, 4 * S), (unsigned)resident);
        k_jacobi<real, D, S, SHX><<<std::max(g, 1u), 128, 0, h->stream>>>(p, src, dst);
    }
    static void launch_jacobi(lbm_handle *h, const ProjArgs<real> &p, const real *src, real *dst) {
        const int js = h->tune_jseg ? h->tune_jseg : kJacobiSegs;
        if (js == 4) launch_jacobi_s<4>(h, p, src, dst);
        else if (js == 1) launch_jacobi_s<1>(h, p, src, dst);
        else launch_jacobi_s<2>(h, p, src, dst);
    }

    static const TmaMaps *maps_of(lbm_handle *h, const void *buf) {
        return h->tma_buf[0] == buf ? &h->tma_maps[0] : &h->tma_maps[1];
    }

    static int link_build(lbm_handle *h) {
        NvtxRange range("cut-link geometry");
        setup_tma(h);
        if (h->nseg == 0) return LBM_OK;
        k_link_build<real, D><<<grid_for(h->nseg, 4), 128, 0, h->stream>>>(
            h->box, h->seg, (int)h->nseg, h->flags, h->dmask, h->lstart, levelset_view(h), h->dbcs, h->nbc,
            links(h), h->status);
        CKL();
        if constexpr (sizeof(real) == 4) {
            if (h->n_cut > 0) {
                k_link_cu<D><<<grid_for(h->n_cut, 256), 256, 0, h->stream>>>(links(h), h->flags, h->dbcs);
                CKL();
            }
        }
        return setup_jpair(h);
    }

    // two-sweep Jacobi: maps, kernel attributes and the list of tiles holding an active node (the
    // geometry pass's window scratch holds the tile flags and their scan)
    static int setup_jpair(lbm_handle *h) {
        h->jp_ok = false;
        h->jp_ntiles = 0;
        if constexpr (sizeof(real) == 4) {
            const Box &b = h->box;
            if (!h->jp_tiles || b.per[0] || b.per[1] || b.per[2] || h->nseg == 0) return LBM_OK;
            int ntx, nty, ntz;
            jp_tile_grid(D, b.nx, b.ny, b.nz, ntx, nty, ntz);
            const long long nt = (long long)ntx * nty * ntz;
            if (nt > h->nsegmax) return LBM_OK;
            bool ok = encode_jpair_maps(D, h->dA, h->dB, h->resid, b.nx, b.ny, b.nz, &h->jp_maps);
            if constexpr (D == 3)
                ok = ok && cudaFuncSetAttribute(k_jacobi_pair3, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                JPairLayout<3>::smem_bytes) == cudaSuccess &&
                     cudaFuncSetAttribute(k_jacobi_pair3, cudaFuncAttributePreferredSharedMemoryCarveout, 100) ==
                         cudaSuccess;
            else
                ok = ok && cudaFuncSetAttribute(k_jacobi_pair2, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                JPairLayout<2>::smem_bytes) == cudaSuccess &&
                     cudaFuncSetAttribute(k_jacobi_pair2, cudaFuncAttributePreferredSharedMemoryCarveout, 100) ==
                         cudaSuccess;
            cudaGetLastError();
            if (!ok) return LBM_OK;
            CK(cudaMemsetAsync(h->segflag, 0, (size_t)nt * sizeof(int), h->stream));
            k_jp_mark<<<grid_for(b.nbox, 256), 256, 0, h->stream>>>(b, h->flags, h->segflag);
            CKL();
            if (scan(h->segflag, h->segidx, nt, h->scan_scratch, h->stream)) return LBM_ERR_CUDA;
            k_jp_compact<<<grid_for(nt, 256), 256, 0, h->stream>>>(h->segflag, h->segidx, (int)nt, h->jp_tiles);
            CKL();
            int last[2] = {0, 0};
            CK(cudaMemcpyAsync(&last[0], h->segidx + (nt - 1), sizeof(int), cudaMemcpyDeviceToHost, h->stream));
            CK(cudaMemcpyAsync(&last[1], h->segflag + (nt - 1), sizeof(int), cudaMemcpyDeviceToHost, h->stream));
            CK(cudaStreamSynchronize(h->stream));
            h->jp_ntiles = last[0] + last[1];
            h->jp_ok = h->jp_ntiles > 0;
        }
        return LBM_OK;
    }

    // two sweeps from src (nullptr: d = 0) into dst with the two-sweep kernel
    static void launch_jpair(lbm_handle *h, const ProjArgs<real> &p, const real *src, real *dst) {
        if constexpr (sizeof(real) == 4) {
            const CUtensorMap &dm = h->jp_maps.d[src == static_cast<const real *>(h->dB) ? 1 : 0];
            const int spin = h->wait_limit >= 0 ? h->wait_limit : kTmaSpin;
            if constexpr (D == 3)
                k_jacobi_pair3<<<h->jp_ntiles, JPairLayout<3>::threads, JPairLayout<3>::smem_bytes, h->stream>>>(
                    p, dm, h->jp_maps.r, src == nullptr, dst, h->jp_tiles, spin);
            else
                k_jacobi_pair2<<<h->jp_ntiles, JPairLayout<2>::threads, JPairLayout<2>::smem_bytes, h->stream>>>(
                    p, dm, h->jp_maps.r, h->jp_maps.rt, src == nullptr, dst, h->jp_tiles, spin);
        }
    }
    // two sweeps per launch: chosen by the tuning, else the default of the dimension (2D: on; 3D:
    // off, the 3D tiles' halos and per-plane barriers cost more than the second pass over memory)
    static bool jpair_on(const lbm_handle *h) {
        return h->jp_ok && (h->tune_jsweeps ? h->tune_jsweeps == 2 : D == 2);
    }

    static int init(lbm_handle *h, int mode, const double *v0, const double *F0, const double *u0, const double *dU0) {
        const double dt = h->grid.dx / h->opt.c;
        k_init<real, D, pop><<<grid_for(h->nseg, 4), 128, 0, h->stream>>>(
            h->box, h->seg, (int)h->nseg, h->flags, v0, F0, u0, dU0, mode == LBM_INIT_CHARACTERISTIC, h->opt.c, dt,
            h->mat.mu, h->mat.lambda, h->gidx, h->ngroups > 0 ? h->mtab_d : nullptr,
            h->mu_field_on ? static_cast<const real *>(h->mu_field) : nullptr, h->opt.gamma,
            h->opt.body_force[0], h->opt.body_force[1], h->opt.body_force[2], static_cast<real *>(h->fA),
            static_cast<real *>(h->ustar));
        CKL();
        return LBM_OK;
    }

    // boundary values of every boundary condition at time th as M g_l + k (FP32 link kernel): the
    // ramp and the time factors in FP64 on the host, once per launch
    static BCTimes bc_times(const lbm_handle *h, double th) {
        BCTimes T;
        std::memset(&T, 0, sizeof(T));
        for (int b = 0; b < h->nbc; ++b) {
            const BCD &bc = h->bcs[b];
            double s = 1.0, sd = 0.0;
            ramp_eval(bc.ramp, bc.t_ramp, th, s, sd);
            double M[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0}, k[3] = {0, 0, 0};
            if (bc.kind == LBM_BC_DIRICHLET) {  // the lattice sees v_D = d u_D / dt
                switch (bc.profile) {
                case LBM_PROFILE_AFFINE:
                    for (int i = 0; i < 9; ++i) M[i] = sd * bc.A[i];
                    break;
                case LBM_PROFILE_RADIAL:
                    for (int i = 0; i < D; ++i) M[4 * i] = bc.amp * sd;
                    break;
                case LBM_PROFILE_TWIST_STRETCH: {
                    const double al = s * bc.amp, ald = sd * bc.amp;
                    M[0] = -ald * std::sin(al);
                    M[1] = -ald * std::cos(al);
                    M[3] = ald * std::cos(al);
                    M[4] = -ald * std::sin(al);
                    if (D == 3) k[2] = sd * bc.vec[2];
                    break;
                }
                case LBM_PROFILE_CONST:
                    for (int i = 0; i < D; ++i) k[i] = sd * bc.vec[i];
                    break;
                default:
                    break;
                }
            } else {  // nominal traction
                if (bc.profile == LBM_PROFILE_RADIAL)
                    for (int i = 0; i < D; ++i) M[4 * i] = bc.amp * s;
                else if (bc.profile == LBM_PROFILE_CONST)
                    for (int i = 0; i < D; ++i) k[i] = s * bc.vec[i];
            }
            BCTimeF &o = T.bc[b];
            for (int i = 0; i < 9; ++i) o.M[i] = (float)M[i];
            for (int i = 0; i < 3; ++i) o.k[i] = (float)k[i];
            o.kind = bc.kind;
        }
        return T;
    }

    static int cutlinks(lbm_handle *h, double t) {
        if (h->n_cut == 0) return LBM_OK;
        CutArgs<real> a;
        a.L = links(h);
        a.b = h->box;
        a.flags = h->flags;
        a.fstar = static_cast<const real *>(h->fA);  // this step's post-collision state, read by the next gather
        a.bcs = h->dbcs;
        a.un = static_cast<const real *>(h->un);
        a.npad = h->box.npad;
        a.t = t;
        a.dt = h->grid.dx / h->opt.c;
        a.c = h->opt.c;
        a.mu = h->mat.mu;
        a.lam = h->mat.lambda;
        a.mat = h->ngroups > 0 ? h->gidx : nullptr;
        a.mtab = h->ngroups > 0 ? mtab(h) : nullptr;
        a.mu_field = h->mu_field_on ? static_cast<const real *>(h->mu_field) : nullptr;
        a.D = D;
        a.status = h->status;
        EventPair ep;
        if (h->timing) timing_begin(h, ep, 1);
        const int lb = h->tune_lblock ? h->tune_lblock : 128;
        if constexpr (sizeof(real) == 4) {
            if (h->n_neu > 0) {
                k_link_sums<D><<<grid_for(h->n_cut * kLinkLanes<D>, 256), 256, 0, h->stream>>>(a, h->l_gsum);
                h->launches++;
            }
            k_links_f32<D, pop><<<grid_for(h->n_cut, lb), lb, 0, h->stream>>>(a, bc_times(h, t + 0.5 * a.dt), h->l_gsum);
        }
        else
            k_cutlinks<real, D><<<grid_for(h->n_cut, lb), lb, 0, h->stream>>>(a);
        if (h->timing) timing_end(h, ep);
        h->launches++;
        CKL();
        return LBM_OK;
    }

    // one projection solve from the warm start `warm`: FP64-accumulated residual, proj_iters damped-Jacobi
    // sweeps on the correction d (population precision), gauge shift into h->mean (zero when Dirichlet
    // anchors exist).  Returns the final correction buffer in *d.
    static int solve(lbm_handle *h, double t, const real *warm, real **d) {
        ProjArgs<real> p = proj_args(h, t, warm);
        const unsigned g = grid_for(h->nseg, 4);
        k_proj_residual<real, D><<<g, 128, 0, h->stream>>>(p);
        h->launches++;
        CKL();
        real *A = static_cast<real *>(h->dA), *B = static_cast<real *>(h->dB);
        const real *src = nullptr;
        real *dst = A;
        EventPair ep;
        if (h->timing && h->opt.proj_iters > 0) timing_begin(h, ep, 3, h->opt.proj_iters);
        for (int it = 0; it < h->opt.proj_iters;) {
            if (jpair_on(h) && it + 1 < h->opt.proj_iters) {
                launch_jpair(h, p, src, dst);
                it += 2;
            } else {
                launch_jacobi(h, p, src, dst);
                it += 1;
            }
            h->launches++;
            src = dst;
            dst = (dst == A) ? B : A;
        }
        if (h->timing && h->opt.proj_iters > 0) timing_end(h, ep);
        CKL();
        if (!src) {  // no sweeps: zero correction
            CK(cudaMemsetAsync(A, 0, (size_t)kDV<D> * h->box.npad * sizeof(real), h->stream));
            src = A;
        }
        if (h->n_dir == 0) {
            const unsigned gr = std::min<unsigned>(g, kReduceBlocks);
            k_reduce_partial<real, D><<<gr, 128, 0, h->stream>>>(p, src, h->partial);
            k_reduce_final<D><<<1, 256, 0, h->stream>>>(h->partial, (int)gr, 1.0 / (double)h->n_active, h->mean);
            h->launches += 2;
            CKL();
        } else {
            CK(cudaMemsetAsync(h->mean, 0, D * sizeof(double), h->stream));
        }
        *d = const_cast<real *>(src);
        return LBM_OK;
    }

    static int step(lbm_handle *h, int nsteps) {
        NvtxRange range("lbm_step");
        const double dt = h->grid.dx / h->opt.c;
        for (int n = 0; n < nsteps; ++n) {
            const double t = h->step * dt;
            StepArgs<real> a = step_args(h);
            const bool proj = h->n_neu > 0 && h->opt.proj_every > 0 && (h->step % h->opt.proj_every) == 0;
            const unsigned g = grid_for(h->nseg, 4);
            bool post_in_B = true;  // where this step leaves the post-collision populations
            if (!proj) {
                EventPair ep;
                if (h->timing) timing_begin(h, ep, 0);
                if (h->phase == 0) k_stream_collide<real, D, 0, pop><<<g, 128, 0, h->stream>>>(a);
                else if constexpr (sizeof(real) == 4) {
                    if (h->tma_ok)
                        launch_fused(h, a);
                    else
                        k_stream_collide<real, D, 1, pop><<<g, 128, 0, h->stream>>>(a);
                } else k_stream_collide<real, D, 1, pop><<<g, 128, 0, h->stream>>>(a);
                if (h->timing) timing_end(h, ep);
                h->launches++;
                CKL();
            } else {
                NvtxRange prange("projection step");
                EventPair ep;
                if (h->timing) timing_begin(h, ep, 2);
                // bulk-copy path (FP32 forms after the first step): the gather stores the moments
                // only, the repair re-gathers f^n from fA and writes f*^n into fB (a regular step's
                // buffers); otherwise the gather stores f^n into fB and the plain repair writes f*^n
                // into fA
                bool staged = false;
                if constexpr (sizeof(real) == 4) staged = h->tma_ok && h->phase == 1;
                if (h->phase == 0) k_gather_moments<real, D, 0, pop><<<g, 128, 0, h->stream>>>(a);
                else if constexpr (sizeof(real) == 4) {
                    if (staged)
                        k_gather_moments_tma<D, pop, false><<<g, 128, TmaLayout<D, sizeof(pop)>::block_bytes(4), h->stream>>>(
                            a, *maps_of(h, h->fA));
                    else
                        k_gather_moments<real, D, 1, pop><<<g, 128, 0, h->stream>>>(a);
                } else k_gather_moments<real, D, 1, pop><<<g, 128, 0, h->stream>>>(a);
                h->launches++;
                CKL();
                real *d = nullptr;
                int rc = solve(h, t, static_cast<const real *>(h->u0), &d);
                if (rc) return rc;
                if constexpr (sizeof(real) == 4) {
                    if (staged) {
                        RepairArgs rp;
                        rp.u0 = static_cast<const float *>(h->u0);
                        rp.dc = d;
                        rp.mean = h->mean;
                        rp.theta = (float)h->opt.theta_F;
                        rp.u1 = static_cast<float *>(h->u1);
                        k_stream_collide_tma<D, pop, 1, true><<<grid_for(h->nseg, 1), 32, fused_smem<1>(), h->stream>>>(
                            a, *maps_of(h, h->fA), rp);
                    }
                }
                if (!staged) {
                    // out of place: f^n (from the gather, in fB) in, f*^n out into fA, whose f*^{n-1}
                    // the gather has consumed
                    StepArgs<real> ar = a;
                    ar.fsrc = static_cast<const real *>(h->fB);
                    ar.fdst = static_cast<real *>(h->fA);
                    k_repair_collide<real, D, pop><<<g, 128, 0, h->stream>>>(ar, static_cast<const real *>(h->u0), d,
                                                                         h->mean, h->opt.theta_F,
                                                                         static_cast<real *>(h->u1));
                }
                post_in_B = staged;
                h->launches++;
                CKL();
                rc = solve(h, t, static_cast<const real *>(h->u1), &d);
                if (rc) return rc;
                k_proj_reset<real, D><<<g, 128, 0, h->stream>>>(a, static_cast<const real *>(h->u1), d, h->mean);
                h->launches++;
                CKL();
                if (h->timing) timing_end(h, ep);
            }
            // the post-collision state: fB after a regular step or a bulk-copy projection step, fA
            // after a plain-load projection step
            if (post_in_B) std::swap(h->fA, h->fB);
            int rc = cutlinks(h, t);
            if (rc) return rc;
            h->phase = 1;
            h->step++;
        }
        return LBM_OK;
    }

    static AdjArgs<real> adj_args(lbm_handle *h, int in) {
        AdjArgs<real> j;
        j.mom = nullptr;
        j.g_in = static_cast<const real *>(h->adj_g[in]);
        j.g_out = static_cast<real *>(h->adj_g[in ^ 1]);
        j.mubar = h->adj_mubar;
        j.bslot = h->adj_bslot;
        j.lu = static_cast<const real *>(h->adj_lu);
        j.grad_u = nullptr;
        j.coef = static_cast<const real *>(h->adj_coef);
        j.side = static_cast<real *>(h->adj_side);
        j.nbox = h->box.nbox;
        return j;
    }

    // seed of a reverse sweep at the current state (after h->step steps)
    static int adjoint_begin(lbm_handle *h, const double *grad_u) {
        const size_t np = (size_t)h->box.npad;
        CK(cudaMemsetAsync(h->adj_mubar, 0, np * sizeof(double), h->stream));
        CK(cudaMemsetAsync(h->adj_bslot, 0, 4 * kAdjSlots * sizeof(double), h->stream));
        CK(cudaMemsetAsync(h->adj_g[0], 0, (size_t)Q * K * np * sizeof(real), h->stream));
        CK(cudaMemsetAsync(h->adj_g[1], 0, (size_t)Q * K * np * sizeof(real), h->stream));
        if (h->n_cut > 0) {
            k_adj_coef<real><<<grid_for(h->n_cut, 256), 256, 0, h->stream>>>(
                h->flags, h->l_node, h->l_q, h->l_bc, h->l_eta, h->dbcs, h->n_cut, static_cast<real *>(h->adj_coef));
            CKL();
        }
        StepArgs<real> a = step_args(h);
        AdjArgs<real> j = adj_args(h, 1);  // seed writes adj_g[0]
        j.grad_u = grad_u;
        k_adj_seed<real, D><<<grid_for(h->nseg, 4), 128, 0, h->stream>>>(a, j, static_cast<real *>(h->adj_lu));
        CKL();
        h->adj_cur = 0;
        h->adj_next = h->step - 1;
        return LBM_OK;
    }

    // reverse of step n = h->adj_next, given F of that step as lbm_step_moments recorded it
    static int adjoint_step(lbm_handle *h, const void *moments) {
        NvtxRange range("lbm_adjoint_step");
        const long long n = h->adj_next;
        StepArgs<real> a = step_args(h);
        AdjArgs<real> j = adj_args(h, h->adj_cur);
        j.mom = static_cast<const real *>(moments);
        bool staged = false;
        if constexpr (sizeof(real) == 4) {
            if (h->tma_ok && h->adj_maps_ok) {
                k_adj_step_tma<D><<<(unsigned)h->nseg, 32, AdjLayout<D>::bytes + 8, h->stream>>>(
                    a, j, h->adj_maps[h->adj_cur]);
                staged = true;
            }
        }
        if (!staged) k_adj_step<real, D><<<grid_for(h->nseg, 4), 128, 0, h->stream>>>(a, j);
        CKL();
        h->adj_cur ^= 1;
        h->adj_next = n - 1;
        return LBM_OK;
    }

    static int fields(lbm_handle *h, const FieldOut &o) {
        StepArgs<real> a = step_args(h);
        const unsigned g = grid_for(h->nseg, 4);
        if (h->phase == 0) k_fields<real, D, 0, pop><<<g, 128, 0, h->stream>>>(a, o);
        else k_fields<real, D, 1, pop><<<g, 128, 0, h->stream>>>(a, o);
        CKL();
        return LBM_OK;
    }

    // whole-body diagnostics: partial records over a fixed grid of kReduceBlocks blocks into h->diag,
    // the combined record into h->diag + kReduceBlocks * kDiagRec
    static int diagnostics(lbm_handle *h) {
        NvtxRange range("lbm_diagnostics");
        StepArgs<real> a = step_args(h);
        const unsigned gr = (unsigned)std::max<long long>(1, std::min<long long>(grid_for(h->nseg, 4), kReduceBlocks));
        if (h->phase == 0) k_diag<real, D, 0, pop><<<gr, 128, 0, h->stream>>>(a, h->diag);
        else k_diag<real, D, 1, pop><<<gr, 128, 0, h->stream>>>(a, h->diag);
        k_diag_final<<<1, 256, 0, h->stream>>>(h->diag, (int)gr, h->diag + (size_t)kReduceBlocks * kDiagRec);
        CKL();
        return LBM_OK;
    }
};

