// Host runtime and C ABI (include/lbm.h) of the sm_103a total-Lagrangian vectorial LBM.
//
// The handle owns host metadata only; all device memory is caller-provided.  Every
// operation is enqueued on the stream given to lbm_create.  Kernels live in
// lbm_kernels.cuh; this file validates descriptors, carves caller storage, and
// schedules one update of Algorithm 1 per step:
//   regular step     K3 fused gather/closure/collision  ->  K4 boundary sources
//   projection step  gather+moments -> projection solve -> repair+collision
//                    -> projection solve -> displacement reset -> K4
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <new>
#include <vector>

#include "lbm_ops.cuh"

static const PrecOps &ops(const lbm_handle *h) {
    return h->real_size == 8 ? ops_fp64() : (h->pop_size == 2 ? ops_bf16s() : ops_fp32());
}

// =============================================================================================
// storage layouts
// =============================================================================================

static void carve_geometry(lbm_handle *h, char *base, size_t *bytes) {
    Carver c{base};
    const long long np = h->box.npad;
    h->flags = c.take<uint8_t>(np + 64);
    h->lstart = c.take<int>(np);
    h->cnt = c.take<int>(np);
    h->segflag = c.take<int>(h->nsegmax + 1);
    h->segidx = c.take<int>(h->nsegmax + 1);
    h->seg = c.take<int2>(h->nsegmax + 1);
    h->scan_scratch = c.take<int>(scan_scratch_ints(std::max<long long>(np, h->nsegmax)));
    h->counters = c.take<unsigned long long>(8);
    h->dshapes = c.take<ShapeD>(kMaxShapes);
    h->dgroups = c.take<GroupD>(kMaxGroups);
    h->mtab_d = c.take<double>(2 * kMaxGroups);
    h->mtab_f = c.take<float>(2 * kMaxGroups);
    h->gidx = c.take<uint8_t>(np);
    h->dbcs = c.take<BCD>(kMaxBCs);
    h->status = c.take<int>(8);
    *bytes = c.off;
}

static void carve_solver(lbm_handle *h, char *base, size_t *bytes) {
    Carver c{base};
    const long long np = h->box.npad, nc = std::max<long long>(h->n_cut, 1);
    const int D = h->D, K = h->K, Q = h->Q, rs = h->real_size, ps = h->pop_size;
    h->fA = c.take<char>((size_t)Q * K * np * ps);
    h->fB = c.take<char>((size_t)Q * K * np * ps);
    // displacement accumulators: one FP64 plane per component, or a (hi, lo) pair of FP32 planes
    h->ustar = c.take<char>((size_t)D * np * 8);
    h->un = c.take<char>((size_t)(D == 3 ? 32 : 16) * np);  // node-major u^n (see kUnStride)
    h->dmask = c.take<uint8_t>(np);
    h->l_node = c.take<int>(nc);
    h->l_q = c.take<int>(nc);
    h->l_bc = c.take<int>(nc);
    h->l_ns = c.take<int>(nc);
    h->l_eta = c.take<double>(nc);
    h->l_Xb = c.take<double>(3 * nc);
    h->l_Nb = c.take<double>(3 * nc);
    h->l_tan = c.take<double>(6 * nc);
    h->l_h = c.take<char>((size_t)3 * nc * rs);
    h->l_rec = c.take<char>((size_t)K * nc * rs);
    h->l_fo = c.take<char>((size_t)2 * K * nc * rs);
    h->l_bvec = rs == 4 ? c.take<float4>(nc) : nullptr;
    h->l_cu = rs == 4 ? c.take<float>(nc) : nullptr;
    h->l_gsum = (rs == 4 && h->has_neumann_bc) ? c.take<float>((size_t)8 * nc) : nullptr;
    if (h->has_neumann_bc) {
        h->l_sidx = c.take<int>((size_t)kLsqCap * nc);
        h->l_w = c.take<char>((size_t)2 * kLsqCap * nc * rs);
        h->u0 = c.take<char>((size_t)D * np * 8);  // FP64 planes or FP32 (hi, lo) pairs
        h->u1 = c.take<char>((size_t)D * np * 8);
        // correction d (2 or 4 values per node) and residual (4 values per node), node-major
        h->dA = c.take<char>((size_t)(D == 3 ? 4 : 2) * np * rs);
        h->dB = c.take<char>((size_t)(D == 3 ? 4 : 2) * np * rs);
        h->resid = c.take<char>((size_t)4 * np * rs);
        int ntx, nty, ntz;
        jp_tile_grid(D, h->box.nx, h->box.ny, h->box.nz, ntx, nty, ntz);
        h->jp_tiles = c.take<int>((size_t)ntx * nty * ntz);
        h->vst = c.take<char>((size_t)D * np * rs);
        h->Gst = c.take<char>((size_t)D * D * np * rs);
        h->partial = c.take<double>((size_t)D * (std::max<size_t>(grid_for(h->nseg, 4), kReduceBlocks) + 1));
        h->mean = c.take<double>(4);
    } else {
        h->l_sidx = nullptr;
        h->l_w = nullptr;
        h->u0 = h->u1 = nullptr;
        h->partial = h->mean = nullptr;
        h->dA = h->dB = h->resid = h->vst = h->Gst = nullptr;
        h->jp_tiles = nullptr;
    }
    h->staging = h->opt.host_staging ? c.take<double>((size_t)(2 * D + D * D + D * K) * h->box.nbox) : nullptr;
    h->diag = c.take<double>((size_t)kDiagRec * (kReduceBlocks + 1));
    if (h->opt.adjoint) {
        h->mu_field = c.take<char>((size_t)np * rs);
        h->adj_g[0] = c.take<char>((size_t)Q * K * np * rs);
        h->adj_g[1] = c.take<char>((size_t)Q * K * np * rs);
        h->adj_mubar = c.take<double>((size_t)np);
        h->adj_bslot = c.take<double>((size_t)4 * kAdjSlots);
        h->adj_lu = c.take<char>((size_t)D * np * rs);
        h->adj_coef = c.take<char>((size_t)4 * nc * rs);
        h->adj_side = c.take<char>((size_t)K * nc * rs);
    } else {
        h->mu_field = h->adj_g[0] = h->adj_g[1] = nullptr;
        h->adj_mubar = h->adj_bslot = nullptr;
        h->adj_lu = h->adj_coef = h->adj_side = nullptr;
    }
    *bytes = c.off;
}

// saved state: a header (step, phase), the stored populations, u*, u^n, the reconstructed link
// values and the Newton states of the links
struct StateLayout {
    size_t pop, ustar, un, rec, lh, bytes;
};
static StateLayout state_layout(const lbm_handle *h) {
    Carver c{nullptr};
    const size_t np = (size_t)h->box.npad, nc = (size_t)std::max<long long>(h->n_cut, 1);
    const int D = h->D, K = h->K, Q = h->Q, rs = h->real_size;
    StateLayout L;
    c.take<char>(256);
    L.pop = c.off;
    c.take<char>((size_t)Q * K * np * h->pop_size);
    L.ustar = c.off;
    c.take<char>((size_t)D * np * 8);
    L.un = c.off;
    c.take<char>((size_t)(D == 3 ? 32 : 16) * np);
    L.rec = c.off;
    c.take<char>((size_t)K * nc * rs);
    L.lh = c.off;
    c.take<char>((size_t)3 * nc * rs);
    L.bytes = c.off;
    return L;
}

// =============================================================================================
// C ABI
// =============================================================================================

extern "C" {

const char *lbm_error_string(int code) {
    switch (code) {
    case LBM_OK: return "ok";
    case LBM_ERR_ARG: return "invalid argument or descriptor";
    case LBM_ERR_DOMAIN: return "empty body, or the body extends past a non-periodic box face";
    case LBM_ERR_CUDA: return "CUDA runtime error";
    case LBM_ERR_STORAGE: return "storage missing, too small or misaligned";
    case LBM_ERR_STATE: return "call out of order";
    case LBM_ERR_DEVICE: return "device status word is non-zero";
    case LBM_ERR_CAPACITY: return "a fixed capacity was exceeded (LSQ stencil, census box)";
    case LBM_ERR_UNSTABLE_C: return "lattice speed c below the wave-speed audit's bound";
    default: return "unknown error";
    }
}

// the lattice a sampled shape's node values sit on
static void set_sampled(ShapeD &d, const lbm_shape &sh, const lbm_grid &g) {
    d.phi = sh.kind == LBM_SHAPE_SAMPLED ? sh.phi : nullptr;
    d.per = 0;
    for (int a = 0; a < 3; ++a) {
        d.n[a] = a < g.dim ? g.n[a] : 1;
        d.org[a] = a < g.dim ? g.origin[a] : 0.0;
        if (a < g.dim && g.periodic[a]) d.per |= 1 << a;
    }
    d.dx = g.dx;
}

static int validate_grid(const lbm_grid *g) {
    if (!g || (g->dim != 2 && g->dim != 3) || !(g->dx > 0.0) || !std::isfinite(g->dx)) return LBM_ERR_ARG;
    for (int a = 0; a < g->dim; ++a)
        if (g->n[a] < 1) return LBM_ERR_ARG;
    long long nz = g->dim == 3 ? g->n[2] : 1;
    long long nbox = (long long)g->n[0] * g->n[1] * nz;
    if (nbox >= (1LL << 31) - 64) return LBM_ERR_ARG;
    return LBM_OK;
}

// Wave-speed audit (Sec. 2, Eq. acoustic-tensor-general-d): c >= factor * c_T with c_T^2 the largest
// squared tangent speed; factor = options.c_audit, 2.5 when 0, no audit when negative
static bool audit_ok(const lbm_options *opt, int dim, double cT2) {
    (void)dim;
    if (opt->c_audit < 0.0) return true;
    const double factor = opt->c_audit > 0.0 ? opt->c_audit : 2.5;
    if (!(cT2 >= 0.0)) return false;  // NaN or an unphysical material
    return opt->c >= factor * std::sqrt(cT2) * (1.0 - 1e-12);
}

int lbm_geometry_bytes(const lbm_grid *grid, size_t *bytes) {
    if (!bytes || validate_grid(grid)) return LBM_ERR_ARG;
    lbm_handle tmp;
    tmp.grid = *grid;
    long long nz = grid->dim == 3 ? grid->n[2] : 1;
    tmp.box.nbox = (long long)grid->n[0] * grid->n[1] * nz;
    tmp.box.npad = (tmp.box.nbox + 31) / 32 * 32 + 32;
    tmp.segs_per_row = (grid->n[0] + kSegAlign - 1) / kSegAlign;
    tmp.nsegmax = (long long)tmp.segs_per_row * grid->n[1] * nz;
    carve_geometry(&tmp, nullptr, bytes);
    return LBM_OK;
}

int lbm_create(const lbm_grid *grid, const lbm_levelset *ls, const lbm_material *mat, const lbm_bc *bcs, int nbc,
               const lbm_options *opt, void *geometry_storage, size_t geometry_bytes, void *cuda_stream,
               lbm_handle **out) {
    if (!out) return LBM_ERR_ARG;
    *out = nullptr;
    if (validate_grid(grid) || !ls || !mat || !opt || nbc < 0 || nbc > kMaxBCs || (nbc > 0 && !bcs))
        return LBM_ERR_ARG;
    if (ls->nshapes < 0 || ls->nshapes > kMaxShapes || (ls->nshapes > 0 && !ls->shapes)) return LBM_ERR_ARG;
    if (!(mat->mu > 0.0) || !(mat->lambda > -mat->mu)) return LBM_ERR_ARG;
    if (ls->ngroups < 0 || ls->ngroups > kMaxGroups || (ls->ngroups > 0 && (!ls->groups || ls->nshapes == 0)))
        return LBM_ERR_ARG;
    for (int g = 0; g < ls->ngroups; ++g) {
        const lbm_group &G = ls->groups[g];
        if (G.first_shape < 0 || G.nshapes < 1 || G.first_shape + G.nshapes > ls->nshapes) return LBM_ERR_ARG;
        if (!(G.material.mu > 0.0) || !(G.material.lambda > -G.material.mu)) return LBM_ERR_ARG;
        for (int a = 0; a < grid->dim; ++a)
            if (!(G.lo[a] <= G.hi[a])) return LBM_ERR_ARG;
    }
    if (opt->precision != LBM_PREC_FP64 && opt->precision != LBM_PREC_FP32 && opt->precision != LBM_PREC_BF16S)
        return LBM_ERR_ARG;
    if (opt->precision == LBM_PREC_BF16S && opt->adjoint) return LBM_ERR_ARG;
    if (!(opt->c > 0.0) || !(opt->omega > 0.0 && opt->omega <= 2.0) || !(opt->gamma >= 0.0)) return LBM_ERR_ARG;
    if (opt->proj_every < 0 || opt->proj_iters < 0 || !(opt->theta_F > 0.0 && opt->theta_F <= 1.0) ||
        !(opt->proj_beta > 0.0 && opt->proj_beta <= 1.0))
        return LBM_ERR_ARG;
    for (int s = 0; s < ls->nshapes; ++s) {
        const lbm_shape &sh = ls->shapes[s];
        if (sh.kind < 0 || sh.kind > LBM_SHAPE_SAMPLED) return LBM_ERR_ARG;
        if (sh.kind == LBM_SHAPE_SUPERELLIPSE && (grid->dim != 2 || !(sh.p >= 1.0))) return LBM_ERR_ARG;
        if (sh.kind == LBM_SHAPE_SAMPLED && !is_device_ptr(sh.phi)) return LBM_ERR_ARG;
    }
    for (int b = 0; b < nbc; ++b) {
        const lbm_bc &bc = bcs[b];
        if (bc.kind != LBM_BC_DIRICHLET && bc.kind != LBM_BC_NEUMANN) return LBM_ERR_ARG;
        if (bc.ramp < 0 || bc.ramp > LBM_RAMP_TIME) return LBM_ERR_ARG;
        if ((bc.ramp == LBM_RAMP_LINEAR || bc.ramp == LBM_RAMP_SIN2 || bc.ramp == LBM_RAMP_COS) && !(bc.t_ramp > 0.0))
            return LBM_ERR_ARG;
        if (bc.kind == LBM_BC_DIRICHLET && !(bc.profile >= LBM_PROFILE_ZERO && bc.profile <= LBM_PROFILE_CONST))
            return LBM_ERR_ARG;
        if (bc.kind == LBM_BC_NEUMANN && !(bc.profile == LBM_PROFILE_ZERO || bc.profile == LBM_PROFILE_RADIAL ||
                                           bc.profile == LBM_PROFILE_CONST))
            return LBM_ERR_ARG;
    }
    if (!std::isfinite(opt->c_audit)) return LBM_ERR_ARG;
    // wave-speed audit of the reference state F = I: c_T^2 = lambda + 2 mu for every material
    {
        double c2 = mat->lambda + 2.0 * mat->mu;
        for (int g = 0; g < ls->ngroups; ++g) c2 = std::max(c2, ls->groups[g].material.lambda + 2.0 * ls->groups[g].material.mu);
        if (!audit_ok(opt, grid->dim, c2)) return LBM_ERR_UNSTABLE_C;
    }
    size_t need = 0;
    lbm_geometry_bytes(grid, &need);
    if (!geometry_storage || geometry_bytes < need || (reinterpret_cast<uintptr_t>(geometry_storage) % kAlign))
        return LBM_ERR_STORAGE;

    lbm_handle *h = new (std::nothrow) lbm_handle();
    if (!h) return LBM_ERR_ARG;
    h->grid = *grid;
    if (grid->dim == 2) {
        h->grid.n[2] = 1;
        h->grid.periodic[2] = 1;
        h->grid.origin[2] = 0.0;
    }
    h->opt = *opt;
    h->mat = *mat;
    h->stream = static_cast<cudaStream_t>(cuda_stream);
    h->D = grid->dim;
    h->K = h->D + h->D * h->D;
    h->Q = 2 * h->D;
    h->real_size = opt->precision == LBM_PREC_FP64 ? 8 : 4;
    h->pop_size = opt->precision == LBM_PREC_BF16S ? 2 : h->real_size;
    h->nshapes = ls->nshapes;
    for (int s = 0; s < ls->nshapes; ++s) {
        const lbm_shape &sh = ls->shapes[s];
        ShapeD &d = h->shapes[s];
        d.kind = sh.kind;
        d.complement = sh.complement != 0;
        d.bid = sh.boundary_id;
        for (int a = 0; a < 3; ++a) { d.c[a] = sh.center[a]; d.a[a] = sh.axes[a]; }
        for (int a = 0; a < 9; ++a) d.Q[a] = sh.rot[a];
        d.p = sh.p;
        set_sampled(d, sh, *grid);
    }
    h->ngroups = ls->ngroups;
    for (int g = 0; g < ls->ngroups; ++g) {
        const lbm_group &G = ls->groups[g];
        GroupD &d = h->groups[g];
        d.first = G.first_shape;
        d.count = G.nshapes;
        for (int a = 0; a < 3; ++a) { d.lo[a] = G.lo[a]; d.hi[a] = G.hi[a]; }
        if (grid->dim == 2) { d.lo[2] = -1.0; d.hi[2] = 1.0; }
        h->gmat[2 * g] = G.material.mu;
        h->gmat[2 * g + 1] = G.material.lambda;
    }
    h->nbc = nbc;
    for (int b = 0; b < nbc; ++b) {
        const lbm_bc &bc = bcs[b];
        BCD &d = h->bcs[b];
        d.bid = bc.boundary_id;
        d.kind = bc.kind;
        d.profile = bc.profile;
        d.ramp = bc.ramp;
        d.t_ramp = bc.t_ramp;
        for (int a = 0; a < 3; ++a) { d.center[a] = bc.center[a]; d.vec[a] = bc.vec[a]; }
        for (int a = 0; a < 9; ++a) d.A[a] = bc.A[a];
        d.amp = bc.amp;
        if (bc.kind == LBM_BC_NEUMANN) h->has_neumann_bc = true;
    }
    Box &bx = h->box;
    bx.D = h->D;
    bx.nx = h->grid.n[0];
    bx.ny = h->grid.n[1];
    bx.nz = h->grid.n[2];
    // a 2D body's single z plane is marked periodic in its grid, but no kernel reads a z neighbour in
    // 2D: the box keeps z non-periodic so that 2D neighbour indices take the plain-offset path
    for (int a = 0; a < 3; ++a) {
        bx.per[a] = a < h->D && h->grid.periodic[a] != 0;
        bx.origin[a] = h->grid.origin[a];
    }
    bx.dx = h->grid.dx;
    bx.nbox = (long long)bx.nx * bx.ny * bx.nz;
    // plane length: the box rounded up to 32 nodes plus one spare window, so that a 32-node window
    // starting anywhere in the box stays inside every plane
    bx.npad = (bx.nbox + 31) / 32 * 32 + 32;
    h->segs_per_row = (bx.nx + kSegAlign - 1) / kSegAlign;  // possible window starts per row
    h->nsegmax = (long long)h->segs_per_row * bx.ny * bx.nz;
    h->geo = static_cast<char *>(geometry_storage);
    carve_geometry(h, h->geo, &h->geo_bytes);

    auto fail = [&](int rc) { delete h; return rc; };
    NvtxRange range("lbm_create geometry pass");
    cudaStream_t st = h->stream;
    if (cudaMemsetAsync(h->geo, 0, h->geo_bytes, st) != cudaSuccess) return fail(LBM_ERR_CUDA);
    if (cudaMemcpyAsync(h->dshapes, h->shapes, sizeof(h->shapes), cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaMemcpyAsync(h->dbcs, h->bcs, sizeof(h->bcs), cudaMemcpyHostToDevice, st) != cudaSuccess)
        return fail(LBM_ERR_CUDA);
    if (h->ngroups > 0) {
        for (int g = 0; g < 2 * h->ngroups; ++g) h->gmat_f[g] = (float)h->gmat[g];
        if (cudaMemcpyAsync(h->dgroups, h->groups, sizeof(GroupD) * h->ngroups, cudaMemcpyHostToDevice, st) !=
                cudaSuccess ||
            cudaMemcpyAsync(h->mtab_d, h->gmat, sizeof(double) * 2 * h->ngroups, cudaMemcpyHostToDevice, st) !=
                cudaSuccess ||
            cudaMemcpyAsync(h->mtab_f, h->gmat_f, sizeof(float) * 2 * h->ngroups, cudaMemcpyHostToDevice, st) !=
                cudaSuccess)
            return fail(LBM_ERR_CUDA);
    }
    k_mask<<<grid_for(bx.nbox, 256), 256, 0, st>>>(bx, levelset_view(h), h->flags, h->gidx);
    k_cutbits<<<grid_for(bx.nbox, 256), 256, 0, st>>>(bx, levelset_view(h), h->flags, h->cnt, h->counters,
                                                       h->status);
    if (cudaGetLastError() != cudaSuccess) return fail(LBM_ERR_CUDA);
    if (scan(h->cnt, h->lstart, bx.nbox, h->scan_scratch, st)) return fail(LBM_ERR_CUDA);
    k_seg_flags<<<grid_for((long long)bx.ny * bx.nz, 128), 128, 0, st>>>(bx, h->flags, h->segs_per_row,
                                                                      (long long)bx.ny * bx.nz, h->segflag);
    if (cudaGetLastError() != cudaSuccess) return fail(LBM_ERR_CUDA);
    if (scan(h->segflag, h->segidx, h->nsegmax, h->scan_scratch, st)) return fail(LBM_ERR_CUDA);
    k_seg_write<<<grid_for(h->nsegmax, 256), 256, 0, st>>>(bx, h->segflag, h->segidx, h->segs_per_row, h->nsegmax,
                                                            h->seg);
    if (cudaGetLastError() != cudaSuccess) return fail(LBM_ERR_CUDA);
    int last[4] = {0, 0, 0, 0}, stv = 0;
    unsigned long long nact = 0;
    if (cudaMemcpyAsync(&last[0], h->lstart + (bx.nbox - 1), sizeof(int), cudaMemcpyDeviceToHost, st) ||
        cudaMemcpyAsync(&last[1], h->cnt + (bx.nbox - 1), sizeof(int), cudaMemcpyDeviceToHost, st) ||
        cudaMemcpyAsync(&last[2], h->segidx + (h->nsegmax - 1), sizeof(int), cudaMemcpyDeviceToHost, st) ||
        cudaMemcpyAsync(&last[3], h->segflag + (h->nsegmax - 1), sizeof(int), cudaMemcpyDeviceToHost, st) ||
        cudaMemcpyAsync(&nact, h->counters, sizeof(nact), cudaMemcpyDeviceToHost, st) ||
        cudaMemcpyAsync(&stv, h->status, sizeof(int), cudaMemcpyDeviceToHost, st) || cudaStreamSynchronize(st))
        return fail(LBM_ERR_CUDA);
    h->n_cut = (long long)last[0] + last[1];
    h->nseg = (long long)last[2] + last[3];
    h->n_active = (long long)nact;
    if (h->n_active == 0 || (stv & kStDomain)) return fail(LBM_ERR_DOMAIN);
    *out = h;
    return LBM_OK;
}

int lbm_storage_bytes(const lbm_handle *h, size_t *bytes) {
    if (!h || !bytes) return LBM_ERR_ARG;
    lbm_handle tmp = *h;
    tmp.events.clear();
    carve_solver(&tmp, nullptr, bytes);
    return LBM_OK;
}

int lbm_bind_storage(lbm_handle *h, void *storage, size_t bytes) {
    if (!h) return LBM_ERR_ARG;
    size_t need = 0;
    lbm_storage_bytes(h, &need);
    if (!storage || bytes < need || (reinterpret_cast<uintptr_t>(storage) % kAlign)) return LBM_ERR_STORAGE;
    h->sto = static_cast<char *>(storage);
    carve_solver(h, h->sto, &h->sto_bytes);
    cudaStream_t st = h->stream;
    // zero everything except the large LSQ tables, which are written before use
    CK(cudaMemsetAsync(h->sto, 0, h->sto_bytes, st));
    int rc = ops(h).link_build(h);
    if (rc) return rc;
    int stv = 0;
    CK(cudaMemcpyAsync(&stv, h->status, sizeof(int), cudaMemcpyDeviceToHost, st));
    std::vector<int> bc(h->n_cut), ns(h->n_cut);
    if (h->n_cut) {
        CK(cudaMemcpyAsync(bc.data(), h->l_bc, h->n_cut * sizeof(int), cudaMemcpyDeviceToHost, st));
        CK(cudaMemcpyAsync(ns.data(), h->l_ns, h->n_cut * sizeof(int), cudaMemcpyDeviceToHost, st));
    }
    CK(cudaStreamSynchronize(st));
    if (stv & kStNoBC) return LBM_ERR_ARG;
    if (stv & kStCapacity) return LBM_ERR_CAPACITY;
    h->n_neu = h->n_dir = h->lsq_entries = 0;
    for (long long l = 0; l < h->n_cut; ++l) {
        if (h->bcs[bc[l]].kind == LBM_BC_NEUMANN) { h->n_neu++; h->lsq_entries += ns[l]; }
        else h->n_dir++;
    }
    h->bound = true;
    h->initialized = false;
    return LBM_OK;
}

int lbm_set_initial(lbm_handle *h, int mode, const double *v0, const double *F0, const double *u0, const double *dU0) {
    if (!h) return LBM_ERR_ARG;
    if (!h->bound) return LBM_ERR_STATE;
    if (!v0 || !F0 || !u0 || (mode != LBM_INIT_EQUILIBRIUM && mode != LBM_INIT_CHARACTERISTIC)) return LBM_ERR_ARG;
    const int D = h->D, K = h->K;
    const long long N = h->box.nbox;
    const double *pv = v0, *pF = F0, *pu = u0, *pd = dU0;
    if (!is_device_ptr(v0) || !is_device_ptr(F0) || !is_device_ptr(u0) || (dU0 && !is_device_ptr(dU0))) {
        if (!h->staging) return LBM_ERR_ARG;
        double *s = h->staging;
        auto stage = [&](const double *src, double *dst, size_t n) {
            return cudaMemcpyAsync(dst, src, n * sizeof(double), cudaMemcpyDefault, h->stream);
        };
        pv = s;
        pF = s + (size_t)D * N;
        pu = s + (size_t)(D + D * D) * N;
        pd = dU0 ? s + (size_t)(2 * D + D * D) * N : nullptr;
        CK(stage(v0, const_cast<double *>(pv), (size_t)D * N));
        CK(stage(F0, const_cast<double *>(pF), (size_t)D * D * N));
        CK(stage(u0, const_cast<double *>(pu), (size_t)D * N));
        if (dU0) CK(stage(dU0, const_cast<double *>(pd), (size_t)D * K * N));
    }
    if (h->opt.c_audit >= 0.0) {  // wave-speed audit of the initial F0 over the active nodes
        const unsigned gr = (unsigned)std::max<long long>(1, std::min<long long>(grid_for(h->nseg, 4), kReduceBlocks));
        const uint8_t *mt = h->ngroups > 0 ? h->gidx : nullptr;
        const double *mtab = h->ngroups > 0 ? h->mtab_d : nullptr;
        if (h->D == 2) {
            if (h->real_size == 8)
                k_audit_f0<2, double><<<gr, 128, 0, h->stream>>>(h->box, h->seg, (int)h->nseg, h->flags, pF, h->mat.mu, h->mat.lambda, mt, mtab,
                                                                 h->mu_field_on ? static_cast<const double *>(h->mu_field) : nullptr, h->diag);
            else
                k_audit_f0<2, float><<<gr, 128, 0, h->stream>>>(h->box, h->seg, (int)h->nseg, h->flags, pF, h->mat.mu, h->mat.lambda, mt, mtab,
                                                                h->mu_field_on ? static_cast<const float *>(h->mu_field) : nullptr, h->diag);
        } else {
            if (h->real_size == 8)
                k_audit_f0<3, double><<<gr, 128, 0, h->stream>>>(h->box, h->seg, (int)h->nseg, h->flags, pF, h->mat.mu, h->mat.lambda, mt, mtab,
                                                                 h->mu_field_on ? static_cast<const double *>(h->mu_field) : nullptr, h->diag);
            else
                k_audit_f0<3, float><<<gr, 128, 0, h->stream>>>(h->box, h->seg, (int)h->nseg, h->flags, pF, h->mat.mu, h->mat.lambda, mt, mtab,
                                                                h->mu_field_on ? static_cast<const float *>(h->mu_field) : nullptr, h->diag);
        }
        CKL();
        std::vector<double> part(gr);
        CK(cudaMemcpyAsync(part.data(), h->diag, gr * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
        CK(cudaStreamSynchronize(h->stream));
        double c2 = 0.0;
        for (double x : part) c2 = std::isnan(x) ? x : std::max(c2, x);
        if (!audit_ok(&h->opt, h->D, c2)) return LBM_ERR_UNSTABLE_C;
    }
    int rc = ops(h).init(h, mode, pv, pF, pu, pd);
    if (rc) return rc;
    h->phase = 0;
    h->step = 0;
    h->initialized = true;
    return LBM_OK;
}

int lbm_step(lbm_handle *h, int nsteps) {
    if (!h || nsteps < 0) return LBM_ERR_ARG;
    if (!h->initialized) return LBM_ERR_STATE;
    return ops(h).step(h, nsteps);
}

int lbm_step_graph(lbm_handle *h, int nsteps) {
    if (!h || nsteps < 0) return LBM_ERR_ARG;
    if (!h->initialized || h->timing) return LBM_ERR_STATE;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    CK(cudaStreamIsCapturing(h->stream, &cs));
    if (cs != cudaStreamCaptureStatusNone) return LBM_ERR_STATE;
    if (h->graph_exec) {  // the previous graph was launched on this stream; its work is ordered before ours
        cudaGraphExecDestroy(h->graph_exec);
        h->graph_exec = nullptr;
    }
    // Record on a private non-blocking stream (the caller's may be the legacy default stream,
    // which cannot be captured); recording executes nothing, and the graph is then launched on
    // the caller's stream after its earlier work.
    if (!h->capture_stream) CK(cudaStreamCreateWithFlags(&h->capture_stream, cudaStreamNonBlocking));
    const cudaStream_t caller = h->stream;
    h->stream = h->capture_stream;
    if (cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
        h->stream = caller;
        cudaGetLastError();
        return LBM_ERR_CUDA;
    }
    const int rc = ops(h).step(h, nsteps);
    cudaGraph_t graph = nullptr;
    const cudaError_t ec = cudaStreamEndCapture(h->stream, &graph);
    h->stream = caller;
    if (rc != LBM_OK || ec != cudaSuccess || !graph) {
        if (graph) cudaGraphDestroy(graph);
        cudaGetLastError();
        return rc != LBM_OK ? rc : LBM_ERR_CUDA;
    }
    cudaGraphExec_t exec = nullptr;
    const cudaError_t ei = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    if (ei != cudaSuccess) {
        cudaGetLastError();
        return LBM_ERR_CUDA;
    }
    h->graph_exec = exec;
    CK(cudaGraphLaunch(exec, h->stream));
    return LBM_OK;
}

// ---- tile shapes and the autotuner ----------------------------------------------------------

static bool one_of(int v, int a, int b, int c) { return v == 0 || v == a || v == b || v == c; }

int lbm_set_tuning(lbm_handle *h, const lbm_tuning *t) {
    if (!h || !t) return LBM_ERR_ARG;
    if (!one_of(t->windows_per_warp, 1, 2, 4) || !one_of(t->jacobi_segments, 1, 2, 4) ||
        !one_of(t->link_block, 64, 128, 256) || !one_of(t->jacobi_sweeps, 1, 2, 0))
        return LBM_ERR_ARG;
    h->tune_nw = t->windows_per_warp;
    h->tune_jseg = t->jacobi_segments;
    h->tune_lblock = t->link_block;
    h->tune_jsweeps = t->jacobi_sweeps;
    return LBM_OK;
}

int lbm_get_tuning(const lbm_handle *h, lbm_tuning *t) {
    if (!h || !t) return LBM_ERR_ARG;
    std::memset(t, 0, sizeof(*t));
    t->windows_per_warp = h->tma_ok ? (h->tune_nw ? h->tune_nw : (h->pop_size == 2 ? 2 : 1)) : 0;
    t->jacobi_segments = h->tune_jseg ? h->tune_jseg : 1;
    t->link_block = h->tune_lblock ? h->tune_lblock : 128;
    t->jacobi_sweeps = (h->jp_ok && (h->tune_jsweeps ? h->tune_jsweeps == 2 : h->D == 2)) ? 2 : 1;
    return LBM_OK;
}

// restores the saved state, takes one untimed step with the current shapes, then times `steps`
// steps on the handle's stream; a latched device status ends the tuning
static int time_shapes(lbm_handle *h, int steps, void *scratch, double *ms_per_step) {
    int rc = lbm_load_state(h, scratch);
    if (rc) return rc;
    rc = ops(h).step(h, 1);
    if (rc) return rc;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    CK(cudaEventCreate(&e0));
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return LBM_ERR_CUDA;
    }
    cudaEventRecord(e0, h->stream);
    rc = ops(h).step(h, steps);
    cudaEventRecord(e1, h->stream);
    float ms = 0.0f;
    const bool ok = cudaEventSynchronize(e1) == cudaSuccess && cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc) return rc;
    if (!ok) return LBM_ERR_CUDA;
    rc = lbm_sync(h, nullptr);
    if (rc) return rc;
    *ms_per_step = (double)ms / steps;
    return LBM_OK;
}

int lbm_autotune(lbm_handle *h, int steps, void *scratch, lbm_tuning *out) {
    if (!h || steps < 1 || !scratch || (reinterpret_cast<uintptr_t>(scratch) % kAlign)) return LBM_ERR_ARG;
    NvtxRange range("lbm_autotune");
    if (!h->initialized || h->timing || (h->opt.adjoint && h->adj_next >= 0)) return LBM_ERR_STATE;
    int rc = lbm_save_state(h, scratch);
    if (rc) return rc;
    constexpr int NC = 4;
    int *const shape[NC] = {&h->tune_nw, &h->tune_jseg, &h->tune_jsweeps, &h->tune_lblock};
    const int saved[NC] = {h->tune_nw, h->tune_jseg, h->tune_jsweeps, h->tune_lblock};
    const int cand[NC][3] = {{1, 2, 4}, {1, 2, 4}, {2, 1, 0}, {64, 128, 256}};
    const int dflt[NC] = {h->pop_size == 2 ? 2 : 1, 1, h->D == 2 ? 2 : 1, 128};
    const bool proj = h->n_neu > 0 && h->opt.proj_every > 0;
    const bool used[NC] = {h->tma_ok, proj, proj && h->jp_ok, h->n_cut > 0};
    for (int c = 0; c < NC; ++c) *shape[c] = 0;
    double best = 0.0;
    int count = 0;
    rc = time_shapes(h, steps, scratch, &best);
    count++;
    const double def_ms = best;
    // coordinate by coordinate; a candidate must beat the best by 1 % to replace it
    for (int c = 0; c < NC && rc == LBM_OK; ++c) {
        if (!used[c]) continue;
        int chosen = 0;
        for (int i = 0; i < 3 && rc == LBM_OK; ++i) {
            if (cand[c][i] == dflt[c] || cand[c][i] == 0) continue;
            *shape[c] = cand[c][i];
            double ms = 0.0;
            rc = time_shapes(h, steps, scratch, &ms);
            count++;
            if (rc == LBM_OK && ms < 0.99 * best) {
                best = ms;
                chosen = cand[c][i];
            }
        }
        *shape[c] = chosen;
    }
    const int rl = lbm_load_state(h, scratch);
    if (rc != LBM_OK) {
        for (int c = 0; c < NC; ++c) *shape[c] = saved[c];
        return rc;
    }
    if (rl) return rl;
    if (out) {
        lbm_get_tuning(h, out);
        out->candidates = count;
        out->ms_per_step = best;
        out->default_ms_per_step = def_ms;
    }
    return LBM_OK;
}

int lbm_set_wait_limit(lbm_handle *h, int polls) {
    if (!h) return LBM_ERR_ARG;
    h->wait_limit = polls < 0 ? -1 : polls;
    return LBM_OK;
}

int lbm_set_mu_field(lbm_handle *h, const double *mu) {
    if (!h || !mu) return LBM_ERR_ARG;
    if (!h->bound || !h->opt.adjoint) return LBM_ERR_STATE;
    const size_t n = (size_t)h->box.nbox;
    // stage the FP64 field in the first gradient buffer (n doubles fit in its Q*K*npad values),
    // then convert into the field in the population precision
    double *tmp = reinterpret_cast<double *>(h->adj_g[0]);
    CK(cudaMemcpyAsync(tmp, mu, n * sizeof(double), is_device_ptr(mu) ? cudaMemcpyDeviceToDevice
                                                                      : cudaMemcpyHostToDevice, h->stream));
    CK(convert_field(tmp, h->mu_field, n, h->real_size, h->stream));
    h->mu_field_on = true;
    return LBM_OK;
}

int lbm_set_body_force(lbm_handle *h, const double *b) {
    if (!h || !b) return LBM_ERR_ARG;
    for (int i = 0; i < 3; ++i) {
        if (!std::isfinite(b[i])) return LBM_ERR_ARG;
        h->opt.body_force[i] = i < h->D ? b[i] : 0.0;
    }
    return LBM_OK;
}

int lbm_state_bytes(const lbm_handle *h, size_t *bytes) {
    if (!h || !bytes) return LBM_ERR_ARG;
    *bytes = state_layout(h).bytes;
    return LBM_OK;
}

static __global__ void k_state_header(long long *dst, long long step, long long phase) {
    dst[0] = step;
    dst[1] = phase;
}

int lbm_save_state(lbm_handle *h, void *dst) {
    if (!h || !dst || (reinterpret_cast<uintptr_t>(dst) % kAlign)) return LBM_ERR_ARG;
    if (!h->initialized) return LBM_ERR_STATE;
    const StateLayout L = state_layout(h);
    char *d = static_cast<char *>(dst);
    const size_t np = (size_t)h->box.npad, nc = (size_t)h->n_cut;
    const int D = h->D, K = h->K, Q = h->Q, rs = h->real_size;
    cudaStream_t st = h->stream;
    k_state_header<<<1, 1, 0, st>>>(reinterpret_cast<long long *>(d), h->step, h->phase);
    CKL();
    CK(cudaMemcpyAsync(d + L.pop, h->fA, (size_t)Q * K * np * h->pop_size, cudaMemcpyDeviceToDevice, st));
    CK(cudaMemcpyAsync(d + L.ustar, h->ustar, (size_t)D * np * 8, cudaMemcpyDeviceToDevice, st));
    CK(cudaMemcpyAsync(d + L.un, h->un, (size_t)(D == 3 ? 32 : 16) * np, cudaMemcpyDeviceToDevice, st));
    if (nc) {
        CK(cudaMemcpyAsync(d + L.rec, h->l_rec, (size_t)K * nc * rs, cudaMemcpyDeviceToDevice, st));
        CK(cudaMemcpyAsync(d + L.lh, h->l_h, (size_t)3 * nc * rs, cudaMemcpyDeviceToDevice, st));
    }
    return LBM_OK;
}

int lbm_load_state(lbm_handle *h, const void *src) {
    if (!h || !src || (reinterpret_cast<uintptr_t>(src) % kAlign)) return LBM_ERR_ARG;
    if (!h->bound) return LBM_ERR_STATE;
    const StateLayout L = state_layout(h);
    const char *s = static_cast<const char *>(src);
    const size_t np = (size_t)h->box.npad, nc = (size_t)h->n_cut;
    const int D = h->D, K = h->K, Q = h->Q, rs = h->real_size;
    long long hdr[2] = {0, 0};
    cudaStream_t st = h->stream;
    CK(cudaMemcpyAsync(hdr, s, sizeof(hdr), cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(h->fA, s + L.pop, (size_t)Q * K * np * h->pop_size, cudaMemcpyDeviceToDevice, st));
    CK(cudaMemcpyAsync(h->ustar, s + L.ustar, (size_t)D * np * 8, cudaMemcpyDeviceToDevice, st));
    CK(cudaMemcpyAsync(h->un, s + L.un, (size_t)(D == 3 ? 32 : 16) * np, cudaMemcpyDeviceToDevice, st));
    if (nc) {
        CK(cudaMemcpyAsync(h->l_rec, s + L.rec, (size_t)K * nc * rs, cudaMemcpyDeviceToDevice, st));
        CK(cudaMemcpyAsync(h->l_h, s + L.lh, (size_t)3 * nc * rs, cudaMemcpyDeviceToDevice, st));
    }
    CK(cudaStreamSynchronize(st));
    if (hdr[0] < 0 || (hdr[1] != 0 && hdr[1] != 1)) return LBM_ERR_ARG;
    h->step = hdr[0];
    h->phase = (int)hdr[1];
    h->initialized = true;
    return LBM_OK;
}

int lbm_moments_bytes(const lbm_handle *h, size_t *bytes) {
    if (!h || !bytes) return LBM_ERR_ARG;
    *bytes = (size_t)h->D * h->D * h->box.npad * h->real_size;
    return LBM_OK;
}

int lbm_step_moments(lbm_handle *h, void *dst) {
    if (!h || !dst || (reinterpret_cast<uintptr_t>(dst) % kAlign)) return LBM_ERR_ARG;
    if (!h->initialized || h->n_neu > 0) return LBM_ERR_STATE;
    h->mom_out = dst;
    const int rc = ops(h).step(h, 1);
    h->mom_out = nullptr;
    return rc;
}

int lbm_adjoint_begin(lbm_handle *h, const double *grad_u) {
    if (!h || !grad_u) return LBM_ERR_ARG;
    if (!h->initialized || !h->opt.adjoint || h->n_neu > 0 || h->step < 1) return LBM_ERR_STATE;
    return ops(h).adjoint_begin(h, grad_u);
}

int lbm_adjoint_step(lbm_handle *h, const void *moments) {
    if (!h || !moments || (reinterpret_cast<uintptr_t>(moments) % kAlign)) return LBM_ERR_ARG;
    if (!h->opt.adjoint || h->adj_next < 0) return LBM_ERR_STATE;
    return ops(h).adjoint_step(h, moments);
}

int lbm_adjoint_gradients(lbm_handle *h, double *grad_mu, double *grad_b) {
    if (!h) return LBM_ERR_ARG;
    if (!h->opt.adjoint) return LBM_ERR_STATE;
    cudaStream_t st = h->stream;
    if (grad_mu) CK(gather_box(h->adj_mubar, grad_mu, h->box.nbox, st));
    // dL/db: the sum of the windows' slots
    std::vector<double> slots((size_t)4 * tlv::kAdjSlots);
    CK(cudaMemcpyAsync(slots.data(), h->adj_bslot, slots.size() * sizeof(double), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    if (grad_b)
        for (int i = 0; i < 3; ++i) {
            double b = 0.0;
            for (int s = 0; s < tlv::kAdjSlots; ++s) b += slots[(size_t)4 * s + i];
            grad_b[i] = b;
        }
    return LBM_OK;
}

int lbm_fields_ex(lbm_handle *h, double *v, double *F, double *u, double *sigma, double *J, int layout) {
    if (!h || (layout != LBM_LAYOUT_PLANES && layout != LBM_LAYOUT_NODES)) return LBM_ERR_ARG;
    if (!h->initialized) return LBM_ERR_STATE;
    const int D = h->D;
    const long long N = h->box.nbox;
    double *ptr[5] = {v, F, u, sigma, J};
    const size_t cnt[5] = {(size_t)D * N, (size_t)D * D * N, (size_t)D * N, (size_t)D * D * N, (size_t)N};
    double *dev[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
    bool host[5] = {false, false, false, false, false};
    size_t off = 0;  // staging holds (2D + D^2 + D K) n_box values, more than the 2D + 2D^2 + 1 used here
    for (int j = 0; j < 5; ++j) {
        if (!ptr[j]) continue;
        if (is_device_ptr(ptr[j])) {
            dev[j] = ptr[j];
        } else {
            if (!h->staging) return LBM_ERR_ARG;
            dev[j] = h->staging + off;
            host[j] = true;
            off += cnt[j];
        }
        CK(cudaMemsetAsync(dev[j], 0, cnt[j] * sizeof(double), h->stream));
    }
    FieldOut o;
    o.v = dev[0];
    o.F = dev[1];
    o.u = dev[2];
    o.sigma = dev[3];
    o.J = dev[4];
    o.layout = layout;
    int rc = ops(h).fields(h, o);
    if (rc) return rc;
    for (int j = 0; j < 5; ++j)
        if (host[j]) CK(cudaMemcpyAsync(ptr[j], dev[j], cnt[j] * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    return LBM_OK;
}

int lbm_fields(lbm_handle *h, double *v, double *F, double *u) {
    return lbm_fields_ex(h, v, F, u, nullptr, nullptr, LBM_LAYOUT_PLANES);
}

int lbm_diagnostics(lbm_handle *h, lbm_diag *out) {
    if (!h || !out) return LBM_ERR_ARG;
    if (!h->initialized) return LBM_ERR_STATE;
    int rc = ops(h).diagnostics(h);
    if (rc) return rc;
    double r[kDiagRec];
    CK(cudaMemcpyAsync(r, h->diag + (size_t)kReduceBlocks * kDiagRec, sizeof(r), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    std::memset(out, 0, sizeof(*out));
    out->n_active = h->n_active;
    out->J_min = r[2];
    out->J_max = r[3];
    out->v_rms = std::sqrt(r[0] / (double)h->n_active);
    out->v_max = std::sqrt(r[1]);
    out->c_tangent = std::sqrt(r[4]);
    out->n_edges = (long long)r[6];
    out->incompat_rms = r[6] > 0.0 ? std::sqrt(r[5] / r[6]) : 0.0;
    out->step = h->step;
    out->t = h->step * (h->grid.dx / h->opt.c);
    return LBM_OK;
}

int lbm_sync(lbm_handle *h, int *device_status) {
    if (!h) return LBM_ERR_ARG;
    int stv = 0;
    CK(cudaMemcpyAsync(&stv, h->status, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    if (device_status) *device_status = stv & (31 | kStTimeout | kStBounds);
    if (stv & (31 | kStTimeout | kStBounds)) {
        CK(cudaMemsetAsync(h->status, 0, sizeof(int), h->stream));
        CK(cudaStreamSynchronize(h->stream));
        return LBM_ERR_DEVICE;
    }
    return LBM_OK;
}

int lbm_get_info(const lbm_handle *h, lbm_info *info) {
    if (!h || !info) return LBM_ERR_ARG;
    std::memset(info, 0, sizeof(*info));
    info->n_box = h->box.nbox;
    info->n_active = h->n_active;
    info->n_cut = h->n_cut;
    info->n_neumann = h->n_neu;
    info->n_dirichlet = h->n_dir;
    info->n_segments = h->nseg;
    info->step = h->step;
    info->dt = h->grid.dx / h->opt.c;
    info->t = h->step * info->dt;
    info->geometry_bytes = h->geo_bytes;
    size_t sb = 0;
    lbm_storage_bytes(h, &sb);
    info->storage_bytes = sb;
    info->launches = h->launches;
    info->lsq_entries = h->lsq_entries;
    return LBM_OK;
}

int lbm_enable_timing(lbm_handle *h, int enable) {
    if (!h) return LBM_ERR_ARG;
    timing_fold(h);
    h->timing = enable != 0;
    for (int i = 0; i < 4; ++i) { h->acc_ms[i] = 0.0; h->acc_n[i] = 0; }
    return LBM_OK;
}

int lbm_kernel_times(lbm_handle *h, lbm_kernel_time *out) {
    if (!h || !out) return LBM_ERR_ARG;
    timing_fold(h);
    out->stream_collide_ms = h->acc_ms[0];
    out->cutlink_ms = h->acc_ms[1];
    out->projection_ms = h->acc_ms[2];
    out->stream_collide_launches = h->acc_n[0];
    out->cutlink_launches = h->acc_n[1];
    out->projection_launches = h->acc_n[2];
    out->jacobi_ms = h->acc_ms[3];
    out->jacobi_launches = h->acc_n[3];
    return LBM_OK;
}

int lbm_copy_links(lbm_handle *h, long long *node, int *q, double *eta, double *Xb, double *Nb, int *bid, int *ns) {
    if (!h) return LBM_ERR_ARG;
    if (!h->bound) return LBM_ERR_STATE;
    const long long n = h->n_cut;
    if (n == 0) return LBM_OK;
    std::vector<int> nd(n), bc(n);
    cudaStream_t st = h->stream;
    CK(cudaMemcpyAsync(nd.data(), h->l_node, n * sizeof(int), cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(bc.data(), h->l_bc, n * sizeof(int), cudaMemcpyDeviceToHost, st));
    if (q) CK(cudaMemcpyAsync(q, h->l_q, n * sizeof(int), cudaMemcpyDeviceToHost, st));
    if (eta) CK(cudaMemcpyAsync(eta, h->l_eta, n * sizeof(double), cudaMemcpyDeviceToHost, st));
    if (Xb) CK(cudaMemcpyAsync(Xb, h->l_Xb, 3 * n * sizeof(double), cudaMemcpyDeviceToHost, st));
    if (Nb) CK(cudaMemcpyAsync(Nb, h->l_Nb, 3 * n * sizeof(double), cudaMemcpyDeviceToHost, st));
    if (ns) CK(cudaMemcpyAsync(ns, h->l_ns, n * sizeof(int), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    for (long long l = 0; l < n; ++l) {
        if (node) node[l] = nd[l];
        if (bid) bid[l] = h->bcs[bc[l]].bid;
    }
    return LBM_OK;
}

int lbm_copy_active(lbm_handle *h, unsigned char *mask) {
    if (!h || !mask) return LBM_ERR_ARG;
    const long long N = h->box.nbox;
    std::vector<uint8_t> fl(N);
    CK(cudaMemcpyAsync(fl.data(), h->flags, N, cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    for (long long i = 0; i < N; ++i) mask[i] = (fl[i] & kActive) ? 1 : 0;
    return LBM_OK;
}

void lbm_destroy(lbm_handle *h) {
    if (!h) return;
    timing_fold(h);
    if (h->graph_exec) {
        cudaStreamSynchronize(h->stream);
        cudaGraphExecDestroy(h->graph_exec);
    }
    if (h->capture_stream) cudaStreamDestroy(h->capture_stream);
    delete h;
}

}  // extern "C"
