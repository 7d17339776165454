// BF16-storage instantiation of the update: FP32 arithmetic (the FP32 form's kernels) with the
// shifted populations stored as BF16 (see lbm_impl.cuh).  The reverse mode is not offered in this
// form (lbm_create refuses options.adjoint with it).
#include <cuda_bf16.h>

#include "lbm_ops.cuh"

namespace {
using pop_t = __nv_bfloat16;
template <int D> using ImplB = Impl<float, D, pop_t>;

int link_build_any(lbm_handle *h) { return h->D == 2 ? ImplB<2>::link_build(h) : ImplB<3>::link_build(h); }
int init_any(lbm_handle *h, int m, const double *v, const double *F, const double *u, const double *d) {
    return h->D == 2 ? ImplB<2>::init(h, m, v, F, u, d) : ImplB<3>::init(h, m, v, F, u, d);
}
int step_any(lbm_handle *h, int n) { return h->D == 2 ? ImplB<2>::step(h, n) : ImplB<3>::step(h, n); }
int fields_any(lbm_handle *h, const FieldOut &o) { return h->D == 2 ? ImplB<2>::fields(h, o) : ImplB<3>::fields(h, o); }
int diagnostics_any(lbm_handle *h) { return h->D == 2 ? ImplB<2>::diagnostics(h) : ImplB<3>::diagnostics(h); }
int adjoint_begin_none(lbm_handle *, const double *) { return LBM_ERR_STATE; }
int adjoint_step_none(lbm_handle *, const void *) { return LBM_ERR_STATE; }
}  // namespace

const PrecOps &ops_bf16s() {
    static const PrecOps ops = {link_build_any, init_any, step_any, fields_any, diagnostics_any,
                                   adjoint_begin_none, adjoint_step_none};
    return ops;
}
