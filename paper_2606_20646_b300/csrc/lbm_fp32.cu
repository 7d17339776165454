// FP32 instantiation of the update (see lbm_impl.cuh).
#include "lbm_ops.cuh"

namespace {
template <int D> int link_build(lbm_handle *h) { return Impl<float, D>::link_build(h); }
template <int D> int init(lbm_handle *h, int m, const double *v, const double *F, const double *u, const double *d) {
    return Impl<float, D>::init(h, m, v, F, u, d);
}
template <int D> int step(lbm_handle *h, int n) { return Impl<float, D>::step(h, n); }
template <int D> int fields(lbm_handle *h, const FieldOut &o) { return Impl<float, D>::fields(h, o); }

int link_build_any(lbm_handle *h) { return h->D == 2 ? link_build<2>(h) : link_build<3>(h); }
int init_any(lbm_handle *h, int m, const double *v, const double *F, const double *u, const double *d) {
    return h->D == 2 ? init<2>(h, m, v, F, u, d) : init<3>(h, m, v, F, u, d);
}
int step_any(lbm_handle *h, int n) { return h->D == 2 ? step<2>(h, n) : step<3>(h, n); }
int fields_any(lbm_handle *h, const FieldOut &o) { return h->D == 2 ? fields<2>(h, o) : fields<3>(h, o); }
int diagnostics_any(lbm_handle *h) {
    return h->D == 2 ? Impl<float, 2>::diagnostics(h) : Impl<float, 3>::diagnostics(h);
}
int adjoint_begin_any(lbm_handle *h, const double *gu) {
    return h->D == 2 ? Impl<float, 2>::adjoint_begin(h, gu) : Impl<float, 3>::adjoint_begin(h, gu);
}
int adjoint_step_any(lbm_handle *h, const void *pop) {
    return h->D == 2 ? Impl<float, 2>::adjoint_step(h, pop) : Impl<float, 3>::adjoint_step(h, pop);
}
}  // namespace

const PrecOps &ops_fp32() {
    static const PrecOps ops = {link_build_any, init_any, step_any, fields_any, diagnostics_any,
                                   adjoint_begin_any, adjoint_step_any};
    return ops;
}
