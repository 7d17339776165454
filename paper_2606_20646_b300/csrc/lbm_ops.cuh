// Entry points of one precision: defined in lbm_fp64.cu (built with -fmad=false so its
// arithmetic matches the FP64 oracle operation for operation), lbm_fp32.cu and lbm_bf16s.cu (FP32
// arithmetic, BF16 population storage).
#pragma once
#include "lbm_impl.cuh"

struct PrecOps {
    int (*link_build)(lbm_handle *);
    int (*init)(lbm_handle *, int, const double *, const double *, const double *, const double *);
    int (*step)(lbm_handle *, int);
    int (*fields)(lbm_handle *, const FieldOut &);
    int (*diagnostics)(lbm_handle *);
    int (*adjoint_begin)(lbm_handle *, const double *);
    int (*adjoint_step)(lbm_handle *, const void *);
};

const PrecOps &ops_fp64();
const PrecOps &ops_fp32();
const PrecOps &ops_bf16s();
