// Tensor-core (tcgen05) sigma for KPM_MIXED contexts.
#pragma once
#include "common.cuh"

namespace kpm {

struct TcSigma {
    void init(const SpinTables& ta, const SpinTables& tb, const double* h1_host,
              const double* eri_host, int n, cudaStream_t st);
    void apply(const float* x, float* y, int ncol, cudaStream_t st);
};

}  // namespace kpm
