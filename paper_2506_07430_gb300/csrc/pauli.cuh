// Jordan-Wigner Pauli-string form of H (see pauli.cu).
#pragma once
#include "common.cuh"

namespace kpm {

struct PauliH {
    int n = 0, na = 0, nb = 0;
    int64_t nterms = 0;   // distinct Pauli strings X^x Z^z with nonzero coefficient
    int ngroups = 0;      // distinct flip masks x
    bool built = false;
    DevBuf gx, gstart, tz, tc;   // per group: x mask, first term; per term: z mask, coefficient
    // Expands H (h1 [n*n], eri [n^4] chemist, host FP64) into Pauli strings.
    void build(const double* h1, const double* eri, int norb, int nalpha, int nbeta);
    // y = H x over the (nalpha, nbeta) sector, ncol columns, FP64 sums.
    void apply(const SpinTables& A, const SpinTables& B, const void* x, void* y, int ncol,
               bool f64, cudaStream_t st) const;
};

}  // namespace kpm
