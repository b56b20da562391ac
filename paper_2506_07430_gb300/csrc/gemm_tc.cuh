// Dense same-spin products on tcgen05 tensor cores (see gemm_tc.cu).
#pragma once
#include "common.cuh"

namespace kpm {

// Row pitch (elements) of an FP16 matrix with `cols` columns: 16-byte rows.
int64_t half_pitch(int64_t cols);

// sigma += F_b-part + F_a-part of H applied to x (FP32 [N_a][N_b]); see gemm_tc.cu.
struct DenseSS {
    int64_t na = 0, nb = 0, pa = 0, pb = 0;   // strings and FP16 row pitches per spin
    double wscale_a = 1.0, wscale_b = 1.0;    // power-of-two scales of the split matrices
    DevBuf fa_hi_own, fa_lo_own, da_own;      // alpha matrices (own copy if N_a != N_b)
    DevBuf fb_hi, fb_lo, db;                  // beta matrices, diagonal of F_b (float hi/lo)
    DevBuf* fa_hi = nullptr;
    DevBuf* fa_lo = nullptr;
    DevBuf* da = nullptr;
    int64_t xpitch = 0;                       // row pitch of xh/xl: N_b rounded up to 128
    DevBuf xh, xl, th, tl;                    // split copies of x and x^T
    DevBuf fmax;                              // scratch for max |F_off|
    // per tile of the split matrix, the k-blocks that hold a nonzero (CSR; see
    // block_lists): beta GEMM (F_b, 128-row tiles), alpha GEMM (F_a, 256-row tiles)
    DevBuf kbs_b, kbl_b, kbs_a, kbl_a;
    int64_t kb_nonzero[2] = {0, 0}, kb_total[2] = {0, 0};
    size_t smem = 0;
    int* err = nullptr;
    // exact diagonal H_II of the whole H (same-spin diagonals and the opposite-spin
    // Coulomb sum, FP64 stored as float hi + lo, [N_a][N_b]), added by the alpha
    // product's epilogue; the split matrices and the row pass leave it out
    const float2* diag_full = nullptr;

    // Builds the split matrices; `same`: alpha and beta strings are identical.
    void init(const SpinTables& A, const SpinTables& B, bool same, int* err_flag,
              cudaStream_t st);
    // xh/xl = x split into scaled FP16 pieces [N_a][xpitch] (zero padding).
    void split(const float* x, const float* amax, cudaStream_t st);
    // y += (F_a (x) 1 + 1 (x) F_b) x with the off-diagonal parts of F_a, F_b, plus
    // diag_full * x (the whole exact diagonal of H); amax = device max|x|.
    // Uses xh/xl from split(x) on the same stream.
    void apply(const float* x, float* y, const float* amax, cudaStream_t st);
    // Rasterisation group (row tiles per group) of the beta and alpha GEMMs, chosen
    // by autotune() at set-up; 16 by default.
    int group_m[2] = {16, 16};
    void autotune(cudaStream_t st);
    void launch_beta(float* y, const float* amax, int group, cudaStream_t st);
    void launch_alpha(const float* x, float* y, const float* amax, int group, cudaStream_t st);
};

}  // namespace kpm
