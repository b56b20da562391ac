// Tensor-core (tcgen05) sigma for KPM_MIXED contexts.
#pragma once
#include "common.cuh"
#include "gemm_tc.cuh"

#include <vector>

namespace kpm {

// sigma = H x with the two-electron terms contracted on the 5th-generation
// tensor cores.  See sigma_tc.cu for the formulation.
struct TcSigma {
    int n = 0, NS = 0, P = 0;     // orbitals, unordered pairs n(n+1)/2, padded N (output slots)
    int KR = 0;                   // K of the row GEMM: noff + ndiag rounded up to 16
    int64_t nsa = 0, nsb = 0, dim = 0;
    int nsm = 0;                  // SMs of the device (persistent grid)
    bool fp16 = false;            // operand format: split FP16 (scaled) or split BF16
    int nw = 3;                   // 16-bit pieces of W
    float wscale = 1.0f;          // power-of-two scale of W in the image
    void* kernel = nullptr;       // k_rowpass instantiation for P
    const SpinTables* ta = nullptr;
    const SpinTables* tb = nullptr;
    DevBuf wimg;                  // W = (pq|rs) over slot pairs, split into 16-bit pieces
    int noff = 0;                 // off-diagonal table entries per alpha string, m (n - m)
    int ndiag = 0;                // 1: one K column for the diagonal entries (m >= 1)
    DevBuf rslot_a;               // uint16 [N_a][noff] off-diagonal entry -> slot | sign << 15
    DevBuf rtgt_a;                // int32  [N_a][noff] off-diagonal entry -> target string
    DevBuf wdiag;                 // double [n][P] W[qq][s] (diagonal slots zero)
    DevBuf xbh, xbl;              // BF16 pieces of x (KPM_MIXED_BF16; FP16 pieces live in dense)
    DevBuf slot_b;                // uint16 [P/8][N_b][8] pair-slot -> target | sign << 15 (N_b: none)
    DenseSS dense;                // same-spin parts (dense GEMMs with F_a, F_b)
    DevBuf err;                   // int error flag (1: a bounded wait ran out)
    DevBuf amax;                  // max |x| (float bits): operand scale, fixed-point range
    DevBuf rowmax;                // [N_a] max |x| per row: per-row fixed-point range of the row pass
    int nst = 2;                  // A stages of the row pass (at most 3, where shared memory
                                  // allows; autotuned)
    int rp_prefetch = 4;          // L2 prefetch distance of the row pass, tiles (autotuned)
    // row-pass layout: plain (15-bit targets with the sign, one pass) or wide (16-bit
    // targets, sign from the column string, targets split into npass ranges of span)
    bool wide = false;
    int npass = 1;
    int64_t span = 0;
    size_t smem_optin = 0;
    bool stall_next = false;      // test of the bounded waits: the next row pass stalls (see
                                  // kpm_test_rowpass_stall)
    size_t smem_bytes = 0;

    // wmax: max |W| over (pq|rs) and k_pq (host-computed), for the FP16 scale;
    // wcolsum: max over output slots s of sum over input slots k of |W[k][s]|;
    // d_diag: the exact diagonal H_II [N_a][N_b] (float hi, lo), kept by the caller.
    void init(const SpinTables& ta, const SpinTables& tb, const double* d_h1,
              const double* d_eri, const float2* d_diag, int n, double wmax, double wcolsum,
              bool use_fp16, cudaStream_t st);
    void apply(const float* x, float* y, int ncol, cudaStream_t st);
    // One row-pass launch (opposite-spin part of y, overwriting it) from the split
    // rows xh, xl, with the given A stages and prefetch distance.
    void launch_rowpass(const uint16_t* xh, const uint16_t* xl, float* y, int stages,
                        int prefetch, cudaStream_t st);
    // Times the row pass's stages x prefetch candidates once per device and shape.
    void autotune(cudaStream_t st);
    // Row-pass layout: passes = 0 automatic, >= 1 the wide layout with that many
    // passes (KPM_EINVAL where no wide kernel is instantiated for P).
    void set_layout(int passes, cudaStream_t st);
    // Reads and clears the device error flag (synchronises the stream).
    int check(cudaStream_t st);

    // Row-pass timing: while prof is set, every row-pass launch is bracketed by
    // a CUDA event pair on the launch stream; read_prof synchronises the stream,
    // returns the summed device time (ms) and launch count, and resets both.
    bool prof = false;
    std::vector<cudaEvent_t> ev;
    int ev_used = 0;
    double read_prof(cudaStream_t st, int* count);
    ~TcSigma();
};

// Dynamic shared memory of one row-pass CTA with the given number of A stages.
size_t rowpass_smem_bytes(const TcSigma& t, int stages);

}  // namespace kpm
