// Internal declarations shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <cstdio>
#include <string>
#include <vector>

#include "kpm.h"

namespace kpm {

// ---------------------------------------------------------------- errors

struct Error {
    kpm_status status;
    std::string msg;
};

// Thrown inside the library only; every extern "C" entry point catches it.
#define KPM_THROW(st, ...)                                                       \
    do {                                                                         \
        char _buf[512];                                                          \
        snprintf(_buf, sizeof(_buf), __VA_ARGS__);                               \
        throw ::kpm::Error{(st), std::string(_buf)};                             \
    } while (0)

#define KPM_CUDA(call)                                                           \
    do {                                                                         \
        cudaError_t _e = (call);                                                 \
        if (_e != cudaSuccess)                                                   \
            KPM_THROW(KPM_ECUDA, "%s:%d %s: %s", __FILE__, __LINE__, #call,      \
                      cudaGetErrorString(_e));                                   \
    } while (0)

// Message returned by kpm_last_error(NULL) on the calling thread.
void set_thread_error(const std::string& msg);

// Every kernel launch of the library goes through this counter.
extern std::atomic<uint64_t> g_launches;

#define KPM_LAUNCHED()                                                           \
    do {                                                                         \
        ::kpm::g_launches.fetch_add(1, std::memory_order_relaxed);               \
        cudaError_t _e = cudaGetLastError();                                     \
        if (_e != cudaSuccess)                                                   \
            KPM_THROW(KPM_ECUDA, "%s:%d launch: %s", __FILE__, __LINE__,         \
                      cudaGetErrorString(_e));                                   \
    } while (0)

// ---------------------------------------------------------------- device buffers

struct DevBuf {
    void* p = nullptr;
    size_t bytes = 0;
    DevBuf() = default;
    DevBuf(const DevBuf&) = delete;
    DevBuf& operator=(const DevBuf&) = delete;
    ~DevBuf() { release(); }
    void alloc(size_t n) {
        release();
        if (n == 0) return;
        cudaError_t e = cudaMalloc(&p, n);
        if (e != cudaSuccess) {
            p = nullptr;
            cudaGetLastError();
            KPM_THROW(KPM_ENOMEM, "cudaMalloc(%zu bytes) failed: %s", n, cudaGetErrorString(e));
        }
        bytes = n;
    }
    void ensure(size_t n) {
        if (n > bytes) alloc(n);
    }
    void release() {
        if (p) cudaFree(p);
        p = nullptr;
        bytes = 0;
    }
    template <class T> T* as() const { return static_cast<T*>(p); }
};

// ---------------------------------------------------------------- string tables

// One spin's occupation strings and single-excitation tables, all on the device.
struct SpinTables {
    int n = 0, m = 0;        // orbitals, electrons of this spin
    int64_t ns = 0;          // number of strings C(n, m)
    int nexc = 0;            // m (n - m + 1)
    int nnbr = 0;            // same-spin neighbours incl. itself: 1 + m(n-m) + C(m,2) C(n-m,2)
    DevBuf masks;            // uint32 [ns]
    DevBuf tgt, pq, sgn;     // int32/uint16/int8 [ns][nexc]  (API layout)
    DevBuf tgtT, pqT, sgnT;  // int32/uint16/int8 [nexc][ns]  (string-fastest, coalesced)
    DevBuf pkT;              // uint32 [nexc][ns]: target | pq << 16 | (sign < 0) << 31
    DevBuf fcol;             // int32  [nnbr][ns]  same-spin string Hamiltonian columns
    DevBuf fval64;           // double [nnbr][ns]
    DevBuf fval32;           // float  [nnbr][ns]
};

// Device binomial table C(p, k) for p, k <= KPM_MAX_ORB.
struct Binom {
    uint32_t c[KPM_MAX_ORB + 1][KPM_MAX_ORB + 1];
};
Binom make_binom();

void build_spin_tables(SpinTables& t, int n, int m, const double* d_h1, const double* d_eri,
                       cudaStream_t st);

// y[i] = (float) x[i]
void to_f32(const double* x, float* y, int64_t n, cudaStream_t st);

// ---------------------------------------------------------------- sigma (gather kernels)

struct SigmaArgs {
    const SpinTables* ta;
    const SpinTables* tb;
    const void* V;     // (pq|rs) as [n*n][n*n], double or float by path
    int n;
    int64_t dim;
    const float2* diag = nullptr;  // FP32 path: exact diagonal H_II as (hi, lo)
};

// diag[I] = H_II (FP64 evaluation, stored as float hi + float lo).
void exact_diagonal(const SpinTables& A, const SpinTables& B, const double* eri, int n,
                    float2* diag, cudaStream_t st);

void sigma_gather_f64(const SigmaArgs& a, const double* x, double* y, int ncol, cudaStream_t st);
void sigma_gather_f32(const SigmaArgs& a, const float* x, float* y, int ncol, cudaStream_t st);

void dipole_apply_f64(const SpinTables& ta, const SpinTables& tb, const double* d_dip,
                      const double* psi, double* y, cudaStream_t st);
void dipole_apply_f32(const SpinTables& ta, const SpinTables& tb, const double* d_dip,
                      const double* psi, float* y, cudaStream_t st);

// ---------------------------------------------------------------- batched steps

// One molecule of a batched recursion step (kpm_moments_batch): the operands of
// its sigma and update work and its first block in each flattened grid.  All
// molecules of a batch share the path (FP64, or FP32 with the exact diagonal).
struct BatchMol {
    // sigma: y = H x (gather path), x and y [ncol][nsa * nsb]
    const void* x;
    void* y;
    int64_t nsa, nsb;
    const int32_t* tgtA;
    const uint16_t* pqA;
    const int8_t* sgnA;
    const int32_t* fcolA;
    const void* fvalA;
    const int32_t* tgtBT;
    const uint16_t* pqBT;
    const int8_t* sgnBT;
    const int32_t* fcolB;
    const void* fvalB;
    const void* V;
    const float2* diag;
    int nexcA, nnbrA, nexcB, nnbrB, n, ncol;
    // update: prev <- 2 (y - b x) / a - prev; dots of step n at dots[col * dstride + 2n],
    // n = step0 + (the step's index within the batch)
    void* prev;
    double a, b;
    double* partials;
    unsigned* counters;
    double* dots;
    int64_t dstride;
    int64_t step0;      // recursion steps done before the batch
    int nblk;           // reduction blocks per column: reduce_blocks(nsa * nsb)
    int64_t sblk0;      // first block of this molecule in the flattened sigma grid
    int64_t ublk0;      // first block of this molecule in the flattened update grid
};

// Sigma of every molecule of mols[0 .. nmol) in one launch of `blocks` blocks
// (sum over molecules of ceil(nsb / 128) * nsa * ncol); smem: the largest
// per-molecule staging size.  Per element the same arithmetic as sigma_gather_*.
void sigma_gather_batch_f64(const BatchMol* mols, int nmol, int64_t blocks, size_t smem,
                            cudaStream_t st);
void sigma_gather_batch_f32(const BatchMol* mols, int nmol, int64_t blocks, size_t smem,
                            cudaStream_t st);
// Non-first update of every molecule in one launch (blocks = sum of nblk * ncol),
// batch step k (dots of step step0 + k); per element and per reduction the same
// as cheb_update_*.
void cheb_update_batch_f64(const BatchMol* mols, int nmol, int64_t blocks, int k,
                           cudaStream_t st);
void cheb_update_batch_f32(const BatchMol* mols, int nmol, int64_t blocks, int k,
                           cudaStream_t st);

// ---------------------------------------------------------------- recursion helpers

// Fixed reduction grid for a vector of length dim (deterministic partial order).
int reduce_blocks(int64_t dim);

// alpha_next = first ? (s - b c)/a : 2 (s - b c)/a - prev, written over prev;
// dots[col*stride + 0] = <c|c>, dots[col*stride + 1] = <next|c> (FP64).
// dots of the step go to dots[2n], dots[2n+1] (per column, stride dots_col_stride),
// n = *step when step is non-null (device counter), else n = 0 at `dots`.
void cheb_update_f64(const double* s, const double* c, double* prev, int64_t dim, int ncol,
                     double a, double b, int first, double* partials, unsigned* counters,
                     double* dots, int64_t dots_col_stride, const unsigned* step,
                     cudaStream_t st);
void cheb_update_f32(const float* s, const float* c, float* prev, int64_t dim, int ncol,
                     double a, double b, int first, double* partials, unsigned* counters,
                     double* dots, int64_t dots_col_stride, const unsigned* step,
                     cudaStream_t st);
void step_set(unsigned* step, unsigned v, cudaStream_t st);
void step_inc(unsigned* step, cudaStream_t st);

// moments[col][2n], [2n+1] from dots[col][n][2] (doubling identities); with defl
// (deflated recursions) defl[col] T_n(x0) is added to moment n.
void doubling_combine(const double* dots, int ncol, int nsteps, int64_t dots_col_stride,
                      double* moments, int nmoments_stride, const double* defl, double x0,
                      cudaStream_t st);
// al -= coef[0] p (FP64, in place) and out = al in the context precision.
void deflate(double* al, const double* p, int64_t dim, const double* coef, void* out, bool f64,
             cudaStream_t st);
// Two-column block (a, b) cross dots: out[0] = <a_n|b_n> (cur), out[1] = <a_n+1|b_n>.
void cross_dots(const void* cur, const void* next, int64_t dim, bool f64, double* partials,
                unsigned* counters, double* out, cudaStream_t st);
// Cross moments from the cross dots c[2n], c[2n+1] (doubling identities).
void cross_doubling(const double* cross, int nsteps, double* moments, cudaStream_t st);
// *c2 = (*c)^2 on the device.
void square_into(const double* c, double* c2, cudaStream_t st);

// Lanczos pieces (FP64 scalars on the device).
void dot_dev(const void* x, const void* y, int64_t dim, bool f64, double* partials,
             unsigned* counters, double* out, cudaStream_t st);
void lanczos_orth(void* w, const void* v, const void* vprev, int64_t dim, bool f64,
                  const double* alpha, const double* beta_prev, double* partials,
                  unsigned* counters, double* norm2_out, cudaStream_t st);
void lanczos_scale(void* vnext, const void* w, int64_t dim, bool f64, const double* norm2,
                   double* beta_out, cudaStream_t st);
void fill_random(void* v, int64_t dim, bool f64, uint64_t seed, cudaStream_t st);
void scale_inplace(void* v, int64_t dim, bool f64, const double* norm2, cudaStream_t st);
// scratch: 3k doubles of device memory.
void tridiag_extremes(const double* alpha, const double* beta, int k, double* out4,
                      double* scratch, cudaStream_t st);

// Lowest eigenpair of a k x k symmetric tridiagonal (device): *theta and the unit
// eigenvector s[0..k); scratch: 2k doubles.
void tridiag_lowest(const double* alpha, const double* beta, int k, double* theta, double* s,
                    double* scratch, cudaStream_t st);
// acc += coef[0] * v, acc FP64 [dim], v FP64 or FP32; coef read on the device.
void axpy_dev(double* acc, const void* v, int64_t dim, bool f64, const double* coef,
              cudaStream_t st);

// Spectrum on the device: moments (device) -> omega, intensity (device);
// `damped` is device scratch of N doubles (g_n Omega_n with the factor 2 for n >= 1).
// kernel: 0 none, 1 Jackson, 2 Lorentz with parameter lambda.
void spectrum_dev(const double* moments, int N, double a, double b, int M, int kernel,
                  double* damped, double* omega, double* intensity, cudaStream_t st,
                  double lambda = KPM_LORENTZ_LAMBDA);

}  // namespace kpm
