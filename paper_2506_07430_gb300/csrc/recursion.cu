// Chebyshev recursion step, moment dot products, doubling identities and the
// Lanczos pieces used for the spectral bounds.
//
// Step (Methods, KPM recursion on the rescaled H~ = (H - b)/a):
//   alpha_1     = (sigma - b alpha_0) / a                   (first step)
//   alpha_{n+1} = 2 (sigma - b alpha_n) / a - alpha_{n-1}   (written over alpha_{n-1})
// with sigma = H alpha_n, fused with the two dot products the doubling
// identities need, s_n = <alpha_n|alpha_n> and t_n = <alpha_{n+1}|alpha_n>:
//   Omega_2n = 2 s_n - s_0,  Omega_2n+1 = 2 t_n - t_0       (Methods, doubling)
//
// Reductions are deterministic: a fixed grid (depending only on the vector
// length), warp-shuffle and shared-memory trees in a fixed order, per-block
// FP64 partials, and a final fixed-order sum done by whichever block finishes
// last (the order of the final sum does not depend on which block that is).
// In the FP32 path, products of groups of 4 consecutive elements of a thread's
// stride are summed in FP32 and each group sum is added in FP64.
#include "common.cuh"

namespace kpm {

static constexpr int RED_THREADS = 256;
static constexpr int RED_MAX_BLOCKS = 1216;  // 8 x 152, fixed for determinism

int reduce_blocks(int64_t dim) {
    int64_t b = (dim + RED_THREADS * 8 - 1) / (RED_THREADS * 8);
    if (b < 1) b = 1;
    if (b > RED_MAX_BLOCKS) b = RED_MAX_BLOCKS;
    return (int)b;
}

// Block-wide sum of two doubles, result valid in thread 0.
__device__ __forceinline__ void block_sum2(double& u, double& v) {
    __shared__ double su[32], sv[32];
    for (int o = 16; o > 0; o >>= 1) {
        u += __shfl_down_sync(0xffffffffu, u, o);
        v += __shfl_down_sync(0xffffffffu, v, o);
    }
    int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) { su[w] = u; sv[w] = v; }
    __syncthreads();
    int nw = (blockDim.x + 31) >> 5;
    if (w == 0) {
        u = l < nw ? su[l] : 0.0;
        v = l < nw ? sv[l] : 0.0;
        for (int o = 16; o > 0; o >>= 1) {
            u += __shfl_down_sync(0xffffffffu, u, o);
            v += __shfl_down_sync(0xffffffffu, v, o);
        }
    }
}

// Stores the partials of block blk (of nblk); the last block to finish sums
// them in a fixed order into out[0], out[1] and re-arms the counter.
__device__ __forceinline__ void finish_reduce(double u, double v, double* partials,
                                              unsigned* counter, int nblk, int blk, double* out0,
                                              double* out1) {
    block_sum2(u, v);
    __shared__ bool last;
    if (threadIdx.x == 0) {
        partials[2 * blk] = u;
        partials[2 * blk + 1] = v;
        __threadfence();
        unsigned prev = atomicAdd(counter, 1u);
        last = (prev == (unsigned)nblk - 1);
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    double a = 0.0, b = 0.0;
    for (int i = threadIdx.x; i < nblk; i += blockDim.x) {
        a += __ldcg(partials + 2 * i);
        b += __ldcg(partials + 2 * i + 1);
    }
    block_sum2(a, b);
    if (threadIdx.x == 0) {
        if (out0) *out0 = a;
        if (out1) *out1 = b;
        *counter = 0u;
    }
}

// Block blk (of nblk) of column col of the update; dots of step n go to
// dots[2n], dots[2n+1].  Shared by the single-molecule kernel and the batched
// one, so that both do the same arithmetic and reduction.
template <class T>
__device__ __forceinline__ void cheb_update_cta(int blk, int nblk, int col,
                                                const T* __restrict__ s, const T* __restrict__ c,
                                                T* __restrict__ prev, int64_t dim, double a,
                                                double b, int first, double* partials,
                                                unsigned* counters, double* dots, int64_t dstride,
                                                int64_t n) {
    dots += 2 * n;
    s += col * dim;
    c += col * dim;
    prev += col * dim;
    const int64_t stride = (int64_t)nblk * blockDim.x;
    double ss = 0.0, tt = 0.0;
    if constexpr (sizeof(T) == 8) {
        const double k1 = (first ? 1.0 : 2.0) / a, k2 = b * k1;
        for (int64_t i = (int64_t)blk * blockDim.x + threadIdx.x; i < dim; i += stride) {
            double cv = c[i];
            double nx = k1 * s[i] - k2 * cv;
            if (!first) nx -= prev[i];
            prev[i] = nx;
            ss += cv * cv;
            tt += nx * cv;
        }
    } else {
        // k1 = 2/a and k2 = 2b/a as float pairs (hi + lo): rounding them to one float
        // each would shift every eigenvalue of H~ by the same relative 2^-24, an
        // error that grows linearly with the moment index
        const double k1d = (first ? 1.0 : 2.0) / a, k2d = b * k1d;
        const float k1 = (float)k1d, k1l = (float)(k1d - (double)k1);
        const float k2 = (float)k2d, k2l = (float)(k2d - (double)k2);
        int64_t i = (int64_t)blk * blockDim.x + threadIdx.x;
        while (i < dim) {
            float gs = 0.f, gt = 0.f;
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                if (i < dim) {
                    float cv = c[i];
                    const float sv = s[i];
                    float nx = fmaf(k1, sv, fmaf(-k2, cv, fmaf(k1l, sv, -k2l * cv)));
                    if (!first) nx -= prev[i];
                    prev[i] = nx;
                    gs = fmaf(cv, cv, gs);
                    gt = fmaf(nx, cv, gt);
                }
                i += stride;
            }
            ss += (double)gs;
            tt += (double)gt;
        }
    }
    finish_reduce(ss, tt, partials + (int64_t)col * 2 * nblk, counters + col, nblk, blk,
                  dots + col * dstride, dots + col * dstride + 1);
}

template <class T>
__global__ void __launch_bounds__(RED_THREADS)
k_cheb_update(const T* __restrict__ s, const T* __restrict__ c, T* __restrict__ prev, int64_t dim,
              double a, double b, int first, double* partials, unsigned* counters, double* dots,
              int64_t dstride, const unsigned* step) {
    // n from the device counter if given (replayable captured steps), else 0
    const int64_t n = step ? (int64_t)(*step) : 0;
    cheb_update_cta<T>(blockIdx.x, gridDim.x, blockIdx.y, s, c, prev, dim, a, b, first, partials,
                       counters, dots, dstride, n);
}

// Batched non-first update: the flattened grid covers every molecule's
// (reduction block, column) blocks; each molecule keeps its own fixed
// reduction grid, partials and counters.
template <class T>
__global__ void __launch_bounds__(RED_THREADS)
k_cheb_update_batch(const BatchMol* __restrict__ mols, int nmol, int64_t k) {
    const int64_t blk = blockIdx.x;
    int lo = 0, hi = nmol - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (mols[mid].ublk0 <= blk) lo = mid; else hi = mid - 1;
    }
    const BatchMol& m = mols[lo];
    const int64_t local = blk - m.ublk0;
    const int b = (int)(local % m.nblk);
    const int col = (int)(local / m.nblk);
    cheb_update_cta<T>(b, m.nblk, col, static_cast<const T*>(m.y), static_cast<const T*>(m.x),
                       static_cast<T*>(m.prev), m.nsa * m.nsb, m.a, m.b, 0, m.partials,
                       m.counters, m.dots, m.dstride, m.step0 + k);
}

template <class T>
static void launch_update_batch(const BatchMol* mols, int nmol, int64_t blocks, int k,
                                cudaStream_t st) {
    if (nmol <= 0 || blocks <= 0) return;
    if (blocks > 0x7FFFFFFFLL) KPM_THROW(KPM_EINVAL, "batched update grid too large");
    k_cheb_update_batch<T><<<(unsigned)blocks, RED_THREADS, 0, st>>>(mols, nmol, (int64_t)k);
    KPM_LAUNCHED();
}

void cheb_update_batch_f64(const BatchMol* mols, int nmol, int64_t blocks, int k,
                           cudaStream_t st) {
    launch_update_batch<double>(mols, nmol, blocks, k, st);
}
void cheb_update_batch_f32(const BatchMol* mols, int nmol, int64_t blocks, int k,
                           cudaStream_t st) {
    launch_update_batch<float>(mols, nmol, blocks, k, st);
}

template <class T>
static void launch_update(const T* s, const T* c, T* prev, int64_t dim, int ncol, double a,
                          double b, int first, double* partials, unsigned* counters, double* dots,
                          int64_t dstride, const unsigned* step, cudaStream_t st) {
    dim3 grid(reduce_blocks(dim), ncol);
    k_cheb_update<T><<<grid, RED_THREADS, 0, st>>>(s, c, prev, dim, a, b, first, partials,
                                                   counters, dots, dstride, step);
    KPM_LAUNCHED();
}

void cheb_update_f64(const double* s, const double* c, double* prev, int64_t dim, int ncol,
                     double a, double b, int first, double* partials, unsigned* counters,
                     double* dots, int64_t dstride, const unsigned* step, cudaStream_t st) {
    launch_update<double>(s, c, prev, dim, ncol, a, b, first, partials, counters, dots, dstride,
                          step, st);
}
void cheb_update_f32(const float* s, const float* c, float* prev, int64_t dim, int ncol, double a,
                     double b, int first, double* partials, unsigned* counters, double* dots,
                     int64_t dstride, const unsigned* step, cudaStream_t st) {
    launch_update<float>(s, c, prev, dim, ncol, a, b, first, partials, counters, dots, dstride,
                         step, st);
}

__global__ void k_step_set(unsigned* step, unsigned v) { *step = v; }
__global__ void k_step_inc(unsigned* step) { *step += 1u; }

// device-side step counter of the recursion (read by k_cheb_update), so that a
// captured step is replayable
void step_set(unsigned* step, unsigned v, cudaStream_t st) {
    k_step_set<<<1, 1, 0, st>>>(step, v);
    KPM_LAUNCHED();
}
void step_inc(unsigned* step, cudaStream_t st) {
    k_step_inc<<<1, 1, 0, st>>>(step);
    KPM_LAUNCHED();
}

// With `defl` (deflated recursion, see rec_begin_deflated): the permanent-dipole
// term defl[col] T_n(x0), T_n(x0) = cos(n arccos x0), is added to moment n.
__global__ void k_doubling(const double* __restrict__ dots, int nsteps, int64_t dstride,
                           double* __restrict__ mom, int mstride, const double* defl, double x0) {
    const int col = blockIdx.y;
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= nsteps) return;
    const double* d = dots + col * dstride;
    double s0 = d[0], t0 = d[1];
    double sn = d[2 * n], tn = d[2 * n + 1];
    double* m = mom + (int64_t)col * mstride;
    double m0 = n == 0 ? s0 : 2.0 * sn - s0;
    double m1 = n == 0 ? t0 : 2.0 * tn - t0;
    if (defl) {
        const double th = acos(x0), c2 = defl[col];
        m0 += c2 * cos((double)(2 * n) * th);
        m1 += c2 * cos((double)(2 * n + 1) * th);
    }
    m[2 * n] = m0;
    m[2 * n + 1] = m1;
}

void doubling_combine(const double* dots, int ncol, int nsteps, int64_t dstride, double* moments,
                      int mstride, const double* defl, double x0, cudaStream_t st) {
    if (nsteps <= 0) return;
    dim3 grid((nsteps + 127) / 128, ncol);
    k_doubling<<<grid, 128, 0, st>>>(dots, nsteps, dstride, moments, mstride, defl, x0);
    KPM_LAUNCHED();
}

// Cross dots of a two-column block recursion (columns a, b): out[0] = <a_n|b_n>
// from cur, out[1] = <a_n+1|b_n> from next (column a) and cur (column b).
template <class T>
__global__ void __launch_bounds__(RED_THREADS)
k_cross_dots(const T* __restrict__ cur, const T* __restrict__ next, int64_t dim, double* partials,
             unsigned* counter, double* out) {
    double u = 0.0, v = 0.0;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < dim; i += stride) {
        const double bn = (double)cur[dim + i];
        u += (double)cur[i] * bn;
        v += (double)next[i] * bn;
    }
    finish_reduce(u, v, partials, counter, gridDim.x, blockIdx.x, out, out + 1);
}

void cross_dots(const void* cur, const void* next, int64_t dim, bool f64, double* partials,
                unsigned* counters, double* out, cudaStream_t st) {
    int g = reduce_blocks(dim);
    if (f64)
        k_cross_dots<double><<<g, RED_THREADS, 0, st>>>((const double*)cur, (const double*)next,
                                                        dim, partials, counters, out);
    else
        k_cross_dots<float><<<g, RED_THREADS, 0, st>>>((const float*)cur, (const float*)next, dim,
                                                       partials, counters, out);
    KPM_LAUNCHED();
}

// Omega_0 = c[0], Omega_1 = c[1], Omega_2n = 2 c[2n] - c[0], Omega_2n+1 = 2 c[2n+1] - c[1]
__global__ void k_cross_doubling(const double* __restrict__ c, int nsteps, double* __restrict__ m) {
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= nsteps) return;
    m[2 * n] = n == 0 ? c[0] : 2.0 * c[2 * n] - c[0];
    m[2 * n + 1] = n == 0 ? c[1] : 2.0 * c[2 * n + 1] - c[1];
}

void cross_doubling(const double* cross, int nsteps, double* moments, cudaStream_t st) {
    if (nsteps <= 0) return;
    k_cross_doubling<<<(nsteps + 127) / 128, 128, 0, st>>>(cross, nsteps, moments);
    KPM_LAUNCHED();
}

// a[i] -= coef[0] * p[i]; out (context precision) = a, FP64 in place
template <class T>
__global__ void k_deflate(double* __restrict__ al, const double* __restrict__ p, int64_t dim,
                          const double* coef, T* __restrict__ out) {
    const double c = *coef;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < dim; i += stride) {
        const double v = al[i] - c * p[i];
        al[i] = v;
        out[i] = (T)v;
    }
}

void deflate(double* al, const double* p, int64_t dim, const double* coef, void* out, bool f64,
             cudaStream_t st) {
    int g = reduce_blocks(dim);
    if (f64) k_deflate<double><<<g, RED_THREADS, 0, st>>>(al, p, dim, coef, (double*)out);
    else k_deflate<float><<<g, RED_THREADS, 0, st>>>(al, p, dim, coef, (float*)out);
    KPM_LAUNCHED();
}

__global__ void k_square_into(const double* __restrict__ c, double* __restrict__ c2) {
    *c2 = (*c) * (*c);
}

void square_into(const double* c, double* c2, cudaStream_t st) {
    k_square_into<<<1, 1, 0, st>>>(c, c2);
    KPM_LAUNCHED();
}

// ---------------------------------------------------------------- Lanczos pieces

template <class T>
__global__ void __launch_bounds__(RED_THREADS)
k_dot(const T* __restrict__ x, const T* __restrict__ y, int64_t dim, double* partials,
      unsigned* counter, double* out) {
    double u = 0.0, v = 0.0;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < dim; i += stride)
        u += (double)x[i] * (double)y[i];
    finish_reduce(u, v, partials, counter, gridDim.x, blockIdx.x, out, nullptr);
}

void dot_dev(const void* x, const void* y, int64_t dim, bool f64, double* partials,
             unsigned* counters, double* out, cudaStream_t st) {
    int g = reduce_blocks(dim);
    if (f64)
        k_dot<double><<<g, RED_THREADS, 0, st>>>((const double*)x, (const double*)y, dim,
                                                 partials, counters, out);
    else
        k_dot<float><<<g, RED_THREADS, 0, st>>>((const float*)x, (const float*)y, dim, partials,
                                                counters, out);
    KPM_LAUNCHED();
}

// w -= alpha v + beta_prev vprev;  norm2 = <w|w>
template <class T>
__global__ void __launch_bounds__(RED_THREADS)
k_lanczos_orth(T* __restrict__ w, const T* __restrict__ v, const T* __restrict__ vp, int64_t dim,
               const double* alpha, const double* beta_prev, double* partials, unsigned* counter,
               double* norm2) {
    const double al = *alpha, be = beta_prev ? *beta_prev : 0.0;
    double u = 0.0;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < dim; i += stride) {
        double x = (double)w[i] - al * (double)v[i];
        if (vp) x -= be * (double)vp[i];
        T xt = (T)x;
        w[i] = xt;
        u += (double)xt * (double)xt;
    }
    finish_reduce(u, 0.0, partials, counter, gridDim.x, blockIdx.x, norm2, nullptr);
}

void lanczos_orth(void* w, const void* v, const void* vprev, int64_t dim, bool f64,
                  const double* alpha, const double* beta_prev, double* partials,
                  unsigned* counters, double* norm2_out, cudaStream_t st) {
    int g = reduce_blocks(dim);
    if (f64)
        k_lanczos_orth<double><<<g, RED_THREADS, 0, st>>>(
            (double*)w, (const double*)v, (const double*)vprev, dim, alpha, beta_prev, partials,
            counters, norm2_out);
    else
        k_lanczos_orth<float><<<g, RED_THREADS, 0, st>>>(
            (float*)w, (const float*)v, (const float*)vprev, dim, alpha, beta_prev, partials,
            counters, norm2_out);
    KPM_LAUNCHED();
}

template <class T>
__global__ void k_lanczos_scale(T* __restrict__ vn, const T* __restrict__ w, int64_t dim,
                                const double* norm2, double* beta_out) {
    const double be = sqrt(*norm2);
    const double inv = be > 0.0 ? 1.0 / be : 0.0;
    if (blockIdx.x == 0 && threadIdx.x == 0 && beta_out) *beta_out = be;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < dim; i += stride)
        vn[i] = (T)((double)w[i] * inv);
}

void lanczos_scale(void* vnext, const void* w, int64_t dim, bool f64, const double* norm2,
                   double* beta_out, cudaStream_t st) {
    int g = reduce_blocks(dim);
    if (f64)
        k_lanczos_scale<double><<<g, RED_THREADS, 0, st>>>((double*)vnext, (const double*)w, dim,
                                                           norm2, beta_out);
    else
        k_lanczos_scale<float><<<g, RED_THREADS, 0, st>>>((float*)vnext, (const float*)w, dim,
                                                          norm2, beta_out);
    KPM_LAUNCHED();
}

void scale_inplace(void* v, int64_t dim, bool f64, const double* norm2, cudaStream_t st) {
    lanczos_scale(v, v, dim, f64, norm2, nullptr, st);
}

// SplitMix64 (Steele, Lea, Flood 2014): z = seed + (i+1) * 0x9e3779b97f4a7c15, then the
// standard finaliser; the top 53 bits give a uniform double in [0,1), mapped to [-1,1).
__device__ __forceinline__ uint64_t splitmix64(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
    return z ^ (z >> 31);
}

template <class T>
__global__ void k_fill_random(T* __restrict__ v, int64_t dim, uint64_t seed) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < dim; i += stride) {
        uint64_t z = splitmix64(seed + (uint64_t)(i + 1) * 0x9e3779b97f4a7c15ull);
        double u = (double)(z >> 11) * (1.0 / 9007199254740992.0);
        v[i] = (T)(2.0 * u - 1.0);
    }
}

void fill_random(void* v, int64_t dim, bool f64, uint64_t seed, cudaStream_t st) {
    int g = reduce_blocks(dim);
    if (f64)
        k_fill_random<double><<<g, RED_THREADS, 0, st>>>((double*)v, dim, seed);
    else
        k_fill_random<float><<<g, RED_THREADS, 0, st>>>((float*)v, dim, seed);
    KPM_LAUNCHED();
}

// Extreme eigenvalues of the k x k symmetric tridiagonal T (diagonal alpha[0..k),
// off-diagonal beta[0..k-1)) by Sturm-sequence bisection, and the Ritz residual
// estimates |beta[k-1] * (last component of the unit eigenvector)|.
// out4 = {theta_min, theta_max, res_min, res_max}.  One thread.
__device__ int sturm_below(const double* al, const double* be, int k, double x) {
    int cnt = 0;
    double q = 1.0;
    for (int i = 0; i < k; ++i) {
        double off = i ? be[i - 1] * be[i - 1] : 0.0;
        q = (al[i] - x) - (i ? off / q : 0.0);
        if (q == 0.0) q = -1e-300;
        if (q < 0.0) ++cnt;
    }
    return cnt;
}

__device__ double tri_eig(const double* al, const double* be, int k, int idx, double lo, double hi) {
    for (int it = 0; it < 200; ++it) {
        double mid = 0.5 * (lo + hi);
        if (mid <= lo || mid >= hi) break;
        if (sturm_below(al, be, k, mid) > idx) hi = mid; else lo = mid;
    }
    return 0.5 * (lo + hi);
}

// Last component of the unit eigenvector of T for eigenvalue th, by inverse
// iteration with the tridiagonal (Thomas) solver; w is scratch of 3k doubles.
__device__ double last_component(const double* al, const double* be, int k, double th,
                                 double* w) {
    double* x = w;
    double* c = w + k;
    double* d = w + 2 * k;
    double scale = 0.0;
    for (int i = 0; i < k; ++i) scale = fmax(scale, fabs(al[i]) + (i + 1 < k ? fabs(be[i]) : 0.0));
    const double shift = th + 1e-10 * (scale + 1e-300);
    for (int i = 0; i < k; ++i) x[i] = 1.0;
    for (int it = 0; it < 4; ++it) {
        // solve (T - shift) y = x; y overwrites x
        double piv = al[0] - shift;
        if (fabs(piv) < 1e-300) piv = 1e-300;
        c[0] = (k > 1 ? be[0] : 0.0) / piv;
        d[0] = x[0] / piv;
        for (int i = 1; i < k; ++i) {
            piv = (al[i] - shift) - be[i - 1] * c[i - 1];
            if (fabs(piv) < 1e-300) piv = 1e-300;
            c[i] = (i + 1 < k ? be[i] : 0.0) / piv;
            d[i] = (x[i] - be[i - 1] * d[i - 1]) / piv;
        }
        x[k - 1] = d[k - 1];
        for (int i = k - 2; i >= 0; --i) x[i] = d[i] - c[i] * x[i + 1];
        double nrm = 0.0;
        for (int i = 0; i < k; ++i) nrm += x[i] * x[i];
        nrm = sqrt(nrm);
        if (!(nrm > 0.0) || !isfinite(nrm)) return 1.0;
        for (int i = 0; i < k; ++i) x[i] /= nrm;
    }
    return fabs(x[k - 1]);
}

__global__ void k_tridiag(const double* al, const double* be, int k, double* out, double* w) {
    if (threadIdx.x || blockIdx.x) return;
    double lo = al[0], hi = al[0];
    for (int i = 0; i < k; ++i) {
        double r = (i ? fabs(be[i - 1]) : 0.0) + (i + 1 < k ? fabs(be[i]) : 0.0);
        lo = fmin(lo, al[i] - r);
        hi = fmax(hi, al[i] + r);
    }
    lo -= 1e-9 * (1.0 + fabs(lo));
    hi += 1e-9 * (1.0 + fabs(hi));
    double tmin = tri_eig(al, be, k, 0, lo, hi);
    double tmax = tri_eig(al, be, k, k - 1, lo, hi);
    double bk = fabs(be[k - 1]);
    out[0] = tmin;
    out[1] = tmax;
    out[2] = bk * last_component(al, be, k, tmin, w);
    out[3] = bk * last_component(al, be, k, tmax, w);
}

void tridiag_extremes(const double* alpha, const double* beta, int k, double* out4,
                      double* scratch, cudaStream_t st) {
    k_tridiag<<<1, 1, 0, st>>>(alpha, beta, k, out4, scratch);
    KPM_LAUNCHED();
}

// Lowest eigenpair of the k x k symmetric tridiagonal T: theta by Sturm
// bisection, its unit eigenvector s by inverse iteration with the tridiagonal
// (Thomas) solver, shifted just below theta.  out[0] = theta, s_out[0..k).
__global__ void k_tridiag_lowest(const double* al, const double* be, int k, double* out,
                                 double* s_out, double* w) {
    if (threadIdx.x || blockIdx.x) return;
    double lo = al[0], hi = al[0];
    for (int i = 0; i < k; ++i) {
        double r = (i ? fabs(be[i - 1]) : 0.0) + (i + 1 < k ? fabs(be[i]) : 0.0);
        lo = fmin(lo, al[i] - r);
        hi = fmax(hi, al[i] + r);
    }
    lo -= 1e-9 * (1.0 + fabs(lo));
    hi += 1e-9 * (1.0 + fabs(hi));
    const double th = tri_eig(al, be, k, 0, lo, hi);
    double* c = w;
    double* d = w + k;
    double scale = 0.0;
    for (int i = 0; i < k; ++i) scale = fmax(scale, fabs(al[i]) + (i + 1 < k ? fabs(be[i]) : 0.0));
    const double shift = th - 1e-12 * (scale + 1e-300);
    for (int i = 0; i < k; ++i) s_out[i] = 1.0;
    for (int it = 0; it < 6; ++it) {
        double piv = al[0] - shift;
        if (fabs(piv) < 1e-300) piv = 1e-300;
        c[0] = (k > 1 ? be[0] : 0.0) / piv;
        d[0] = s_out[0] / piv;
        for (int i = 1; i < k; ++i) {
            piv = (al[i] - shift) - be[i - 1] * c[i - 1];
            if (fabs(piv) < 1e-300) piv = 1e-300;
            c[i] = (i + 1 < k ? be[i] : 0.0) / piv;
            d[i] = (s_out[i] - be[i - 1] * d[i - 1]) / piv;
        }
        s_out[k - 1] = d[k - 1];
        for (int i = k - 2; i >= 0; --i) s_out[i] = d[i] - c[i] * s_out[i + 1];
        double nrm = 0.0;
        for (int i = 0; i < k; ++i) nrm += s_out[i] * s_out[i];
        nrm = sqrt(nrm);
        if (!(nrm > 0.0) || !isfinite(nrm)) {
            for (int i = 0; i < k; ++i) s_out[i] = i == 0 ? 1.0 : 0.0;
            break;
        }
        for (int i = 0; i < k; ++i) s_out[i] /= nrm;
    }
    out[0] = th;
}

void tridiag_lowest(const double* alpha, const double* beta, int k, double* theta, double* s,
                    double* scratch, cudaStream_t st) {
    k_tridiag_lowest<<<1, 1, 0, st>>>(alpha, beta, k, theta, s, scratch);
    KPM_LAUNCHED();
}

// acc[i] += coef[0] * v[i] (FP64 accumulation; the coefficient is read on the device)
template <class T>
__global__ void k_axpy_dev(double* __restrict__ acc, const T* __restrict__ v, int64_t dim,
                           const double* coef) {
    const double c = *coef;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < dim; i += stride)
        acc[i] += c * (double)v[i];
}

void axpy_dev(double* acc, const void* v, int64_t dim, bool f64, const double* coef,
              cudaStream_t st) {
    int g = reduce_blocks(dim);
    if (f64)
        k_axpy_dev<double><<<g, RED_THREADS, 0, st>>>(acc, (const double*)v, dim, coef);
    else
        k_axpy_dev<float><<<g, RED_THREADS, 0, st>>>(acc, (const float*)v, dim, coef);
    KPM_LAUNCHED();
}

}  // namespace kpm
