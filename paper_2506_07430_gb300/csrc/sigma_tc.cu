// sigma = H x on tcgen05 tensor cores (KPM_MIXED, KPM_MIXED_BF16).
//
// With the alpha/beta string factorisation of the paper's second-quantized H
// (Methods),
//   H = F_a (x) 1 + 1 (x) F_b + sum_{pq,rs} (pq|rs) E^a_pq E^b_rs,
// where F_s is one spin's string Hamiltonian (tables.cu).  The same-spin parts
// are dense GEMMs with F_a, F_b (gemm_tc.cu).  This file holds the
// opposite-spin part.  Because (pq|rs) = (qp|rs) = (pq|sr), sums over ordered
// pairs fold onto the NS = n(n+1)/2 unordered pairs ("slots"); a string has at
// most one table entry per slot.  For one alpha string R (a row of X[R][C]) and
// a tile of 128 beta strings J:
//   A[J][e] = X[tgt_e, J]                    for the entries e of tab(R)  (gather)
//   B_R[s][e] = sgn_e W[slot(e)][s],         W[s][s'] = (pq|rs)
//   G = A B_R^T
//   sigma[R, tgt_f] += sgn_f G[J][slot(f)]   for every f in tab(J)        (scatter)
// (<I|E_pq|J> = <J|E_qp|I> turns the outer excitation into a scatter from J.)
//
// GEMM per tile: M = 128 columns J, K = KR (the row's nexc entries rounded up
// to 16), N = P (NS + 1 rounded up to 16).  A is written by the CUDA cores
// straight into tensor memory (tcgen05.st, one TMEM lane per column J); B_R is
// gathered once per row from the W image into shared memory (canonical K-major
// layout without swizzle, signs folded in); D accumulates in tensor memory in
// FP32.  Operands are split into 16-bit pieces (FP16 with power-of-two scales:
// x in 2, W in 3 pieces, 4 MMAs; or BF16 2 + 2, 3 MMAs).  The epilogue reads D
// (tcgen05.ld) and scatters into the row's sigma in shared memory with 32-bit
// fixed-point integer atomics (order-independent, so the result is
// reproducible bit for bit).
//
// One CTA (16 warps) per SM, persistent over rows; the 4 warps of each TMEM lane
// quadrant take chunks of 8 (entries or slots) round-robin.  Per tile t the CTA waits for MMA(t),
// copies D(t) to registers, issues MMA(t+1), builds A(t+2) and scatters D(t),
// so the tensor core runs while the CUDA cores build and scatter.  Waits on the
// MMA-completion mbarrier are bounded (about two seconds); on expiry the kernel
// records an error, frees its TMEM and returns.
#include "sigma_tc.cuh"

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <cmath>

namespace kpm {

namespace {

constexpr long long WAIT_CYCLES = 4000000000LL;  // ~2 s at 2 GHz

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void tmem_alloc(uint32_t* holder, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                 ::"r"(smem_u32(holder)), "r"(ncols) : "memory");
}
__device__ __forceinline__ void tmem_relinquish() {
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols)
                 : "memory");
}
__device__ __forceinline__ void tc_fence_before() {
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tmem_st4(uint32_t taddr, uint32_t a, uint32_t b, uint32_t c,
                                         uint32_t d) {
    asm volatile("tcgen05.st.sync.aligned.32x32b.x4.b32 [%0], {%1, %2, %3, %4};"
                 ::"r"(taddr), "r"(a), "r"(b), "r"(c), "r"(d) : "memory");
}
__device__ __forceinline__ void tmem_st_wait() {
    asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_ld8(uint32_t taddr, uint32_t (&r)[8]) {
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]),
                   "=r"(r[6]), "=r"(r[7])
                 : "r"(taddr)
                 : "memory");
}
__device__ __forceinline__ void tmem_ld_wait() {
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}
// D[tmem] (+)= A[tmem] * B[smem]^T, kind::f16 (BF16 or FP16 operands, FP32 accumulate)
__device__ __forceinline__ void mma_ts(uint32_t d, uint32_t a, uint64_t bdesc, uint32_t idesc,
                                       uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n\t}"
        ::"r"(d), "r"(a), "l"(bdesc), "r"(idesc), "r"(accumulate) : "memory");
}
__device__ __forceinline__ void mma_commit(uint64_t* mbar) {
    asm volatile(
        "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
        ::"r"(smem_u32(mbar)) : "memory");
}
__device__ __forceinline__ void mbar_init(uint64_t* mbar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(mbar)), "r"(count)
                 : "memory");
}
__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* mbar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(mbar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// 4-byte asynchronous global -> shared copy; src_bytes = 0 writes zero
__device__ __forceinline__ void cp_async4(uint32_t dst, const void* src, uint32_t src_bytes) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(dst), "l"(src),
                 "r"(src_bytes) : "memory");
}
__device__ __forceinline__ void cp_async_commit() {
    asm volatile("cp.async.commit_group;" ::: "memory");
}
template <int N>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// Shared-memory matrix descriptor, canonical K-major layout without swizzle:
// 8-row x 16-byte core matrices; LBO = byte distance between core matrices
// adjacent along K, SBO = between core matrices adjacent along M/N.
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
    d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1 << 46;  // descriptor version for tcgen05
    return d;                // base offset 0, swizzle none
}

// Instruction descriptor, kind::f16: D = F32, A/B = BF16 (1) or F16 (0), both
// K-major, N >> 3 at bit 17, M >> 4 at bit 24.
__host__ __device__ constexpr uint32_t instr_desc(int M, int N, bool bf16) {
    return (1u << 4) | ((bf16 ? 1u : 0u) << 7) | ((bf16 ? 1u : 0u) << 10) |
           ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

template <bool FP16>
__device__ __forceinline__ uint32_t pack2(float a, float b) {
    if (FP16) {
        __half2 h = __floats2half2_rn(a, b);
        return *reinterpret_cast<uint32_t*>(&h);
    } else {
        __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
        return *reinterpret_cast<uint32_t*>(&h);
    }
}
template <bool FP16>
__device__ __forceinline__ float round16(float a) {
    if (FP16) return __half2float(__float2half_rn(a));
    return __bfloat162float(__float2bfloat16_rn(a));
}

__device__ __forceinline__ void slot_pair(int s, int& p, int& q) {
    // s = q (q + 1) / 2 + p, 0 <= p <= q
    q = (int)((sqrtf(8.0f * s + 1.0f) - 1.0f) * 0.5f);
    while ((q + 1) * (q + 2) / 2 <= s) ++q;
    while (q * (q + 1) / 2 > s) --q;
    p = s - q * (q + 1) / 2;
}

struct RowPass {
    const float* X;
    float* Y;
    int64_t Nr, Nc;
    const uint4* tslot8;     // [P/8][Nc]: 8 16-bit entries per chunk of 8 slots (slot 8c+u in
                             // half u of the 128-bit word): target string | sign << 15,
                             // Nc when the slot is absent
    const int32_t* rtgt;     // [Nr][rnexc] row-string tables
    const uint16_t* rpq;
    const int8_t* rsgn;
    int rnexc;               // table entries per row string (K of the row's GEMM)
    int KR;                  // rnexc rounded up to 16
    const __half* wrow;      // W by input slot: NW pieces of [P][P] 16-bit (bits of the format)
    int NS, n;
    uint32_t ncols;          // TMEM columns allocated
    const float* amax;       // device max|X| (operand scaling and fixed-point range)
    float wscale;            // power-of-two scale applied to W in the image
    float gbound;            // max over output slots of sum_k |W[k][s]| (unscaled W)
    int nexc_c;              // table entries per column string (contributions per target)
    int* err;
};

constexpr int RP_WARPS = 16;                 // 4 warps per TMEM lane quadrant
constexpr int RP_THREADS = 32 * RP_WARPS;
constexpr int RP_MAXK = 96;                  // largest KR: 9 * 10 = 90 entries rounded up

// P: padded N (multiple of 16); FP16: operand format (else BF16); NW: pieces of W.
// Per row R the K dimension holds R's own table entries e (KR = rnexc rounded up
// to 16): A[J][e] = X[tgt_e, J], and the row's B, B_R[s][e] = sgn_e W[slot(e)][s],
// is gathered from the W image into shared memory (canonical K-major layout
// without swizzle).  MMA passes: A_hi B_j for every piece j, plus A_lo B_0.
//
// Work split: the KR entries form KR/8 chunks of 8 (A build) and the P output
// slots P/8 chunks (scatter); the 4 warps of a lane quadrant take chunks
// round-robin.  Per tile t the CTA waits for MMA(t), copies D(t) into
// registers, issues MMA(t+1), builds A(t+2) into the buffer MMA(t) has finished
// with, starts the asynchronous gather copies of tile t+3 into shared memory
// and scatters D(t).  The gather of a tile is thus in flight for a whole
// iteration, and the scatter's table words, loaded at the start of the
// iteration, arrive during the build.
template <int P, bool FP16, int NW>
__global__ void __launch_bounds__(RP_THREADS, 1) k_rowpass(const RowPass p) {
    constexpr int NCH = P / 8;                     // output chunks of 8 slots
    constexpr int MAXC = (NCH + 3) / 4;            // output chunks per warp (upper bound)
    constexpr int MAXA = (RP_MAXK / 8 + 3) / 4;    // input chunks per warp (upper bound)
    extern __shared__ __align__(1024) unsigned char smem[];
    const int KR = p.KR;
    const int64_t Nc = p.Nc;
    uint8_t* sB = smem;                                               // NW pieces of P x KR
    const uint32_t piece_bytes = (uint32_t)(P * KR * 2);
    int* srow = reinterpret_cast<int*>(smem + NW * piece_bytes);      // Nc + 1, fixed point
    int32_t* rje = srow + (Nc + 1);                                   // [RP_MAXK] source rows
    float* sX = reinterpret_cast<float*>(
        (reinterpret_cast<uintptr_t>(rje + RP_MAXK) + 15) & ~uintptr_t(15));  // [2][KR][128]
    uintptr_t tail = reinterpret_cast<uintptr_t>(sX + 2 * KR * 128);
    uint64_t* mbar = reinterpret_cast<uint64_t*>(tail);
    uint32_t* tmem_holder = reinterpret_cast<uint32_t*>(mbar + 1);
    int* abort_flag = reinterpret_cast<int*>(tmem_holder + 1);

    const int tid = threadIdx.x;
    const int warp = tid >> 5, lane = tid & 31;
    const int quad = warp & 3, wq = warp >> 2;
    const int m = quad * 32 + lane;

    if (tid == 0) {
        mbar_init(mbar, 1);
        *abort_flag = 0;
        fence_mbar_init();
    }
    if (warp == 0) {
        tmem_alloc(tmem_holder, p.ncols);
        tmem_relinquish();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tbase = *tmem_holder;
    const uint32_t lane_base = (uint32_t)(quad * 32) << 16;
    constexpr uint32_t idesc = instr_desc(128, P, !FP16);
    const uint32_t sB_addr = smem_u32(sB);
    const uint32_t sX_addr = smem_u32(sX);
    const uint32_t SBO = 16u * (uint32_t)KR, LBO = 128u;
    const int ntiles = (int)((Nc + 127) / 128);
    const int nchA = KR / 8;
    float sa = 1.f, fx = 1.f;
    {
        const float mx = *p.amax;
        if (mx > 0.f && isfinite(mx)) {
            int e;
            frexpf(mx, &e);  // mx < 2^e; A entries are single values of x
            if (FP16) sa = ldexpf(1.f, 14 - max(e, -90));
            // every target receives nexc_c terms of magnitude <= max|x| gbound
            const float bound = 1.02f * (float)p.nexc_c * mx * p.gbound;
            int f = -90;
            if (bound > 0.f) frexpf(bound, &f);  // bound < 2^f
            fx = ldexpf(1.f, 31 - max(f, -90));
        }
    }
    const float unscale = fx / (sa * p.wscale);   // D -> fixed point
    const float inv_fx = 1.f / fx;
    const uint32_t absent = (uint32_t)Nc;
    uint32_t phase = 0;

    // stage the gather X[tgt_e, J] of tile t for this thread's entry chunks
    // (4-byte cp.async: rows of X are not 16-byte aligned in general)
    auto copies = [&](int t) {
        const int64_t jc = (int64_t)t * 128 + m;
        const bool valid = jc < Nc;
        const uint32_t dst0 = sX_addr + (uint32_t)((t & 1) * KR) * 512u + (uint32_t)m * 4u;
#pragma unroll
        for (int k = 0; k < MAXA; ++k) {
            const int c = wq + 4 * k;
            if (c < nchA) {
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    const int e = c * 8 + u;
                    const int r = rje[e];
                    const bool ok = valid && r >= 0;
                    const float* src = ok ? p.X + (int64_t)r * Nc + jc : p.X;
                    cp_async4(dst0 + (uint32_t)e * 512u, src, ok ? 4u : 0u);
                }
            }
        }
        cp_async_commit();
    };

    // A(t) = split X gather of tile t (staged by copies(t)) -> TMEM buffer buf
    auto build = [&](int t, int buf) {
        const float* xs = sX + (size_t)((t & 1) * KR) * 128 + m;
        const uint32_t a_hi = tbase + lane_base + (uint32_t)(buf * KR);
        const uint32_t a_lo = a_hi + (uint32_t)(KR / 2);
#pragma unroll
        for (int k = 0; k < MAXA; ++k) {
            const int c = wq + 4 * k;
            if (c < nchA) {
                uint32_t hi[4], lo[4];
#pragma unroll
                for (int u = 0; u < 8; u += 2) {
                    const float v0 = xs[(c * 8 + u) * 128] * sa;
                    const float v1 = xs[(c * 8 + u + 1) * 128] * sa;
                    const float h0 = round16<FP16>(v0), h1 = round16<FP16>(v1);
                    hi[u / 2] = pack2<FP16>(h0, h1);
                    lo[u / 2] = pack2<FP16>(v0 - h0, v1 - h1);
                }
                const uint32_t col = (uint32_t)(c * 4);
                tmem_st4(a_hi + col, hi[0], hi[1], hi[2], hi[3]);
                tmem_st4(a_lo + col, lo[0], lo[1], lo[2], lo[3]);
            }
        }
    };

    auto issue = [&](int t) {
        const int buf = t & 1;
        const uint32_t a_hi = tbase + (uint32_t)(buf * KR);
        const uint32_t a_lo = a_hi + (uint32_t)(KR / 2);
        const uint32_t d = tbase + (uint32_t)(2 * KR);
        const int ksteps = KR / 16;
#pragma unroll
        for (int pass = 0; pass < NW + 1; ++pass) {
            // pass 0: A_hi W_0, pass 1: A_lo W_0, pass j+1 (j >= 1): A_hi W_j
            const uint32_t a = (pass == 1) ? a_lo : a_hi;
            const int piece = pass <= 1 ? 0 : pass - 1;
            const uint32_t bbase = sB_addr + (uint32_t)piece * piece_bytes;
            for (int j = 0; j < ksteps; ++j) {
                uint64_t bd = smem_desc(bbase + (uint32_t)(j * 256), LBO, SBO);
                mma_ts(d, a + (uint32_t)(j * 8), bd, idesc, (pass | j) != 0);
            }
        }
        mma_commit(mbar);
    };

    auto load_d = [&](uint32_t (&dr)[MAXC][8]) {
        const uint32_t dcol = tbase + lane_base + (uint32_t)(2 * KR);
#pragma unroll
        for (int k = 0; k < MAXC; ++k) {
            const int c = wq + 4 * k;
            if (c < NCH) tmem_ld8(dcol + (uint32_t)(c * 8), dr[k]);
        }
        tmem_ld_wait();
    };

    auto load_words = [&](int t, uint4 (&w4)[MAXC]) {
        const int64_t jc = (int64_t)t * 128 + m;
        const int64_t jcc = jc < Nc ? jc : Nc - 1;
#pragma unroll
        for (int k = 0; k < MAXC; ++k) {
            const int c = wq + 4 * k;
            if (c < NCH) w4[k] = __ldg(p.tslot8 + (int64_t)c * Nc + jcc);
        }
    };

    auto scatter = [&](int t, const uint32_t (&dr)[MAXC][8], const uint4 (&w4)[MAXC]) {
        const bool valid = (int64_t)t * 128 + m < Nc;
#pragma unroll
        for (int k = 0; k < MAXC; ++k) {
            const int c = wq + 4 * k;
            if (c < NCH) {
                const uint32_t w[4] = {w4[k].x, w4[k].y, w4[k].z, w4[k].w};
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    const uint32_t e = (w[u >> 1] >> (16 * (u & 1))) & 0xFFFFu;
                    const uint32_t tg = e & 0x7FFFu;
                    const int q = __float2int_rn(__uint_as_float(dr[k][u]) * unscale);
                    if (valid && tg != absent) atomicAdd(srow + tg, (e & 0x8000u) ? -q : q);
                }
            }
        }
    };

    auto wait_mma = [&]() {
        if (tid == 0) {
            long long t0 = clock64();
            while (!mbar_try_wait(mbar, phase)) {
                if (clock64() - t0 > WAIT_CYCLES) {
                    *abort_flag = 1;
                    atomicExch(p.err, 1);
                    break;
                }
            }
        }
        phase ^= 1u;
    };

    for (int64_t ir = blockIdx.x; ir < p.Nr; ir += gridDim.x) {
        // row set-up: zero sigma, the row's source rows, and its B (signs folded in)
        for (int64_t j = tid; j <= Nc; j += RP_THREADS) srow[j] = 0;
        for (int e = tid; e < RP_MAXK; e += RP_THREADS)
            rje[e] = e < p.rnexc ? p.rtgt[ir * p.rnexc + e] : -1;
        {
            const uint16_t* wsrc = reinterpret_cast<const uint16_t*>(p.wrow);
            const int tot = NW * P * KR;
            for (int i = tid; i < tot; i += RP_THREADS) {
                const int piece = i / (P * KR);
                const int rem = i % (P * KR);
                const int e = rem / P, nn = rem % P;   // consecutive threads: consecutive nn
                uint16_t v = 0;
                if (e < p.rnexc) {
                    const int g = p.rpq[ir * p.rnexc + e];
                    int a = g / p.n, b = g % p.n;
                    if (a > b) { int t = a; a = b; b = t; }
                    const int sl = b * (b + 1) / 2 + a;
                    v = wsrc[((size_t)piece * P + sl) * P + nn];
                    if (p.rsgn[ir * p.rnexc + e] < 0) v ^= 0x8000u;   // exact negation
                }
                const uint32_t off = (uint32_t)piece * piece_bytes + (uint32_t)(nn / 8) * SBO +
                                     (uint32_t)(e / 8) * 128 + (uint32_t)(nn % 8) * 16 +
                                     (uint32_t)(e % 8) * 2;
                *reinterpret_cast<uint16_t*>(sB + off) = v;
            }
        }
        fence_proxy_async_smem();
        __syncthreads();

        // tiles: copies(t + 3) and build(t + 2) run while MMA(t + 1) does;
        // stage t & 1 holds tile t's gather from copies(t) until build(t)
        copies(0);
        if (ntiles > 1) copies(1);
        if (ntiles > 1) cp_async_wait<1>(); else cp_async_wait<0>();
        build(0, 0);
        tmem_st_wait();
        tc_fence_before();
        __syncthreads();
        if (tid == 0) {
            tc_fence_after();
            issue(0);
        }
        if (ntiles > 1) {
            cp_async_wait<0>();
            build(1, 1);
        }
        if (ntiles > 2) copies(2);
        for (int t = 0; t < ntiles; ++t) {
            uint4 w4[MAXC];
            load_words(t, w4);
            wait_mma();
            __syncthreads();
            if (*abort_flag) break;
            tc_fence_after();
            uint32_t dr[MAXC][8];
            load_d(dr);
            tmem_st_wait();
            tc_fence_before();
            __syncthreads();
            if (t + 1 < ntiles && tid == 0) {
                tc_fence_after();
                issue(t + 1);
            }
            if (t + 2 < ntiles) {
                cp_async_wait<0>();
                build(t + 2, t & 1);
            }
            if (t + 3 < ntiles) copies(t + 3);
            scatter(t, dr, w4);
        }
        cp_async_wait<0>();
        __syncthreads();
        if (*abort_flag) break;
        for (int64_t j = tid; j < Nc; j += RP_THREADS) p.Y[ir * Nc + j] = (float)srow[j] * inv_fx;
        __syncthreads();
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) tmem_dealloc(tbase, p.ncols);
}

// max |x| as float bits (non-negative floats order like unsigned integers)
__global__ void k_absmax(const float* __restrict__ x, int64_t n, unsigned* out) {
    float mx = 0.f;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        mx = fmaxf(mx, fabsf(x[i]));
    for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_down_sync(0xffffffffu, mx, o));
    if ((threadIdx.x & 31) == 0) atomicMax(out, __float_as_uint(mx));
}

// ---------------------------------------------------------------- set-up kernels

// W image by input slot: NW pieces of a P x P row-major array of 16-bit values,
// element (s_in, s_out) = piece j of W[s_in][s_out] = (pq|rs) (scaled by the
// power of two wscale), piece j = round(W - sum_{i<j} piece_i).
template <bool FP16>
__global__ void k_wimg(const double* __restrict__ eri, int n, int P, int NS, int NW,
                       uint16_t* __restrict__ img, double wscale) {
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= P * P) return;
    const int si = idx / P, so = idx % P;
    double w = 0.0;
    if (si < NS && so < NS) {
        int pi, qi, po, qo;
        slot_pair(si, pi, qi);
        slot_pair(so, po, qo);
        w = eri[(((int64_t)pi * n + qi) * n + po) * n + qo];
    }
    w *= wscale;
    double rest = w;
    for (int j = 0; j < NW; ++j) {
        uint16_t bits;
        double part;
        if (FP16) {
            __half h = __double2half(rest);
            part = (double)__half2float(h);
            bits = *reinterpret_cast<uint16_t*>(&h);
        } else {
            __nv_bfloat16 h = __double2bfloat16(rest);
            part = (double)__bfloat162float(h);
            bits = *reinterpret_cast<uint16_t*>(&h);
        }
        img[(size_t)j * P * P + idx] = bits;
        rest -= part;
    }
}

// slot table: for string j and its entry (pq -> tgt, sgn), slot s = {p,q} holds
// tgt | (sgn < 0) << 15; slots without an entry hold ns.  Stored per chunk of 8
// slots: the 128-bit word (s/8, j) holds slots 8*(s/8) .. 8*(s/8)+7, slot s in
// 16-bit half s%8.
__global__ void k_slot_fill(uint16_t* __restrict__ tslot, int64_t count, uint16_t v) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count;
         i += (int64_t)gridDim.x * blockDim.x)
        tslot[i] = v;
}

__global__ void k_slot_table(const int32_t* __restrict__ tgt, const uint16_t* __restrict__ pq,
                             const int8_t* __restrict__ sgn, int64_t ns, int nexc, int n,
                             uint16_t* __restrict__ tslot) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= ns * nexc) return;
    const int64_t j = i / nexc;
    int a = pq[i] / n, b = pq[i] % n;
    if (a > b) { int t = a; a = b; b = t; }
    const int s = b * (b + 1) / 2 + a;
    tslot[((int64_t)(s >> 3) * ns + j) * 8 + (s & 7)] =
        (uint16_t)(tgt[i] | (sgn[i] < 0 ? 0x8000 : 0));
}

uint32_t tmem_cols(int P, int KR) {
    uint32_t need = (uint32_t)(2 * KR + P), c = 32;
    while (c < need) c <<= 1;
    return c;
}

size_t rowpass_smem(int P, int NW, int KR, int64_t Nc) {
    return (size_t)2 * NW * P * KR + 4 * (size_t)(Nc + 1) + 4 * RP_MAXK + 16 +
           (size_t)2 * KR * 128 * 4 + 64;
}

template <int P>
void* rowpass_fn(bool fp16) {
    return fp16 ? (void*)k_rowpass<P, true, 3> : (void*)k_rowpass<P, false, 2>;
}

void* rowpass_kernel(int P, bool fp16) {
    switch (P) {
        case 16: return rowpass_fn<16>(fp16);
        case 32: return rowpass_fn<32>(fp16);
        case 48: return rowpass_fn<48>(fp16);
        case 64: return rowpass_fn<64>(fp16);
        case 80: return rowpass_fn<80>(fp16);
        case 96: return rowpass_fn<96>(fp16);
        case 112: return rowpass_fn<112>(fp16);
        case 128: return rowpass_fn<128>(fp16);
        case 144: return rowpass_fn<144>(fp16);
        default: return nullptr;
    }
}

}  // namespace

void TcSigma::init(const SpinTables& A, const SpinTables& B, const double* d_h1,
                   const double* d_eri, int norb, double wmax, double wcolsum, bool use_fp16,
                   cudaStream_t st) {
    ta = &A;
    tb = &B;
    n = norb;
    NS = n * (n + 1) / 2;
    P = ((NS + 1 + 15) / 16) * 16;
    nsa = A.ns;
    nsb = B.ns;
    dim = nsa * nsb;
    fp16 = use_fp16;
    nw = fp16 ? 3 : 2;
    kernel = rowpass_kernel(P, fp16);
    KR = ((A.nexc + 15) / 16) * 16;
    if (!kernel || KR > RP_MAXK || tmem_cols(P, KR) > 512 || A.ns > 32766 || B.ns > 32766)
        KPM_THROW(KPM_EUNSUPPORTED, "tensor-core sigma supports up to 16 orbitals");
    int dev = 0;
    KPM_CUDA(cudaGetDevice(&dev));
    cudaDeviceProp prop;
    KPM_CUDA(cudaGetDeviceProperties(&prop, dev));
    if (prop.major != 10)
        KPM_THROW(KPM_EUNSUPPORTED, "tensor-core sigma needs a Blackwell (sm_10x) GPU");
    nsm = prop.multiProcessorCount;
    gbound = (float)(wcolsum * (1.0 + 1e-6));
    int64_t ncmax = nsa > nsb ? nsa : nsb;
    smem_bytes = rowpass_smem(P, nw, KR, ncmax);
    // at least ~116 KB so that exactly one CTA (and one TMEM allocation) fits per SM
    size_t floor_bytes = 116 * 1024;
    if (smem_bytes < floor_bytes) smem_bytes = floor_bytes;
    if (smem_bytes > (size_t)prop.sharedMemPerBlockOptin)
        KPM_THROW(KPM_EUNSUPPORTED, "tensor-core sigma: rows of %lld strings need %zu B of shared memory",
                  (long long)ncmax, smem_bytes);
    KPM_CUDA(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)smem_bytes));
    // W scaled by a power of two so that |W| < 2^14 (FP16 range); BF16 needs none
    wscale = 1.0f;
    if (fp16 && wmax > 0.0) {
        int e;
        std::frexp(wmax, &e);
        wscale = std::ldexp(1.0f, 14 - e);
    }
    size_t wbytes = (size_t)2 * nw * P * P;
    wimg.alloc(wbytes);
    KPM_CUDA(cudaMemsetAsync(wimg.p, 0, wbytes, st));
    if (fp16)
        k_wimg<true><<<(P * P + 255) / 256, 256, 0, st>>>(d_eri, n, P, NS, nw,
                                                          wimg.as<uint16_t>(), (double)wscale);
    else
        k_wimg<false><<<(P * P + 255) / 256, 256, 0, st>>>(d_eri, n, P, NS, nw,
                                                           wimg.as<uint16_t>(), (double)wscale);
    KPM_LAUNCHED();

    auto build_slots = [&](const SpinTables& T, DevBuf& out) {
        size_t count = (size_t)P * T.ns;
        out.alloc(count * sizeof(uint16_t));
        k_slot_fill<<<1024, 256, 0, st>>>(out.as<uint16_t>(), (int64_t)count, (uint16_t)T.ns);
        KPM_LAUNCHED();
        int64_t ne = T.ns * T.nexc;
        if (ne > 0) {
            k_slot_table<<<(unsigned)((ne + 255) / 256), 256, 0, st>>>(
                T.tgt.as<int32_t>(), T.pq.as<uint16_t>(), T.sgn.as<int8_t>(), T.ns, T.nexc, n,
                out.as<uint16_t>());
            KPM_LAUNCHED();
        }
    };
    build_slots(B, slot_b);
    err.alloc(sizeof(int));
    amax.alloc(2 * sizeof(unsigned));
    KPM_CUDA(cudaMemsetAsync(err.p, 0, sizeof(int), st));
    dense.init(A, B, &A == &B, err.as<int>(), st);
}

void TcSigma::apply(const float* x, float* y, int ncol, cudaStream_t st) {
    const uint32_t nc = tmem_cols(P, KR);
    for (int c = 0; c < ncol; ++c) {
        const float* X = x + (size_t)c * dim;
        float* Y = y + (size_t)c * dim;
        // max|x|: FP16 operand scales and the fixed-point range of the scatter
        KPM_CUDA(cudaMemsetAsync(amax.p, 0, sizeof(unsigned), st));
        k_absmax<<<1024, 256, 0, st>>>(X, dim, amax.as<unsigned>());
        KPM_LAUNCHED();
        const float* am = reinterpret_cast<const float*>(amax.p);
        // opposite-spin part: rows alpha, columns beta; writes Y
        RowPass p1{X, Y, nsa, nsb, slot_b.as<uint4>(),
                   ta->tgt.as<int32_t>(), ta->pq.as<uint16_t>(), ta->sgn.as<int8_t>(), ta->nexc,
                   KR, wimg.as<__half>(), NS, n, nc, am, wscale, gbound, tb->nexc, err.as<int>()};
        int g1 = (int)(nsa < nsm ? nsa : nsm);
        void* args1[] = {&p1};
        KPM_CUDA(cudaLaunchKernel(kernel, dim3(g1), dim3(RP_THREADS), args1, smem_bytes, st));
        KPM_LAUNCHED();
        // same-spin parts (dense GEMMs) and the exact diagonal, added into Y
        dense.apply(X, Y, am, st);
    }
}

int TcSigma::check(cudaStream_t st) {
    int h = 0;
    KPM_CUDA(cudaMemcpyAsync(&h, err.p, sizeof(int), cudaMemcpyDeviceToHost, st));
    KPM_CUDA(cudaStreamSynchronize(st));
    if (h) KPM_CUDA(cudaMemsetAsync(err.p, 0, sizeof(int), st));
    return h;
}

}  // namespace kpm
