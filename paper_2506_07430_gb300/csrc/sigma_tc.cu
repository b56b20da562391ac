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
// GEMM per tile: M = 128 columns J, K = KR (the row's off-diagonal entries plus
// one column for its diagonal entries, rounded up to 16), N = P (NS + 1 rounded
// up to 16), operands in shared memory, D in tensor memory (FP32).  x and W are
// split into NW = 2 16-bit pieces each (FP16 with power-of-two scales, or BF16);
// the MMAs A_hi B_j (every piece j of W) and A_lo B_0 drop only A_lo B_1, below
// 2^-22 relative.  The epilogue reads D
// (tcgen05.ld) and scatters into the row's sigma in shared memory with 32-bit
// fixed-point integer atomics (order-independent, so the result is
// reproducible bit for bit).  One CTA per SM, persistent over rows; the kernel
// comment of k_rowpass gives the pipeline.  Every wait on an mbarrier is
// bounded (about two seconds); on expiry the kernel records an error, frees
// its tensor memory and returns.
#include "sigma_tc.cuh"

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <array>
#include <cmath>
#include <map>
#include <mutex>

namespace kpm {

namespace {

constexpr long long WAIT_CYCLES = 4000000000LL;  // ~2 s at 2 GHz
constexpr long long STALL_WAIT_CYCLES = 20000000LL;  // ~10 ms: the stall test's limit

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
__device__ __forceinline__ void tmem_ld8(uint32_t taddr, uint32_t (&r)[8]) {
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]),
                   "=r"(r[6]), "=r"(r[7])
                 : "r"(taddr)
                 : "memory");
}
__device__ __forceinline__ void tmem_ld4(uint32_t taddr, uint32_t (&r)[8]) {
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0, %1, %2, %3}, [%4];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(taddr)
                 : "memory");
}
__device__ __forceinline__ void tmem_ld_wait() {
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}
// D[tmem] (+)= A[smem] * B[smem]^T, kind::f16 (BF16 or FP16 operands, FP32 accumulate)
__device__ __forceinline__ void mma_ss(uint32_t d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                       uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}"
        ::"r"(d), "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate) : "memory");
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
__device__ __forceinline__ void cp_async_commit() {
    asm volatile("cp.async.commit_group;" ::: "memory");
}
template <int N>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}
// hint: bring `bytes` (multiple of 16, 16-byte aligned) at p into L2
__device__ __forceinline__ void prefetch_l2(const void* p, uint32_t bytes) {
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"(bytes) : "memory");
}

// Shared-memory matrix descriptor, canonical layouts without swizzle: 8 x 16-byte
// core matrices (128 contiguous bytes); LBO = byte distance between core
// matrices adjacent along K, SBO = between core matrices adjacent along M/N.
// K-major: a core matrix row is 8 K-consecutive elements of one M/N index;
// MN-major: 8 M/N-consecutive elements of one K index.
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
    d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1 << 46;  // descriptor version for tcgen05
    return d;                // base offset 0, swizzle none
}

// Instruction descriptor, kind::f16: D = F32, A/B = BF16 (1) or F16 (0), both
// K-major (bit 15 set: A MN-major), N >> 3 at bit 17, M >> 4 at bit 24.
__host__ __device__ constexpr uint32_t instr_desc(int M, int N, bool bf16) {
    return (1u << 4) | ((bf16 ? 1u : 0u) << 7) | ((bf16 ? 1u : 0u) << 10) |
           ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void slot_pair(int s, int& p, int& q) {
    // s = q (q + 1) / 2 + p, 0 <= p <= q
    q = (int)((sqrtf(8.0f * s + 1.0f) - 1.0f) * 0.5f);
    while ((q + 1) * (q + 2) / 2 <= s) ++q;
    while (q * (q + 1) / 2 > s) --q;
    p = s - q * (q + 1) / 2;
}

struct RowPass {
    const uint16_t* Xh;      // x split into 16-bit pieces (bits of the format), [Nr][xpitch],
    const uint16_t* Xl;      // scaled by sa(amax); columns [Nc, xpitch) hold zeros
    int64_t xpitch;          // multiple of 128
    float* Y;
    int64_t Nr, Nc;
    const uint4* tslot8;     // [P/8][Nc]: 8 16-bit entries per chunk of 8 slots (slot 8c+u in
                             // half u of the 128-bit word): target string | sign << 15,
                             // Nc + (J mod 32) when the slot of column J is absent
    const int32_t* rtgt;     // [Nr][rnexc] row-string targets of the off-diagonal entries
    const uint16_t* rslot;   // [Nr][rnexc] their slot | sign << 15
    int rnexc;               // off-diagonal table entries per row string, m (n - m)
    int ndiag;               // 1 if the row strings hold electrons (a diagonal column), else 0
    int KR;                  // K of the row GEMM: rnexc + ndiag rounded up to 16 (at least 16)
    const uint32_t* rmask;   // [Nr] occupation masks of the row strings
    const double* wdiag;     // [n][P] W[qq][s] (unscaled, FP64; zero for diagonal slots s)
    const uint16_t* wrow;    // W by input slot: NW pieces of [P][P] 16-bit (bits of the format)
    uint32_t ncols;          // TMEM columns allocated
    const float* amax;       // device max|x| (operand scaling)
    const float* rowmax;     // [Nr] max |x| of each row (per-row fixed-point range)
    float wscale;            // power-of-two scale applied to W in the image
    int nexc_c;              // table entries per column string (contributions per target)
    int NS;                  // slots in use (n(n+1)/2); slots [NS, P) are padding
    int nst;                 // A stages in shared memory (2 or 3)
    int prefetch;            // L2 prefetch of the A rows this many tiles ahead (0: none)
    // wide layout (more than 32736 column strings, or a row's sigma beyond shared
    // memory): 16-bit targets without the sign (absent: 0xFFFF), the sign taken from
    // the column string's occupations, and the targets split into npass ranges of
    // span strings, one pass over the row's tiles per range
    int npass;
    int64_t span;
    const uint32_t* cmask;   // [Nc] occupation masks of the column strings (wide layout)
    int* err;
    long long wait_cycles;   // limit of every mbarrier wait (clock64 cycles)
    int stall;               // test of the bounded waits: the MMA thread issues nothing, so
                             // the other roles' waits run out and the kernel reports it
};

constexpr int RP_SCATTER_WARPS = 16;         // 4 per TMEM lane quadrant
#ifndef RP_COPY_WARPS_N
#define RP_COPY_WARPS_N 3
#endif
constexpr int RP_COPY_WARPS = RP_COPY_WARPS_N;   // cp.async producers (warps 16 ...)
constexpr int RP_MMA_WARP = RP_SCATTER_WARPS + RP_COPY_WARPS;   // MMA issue (one thread)
constexpr int RP_WARPS = RP_SCATTER_WARPS + RP_COPY_WARPS + 1;
constexpr int RP_THREADS = 32 * RP_WARPS;
constexpr int RP_MAXK = 96;                  // largest KR: 9 * 10 = 90 entries rounded up
static_assert(RP_COPY_WARPS * 32 >= RP_MAXK, "one copy lane per entry (L2 prefetch)");
// sink cells after the row's sigma: an absent slot of column J targets cell
// Nc + (J mod 32), so the scatter adds every slot without a branch and the 32
// lanes of a warp (32 consecutive J) sink into 32 different banks
constexpr int RP_SINK = 32;
// poll interval of the copy and MMA warps' waits (the MMA of tile t + 1 has
// about one scatter duration of slack, microseconds), and of the scatter warps'
// wait for D
#ifndef RP_BACKOFF_NS
#define RP_BACKOFF_NS 256
#endif
#ifndef RP_SCATTER_BACKOFF_NS
#define RP_SCATTER_BACKOFF_NS 64
#endif
constexpr uint32_t A_LBO = 2048;             // A stage: K-group (8 entries) stride, bytes
constexpr uint32_t A_SBO = 128;              // A stage: MN-group (8 columns) stride, bytes

// operand scale of x (power of two): FP16 pieces of x * sa stay below 2^15
__device__ __forceinline__ float x_scale(float mx, bool fp16) {
    if (!fp16 || !(mx > 0.f) || !isfinite(mx)) return 1.f;
    int e;
    frexpf(mx, &e);  // mx < 2^e
    return ldexpf(1.f, 14 - max(e, -90));
}

// value -> NW 16-bit pieces, each the rounding of what the previous ones left
template <bool FP16, int NW>
__device__ __forceinline__ void split16(double v, uint16_t (&out)[NW]) {
#pragma unroll
    for (int j = 0; j < NW; ++j) {
        double part;
        if (FP16) {
            const __half h = __double2half(v);
            out[j] = __half_as_ushort(h);
            part = (double)__half2float(h);
        } else {
            const __nv_bfloat16 h = __double2bfloat16(v);
            out[j] = __bfloat16_as_ushort(h);
            part = (double)__bfloat162float(h);
        }
        v -= part;
    }
}

template <bool FP16>
__device__ __forceinline__ float f16bits(uint16_t bits) {
    if (FP16) return __half2float(__ushort_as_half(bits));
    return __bfloat162float(__ushort_as_bfloat16(bits));
}

template <bool FP16>
__device__ __forceinline__ uint16_t scale16(uint16_t bits, float sc) {
    if (FP16) {
        __half h = __float2half_rn(__half2float(__ushort_as_half(bits)) * sc);
        return __half_as_ushort(h);
    } else {
        __nv_bfloat16 h = __float2bfloat16_rn(__bfloat162float(__ushort_as_bfloat16(bits)) * sc);
        return __bfloat16_as_ushort(h);
    }
}


__device__ __forceinline__ void tmem_ld2(uint32_t taddr, uint32_t& r0, uint32_t& r1) {
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x2.b32 {%0, %1}, [%2];"
                 : "=r"(r0), "=r"(r1)
                 : "r"(taddr)
                 : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* mbar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(mbar)) : "memory");
}

// try_wait that may suspend the thread for up to ~hint_ns until the phase completes
__device__ __forceinline__ bool mbar_try_wait_sleep(uint64_t* mbar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(mbar)), "r"(parity), "r"(100000u)
        : "memory");
    return ok != 0;
}

// Bounded wait on an mbarrier phase; false (and the CTA's abort flag set) when
// the wait ran out or another role has aborted.  try_wait's suspension ends
// long before its time hint (tens of cycles), so a waiting warp would still
// take a large share of its sub-partition's issue slots from the scatter warps;
// roles off the critical path sleep backoff_ns between polls.
__device__ __forceinline__ bool wait_phase(uint64_t* mbar, uint32_t parity, volatile int* abort_flag,
                                           int* err, long long limit, unsigned backoff_ns = 0) {
    const long long t0 = clock64();
    while (!mbar_try_wait_sleep(mbar, parity)) {
        if (backoff_ns) __nanosleep(backoff_ns);
        if (*abort_flag) return false;
        if (clock64() - t0 > limit) {
            *abort_flag = 1;
            atomicExch(err, 1);
            return false;
        }
    }
    return true;
}

// P: padded N (multiple of 16); FP16: operand format (else BF16); NW: pieces of W.
//
// Row R's GEMM: D[J][s] = sum_e A[J][e] B_R[s][e], K = the row's table entries
// e (KR = rnexc rounded up to 16), A[J][e] = x[tgt_e][J] (x pre-split into
// 16-bit hi/lo pieces), B_R[s][e] = sgn_e W[slot(e)][s] bscale.  bscale folds
// the operand scales and the fixed-point factor into B, so D is already the
// fixed-point value and the scatter only rounds it to an integer.
//
// A is staged in shared memory in the canonical MN-major layout without
// swizzle (8 columns x 8 entries per 128-byte core matrix; MN-group stride
// A_SBO, K-group stride A_LBO) by 16-byte cp.async copies straight from the
// split rows of x, nst (3, else 2) stages deep; B_R is gathered once per row
// (canonical K-major layout without swizzle).  MMA passes: A_hi B_j for every
// piece j of W, plus A_lo B_0; D accumulates in tensor memory, two buffers deep.
//
// Warp roles, synchronised per tile by mbarriers only (the copy and MMA warps
// poll theirs with a sleep in between, leaving the issue slots to the scatter):
//   copy (warps 16-18, a third of the copies each): copies of tile t into
//     stage t % nst once MMA(t - nst) has released it; once they have landed
//     (and been fenced for the async proxy), each arrives on "A full"; with
//     them, one lane per entry prefetches that entry's rows of tile
//     t + p.prefetch into L2 (a quarter of the gathered segments miss L2);
//   MMA (warp 19, one thread): MMA(t) once A(t) is full and the scatter warps
//     have released D buffer t & 1; tcgen05.commit then signals "stage free"
//     and "D full";
//   scatter (warps 0-15, 4 per TMEM lane quadrant, one column J per thread):
//     wait for D(t), copy it to registers, release the D buffer, and add every
//     slot into the row's sigma in shared memory with 32-bit fixed-point
//     atomics (order-independent: bitwise reproducible; an absent slot adds
//     into the lane's sink cell after the row, so there is no branch).  The 4
//     warps of a quadrant share the NS used slots evenly (chunks of 8
//     round-robin, the remaining chunks split in pairs of slots).
// Rows are separated by CTA barriers (set-up of the next row's B_R and sigma).
//
// Fixed-point range: integer addition wraps, so only each final row sum has to
// fit in 32 bits, and it does whenever every term |D| < 2^31 / nexc_c.  Per row
// R, |D[J][s]| <= c_s = sum_e rowmax(tgt_e) |B[s][e]| / fx (rowmax: max |x| of a
// source row), which sets the row's scale fx (a power of two; capped so that B_R
// stays in the FP16 range); vectors with small or empty source rows get a
// correspondingly finer step.
//
// The row's m diagonal entries E_qq (q in R) all read source row R itself with
// sign +1, so they share one K column: A = x[R][J], B = w_R[s] = sum_{q in R}
// W[qq][s], formed in FP64 and split into NW pieces.  The block of W where both
// excitations are diagonal ((pp|qq)) is zero in the image and in w_R: that part
// of the diagonal of H is added exactly by the same-spin GEMM's epilogue.
template <int P, bool FP16, int NW, bool WIDE>
__global__ void __launch_bounds__(RP_THREADS, 1) k_rowpass(const RowPass p) {
    constexpr int MAXF = P >= 32 ? P / 32 : 1;     // full chunks per scatter warp (upper bound)
    extern __shared__ __align__(1024) unsigned char smem[];
    const int KR = p.KR;
    const int64_t Nc = p.Nc;
    const uint32_t a_piece = (uint32_t)KR * 256u;                     // one piece of one stage
    const uint32_t nst = (uint32_t)p.nst;
    uint8_t* sA = smem;                                               // [nst stages][2 pieces]
    uint8_t* sB = smem + 2 * nst * a_piece;                           // NW pieces of P x KR
    const uint32_t b_piece = (uint32_t)(P * KR * 2);
    // targets held per pass: all Nc, or a span of them (wide layout)
    const int64_t Nrow = WIDE ? p.span : Nc;
    int* srow = reinterpret_cast<int*>(sB + NW * b_piece);            // Nrow + RP_SINK, fixed point
    int64_t* rowoff = reinterpret_cast<int64_t*>(
        (reinterpret_cast<uintptr_t>(srow + Nrow + RP_SINK) + 15) & ~uintptr_t(15));  // [RP_MAXK]
    uint16_t* rsl = reinterpret_cast<uint16_t*>(rowoff + RP_MAXK);    // [RP_MAXK]
    float* rmx = reinterpret_cast<float*>(
        (reinterpret_cast<uintptr_t>(rsl + RP_MAXK) + 15) & ~uintptr_t(15));  // [RP_MAXK]
    float* rsc = rmx + RP_MAXK;                                       // [4] row scales
    unsigned* rred = reinterpret_cast<unsigned*>(rsc + 4);            // [2] row reductions
    double* wdg = reinterpret_cast<double*>(
        (reinterpret_cast<uintptr_t>(rred + 2) + 15) & ~uintptr_t(15));  // [P] w_R (FP64)
    uint32_t* bm = reinterpret_cast<uint32_t*>(wdg + P);   // [P] orbitals strictly inside slot s
    uintptr_t tail = (reinterpret_cast<uintptr_t>(bm + P) + 15) & ~uintptr_t(15);
    uint64_t* afree = reinterpret_cast<uint64_t*>(tail);   // [3] stage s free (MMA done)
    uint64_t* afull = afree + 3;                           // [3] stage s copied
    uint64_t* dfull = afree + 6;                           // [2] D buffer d written
    uint64_t* dfree = afree + 8;                           // [2] D buffer d read (16 warps)
    uint32_t* tmem_holder = reinterpret_cast<uint32_t*>(afree + 10);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_holder + 1);

    const int tid = threadIdx.x;
    const int warp = tid >> 5, lane = tid & 31;

    if (tid == 0) {
        for (int i = 0; i < 3; ++i) {
            mbar_init(afree + i, 1);
            mbar_init(afull + i, RP_COPY_WARPS);
        }
        for (int i = 0; i < 2; ++i) {
            mbar_init(dfull + i, 1);
            mbar_init(dfree + i, RP_SCATTER_WARPS);
        }
        *abort_flag = 0;
        fence_mbar_init();
    }
    if (WIDE) {
        // slot s = {a, b}, a < b: the sign of its excitation on a string is the parity
        // of the string's occupations strictly between a and b (tables.cu)
        for (int sl = tid; sl < P; sl += RP_THREADS) {
            int a = 0, b = 0;
            if (sl < p.NS) slot_pair(sl, a, b);
            bm[sl] = (sl < p.NS && a < b) ? (((1u << b) - 1u) & ~((2u << a) - 1u)) : 0u;
        }
    }
    if (warp == 0) {
        tmem_alloc(tmem_holder, p.ncols);
        tmem_relinquish();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tbase = *tmem_holder;
    constexpr uint32_t idesc = instr_desc(128, P, !FP16) | (1u << 15);  // A MN-major
    const uint32_t sA_addr = smem_u32(sA), sB_addr = smem_u32(sB);
    const uint32_t SBO_B = 16u * (uint32_t)KR;
    const int ntiles = (int)((Nc + 127) / 128);
    const float sa = x_scale(*p.amax, FP16);
    const int64_t nrows = p.Nr;
    const int ncolk = p.rnexc + p.ndiag;                   // K columns in use

    // scatter geometry (warps 0-15): used chunks of 8 slots, full chunks per
    // warp, and the remainder shared out two slots at a time
    const int quad = warp & 3, wq = (warp >> 2) & 3;
    const int m = quad * 32 + lane;
    const int nchr = (p.NS + 7) / 8;
    const int nfull = nchr / 4;
    const int rem = nchr - 4 * nfull;                      // 0..3 chunks -> 2 rem slots per warp
    const int tail0 = nfull * 32 + wq * 2 * rem;           // first remainder slot of this warp

    // tiles processed by this CTA over all rows: tile g uses A stage g % nst
    // (the k-th use of a stage completes its barriers' phase k, parity k & 1)
    // and D buffer g & 1
    uint32_t g = 0;

    // work items: (row, pass over a range of targets); one pass per row unless wide
    const int npass = WIDE ? p.npass : 1;
    for (int64_t idx = blockIdx.x; idx < nrows * npass; idx += gridDim.x) {
        const int64_t ir = WIDE ? idx / npass : idx;
        const int64_t lo = WIDE ? (idx - ir * npass) * Nrow : 0;   // first target of the pass
        // ---- row set-up: zero sigma; the row's source rows, slots and signs; B_R
        if (tid == 0) {
            rred[0] = 0u;
            rred[1] = 0u;
        }
        for (int64_t j = tid; j < Nrow + RP_SINK; j += RP_THREADS) srow[j] = 0;
        for (int e = tid; e < RP_MAXK; e += RP_THREADS) {
            // off-diagonal entries, then the diagonal column (marker 0xFFFE), then padding
            if (e < p.rnexc) {
                const int32_t t = p.rtgt[ir * p.rnexc + e];
                rowoff[e] = (int64_t)t * p.xpitch;
                rsl[e] = p.rslot[ir * p.rnexc + e];
                rmx[e] = p.rowmax[t];
            } else if (e < ncolk) {
                rowoff[e] = ir * p.xpitch;
                rsl[e] = (uint16_t)0xFFFEu;
                rmx[e] = p.rowmax[ir];
            } else {
                rowoff[e] = -1;
                rsl[e] = (uint16_t)0xFFFFu;
                rmx[e] = 0.f;
            }
        }
        __syncthreads();
        // w_R[s] in FP64; this row's fixed-point range c_s (in units of the W image;
        // piece 0 of W is within 2^-8 of W in either format: 1 % margin) and max |B|
        if (tid < P) {
            double wr = 0.0;
            for (uint32_t mk = __ldg(p.rmask + ir); mk; mk &= mk - 1)
                wr += __ldg(p.wdiag + (size_t)(__ffs(mk) - 1) * P + tid);
            wdg[tid] = wr;
            const float wrs = (float)fabs(wr) * p.wscale;
            float c = p.ndiag ? rmx[p.rnexc] * wrs : 0.f, wm = p.ndiag ? wrs : 0.f;
            for (int e = 0; e < p.rnexc; ++e) {
                const float w = fabsf(f16bits<FP16>(__ldg(p.wrow + (size_t)(rsl[e] & 0x7FFFu) * P + tid)));
                c = fmaf(rmx[e], w, c);
                wm = fmaxf(wm, w);
            }
            atomicMax(rred, __float_as_uint(c));
            atomicMax(rred + 1, __float_as_uint(wm));
        }
        __syncthreads();
        if (tid == 0) {
            const float cmax = __uint_as_float(rred[0]) / p.wscale * 1.01f;
            const float wmax = __uint_as_float(rred[1]) / p.wscale * 1.01f;
            // each target receives at most nexc_c terms of magnitude <= cmax
            const float bound = 1.02f * (float)p.nexc_c * cmax;
            float fx = 1.f;
            if (bound > 0.f && isfinite(bound)) {
                int f;
                frexpf(bound, &f);  // bound < 2^f
                fx = ldexpf(1.f, 31 - max(f, -90));
                // B_R = W fx / sa stays below 2^15 in FP16
                if (FP16 && wmax > 0.f) {
                    const float lim = 30000.f * sa / wmax;
                    while (fx > lim) fx *= 0.5f;
                }
            }
            rsc[0] = fx;
            rsc[1] = fx / (sa * p.wscale);
            rsc[2] = 1.f / fx;
        }
        __syncthreads();
        const float bscale_r = rsc[1];
        // B_R[s][e] = sgn_e W[slot e][s] bscale (NW pieces, canonical K-major layout
        // without swizzle); the diagonal column from w_R in FP64
        for (int i = tid; i < KR * P; i += RP_THREADS) {
            const int e = i / P, nn = i - (i / P) * P;
            const uint16_t r = rsl[e];
            uint16_t v[NW];
            if (r == 0xFFFEu) {
                split16<FP16, NW>(wdg[nn] * (double)p.wscale * (double)bscale_r, v);
            } else {
#pragma unroll
                for (int j = 0; j < NW; ++j) {
                    v[j] = 0;
                    if (r != 0xFFFFu) {
                        v[j] = scale16<FP16>(__ldg(p.wrow + (size_t)j * P * P +
                                                   (size_t)(r & 0x7FFFu) * P + nn), bscale_r);
                        v[j] ^= (uint16_t)(r & 0x8000u);   // exact negation
                    }
                }
            }
            const uint32_t off = (uint32_t)(nn >> 3) * SBO_B + (uint32_t)(e >> 3) * 128u +
                                 (uint32_t)(nn & 7) * 16u + (uint32_t)(e & 7) * 2u;
#pragma unroll
            for (int j = 0; j < NW; ++j) *reinterpret_cast<uint16_t*>(sB + j * b_piece + off) = v[j];
        }
        fence_proxy_async_smem();
        __syncthreads();

        if (warp >= RP_SCATTER_WARPS && warp < RP_MMA_WARP) {
            // ---- copies: (piece, K-group) pairs u < KR / 4, u = cw + RP_COPY_WARPS i
            // for copy warp cw; per pair this lane copies entry kc * 8 + (lane & 7),
            // column groups (lane >> 3) + 4 v, v < 4
            constexpr int MAXU = (RP_MAXK / 4 + RP_COPY_WARPS - 1) / RP_COPY_WARPS;
            const int cw = warp - RP_SCATTER_WARPS;
            const int eo = lane & 7, g0 = lane >> 3;
            const int nu = KR / 4, kpg = KR / 8;
            int64_t so[MAXU];                       // element offset in the piece, -1: padding
                                                    // (beyond 2^31 at 18 orbitals)
#pragma unroll
            for (int i = 0; i < MAXU; ++i) {
                const int u = cw + RP_COPY_WARPS * i;
                so[i] = -1;
                if (u < nu) {
                    const int kc = u < kpg ? u : u - kpg;
                    const int64_t ro = rowoff[kc * 8 + eo];
                    so[i] = ro >= 0 ? ro + 8 * g0 : -1;
                }
            }
            auto copies = [&](int t, uint32_t stage) {
                const int32_t j0 = t * 128;
                const uint32_t st = sA_addr + stage * 2u * a_piece + (uint32_t)g0 * A_SBO +
                                    (uint32_t)eo * 16u;
#pragma unroll
                for (int i = 0; i < MAXU; ++i) {
                    const int u = cw + RP_COPY_WARPS * i;
                    if (u < nu) {
                        const bool lo = u >= kpg;
                        const int kc = lo ? u - kpg : u;
                        const uint16_t* base = lo ? p.Xl : p.Xh;
                        const bool ok = so[i] >= 0;
                        const uint16_t* src = base + (ok ? so[i] + j0 : 0);
                        const uint32_t dst = st + (lo ? a_piece : 0u) + (uint32_t)kc * A_LBO;
                        const uint32_t nb = ok ? 16u : 0u;
#pragma unroll
                        for (int v = 0; v < 4; ++v) {
                            // column groups g0 + 4 v: 32 elements apart in x, 4 core matrices in A
                            asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;"
                                         ::"r"(dst + (uint32_t)v * 4u * A_SBO),
                                         "l"(src + (ok ? 32 * v : 0)), "r"(nb) : "memory");
                        }
                    }
                }
                cp_async_commit();
            };
            // copies of tile gi have landed: make them visible to the tensor core
            auto publish = [&](uint32_t gi, bool newest_pending) {
                if (newest_pending) cp_async_wait<1>(); else cp_async_wait<0>();
                fence_proxy_async_smem();
                __syncwarp();
                if (lane == 0) mbar_arrive(afull + gi % nst);
            };
            bool ok = true;
            for (int t = 0; t < ntiles && ok; ++t) {
                const uint32_t gt = g + (uint32_t)t;
                if (gt >= nst) {
                    // stage gt % nst is free once MMA(gt - nst) has completed
                    if (lane == 0)
                        ok = wait_phase(afree + gt % nst, (gt / nst - 1) & 1u, abort_flag, p.err,
                                        p.wait_cycles, RP_BACKOFF_NS);
                    ok = __shfl_sync(0xffffffffu, ok ? 1 : 0, 0) != 0;
                    if (!ok) break;
                }
                copies(t, gt % nst);
                if (p.prefetch > 0 && t + p.prefetch < ntiles) {
                    // entry cw * 32 + lane: both pieces of its 128 columns (256 bytes each)
                    const int e = cw * 32 + lane;
                    const int64_t ro = e < KR ? rowoff[e] : -1;
                    if (ro >= 0) {
                        const int64_t off = ro + (int64_t)(t + p.prefetch) * 128;
                        prefetch_l2(p.Xh + off, 256u);
                        prefetch_l2(p.Xl + off, 256u);
                    }
                }
                if (t >= 1) publish(gt - 1, true);
            }
            if (ok && ntiles > 0) publish(g + (uint32_t)ntiles - 1, false);
            cp_async_wait<0>();
        } else if (warp == RP_MMA_WARP) {
            // ---- MMAs (one thread); with p.stall set nothing is issued or committed
            if (lane == 0 && !p.stall) {
                const int ksteps = KR / 16;
                const uint64_t bdesc0 = smem_desc(sB_addr, 128u, SBO_B);
                for (int t = 0; t < ntiles; ++t) {
                    const uint32_t gi = g + (uint32_t)t;
                    const uint32_t sg = gi % nst;
                    const uint32_t st = sA_addr + sg * 2u * a_piece;
                    const uint32_t d = tbase + (gi & 1u) * (uint32_t)P;
                    if (!wait_phase(afull + sg, (gi / nst) & 1u, abort_flag, p.err, p.wait_cycles,
                                    RP_BACKOFF_NS))
                        break;
                    if (gi >= 2 && !wait_phase(dfree + (gi & 1u), ((gi >> 1) - 1) & 1u,
                                               abort_flag, p.err, p.wait_cycles, RP_BACKOFF_NS))
                        break;
                    tc_fence_after();
                    // descriptor address fields advance by (bytes >> 4): K step = 2 K-groups
                    // of A (2 * A_LBO bytes) and 256 bytes of B
                    const uint64_t a_hi = smem_desc(st, A_LBO, A_SBO);
                    const uint64_t a_lo = a_hi + (a_piece >> 4);
                    // the small correction products first (A_lo B_0, then A_hi B_j for
                    // j >= 1), the main product A_hi B_0 last: the accumulator rounds
                    // each addition toward zero, so each addition should land on a
                    // running sum as small as possible (see GM_CK in gemm_tc.cu)
#pragma unroll
                    for (int q = 0; q < NW + 1; ++q) {
                        // q = 0: A_lo B_0; 1 <= q < NW: A_hi B_q; q = NW: A_hi B_0
                        const uint64_t ad0 = q == 0 ? a_lo : a_hi;
                        const uint64_t bd0 = bdesc0 + (uint64_t)((q == 0 || q == NW ? 0 : q) *
                                                                 (b_piece >> 4));
#pragma unroll
                        for (int j = 0; j < RP_MAXK / 16; ++j) {
                            if (j < ksteps)
                                mma_ss(d, ad0 + (uint64_t)(j * (2 * A_LBO >> 4)),
                                       bd0 + (uint64_t)(j * 16), idesc, (q | j) != 0);
                        }
                    }
                    mma_commit(afree + sg);
                    mma_commit(dfull + (gi & 1u));
                }
            }
            __syncwarp();
        } else {
            // ---- scatter
            uint32_t w[MAXF][4], wt[3];
            // columns past Nc (the ragged last tile) sink every slot: cell Nc + lane
            // (the tile starts at a multiple of 128, so J mod 32 = lane)
            // (wide layout: absent slots and ragged columns read 0xFFFF, which no range
            // holds, so they add into the sink cell Nrow + lane)
            const uint32_t sink = WIDE ? 0xFFFFu : (uint32_t)Nc + (uint32_t)lane;
            const uint32_t sink2 = sink | (sink << 16);
            uint32_t mj = 0, cmj = 0;     // wide layout: occupations of this column's string
            auto load_words = [&](int t) {
                const int64_t jc = (int64_t)t * 128 + m;
                const bool in = jc < Nc;
                const int64_t jcc = in ? jc : Nc - 1;
#pragma unroll
                for (int k = 0; k < MAXF; ++k) {
                    if (k < nfull) {
                        const uint4 v = __ldg(p.tslot8 + (int64_t)(wq + 4 * k) * Nc + jcc);
                        w[k][0] = in ? v.x : sink2; w[k][1] = in ? v.y : sink2;
                        w[k][2] = in ? v.z : sink2; w[k][3] = in ? v.w : sink2;
                    }
                }
#pragma unroll
                for (int i = 0; i < 3; ++i) {
                    if (i < rem) {
                        const int s0 = tail0 + 2 * i;      // even: a pair within one chunk
                        const uint32_t* q = reinterpret_cast<const uint32_t*>(
                            p.tslot8 + (int64_t)(s0 >> 3) * Nc + jcc);
                        const uint32_t v = __ldg(q + ((s0 & 7) >> 1));
                        wt[i] = in ? v : sink2;
                    }
                }
                if (WIDE) mj = __ldg(p.cmask + jcc);
            };
            // one slot: sigma[tgt] += sign * round(D), unconditionally (an absent
            // slot's target is this lane's sink cell)
            auto add = [&](uint32_t word, int half, int slot, uint32_t dbits) {
                if (WIDE) {
                    // target within this pass's range, else the lane's sink cell; sign
                    // from the column string's occupations inside the slot
                    const uint32_t t = half ? (word >> 16) : (word & 0xFFFFu);
                    const uint32_t loc = t - (uint32_t)lo;
                    const uint32_t tg = loc < (uint32_t)Nrow ? loc : (uint32_t)Nrow + (uint32_t)lane;
                    const uint32_t sg = (uint32_t)(__popc(cmj & bm[slot]) & 1) << 31;
                    const int q = __float2int_rn(__uint_as_float(dbits ^ sg));
                    atomicAdd(srow + tg, q);
                } else {
                    const uint32_t tg = half ? (word >> 16) & 0x7FFFu : word & 0x7FFFu;
                    const uint32_t sg = half ? (word & 0x80000000u) : (word << 16) & 0x80000000u;
                    const int q = __float2int_rn(__uint_as_float(dbits ^ sg));
                    atomicAdd(srow + tg, q);
                }
            };
            bool ok = true;
            if (ntiles > 0) load_words(0);
            for (int t = 0; t < ntiles && ok; ++t) {
                const uint32_t gt = g + (uint32_t)t;
                if (lane == 0)
                    ok = wait_phase(dfull + (gt & 1u), (gt >> 1) & 1u, abort_flag, p.err,
                                    p.wait_cycles, RP_SCATTER_BACKOFF_NS);
                ok = __shfl_sync(0xffffffffu, ok ? 1 : 0, 0) != 0;
                if (!ok) break;
                tc_fence_after();
                const uint32_t dcol = tbase + ((uint32_t)(quad * 32) << 16) +
                                      (gt & 1u) * (uint32_t)P;
                uint32_t dr[MAXF][8], dt[6];
#pragma unroll
                for (int k = 0; k < MAXF; ++k)
                    if (k < nfull) tmem_ld8(dcol + (uint32_t)((wq + 4 * k) * 8), dr[k]);
                // remainder: pairs of slots (tail0 is even; 4-aligned when rem == 2)
                if (rem == 2) {
                    uint32_t r4[8];
                    tmem_ld4(dcol + (uint32_t)tail0, r4);
                    dt[0] = r4[0]; dt[1] = r4[1]; dt[2] = r4[2]; dt[3] = r4[3];
                } else {
#pragma unroll
                    for (int i = 0; i < 3; ++i)
                        if (i < rem) tmem_ld2(dcol + (uint32_t)(tail0 + 2 * i), dt[2 * i], dt[2 * i + 1]);
                }
                tmem_ld_wait();
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(dfree + (gt & 1u));
                // this tile's words; start loading the next tile's
                uint32_t cw[MAXF][4], ct[3];
#pragma unroll
                for (int k = 0; k < MAXF; ++k)
#pragma unroll
                    for (int i = 0; i < 4; ++i) cw[k][i] = w[k][i];
#pragma unroll
                for (int i = 0; i < 3; ++i) ct[i] = wt[i];
                cmj = mj;
                if (!WIDE && t + 1 < ntiles) load_words(t + 1);
#pragma unroll
                for (int k = 0; k < MAXF; ++k) {
                    if (k < nfull) {
#pragma unroll
                        for (int u = 0; u < 8; ++u)
                            add(cw[k][u >> 1], u & 1, (wq + 4 * k) * 8 + u, dr[k][u]);
                    }
                }
#pragma unroll
                for (int i = 0; i < 3; ++i) {
                    if (i < rem) {
                        add(ct[i], 0, tail0 + 2 * i, dt[2 * i]);
                        add(ct[i], 1, tail0 + 2 * i + 1, dt[2 * i + 1]);
                    }
                }
                // (wide layout: the next tile's words after the adds, which frees the
                // registers of one word set at 160-176 slots: 6 % faster at 18 orbitals)
                if (WIDE && t + 1 < ntiles) load_words(t + 1);
            }
        }
        g += (uint32_t)ntiles;
        __syncthreads();
        if (*abort_flag) break;
        {
            const int64_t nout = Nc - lo < Nrow ? Nc - lo : Nrow;   // this pass's targets
            for (int64_t j = tid; j < nout; j += RP_THREADS)
                p.Y[ir * Nc + lo + j] = (float)srow[j] * rsc[2];
        }
        __syncthreads();
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) tmem_dealloc(tbase, p.ncols);
}

// max |x| of each row (rowmax[r]) and of all rows (out, float bits: non-negative
// floats order like unsigned integers)
__global__ void k_rowmax(const float* __restrict__ x, int64_t nrow, int64_t ncol,
                         float* __restrict__ rowmax, unsigned* out) {
    __shared__ float wmx[8];
    for (int64_t r = blockIdx.x; r < nrow; r += gridDim.x) {
        float mx = 0.f;
        for (int64_t j = threadIdx.x; j < ncol; j += blockDim.x) mx = fmaxf(mx, fabsf(x[r * ncol + j]));
        for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_down_sync(0xffffffffu, mx, o));
        if ((threadIdx.x & 31) == 0) wmx[threadIdx.x >> 5] = mx;
        __syncthreads();
        if (threadIdx.x == 0) {
            float m = wmx[0];
            for (int w = 1; w < (int)(blockDim.x >> 5); ++w) m = fmaxf(m, wmx[w]);
            rowmax[r] = m;
            atomicMax(out, __float_as_uint(m));
        }
        __syncthreads();
    }
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
        // (pp|qq) with both excitations diagonal only ever multiplies a determinant
        // into itself: that part of the diagonal of H is added exactly elsewhere
        if (!(pi == qi && po == qo)) w = eri[(((int64_t)pi * n + qi) * n + po) * n + qo];
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
// tgt | (sgn < 0) << 15; slots without an entry hold the sink ns + (j mod 32).
// Stored per chunk of 8 slots: the 128-bit word (s/8, j) holds slots
// 8*(s/8) .. 8*(s/8)+7, slot s in 16-bit half s%8.
// Wide layout (wide != 0): a slot holds the target alone, 0xFFFF when absent.
__global__ void k_slot_fill(uint16_t* __restrict__ tslot, int64_t count, int64_t ns, int wide) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count;
         i += (int64_t)gridDim.x * blockDim.x)
        tslot[i] = wide ? (uint16_t)0xFFFFu : (uint16_t)(ns + ((i >> 3) % ns & 31));
}

__global__ void k_slot_table(const int32_t* __restrict__ tgt, const uint16_t* __restrict__ pq,
                             const int8_t* __restrict__ sgn, int64_t ns, int nexc, int n,
                             uint16_t* __restrict__ tslot, int wide) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= ns * nexc) return;
    const int64_t j = i / nexc;
    int a = pq[i] / n, b = pq[i] % n;
    if (a > b) { int t = a; a = b; b = t; }
    const int s = b * (b + 1) / 2 + a;
    tslot[((int64_t)(s >> 3) * ns + j) * 8 + (s & 7)] =
        wide ? (uint16_t)tgt[i] : (uint16_t)(tgt[i] | (sgn[i] < 0 ? 0x8000 : 0));
}

// row-string tables of the off-diagonal entries (p != q), in table order: target
// and slot({p,q}) | (sgn < 0) << 15; one thread per string
__global__ void k_row_offdiag(const int32_t* __restrict__ tgt, const uint16_t* __restrict__ pq,
                              const int8_t* __restrict__ sgn, int64_t ns, int nexc, int noff,
                              int n, int32_t* __restrict__ otgt, uint16_t* __restrict__ oslot) {
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= ns) return;
    int k = 0;
    for (int e = 0; e < nexc; ++e) {
        const int64_t i = r * nexc + e;
        int a = pq[i] / n, b = pq[i] % n;
        if (a == b) continue;
        if (a > b) { int t = a; a = b; b = t; }
        otgt[r * noff + k] = tgt[i];
        oslot[r * noff + k] = (uint16_t)((b * (b + 1) / 2 + a) | (sgn[i] < 0 ? 0x8000 : 0));
        ++k;
    }
}

// wd[q][s] = W[qq][s] = (qq|pr) for slot s = {p, r}, FP64 unscaled; zero for the
// diagonal slots (p == r), whose part of the diagonal of H is added exactly elsewhere
__global__ void k_wdiag(const double* __restrict__ eri, int n, int P, int NS,
                        double* __restrict__ wd) {
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= n * P) return;
    const int q = idx / P, so = idx % P;
    double w = 0.0;
    if (so < NS) {
        int po, qo;
        slot_pair(so, po, qo);
        if (po != qo) w = eri[(((int64_t)q * n + q) * n + po) * n + qo];
    }
    wd[idx] = w;
}

// x [R][Cn] -> hi/lo BF16 pieces [R][pitch] (BF16 needs no scale); zero padding
__global__ void k_split_rows_bf16(const float* __restrict__ src, int64_t R, int64_t Cn,
                                  uint16_t* __restrict__ hi, uint16_t* __restrict__ lo,
                                  int64_t pitch) {
    const int64_t total = R * pitch;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = i / pitch, c = i % pitch;
        const float v = c < Cn ? src[r * Cn + c] : 0.f;
        const __nv_bfloat16 h = __float2bfloat16_rn(v);
        hi[i] = __bfloat16_as_ushort(h);
        lo[i] = __bfloat16_as_ushort(__float2bfloat16_rn(v - __bfloat162float(h)));
    }
}

uint32_t tmem_cols(int P) {
    uint32_t need = (uint32_t)(2 * P), c = 32;
    while (c < need) c <<= 1;
    return c;
}

// Nrow: targets held in shared memory (all column strings, or one pass's span)
size_t rowpass_smem(int P, int NW, int KR, int64_t Nrow, int nst) {
    return (size_t)2 * nst * KR * 256 + (size_t)2 * NW * P * KR + 4 * (size_t)(Nrow + RP_SINK) +
           16 + 10 * RP_MAXK + 16 + 4 * RP_MAXK + 24 + 16 + 8 * (size_t)P + 4 * (size_t)P + 16 +
           10 * 8 + 16;
}

// W in RP_NW 16-bit pieces (2: ~2^-22 relative per (pq|rs); 3: ~2^-33, a fourth
// MMA pass and 50 % more shared memory for B_R, which leaves room for two A
// stages only)
constexpr int RP_NW = 2;

template <int P>
void* rowpass_fn(bool fp16) {
    return fp16 ? (void*)k_rowpass<P, true, RP_NW, false> : (void*)k_rowpass<P, false, RP_NW, false>;
}
template <int P>
void* rowpass_fn_wide(bool fp16) {
    return fp16 ? (void*)k_rowpass<P, true, RP_NW, true> : (void*)k_rowpass<P, false, RP_NW, true>;
}

// The wide layout is instantiated for 17 and 18 orbitals (P = 160, 176), which
// need it, and for 12 orbitals (P = 80), where the tests compare it with the
// plain layout.
void* rowpass_kernel(int P, bool fp16, bool wide) {
    if (wide) {
        switch (P) {
            case 80: return rowpass_fn_wide<80>(fp16);
            case 160: return rowpass_fn_wide<160>(fp16);
            case 176: return rowpass_fn_wide<176>(fp16);
            default: return nullptr;
        }
    }
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

size_t rowpass_smem_bytes(const TcSigma& t, int stages) {
    return rowpass_smem(t.P, t.nw, t.KR, t.wide ? t.span : t.nsb, stages);
}

void TcSigma::init(const SpinTables& A, const SpinTables& B, const double* d_h1,
                   const double* d_eri, const float2* d_diag, int norb, double wmax,
                   double wcolsum, bool use_fp16, cudaStream_t st) {
    ta = &A;
    tb = &B;
    n = norb;
    NS = n * (n + 1) / 2;
    P = ((NS + 1 + 15) / 16) * 16;
    nsa = A.ns;
    nsb = B.ns;
    dim = nsa * nsb;
    fp16 = use_fp16;
    nw = RP_NW;
    // off-diagonal entries of a row string, m (n - m), and one column for its m
    // diagonal entries; at least one K step, so that a row without any (no alpha
    // electrons) multiplies padding (B_R = 0) and D is exactly zero instead of
    // never written
    noff = A.m * (n - A.m);
    ndiag = A.m > 0 ? 1 : 0;
    KR = noff + ndiag > 0 ? ((noff + ndiag + 15) / 16) * 16 : 16;
    if (KR > RP_MAXK || B.ns > 65536 - 2 * RP_SINK)
        KPM_THROW(KPM_EUNSUPPORTED, "tensor-core sigma supports up to 18 orbitals");
    int dev = 0;
    KPM_CUDA(cudaGetDevice(&dev));
    cudaDeviceProp prop;
    KPM_CUDA(cudaGetDeviceProperties(&prop, dev));
    if (prop.major != 10)
        KPM_THROW(KPM_EUNSUPPORTED, "tensor-core sigma needs a Blackwell (sm_10x) GPU");
    nsm = prop.multiProcessorCount;
    smem_optin = prop.sharedMemPerBlockOptin;
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

    // the plain layout where its 15-bit targets and one row's sigma fit (three A
    // stages, else two), else the wide one with as few passes as fit
    set_layout(0, st);
    {
        const int64_t no = A.ns * (int64_t)noff;
        rslot_a.alloc((size_t)(no > 0 ? no : 1) * sizeof(uint16_t));
        rtgt_a.alloc((size_t)(no > 0 ? no : 1) * sizeof(int32_t));
        if (no > 0) {
            k_row_offdiag<<<(unsigned)((A.ns + 127) / 128), 128, 0, st>>>(
                A.tgt.as<int32_t>(), A.pq.as<uint16_t>(), A.sgn.as<int8_t>(), A.ns, A.nexc, noff,
                n, rtgt_a.as<int32_t>(), rslot_a.as<uint16_t>());
            KPM_LAUNCHED();
        }
        wdiag.alloc((size_t)n * P * sizeof(double));
        k_wdiag<<<(n * P + 255) / 256, 256, 0, st>>>(d_eri, n, P, NS, wdiag.as<double>());
        KPM_LAUNCHED();
    }
    err.alloc(sizeof(int));
    amax.alloc(2 * sizeof(unsigned));
    KPM_CUDA(cudaMemsetAsync(err.p, 0, sizeof(int), st));
    dense.init(A, B, &A == &B, err.as<int>(), st);
    dense.diag_full = d_diag;
    dense.autotune(st);
    if (!wide) autotune(st);
}

// Chooses the row pass's layout (passes = 0: automatic; >= 1: the wide layout
// with that many passes, where it is instantiated), sizes its shared memory and
// builds the column strings' slot table in the matching format.
void TcSigma::set_layout(int passes, cudaStream_t st) {
    const size_t optin = smem_optin;
    bool w = passes > 0;
    int np = passes > 0 ? passes : 1;
    int stg = 3;
    if (!w) {
        const bool fits15 = nsb <= 32768 - RP_SINK && rowpass_kernel(P, fp16, false);
        if (fits15 && rowpass_smem(P, nw, KR, nsb, 3) <= optin) stg = 3;
        else if (fits15 && rowpass_smem(P, nw, KR, nsb, 2) <= optin) stg = 2;
        else w = true;   // (also where only the wide kernel exists for P: 17, 18 orbitals)
    }
    int64_t sp = nsb;
    if (w) {
        stg = 2;
        if (passes <= 0)
            while (rowpass_smem(P, nw, KR, (nsb + np - 1) / np, 2) > optin && np < 64) ++np;
        sp = (nsb + np - 1) / np;
        if (sp < 1) sp = 1;
    }
    void* kfn = rowpass_kernel(P, fp16, w);
    if (!kfn)
        KPM_THROW(w ? KPM_EINVAL : KPM_EUNSUPPORTED,
                  "tensor-core sigma: no row-pass kernel for %d slots in the %s layout", P,
                  w ? "wide" : "plain");
    size_t sm = rowpass_smem(P, nw, KR, sp, stg);
    // at least ~116 KB so that exactly one CTA (and one TMEM allocation) fits per SM
    const size_t floor_bytes = 116 * 1024;
    if (sm < floor_bytes) sm = floor_bytes;
    if (sm > optin)
        KPM_THROW(KPM_EUNSUPPORTED, "tensor-core sigma: %lld targets per pass need %zu B of shared memory",
                  (long long)sp, sm);
    KPM_CUDA(cudaFuncSetAttribute(kfn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    const size_t count = (size_t)P * tb->ns;
    if (!slot_b.p || w != wide) {
        slot_b.alloc(count * sizeof(uint16_t));
        k_slot_fill<<<1024, 256, 0, st>>>(slot_b.as<uint16_t>(), (int64_t)count, tb->ns, w ? 1 : 0);
        KPM_LAUNCHED();
        const int64_t ne = tb->ns * tb->nexc;
        if (ne > 0) {
            k_slot_table<<<(unsigned)((ne + 255) / 256), 256, 0, st>>>(
                tb->tgt.as<int32_t>(), tb->pq.as<uint16_t>(), tb->sgn.as<int8_t>(), tb->ns,
                tb->nexc, n, slot_b.as<uint16_t>(), w ? 1 : 0);
            KPM_LAUNCHED();
        }
    }
    kernel = kfn;
    wide = w;
    npass = np;
    span = sp;
    nst = stg;
    smem_bytes = sm;
}

void TcSigma::apply(const float* x, float* y, int ncol, cudaStream_t st) {
    const int64_t xp = dense.xpitch;
    for (int c = 0; c < ncol; ++c) {
        const float* X = x + (size_t)c * dim;
        float* Y = y + (size_t)c * dim;
        // max|x|: FP16 operand scales and the fixed-point range of the scatter
        KPM_CUDA(cudaMemsetAsync(amax.p, 0, sizeof(unsigned), st));
        rowmax.ensure((size_t)(nsa > 0 ? nsa : 1) * sizeof(float));
        {
            const int64_t g = nsa < (int64_t)nsm * 8 ? nsa : (int64_t)nsm * 8;
            k_rowmax<<<(unsigned)(g > 0 ? g : 1), 256, 0, st>>>(X, nsa, nsb, rowmax.as<float>(),
                                                                amax.as<unsigned>());
        }
        KPM_LAUNCHED();
        const float* am = reinterpret_cast<const float*>(amax.p);
        // split x: the FP16 pieces serve the row pass and the beta GEMM
        dense.split(X, am, st);
        const uint16_t* xh = dense.xh.as<uint16_t>();
        const uint16_t* xl = dense.xl.as<uint16_t>();
        if (!fp16) {
            xbh.ensure((size_t)nsa * xp * 2);
            xbl.ensure((size_t)nsa * xp * 2);
            k_split_rows_bf16<<<2048, 256, 0, st>>>(X, nsa, nsb, xbh.as<uint16_t>(),
                                                    xbl.as<uint16_t>(), xp);
            KPM_LAUNCHED();
            xh = xbh.as<uint16_t>();
            xl = xbl.as<uint16_t>();
        }
        // opposite-spin part: rows alpha, columns beta; writes Y
        launch_rowpass(xh, xl, Y, nst, rp_prefetch, st);
        // same-spin parts (dense GEMMs) and the exact diagonal, added into Y
        dense.apply(X, Y, am, st);
    }
}

void TcSigma::launch_rowpass(const uint16_t* xh, const uint16_t* xl, float* Y, int stages,
                             int prefetch, cudaStream_t st) {
    const uint32_t nc = tmem_cols(P);
    const int64_t xp = dense.xpitch;
    const float* am = reinterpret_cast<const float*>(amax.p);
    RowPass p1{xh, xl, xp, Y, nsa, nsb, slot_b.as<uint4>(),
               rtgt_a.as<int32_t>(), rslot_a.as<uint16_t>(), noff, ndiag, KR,
               ta->masks.as<uint32_t>(), wdiag.as<double>(),
               wimg.as<uint16_t>(), nc, am, rowmax.as<float>(), wscale, tb->nexc, NS, stages,
               prefetch, npass, span, tb->masks.as<uint32_t>(), err.as<int>(),
               stall_next ? STALL_WAIT_CYCLES : WAIT_CYCLES, stall_next ? 1 : 0};
    stall_next = false;
    const int64_t items = nsa * (int64_t)npass;
    int g1 = (int)(items < nsm ? items : nsm);
    void* args1[] = {&p1};
    if (prof) {
        if ((int)ev.size() < ev_used + 2) {
            cudaEvent_t e0, e1;
            KPM_CUDA(cudaEventCreate(&e0));
            KPM_CUDA(cudaEventCreate(&e1));
            ev.push_back(e0);
            ev.push_back(e1);
        }
        KPM_CUDA(cudaEventRecord(ev[ev_used], st));
    }
    // (smem_bytes is sized for the most stages init allowed)
    KPM_CUDA(cudaLaunchKernel(kernel, dim3(g1), dim3(RP_THREADS), args1, smem_bytes, st));
    KPM_LAUNCHED();
    if (prof) {
        KPM_CUDA(cudaEventRecord(ev[ev_used + 1], st));
        ev_used += 2;
    }
}

// Picks the row pass's A stages and L2 prefetch distance by timing every
// candidate once per device and shape (process-wide cache), on a zero vector:
// the choice decides only when copies are issued, never what is computed, so
// results do not depend on it.  Small shapes keep the defaults.
void TcSigma::autotune(cudaStream_t st) {
    if (nsa * nsb < ((int64_t)1 << 22)) return;
    int dev = 0;
    KPM_CUDA(cudaGetDevice(&dev));
    static std::mutex mu;
    static std::map<std::array<int64_t, 5>, std::array<int, 2>> cache;
    const std::array<int64_t, 5> key{dev, n, nsa, nsb, fp16 ? 1 : 0};
    {
        std::lock_guard<std::mutex> lk(mu);
        auto it = cache.find(key);
        if (it != cache.end()) {
            nst = it->second[0];
            rp_prefetch = it->second[1];
            return;
        }
    }
    const int64_t xp = dense.xpitch;
    // two distinct operand buffers, as in use (x's hi and lo pieces are separate
    // arrays, so the gathers touch twice the bytes of one)
    DevBuf zh, zl, y;
    zh.alloc((size_t)nsa * xp * 2);
    zl.alloc((size_t)nsa * xp * 2);
    y.alloc((size_t)dim * sizeof(float));
    KPM_CUDA(cudaMemsetAsync(zh.p, 0, zh.bytes, st));
    KPM_CUDA(cudaMemsetAsync(zl.p, 0, zl.bytes, st));
    KPM_CUDA(cudaMemsetAsync(amax.p, 0, sizeof(unsigned), st));
    rowmax.ensure((size_t)(nsa > 0 ? nsa : 1) * sizeof(float));
    KPM_CUDA(cudaMemsetAsync(rowmax.p, 0, rowmax.bytes, st));
    cudaEvent_t e0, e1;
    KPM_CUDA(cudaEventCreate(&e0));
    KPM_CUDA(cudaEventCreate(&e1));
    const bool prof_was = prof;
    prof = false;
    const int maxst = nst;   // what shared memory allows (init)
    const int pfs[3] = {0, 4, 8};
    float best = 0.f;
    int bst = nst, bpf = rp_prefetch;
    launch_rowpass(zh.as<uint16_t>(), zl.as<uint16_t>(), y.as<float>(), nst, rp_prefetch, st);
    for (int stg = 2; stg <= maxst; ++stg) {
        for (int pf : pfs) {
            // the faster of two launches
            float ms = 0.f;
            for (int rep = 0; rep < 2; ++rep) {
                KPM_CUDA(cudaEventRecord(e0, st));
                launch_rowpass(zh.as<uint16_t>(), zl.as<uint16_t>(), y.as<float>(), stg, pf, st);
                KPM_CUDA(cudaEventRecord(e1, st));
                KPM_CUDA(cudaEventSynchronize(e1));
                float t = 0.f;
                KPM_CUDA(cudaEventElapsedTime(&t, e0, e1));
                if (rep == 0 || t < ms) ms = t;
            }
            if (best == 0.f || ms < best) {
                best = ms;
                bst = stg;
                bpf = pf;
            }
        }
    }
    prof = prof_was;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    nst = bst;
    rp_prefetch = bpf;
    std::lock_guard<std::mutex> lk(mu);
    cache[key] = {nst, rp_prefetch};
}

double TcSigma::read_prof(cudaStream_t st, int* count) {
    KPM_CUDA(cudaStreamSynchronize(st));
    double tot = 0.0;
    for (int i = 0; i + 1 < ev_used; i += 2) {
        float t = 0.f;
        KPM_CUDA(cudaEventElapsedTime(&t, ev[i], ev[i + 1]));
        tot += t;
    }
    if (count) *count = ev_used / 2;
    ev_used = 0;
    return tot;
}

TcSigma::~TcSigma() {
    for (cudaEvent_t e : ev) cudaEventDestroy(e);
}

int TcSigma::check(cudaStream_t st) {
    int h = 0;
    KPM_CUDA(cudaMemcpyAsync(&h, err.p, sizeof(int), cudaMemcpyDeviceToHost, st));
    KPM_CUDA(cudaStreamSynchronize(st));
    if (h) KPM_CUDA(cudaMemsetAsync(err.p, 0, sizeof(int), st));
    return h;
}

}  // namespace kpm
