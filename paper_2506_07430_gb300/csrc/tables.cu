// Occupation strings, single-excitation tables and the same-spin string
// Hamiltonian, built on the device.
//
// Strings: the (N_alpha, N_beta) sector of the paper's number-conserving
// sampler (Results, "Parallel sampling") factorises into alpha and beta
// occupation strings: n-bit masks with m bits set.  A string's rank is its
// position in ascending integer order, which is the combinatorial number
// system rank sum_{k=1..m} C(p_k, k) over its occupied orbitals
// p_1 < ... < p_m; strings are produced by unranking and targets are located by
// ranking, so no lookup table of size 2^n is needed.
//
// Single-excitation table: for string I and each (p, q) with a+_p a_q |I> != 0
// (q occupied, p vacant or p == q): target rank, pair index p*n+q and sign
// (-1)^(occupied orbitals strictly between p and q).  Entry order: q ascending
// over occupied orbitals, p ascending over {q} union vacant.
//
// Same-spin string Hamiltonian F (the part of the paper's second-quantized H,
// Methods, that moves electrons of one spin only), by the Slater-Condon rules
// on one spin's strings with one-body h and two-body (pq|rs):
//   F[I,I]           = sum_{i in I} h_ii + 1/2 sum_{i,j in I} ((ii|jj) - (ij|ji))
//   F[I - i + a, I]  = s * (h_ai + sum_{j in I} ((ai|jj) - (aj|ji)))
//   F[I - ij + ab, I]= s * ((ai|bj) - (aj|bi))
// with s the sign of a+_a a_i (or a+_a a+_b a_j a_i) acting on I.  The
// neighbours of each string are stored in one fixed order: itself, singles
// (i occupied ascending, a vacant ascending), doubles (i<j, a<b).
#include "common.cuh"

namespace kpm {

std::atomic<uint64_t> g_launches{0};

Binom make_binom() {
    Binom b{};
    for (int p = 0; p <= KPM_MAX_ORB; ++p) {
        b.c[p][0] = 1;
        for (int k = 1; k <= KPM_MAX_ORB; ++k)
            b.c[p][k] = (p == 0) ? 0u : b.c[p - 1][k - 1] + b.c[p - 1][k];
    }
    return b;
}

__device__ __forceinline__ uint32_t rank_of(uint32_t mask, const Binom& B) {
    uint32_t r = 0;
    int k = 1;
    while (mask) {
        int p = __ffs(mask) - 1;
        r += B.c[p][k];
        ++k;
        mask &= mask - 1;
    }
    return r;
}

__device__ __forceinline__ int parity_below(uint32_t mask, int p) {
    return __popc(mask & ((1u << p) - 1u)) & 1;
}

__global__ void k_masks(uint32_t* __restrict__ masks, int n, int m, int64_t ns, Binom B) {
    int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= ns) return;
    uint32_t rr = (uint32_t)r, mask = 0;
    for (int k = m; k >= 1; --k) {
        int p = k - 1;
        while (p + 1 < n && B.c[p + 1][k] <= rr) ++p;
        mask |= 1u << p;
        rr -= B.c[p][k];
    }
    masks[r] = mask;
}

__global__ void k_tables(const uint32_t* __restrict__ masks, int n, int64_t ns, int nexc, Binom B,
                         int32_t* __restrict__ tgt, uint16_t* __restrict__ pq,
                         int8_t* __restrict__ sgn, int32_t* __restrict__ tgtT,
                         uint16_t* __restrict__ pqT, int8_t* __restrict__ sgnT) {
    int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= ns) return;
    uint32_t I = masks[r];
    int k = 0;
    for (int q = 0; q < n; ++q) {
        if (!((I >> q) & 1u)) continue;
        for (int p = 0; p < n; ++p) {
            if (p != q && ((I >> p) & 1u)) continue;
            uint32_t J = (I & ~(1u << q)) | (1u << p);
            int lo = p < q ? p : q, hi = p < q ? q : p;
            uint32_t between = I & ((1u << hi) - 1u) & ~((2u << lo) - 1u);
            int8_t s = (__popc(between) & 1) ? -1 : 1;
            int32_t t = (int32_t)rank_of(J, B);
            uint16_t g = (uint16_t)(p * n + q);
            tgt[r * nexc + k] = t;
            pq[r * nexc + k] = g;
            sgn[r * nexc + k] = s;
            tgtT[(int64_t)k * ns + r] = t;
            pqT[(int64_t)k * ns + r] = g;
            sgnT[(int64_t)k * ns + r] = s;
            ++k;
        }
    }
}

__device__ __forceinline__ double eri4(const double* __restrict__ e, int n, int p, int q, int r,
                                       int s) {
    return __ldg(e + (((int64_t)p * n + q) * n + r) * n + s);
}

__global__ void k_same_spin(const uint32_t* __restrict__ masks, int n, int64_t ns, int nnbr,
                            Binom B, const double* __restrict__ h1, const double* __restrict__ eri,
                            int32_t* __restrict__ fcol, double* __restrict__ fval) {
    int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= ns) return;
    uint32_t I = masks[r];
    int occ[KPM_MAX_ORB], vac[KPM_MAX_ORB], no = 0, nv = 0;
    for (int p = 0; p < n; ++p) {
        if ((I >> p) & 1u) occ[no++] = p; else vac[nv++] = p;
    }
    int64_t t = 0;
    // itself
    double e = 0.0;
    for (int x = 0; x < no; ++x) {
        int i = occ[x];
        e += h1[i * n + i];
        for (int y = 0; y < no; ++y) {
            int j = occ[y];
            e += 0.5 * (eri4(eri, n, i, i, j, j) - eri4(eri, n, i, j, j, i));
        }
    }
    fcol[t * ns + r] = (int32_t)r;
    fval[t * ns + r] = e;
    ++t;
    // singles i -> a
    for (int x = 0; x < no; ++x) {
        int i = occ[x];
        for (int z = 0; z < nv; ++z) {
            int a = vac[z];
            uint32_t J = I ^ (1u << i) ^ (1u << a);
            int lo = a < i ? a : i, hi = a < i ? i : a;
            uint32_t between = I & ((1u << hi) - 1u) & ~((2u << lo) - 1u);
            double s = (__popc(between) & 1) ? -1.0 : 1.0;
            double v = h1[a * n + i];
            for (int y = 0; y < no; ++y) {
                int j = occ[y];
                v += eri4(eri, n, a, i, j, j) - eri4(eri, n, a, j, j, i);
            }
            fcol[t * ns + r] = (int32_t)rank_of(J, B);
            fval[t * ns + r] = s * v;
            ++t;
        }
    }
    // doubles i<j -> a<b
    for (int x = 0; x < no; ++x)
        for (int y = x + 1; y < no; ++y) {
            int i = occ[x], j = occ[y];
            for (int z = 0; z < nv; ++z)
                for (int w = z + 1; w < nv; ++w) {
                    int a = vac[z], b = vac[w];
                    uint32_t M = I;
                    int par = parity_below(M, i);
                    M &= ~(1u << i);
                    par ^= parity_below(M, j);
                    M &= ~(1u << j);
                    par ^= parity_below(M, b);
                    M |= 1u << b;
                    par ^= parity_below(M, a);
                    M |= 1u << a;
                    double v = eri4(eri, n, a, i, b, j) - eri4(eri, n, a, j, b, i);
                    fcol[t * ns + r] = (int32_t)rank_of(M, B);
                    fval[t * ns + r] = par ? -v : v;
                    ++t;
                }
        }
}

__global__ void k_to_f32(const double* __restrict__ x, float* __restrict__ y, int64_t n) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        y[i] = (float)x[i];
}

void to_f32(const double* x, float* y, int64_t n, cudaStream_t st) {
    if (n <= 0) return;
    k_to_f32<<<1024, 256, 0, st>>>(x, y, n);
    KPM_LAUNCHED();
}

static int64_t binom64(int n, int k) {
    if (k < 0 || k > n) return 0;
    int64_t r = 1;
    for (int i = 1; i <= k; ++i) r = r * (n - k + i) / i;
    return r;
}

// packed transposed table: one 32-bit word per entry (targets < 2^16 for n <= 18)
__global__ void k_pack_tables(const int32_t* __restrict__ tgtT, const uint16_t* __restrict__ pqT,
                              const int8_t* __restrict__ sgnT, int64_t ne,
                              uint32_t* __restrict__ pkT) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= ne) return;
    pkT[i] = (uint32_t)tgtT[i] | ((uint32_t)pqT[i] << 16) | (sgnT[i] < 0 ? 0x80000000u : 0u);
}

void build_spin_tables(SpinTables& t, int n, int m, const double* d_h1, const double* d_eri,
                       cudaStream_t st) {
    t.n = n;
    t.m = m;
    t.ns = binom64(n, m);
    t.nexc = m * (n - m + 1);
    t.nnbr = (int)(1 + (int64_t)m * (n - m) + binom64(m, 2) * binom64(n - m, 2));
    Binom B = make_binom();
    t.masks.alloc(t.ns * sizeof(uint32_t));
    size_t ne = (size_t)t.ns * t.nexc;
    t.tgt.alloc(ne * 4 + 4);
    t.pq.alloc(ne * 2 + 4);
    t.sgn.alloc(ne + 4);
    t.tgtT.alloc(ne * 4 + 4);
    t.pqT.alloc(ne * 2 + 4);
    t.sgnT.alloc(ne + 4);
    size_t nf = (size_t)t.ns * t.nnbr;
    t.fcol.alloc(nf * 4);
    t.fval64.alloc(nf * 8);
    t.fval32.alloc(nf * 4);
    int th = 128;
    int bl = (int)((t.ns + th - 1) / th);
    k_masks<<<bl, th, 0, st>>>(t.masks.as<uint32_t>(), n, m, t.ns, B);
    KPM_LAUNCHED();
    k_tables<<<bl, th, 0, st>>>(t.masks.as<uint32_t>(), n, t.ns, t.nexc, B, t.tgt.as<int32_t>(),
                               t.pq.as<uint16_t>(), t.sgn.as<int8_t>(), t.tgtT.as<int32_t>(),
                               t.pqT.as<uint16_t>(), t.sgnT.as<int8_t>());
    KPM_LAUNCHED();
    t.pkT.alloc(ne * 4 + 4);
    if (ne > 0) {
        k_pack_tables<<<(unsigned)((ne + 255) / 256), 256, 0, st>>>(
            t.tgtT.as<int32_t>(), t.pqT.as<uint16_t>(), t.sgnT.as<int8_t>(), (int64_t)ne,
            t.pkT.as<uint32_t>());
        KPM_LAUNCHED();
    }
    k_same_spin<<<bl, th, 0, st>>>(t.masks.as<uint32_t>(), n, t.ns, t.nnbr, B, d_h1, d_eri,
                                  t.fcol.as<int32_t>(), t.fval64.as<double>());
    KPM_LAUNCHED();
    k_to_f32<<<1024, 256, 0, st>>>(t.fval64.as<double>(), t.fval32.as<float>(), (int64_t)nf);
    KPM_LAUNCHED();
}

}  // namespace kpm
