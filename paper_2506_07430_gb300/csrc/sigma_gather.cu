// Gather-form sigma = H x and dipole mu x (FP64 and FP32 CUDA-core paths).
//
// H (Methods, second-quantized Hamiltonian) splits over the alpha/beta string
// product basis as
//   H = F_alpha (x) 1 + 1 (x) F_beta + sum_{pq,rs} (pq|rs) E^alpha_pq E^beta_rs,
// where F_sigma is the same-spin string Hamiltonian (built in tables.cu) and the
// last term is the opposite-spin two-electron part.  For determinant
// (I_a, I_b) and x laid out as x[J_a * N_b + J_b]:
//   y = sum_t F_b[I_b,t] x[I_a, J_t] + sum_t F_a[I_a,t] x[J_t, I_b]
//     + sum_{e in tab(I_a)} s_e sum_{f in tab(I_b)} s_f (pq_e|pq_f) x[J_e, J_f]
// using <I|E_pq|J> = <J|E_qp|I> and (pq|rs) = (qp|sr) for real orbitals.
//
// The dipole (Methods, mu = -sum_pq d_pq (E^alpha_pq + E^beta_pq)) is a
// one-body gather over the same tables.
//
// One CTA row handles one alpha string and 128 consecutive beta strings; the
// alpha-side table row and F_alpha row are staged in shared memory and read
// uniformly; beta-side rows are read from the string-fastest tables, so
// neighbouring threads load neighbouring words.
#include "common.cuh"

namespace kpm {

// EXACT_DIAG (FP32 path): the diagonal H_II is taken from `diag` (FP64 value stored
// as a float hi/lo pair) and every diagonal contribution is skipped in the
// gathers: F entries t = 0 of both spins and the alpha-beta products whose alpha
// and beta excitations are both diagonal (p == q).  Large diagonal energies
// then carry no FP32 representation error, which would otherwise shift every
// eigenvalue systematically and grow the moment error linearly in n.
// One CTA of the gather sigma: beta tile bx (128 strings), alpha string ia,
// column col.  Shared by the single-molecule kernel and the batched one, so that
// both do the same arithmetic per element.
template <class T, bool EXACT_DIAG>
__device__ __forceinline__ void sigma_gather_cta(
    int64_t bx, int64_t ia, int64_t col, const T* __restrict__ x, T* __restrict__ y, int64_t nsa,
    int64_t nsb, const int32_t* __restrict__ tgtA, const uint16_t* __restrict__ pqA,
    const int8_t* __restrict__ sgnA, int nexcA, const int32_t* __restrict__ fcolA,
    const T* __restrict__ fvalA, int nnbrA, const int32_t* __restrict__ tgtBT,
    const uint16_t* __restrict__ pqBT, const int8_t* __restrict__ sgnBT, int nexcB,
    const int32_t* __restrict__ fcolB, const T* __restrict__ fvalB, int nnbrB,
    const T* __restrict__ V, int n, const float2* __restrict__ diag) {
    extern __shared__ __align__(16) unsigned char smem[];
    T* sFv = reinterpret_cast<T*>(smem);
    int32_t* sFc = reinterpret_cast<int32_t*>(sFv + nnbrA);
    int32_t* sJ = sFc + nnbrA;
    int32_t* sP = sJ + nexcA;
    int32_t* sS = sP + nexcA;
    __shared__ int sNoff;

    const int n2 = n * n;
    const int64_t ib = bx * blockDim.x + threadIdx.x;
    const int64_t dim = nsa * nsb;
    x += col * dim;
    y += col * dim;

    for (int t = threadIdx.x; t < nnbrA; t += blockDim.x) {
        sFv[t] = fvalA[(int64_t)t * nsa + ia];
        sFc[t] = fcolA[(int64_t)t * nsa + ia];
    }
    if (EXACT_DIAG) {
        // alpha entries reordered: off-diagonal (p != q) first, then diagonal
        if (threadIdx.x == 0) {
            int k = 0;
            for (int pass = 0; pass < 2; ++pass)
                for (int e = 0; e < nexcA; ++e) {
                    int g = pqA[ia * nexcA + e];
                    bool dg = (g % (n + 1)) == 0;
                    if (dg != (pass == 1)) continue;
                    sJ[k] = tgtA[ia * nexcA + e];
                    sP[k] = g;
                    sS[k] = sgnA[ia * nexcA + e];
                    ++k;
                }
            int noff = 0;
            for (int e = 0; e < nexcA; ++e) noff += (pqA[ia * nexcA + e] % (n + 1)) != 0;
            sNoff = noff;
        }
    } else {
        for (int e = threadIdx.x; e < nexcA; e += blockDim.x) {
            sJ[e] = tgtA[ia * nexcA + e];
            sP[e] = pqA[ia * nexcA + e];
            sS[e] = sgnA[ia * nexcA + e];
        }
    }
    __syncthreads();
    if (ib >= nsb) return;

    const T* xrow = x + ia * nsb;
    const int t0 = EXACT_DIAG ? 1 : 0;
    T acc = T(0);
    // same-spin beta: row I_a of x, columns = F_beta neighbours of I_b
    for (int t = t0; t < nnbrB; ++t)
        acc += fvalB[(int64_t)t * nsb + ib] * xrow[fcolB[(int64_t)t * nsb + ib]];
    // same-spin alpha: column I_b of x, rows = F_alpha neighbours of I_a
    for (int t = t0; t < nnbrA; ++t) acc += sFv[t] * x[(int64_t)sFc[t] * nsb + ib];
    // opposite-spin two-electron part
    const int noff = EXACT_DIAG ? sNoff : nexcA;
    for (int f = 0; f < nexcB; ++f) {
        const int64_t jb = tgtBT[(int64_t)f * nsb + ib];
        const int pb = pqBT[(int64_t)f * nsb + ib];
        const T sb = T(sgnBT[(int64_t)f * nsb + ib]);
        const int ne = (EXACT_DIAG && (pb % (n + 1)) == 0) ? noff : nexcA;
        T inner = T(0);
        for (int e = 0; e < ne; ++e)
            inner += T(sS[e]) * V[(int64_t)sP[e] * n2 + pb] * x[(int64_t)sJ[e] * nsb + jb];
        acc += sb * inner;
    }
    if (EXACT_DIAG) {
        const float2 d = diag[ia * nsb + ib];
        const T xv = xrow[ib];
        acc += fmaf(d.x, xv, d.y * xv);
    }
    y[ia * nsb + ib] = acc;
}

template <class T, bool EXACT_DIAG>
__global__ void __launch_bounds__(128)
k_sigma_gather(const T* __restrict__ x, T* __restrict__ y, int64_t nsa, int64_t nsb,
               const int32_t* __restrict__ tgtA, const uint16_t* __restrict__ pqA,
               const int8_t* __restrict__ sgnA, int nexcA, const int32_t* __restrict__ fcolA,
               const T* __restrict__ fvalA, int nnbrA, const int32_t* __restrict__ tgtBT,
               const uint16_t* __restrict__ pqBT, const int8_t* __restrict__ sgnBT, int nexcB,
               const int32_t* __restrict__ fcolB, const T* __restrict__ fvalB, int nnbrB,
               const T* __restrict__ V, int n, const float2* __restrict__ diag) {
    sigma_gather_cta<T, EXACT_DIAG>(blockIdx.x, blockIdx.y, blockIdx.z, x, y, nsa, nsb, tgtA, pqA,
                                    sgnA, nexcA, fcolA, fvalA, nnbrA, tgtBT, pqBT, sgnBT, nexcB,
                                    fcolB, fvalB, nnbrB, V, n, diag);
}

// Batched gather sigma: the flattened grid covers every molecule's
// (beta tile, alpha string, column) blocks; a block finds its molecule by binary
// search over the molecules' first blocks.
template <class T, bool EXACT_DIAG>
__global__ void __launch_bounds__(128)
k_sigma_gather_batch(const BatchMol* __restrict__ mols, int nmol) {
    const int64_t blk = blockIdx.x;
    int lo = 0, hi = nmol - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (mols[mid].sblk0 <= blk) lo = mid; else hi = mid - 1;
    }
    const BatchMol& m = mols[lo];
    const int64_t tiles = (m.nsb + 127) / 128;
    const int64_t local = blk - m.sblk0;
    const int64_t bx = local % tiles;
    const int64_t ia = (local / tiles) % m.nsa;
    const int64_t col = local / (tiles * m.nsa);
    sigma_gather_cta<T, EXACT_DIAG>(
        bx, ia, col, static_cast<const T*>(m.x), static_cast<T*>(m.y), m.nsa, m.nsb, m.tgtA,
        m.pqA, m.sgnA, m.nexcA, m.fcolA, static_cast<const T*>(m.fvalA), m.nnbrA, m.tgtBT,
        m.pqBT, m.sgnBT, m.nexcB, m.fcolB, static_cast<const T*>(m.fvalB), m.nnbrB,
        static_cast<const T*>(m.V), m.n, m.diag);
}

template <class T, bool ED>
static void launch_sigma(const SigmaArgs& a, const T* x, T* y, int ncol, const T* fvA,
                         const T* fvB, cudaStream_t st) {
    const SpinTables& A = *a.ta;
    const SpinTables& B = *a.tb;
    if (ncol <= 0 || a.dim == 0) return;
    dim3 grid((unsigned)((B.ns + 127) / 128), (unsigned)A.ns, (unsigned)ncol);
    size_t sm = (size_t)A.nnbr * (sizeof(T) + 4) + (size_t)A.nexc * 12 + 16;
    if (sm > 48 * 1024)
        KPM_CUDA(cudaFuncSetAttribute(k_sigma_gather<T, ED>,
                                      cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    k_sigma_gather<T, ED><<<grid, 128, sm, st>>>(
        x, y, A.ns, B.ns, A.tgt.as<int32_t>(), A.pq.as<uint16_t>(), A.sgn.as<int8_t>(), A.nexc,
        A.fcol.as<int32_t>(), fvA, A.nnbr, B.tgtT.as<int32_t>(), B.pqT.as<uint16_t>(),
        B.sgnT.as<int8_t>(), B.nexc, B.fcol.as<int32_t>(), fvB, B.nnbr,
        static_cast<const T*>(a.V), a.n, a.diag);
    KPM_LAUNCHED();
}

template <class T, bool ED>
static void launch_sigma_batch(const BatchMol* mols, int nmol, int64_t blocks, size_t smem,
                               cudaStream_t st) {
    if (nmol <= 0 || blocks <= 0) return;
    if (blocks > 0x7FFFFFFFLL) KPM_THROW(KPM_EINVAL, "batched sigma grid too large");
    if (smem > 48 * 1024)
        KPM_CUDA(cudaFuncSetAttribute(k_sigma_gather_batch<T, ED>,
                                      cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    k_sigma_gather_batch<T, ED><<<(unsigned)blocks, 128, smem, st>>>(mols, nmol);
    KPM_LAUNCHED();
}

void sigma_gather_batch_f64(const BatchMol* mols, int nmol, int64_t blocks, size_t smem,
                            cudaStream_t st) {
    launch_sigma_batch<double, false>(mols, nmol, blocks, smem, st);
}
void sigma_gather_batch_f32(const BatchMol* mols, int nmol, int64_t blocks, size_t smem,
                            cudaStream_t st) {
    launch_sigma_batch<float, true>(mols, nmol, blocks, smem, st);
}

void sigma_gather_f64(const SigmaArgs& a, const double* x, double* y, int ncol, cudaStream_t st) {
    launch_sigma<double, false>(a, x, y, ncol, a.ta->fval64.as<double>(),
                                a.tb->fval64.as<double>(), st);
}
void sigma_gather_f32(const SigmaArgs& a, const float* x, float* y, int ncol, cudaStream_t st) {
    launch_sigma<float, true>(a, x, y, ncol, a.ta->fval32.as<float>(), a.tb->fval32.as<float>(),
                              st);
}

// ---------------------------------------------------------------- exact diagonal

// H_II = F_alpha[I_a,I_a] + F_beta[I_b,I_b] + sum_{i in I_a, j in I_b} (ii|jj), FP64,
// stored as hi = float(H_II), lo = float(H_II - hi).
__global__ void __launch_bounds__(128)
k_diag(const uint32_t* __restrict__ maskA, const uint32_t* __restrict__ maskB, int64_t nsa,
       int64_t nsb, const double* __restrict__ fA0, const double* __restrict__ fB0,
       const double* __restrict__ eri, int n, float2* __restrict__ diag) {
    __shared__ double v[KPM_MAX_ORB];
    const int64_t ia = blockIdx.y;
    const uint32_t Ia = maskA[ia];
    if (threadIdx.x < n) {
        int j = threadIdx.x;
        double s = 0.0;
        for (int i = 0; i < n; ++i)
            if ((Ia >> i) & 1u) s += eri[(((int64_t)i * n + i) * n + j) * n + j];
        v[j] = s;
    }
    __syncthreads();
    const int64_t ib = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (ib >= nsb) return;
    uint32_t Ib = maskB[ib];
    double d = fA0[ia] + fB0[ib];
    while (Ib) {
        int j = __ffs(Ib) - 1;
        d += v[j];
        Ib &= Ib - 1;
    }
    float hi = (float)d;
    diag[ia * nsb + ib] = make_float2(hi, (float)(d - (double)hi));
}

void exact_diagonal(const SpinTables& A, const SpinTables& B, const double* eri, int n,
                    float2* diag, cudaStream_t st) {
    if (A.ns * B.ns == 0) return;
    dim3 grid((unsigned)((B.ns + 127) / 128), (unsigned)A.ns);
    k_diag<<<grid, 128, 0, st>>>(A.masks.as<uint32_t>(), B.masks.as<uint32_t>(), A.ns, B.ns,
                                 A.fval64.as<double>(), B.fval64.as<double>(), eri, n, diag);
    KPM_LAUNCHED();
}

// ---------------------------------------------------------------- dipole

template <class T>
__global__ void __launch_bounds__(128)
k_dipole(const double* __restrict__ psi, T* __restrict__ y, int64_t nsa, int64_t nsb,
         const int32_t* __restrict__ tgtA, const uint16_t* __restrict__ pqA,
         const int8_t* __restrict__ sgnA, int nexcA, const int32_t* __restrict__ tgtBT,
         const uint16_t* __restrict__ pqBT, const int8_t* __restrict__ sgnBT, int nexcB,
         const double* __restrict__ d) {
    const int64_t ia = blockIdx.y;
    const int64_t ib = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (ib >= nsb) return;
    double acc = 0.0;
    for (int e = 0; e < nexcA; ++e) {
        int64_t ja = tgtA[ia * nexcA + e];
        acc += d[pqA[ia * nexcA + e]] * (double)sgnA[ia * nexcA + e] * psi[ja * nsb + ib];
    }
    const double* prow = psi + ia * nsb;
    for (int f = 0; f < nexcB; ++f) {
        int64_t jb = tgtBT[(int64_t)f * nsb + ib];
        acc += d[pqBT[(int64_t)f * nsb + ib]] * (double)sgnBT[(int64_t)f * nsb + ib] * prow[jb];
    }
    y[ia * nsb + ib] = (T)(-acc);
}

// One block per alpha row I_a: the row psi[I_a][:] is staged in shared memory,
// so the beta terms (targets within the row) are read there; the alpha terms
// read whole rows psi[J_a][:] (coalesced across the block's threads).  Beta
// entries come from the packed table, 4 bytes per term.
template <class T>
__global__ void __launch_bounds__(256)
k_dipole_rows(const double* __restrict__ psi, T* __restrict__ y, int64_t nsb,
              const int32_t* __restrict__ tgtA, const uint16_t* __restrict__ pqA,
              const int8_t* __restrict__ sgnA, int nexcA, const uint32_t* __restrict__ pkB,
              int nexcB, const double* __restrict__ d, int nn) {
    extern __shared__ double sd[];
    double* row = sd;                                    // [nsb]
    double* cA = row + nsb;                              // [nexcA] signed coefficients
    int64_t* oA = reinterpret_cast<int64_t*>(cA + nexcA);  // [nexcA] row offsets
    double* dd = reinterpret_cast<double*>(oA + nexcA);  // [nn] dipole integrals
    const int64_t ia = blockIdx.x;
    for (int64_t j = threadIdx.x; j < nsb; j += blockDim.x) row[j] = psi[ia * nsb + j];
    for (int i = threadIdx.x; i < nn; i += blockDim.x) dd[i] = d[i];
    for (int e = threadIdx.x; e < nexcA; e += blockDim.x) {
        const int64_t k = ia * nexcA + e;
        cA[e] = d[pqA[k]] * (double)sgnA[k];
        oA[e] = (int64_t)tgtA[k] * nsb;
    }
    __syncthreads();
    for (int64_t ib = threadIdx.x; ib < nsb; ib += blockDim.x) {
        double acc = 0.0;
        for (int e = 0; e < nexcA; ++e) acc += cA[e] * psi[oA[e] + ib];
        for (int f = 0; f < nexcB; ++f) {
            const uint32_t w = pkB[(int64_t)f * nsb + ib];
            const double c = dd[(w >> 16) & 0x7FFFu];
            acc += ((w >> 31) ? -c : c) * row[w & 0xFFFFu];
        }
        y[ia * nsb + ib] = (T)(-acc);
    }
}

template <class T>
static void launch_dipole(const SpinTables& A, const SpinTables& B, const double* d,
                          const double* psi, T* y, cudaStream_t st) {
    if (A.ns * B.ns == 0) return;
    const int nn = A.n * A.n;
    const size_t smem = sizeof(double) * ((size_t)B.ns + 2 * (size_t)A.nexc + nn);
    if (smem <= 200 * 1024) {
        // per device; cheap, and the dipole runs once per request
        KPM_CUDA(cudaFuncSetAttribute(k_dipole_rows<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      200 * 1024));
        k_dipole_rows<T><<<(unsigned)A.ns, 256, smem, st>>>(
            psi, y, B.ns, A.tgt.as<int32_t>(), A.pq.as<uint16_t>(), A.sgn.as<int8_t>(), A.nexc,
            B.pkT.as<uint32_t>(), B.nexc, d, nn);
        KPM_LAUNCHED();
        return;
    }
    // rows too long for shared memory: gather the beta terms from global memory
    dim3 grid((unsigned)((B.ns + 127) / 128), (unsigned)A.ns);
    k_dipole<T><<<grid, 128, 0, st>>>(psi, y, A.ns, B.ns, A.tgt.as<int32_t>(),
                                      A.pq.as<uint16_t>(), A.sgn.as<int8_t>(), A.nexc,
                                      B.tgtT.as<int32_t>(), B.pqT.as<uint16_t>(),
                                      B.sgnT.as<int8_t>(), B.nexc, d);
    KPM_LAUNCHED();
}

void dipole_apply_f64(const SpinTables& ta, const SpinTables& tb, const double* d,
                      const double* psi, double* y, cudaStream_t st) {
    launch_dipole<double>(ta, tb, d, psi, y, st);
}
void dipole_apply_f32(const SpinTables& ta, const SpinTables& tb, const double* d,
                      const double* psi, float* y, cudaStream_t st) {
    launch_dipole<float>(ta, tb, d, psi, y, st);
}

}  // namespace kpm
