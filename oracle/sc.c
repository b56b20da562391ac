/*
 * Plain FP64 determinant-pair Slater-Condon Hamiltonian and one-body dipole.
 *
 * Test infrastructure: this file is part of the CPU oracle; only the tests, the
 * smoke check and the benchmark's CPU baseline load it.  It shares no code with
 * the CUDA library.
 *
 * Operator (Methods, "Mapping fermionic Hamiltonians to the qubits"): the
 * second-quantized electronic Hamiltonian with one-body integrals h_pq and
 * two-body integrals, here in chemist order (pq|rs):
 *     H = sum_{PQ} h_PQ a+_P a_Q + 1/2 sum_{PQRS} <PQ|RS> a+_P a+_Q a_S a_R,
 * over spin orbitals P = (p, sigma), with <PQ|RS> = (pr|qs) d(sP,sR) d(sQ,sS).
 * Dipole (Methods, "KPM for absorption spectra"): mu = -sum_pq d_pq
 * (c+_{p up} c_{q up} + c+_{p dn} c_{q dn}) - mu_c, with mu_c = 0 (no frozen
 * core in the synthetic systems).
 *
 * Determinants: spin orbital P = p for alpha, P = n + p for beta; a determinant
 * is the 2n-bit mask D = I_alpha | (I_beta << n) and its state is the product of
 * creators in ascending P order on the vacuum.  Its index is
 * rank_a(I_alpha) * N_beta + rank_b(I_beta).
 *
 * Matrix elements follow the Slater-Condon rules; every sign is obtained by
 * applying the annihilators and creators one at a time to the mask with the
 * Jordan-Wigner rule (sign (-1)^(occupied spin orbitals below the index)):
 *   diagonal:        sum_I h_II + 1/2 sum_{I,J} <IJ||IJ>
 *   single I->A:     s * (h_AI + sum_{J in D} <AJ||IJ>),   s = <D'|a+_A a_I|D>
 *   double IJ->AB:   s * <AB||IJ>,                         s = <D'|a+_A a+_B a_J a_I|D>
 * with <PQ||RS> = <PQ|RS> - <PQ|SR>.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
    int n, na, nb;
    int64_t nsa, nsb;
    const double* h1;      /* n*n */
    const double* eri;     /* n^4, (pq|rs) at ((p*n+q)*n+r)*n+s */
    const int64_t* masks_a;
    const int64_t* masks_b;
    const int64_t* rank_a; /* 2^n, -1 outside the sector */
    const int64_t* rank_b;
} sc_system;

static inline int popc64(uint64_t x) { return __builtin_popcountll(x); }

/* a_P |D>: returns 0 if empty, else +1/-1 and updates *D. */
static inline int annihilate(uint64_t* D, int P) {
    uint64_t b = (uint64_t)1 << P;
    if (!(*D & b)) return 0;
    int s = (popc64(*D & (b - 1)) & 1) ? -1 : 1;
    *D &= ~b;
    return s;
}
static inline int create(uint64_t* D, int P) {
    uint64_t b = (uint64_t)1 << P;
    if (*D & b) return 0;
    int s = (popc64(*D & (b - 1)) & 1) ? -1 : 1;
    *D |= b;
    return s;
}

static inline double chem(const sc_system* S, int p, int q, int r, int s) {
    int n = S->n;
    return S->eri[(((int64_t)p * n + q) * n + r) * n + s];
}
/* <PQ|RS> in spin orbitals */
static inline double phys(const sc_system* S, int P, int Q, int R, int Sx) {
    int n = S->n;
    if (P / n != R / n || Q / n != Sx / n) return 0.0;
    return chem(S, P % n, R % n, Q % n, Sx % n);
}
static inline double anti(const sc_system* S, int P, int Q, int R, int Sx) {
    return phys(S, P, Q, R, Sx) - phys(S, P, Q, Sx, R);
}
static inline double hso(const sc_system* S, int P, int Q) {
    int n = S->n;
    if (P / n != Q / n) return 0.0;
    return S->h1[(P % n) * n + (Q % n)];
}

static inline int64_t det_index(const sc_system* S, uint64_t D) {
    int n = S->n;
    uint64_t lo = D & (((uint64_t)1 << n) - 1);
    uint64_t hi = D >> n;
    int64_t ra = S->rank_a[lo], rb = S->rank_b[hi];
    if (ra < 0 || rb < 0) return -1;
    return ra * S->nsb + rb;
}

static inline uint64_t det_mask(const sc_system* S, int64_t row) {
    int64_t ia = row / S->nsb, ib = row % S->nsb;
    return (uint64_t)S->masks_a[ia] | ((uint64_t)S->masks_b[ib] << S->n);
}

int64_t sc_row_capacity(const sc_system* S) {
    int N = S->na + S->nb, V = 2 * S->n - N;
    return 1 + (int64_t)N * V + (int64_t)(N * (N - 1) / 2) * (V * (V - 1) / 2);
}

/* Row `row` of H: writes (column, value) pairs, returns how many. */
int64_t sc_row(const sc_system* S, int64_t row, int64_t* cols, double* vals) {
    int n2 = 2 * S->n;
    uint64_t D = det_mask(S, row);
    int occ[64], vac[64], no = 0, nv = 0;
    for (int P = 0; P < n2; ++P) {
        if ((D >> P) & 1) occ[no++] = P; else vac[nv++] = P;
    }
    int64_t k = 0;
    /* diagonal */
    double e = 0.0;
    for (int i = 0; i < no; ++i) {
        e += hso(S, occ[i], occ[i]);
        for (int j = 0; j < no; ++j) e += 0.5 * anti(S, occ[i], occ[j], occ[i], occ[j]);
    }
    cols[k] = row; vals[k] = e; ++k;
    /* singles */
    for (int i = 0; i < no; ++i) {
        int I = occ[i];
        for (int a = 0; a < nv; ++a) {
            int A = vac[a];
            if (I / S->n != A / S->n) continue;
            uint64_t Dp = D;
            int s = annihilate(&Dp, I);
            s *= create(&Dp, A);
            double v = hso(S, A, I);
            for (int j = 0; j < no; ++j) v += anti(S, A, occ[j], I, occ[j]);
            cols[k] = det_index(S, Dp); vals[k] = s * v; ++k;
        }
    }
    /* doubles */
    for (int i = 0; i < no; ++i)
        for (int j = i + 1; j < no; ++j) {
            int I = occ[i], J = occ[j];
            int si = I / S->n, sj = J / S->n;
            for (int a = 0; a < nv; ++a)
                for (int b = a + 1; b < nv; ++b) {
                    int A = vac[a], B = vac[b];
                    int sa = A / S->n, sb = B / S->n;
                    /* spin conservation: {sA, sB} == {sI, sJ} */
                    if (sa + sb != si + sj) continue;
                    uint64_t Dp = D;
                    int s = annihilate(&Dp, I);
                    s *= annihilate(&Dp, J);
                    s *= create(&Dp, B);
                    s *= create(&Dp, A);
                    double v = anti(S, A, B, I, J);
                    cols[k] = det_index(S, Dp); vals[k] = s * v; ++k;
                }
        }
    return k;
}

/* y[r] = sum_c H[rows[r], c] x[c] for the listed rows. */
void sc_sigma_rows(const sc_system* S, const int64_t* rows, int64_t nrows,
                   const double* x, double* y) {
    int64_t cap = sc_row_capacity(S);
#pragma omp parallel
    {
        int64_t* cols = (int64_t*)malloc(sizeof(int64_t) * cap);
        double* vals = (double*)malloc(sizeof(double) * cap);
#pragma omp for schedule(dynamic, 64)
        for (int64_t r = 0; r < nrows; ++r) {
            int64_t k = sc_row(S, rows[r], cols, vals);
            double acc = 0.0;
            for (int64_t t = 0; t < k; ++t) acc += vals[t] * x[cols[t]];
            y[r] = acc;
        }
        free(cols);
        free(vals);
    }
}

/* Test vector defined by an integer hash of the index, exactly representable in
 * FP32 and FP64: x(i) = ((((i * 0x9E3779B97F4A7C15) >> 48) & 0xFFFF) - 32768) * 2^-24
 * (64-bit wrap-around multiply).  Lets huge vectors be checked on sampled rows
 * without storing x on the host. */
static inline double hashvec(uint64_t i) {
    uint64_t h = (i * 0x9E3779B97F4A7C15ull) >> 48;
    return ((double)(int64_t)(h & 0xFFFFu) - 32768.0) * (1.0 / 16777216.0);
}

double sc_hashvec(int64_t i) { return hashvec((uint64_t)i); }

/* y[r] = sum_c H[rows[r], c] x(c) with x the hash vector above. */
void sc_sigma_rows_hash(const sc_system* S, const int64_t* rows, int64_t nrows, double* y) {
    int64_t cap = sc_row_capacity(S);
#pragma omp parallel
    {
        int64_t* cols = (int64_t*)malloc(sizeof(int64_t) * cap);
        double* vals = (double*)malloc(sizeof(double) * cap);
#pragma omp for schedule(dynamic, 16)
        for (int64_t r = 0; r < nrows; ++r) {
            int64_t k = sc_row(S, rows[r], cols, vals);
            double acc = 0.0;
            for (int64_t t = 0; t < k; ++t) acc += vals[t] * hashvec((uint64_t)cols[t]);
            y[r] = acc;
        }
        free(cols);
        free(vals);
    }
}

/* Full y = H x. */
void sc_sigma(const sc_system* S, const double* x, double* y) {
    int64_t dim = S->nsa * S->nsb;
    int64_t cap = sc_row_capacity(S);
#pragma omp parallel
    {
        int64_t* cols = (int64_t*)malloc(sizeof(int64_t) * cap);
        double* vals = (double*)malloc(sizeof(double) * cap);
#pragma omp for schedule(dynamic, 64)
        for (int64_t r = 0; r < dim; ++r) {
            int64_t k = sc_row(S, r, cols, vals);
            double acc = 0.0;
            for (int64_t t = 0; t < k; ++t) acc += vals[t] * x[cols[t]];
            y[r] = acc;
        }
        free(cols);
        free(vals);
    }
}

/* Y[c] = H X[c] for ncol columns stored one after the other ([ncol][dim]): each
 * row of H is generated once and applied to every column; per column the sum
 * is the one sc_sigma forms, term for term in the same order. */
void sc_sigma_block(const sc_system* S, const double* X, double* Y, int ncol) {
    int64_t dim = S->nsa * S->nsb;
    int64_t cap = sc_row_capacity(S);
#pragma omp parallel
    {
        int64_t* cols = (int64_t*)malloc(sizeof(int64_t) * cap);
        double* vals = (double*)malloc(sizeof(double) * cap);
#pragma omp for schedule(dynamic, 64)
        for (int64_t r = 0; r < dim; ++r) {
            int64_t k = sc_row(S, r, cols, vals);
            for (int c = 0; c < ncol; ++c) {
                const double* x = X + (int64_t)c * dim;
                double acc = 0.0;
                for (int64_t t = 0; t < k; ++t) acc += vals[t] * x[cols[t]];
                Y[(int64_t)c * dim + r] = acc;
            }
        }
        free(cols);
        free(vals);
    }
}

/* Number of stored entries of each row (for a CSR build). */
void sc_row_counts(const sc_system* S, int64_t* counts) {
    int64_t dim = S->nsa * S->nsb;
    int64_t cap = sc_row_capacity(S);
#pragma omp parallel
    {
        int64_t* cols = (int64_t*)malloc(sizeof(int64_t) * cap);
        double* vals = (double*)malloc(sizeof(double) * cap);
#pragma omp for schedule(dynamic, 64)
        for (int64_t r = 0; r < dim; ++r) counts[r] = sc_row(S, r, cols, vals);
        free(cols);
        free(vals);
    }
}

/* Fill CSR arrays; indptr must hold the prefix sums of sc_row_counts. */
void sc_fill_csr(const sc_system* S, const int64_t* indptr, int64_t* indices, double* data) {
    int64_t dim = S->nsa * S->nsb;
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t r = 0; r < dim; ++r) sc_row(S, r, indices + indptr[r], data + indptr[r]);
}

/* One-body dipole row-pull: y[r] = sum_c mu[rows[r], c] x[c],
 * mu = -sum_pq d_pq (E^alpha_pq + E^beta_pq). */
void sc_dipole_rows(const sc_system* S, const double* d, const int64_t* rows, int64_t nrows,
                    const double* x, double* y) {
    int n = S->n, n2 = 2 * n;
#pragma omp parallel for schedule(dynamic, 256)
    for (int64_t r = 0; r < nrows; ++r) {
        uint64_t D = det_mask(S, rows[r]);
        double acc = 0.0;
        for (int I = 0; I < n2; ++I) {
            if (!((D >> I) & 1)) continue;
            acc += -d[(I % n) * n + (I % n)] * x[rows[r]];
            for (int A = 0; A < n2; ++A) {
                if ((D >> A) & 1) continue;
                if (A / n != I / n) continue;
                uint64_t Dp = D;
                int s = annihilate(&Dp, I);
                s *= create(&Dp, A);
                acc += -d[(A % n) * n + (I % n)] * s * x[det_index(S, Dp)];
            }
        }
        y[r] = acc;
    }
}

int sc_omp_threads(void) {
#ifdef _OPENMP
    extern int omp_get_max_threads(void);
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* Sets the number of OpenMP threads of the later calls (n >= 1; a no-op without
   OpenMP): lets a caller time the oracle on one core as well as on all. */
void sc_set_threads(int n) {
#ifdef _OPENMP
    extern void omp_set_num_threads(int);
    if (n >= 1) omp_set_num_threads(n);
#else
    (void)n;
#endif
}
