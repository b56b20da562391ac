// H x in the Jordan-Wigner Pauli-string representation of the paper's qubit
// Hamiltonian (Methods, "Mapping fermionic Hamiltonians to the qubits"): a
// second way to apply the same H, for comparison with the determinant form.
//
// Qubits are the spin orbitals in this library's determinant order, alpha
// orbitals 0..n-1 then beta orbitals n..2n-1, so that the basis state of
// occupation bits b is the determinant (alpha creators ascending)(beta creators
// ascending)|vac> of the string tables.  With Z_{<q} the product of Z over qubits
// below q (|1> = occupied, Z|1> = -|1>),
//   a+_q = (X_q - i Y_q)/2 Z_{<q} = (X_q + X_q Z_q)/2 Z_{<q},
//   a_q  = (X_q + i Y_q)/2 Z_{<q} = (X_q - X_q Z_q)/2 Z_{<q},
// so every operator product is a real combination of strings X^x Z^z (x, z bit
// masks; Y never appears explicitly), and
//   (X^x1 Z^z1)(X^x2 Z^z2) = (-1)^{|z1 & x2|} X^(x1^x2) Z^(z1^z2).
// H = sum_PQ h_PQ a+_P a_Q + 1/2 sum_PQRS <PQ|RS> a+_P a+_Q a_S a_R over spin
// orbitals, <PQ|RS> = (pr|qs) for equal spins of P, R and of Q, S, expands into
// such strings on the host (a hash map merges equal ones); the device applies
// H x as a pull over strings grouped by their flip mask x:
//   sigma[b'] = sum_groups [b = b' ^ x in the sector] x[rank(b)] sum_t c_t (-1)^{|z_t & b|}.
#include <algorithm>
#include <cmath>
#include <unordered_map>
#include <vector>

#include "common.cuh"
#include "pauli.cuh"

namespace kpm {
namespace {

struct Term {
    uint64_t x, z;
    double c;
};

// a+_q or a_q as two X^x Z^z strings with coefficients 1/2, +-1/2
void ladder(int q, bool create, Term out[2]) {
    const uint64_t e = (uint64_t)1 << q, below = e - 1;
    out[0] = {e, below, 0.5};
    out[1] = {e, below ^ e, create ? 0.5 : -0.5};
}

// product of strings: (X^x1 Z^z1)(X^x2 Z^z2)
inline Term mul(const Term& a, const Term& b) {
    const int s = __builtin_popcountll(a.z & b.x) & 1;
    return {a.x ^ b.x, a.z ^ b.z, (s ? -1.0 : 1.0) * a.c * b.c};
}

struct Key {
    uint64_t x, z;
    bool operator==(const Key& o) const { return x == o.x && z == o.z; }
};
struct KeyHash {
    size_t operator()(const Key& k) const {
        uint64_t h = k.x * 0x9E3779B97F4A7C15ull ^ (k.z + 0x7F4A7C159E3779B9ull + (k.x << 6));
        return (size_t)(h ^ (h >> 29));
    }
};

// adds coef * (product of the ladder operators ops) to the map
void add_product(std::unordered_map<Key, double, KeyHash>& m, const int* qs, const bool* cr,
                 int k, double coef) {
    std::vector<Term> cur{{0, 0, coef}};
    for (int i = 0; i < k; ++i) {
        Term l[2];
        ladder(qs[i], cr[i], l);
        std::vector<Term> nxt;
        nxt.reserve(cur.size() * 2);
        for (const Term& t : cur)
            for (const Term& u : l) nxt.push_back(mul(t, u));
        cur.swap(nxt);
    }
    for (const Term& t : cur) m[Key{t.x, t.z}] += t.c;
}

template <class T>
__global__ void __launch_bounds__(128)
k_sigma_pauli(const T* __restrict__ x, T* __restrict__ y, int64_t nsa, int64_t nsb,
              const uint32_t* __restrict__ ma, const uint32_t* __restrict__ mb, int n, int na,
              int nb, int ngroups, const uint64_t* __restrict__ gx,
              const int32_t* __restrict__ gstart, const uint64_t* __restrict__ tz,
              const double* __restrict__ tc, Binom B) {
    const int64_t ia = blockIdx.y;
    const int64_t ib = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t col = blockIdx.z;
    if (ib >= nsb) return;
    const int64_t dim = nsa * nsb;
    x += col * dim;
    const uint64_t lowm = ((uint64_t)1 << n) - 1;
    const uint64_t bp = (uint64_t)ma[ia] | ((uint64_t)mb[ib] << n);
    double acc = 0.0;
    for (int g = 0; g < ngroups; ++g) {
        const uint64_t b = bp ^ gx[g];
        const uint32_t ba = (uint32_t)(b & lowm), bb = (uint32_t)(b >> n);
        if (__popc(ba) != na || __popc(bb) != nb) continue;
        double s = 0.0;
        for (int t = gstart[g]; t < gstart[g + 1]; ++t)
            s += (__popcll(tz[t] & b) & 1) ? -tc[t] : tc[t];
        uint32_t ra = 0, rb = 0;
        int k = 1;
        for (uint32_t mk = ba; mk; mk &= mk - 1, ++k) ra += B.c[__ffs(mk) - 1][k];
        k = 1;
        for (uint32_t mk = bb; mk; mk &= mk - 1, ++k) rb += B.c[__ffs(mk) - 1][k];
        acc += s * (double)x[(int64_t)ra * nsb + rb];
    }
    y[col * dim + ia * nsb + ib] = (T)acc;
}

}  // namespace

void PauliH::build(const double* h1, const double* eri, int norb, int nalpha, int nbeta) {
    n = norb;
    na = nalpha;
    nb = nbeta;
    const int N = 2 * n;
    std::unordered_map<Key, double, KeyHash> m;
    m.reserve(1 << 16);
    auto hso = [&](int P, int Q) { return (P / n == Q / n) ? h1[(P % n) * n + (Q % n)] : 0.0; };
    auto phys = [&](int P, int Q, int R, int S) {
        if (P / n != R / n || Q / n != S / n) return 0.0;
        const int p = P % n, q = Q % n, r = R % n, s = S % n;
        return eri[(((size_t)p * n + r) * n + q) * n + s];   // <PQ|RS> = (pr|qs)
    };
    for (int P = 0; P < N; ++P)
        for (int Q = 0; Q < N; ++Q) {
            const double c = hso(P, Q);
            if (c == 0.0) continue;
            const int qs[2] = {P, Q};
            const bool cr[2] = {true, false};
            add_product(m, qs, cr, 2, c);
        }
    for (int P = 0; P < N; ++P)
        for (int Q = 0; Q < N; ++Q) {
            if (P == Q) continue;
            for (int R = 0; R < N; ++R)
                for (int S = 0; S < N; ++S) {
                    if (R == S) continue;
                    const double c = 0.5 * phys(P, Q, R, S);
                    if (c == 0.0) continue;
                    const int qs[4] = {P, Q, S, R};
                    const bool cr[4] = {true, true, false, false};
                    add_product(m, qs, cr, 4, c);
                }
        }
    double mx = 0.0;
    for (auto& kv : m) mx = std::max(mx, std::fabs(kv.second));
    std::vector<Term> terms;
    terms.reserve(m.size());
    for (auto& kv : m)
        if (std::fabs(kv.second) > 1e-14 * mx) terms.push_back({kv.first.x, kv.first.z, kv.second});
    std::sort(terms.begin(), terms.end(), [](const Term& a, const Term& b) {
        return a.x != b.x ? a.x < b.x : a.z < b.z;
    });
    std::vector<uint64_t> hx, hz;
    std::vector<int32_t> hs;
    std::vector<double> hc;
    for (size_t i = 0; i < terms.size(); ++i) {
        if (i == 0 || terms[i].x != terms[i - 1].x) {
            hx.push_back(terms[i].x);
            hs.push_back((int32_t)i);
        }
        hz.push_back(terms[i].z);
        hc.push_back(terms[i].c);
    }
    hs.push_back((int32_t)terms.size());
    nterms = (int64_t)terms.size();
    ngroups = (int)hx.size();
    gx.alloc(std::max<size_t>(1, hx.size()) * 8);
    gstart.alloc(hs.size() * 4);
    tz.alloc(std::max<size_t>(1, hz.size()) * 8);
    tc.alloc(std::max<size_t>(1, hc.size()) * 8);
    if (!hx.empty()) KPM_CUDA(cudaMemcpy(gx.p, hx.data(), hx.size() * 8, cudaMemcpyHostToDevice));
    KPM_CUDA(cudaMemcpy(gstart.p, hs.data(), hs.size() * 4, cudaMemcpyHostToDevice));
    if (!hz.empty()) {
        KPM_CUDA(cudaMemcpy(tz.p, hz.data(), hz.size() * 8, cudaMemcpyHostToDevice));
        KPM_CUDA(cudaMemcpy(tc.p, hc.data(), hc.size() * 8, cudaMemcpyHostToDevice));
    }
    built = true;
}

template <class T>
static void launch_pauli(const PauliH& ph, const SpinTables& A, const SpinTables& B, const T* x,
                         T* y, int ncol, cudaStream_t st) {
    if (A.ns * B.ns == 0 || ncol <= 0) return;
    dim3 grid((unsigned)((B.ns + 127) / 128), (unsigned)A.ns, (unsigned)ncol);
    k_sigma_pauli<T><<<grid, 128, 0, st>>>(x, y, A.ns, B.ns, A.masks.as<uint32_t>(),
                                           B.masks.as<uint32_t>(), ph.n, ph.na, ph.nb,
                                           ph.ngroups, ph.gx.as<uint64_t>(),
                                           ph.gstart.as<int32_t>(), ph.tz.as<uint64_t>(),
                                           ph.tc.as<double>(), make_binom());
    KPM_LAUNCHED();
}

void PauliH::apply(const SpinTables& A, const SpinTables& B, const void* x, void* y, int ncol,
                   bool f64, cudaStream_t st) const {
    if (f64) launch_pauli<double>(*this, A, B, (const double*)x, (double*)y, ncol, st);
    else launch_pauli<float>(*this, A, B, (const float*)x, (float*)y, ncol, st);
}

}  // namespace kpm
