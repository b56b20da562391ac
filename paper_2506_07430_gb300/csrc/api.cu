// extern "C" entry points of include/kpm.h: context set-up, sigma/dipole
// dispatch, the KPM recursion loop, Lanczos bounds and the spectrum.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <memory>
#include <vector>

#include "common.cuh"
#include "pauli.cuh"
#include "sigma_tc.cuh"

using namespace kpm;

static thread_local std::string g_err = "no error";

namespace kpm {
void set_thread_error(const std::string& msg) { g_err = msg; }
}  // namespace kpm

struct kpm_ctx {
    int n = 0, na = 0, nb = 0;
    kpm_precision prec = KPM_FP64;
    cudaStream_t st = nullptr;
    int device = 0;
    int64_t dim = 0;
    std::string err = "no error";

    DevBuf d_h1, d_eri, d_dip, d_V32, d_diag;
    SpinTables ta, tb_own;
    SpinTables* tb = nullptr;
    std::unique_ptr<TcSigma> tc;  // tensor-core sigma (KPM_MIXED)
    std::unique_ptr<PauliH> pauli;  // Pauli-string form of H (built on first use)

    // recursion state
    int rec_ncol = 0, rec_steps = 0, rec_max_steps = 0;
    double rec_a = 1.0, rec_b = 0.0;
    DevBuf vA, vB, vS, dots, moments_dev, partials, counters, psi_tmp;
    void* rec_prev = nullptr;
    void* rec_cur = nullptr;
    // deflated recursion (kpm_recursion_begin_deflated): per column the weight c0^2
    // of the ground state in alpha_0 and x0 = (e0 - b)/a; FP64 scratch vectors
    bool rec_deflated = false;
    double rec_x0 = 0.0;
    DevBuf dfl_c, dfl_p, dfl_a;
    DevBuf x_ops, x_cross;            // kpm_moments_cross: operator integrals, cross dots

    // Lanczos state (spectral bounds, ground state)
    DevBuf lz_v0, lz_v1, lz_w, lz_ab, lz_scalar, lz_start;

    // profiling of H applications
    bool prof = false;
    std::vector<cudaEvent_t> ev;
    int ev_used = 0;

    // recursion steps replayed from CUDA graphs of two steps, one graph per
    // assignment of the two rotating vectors; the step index lives on the device
    bool graphs = true;
    cudaGraphExec_t gexec[2] = {nullptr, nullptr};
    uint64_t glaunches[2] = {0, 0};   // kernels in one replay (launch accounting)
    DevBuf step_ctr;                  // unsigned: index n of the next step's dots
    // batched steps led by this context: device BatchMol tables, their pinned
    // staging copy (reused once the event of the previous upload has passed), and
    // an event that orders this context's stream against a batch's stream
    DevBuf batch_desc;
    BatchMol* desc_host = nullptr;
    size_t desc_host_cap = 0;
    cudaEvent_t ev_desc = nullptr;
    cudaEvent_t ev_order = nullptr;
    cudaStream_t cap_st = nullptr;    // private stream for capture (any user stream may be
                                      // the legacy default stream, which cannot be captured)
    void drop_graphs() {
        for (auto& g : gexec) {
            if (g) cudaGraphExecDestroy(g);
            g = nullptr;
        }
    }

    ~kpm_ctx() {
        for (cudaEvent_t e : ev) cudaEventDestroy(e);
        drop_graphs();
        if (cap_st) cudaStreamDestroy(cap_st);
        if (ev_desc) cudaEventDestroy(ev_desc);
        if (ev_order) cudaEventDestroy(ev_order);
        if (desc_host) cudaFreeHost(desc_host);
    }

    size_t esz() const { return prec == KPM_FP64 ? 8 : 4; }
};

namespace {

struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        if (prev != dev) KPM_CUDA(cudaSetDevice(dev));
    }
    ~DeviceGuard() {
        int cur = -1;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

template <class F>
kpm_status guarded(kpm_ctx* ctx, F&& f) {
    try {
        f();
        return KPM_OK;
    } catch (const Error& e) {
        if (ctx) ctx->err = e.msg; else g_err = e.msg;
        return e.status;
    } catch (const std::bad_alloc&) {
        if (ctx) ctx->err = "host allocation failed"; else g_err = "host allocation failed";
        return KPM_ENOMEM;
    } catch (...) {
        if (ctx) ctx->err = "unknown error"; else g_err = "unknown error";
        return KPM_ECUDA;
    }
}

void check_sym(const double* m, int n, const char* what) {
    double mx = 0.0, d = 0.0;
    for (int i = 0; i < n * n; ++i) mx = std::fmax(mx, std::fabs(m[i]));
    for (int p = 0; p < n; ++p)
        for (int q = 0; q < n; ++q) d = std::fmax(d, std::fabs(m[p * n + q] - m[q * n + p]));
    if (!(d <= 1e-12 * std::fmax(1.0, mx)))
        KPM_THROW(KPM_EINVAL, "%s is not symmetric (max asymmetry %.3e)", what, d);
}

void check_eri(const double* e, int n) {
    double mx = 0.0, d = 0.0;
    int64_t n4 = (int64_t)n * n * n * n;
    for (int64_t i = 0; i < n4; ++i) {
        if (!std::isfinite(e[i])) KPM_THROW(KPM_EINVAL, "eri has a non-finite entry");
        mx = std::fmax(mx, std::fabs(e[i]));
    }
    auto at = [&](int p, int q, int r, int s) { return e[(((int64_t)p * n + q) * n + r) * n + s]; };
    for (int p = 0; p < n; ++p)
        for (int q = 0; q < n; ++q)
            for (int r = 0; r < n; ++r)
                for (int s = 0; s < n; ++s) {
                    double v = at(p, q, r, s);
                    d = std::fmax(d, std::fabs(v - at(q, p, r, s)));
                    d = std::fmax(d, std::fabs(v - at(p, q, s, r)));
                    d = std::fmax(d, std::fabs(v - at(r, s, p, q)));
                }
    if (!(d <= 1e-12 * std::fmax(1.0, mx)))
        KPM_THROW(KPM_EINVAL, "eri lacks 8-fold symmetry (max deviation %.3e)", d);
}

void require_device() {
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
        cudaGetLastError();
        KPM_THROW(KPM_ECUDA, "no CUDA device available");
    }
}

void sigma_dispatch(kpm_ctx* c, const void* x, void* y, int ncol) {
    if (c->prec == KPM_FP64) {
        SigmaArgs a{&c->ta, c->tb, c->d_eri.p, c->n, c->dim};
        sigma_gather_f64(a, (const double*)x, (double*)y, ncol, c->st);
    } else if (c->prec == KPM_FP32) {
        SigmaArgs a{&c->ta, c->tb, c->d_V32.p, c->n, c->dim, c->d_diag.as<float2>()};
        sigma_gather_f32(a, (const float*)x, (float*)y, ncol, c->st);
    } else {
        c->tc->apply((const float*)x, (float*)y, ncol, c->st);
    }
}

void dipole_dispatch(kpm_ctx* c, int comp, const double* psi, void* y) {
    const double* d = c->d_dip.as<double>() + (int64_t)comp * c->n * c->n;
    if (c->prec == KPM_FP64) dipole_apply_f64(c->ta, *c->tb, d, psi, (double*)y, c->st);
    else dipole_apply_f32(c->ta, *c->tb, d, psi, (float*)y, c->st);
}

void update_dispatch(kpm_ctx* c, const void* s, const void* cur, void* prev, int first,
                     double* dots, const unsigned* step) {
    int64_t dstride = (int64_t)c->rec_max_steps * 2;
    if (c->prec == KPM_FP64)
        cheb_update_f64((const double*)s, (const double*)cur, (double*)prev, c->dim, c->rec_ncol,
                        c->rec_a, c->rec_b, first, c->partials.as<double>(),
                        c->counters.as<unsigned>(), dots, dstride, step, c->st);
    else
        cheb_update_f32((const float*)s, (const float*)cur, (float*)prev, c->dim, c->rec_ncol,
                        c->rec_a, c->rec_b, first, c->partials.as<double>(),
                        c->counters.as<unsigned>(), dots, dstride, step, c->st);
}

void ensure_reduce_scratch(kpm_ctx* c, int ncol) {
    size_t pb = (size_t)ncol * 1216 * 2 * sizeof(double);
    if (c->partials.bytes < pb) c->partials.alloc(pb);
    size_t cb = (size_t)ncol * sizeof(unsigned) + 64;
    if (c->counters.bytes < cb) {
        c->counters.alloc(cb);
        KPM_CUDA(cudaMemsetAsync(c->counters.p, 0, cb, c->st));
    }
}

void rec_begin(kpm_ctx* c, const double* psi0, unsigned mask, double a, double b, int max_moments) {
    if (!psi0) KPM_THROW(KPM_EINVAL, "psi0 is NULL");
    if ((mask & ~7u) || !mask) KPM_THROW(KPM_EINVAL, "comp_mask must be a non-empty subset of {1,2,4}");
    if (max_moments < 2 || (max_moments & 1)) KPM_THROW(KPM_EINVAL, "nmoments must be even and >= 2");
    if (!(a > 0.0) || !std::isfinite(a) || !std::isfinite(b)) KPM_THROW(KPM_EINVAL, "need a > 0 and finite a, b");
    int ncol = __builtin_popcount(mask);
    c->rec_ncol = ncol;
    c->rec_max_steps = max_moments / 2;
    c->rec_a = a;
    c->rec_b = b;
    size_t vb = (size_t)ncol * c->dim * c->esz();
    c->vA.ensure(vb);
    c->vB.ensure(vb);
    c->vS.ensure(vb);
    size_t db = (size_t)ncol * c->rec_max_steps * 2 * sizeof(double);
    c->dots.ensure(db);
    c->moments_dev.ensure(db);
    ensure_reduce_scratch(c, ncol);
    int j = 0;
    for (int comp = 0; comp < 3; ++comp) {
        if (!((mask >> comp) & 1)) continue;
        dipole_dispatch(c, comp, psi0, (char*)c->vB.p + (size_t)j * c->dim * c->esz());
        ++j;
    }
    sigma_dispatch(c, c->vB.p, c->vS.p, ncol);
    update_dispatch(c, c->vS.p, c->vB.p, c->vA.p, 1, c->dots.as<double>(), nullptr);
    c->rec_prev = c->vB.p;  // alpha_0
    c->rec_cur = c->vA.p;   // alpha_1
    c->rec_steps = 1;
    c->rec_deflated = false;
    // buffers may have moved: captured steps are stale
    c->drop_graphs();
    c->step_ctr.ensure(sizeof(unsigned));
    step_set(c->step_ctr.as<unsigned>(), 1u, c->st);
}

// As rec_begin for a ground state psi0 with eigenvalue e0: alpha_0 = mu psi0 is
// split into c0 p + alpha_perp (p = psi0 / |psi0|, c0 = <p|alpha_0>, all in FP64,
// alpha_perp then stored in the context precision)
// and the recursion runs on alpha_perp; the collected moments add c0^2 T_n(x0),
// x0 = (e0 - b)/a, which is <c0 p|T_n(H~)|c0 p> for an eigenvector (the cross
// terms vanish since T_n(H~) p = T_n(x0) p is orthogonal to alpha_perp).
void rec_begin_deflated(kpm_ctx* c, const double* psi0, double e0, unsigned mask, double a,
                        double b, int max_moments) {
    if (!psi0) KPM_THROW(KPM_EINVAL, "psi0 is NULL");
    if ((mask & ~7u) || !mask) KPM_THROW(KPM_EINVAL, "comp_mask must be a non-empty subset of {1,2,4}");
    if (max_moments < 2 || (max_moments & 1)) KPM_THROW(KPM_EINVAL, "nmoments must be even and >= 2");
    if (!(a > 0.0) || !std::isfinite(a) || !std::isfinite(b)) KPM_THROW(KPM_EINVAL, "need a > 0 and finite a, b");
    const double x0 = (e0 - b) / a;
    if (!std::isfinite(e0) || !(std::fabs(x0) <= 1.0))
        KPM_THROW(KPM_EINVAL, "e0 must lie in [b - a, b + a]");
    const int ncol = __builtin_popcount(mask);
    c->rec_ncol = ncol;
    c->rec_max_steps = max_moments / 2;
    c->rec_a = a;
    c->rec_b = b;
    const size_t vb = (size_t)ncol * c->dim * c->esz();
    c->vA.ensure(vb);
    c->vB.ensure(vb);
    c->vS.ensure(vb);
    const size_t db = (size_t)ncol * c->rec_max_steps * 2 * sizeof(double);
    c->dots.ensure(db);
    c->moments_dev.ensure(db);
    ensure_reduce_scratch(c, ncol);
    const bool f64 = c->prec == KPM_FP64;
    const int64_t dim = c->dim;
    c->dfl_c.ensure(sizeof(double) * 8);
    c->dfl_p.ensure((size_t)dim * 8);
    c->dfl_a.ensure((size_t)dim * 8);
    double* cc = c->dfl_c.as<double>();         // [0] |psi0|^2, [1] c0 of a column, [4 + col] c0^2
    double* p = c->dfl_p.as<double>();
    double* al = c->dfl_a.as<double>();
    double* parts = c->partials.as<double>();
    unsigned* cnt = c->counters.as<unsigned>();
    KPM_CUDA(cudaMemcpyAsync(p, psi0, (size_t)dim * 8, cudaMemcpyDeviceToDevice, c->st));
    dot_dev(p, p, dim, true, parts, cnt, cc, c->st);
    scale_inplace(p, dim, true, cc, c->st);
    int j = 0;
    for (int comp = 0; comp < 3; ++comp) {
        if (!((mask >> comp) & 1)) continue;
        const double* d = c->d_dip.as<double>() + (int64_t)comp * c->n * c->n;
        dipole_apply_f64(c->ta, *c->tb, d, psi0, al, c->st);
        dot_dev(p, al, dim, true, parts, cnt, cc + 1, c->st);
        deflate(al, p, dim, cc + 1, (char*)c->vB.p + (size_t)j * dim * c->esz(), f64, c->st);
        square_into(cc + 1, cc + 4 + j, c->st);
        ++j;
    }
    sigma_dispatch(c, c->vB.p, c->vS.p, ncol);
    update_dispatch(c, c->vS.p, c->vB.p, c->vA.p, 1, c->dots.as<double>(), nullptr);
    c->rec_prev = c->vB.p;
    c->rec_cur = c->vA.p;
    c->rec_steps = 1;
    c->rec_deflated = true;
    c->rec_x0 = x0;
    c->drop_graphs();
    c->step_ctr.ensure(sizeof(unsigned));
    step_set(c->step_ctr.as<unsigned>(), 1u, c->st);
}

// one Chebyshev step alpha_{n+1} = 2 (H~ alpha_n) - alpha_{n-1}, dots of step n
void step_direct(kpm_ctx* c) {
    if (c->prof) {
        if ((int)c->ev.size() < c->ev_used + 2) {
            cudaEvent_t e0, e1;
            KPM_CUDA(cudaEventCreate(&e0));
            KPM_CUDA(cudaEventCreate(&e1));
            c->ev.push_back(e0);
            c->ev.push_back(e1);
        }
        KPM_CUDA(cudaEventRecord(c->ev[c->ev_used], c->st));
        sigma_dispatch(c, c->rec_cur, c->vS.p, c->rec_ncol);
        KPM_CUDA(cudaEventRecord(c->ev[c->ev_used + 1], c->st));
        c->ev_used += 2;
    } else {
        sigma_dispatch(c, c->rec_cur, c->vS.p, c->rec_ncol);
    }
    update_dispatch(c, c->vS.p, c->rec_cur, c->rec_prev, 0, c->dots.as<double>(),
                    c->step_ctr.as<unsigned>());
    step_inc(c->step_ctr.as<unsigned>(), c->st);
    std::swap(c->rec_prev, c->rec_cur);
    ++c->rec_steps;
}

// Captures two steps from the current vector assignment into graph slot gi, on
// the context's private capture stream; host state is restored (capture
// executes nothing).  Returns false, with graphs disabled for the context, if
// the capture fails.
bool capture_two_steps(kpm_ctx* c, int gi) {
    if (!c->cap_st && cudaStreamCreateWithFlags(&c->cap_st, cudaStreamNonBlocking) != cudaSuccess) {
        cudaGetLastError();
        c->cap_st = nullptr;
        c->graphs = false;
        return false;
    }
    void* cur0 = c->rec_cur;
    void* prev0 = c->rec_prev;
    const int steps0 = c->rec_steps;
    const uint64_t l0 = g_launches.load();
    cudaStream_t user_st = c->st;
    cudaGraph_t graph = nullptr;
    c->st = c->cap_st;
    bool ok = cudaStreamBeginCapture(c->st, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
    if (ok) {
        try {
            step_direct(c);
            step_direct(c);
        } catch (...) {
            ok = false;
        }
        ok = (cudaStreamEndCapture(c->st, &graph) == cudaSuccess) && ok && graph;
    }
    c->st = user_st;
    if (ok) ok = cudaGraphInstantiate(&c->gexec[gi], graph, 0) == cudaSuccess;
    if (graph) cudaGraphDestroy(graph);
    c->glaunches[gi] = g_launches.load() - l0;
    g_launches.fetch_sub(c->glaunches[gi]);
    c->rec_cur = cur0;
    c->rec_prev = prev0;
    c->rec_steps = steps0;
    if (!ok) {
        cudaGetLastError();
        c->gexec[gi] = nullptr;
        c->graphs = false;
    }
    return ok;
}

void rec_advance(kpm_ctx* c, int nsteps) {
    if (c->rec_steps <= 0) KPM_THROW(KPM_EINVAL, "no recursion in progress");
    if (nsteps < 0 || c->rec_steps + nsteps > c->rec_max_steps)
        KPM_THROW(KPM_EINVAL, "advance past the requested number of moments");
    int k = 0;
    while (k < nsteps) {
        if (c->graphs && !c->prof && nsteps - k >= 2) {
            // two steps leave the two rotating vectors where they were
            const int gi = c->rec_cur == c->vA.p ? 0 : 1;
            if (c->gexec[gi] || capture_two_steps(c, gi)) {
                KPM_CUDA(cudaGraphLaunch(c->gexec[gi], c->st));
                g_launches.fetch_add(c->glaunches[gi]);
                c->rec_steps += 2;
                k += 2;
                continue;
            }
        }
        step_direct(c);
        ++k;
    }
}

// Batched steps (kpm_moments_batch, kpm_recursion_advance_batch): contexts of
// one batch are distinct, on one device, all on the gather path (FP64 or FP32).
void check_batch(kpm_ctx* const* ctxs, int count) {
    const kpm_ctx* c0 = ctxs[0];
    for (int i = 0; i < count; ++i) {
        const kpm_ctx* c = ctxs[i];
        if (!c) KPM_THROW(KPM_EINVAL, "context %d is NULL", i);
        if (c->prec != KPM_FP64 && c->prec != KPM_FP32)
            KPM_THROW(KPM_EINVAL, "batched steps run the gather path: FP64 or FP32 contexts "
                                  "only (context %d)", i);
        if (c->prec != c0->prec) KPM_THROW(KPM_EINVAL, "contexts of a batch share one precision");
        if (c->device != c0->device) KPM_THROW(KPM_EINVAL, "contexts of a batch share one device");
        for (int j = 0; j < i; ++j)
            if (ctxs[j] == c) KPM_THROW(KPM_EINVAL, "context %d appears twice", i);
    }
}

cudaEvent_t order_event(kpm_ctx* c) {
    if (!c->ev_order) KPM_CUDA(cudaEventCreateWithFlags(&c->ev_order, cudaEventDisableTiming));
    return c->ev_order;
}

// nsteps Chebyshev steps of every context's recursion (each mid-recursion, at its
// own step) as one sigma and one update launch per step on ctxs[0]'s stream,
// ordered after each context's queued work and before its later work by events.
void batch_steps(kpm_ctx* const* ctxs, int count, int nsteps) {
    if (nsteps <= 0) return;
    kpm_ctx* c0 = ctxs[0];
    cudaStream_t st = c0->st;
    for (int i = 1; i < count; ++i)
        if (ctxs[i]->st != st) {
            KPM_CUDA(cudaEventRecord(order_event(ctxs[i]), ctxs[i]->st));
            KPM_CUDA(cudaStreamWaitEvent(st, ctxs[i]->ev_order, 0));
        }
    const bool f64 = c0->prec == KPM_FP64;
    // operand tables for the two assignments of the rotating vectors, staged in
    // pinned memory (the previous upload from it must have been read first)
    const size_t need = (size_t)2 * count;
    if (c0->ev_desc) KPM_CUDA(cudaEventSynchronize(c0->ev_desc));
    else KPM_CUDA(cudaEventCreateWithFlags(&c0->ev_desc, cudaEventDisableTiming));
    if (c0->desc_host_cap < need) {
        if (c0->desc_host) cudaFreeHost(c0->desc_host);
        c0->desc_host = nullptr;
        c0->desc_host_cap = 0;
        KPM_CUDA(cudaMallocHost(&c0->desc_host, need * sizeof(BatchMol)));
        c0->desc_host_cap = need;
    }
    BatchMol* h = c0->desc_host;
    int64_t sblk = 0, ublk = 0;
    size_t smem = 16;
    for (int i = 0; i < count; ++i) {
        kpm_ctx* c = ctxs[i];
        const SpinTables& A = c->ta;
        const SpinTables& B = *c->tb;
        BatchMol m{};
        m.nsa = A.ns;
        m.nsb = B.ns;
        m.tgtA = A.tgt.as<int32_t>();
        m.pqA = A.pq.as<uint16_t>();
        m.sgnA = A.sgn.as<int8_t>();
        m.fcolA = A.fcol.as<int32_t>();
        m.fvalA = f64 ? A.fval64.p : A.fval32.p;
        m.tgtBT = B.tgtT.as<int32_t>();
        m.pqBT = B.pqT.as<uint16_t>();
        m.sgnBT = B.sgnT.as<int8_t>();
        m.fcolB = B.fcol.as<int32_t>();
        m.fvalB = f64 ? B.fval64.p : B.fval32.p;
        m.V = f64 ? c->d_eri.p : c->d_V32.p;
        m.diag = f64 ? nullptr : c->d_diag.as<float2>();
        m.nexcA = A.nexc;
        m.nnbrA = A.nnbr;
        m.nexcB = B.nexc;
        m.nnbrB = B.nnbr;
        m.n = c->n;
        m.ncol = c->rec_ncol;
        m.a = c->rec_a;
        m.b = c->rec_b;
        m.partials = c->partials.as<double>();
        m.counters = c->counters.as<unsigned>();
        m.dots = c->dots.as<double>();
        m.dstride = (int64_t)c->rec_max_steps * 2;
        m.step0 = c->rec_steps;
        m.nblk = reduce_blocks(c->dim);
        m.sblk0 = sblk;
        m.ublk0 = ublk;
        sblk += (B.ns + 127) / 128 * A.ns * m.ncol;
        ublk += (int64_t)m.nblk * m.ncol;
        smem = std::max(smem, (size_t)A.nnbr * ((f64 ? 8 : 4) + 4) + (size_t)A.nexc * 12 + 16);
        // even batch steps: the current assignment; odd: swapped
        m.x = c->rec_cur;
        m.y = c->vS.p;
        m.prev = c->rec_prev;
        h[i] = m;
        m.x = c->rec_prev;
        m.prev = c->rec_cur;
        h[(size_t)count + i] = m;
    }
    c0->batch_desc.ensure(need * sizeof(BatchMol));
    KPM_CUDA(cudaMemcpyAsync(c0->batch_desc.p, h, need * sizeof(BatchMol), cudaMemcpyHostToDevice,
                             st));
    KPM_CUDA(cudaEventRecord(c0->ev_desc, st));
    const BatchMol* d = c0->batch_desc.as<BatchMol>();
    for (int k = 0; k < nsteps; ++k) {
        const BatchMol* dk = d + (size_t)(k & 1) * count;
        if (f64) {
            sigma_gather_batch_f64(dk, count, sblk, smem, st);
            cheb_update_batch_f64(dk, count, ublk, k, st);
        } else {
            sigma_gather_batch_f32(dk, count, sblk, smem, st);
            cheb_update_batch_f32(dk, count, ublk, k, st);
        }
    }
    for (int i = 0; i < count; ++i) {
        kpm_ctx* c = ctxs[i];
        if (nsteps & 1) std::swap(c->rec_prev, c->rec_cur);
        c->rec_steps += nsteps;
        // device step counter for later graph-replayed steps of this context
        step_set(c->step_ctr.as<unsigned>(), (unsigned)c->rec_steps, st);
    }
    KPM_CUDA(cudaEventRecord(order_event(c0), st));
    for (int i = 1; i < count; ++i)
        if (ctxs[i]->st != st) KPM_CUDA(cudaStreamWaitEvent(ctxs[i]->st, c0->ev_order, 0));
}

void check_device_errors(kpm_ctx* c) {
    if (c->tc && c->tc->check(c->st))
        KPM_THROW(KPM_ETIMEOUT, "a bounded wait in the tensor-core sigma kernel ran out");
}

kpm_status rec_collect(kpm_ctx* c, double* out, int nm_stride) {
    int ns = c->rec_steps;
    doubling_combine(c->dots.as<double>(), c->rec_ncol, ns, (int64_t)c->rec_max_steps * 2,
                     c->moments_dev.as<double>(), 2 * c->rec_max_steps,
                     c->rec_deflated ? c->dfl_c.as<double>() + 4 : nullptr, c->rec_x0, c->st);
    for (int j = 0; j < c->rec_ncol; ++j)
        KPM_CUDA(cudaMemcpyAsync(out + (size_t)j * nm_stride,
                                 c->moments_dev.as<double>() + (size_t)j * 2 * c->rec_max_steps,
                                 sizeof(double) * 2 * ns, cudaMemcpyDeviceToHost, c->st));
    KPM_CUDA(cudaStreamSynchronize(c->st));
    check_device_errors(c);
    for (int j = 0; j < c->rec_ncol; ++j) {
        const double* m = out + (size_t)j * nm_stride;
        double lim = m[0] * (1.0 + 1e-6);
        for (int i = 0; i < 2 * ns; ++i)
            if (!std::isfinite(m[i]) || std::fabs(m[i]) > lim) {
                c->err = "|Omega_n| exceeds Omega_0: [b-a, b+a] does not contain the spectrum";
                return KPM_EBOUNDS;
            }
    }
    return KPM_OK;
}

}  // namespace

extern "C" {

kpm_status kpm_create(const double* h1, const double* eri, const double* dipole, int norb,
                      int nalpha, int nbeta, kpm_precision prec, void* cuda_stream,
                      kpm_ctx** out) {
    if (out) *out = nullptr;
    std::unique_ptr<kpm_ctx> c;
    kpm_status s = guarded(nullptr, [&] {
        if (!out || !h1 || !eri || !dipole) KPM_THROW(KPM_EINVAL, "NULL argument");
        if (norb < 1 || norb > KPM_MAX_ORB)
            KPM_THROW(KPM_EINVAL, "norb must be in 1..%d", KPM_MAX_ORB);
        if (nalpha < 0 || nbeta < 0 || nalpha > norb || nbeta > norb)
            KPM_THROW(KPM_EINVAL, "electron counts must be in 0..norb");
        if (prec != KPM_FP64 && prec != KPM_FP32 && prec != KPM_MIXED && prec != KPM_MIXED_BF16)
            KPM_THROW(KPM_EINVAL, "unknown precision %d", (int)prec);
        check_sym(h1, norb, "h1");
        for (int cc = 0; cc < 3; ++cc) check_sym(dipole + (size_t)cc * norb * norb, norb, "dipole");
        check_eri(eri, norb);
        require_device();
        c.reset(new kpm_ctx());
        KPM_CUDA(cudaGetDevice(&c->device));
        c->n = norb;
        c->na = nalpha;
        c->nb = nbeta;
        c->prec = prec;
        c->st = (cudaStream_t)cuda_stream;
        int64_t n2 = (int64_t)norb * norb, n4 = n2 * n2;
        c->d_h1.alloc(n2 * 8);
        c->d_eri.alloc(n4 * 8);
        c->d_dip.alloc(3 * n2 * 8);
        KPM_CUDA(cudaMemcpyAsync(c->d_h1.p, h1, n2 * 8, cudaMemcpyHostToDevice, c->st));
        KPM_CUDA(cudaMemcpyAsync(c->d_eri.p, eri, n4 * 8, cudaMemcpyHostToDevice, c->st));
        KPM_CUDA(cudaMemcpyAsync(c->d_dip.p, dipole, 3 * n2 * 8, cudaMemcpyHostToDevice, c->st));
        build_spin_tables(c->ta, norb, nalpha, c->d_h1.as<double>(), c->d_eri.as<double>(), c->st);
        if (nbeta == nalpha) {
            c->tb = &c->ta;
        } else {
            build_spin_tables(c->tb_own, norb, nbeta, c->d_h1.as<double>(), c->d_eri.as<double>(),
                              c->st);
            c->tb = &c->tb_own;
        }
        c->dim = c->ta.ns * c->tb->ns;
        if (prec == KPM_FP32) {
            c->d_V32.alloc(n4 * 4);
            to_f32(c->d_eri.as<double>(), c->d_V32.as<float>(), n4, c->st);
            c->d_diag.alloc((size_t)c->dim * sizeof(float2));
            exact_diagonal(c->ta, *c->tb, c->d_eri.as<double>(), norb, c->d_diag.as<float2>(), c->st);
        }
        if (prec == KPM_MIXED || prec == KPM_MIXED_BF16) {
            // W over unordered pairs {p<=q}: rows (pq|rs) and the one-body row k_pq.
            // wmax = max |W|, wcol = max over output pairs of the column sum of |W|.
            double wmax = 0.0, wcol = 0.0;
            auto eri_at = [&](int p, int q, int r, int s) {
                return eri[(((int64_t)p * norb + q) * norb + r) * norb + s];
            };
            for (int r = 0; r < norb; ++r)
                for (int s = r; s < norb; ++s) {
                    double k = h1[r * norb + s];
                    for (int t = 0; t < norb; ++t) k -= 0.5 * eri_at(r, t, t, s);
                    double col = std::fabs(k);
                    wmax = std::fmax(wmax, std::fabs(k));
                    for (int p = 0; p < norb; ++p)
                        for (int q = p; q < norb; ++q) {
                            double v = std::fabs(eri_at(p, q, r, s));
                            col += v;
                            wmax = std::fmax(wmax, v);
                        }
                    wcol = std::fmax(wcol, col);
                }
            // the diagonal of H in FP64 (hi + lo floats), added exactly after the
            // reduced-precision products, which leave it out
            c->d_diag.alloc((size_t)c->dim * sizeof(float2));
            exact_diagonal(c->ta, *c->tb, c->d_eri.as<double>(), norb, c->d_diag.as<float2>(), c->st);
            c->tc.reset(new TcSigma());
            c->tc->init(c->ta, *c->tb, c->d_h1.as<double>(), c->d_eri.as<double>(),
                        c->d_diag.as<float2>(), norb, wmax, wcol, prec == KPM_MIXED, c->st);
        }
        KPM_CUDA(cudaStreamSynchronize(c->st));
    });
    if (s == KPM_OK) *out = c.release();
    return s;
}

void kpm_destroy(kpm_ctx* ctx) {
    if (!ctx) return;
    cudaStreamSynchronize(ctx->st);
    delete ctx;
}

const char* kpm_last_error(const kpm_ctx* ctx) { return ctx ? ctx->err.c_str() : g_err.c_str(); }

int64_t kpm_dim(const kpm_ctx* ctx) { return ctx ? ctx->dim : -1; }

int64_t kpm_nstrings(const kpm_ctx* ctx, int spin) {
    if (!ctx || (spin != 0 && spin != 1)) return -1;
    return spin == 0 ? ctx->ta.ns : ctx->tb->ns;
}

int kpm_nexc(const kpm_ctx* ctx, int spin) {
    if (!ctx || (spin != 0 && spin != 1)) return -1;
    return spin == 0 ? ctx->ta.nexc : ctx->tb->nexc;
}

kpm_status kpm_string_table(const kpm_ctx* ctx_c, int spin, uint32_t* masks, int32_t* tgt,
                            uint16_t* pq, int8_t* sgn) {
    kpm_ctx* ctx = const_cast<kpm_ctx*>(ctx_c);
    if (!ctx) { g_err = "NULL context"; return KPM_EINVAL; }
    return guarded(ctx, [&] {
        if (spin != 0 && spin != 1) KPM_THROW(KPM_EINVAL, "spin must be 0 or 1");
        DeviceGuard g(ctx->device);
        const SpinTables& t = spin == 0 ? ctx->ta : *ctx->tb;
        size_t ne = (size_t)t.ns * t.nexc;
        KPM_CUDA(cudaStreamSynchronize(ctx->st));
        if (masks) KPM_CUDA(cudaMemcpy(masks, t.masks.p, t.ns * 4, cudaMemcpyDeviceToHost));
        if (tgt && ne) KPM_CUDA(cudaMemcpy(tgt, t.tgt.p, ne * 4, cudaMemcpyDeviceToHost));
        if (pq && ne) KPM_CUDA(cudaMemcpy(pq, t.pq.p, ne * 2, cudaMemcpyDeviceToHost));
        if (sgn && ne) KPM_CUDA(cudaMemcpy(sgn, t.sgn.p, ne, cudaMemcpyDeviceToHost));
    });
}

kpm_status kpm_sigma(kpm_ctx* ctx, const void* x, void* y, int ncol) {
    if (!ctx) { g_err = "NULL context"; return KPM_EINVAL; }
    return guarded(ctx, [&] {
        if (!x || !y || ncol < 1 || ncol > 64) KPM_THROW(KPM_EINVAL, "bad sigma arguments");
        if (x == y) KPM_THROW(KPM_EINVAL, "x and y must not alias");
        DeviceGuard g(ctx->device);
        sigma_dispatch(ctx, x, y, ncol);
    });
}

// builds the Pauli-string form of H from the context's integrals on first use
static PauliH& pauli_of(kpm_ctx* ctx) {
    if (!ctx->pauli) {
        const int n = ctx->n;
        std::vector<double> h1((size_t)n * n), eri((size_t)n * n * n * n);
        KPM_CUDA(cudaStreamSynchronize(ctx->st));
        KPM_CUDA(cudaMemcpy(h1.data(), ctx->d_h1.p, h1.size() * 8, cudaMemcpyDeviceToHost));
        KPM_CUDA(cudaMemcpy(eri.data(), ctx->d_eri.p, eri.size() * 8, cudaMemcpyDeviceToHost));
        auto p = std::make_unique<PauliH>();
        p->build(h1.data(), eri.data(), n, ctx->na, ctx->nb);
        ctx->pauli = std::move(p);
    }
    return *ctx->pauli;
}

kpm_status kpm_sigma_pauli(kpm_ctx* ctx, const void* x, void* y, int ncol) {
    if (!ctx) { g_err = "NULL context"; return KPM_EINVAL; }
    return guarded(ctx, [&] {
        if (!x || !y || ncol < 1 || ncol > 64) KPM_THROW(KPM_EINVAL, "bad sigma arguments");
        if (x == y) KPM_THROW(KPM_EINVAL, "x and y must not alias");
        DeviceGuard g(ctx->device);
        PauliH& ph = pauli_of(ctx);
        ph.apply(ctx->ta, *ctx->tb, x, y, ncol, ctx->prec == KPM_FP64, ctx->st);
    });
}

kpm_status kpm_pauli_terms(kpm_ctx* ctx, int64_t* nterms, int* ngroups) {
    if (!ctx) { g_err = "NULL context"; return KPM_EINVAL; }
    return guarded(ctx, [&] {
        DeviceGuard g(ctx->device);
        PauliH& ph = pauli_of(ctx);
        if (nterms) *nterms = ph.nterms;
        if (ngroups) *ngroups = ph.ngroups;
    });
}

kpm_status kpm_apply_dipole(kpm_ctx* ctx, int comp, const double* psi, void* y) {
    if (!ctx) { g_err = "NULL context"; return KPM_EINVAL; }
    return guarded(ctx, [&] {
        if (comp < 0 || comp > 2 || !psi || !y) KPM_THROW(KPM_EINVAL, "bad dipole arguments");
        DeviceGuard g(ctx->device);
        dipole_dispatch(ctx, comp, psi, y);
    });
}

void kpm_scale(double emin, double emax, double eps, double* a, double* b) {
    if (a) *a = (emax - emin) / (2.0 - eps);
    if (b) *b = 0.5 * (emax + emin);
}

kpm_status kpm_bounds(kpm_ctx* ctx, int iters, uint64_t seed, double* emin, double* emax) {
    if (!ctx) { g_err = "NULL context"; return KPM_EINVAL; }
    return guarded(ctx, [&] {
        if (iters < 1 || iters > 4096 || !emin || !emax) KPM_THROW(KPM_EINVAL, "bad bounds arguments");
        DeviceGuard g(ctx->device);
        int k = (int)std::min<int64_t>(iters, ctx->dim);
        bool f64 = ctx->prec == KPM_FP64;
        size_t vb = (size_t)ctx->dim * ctx->esz();
        ctx->lz_v0.ensure(vb);
        ctx->lz_v1.ensure(vb);
        ctx->lz_w.ensure(vb);
        ctx->lz_ab.ensure(sizeof(double) * (5 * (k + 1)));
        ctx->lz_scalar.ensure(sizeof(double) * 8);
        ensure_reduce_scratch(ctx, 1);
        double* al = ctx->lz_ab.as<double>();
        double* be = al + (k + 1);
        double* sc = ctx->lz_scalar.as<double>();
        double* parts = ctx->partials.as<double>();
        unsigned* cnt = ctx->counters.as<unsigned>();
        void* v = ctx->lz_v0.p;
        void* vp = ctx->lz_v1.p;
        void* w = ctx->lz_w.p;
        fill_random(v, ctx->dim, f64, seed, ctx->st);
        dot_dev(v, v, ctx->dim, f64, parts, cnt, sc, ctx->st);
        scale_inplace(v, ctx->dim, f64, sc, ctx->st);
        for (int j = 0; j < k; ++j) {
            sigma_dispatch(ctx, v, w, 1);
            dot_dev(w, v, ctx->dim, f64, parts, cnt, al + j, ctx->st);
            lanczos_orth(w, v, j ? vp : nullptr, ctx->dim, f64, al + j, j ? be + j - 1 : nullptr,
                         parts, cnt, sc, ctx->st);
            lanczos_scale(vp, w, ctx->dim, f64, sc, be + j, ctx->st);
            std::swap(v, vp);  // v <- v_{j+1}, vp <- v_j
        }
        tridiag_extremes(al, be, k, sc + 2, be + (k + 1), ctx->st);
        double out4[4];
        KPM_CUDA(cudaMemcpyAsync(out4, sc + 2, sizeof(out4), cudaMemcpyDeviceToHost, ctx->st));
        KPM_CUDA(cudaStreamSynchronize(ctx->st));
        check_device_errors(ctx);
        *emin = out4[0] - out4[2];
        *emax = out4[1] + out4[3];
    });
}

kpm_status kpm_ground_state(kpm_ctx* ctx, int iters, int max_cycles, double tol, uint64_t seed,
                            double* psi_dev, double* e0, double* resid) {
    if (!ctx) { g_err = "NULL context"; return KPM_EINVAL; }
    return guarded(ctx, [&] {
        if (iters < 2 || iters > 4096 || max_cycles < 1 || max_cycles > 10000 || !psi_dev ||
            !(tol > 0.0) || !e0 || !resid)
            KPM_THROW(KPM_EINVAL, "bad ground-state arguments");
        DeviceGuard g(ctx->device);
        const int64_t dim = ctx->dim;
        const int k = (int)std::min<int64_t>(iters, dim);
        const bool f64 = ctx->prec == KPM_FP64;
        const size_t vb = (size_t)dim * ctx->esz();
        ctx->lz_v0.ensure(vb);
        ctx->lz_v1.ensure(vb);
        ctx->lz_w.ensure(vb);
        ctx->lz_start.ensure(vb);
        ctx->lz_ab.ensure(sizeof(double) * (6 * (k + 1)));
        ctx->lz_scalar.ensure(sizeof(double) * 8);
        ensure_reduce_scratch(ctx, 1);
        double* al = ctx->lz_ab.as<double>();
        double* be = al + (k + 1);
        double* sv = be + (k + 1);          // eigenvector of T
        double* scr = sv + (k + 1);         // 2k scratch
        double* sc = ctx->lz_scalar.as<double>();
        double* parts = ctx->partials.as<double>();
        unsigned* cnt = ctx->counters.as<unsigned>();
        void* start = ctx->lz_start.p;
        fill_random(start, dim, f64, seed, ctx->st);
        dot_dev(start, start, dim, f64, parts, cnt, sc, ctx->st);
        scale_inplace(start, dim, f64, sc, ctx->st);
        // one pass of k Lanczos steps from `start`; with `acc`, psi += s_j v_j as
        // v_j is regenerated (the kernels are deterministic, so pass 2 repeats
        // pass 1's vectors bit for bit)
        auto pass = [&](bool acc) {
            void* v = ctx->lz_v0.p;
            void* vp = ctx->lz_v1.p;
            void* w = ctx->lz_w.p;
            KPM_CUDA(cudaMemcpyAsync(v, start, vb, cudaMemcpyDeviceToDevice, ctx->st));
            for (int j = 0; j < k; ++j) {
                if (acc) axpy_dev(psi_dev, v, dim, f64, sv + j, ctx->st);
                if (acc && j == k - 1) break;
                sigma_dispatch(ctx, v, w, 1);
                dot_dev(w, v, dim, f64, parts, cnt, al + j, ctx->st);
                lanczos_orth(w, v, j ? vp : nullptr, dim, f64, al + j, j ? be + j - 1 : nullptr,
                             parts, cnt, sc, ctx->st);
                lanczos_scale(vp, w, dim, f64, sc, be + j, ctx->st);
                std::swap(v, vp);
            }
        };
        double e = 0.0, r = INFINITY;
        for (int cyc = 0; cyc < max_cycles; ++cyc) {
            pass(false);
            tridiag_lowest(al, be, k, sc + 4, sv, scr, ctx->st);
            KPM_CUDA(cudaMemsetAsync(psi_dev, 0, (size_t)dim * 8, ctx->st));
            pass(true);
            // psi /= |psi|; residual |H psi - E psi| with E = <psi|H|psi>, in the
            // context precision (psi rounded to it for the product)
            dot_dev(psi_dev, psi_dev, dim, true, parts, cnt, sc, ctx->st);
            scale_inplace(psi_dev, dim, true, sc, ctx->st);
            void* v = ctx->lz_v0.p;
            void* w = ctx->lz_w.p;
            if (f64) KPM_CUDA(cudaMemcpyAsync(v, psi_dev, vb, cudaMemcpyDeviceToDevice, ctx->st));
            else to_f32(psi_dev, (float*)v, dim, ctx->st);
            sigma_dispatch(ctx, v, w, 1);
            dot_dev(w, v, dim, f64, parts, cnt, sc + 1, ctx->st);
            dot_dev(v, v, dim, f64, parts, cnt, sc + 2, ctx->st);
            lanczos_orth(w, v, nullptr, dim, f64, sc + 1, nullptr, parts, cnt, sc + 3, ctx->st);
            double h[4];
            KPM_CUDA(cudaMemcpyAsync(h, sc, sizeof(h), cudaMemcpyDeviceToHost, ctx->st));
            KPM_CUDA(cudaStreamSynchronize(ctx->st));
            check_device_errors(ctx);
            // v is psi rounded to the context precision: |v| = 1 up to that rounding
            e = h[1] / h[2];
            r = std::sqrt(std::fmax(h[3], 0.0));
            if (r <= tol) break;
            // restart from psi
            KPM_CUDA(cudaMemcpyAsync(start, v, vb, cudaMemcpyDeviceToDevice, ctx->st));
            dot_dev(start, start, dim, f64, parts, cnt, sc, ctx->st);
            scale_inplace(start, dim, f64, sc, ctx->st);
        }
        *e0 = e;
        *resid = r;
    });
}

kpm_status kpm_recursion_begin(kpm_ctx* ctx, const double* psi0_dev, unsigned comp_mask, double a,
                               double b, int max_moments) {
    if (!ctx) { g_err = "NULL context"; return KPM_EINVAL; }
    return guarded(ctx, [&] {
        DeviceGuard g(ctx->device);
        rec_begin(ctx, psi0_dev, comp_mask, a, b, max_moments);
    });
}

kpm_status kpm_recursion_begin_deflated(kpm_ctx* ctx, const double* psi0_dev, double e0,
                                        unsigned comp_mask, double a, double b, int max_moments) {
    if (!ctx) { g_err = "NULL context"; return KPM_EINVAL; }
    return guarded(ctx, [&] {
        DeviceGuard g(ctx->device);
        rec_begin_deflated(ctx, psi0_dev, e0, comp_mask, a, b, max_moments);
    });
}

kpm_status kpm_moments_deflated(kpm_ctx* ctx, const double* psi0_dev, double e0,
                                unsigned comp_mask, double a, double b, int nmoments,
                                double* moments_host) {
    if (!ctx) { g_err = "NULL context"; return KPM_EINVAL; }
    kpm_status r = KPM_OK;
    kpm_status s = guarded(ctx, [&] {
        if (!moments_host) KPM_THROW(KPM_EINVAL, "NULL output");
        DeviceGuard g(ctx->device);
        rec_begin_deflated(ctx, psi0_dev, e0, comp_mask, a, b, nmoments);
        rec_advance(ctx, nmoments / 2 - 1);
        r = rec_collect(ctx, moments_host, nmoments);
    });
    return s != KPM_OK ? s : r;
}

kpm_status kpm_moments_cross(kpm_ctx* ctx, const double* psi0, const double* op_a,
                             const double* op_b, double a, double b, int nmoments,
                             double* moments_host) {
    if (!ctx) { g_err = "NULL context"; return KPM_EINVAL; }
    kpm_status r = KPM_OK;
    kpm_status s = guarded(ctx, [&] {
        if (!psi0 || !op_a || !op_b || !moments_host) KPM_THROW(KPM_EINVAL, "NULL argument");
        if (nmoments < 2 || (nmoments & 1)) KPM_THROW(KPM_EINVAL, "nmoments must be even and >= 2");
        if (!(a > 0.0) || !std::isfinite(a) || !std::isfinite(b))
            KPM_THROW(KPM_EINVAL, "need a > 0 and finite a, b");
        const int n = ctx->n;
        check_sym(op_a, n, "op_a");
        check_sym(op_b, n, "op_b");
        DeviceGuard g(ctx->device);
        kpm_ctx* c = ctx;
        const int64_t dim = c->dim;
        const bool f64 = c->prec == KPM_FP64;
        // the dipole kernels apply -sum d_pq E_pq: upload -op
        std::vector<double> neg((size_t)2 * n * n);
        for (int i = 0; i < n * n; ++i) {
            neg[i] = -op_a[i];
            neg[(size_t)n * n + i] = -op_b[i];
        }
        c->x_ops.ensure(neg.size() * sizeof(double));
        KPM_CUDA(cudaMemcpyAsync(c->x_ops.p, neg.data(), neg.size() * sizeof(double),
                                 cudaMemcpyHostToDevice, c->st));
        const int nsteps = nmoments / 2;
        c->rec_ncol = 2;
        c->rec_max_steps = nsteps;
        c->rec_a = a;
        c->rec_b = b;
        c->rec_deflated = false;
        const size_t vb = (size_t)2 * dim * c->esz();
        c->vA.ensure(vb);
        c->vB.ensure(vb);
        c->vS.ensure(vb);
        c->dots.ensure((size_t)2 * nsteps * 2 * sizeof(double));
        c->moments_dev.ensure((size_t)nmoments * sizeof(double));
        c->x_cross.ensure((size_t)nmoments * sizeof(double));
        ensure_reduce_scratch(c, 2);
        c->drop_graphs();
        double* xc = c->x_cross.as<double>();
        double* parts = c->partials.as<double>();
        unsigned* cnt = c->counters.as<unsigned>() + 2;    // counters 0, 1: the update's columns
        for (int j = 0; j < 2; ++j) {
            const double* d = c->x_ops.as<double>() + (size_t)j * n * n;
            void* y = (char*)c->vB.p + (size_t)j * dim * c->esz();
            if (f64) dipole_apply_f64(c->ta, *c->tb, d, psi0, (double*)y, c->st);
            else dipole_apply_f32(c->ta, *c->tb, d, psi0, (float*)y, c->st);
        }
        void* prev = c->vB.p;   // (a_0, b_0)
        void* cur = c->vA.p;    // (a_1, b_1) after the first update
        sigma_dispatch(c, prev, c->vS.p, 2);
        update_dispatch(c, c->vS.p, prev, cur, 1, c->dots.as<double>(), nullptr);
        cross_dots(prev, cur, dim, f64, parts, cnt, xc, c->st);
        // prev = step k - 1, cur = step k
        for (int k = 1; k < nsteps; ++k) {
            sigma_dispatch(c, cur, c->vS.p, 2);
            // update writes step n + 1 over step n - 1; its own dots (at index k) are unused
            update_dispatch(c, c->vS.p, cur, prev, 0, c->dots.as<double>() + 2 * k, nullptr);
            cross_dots(cur, prev, dim, f64, parts, cnt, xc + 2 * k, c->st);
            std::swap(prev, cur);
        }
        cross_doubling(xc, nsteps, c->moments_dev.as<double>(), c->st);
        double self[2];
        KPM_CUDA(cudaMemcpyAsync(moments_host, c->moments_dev.p, sizeof(double) * nmoments,
                                 cudaMemcpyDeviceToHost, c->st));
        KPM_CUDA(cudaMemcpyAsync(&self[0], c->dots.as<double>(), sizeof(double),
                                 cudaMemcpyDeviceToHost, c->st));
        KPM_CUDA(cudaMemcpyAsync(&self[1], c->dots.as<double>() + (size_t)2 * nsteps,
                                 sizeof(double), cudaMemcpyDeviceToHost, c->st));
        KPM_CUDA(cudaStreamSynchronize(c->st));
        check_device_errors(c);
        c->rec_steps = 0;     // the context holds no resumable recursion now
        const double lim = std::sqrt(std::fabs(self[0] * self[1])) * (1.0 + 1e-6);
        for (int i = 0; i < nmoments; ++i)
            if (!std::isfinite(moments_host[i]) || std::fabs(moments_host[i]) > lim) {
                c->err = "|Omega_n| exceeds the Cauchy-Schwarz bound: [b-a, b+a] misses the spectrum";
                r = KPM_EBOUNDS;
                break;
            }
    });
    return s != KPM_OK ? s : r;
}

kpm_status kpm_recursion_advance(kpm_ctx* ctx, int nsteps) {
    if (!ctx) { g_err = "NULL context"; return KPM_EINVAL; }
    return guarded(ctx, [&] {
        DeviceGuard g(ctx->device);
        rec_advance(ctx, nsteps);
    });
}

kpm_status kpm_recursion_moments(kpm_ctx* ctx, double* out, int* nm_out) {
    if (!ctx) { g_err = "NULL context"; return KPM_EINVAL; }
    kpm_status r = KPM_OK;
    kpm_status s = guarded(ctx, [&] {
        if (!out) KPM_THROW(KPM_EINVAL, "NULL output");
        if (ctx->rec_steps <= 0) KPM_THROW(KPM_EINVAL, "no recursion in progress");
        DeviceGuard g(ctx->device);
        r = rec_collect(ctx, out, 2 * ctx->rec_steps);
        if (nm_out) *nm_out = 2 * ctx->rec_steps;
    });
    return s != KPM_OK ? s : r;
}

kpm_status kpm_moments(kpm_ctx* ctx, const double* psi0_dev, unsigned comp_mask, double a,
                       double b, int nmoments, double* moments_host) {
    if (!ctx) { g_err = "NULL context"; return KPM_EINVAL; }
    kpm_status r = KPM_OK;
    kpm_status s = guarded(ctx, [&] {
        if (!moments_host) KPM_THROW(KPM_EINVAL, "NULL output");
        DeviceGuard g(ctx->device);
        rec_begin(ctx, psi0_dev, comp_mask, a, b, nmoments);
        rec_advance(ctx, nmoments / 2 - 1);
        r = rec_collect(ctx, moments_host, nmoments);
    });
    return s != KPM_OK ? s : r;
}

kpm_status kpm_moments_batch(kpm_ctx* const* ctxs, int count, const double* const* psi0_dev,
                             unsigned comp_mask, const double* a, const double* b, int nmoments,
                             double* moments_host) {
    if (!ctxs || count < 1 || !ctxs[0]) {
        g_err = "NULL or empty context list";
        return KPM_EINVAL;
    }
    kpm_ctx* c0 = ctxs[0];
    kpm_status r = KPM_OK;
    kpm_status s = guarded(c0, [&] {
        if (!psi0_dev || !a || !b || !moments_host) KPM_THROW(KPM_EINVAL, "NULL argument");
        check_batch(ctxs, count);
        DeviceGuard g(c0->device);
        for (int i = 0; i < count; ++i)
            rec_begin(ctxs[i], psi0_dev[i], comp_mask, a[i], b[i], nmoments);
        batch_steps(ctxs, count, nmoments / 2 - 1);
        const int ncomp = __builtin_popcount(comp_mask);
        for (int i = 0; i < count; ++i) {
            kpm_status ri = rec_collect(ctxs[i], moments_host + (size_t)i * ncomp * nmoments,
                                        nmoments);
            if (r == KPM_OK) r = ri;
        }
    });
    return s != KPM_OK ? s : r;
}

kpm_status kpm_recursion_advance_batch(kpm_ctx* const* ctxs, int count, int nsteps) {
    if (!ctxs || count < 1 || !ctxs[0]) {
        g_err = "NULL or empty context list";
        return KPM_EINVAL;
    }
    return guarded(ctxs[0], [&] {
        check_batch(ctxs, count);
        for (int i = 0; i < count; ++i) {
            const kpm_ctx* c = ctxs[i];
            if (c->rec_steps <= 0) KPM_THROW(KPM_EINVAL, "context %d: no recursion in progress", i);
            if (nsteps < 0 || c->rec_steps + nsteps > c->rec_max_steps)
                KPM_THROW(KPM_EINVAL, "context %d: advance past the requested number of moments", i);
        }
        DeviceGuard g(ctxs[0]->device);
        batch_steps(ctxs, count, nsteps);
    });
}

kpm_status kpm_moments_host(kpm_ctx* ctx, const double* psi0_host, unsigned comp_mask, double a,
                            double b, int nmoments, double* moments_host) {
    if (!ctx) { g_err = "NULL context"; return KPM_EINVAL; }
    kpm_status s = guarded(ctx, [&] {
        if (!psi0_host) KPM_THROW(KPM_EINVAL, "NULL psi0");
        DeviceGuard g(ctx->device);
        ctx->psi_tmp.ensure((size_t)ctx->dim * 8);
        KPM_CUDA(cudaMemcpyAsync(ctx->psi_tmp.p, psi0_host, (size_t)ctx->dim * 8,
                                 cudaMemcpyHostToDevice, ctx->st));
    });
    if (s != KPM_OK) return s;
    return kpm_moments(ctx, ctx->psi_tmp.as<double>(), comp_mask, a, b, nmoments, moments_host);
}

kpm_status kpm_spectrum(const double* moments, int nmoments, double a, double b, int npoints,
                        int kernel, double* omega_out, double* intensity_out) {
    return guarded(nullptr, [&] {
        if (!moments || !omega_out || !intensity_out) KPM_THROW(KPM_EINVAL, "NULL argument");
        if (nmoments < 1 || npoints < 1 || kernel < 0 || kernel > 2)
            KPM_THROW(KPM_EINVAL, "bad spectrum arguments");
        if (!(a > 0.0)) KPM_THROW(KPM_EINVAL, "a must be > 0");
        require_device();
        DevBuf dm, dd, dom, din;
        dm.alloc(sizeof(double) * nmoments);
        dd.alloc(sizeof(double) * nmoments);
        dom.alloc(sizeof(double) * npoints);
        din.alloc(sizeof(double) * npoints);
        KPM_CUDA(cudaMemcpy(dm.p, moments, sizeof(double) * nmoments, cudaMemcpyHostToDevice));
        spectrum_dev(dm.as<double>(), nmoments, a, b, npoints, kernel, dd.as<double>(),
                     dom.as<double>(), din.as<double>(), nullptr);
        KPM_CUDA(cudaMemcpy(omega_out, dom.p, sizeof(double) * npoints, cudaMemcpyDeviceToHost));
        KPM_CUDA(cudaMemcpy(intensity_out, din.p, sizeof(double) * npoints, cudaMemcpyDeviceToHost));
    });
}

kpm_status kpm_spectrum_lorentz(const double* moments, int nmoments, double a, double b,
                                int npoints, double lambda, double* omega_out,
                                double* intensity_out) {
    return guarded(nullptr, [&] {
        if (!moments || !omega_out || !intensity_out) KPM_THROW(KPM_EINVAL, "NULL argument");
        if (nmoments < 1 || npoints < 1 || !(lambda > 0.0) || !std::isfinite(lambda))
            KPM_THROW(KPM_EINVAL, "bad spectrum arguments");
        if (!(a > 0.0)) KPM_THROW(KPM_EINVAL, "a must be > 0");
        require_device();
        DevBuf dm, dd, dom, din;
        dm.alloc(sizeof(double) * nmoments);
        dd.alloc(sizeof(double) * nmoments);
        dom.alloc(sizeof(double) * npoints);
        din.alloc(sizeof(double) * npoints);
        KPM_CUDA(cudaMemcpy(dm.p, moments, sizeof(double) * nmoments, cudaMemcpyHostToDevice));
        spectrum_dev(dm.as<double>(), nmoments, a, b, npoints, 2, dd.as<double>(),
                     dom.as<double>(), din.as<double>(), nullptr, lambda);
        KPM_CUDA(cudaMemcpy(omega_out, dom.p, sizeof(double) * npoints, cudaMemcpyDeviceToHost));
        KPM_CUDA(cudaMemcpy(intensity_out, din.p, sizeof(double) * npoints, cudaMemcpyDeviceToHost));
    });
}

kpm_status kpm_synchronize(kpm_ctx* ctx) {
    if (!ctx) { g_err = "NULL context"; return KPM_EINVAL; }
    return guarded(ctx, [&] {
        DeviceGuard g(ctx->device);
        KPM_CUDA(cudaStreamSynchronize(ctx->st));
        KPM_CUDA(cudaGetLastError());
        check_device_errors(ctx);
    });
}

kpm_status kpm_profile_enable(kpm_ctx* ctx, int enable) {
    if (!ctx) { g_err = "NULL context"; return KPM_EINVAL; }
    ctx->prof = enable != 0;
    if (ctx->tc) ctx->tc->prof = ctx->prof;
    return KPM_OK;
}

kpm_status kpm_profile_read_rowpass(kpm_ctx* ctx, double* ms, int* count) {
    if (!ctx) { g_err = "NULL context"; return KPM_EINVAL; }
    return guarded(ctx, [&] {
        DeviceGuard g(ctx->device);
        double t = 0.0;
        int n = 0;
        if (ctx->tc) t = ctx->tc->read_prof(ctx->st, &n);
        if (ms) *ms = t;
        if (count) *count = n;
    });
}

kpm_status kpm_test_rowpass_stall(kpm_ctx* ctx, int enable) {
    if (!ctx) { g_err = "NULL context"; return KPM_EINVAL; }
    if (!ctx->tc) {
        ctx->err = "not a tensor-core (KPM_MIXED / KPM_MIXED_BF16) context";
        return KPM_EINVAL;
    }
    ctx->tc->stall_next = enable != 0;
    return KPM_OK;
}

kpm_status kpm_tuned_params(const kpm_ctx* ctx, int* group_beta, int* group_alpha) {
    if (!ctx) { g_err = "NULL context"; return KPM_EINVAL; }
    if (group_beta) *group_beta = ctx->tc ? ctx->tc->dense.group_m[0] : 0;
    if (group_alpha) *group_alpha = ctx->tc ? ctx->tc->dense.group_m[1] : 0;
    return KPM_OK;
}

kpm_status kpm_tuned_rowpass(const kpm_ctx* ctx, int* stages, int* prefetch) {
    if (!ctx) { g_err = "NULL context"; return KPM_EINVAL; }
    if (stages) *stages = ctx->tc ? ctx->tc->nst : 0;
    if (prefetch) *prefetch = ctx->tc ? ctx->tc->rp_prefetch : 0;
    return KPM_OK;
}

kpm_status kpm_set_rowpass(kpm_ctx* ctx, int stages, int prefetch) {
    if (!ctx) { g_err = "NULL context"; return KPM_EINVAL; }
    if (!ctx->tc) {
        ctx->err = "not a tensor-core (KPM_MIXED / KPM_MIXED_BF16) context";
        return KPM_EINVAL;
    }
    const size_t need = kpm::rowpass_smem_bytes(*ctx->tc, stages);
    if (stages < 2 || stages > 3 || prefetch < 0 || prefetch > 64 || need > ctx->tc->smem_bytes) {
        ctx->err = "row pass: stages must be 2 or 3 (within the shared memory sized at "
                   "creation) and prefetch 0..64 tiles";
        return KPM_EINVAL;
    }
    ctx->tc->nst = stages;
    ctx->tc->rp_prefetch = prefetch;
    return KPM_OK;
}

kpm_status kpm_set_rowpass_passes(kpm_ctx* ctx, int passes) {
    if (!ctx) { g_err = "NULL context"; return KPM_EINVAL; }
    if (!ctx->tc || passes < 0 || passes > 64) {
        ctx->err = "row pass: a tensor-core context and 0..64 passes";
        return KPM_EINVAL;
    }
    return guarded(ctx, [&] {
        DeviceGuard g(ctx->device);
        ctx->tc->set_layout(passes, ctx->st);
        KPM_CUDA(cudaStreamSynchronize(ctx->st));
    });
}

kpm_status kpm_rowpass_layout(const kpm_ctx* ctx, int* wide, int* passes) {
    if (!ctx) { g_err = "NULL context"; return KPM_EINVAL; }
    if (wide) *wide = ctx->tc ? (ctx->tc->wide ? 1 : 0) : 0;
    if (passes) *passes = ctx->tc ? ctx->tc->npass : 0;
    return KPM_OK;
}

kpm_status kpm_graphs_enable(kpm_ctx* ctx, int enable) {
    if (!ctx) { g_err = "NULL context"; return KPM_EINVAL; }
    ctx->graphs = enable != 0;
    if (!ctx->graphs) ctx->drop_graphs();
    return KPM_OK;
}

kpm_status kpm_profile_read(kpm_ctx* ctx, double* ms, int* count) {
    if (!ctx) { g_err = "NULL context"; return KPM_EINVAL; }
    return guarded(ctx, [&] {
        DeviceGuard g(ctx->device);
        KPM_CUDA(cudaStreamSynchronize(ctx->st));
        double tot = 0.0;
        for (int i = 0; i + 1 < ctx->ev_used; i += 2) {
            float t = 0.f;
            KPM_CUDA(cudaEventElapsedTime(&t, ctx->ev[i], ctx->ev[i + 1]));
            tot += t;
        }
        if (ms) *ms = tot;
        if (count) *count = ctx->ev_used / 2;
        ctx->ev_used = 0;
    });
}

uint64_t kpm_launch_count(void) { return g_launches.load(); }

}  // extern "C"
