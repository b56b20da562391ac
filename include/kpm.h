/*
 * kpm.h -- C-ABI of the GB300 (sm_103a) kernel-polynomial-method library.
 *
 * The library computes the dipole absorption spectrum of a molecule from its
 * ground state with the kernel polynomial method of arXiv 2506.07430:
 *
 *   I(w) = sum_n |<n|mu|0>|^2 delta(w_n - w)                        (Eq. 1)
 *   Omega_n = <0| mu T_n(H~) mu |0>,  H~ = (H - b)/a                (Eq. moments)
 *   alpha_0 = mu|0>, alpha_1 = H~ alpha_0,
 *   alpha_{n+1} = 2 H~ alpha_n - alpha_{n-1}          (Methods, KPM recursion)
 *   Omega_2n = 2<alpha_n|alpha_n> - Omega_0,
 *   Omega_2n+1 = 2<alpha_n+1|alpha_n> - Omega_1       (Methods, doubling)
 *   I(x) = (g_0 Omega_0 + 2 sum_n g_n Omega_n T_n(x)) / (pi sqrt(1-x^2))
 *                                          (Eq. kpm with the Jackson kernel g_n)
 *
 * H is the second-quantized electronic Hamiltonian of the paper's Methods
 * ("Mapping fermionic Hamiltonians to the qubits") with one-body integrals h_pq
 * and two-body integrals, here in chemist order (pq|rs):
 *   H = sum_pq h_pq E_pq + 1/2 sum_pqrs (pq|rs) (E_pq E_rs - delta_qr E_ps),
 * E_pq = sum_sigma a+_{p sigma} a_{q sigma}; mu = -sum_pq d_pq E_pq (the paper's
 * dipole operator without frozen core).  H acts matrix-free on the full
 * configuration-interaction space of a fixed (N_alpha, N_beta) sector.
 *
 * Vector layout (every device vector): determinant (I_alpha, I_beta) is element
 * I_alpha * N_beta + I_beta (int64), where I is the rank of an occupation string
 * (an n-bit mask with bit p = orbital p occupied) in ascending integer order.
 * Block vectors hold ncol columns one after the other: [ncol][dim].
 * The state of a determinant is (alpha creators ascending)(beta creators
 * ascending)|vac>.
 *
 * Conventions for every call:
 *  - Host arrays are read during the call and copied; the caller keeps them.
 *  - Device pointers are owned by the caller, must stay valid until the work
 *    queued on the context's stream has finished, and must not alias each other
 *    unless stated.  Device vectors are double* for KPM_FP64 contexts and float*
 *    otherwise ("void*" below).
 *  - Calls on one context are not thread-safe; distinct contexts are independent.
 *  - Errors are returned as kpm_status; no C++ exception crosses the boundary.
 *    kpm_last_error(ctx) returns the message of the last failing call on ctx
 *    (kpm_last_error(NULL): last failure of a call without a context, or of
 *    kpm_create, on this thread).
 *  - All arithmetic of the path runs in CUDA kernels of this library; there is
 *    no CPU fallback.  A missing or unusable GPU is reported as KPM_ECUDA.
 */
#ifndef KPM_H
#define KPM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct kpm_ctx kpm_ctx;

typedef enum {
    KPM_OK = 0,
    KPM_EINVAL = 1,      /* invalid argument (size, symmetry, range, null pointer) */
    KPM_ENOMEM = 2,      /* device or host allocation failed */
    KPM_ECUDA = 3,       /* CUDA runtime or launch error */
    KPM_EBOUNDS = 4,     /* |Omega_n| > Omega_0 (1 + 1e-6): [b-a, b+a] misses the spectrum */
    KPM_ETIMEOUT = 5,    /* a bounded wait ran out */
    KPM_ECANCELLED = 6,  /* request cancelled */
    KPM_EUNSUPPORTED = 7 /* valid request outside this build's limits */
} kpm_status;

typedef enum {
    KPM_FP64 = 0,      /* FP64 vectors and arithmetic everywhere (reference path)     */
    KPM_FP32 = 1,      /* FP32 vectors, FP32 CUDA-core sigma with the diagonal H_II
                          evaluated in FP64; FP64 dots/moments                        */
    KPM_MIXED = 2,     /* FP32 vectors; the opposite-spin two-electron term and the
                          same-spin string Hamiltonians on tensor cores (tcgen05):
                          x and the integrals each split into 2 FP16 pieces with
                          power-of-two scales, 3 MMAs per product (hi*hi, lo*hi,
                          hi*lo), FP32 accumulation; same-spin diagonals added
                          exactly; FP64 dots/moments; up to 18 orbitals               */
    KPM_MIXED_BF16 = 3 /* as KPM_MIXED with split-BF16 operands (2 pieces each,
                          3 MMAs): ~16 significant bits per product                  */
} kpm_precision;

/* Parameter lambda of the Lorentz kernel (kernel = 2) of kpm_spectrum. */
#define KPM_LORENTZ_LAMBDA 4.0

/* Largest orbital count this build supports (strings are 32-bit masks, string
 * ranks are 16-bit in packed tables: C(18,9) = 48620 < 65536). */
#define KPM_MAX_ORB 18

/*
 * kpm_create -- build a context for one molecule.
 *   h1     [norb*norb]       host, row-major one-body integrals h_pq, symmetric.
 *   eri    [norb^4]          host, chemist (pq|rs) at ((p*n+q)*n+r)*n+s,
 *                            8-fold symmetric.
 *   dipole [3*norb*norb]     host, d^x, d^y, d^z (Methods, d_pq = <p|r|q>),
 *                            each symmetric.
 *   norb   1..KPM_MAX_ORB; 0 <= nalpha, nbeta <= norb.
 *   prec   kpm_precision of every vector this context reads or writes.
 *   cuda_stream  cudaStream_t (NULL = legacy default stream) all work is queued on.
 * Builds the string tables on the device (kernels), uploads the integrals, and
 * allocates the context's own workspaces.  Symmetry is checked to 1e-12
 * (relative to max |entry|) -> KPM_EINVAL.  On success *out owns everything it
 * allocated; release with kpm_destroy.
 * Paper: Methods, "Mapping fermionic Hamiltonians to the qubits" (H) and
 * "KPM for absorption spectra" (mu, d_pq).
 */
kpm_status kpm_create(const double* h1, const double* eri, const double* dipole,
                      int norb, int nalpha, int nbeta, kpm_precision prec,
                      void* cuda_stream, kpm_ctx** out);

/* Releases everything the context allocated (synchronises its stream first). */
void kpm_destroy(kpm_ctx* ctx);

/* Message of the last failing call (see conventions).  Never NULL. */
const char* kpm_last_error(const kpm_ctx* ctx);

/* FCI dimension N_alpha_strings * N_beta_strings; -1 for a NULL context. */
int64_t kpm_dim(const kpm_ctx* ctx);

/* Number of strings, and of single-excitation table entries per string
 * (m (n - m + 1)), of spin 0 (alpha) or 1 (beta); -1 on bad arguments. */
int64_t kpm_nstrings(const kpm_ctx* ctx, int spin);
int kpm_nexc(const kpm_ctx* ctx, int spin);

/*
 * kpm_string_table -- host copies of the device-built tables of one spin.
 *   masks [N_s]          occupation masks in rank order.
 *   tgt   [N_s][n_exc]   rank of the target string J of a+_p a_q |I> = sgn |J>.
 *   pq    [N_s][n_exc]   p * norb + q.
 *   sgn   [N_s][n_exc]   +1 / -1.
 * Entry order per string I: q over occupied orbitals ascending, then p over
 * {q} union (vacant orbitals) ascending.  Any output pointer may be NULL.
 * Synchronises the context's stream.
 */
kpm_status kpm_string_table(const kpm_ctx* ctx, int spin, uint32_t* masks, int32_t* tgt,
                            uint16_t* pq, int8_t* sgn);

/*
 * kpm_sigma -- y = H x for ncol columns (device, [ncol][dim], x and y distinct).
 * Queued on the context's stream (asynchronous).  FP64: plain gathers in FP64;
 * FP32: FP32 gathers with the diagonal H_II evaluated in FP64; KPM_MIXED /
 * KPM_MIXED_BF16: the opposite-spin term and the same-spin products on tensor
 * cores (split FP16 / BF16 operands, FP32 accumulation), the same-spin
 * diagonals added exactly.
 * Paper: Methods, second-quantized Hamiltonian.
 */
kpm_status kpm_sigma(kpm_ctx* ctx, const void* x, void* y, int ncol);

/*
 * kpm_sigma_pauli -- y = H x with H in the Jordan-Wigner Pauli-string form the
 * paper maps the second-quantized Hamiltonian to (Methods, "Mapping fermionic
 * Hamiltonians to the qubits"): qubits are the spin orbitals in this library's
 * determinant order (alpha 0..n-1, beta n..2n-1), a+_q = (X_q - i Y_q)/2 Z_{<q},
 * and H becomes a real sum of strings c X^x Z^z (built on the host at the first
 * call from the context's integrals; equal strings merged).  The kernel pulls
 * every output determinant's terms over the strings' flip masks (FP64 sums; x and
 * y in the context's vector type; FP64 or FP32 contexts, and tensor-core contexts
 * with FP32 vectors).  It is the same H as kpm_sigma, for comparison with the
 * paper's representation; its cost grows with the number of strings (O(n^4)), so
 * it is meant for small systems.  Asynchronous after the first call.
 * Errors: KPM_EINVAL (NULL, ncol outside 1..64, x == y).
 */
kpm_status kpm_sigma_pauli(kpm_ctx* ctx, const void* x, void* y, int ncol);

/* Number of Pauli strings of kpm_sigma_pauli's H and of their distinct flip
 * masks (builds the form if needed; synchronous). */
kpm_status kpm_pauli_terms(kpm_ctx* ctx, int64_t* nterms, int* ngroups);

/*
 * kpm_apply_dipole -- y = mu^comp psi (comp 0,1,2 = x,y,z); psi FP64 device
 * [dim], y device [dim] in the context precision.  Asynchronous.
 * Paper: Methods, dipole operator mu = -sum_pq d_pq (c+_up c_up + c+_dn c_dn).
 */
kpm_status kpm_apply_dipole(kpm_ctx* ctx, int comp, const double* psi_dev, void* y);

/*
 * kpm_bounds -- spectral bounds of H by `iters` Lanczos steps (FP64 dots and
 * tridiagonal, vectors in the context precision) from a start vector drawn with
 * the SplitMix64 counter generator seeded by `seed`.  The extreme Ritz values
 * are widened by their residual estimates |beta_k s_k|.  Synchronous.
 * The paper rescales the spectrum into [-1, 1] (Results, "Resolution of
 * absorption spectra"); pass these bounds to kpm_scale to get a, b.
 */
kpm_status kpm_bounds(kpm_ctx* ctx, int iters, uint64_t seed, double* emin, double* emax);

/*
 * kpm_ground_state -- the lowest eigenpair of H, the |0> that the dipole
 * recursion starts from (the paper obtains |0> from its NQS; here it is found
 * on the GPU with the library's own sigma).  Explicitly restarted Lanczos: each
 * cycle runs `iters` Lanczos steps (FP64 dots and tridiagonal, vectors in the
 * context precision) from the current start vector, takes the lowest Ritz pair
 * of the tridiagonal (Sturm bisection and inverse iteration on the device),
 * regenerates the same Lanczos vectors in a second pass to form the Ritz
 * vector psi = sum_j s_j v_j in FP64, normalises it, and restarts from it,
 * until |H psi - E psi| <= tol or max_cycles cycles have run.  The first start
 * vector is drawn with the SplitMix64 counter generator seeded by `seed`.
 *   psi_dev  FP64 device [dim] (caller-owned), out: the unit Ritz vector
 *            (overall sign arbitrary; moments do not depend on it).
 *   e0       host out: E = <psi|H|psi> (H applied in the context precision).
 *   resid    host out: |H psi - E psi| of the last cycle (2-norm, energy units);
 *            above tol if max_cycles ran out (the call still returns KPM_OK).
 * Each cycle costs 2 iters + 1 H applications.  Synchronous.  Errors:
 * KPM_EINVAL (iters outside 2..4096, max_cycles outside 1..10000, tol <= 0, NULL
 * pointers), KPM_ETIMEOUT / KPM_ECUDA as kpm_synchronize.
 * Paper: Methods, "KPM for absorption spectra" (|alpha> = mu|0> from the ground
 * state |0>); Results, absorption spectra (Lanczos for the FCI baselines).
 */
kpm_status kpm_ground_state(kpm_ctx* ctx, int iters, int max_cycles, double tol, uint64_t seed,
                            double* psi_dev, double* e0, double* resid);

/* a = (emax - emin) / (2 - eps), b = (emax + emin) / 2. */
void kpm_scale(double emin, double emax, double eps, double* a, double* b);

/*
 * kpm_moments -- Omega_0 .. Omega_{N-1} for each dipole component set in
 * comp_mask (bit c = component c), nmoments even and >= 2.
 *   psi0_dev   FP64 device [dim], the ground state |0> (need not be normalised).
 *   moments_host  host [popcount(comp_mask)][nmoments], FP64, components in
 *                 ascending order.
 * The selected components run as one block vector.  Synchronous.  Returns
 * KPM_EBOUNDS if some |Omega_n| > Omega_0 (1 + 1e-6) (moments still written).
 * Paper: Eq. moments; Methods recursion and doubling identities.
 */
kpm_status kpm_moments(kpm_ctx* ctx, const double* psi0_dev, unsigned comp_mask, double a,
                       double b, int nmoments, double* moments_host);

/* As kpm_moments with psi0 in host memory (copied to the device inside). */
kpm_status kpm_moments_host(kpm_ctx* ctx, const double* psi0_host, unsigned comp_mask,
                            double a, double b, int nmoments, double* moments_host);

/*
 * kpm_moments_deflated -- kpm_moments for a ground state psi0 that is an
 * eigenvector of H with eigenvalue e0, known to FP64 accuracy (for example
 * from kpm_ground_state on a KPM_FP64 context).  The same moments (Eq.
 * moments), evaluated with less round-off: alpha_0 = mu psi0 splits into
 * c0 p + alpha_perp with p = psi0/|psi0| and c0 = <p|alpha_0> (FP64), and since
 * T_n(H~) p = T_n(x0) p, x0 = (e0 - b)/a,
 *   Omega_n = c0^2 T_n(x0) + <alpha_perp|T_n(H~)|alpha_perp>.
 * The recursion (context precision) runs on alpha_perp only; the permanent-
 * dipole term c0^2 T_n(x0) (the peak at omega = e0) is added in FP64 in closed
 * form.  With FP32 vectors this removes the error that grows linearly with n
 * from the ground-state component at the edge of the spectrum, where the
 * Chebyshev recursion amplifies round-off most.  If psi0 is not an eigenvector
 * the cross terms c0 <p|T_n(H~)|alpha_perp> are dropped: results are then only
 * as accurate as psi0's residual |H psi0 - e0 psi0| allows.
 * Arguments and errors as kpm_moments; KPM_EINVAL also if e0 lies outside
 * [b - a, b + a].  Paper: Eq. moments; Methods, KPM for absorption spectra
 * (|alpha> = mu|0> with |0> the ground state).
 */
kpm_status kpm_moments_deflated(kpm_ctx* ctx, const double* psi0_dev, double e0,
                                unsigned comp_mask, double a, double b, int nmoments,
                                double* moments_host);

/*
 * kpm_moments_batch -- kpm_moments for `count` molecules at once: after each
 * molecule's first step, every further Chebyshev step of all molecules is one
 * sigma launch and one update launch over a flattened grid (a table of the
 * molecules' operands, with each molecule's own reduction grid), so small
 * molecules do not pay one set of launches each.  Per molecule the arithmetic
 * and reduction order are those of kpm_moments: the moments are identical.
 *   ctxs       [count] distinct contexts, all KPM_FP64 or all KPM_FP32 (the
 *              CUDA-core gather path), on one device.
 *   psi0_dev   [count] FP64 device ground states, psi0_dev[i] of ctxs[i]'s dim.
 *   a, b       [count] host rescaling of each molecule (as kpm_moments).
 *   moments_host  host [count][popcount(comp_mask)][nmoments].
 * Each molecule's first step runs on its own context's stream, the batched
 * steps on ctxs[0]'s stream, ordered between them by CUDA events; each
 * context's recursion state is left as after kpm_moments.
 * Synchronous.  Errors: KPM_EINVAL for NULL or repeated contexts, mixed or
 * tensor-core (KPM_MIXED*) precisions, or invalid a, b, nmoments, comp_mask;
 * KPM_EBOUNDS if some molecule's |Omega_n| > Omega_0 (1 + 1e-6) (all moments
 * still written; kpm_last_error(ctxs[i]) names it).  The paper's serving
 * pattern of many small molecules per launch; Eq. moments, Methods recursion.
 */
kpm_status kpm_moments_batch(kpm_ctx* const* ctxs, int count, const double* const* psi0_dev,
                             unsigned comp_mask, const double* a, const double* b, int nmoments,
                             double* moments_host);

/*
 * Resumable recursion (the same computation as kpm_moments, in pieces):
 *   kpm_recursion_begin  alpha_0 = mu psi0, first step; state kept on device.
 *   kpm_recursion_advance  `nsteps` further Chebyshev steps (asynchronous).
 *   kpm_recursion_moments  the moments so far into host memory (synchronous);
 *                          *nmoments_out = 2 * (steps done).
 * One Chebyshev step = one H~ product, the update and two FP64 dots per column.
 */
kpm_status kpm_recursion_begin(kpm_ctx* ctx, const double* psi0_dev, unsigned comp_mask,
                               double a, double b, int max_moments);
/* kpm_recursion_begin with the ground-state deflation of kpm_moments_deflated. */
kpm_status kpm_recursion_begin_deflated(kpm_ctx* ctx, const double* psi0_dev, double e0,
                                        unsigned comp_mask, double a, double b,
                                        int max_moments);
kpm_status kpm_recursion_advance(kpm_ctx* ctx, int nsteps);
kpm_status kpm_recursion_moments(kpm_ctx* ctx, double* moments_host, int* nmoments_out);

/*
 * kpm_recursion_advance_batch -- kpm_recursion_advance(ctxs[i], nsteps) for
 * every context, as one sigma launch and one update launch per Chebyshev step
 * for all of them (the batched path of kpm_moments_batch; the contexts may be at
 * different steps).  The launches go to ctxs[0]'s stream, ordered after the
 * work already queued on each context's stream and before work queued on it
 * later (CUDA events): asynchronous.  The result of each recursion is identical
 * to advancing it alone.  Errors: KPM_EINVAL as kpm_moments_batch, or if some
 * context has no recursion in progress or would pass its max_moments.
 * Paper: Methods, KPM recursion; the serving pattern of many molecules per launch.
 */
kpm_status kpm_recursion_advance_batch(kpm_ctx* const* ctxs, int count, int nsteps);

/*
 * kpm_spectrum -- Jackson-damped (kernel=1), Lorentz-damped (kernel=2, lambda =
 * KPM_LORENTZ_LAMBDA) or undamped (kernel=0) Chebyshev reconstruction on the
 * npoints Chebyshev nodes x_k = cos(pi (k+1/2)/M):
 *   I(x) = (g_0 Omega_0 + 2 sum_{n>=1} g_n Omega_n T_n(x)) / (pi sqrt(1-x^2)),
 *   omega = a x + b, intensity = I(x) / a (density per unit energy),
 * written in ascending omega.  g_n = [(N-n+1) cos(pi n/(N+1)) +
 * sin(pi n/(N+1)) cot(pi/(N+1))]/(N+1), n = 0..N-1 (Jackson); g_n =
 * sinh(lambda (1 - n/N)) / sinh(lambda) (Lorentz).  moments, omega_out,
 * intensity_out are host arrays; the sums run in a CUDA kernel on the current
 * device's legacy stream.  Synchronous.  No context needed.
 * Paper: Eq. kpm, Eq. jackson (with the (N-n+1) factor of the KPM review the
 * paper cites; the printed (N-n-1) gives g_0 != 1).
 */
kpm_status kpm_spectrum(const double* moments, int nmoments, double a, double b,
                        int npoints, int kernel, double* omega_out, double* intensity_out);

/*
 * kpm_spectrum_lorentz -- kpm_spectrum with the Lorentz kernel g_n =
 * sinh(lambda (1 - n/N)) / sinh(lambda), lambda > 0 chosen by the caller (the
 * KPM review the paper cites recommends 3..5; the broadening is about lambda/N
 * in x).  Paper: Methods, "modified kernels like the Jackson kernel".
 */
kpm_status kpm_spectrum_lorentz(const double* moments, int nmoments, double a, double b,
                                int npoints, double lambda, double* omega_out,
                                double* intensity_out);

/*
 * kpm_moments_cross -- moments of the dynamical correlation function of two
 * one-body operators (Methods, C_AB): Omega_n = <0| A T_n(H~) B |0>, n < N,
 * with A = sum_pq op_a[p][q] E_pq and B = sum_pq op_b[p][q] E_pq (spin-summed,
 * real symmetric n x n host matrices; the dipole component c is op = -d^c).
 * Two recursions run as one block, a_n = T_n(H~) A|0> and b_n = T_n(H~) B|0>,
 * and since T_m T_n = (T_{m+n} + T_{|m-n|})/2 for the symmetric H~,
 *   Omega_2n = 2 <a_n|b_n> - Omega_0,  Omega_2n+1 = 2 <a_n+1|b_n> - Omega_1
 * (FP64 cross dots), N/2 steps of two columns.  A = B reproduces kpm_moments.
 *   psi0_dev       FP64 device [dim], the ground state.
 *   moments_host   host [nmoments], nmoments even and >= 2.
 * Synchronous.  Errors: KPM_EINVAL (NULL, nmoments, a, b, non-symmetric op),
 * KPM_EBOUNDS if some |Omega_n| exceeds sqrt(<0|A^2|0> <0|B^2|0>) (1 + 1e-6)
 * (the Cauchy-Schwarz bound; moments still written).
 */
kpm_status kpm_moments_cross(kpm_ctx* ctx, const double* psi0_dev, const double* op_a,
                             const double* op_b, double a, double b, int nmoments,
                             double* moments_host);

/*
 * kpm_synchronize -- waits for all work queued on the context's stream and
 * reports errors raised on the device: KPM_ETIMEOUT if a bounded wait inside a
 * kernel ran out (the kernel then returned early and its output is invalid),
 * KPM_ECUDA for an asynchronous CUDA error.
 */
kpm_status kpm_synchronize(kpm_ctx* ctx);

/*
 * kpm_tuned_params -- the launch choices the library's autotuner made for this
 * context at creation: the rasterisation group (row tiles that sweep the column
 * tiles together, for L2 reuse) of the beta and alpha same-spin GEMMs of the
 * tensor-core paths, picked from {4, 8, 16, 32} by timing each once per device
 * and shape (16 for shapes too small to tune).  The choice never changes
 * results.  FP64 / FP32 contexts report 0.  Errors: KPM_EINVAL for NULL ctx.
 */
kpm_status kpm_tuned_params(const kpm_ctx* ctx, int* group_beta, int* group_alpha);

/*
 * kpm_tuned_rowpass -- the autotuner's choices for the opposite-spin row pass
 * of a tensor-core context: the number of shared-memory stages of its gathered
 * A tiles (2 or 3; 3 only where shared memory allows) and how many tiles ahead
 * its copy warps prefetch the gathered rows into L2 (0, 4 or 8), picked by
 * timing each pair once per device and shape at creation (shapes below 2^22
 * determinants keep 3 or 2 stages and 4).  FP64 / FP32 contexts report 0, 0.
 * Errors: KPM_EINVAL for NULL ctx.
 *
 * kpm_set_rowpass -- pins those two choices (results do not depend on them: the
 * same products are formed in the same order, only the copies' timing moves).
 * Errors: KPM_EINVAL for NULL ctx, a non-tensor-core context, stages outside
 * 2..3 or beyond the shared memory sized at creation, prefetch outside 0..64.
 */
kpm_status kpm_tuned_rowpass(const kpm_ctx* ctx, int* stages, int* prefetch);
kpm_status kpm_set_rowpass(kpm_ctx* ctx, int stages, int prefetch);

/*
 * kpm_rowpass_layout -- how the opposite-spin row pass of a tensor-core context
 * holds its targets: the plain layout (wide = 0, passes = 1: 15-bit target strings
 * with the excitation sign in the slot table, one output row's sigma in shared
 * memory) or the wide one (wide = 1: 16-bit targets, the sign taken from the
 * column string's occupations, the targets split into `passes` ranges, one pass
 * over the row's tiles per range).  Creation picks the plain layout where it fits
 * and the wide one with the fewest passes otherwise (more than 32736 strings per
 * spin, or a row's sigma beyond shared memory: 17 and 18 orbitals).  FP64 / FP32
 * contexts report 0, 0.  Errors: KPM_EINVAL for NULL ctx.
 *
 * kpm_set_rowpass_passes -- passes >= 1 switches to the wide layout with that
 * many passes, 0 back to the automatic choice.  The row sums are integer and
 * order-independent, so every layout gives the same sigma bit for bit.  The wide
 * kernel is compiled for 12, 17 and 18 orbitals only.  Errors: KPM_EINVAL for
 * NULL ctx, a non-tensor-core context, passes outside 0..64, or no wide kernel for
 * this size; KPM_EUNSUPPORTED if a pass's targets do not fit in shared memory.
 */
kpm_status kpm_rowpass_layout(const kpm_ctx* ctx, int* wide, int* passes);
kpm_status kpm_set_rowpass_passes(kpm_ctx* ctx, int passes);

/*
 * kpm_graphs_enable -- kpm_recursion_advance (and kpm_moments, the server)
 * issue pairs of Chebyshev steps as replays of CUDA graphs captured on first
 * use (one per assignment of the two rotating recursion vectors; the step
 * index is kept on the device), which removes the per-kernel launch cost that
 * dominates small problems.  Enabled by default; enable = 0 issues every kernel
 * directly.  Results are identical either way (same kernels, same arguments).
 * Steps run directly while profiling is enabled, and for good if a capture
 * fails.  Errors: KPM_EINVAL for a NULL context.
 */
kpm_status kpm_graphs_enable(kpm_ctx* ctx, int enable);

/*
 * Per-launch timing of the H application inside the recursion.
 * kpm_profile_enable(ctx, 1): every H application queued by later
 * kpm_recursion_advance calls on ctx is bracketed by a CUDA event pair recorded
 * on the context's stream.  kpm_profile_read synchronises the stream and
 * returns the summed device time (ms) and the number of H applications since
 * the previous read, then resets both.  Disabled by default.
 */
kpm_status kpm_profile_enable(kpm_ctx* ctx, int enable);
kpm_status kpm_profile_read(kpm_ctx* ctx, double* sigma_ms, int* count);

/*
 * kpm_profile_read_rowpass -- device time of the opposite-spin tensor-core
 * kernel (the row pass, the largest part of a KPM_MIXED / KPM_MIXED_BF16 H
 * application) while profiling is enabled: summed milliseconds over the
 * row-pass launches since the previous read, and their number; both reset.
 * The launches are bracketed by CUDA event pairs on the context's stream (no
 * extra synchronisation inside the recursion); the call synchronises the
 * stream.  FP64 / FP32 contexts have no row pass: *rowpass_ms = 0, *count = 0.
 * Errors: KPM_EINVAL for a NULL context, KPM_ECUDA for a CUDA failure.
 */
kpm_status kpm_profile_read_rowpass(kpm_ctx* ctx, double* rowpass_ms, int* count);

/*
 * kpm_test_rowpass_stall -- testing aid for the bounded waits of the
 * tensor-core row pass (KPM_MIXED / KPM_MIXED_BF16 contexts).  With enable != 0
 * the next row pass (the first column of the next H application) issues no
 * MMAs, so the mbarrier waits of its copy and scatter warps run out after about
 * 10 ms instead of the normal ~2 s limit; the kernel records the expiry, waits
 * for its own copies in flight, frees its tensor memory and returns with its
 * rows unwritten.  kpm_synchronize then reports KPM_ETIMEOUT and clears the
 * flag; the context stays usable and later H applications are exact again.
 * Nothing faults and nothing waits without a limit.  The paper has no
 * counterpart (this library's failure detection).  Errors: KPM_EINVAL for a NULL
 * or non-tensor-core context.
 */
kpm_status kpm_test_rowpass_stall(kpm_ctx* ctx, int enable);

/*
 * kpm_spectrum_static -- kpm_spectrum (kernels 0, 1, 2) for callers that cannot allocate device
 * memory.  The paper has no counterpart; this entry point exists for callers
 * that cannot call cudaMalloc: processes whose device memory is entirely
 * reserved by another allocator (a framework's caching pool, a fixed memory
 * plan), where cudaMalloc fails, and latency-critical loops that cannot pay for
 * cudaMalloc/cudaFree, which synchronise the device.
 *   moments_dev   [nmoments] FP64 device array (caller-owned).
 *   omega_dev, intensity_dev  [npoints] FP64 device arrays (caller-owned),
 *                 filled as kpm_spectrum fills its host outputs.
 *   cuda_stream   cudaStream_t the two kernels are queued on (asynchronous).
 * It allocates nothing: its scratch (the damped moments) is a fixed array of
 * KPM_SPECTRUM_STATIC_MAX_MOMENTS doubles (2 MiB) in the library's device
 * memory, held by every GPU that loads the library until the process exits.
 * nmoments above that limit is rejected with KPM_EINVAL.  The first call on a
 * device looks up the array's device address (cudaGetSymbolAddress) and caches
 * it for the life of the process; make that first call before any stream
 * capture, and do not call it again on a device after cudaDeviceReset (the
 * cached address belonged to the destroyed context).  Every call on a device
 * shares the one array, so calls whose work overlaps on the GPU (for example
 * on two streams at once) race and give undefined results; serialise them.
 * The array needs no clearing: every element read is written first in stream
 * order.  Errors: KPM_EINVAL (arguments, size), KPM_ECUDA; message via
 * kpm_last_error(NULL).
 */
#define KPM_SPECTRUM_STATIC_MAX_MOMENTS 262144
kpm_status kpm_spectrum_static(const double* moments_dev, int nmoments, double a, double b,
                               int npoints, int kernel, double* omega_dev,
                               double* intensity_dev, void* cuda_stream);

/* ------------------------------------------------------------------ serving
 *
 * Continuous batching of spectrum requests on one GPU (this library's
 * serving layer; the paper computes one spectrum at a time).  A worker thread
 * admits queued requests (FIFO) when a slot is free and the request's
 * estimated device memory fits in mem_budget_bytes, keeps every admitted
 * request's recursion resident on its own stream, advances all resident
 * requests by steps_per_round Chebyshev steps per round (queued for all of them
 * before waiting on any, so their kernels overlap), and on completion
 * reconstructs the spectrum (Jackson kernel optional) of the moments summed
 * over the requested dipole components and frees the request's memory.
 * A request computes with the same kernels whether it runs alone or beside
 * others, so its result is the same.  Set-up (kpm_create, the dipole and the
 * first step) runs on a second thread, overlapping the rounds of the resident
 * requests.  A request whose set-up or advance fails is finished at once with
 * that status, and its slot and budget are released.
 */
typedef struct kpm_server kpm_server;

typedef struct {
    size_t mem_budget_bytes; /* device memory admitted requests may hold together     */
    int max_slots;           /* requests resident at once (>= 1)                      */
    int steps_per_round;     /* Chebyshev steps per resident request per round (>= 1) */
    kpm_precision precision; /* arithmetic of every request                           */
} kpm_server_config;

typedef struct {
    const double* h1;      /* host [norb*norb], copied at submit                   */
    const double* eri;     /* host [norb^4], chemist (pq|rs), copied               */
    const double* dipole;  /* host [3*norb*norb], copied                           */
    int norb, nalpha, nbeta;
    const double* psi0;    /* host [dim] ground state, copied                       */
    unsigned comp_mask;    /* dipole components (bit c = component c)            */
    double a, b;           /* rescaling H~ = (H - b)/a (e.g. from kpm_bounds)      */
    int nmoments;          /* even, >= 2                                           */
    int npoints;           /* Chebyshev nodes of the spectrum                      */
    int kernel;            /* 1 = Jackson, 2 = Lorentz (KPM_LORENTZ_LAMBDA), 0 = none */
    int deflate;           /* 1: psi0 is an eigenvector of energy e0, use the      */
    double e0;             /*    deflated recursion of kpm_moments_deflated        */
} kpm_request;

typedef struct {
    double* moments;   /* [ncomp][nmoments] or NULL (caller-owned host memory)    */
    double* omega;     /* [npoints] or NULL, ascending                            */
    double* intensity; /* [npoints] or NULL, summed over components, per energy   */
    double t_queue_s;  /* submit -> admission (out)                               */
    double t_run_s;    /* admission -> result (out)                               */
    double t_total_s;  /* submit -> result, the request's latency (out)            */
} kpm_result;

/* Starts the worker thread on the current device.  KPM_EINVAL for a bad
 * configuration, KPM_ECUDA without a device. */
kpm_status kpm_server_create(const kpm_server_config* cfg, kpm_server** out);
/* Queues a request (inputs copied); *id identifies it.  KPM_ENOMEM if it can
 * never fit the budget, KPM_EINVAL for bad arguments. */
kpm_status kpm_server_submit(kpm_server* s, const kpm_request* req, uint64_t* id);
/* Waits up to timeout_ms for request id and copies its results (then forgets
 * it).  KPM_ETIMEOUT if not finished yet (it stays queued/resident), else the
 * request's own status (KPM_EBOUNDS, KPM_ECANCELLED, ...). */
kpm_status kpm_server_wait(kpm_server* s, uint64_t id, int timeout_ms, kpm_result* out);
/* Cancels a queued or resident request; its wait returns KPM_ECANCELLED. */
kpm_status kpm_server_cancel(kpm_server* s, uint64_t id);
/* Device memory held by admitted requests, resident and queued counts. */
kpm_status kpm_server_stats(kpm_server* s, size_t* mem_used, int* resident, int* queued);
/* Cancels what is queued, lets the resident requests (and one being set up)
 * run to their end, then joins the server's threads. */
void kpm_server_destroy(kpm_server* s);

/* Testing aid for the server's failure handling (host-side fault injection;
 * no GPU work faults): the next round that would advance request id treats
 * that advance as having returned `status` (not KPM_OK).  The request is then
 * finished with that status (kpm_server_wait returns it), its slot and budget
 * are released, and the other requests go on unchanged.  The paper has no
 * counterpart.  Errors: KPM_EINVAL for a NULL server, KPM_OK as status, or an
 * unknown (or already collected) id. */
kpm_status kpm_server_inject_failure(kpm_server* s, uint64_t id, kpm_status status);

/* Number of kernels this library launched on the calling process so far. */
uint64_t kpm_launch_count(void);

#ifdef __cplusplus
}
#endif

#endif /* KPM_H */
