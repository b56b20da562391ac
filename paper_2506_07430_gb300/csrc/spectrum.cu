// Kernel damping and Chebyshev reconstruction of the spectrum (Eq. kpm,
// Eq. jackson) on the Chebyshev nodes x_k = cos(theta_k), theta_k = pi(k+1/2)/M:
//   I(x_k) = (g_0 Omega_0 + 2 sum_{n>=1} g_n Omega_n T_n(x_k)) / (pi sin theta_k)
// with the Jackson kernel g_n = [(N-n+1) cos(pi n/(N+1)) + sin(pi n/(N+1))
// cot(pi/(N+1))]/(N+1), or the Lorentz kernel g_n = sinh(lambda (1 - n/N)) /
// sinh(lambda) of the KPM review the paper cites (the Methods name "modified
// kernels like the Jackson kernel"; Lorentz broadening suits Green's functions).
// This is a type-III discrete cosine transform of the damped moments; it is
// evaluated here as a direct FP64 sum (N*M <= a few 1e7 terms per spectrum), with
// T_n(x_k) from the three-term Chebyshev recurrence.  Energy axis
// omega = a x + b, density per unit energy I/a, written in ascending omega.
#include "common.cuh"

namespace kpm {

__global__ void k_damp(const double* __restrict__ mom, int N, int kernel, double lambda,
                       double* __restrict__ mt) {
    int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= N) return;
    double g = 1.0;
    if (kernel == 1) {
        const double q = M_PI / (N + 1);
        double sn, cn;
        sincos(q * n, &sn, &cn);
        g = ((N - n + 1) * cn + sn * (cos(q) / sin(q))) / (N + 1);
    } else if (kernel == 2) {
        g = sinh(lambda * (1.0 - (double)n / N)) / sinh(lambda);
    }
    mt[n] = g * mom[n] * (n == 0 ? 1.0 : 2.0);
}

__global__ void __launch_bounds__(128)
k_reconstruct(const double* __restrict__ mt, int N, double a, double b, int M,
              double* __restrict__ omega, double* __restrict__ inten) {
    __shared__ double sm[1024];
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    double th = M_PI * (k + 0.5) / M;
    double x = cos(th);
    double acc = 0.0, tm1 = 1.0, t = x;  // T_0, T_1
    for (int base = 0; base < N; base += 1024) {
        int cnt = min(1024, N - base);
        __syncthreads();
        for (int i = threadIdx.x; i < cnt; i += blockDim.x) sm[i] = mt[base + i];
        __syncthreads();
        for (int i = 0; i < cnt; ++i) {
            int n = base + i;
            double Tn;
            if (n == 0) Tn = 1.0;
            else if (n == 1) Tn = x;
            else {
                Tn = 2.0 * x * t - tm1;
                tm1 = t;
                t = Tn;
            }
            acc += sm[i] * Tn;
        }
    }
    if (k < M) {
        int o = M - 1 - k;
        omega[o] = a * x + b;
        inten[o] = acc / (M_PI * sin(th)) / a;
    }
}

void spectrum_dev(const double* moments, int N, double a, double b, int M, int kernel,
                  double* damped, double* omega, double* intensity, cudaStream_t st,
                  double lambda) {
    k_damp<<<(N + 127) / 128, 128, 0, st>>>(moments, N, kernel, lambda, damped);
    KPM_LAUNCHED();
    k_reconstruct<<<(M + 127) / 128, 128, 0, st>>>(damped, N, a, b, M, omega, intensity);
    KPM_LAUNCHED();
}

}  // namespace kpm
