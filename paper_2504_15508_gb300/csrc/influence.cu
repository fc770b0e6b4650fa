// Plan-time tables: the optimal influence function of PPPM with ik
// differentiation, and the FFT twiddle factors.  Both are computed in FP64 on
// the device; the FP32 path rounds them once.
//
// Influence function (Hockney and Eastwood's optimal G for ik differentiation,
// with the Gaussian reference interaction of Eq. DPLR:EGt, whose Fourier
// kernel is 4 pi exp(-k^2 / (4 beta^2)) / k^2):
//   G(k) = sum_{n in [-a,a]^3} (k . k_n / |k_n|^2) 4 pi exp(-|k_n|^2 / (4 beta^2)) U^2(k_n)
//          / ( |k|^2 [ prod_d sum_{|n_d| <= 20} U_d^2(k_{n,d}) ]^2 ),
//   k_{n,d} = k_d + 2 pi n_d / h_d,  U_d(k) = sinc(k h_d / 2)^p,  G(0) = 0,
// where k_d = 2 pi m_d / L_d, m_d = i_d for i_d <= N_d/2, else i_d - N_d.
// Since k_{n,d} h_d / 2 = pi (m_d / N_d + n_d), every sinc is evaluated as
// sinpi(a) / (pi a) with a = m_d / N_d + n_d.
#include "internal.cuh"

namespace pppm {

__device__ __forceinline__ double sinc_pi(double a) {  // sin(pi a) / (pi a)
    return a == 0.0 ? 1.0 : sinpi(a) / (3.141592653589793238462643 * a);
}

__device__ __forceinline__ double ipow(double x, int e) {
    double r = 1.0;
    for (int i = 0; i < e; ++i) r *= x;
    return r;
}

__global__ void k_influence(Geo g, double beta, int alias, double* __restrict__ G) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int Nx = g.N[0], Ny = g.N[1], Nz = g.N[2], Hz = g.Hz;
    const int64_t total = (int64_t)Nx * Ny * Hz;
    if (idx >= total) return;
    const int iz = (int)(idx % Hz);
    const int iy = (int)((idx / Hz) % Ny);
    const int ix = (int)(idx / ((int64_t)Ny * Hz));
    const int m[3] = {ix <= Nx / 2 ? ix : ix - Nx, iy <= Ny / 2 ? iy : iy - Ny, iz};
    const double twopi = 6.283185307179586476925;
    double k[3], frac[3];
    for (int d = 0; d < 3; ++d) {
        k[d] = twopi * m[d] / g.L[d];
        frac[d] = (double)m[d] / g.N[d];
    }
    const double k2 = k[0] * k[0] + k[1] * k[1] + k[2] * k[2];
    if (k2 == 0.0) { G[idx] = 0.0; return; }
    const int p2 = 2 * g.order;
    double den = 1.0;
    for (int d = 0; d < 3; ++d) {
        double s = 0.0;
        for (int n = -20; n <= 20; ++n) s += ipow(sinc_pi(frac[d] + n), p2);
        den *= s;
    }
    const double inv4b2 = 1.0 / (4.0 * beta * beta);
    double num = 0.0;
    for (int nx = -alias; nx <= alias; ++nx) {
        const double knx = twopi * (m[0] + (double)nx * Nx) / g.L[0];
        const double ux = ipow(sinc_pi(frac[0] + nx), p2);
        for (int ny = -alias; ny <= alias; ++ny) {
            const double kny = twopi * (m[1] + (double)ny * Ny) / g.L[1];
            const double uy = ipow(sinc_pi(frac[1] + ny), p2);
            for (int nz = -alias; nz <= alias; ++nz) {
                const double knz = twopi * (m[2] + (double)nz * Nz) / g.L[2];
                const double uz = ipow(sinc_pi(frac[2] + nz), p2);
                const double kn2 = knx * knx + kny * kny + knz * knz;
                const double dot = k[0] * knx + k[1] * kny + k[2] * knz;
                num += dot / kn2 * 12.566370614359172953850 * exp(-kn2 * inv4b2) * ux * uy * uz;
            }
        }
    }
    G[idx] = num / (k2 * den * den);
}

cudaError_t launch_influence(cudaStream_t s, const Geo& g, double beta, int alias, double* G) {
    const int64_t total = (int64_t)g.N[0] * g.N[1] * g.Hz;
    k_influence<<<(unsigned)((total + 127) / 128), 128, 0, s>>>(g, beta, alias, G);
    return cudaGetLastError();
}

template <typename T>
__global__ void k_convert(const double* __restrict__ in, T* __restrict__ out, int64_t n) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = (T)in[i];
}

template <typename T>
cudaError_t launch_convert(cudaStream_t s, const double* in, T* out, int64_t n) {
    if (n == 0) return cudaSuccess;
    k_convert<T><<<(unsigned)((n + 255) / 256), 256, 0, s>>>(in, out, n);
    return cudaGetLastError();
}

// tw[t] = exp(-2 pi i t / L) = cospi(2t/L) - i sinpi(2t/L)
template <typename C>
__global__ void k_twiddles(int L, C* __restrict__ tw) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= L) return;
    double sn, cs;
    sincospi(2.0 * t / L, &sn, &cs);
    tw[t].x = cs;
    tw[t].y = -sn;
}

template <typename T>
cudaError_t launch_twiddles(cudaStream_t s, int L, typename Cx<T>::t* tw) {
    k_twiddles<typename Cx<T>::t><<<(L + 127) / 128, 128, 0, s>>>(L, tw);
    return cudaGetLastError();
}

template cudaError_t launch_convert<float>(cudaStream_t, const double*, float*, int64_t);
template cudaError_t launch_convert<double>(cudaStream_t, const double*, double*, int64_t);
template cudaError_t launch_twiddles<float>(cudaStream_t, int, float2*);
template cudaError_t launch_twiddles<double>(cudaStream_t, int, double2*);

}  // namespace pppm
