// lat_init.cu -- DEFROST-style initial conditions on the device (Sec. II.B,
// last paragraph): homogeneous values plus Gaussian vacuum fluctuations.
//
// White noise: one standard normal per (seed, field, quantity, site) from
// Philox-4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11) with counter
// (site, field, quantity, 0) and key (seed lo, seed hi); words 0 and 1 are mapped
// to (0,1) as (u + 1/2) 2^-32 and turned into a normal by Box-Muller's cosine
// branch. The noise is filtered in Fourier space by the vacuum amplitude
// (cuFFT does the transforms), transformed back and added to the homogeneous
// program-unit values, after which the fields are advanced by dt/2.
#include <cufft.h>

#include "lat_kernels.h"

namespace lat {

namespace {

__device__ __forceinline__ uint32_t mulhi32(uint32_t a, uint32_t b) { return __umulhi(a, b); }

// Philox-4x32-10: ten rounds, each two 32x32->64 multiplies (multipliers
// 0xD2511F53, 0xCD9E8D57) and an xor with the key; the key advances by the
// Weyl constants 0x9E3779B9, 0xBB67AE85 between rounds.
__device__ __forceinline__ void philox4x32_10(uint32_t c[4], uint32_t k0, uint32_t k1)
{
#pragma unroll
    for (int round = 0; round < 10; round++) {
        if (round > 0) { k0 += 0x9E3779B9u; k1 += 0xBB67AE85u; }
        const uint32_t lo0 = 0xD2511F53u * c[0], hi0 = mulhi32(0xD2511F53u, c[0]);
        const uint32_t lo1 = 0xCD9E8D57u * c[2], hi1 = mulhi32(0xCD9E8D57u, c[2]);
        const uint32_t n0 = hi1 ^ c[1] ^ k0, n2 = hi0 ^ c[3] ^ k1;
        c[0] = n0; c[1] = lo1; c[2] = n2; c[3] = lo0;
    }
}

__global__ void white_noise_kernel(double* out, size_t count, uint64_t seed, uint32_t field, uint32_t quantity)
{
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (size_t)gridDim.x * blockDim.x) {
        uint32_t c[4] = {(uint32_t)i, field, quantity, 0u};
        philox4x32_10(c, (uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32));
        const double u1 = ((double)c[0] + 0.5) * (1.0 / 4294967296.0);
        const double u2 = ((double)c[1] + 0.5) * (1.0 / 4294967296.0);
        out[i] = sqrt(-2.0 * log(u1)) * cospi(2.0 * u2);
    }
}

// Multiply the half spectrum (kx in [0, N/2], layout [kz][ky][kx]) by the vacuum
// amplitude: fields 1/sqrt(2 w), momenta sqrt(w/2), times amp = fluct A B dx^-3/2,
// with w^2 = k_lat^2 + m_eff^2, k_lat^2 = sum_d (2/dx sin(pi n_d/N))^2. Empty for
// |n| = 0, |n| > kcut or w^2 <= 0.
__global__ void spectral_scale_kernel(cufftDoubleComplex* spec, int n, double dx, double meff2, double amp,
                                      double kcut, int quantity, int stencil)
{
    const int nh = n / 2 + 1;
    const size_t count = (size_t)n * n * nh;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (size_t)gridDim.x * blockDim.x) {
        const int kx = (int)(i % nh);
        const int ky = (int)((i / nh) % n);
        const int kz = (int)(i / ((size_t)nh * n));
        const int nx = kx < n / 2 ? kx : kx - n;
        const int ny = ky < n / 2 ? ky : ky - n;
        const int nz = kz < n / 2 ? kz : kz - n;
        const double nmag = sqrt((double)nx * nx + (double)ny * ny + (double)nz * nz);
        // k_lat^2 = -L(k) of the stencil in s_i = sin^2(pi n_i / N) (no
        // cancellation at small k): 7-point 4 sum s_i / dx^2; 27-point
        // (4 sum s_i - 8/3 sum_{i<j} s_i s_j + 32/15 s_1 s_2 s_3) / dx^2, the weights
        // 14/30, 3/30, 1/30 of face, edge and corner neighbours written with
        // cos(k_i dx) = 1 - 2 s_i
        const double qx = sinpi((double)nx / n), qy = sinpi((double)ny / n), qz = sinpi((double)nz / n);
        const double s1 = qx * qx, s2 = qy * qy, s3 = qz * qz;
        double klat = 4.0 * (s1 + s2 + s3);
        if (stencil == 27) klat += -8.0 / 3.0 * (s1 * s2 + s1 * s3 + s2 * s3) + 32.0 / 15.0 * s1 * s2 * s3;
        const double w2 = klat / (dx * dx) + meff2;
        double scale = 0.0;
        if (nmag > 0.0 && nmag <= kcut && w2 > 0.0) {
            const double w = sqrt(w2);
            scale = amp * (quantity == 0 ? rsqrt(2.0 * w) : sqrt(0.5 * w));
        }
        spec[i].x *= scale;
        spec[i].y *= scale;
    }
}

// f = fh + df + (dt/2) pi and f' = ph + dp + r h0 df, with the inverse DFT's
// 1/N^3 applied here; the half-step drift of Sec. II.B is taken in FP64 before
// rounding to the storage type. Writes ping-pong set 0.
template <typename T>
__global__ void init_combine_kernel(Bufs<T> B, int field, const double* df, const double* dp, double fh, double ph,
                                    double r_h0, double half_dt, double inv_n3, size_t count)
{
    T* f = B.f[0][field];
    T* p = B.p[0][field];
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (size_t)gridDim.x * blockDim.x) {
        const double d = df ? df[i] * inv_n3 : 0.0;
        const double q = dp ? dp[i] * inv_n3 : 0.0;
        const double pv = ph + q + r_h0 * d;
        const double fv = fh + d + half_dt * pv;
        f[i] = (T)fv;
        p[i] = (T)pv;
    }
}

int grid_for(size_t count)
{
    size_t b = (count + 255) / 256;
    return (int)(b < 4096 ? b : 4096);
}

} // namespace

cudaError_t launch_white_noise(double* out, int n, uint64_t seed, uint32_t field, uint32_t quantity,
                               cudaStream_t st)
{
    const size_t count = (size_t)n * n * n;
    white_noise_kernel<<<grid_for(count), 256, 0, st>>>(out, count, seed, field, quantity);
    return cudaGetLastError();
}

cudaError_t launch_spectral_scale(void* spec, int n, double dx, double meff2, double amp, double kcut,
                                  int quantity, int stencil, cudaStream_t st)
{
    const size_t count = (size_t)n * n * (n / 2 + 1);
    spectral_scale_kernel<<<grid_for(count), 256, 0, st>>>((cufftDoubleComplex*)spec, n, dx, meff2, amp, kcut,
                                                           quantity, stencil);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_init_combine(const Bufs<T>& b, int field, const double* df, const double* dp, double fh,
                                double ph, double r_h0, double half_dt, int n, cudaStream_t st)
{
    const size_t count = (size_t)n * n * n;
    init_combine_kernel<T><<<grid_for(count), 256, 0, st>>>(b, field, df, dp, fh, ph, r_h0, half_dt,
                                                            1.0 / (double)count, count);
    return cudaGetLastError();
}

template cudaError_t launch_init_combine<float>(const Bufs<float>&, int, const double*, const double*, double,
                                                double, double, double, int, cudaStream_t);
template cudaError_t launch_init_combine<double>(const Bufs<double>&, int, const double*, const double*, double,
                                                 double, double, double, int, cudaStream_t);

} // namespace lat
