// lat_stencil27.cuh -- the 27-point Laplacian of Sec. II.C (Patra and
// Karttunen, over the 3x3x3 cube) at one site, for the FP64 kernels off the
// step path (sums after a state upload, energies). Weights in units of
// 1/(30 dx^2): 14 for the 6 face neighbours, 3 for the 12 edge neighbours, 1 for
// the 8 corner neighbours (and -128 for the centre); M.lap_scale supplies the
// 1/(30 dx^2).
#pragma once

#include <cuda_runtime.h>

namespace lat {

// integer weight of a neighbour offset with |dx| + |dy| + |dz| = 1, 2, 3
__host__ __device__ constexpr int w27(int cls) { return cls == 1 ? 14 : cls == 2 ? 3 : 1; }

__device__ __forceinline__ int wrap27(int v, int n) { return v < 0 ? v + n : v >= n ? v - n : v; }

// sum over the 26 neighbours of w_b (f(x + b) - f(x)): 30 dx^2 (L f)(x)
template <typename T>
__device__ inline double lap27_sum(const T* f, int n, int x, int y, int z)
{
    const double c = (double)f[((size_t)z * n + y) * n + x];
    double acc = 0.0;
    for (int dz = -1; dz <= 1; dz++)
        for (int dy = -1; dy <= 1; dy++)
            for (int dx = -1; dx <= 1; dx++) {
                const int cls = (dx != 0) + (dy != 0) + (dz != 0);
                if (cls == 0) continue;
                const size_t j = ((size_t)wrap27(z + dz, n) * n + wrap27(y + dy, n)) * n + wrap27(x + dx, n);
                acc += w27(cls) * ((double)f[j] - c);
            }
    return acc;
}

// Sum over the 13 bonds (neighbour pairs) the site owns of w_b (f(x + b) -
// f(x))^2; the gradient average is -<f L f> = < that sum > / (30 dx^2). A site
// owns one offset of each +-b pair, all with dy >= 0, so that a tile of rows
// needs the new fields of one row beyond it (in +y) only: four in its plane,
// six to the plane above, three to the plane below ({dx, dy, dz}). Arithmetic
// in R (the differences are exact in the lattice precision for f = const + small).
template <typename R = double, typename T>
__device__ inline R bonds27_sum(const T* f, int n, int x, int y, int z)
{
    constexpr signed char B[13][3] = {{1, 0, 0},  {0, 1, 0},  {1, 1, 0},  {-1, 1, 0},
                                      {0, 0, 1},  {1, 0, 1},  {-1, 0, 1}, {0, 1, 1}, {1, 1, 1}, {-1, 1, 1},
                                      {0, 1, -1}, {1, 1, -1}, {-1, 1, -1}};
    const R c = (R)__ldg(f + ((size_t)z * n + y) * n + x);
    R acc = R(0);
#pragma unroll
    for (int b = 0; b < 13; b++) {
        const int dx = B[b][0], dy = B[b][1], dz = B[b][2];
        const int cls = (dx != 0) + (dy != 0) + (dz != 0);
        const size_t j = ((size_t)wrap27(z + dz, n) * n + wrap27(y + dy, n)) * n + wrap27(x + dx, n);
        const R d = (R)__ldg(f + j) - c;
        acc += R(w27(cls)) * d * d;
    }
    return acc;
}

} // namespace lat
