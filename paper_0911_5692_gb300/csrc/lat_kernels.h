// lat_kernels.h -- host-side launchers of the lattice kernels (internal to the
// library; the public ABI is include/lattice.h).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "lat_common.cuh"

namespace lat {

// Device buffers of one lattice: [parity][field] for fields f and momenta f'.
template <typename T>
struct Bufs {
    T* f[2][2];
    T* p[2][2];
};

// Plain-load fused step (both precisions, any N % 4 == 0).
constexpr int kSimpleTX = 32, kSimpleTY = 8;
int simple_grid_blocks(int n, int zr);
template <typename T>
cudaError_t launch_step_simple(const Bufs<T>& b, const Model& M, DevScalars* sc, double* partials, int zr,
                               cudaStream_t st);

// Sums of the current fields (no step) followed by the scale-factor solve.
int sums_grid_blocks(int n);
int sums_zruns(int n);
template <typename T>
cudaError_t launch_sums(const Bufs<T>& b, const Model& M, DevScalars* sc, double* partials, cudaStream_t st);

// Register-prefetch z-march fused step (the default fast path).
struct MarchConfig {
    int ty;        // owned rows per tile
    int zr;        // planes per z-chunk (the longest)
    int nzc;       // z-chunks (balanced lengths)
    int depth;     // planes prefetched ahead (1..4)
    int threads;   // threads per block ((ty + 3) rows x 16-byte vectors)
    int maxt;      // launch-bound instance
    size_t smem;   // dynamic shared memory bytes
    int nyt;       // y tiles
    int blocks;    // blocks per step
    int fast;      // 1: the instance specialised for this (N, ty, depth)
    int nzl = 0;   // z-slab: owned planes (0: a whole periodic lattice)
    int zbase = 0; // z-slab: stored plane of z = z + zbase
    int s27 = 0;   // 1: the 27-point Laplacian kernel (lat_step27.cu)
    int nxt = 1;   // 27-point and x-tiled kernels: x tiles per row
    int xt = 0;    // 1: the x-tiled 7-point kernel (lat_step_xt.cu)
};
// kernel specialised for (element bytes, N, ty, depth), or null; *smem gets its
// dynamic shared memory in bytes
const void* fast_kernel(int elem_bytes, int n, int ty, int depth, size_t* smem);
template <typename T>
cudaError_t launch_step_fast(const Bufs<T>& b, const Model& M, DevScalars* sc, double* partials,
                             const MarchConfig& cfg, cudaStream_t st);
bool march_config(int n, int elem_bytes, int ty, int zr, int depth, MarchConfig* cfg);
// geometry of the general plane-ring kernel over a z-slab of nzl owned planes
// (arrays store plane z at z + 1); one resident wave
bool march_slab_config(int n, int elem_bytes, int nzl, MarchConfig* cfg);
template <typename T>
cudaError_t launch_step_march(const Bufs<T>& b, const Model& M, DevScalars* sc, double* partials,
                              const MarchConfig& cfg, cudaStream_t st, double* sums_out = nullptr);
// the same ring with x tiles of at most 32 (or 16) vectors and taller y tiles
// (whole periodic lattices)
bool xt_config(int n, int elem_bytes, int ty, int zr, int depth, MarchConfig* cfg);
template <typename T>
cudaError_t launch_step_xt(const Bufs<T>& b, const Model& M, DevScalars* sc, double* partials, const MarchConfig& cfg,
                           cudaStream_t st);
// the same ring with the 27-point Laplacian (whole periodic lattices)
bool march27_config(int n, int elem_bytes, int ty, int zr, int depth, MarchConfig* cfg);
template <typename T>
cudaError_t launch_step27(const Bufs<T>& b, const Model& M, DevScalars* sc, double* partials, const MarchConfig& cfg,
                          cudaStream_t st);

// TMA plane-ring fused step.
struct TmaGeom {
    int n, ty, zr, depth;
    int bw, nbx;   // TMA box width (elements) and x chunks per row
    int rs;        // shared-memory row stride in bytes (a multiple of 128)
    int tall;      // 1: one multi-row box per field and x chunk where y does not wrap
    int nyt;       // y tiles
    int rf, rp;    // ring slots for f planes and for momentum planes
    int items;     // (ty + 1) * n / (16 / element bytes)
};
struct TmaConfig {
    int ty;        // owned rows per tile
    int zr;        // requested (y tile, z) planes per block; 0 = one resident wave
    int depth;     // planes prefetched ahead
    int threads;   // threads per block
    size_t smem;   // dynamic shared memory bytes
    int blocks;    // blocks per step (persistent: each marches a contiguous run)
    TmaGeom geom;
};
bool tma_config(int n, int elem_bytes, int ty, int zr, TmaConfig* cfg);
template <typename T>
cudaError_t launch_step_tma(const Bufs<T>& b, const Model& M, DevScalars* sc, double* partials,
                            const TmaConfig& cfg, const void* tmaps, cudaStream_t st);
// Encode the 16 tensor maps of the TMA kernel into `out` (16 * 128 bytes,
// 64-byte aligned host memory): one-row boxes for the 8 arrays, then multi-row
// boxes (ty + 3 rows for fields, ty + 1 for momenta).
constexpr int kTmaMaps = 16;
cudaError_t tma_encode_maps(const void* const ptrs[8], int n, int elem_bytes, int ty, void* out);

// Initial conditions (off the timed path).
struct InitWork {
    double* re;      // N^3 doubles
    double* keep;    // N^3 doubles
    void* spec;      // N*N*(N/2+1) complex doubles
    int fft_fwd, fft_inv;  // cufft handles
};
template <typename T>
cudaError_t launch_init_combine(const Bufs<T>& b, int field, const double* df, const double* dp, double fh,
                                double ph, double r_h0, double half_dt, int n, cudaStream_t st);
cudaError_t launch_white_noise(double* out, int n, uint64_t seed, uint32_t field, uint32_t quantity,
                               cudaStream_t st);
cudaError_t launch_spectral_scale(void* spec, int n, double dx, double meff2, double amp, double kcut,
                                  int quantity, int stencil, cudaStream_t st);

// Diagnostics (off the timed path).
constexpr int kEnergySums = 7;
int energies_grid_blocks(int n);
template <typename T>
cudaError_t launch_energies(const Bufs<T>& b, const Model& M, const DevScalars* sc, double* partials,
                            const double* means, int pass, cudaStream_t st);
template <typename T>
cudaError_t launch_to_double(const T* src, double* dst, size_t count, cudaStream_t st);
// energy density and pressure at every site (eq. rho-pres per site)
template <typename T>
cudaError_t launch_energy_field(const Bufs<T>& b, const Model& M, const DevScalars* sc, T* rho, T* pres,
                                cudaStream_t st);

// The L = 1/H form (expansion 2): the read-only pass over the current state
// whose last block solves the next step's coefficients (lat_lform.cu).
template <typename T>
cudaError_t launch_lform(const Bufs<T>& b, const Model& M, DevScalars* sc, double* partials, cudaStream_t st);
int spectrum_grid_blocks(int n);
cudaError_t launch_spectrum_bins(const void* spec, int n, double L, int nbins, double* partials,
                                 cudaStream_t st);

} // namespace lat
