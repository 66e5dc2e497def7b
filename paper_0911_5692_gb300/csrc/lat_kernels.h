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

// Sums of the current fields (no step) followed by the scale-factor solve
// (lat_sums.cu).
int sums_grid_blocks(int n);
int sums_zruns(int n);
template <typename T>
cudaError_t launch_sums(const Bufs<T>& b, const Model& M, DevScalars* sc, double* partials, cudaStream_t st);

// Plane-ring z-march fused steps (lat_step_march.cu, lat_step_fast.cu,
// lat_step_xt.cu, lat_step27.cu).
// Raise a kernel's dynamic shared memory opt-in to at least `bytes` on the
// current device. The opt-in is process-wide per kernel function and is never
// lowered here: lattices of different shapes share kernel functions, and a
// lower limit set for one would refuse the launches of another.
cudaError_t allow_dynamic_smem(const void* fn, size_t bytes);

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
    int xw = 0;    // 1: the compile-time x-tiled kernel one warp wide (lat_step_xw.cu)
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
// x tiles one warp wide with compile-time N, ty, depth and an edge warp for the
// tile's x neighbours (whole periodic lattices; the compiled geometries only)
bool xw_config(int n, int elem_bytes, int ty, int zr, int depth, MarchConfig* cfg);
template <typename T>
cudaError_t launch_step_xw(const Bufs<T>& b, const Model& M, DevScalars* sc, double* partials, const MarchConfig& cfg,
                           cudaStream_t st);
// the same ring with the 27-point Laplacian (whole periodic lattices)
bool march27_config(int n, int elem_bytes, int ty, int zr, int depth, MarchConfig* cfg);
template <typename T>
cudaError_t launch_step27(const Bufs<T>& b, const Model& M, DevScalars* sc, double* partials, const MarchConfig& cfg,
                          cudaStream_t st);
namespace xw {

// What one launch of a SLAB instance steps: z ranges of one or several
// z-slabs of one lattice held by this process, each slab with its own eight
// arrays (f_phi, f_chi, pi_phi, pi_chi of set 0, then of set 1). Range r is
// rn[r] planes stored from plane rzb[r] of slab rslab[r]'s arrays; the ranges
// are laid end to end in z (range r from plane rz[r], nz planes in all) for
// the block layout, and a run never crosses from one range into the next. The
// sum of the ranges' shares of the volume averages goes to sums_out.
constexpr int kMaxSlabRanges = 16, kMaxLocalSlabs = 8;
struct SlabRun {
    int nranges, nz;
    double* sums_out;
    int rz[kMaxSlabRanges], rn[kMaxSlabRanges], rzb[kMaxSlabRanges], rslab[kMaxSlabRanges];
    void* buf[kMaxLocalSlabs][8];
};

} // namespace xw

// the warp-wide x tiles (lat_xw.cuh) on z ranges of the owned planes of z-slabs
// (N = 256, 512 FP32 with two planes in flight and 256 FP64 with one compiled):
// nz = the ranges' planes in all; the launch writes the ranges' summed shares
bool slab_xw_config(int n, int elem_bytes, int nz, MarchConfig* cfg);
template <typename T>
cudaError_t launch_slab_xw(const xw::SlabRun& R, const Model& M, DevScalars* sc, double* partials,
                           const MarchConfig& cfg, cudaStream_t st);
// the 27-point Laplacian over x tiles one warp wide with compile-time N, ty,
// depth and an edge warp (whole periodic lattices; the compiled geometries only)
bool s27w_config(int n, int elem_bytes, int ty, int zr, int depth, MarchConfig* cfg);
template <typename T>
cudaError_t launch_step27w(const Bufs<T>& b, const Model& M, DevScalars* sc, double* partials, const MarchConfig& cfg,
                           cudaStream_t st);

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

// Split storage (lat_split.cu): a[i] += delta (in FP64, rounded once), and
// per-block FP64 sums of two arrays into partials[2 b], [2 b + 1] (at most
// kSum2Blocks blocks; the count is returned in *blocks).
constexpr int kSum2Blocks = 1024;
template <typename T>
cudaError_t launch_shift(T* a, size_t count, double delta, cudaStream_t st);
template <typename T>
cudaError_t launch_sum2(const T* a, const T* b, size_t count, double* partials, int* blocks, cudaStream_t st);

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
