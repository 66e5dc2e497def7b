// lat_internal.h -- the lattice handle behind the opaque pointer of
// include/lattice.h and the host helpers that the ABI translation units share.
#pragma once

#include "lat_kernels.h"

struct lat_handle {
    lat_params p;
    lat::Model M;
    int prec;
    size_t esize;
    size_t nsites;
    cudaStream_t stream;
    void* buf[8];        // f0, f1, p0, p1 of set 0, then of set 1
    bool owns;
    void* arena;         // the one allocation the eight arrays are cut from (owned buffers)
    lat::DevScalars* sc;      // device
    double* partials;    // device, per-block sums
    size_t partials_cap; // doubles
    double* means;       // device, 2 doubles
    bool dirty;          // sums and coefficients must be recomputed
    int variant;         // 2 = plane-ring z-march over full rows, 4 = over x tiles
    int ty, zr;
    lat::MarchConfig mcfg;
    cudaGraphExec_t graph;
    int graph_steps;
    bool slab;           // a z-slab of a larger lattice (lat_slab_create)
    int slab_z0, slab_nzl;
    // lat_evolve_host: one copy stream per direction, its events and the
    // device log of the scalars after each step (created on first use)
    cudaStream_t host_up, host_down;
    cudaEvent_t host_up_done, host_comp_done, host_down_ev[64];
    lat::DevScalars* host_log;
    size_t host_log_cap;   // entries
};

#define LAT_TRY(expr)                          \
    do {                                       \
        lat_status _s = (expr);                \
        if (_s != LAT_OK) return _s;           \
    } while (0)
#define LAT_CUDA(expr)                                   \
    do {                                                 \
        cudaError_t _e = (expr);                         \
        if (_e != cudaSuccess) return LAT_ECUDA;         \
    } while (0)

namespace lat {

// Byte offsets of the eight state arrays in one allocation, and its size.
void buffer_layout(size_t array_bytes, uint64_t offsets[8], uint64_t* total);

template <typename T>
Bufs<T> bufs_of(const lat_handle* h)
{
    Bufs<T> b;
    for (int par = 0; par < 2; par++)
        for (int f = 0; f < 2; f++) {
            b.f[par][f] = (T*)h->buf[4 * par + f];
            b.p[par][f] = (T*)h->buf[4 * par + 2 + f];
        }
    return b;
}

lat_status cuda_status(cudaError_t e);
lat_status derive_model(const lat_params& p, Model* M);
lat_status ensure_prepared(lat_handle* h);
lat_status read_scalars(lat_handle* h, DevScalars* out);
void drop_graph(lat_handle* h);
template <typename T>
cudaError_t launch_step_with(lat_handle* h, const Bufs<T>& b, bool own_buffers);

} // namespace lat
