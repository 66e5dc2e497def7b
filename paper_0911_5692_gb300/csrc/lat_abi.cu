// lat_abi.cu -- the C ABI of include/lattice.h: parameter validation and the
// program-unit rescaling (Sec. II.B), buffer ownership, the graph-captured
// evolution loop, initial conditions and diagnostics.
#include <cufft.h>

#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <tuple>
#include <vector>

#include "lat_internal.h"

using namespace lat;

namespace lat {

constexpr int kGraphChunk = 32;

lat_status cuda_status(cudaError_t e) { return e == cudaSuccess ? LAT_OK : LAT_ECUDA; }

// The eight arrays of a state are read and written at the same site index in
// the same instant. Where their starts are equal modulo 2 KB (arrays of a
// power-of-two size allocated one after another are), those accesses meet in
// the same memory partitions: the 512^3 FP32 step measured 0.79 ms with such
// starts and 0.73 ms with starts that differ modulo 2 KB. Array k starts at
// k * (its size rounded up to 2 KB + 128 bytes): offsets k * 128 mod 2048, all
// eight distinct, 128-byte aligned. Of the staggers measured over several
// placements of the allocation in physical memory, 128 bytes had the best
// worst case at 512^3 (0.728-0.732 ms) and at 256^3 (0.108-0.109 ms); 256
// and 1280 bytes were 3-6 % slower at 256^3.
constexpr uint64_t kArrayAlign = 2048, kArrayStagger = 128;

void buffer_layout(size_t array_bytes, uint64_t offsets[8], uint64_t* total)
{
    const uint64_t stride = (array_bytes + kArrayAlign - 1) / kArrayAlign * kArrayAlign + kArrayStagger;
    for (int k = 0; k < 8; k++) offsets[k] = (uint64_t)k * stride;
    *total = 7 * stride + array_bytes;
}

// Sec. II.B: rescaling for a dominant term cpl/beta phi^beta and the program-unit
// potential V_pr = (A^2/B^2) a^(2r-2s) V(f / (A a^r)), which for
// V = cpl/beta phi^beta + g2/2 phi^2 chi^2 is
// cdom0 a^pdom f^beta/beta + kappa0 a^pint f^2 chi^2/2 with
// cdom0 = cpl A^(2-beta)/B^2, pdom = 2r - 2s - beta r, kappa0 = g2/(A^2 B^2),
// pint = -2r - 2s.
lat_status derive_model(const lat_params& p, Model* M)
{
    if (p.n < 4 || p.n > 1024 || (p.n % 4) != 0) return LAT_EINVAL;
    if (p.precision != 32 && p.precision != 64) return LAT_EINVAL;
    if (!(p.L > 0.0) || !(p.dt > 0.0) || !std::isfinite(p.L) || !std::isfinite(p.dt)) return LAT_EINVAL;
    if (p.expansion < 0 || p.expansion > 2) return LAT_EINVAL;
    if (p.stencil != 0 && p.stencil != 7 && p.stencil != 27) return LAT_EINVAL;
    if (p.split != 0 && p.split != 1) return LAT_EINVAL;
    double cpl, beta;
    if (p.model == LAT_MODEL_LPHI4) { cpl = p.lambda; beta = 4.0; }
    else if (p.model == LAT_MODEL_M2PHI2) { cpl = p.m * p.m; beta = 2.0; }
    else return LAT_EINVAL;
    if (!(cpl > 0.0) || p.phi0[0] == 0.0 || !(p.g2 >= 0.0)) return LAT_EINVAL;
    double A, B, r, s;
    if (p.A == 0.0 && p.B == 0.0 && p.r == 0.0 && p.s == 0.0) {
        A = 1.0 / p.phi0[0];
        B = std::sqrt(cpl) * std::pow(std::fabs(p.phi0[0]), beta / 2.0 - 1.0);
        r = 6.0 / (2.0 + beta);
        s = 3.0 * (2.0 - beta) / (2.0 + beta);
    } else {
        A = p.A; B = p.B; r = p.r; s = p.s;
    }
    if (A == 0.0 || !(B > 0.0) || std::fabs(s - 2.0 * r + 3.0) > 1e-12) return LAT_EINVAL;
    if (p.expansion && !(p.eight_pi_G > 0.0)) return LAT_EINVAL;
    std::memset(M, 0, sizeof(*M));
    M->n = p.n;
    M->expansion = p.expansion;
    M->beta = (int)beta;
    M->dx = p.L / p.n;
    M->dt = p.dt;
    M->inv_dx2 = 1.0 / (M->dx * M->dx);
    M->stencil = p.stencil == 27 ? 27 : 7;
    M->split = p.split;
    M->lap_scale = M->stencil == 27 ? M->inv_dx2 / 30.0 : M->inv_dx2;
    M->A = A; M->B = B; M->r = r; M->s = s;
    M->cdom0 = cpl * std::pow(A, 2.0 - beta) / (B * B);
    M->pdom = 2.0 * r - 2.0 * s - beta * r;
    M->kappa0 = p.g2 / (A * A * B * B);
    M->pint = -2.0 * r - 2.0 * s;
    M->eight_pi_G = p.eight_pi_G;
    M->g8A2 = p.eight_pi_G / (A * A);
    M->inv_sites = 1.0 / ((double)p.n * p.n * p.n);
    return LAT_OK;
}

// Effective masses^2 of the two fields at the homogeneous initial values (a = 1).
void meff2_initial(const lat_params& p, const Model& M, double out[2])
{
    const double fh = M.A * p.phi0[0], ch = M.A * p.phi0[1];
    out[0] = M.cdom0 * (M.beta - 1) * std::pow(fh, M.beta - 2) + M.kappa0 * ch * ch;
    out[1] = M.kappa0 * fh * fh;
}

// Stability of the leapfrog: the largest lattice frequency must satisfy
// w dt < 2, w^2 = k_max^2 + m_eff^2 (a = 1), k_max^2 = max over k of -L(k). For
// the 7-point stencil -L = 4 sum_i s_i / dx^2 with s_i = sin^2(k_i dx / 2); for
// the 27-point one -L = (4 sum s_i - 8/3 sum_{i<j} s_i s_j + 32/15 s_1 s_2 s_3) / dx^2,
// multilinear in s in [0, 1]^3 and largest at s = (1, 1, 1): 12/dx^2 and
// 92/(15 dx^2).
lat_status check_cfl(const lat_params& p, const Model& M)
{
    double m2[2];
    meff2_initial(p, M, m2);
    const double mmax = std::max(0.0, std::max(m2[0], m2[1]));
    const double w2 = (M.stencil == 27 ? 92.0 / 15.0 : 12.0) * M.inv_dx2 + mmax;
    if (!(p.dt * p.dt * w2 <= 4.0)) return LAT_ECFL;
    return LAT_OK;
}

size_t partials_needed(int n)
{
    size_t need = (size_t)sums_grid_blocks(n) * kSums;
    need = std::max(need, (size_t)energies_grid_blocks(n) * kEnergySums);
    // the step kernels: one resident wave, or with an explicit z length at most
    // (y tiles) x (z chunks) <= N^2 blocks (x-tiled: a few more)
    need = std::max(need, ((size_t)n * n + 4096) * kSums);
    return need;
}

// The L = 1/H form (expansion 2) solves the next step's coefficients in a pass
// of its own after the sums (and after every step).
lat_status launch_lform_pass(lat_handle* h)
{
    if (h->M.expansion != 2) return LAT_OK;
    cudaError_t e = h->prec == 32 ? launch_lform<float>(bufs_of<float>(h), h->M, h->sc, h->partials, h->stream)
                                  : launch_lform<double>(bufs_of<double>(h), h->M, h->sc, h->partials, h->stream);
    return cuda_status(e);
}

lat_status launch_prepare(lat_handle* h)
{
    cudaError_t e = h->prec == 32 ? launch_sums<float>(bufs_of<float>(h), h->M, h->sc, h->partials, h->stream)
                                  : launch_sums<double>(bufs_of<double>(h), h->M, h->sc, h->partials, h->stream);
    LAT_TRY(cuda_status(e));
    return launch_lform_pass(h);
}

// One step of the configured kernel on the given buffers (the handle's own for
// lat_evolve; per-step storage for the recomputation of the reverse pass).
template <typename T>
cudaError_t launch_step_with(lat_handle* h, const Bufs<T>& b, bool)
{
    return launch_step_march<T>(b, h->M, h->sc, h->partials, h->mcfg, h->stream);
}
template cudaError_t launch_step_with<float>(lat_handle*, const Bufs<float>&, bool);
template cudaError_t launch_step_with<double>(lat_handle*, const Bufs<double>&, bool);

lat_status launch_one_step(lat_handle* h)
{
    cudaError_t e = h->prec == 32 ? launch_step_with<float>(h, bufs_of<float>(h), true)
                                  : launch_step_with<double>(h, bufs_of<double>(h), true);
    LAT_TRY(cuda_status(e));
    return launch_lform_pass(h);
}

void drop_graph(lat_handle* h)
{
    if (h->graph) cudaGraphExecDestroy(h->graph);
    h->graph = nullptr;
    h->graph_steps = 0;
}

lat_status ensure_prepared(lat_handle* h)
{
    if (h->slab) {   // a slab's coefficients come from lat_slab_advance
        h->dirty = false;
        return LAT_OK;
    }
    if (!h->dirty) return LAT_OK;
    LAT_TRY(launch_prepare(h));
    h->dirty = false;
    return LAT_OK;
}

// The L form's Hubble length l = a_t / a'_t at the momentum time t, with a_t
// taken half a step back from the stored a at the field time: a - (dt/2) a'.
double ell_at_momentum_time(double a, double ad, double dt) { return (a - 0.5 * dt * ad) / ad; }

lat_status read_scalars(lat_handle* h, DevScalars* out)
{
    LAT_CUDA(cudaMemcpyAsync(out, h->sc, sizeof(DevScalars), cudaMemcpyDeviceToHost, h->stream));
    LAT_CUDA(cudaStreamSynchronize(h->stream));
    return LAT_OK;
}

lat_status configure_kernel(lat_handle* h, int variant, int ty, int zr, int depth)
{
    const int n = h->p.n;
    if (variant != 0 && variant != 2 && variant != 4 && variant != 5) return LAT_EINVAL;
    auto take = [&](const MarchConfig& cfg, int v) {
        h->mcfg = cfg;
        h->ty = cfg.ty;
        h->zr = cfg.zr;
        h->variant = v;
        drop_graph(h);
        return LAT_OK;
    };
    auto fits = [&](const MarchConfig& cfg) { return (size_t)cfg.blocks * kSums <= h->partials_cap; };
    if (h->M.stencil == 27) {   // the 27-point Laplacian: its own kernels (variants 2 and 5)
        if (variant == 4) return LAT_EUNSUPPORTED;
        MarchConfig cfg;
        if (variant == 5 || variant == 0) {   // x tiles one warp wide where an instance is compiled
            if (s27w_config(n, (int)h->esize, variant == 0 ? 0 : ty, variant == 0 ? 0 : zr, variant == 0 ? 0 : depth,
                            &cfg) &&
                fits(cfg))
                return take(cfg, 5);
            if (variant == 5) return LAT_EUNSUPPORTED;
        }
        if (!march27_config(n, (int)h->esize, variant == 0 ? 0 : ty, variant == 0 ? 0 : zr,
                            variant == 0 ? 0 : depth, &cfg) || !fits(cfg))
            return LAT_EUNSUPPORTED;
        return take(cfg, 2);
    }
    if (variant == 4) {   // the x-tiled plane ring (7-point)
        MarchConfig cfg;
        if (!xt_config(n, (int)h->esize, ty, zr, depth, &cfg) || !fits(cfg)) return LAT_EUNSUPPORTED;
        return take(cfg, 4);
    }
    if (variant == 5) {   // x tiles one warp wide, compiled geometries (7-point)
        MarchConfig cfg;
        if (!xw_config(n, (int)h->esize, ty, zr, depth, &cfg) || !fits(cfg)) return LAT_EUNSUPPORTED;
        return take(cfg, 5);
    }
    if (variant == 0 && h->esize == 4) {
        // FP32: x tiles one warp wide with compiled geometry where an instance
        // exists (N = 256, 512, 1024): 512^3 0.871 ms per step against 0.901 ms
        // (variant 4); 256^3 0.124 against 0.128 ms (variant 2)
        MarchConfig cfg;
        if (xw_config(n, 4, 16, 0, 0, &cfg) && fits(cfg)) return take(cfg, 5);
    }
    if (variant == 0 && n / (16 / (int)h->esize) >= 128) {
        // rows of 128 16-byte vectors or more: full-row tiles leave room for at
        // most 4 owned rows per 7 staged; x tiles of 32 vectors take 16 rows with
        // two planes in flight (FP32 512^3: 0.89 ms per step against 0.98 ms;
        // FP64 512^3: 16 ms against 24 ms, 256^3: 2.04 against 2.10 ms)
        MarchConfig cfg;
        if (xt_config(n, (int)h->esize, 16, 0, 2, &cfg) && fits(cfg)) return take(cfg, 4);
    }
    MarchConfig cfg;
    if (march_config(n, (int)h->esize, variant == 0 ? 0 : ty, variant == 0 ? 0 : zr, variant == 0 ? 0 : depth, &cfg) &&
        fits(cfg))
        return take(cfg, 2);
    if (variant == 2) return LAT_EUNSUPPORTED;
    // rows too wide for a block of full-row tiles: the x-tiled ring serves any N
    if (xt_config(n, (int)h->esize, 0, 0, 0, &cfg) && fits(cfg)) return take(cfg, 4);
    return LAT_EUNSUPPORTED;
}

// ---- the step-kernel autotuner: the fastest (variant, ty, zr, depth) measured on
// a lattice, remembered for the process per (N, precision, stencil, split,
// expansion) and taken by every handle created later with the same key
struct TuneKey {
    int n, prec, stencil, split, expansion;
    bool operator<(const TuneKey& o) const
    {
        return std::tie(n, prec, stencil, split, expansion) < std::tie(o.n, o.prec, o.stencil, o.split, o.expansion);
    }
};
struct TuneShape {
    int variant, ty, zr, depth;
};
std::mutex g_tune_mx;
std::map<TuneKey, TuneShape> g_tuned;

TuneKey tune_key(const lat_handle* h)
{
    return TuneKey{h->p.n, h->prec, h->M.stencil, h->M.split, h->M.expansion};
}

// Candidate shapes for a lattice: every kernel that can run it, over tile
// heights and prefetch depths (configure_kernel refuses the ones that do not fit).
std::vector<TuneShape> tune_candidates(const lat_handle* h)
{
    std::vector<TuneShape> c;
    if (h->M.stencil == 27) {
        c.push_back({5, 16, 0, 1});
        for (int ty : {16, 8, 4})
            for (int d : {1, 2}) c.push_back({2, ty, 0, d});
        return c;
    }
    for (int d : {1, 2}) c.push_back({5, 16, 0, d});
    for (int ty : {32, 16, 8})
        for (int d : {1, 2}) c.push_back({4, ty, 0, d});
    for (int ty : {16, 8, 4, 2})
        for (int d : {1, 2}) c.push_back({2, ty, 0, d});
    return c;
}

lat_status create_common(const lat_params* params, void* stream, void* const bufs[8], lat_handle** out)
{
    if (!out) return LAT_EINVAL;
    *out = nullptr;
    if (!params) return LAT_EINVAL;
    Model M;
    LAT_TRY(derive_model(*params, &M));
    LAT_TRY(check_cfl(*params, M));
    lat_handle* h = new (std::nothrow) lat_handle();
    if (!h) return LAT_ENOMEM;
    h->p = *params;
    h->M = M;
    h->prec = params->precision;
    h->esize = params->precision == 32 ? 4 : 8;
    h->nsites = (size_t)params->n * params->n * params->n;
    h->stream = (cudaStream_t)stream;
    h->owns = bufs == nullptr;
    lat_status st = LAT_OK;
    if (bufs) {
        for (int i = 0; i < 8 && st == LAT_OK; i++) {
            h->buf[i] = bufs[i];
            if (!bufs[i] || ((uintptr_t)bufs[i] & 15u)) st = LAT_EINVAL;
        }
    } else {   // one allocation, the arrays at staggered offsets (buffer_layout)
        uint64_t off[8], total = 0;
        buffer_layout(h->nsites * h->esize, off, &total);
        if (cudaMalloc(&h->arena, total) != cudaSuccess) {
            h->arena = nullptr;
            st = LAT_ENOMEM;
        } else if (cudaMemsetAsync(h->arena, 0, total, h->stream) != cudaSuccess) {
            st = LAT_ECUDA;
        }
        for (int i = 0; i < 8 && st == LAT_OK; i++) h->buf[i] = (char*)h->arena + off[i];
    }
    h->partials_cap = partials_needed(params->n);
    if (st == LAT_OK && cudaMalloc((void**)&h->sc, sizeof(DevScalars)) != cudaSuccess) st = LAT_ENOMEM;
    if (st == LAT_OK && cudaMalloc((void**)&h->partials, h->partials_cap * sizeof(double)) != cudaSuccess)
        st = LAT_ENOMEM;
    if (st == LAT_OK && cudaMalloc((void**)&h->means, 2 * sizeof(double)) != cudaSuccess) st = LAT_ENOMEM;
    if (st == LAT_OK) {
        DevScalars s;
        std::memset(&s, 0, sizeof(s));
        s.a = 1.0;
        if (cudaMemcpyAsync(h->sc, &s, sizeof(s), cudaMemcpyHostToDevice, h->stream) != cudaSuccess ||
            cudaStreamSynchronize(h->stream) != cudaSuccess)
            st = LAT_ECUDA;
    }
    h->dirty = true;
    if (st == LAT_OK) st = configure_kernel(h, 0, 0, 0, 0);
    if (st == LAT_OK) {   // a shape the autotuner chose for this key earlier in the process
        TuneShape t{0, 0, 0, 0};
        {
            std::lock_guard<std::mutex> lock(g_tune_mx);
            auto it = g_tuned.find(tune_key(h));
            if (it != g_tuned.end()) t = it->second;
        }
        if (t.variant && configure_kernel(h, t.variant, t.ty, t.zr, t.depth) != LAT_OK)
            st = configure_kernel(h, 0, 0, 0, 0);
    }
    if (st != LAT_OK) {
        lat_destroy(h);
        return st;
    }
    *out = h;
    return LAT_OK;
}

} // namespace lat

extern "C" {

const char* lat_status_string(lat_status st)
{
    switch (st) {
    case LAT_OK: return "ok";
    case LAT_EINVAL: return "invalid argument or parameters";
    case LAT_ECFL: return "time step violates the leapfrog stability bound";
    case LAT_ENOMEM: return "out of memory";
    case LAT_ECUDA: return "CUDA runtime or library error";
    case LAT_ENONFINITE: return "non-finite sums or no real root for the scale-factor update";
    case LAT_ETIMEOUT: return "a bounded device wait timed out";
    case LAT_EUNSUPPORTED: return "unsupported configuration";
    case LAT_ESTATE: return "call not valid in the current state";
    }
    return "unknown status";
}

lat_status lat_create(const lat_params* params, void* cuda_stream, lat_handle** out)
{
    return create_common(params, cuda_stream, nullptr, out);
}

lat_status lat_create_with_buffers(const lat_params* params, void* cuda_stream, void* const dev_bufs[8],
                                   lat_handle** out)
{
    if (!dev_bufs) return LAT_EINVAL;
    return create_common(params, cuda_stream, dev_bufs, out);
}

void lat_destroy(lat_handle* h)
{
    if (!h) return;
    if (h->stream) cudaStreamSynchronize(h->stream);
    else cudaDeviceSynchronize();
    drop_graph(h);
    if (h->owns && h->arena) cudaFree(h->arena);
    if (h->sc) cudaFree(h->sc);
    if (h->partials) cudaFree(h->partials);
    if (h->means) cudaFree(h->means);
    for (cudaEvent_t e : h->host_down_ev)
        if (e) cudaEventDestroy(e);
    if (h->host_up_done) cudaEventDestroy(h->host_up_done);
    if (h->host_comp_done) cudaEventDestroy(h->host_comp_done);
    if (h->host_up) cudaStreamDestroy(h->host_up);
    if (h->host_down) cudaStreamDestroy(h->host_down);
    if (h->host_log) cudaFree(h->host_log);
    delete h;
}

lat_status lat_sync(lat_handle* h)
{
    if (!h) return LAT_EINVAL;
    DevScalars s;
    LAT_TRY(read_scalars(h, &s));
    return (lat_status)s.status;
}

lat_status lat_set_g2(lat_handle* h, double g2)
{
    if (!h || !(g2 >= 0.0) || !std::isfinite(g2)) return LAT_EINVAL;
    lat_params p = h->p;
    p.g2 = g2;
    Model M;
    LAT_TRY(derive_model(p, &M));
    LAT_TRY(check_cfl(p, M));
    LAT_CUDA(cudaStreamSynchronize(h->stream));
    h->p = p;
    h->M = M;
    drop_graph(h);      // the captured launches carry the old constants
    h->dirty = true;    // coefficients of the next step follow kappa
    return LAT_OK;
}

lat_status lat_set_kernel(lat_handle* h, int variant, int ty, int zr, int depth)
{
    if (!h || variant < 0 || variant > 5 || ty < 0 || zr < 0 || depth < 0) return LAT_EINVAL;
    if (h->slab) return LAT_ESTATE;
    LAT_CUDA(cudaStreamSynchronize(h->stream));
    return configure_kernel(h, variant, ty, zr, depth);
}

lat_status lat_kernel_info(lat_handle* h, int64_t out[8])
{
    if (!h || !out) return LAT_EINVAL;
    out[0] = h->variant;
    out[1] = h->mcfg.blocks; out[2] = h->mcfg.threads; out[3] = (int64_t)h->mcfg.smem;
    out[4] = h->M.expansion == 2 ? 2 : 1;   // the L form adds its own pass
    out[5] = h->ty;
    out[6] = h->zr;
    out[7] = h->mcfg.depth;
    return LAT_OK;
}

lat_status lat_tune(lat_handle* h, int steps, int64_t out[8])
{
    if (!h || steps < 1 || steps > 100000) return LAT_EINVAL;
    if (h->slab) return LAT_ESTATE;
    LAT_TRY(ensure_prepared(h));
    DevScalars s0;
    LAT_TRY(read_scalars(h, &s0));
    if (s0.status != LAT_OK) return (lat_status)s0.status;
    const int par = (int)(s0.step & 1);
    const size_t bytes = h->nsites * h->esize;
    // the current state, saved and put back before every candidate and at the end
    void* save = nullptr;
    if (cudaMalloc(&save, 4 * bytes) != cudaSuccess) return LAT_ENOMEM;
    lat_status st = LAT_OK;
    for (int k = 0; k < 4 && st == LAT_OK; k++)
        if (cudaMemcpyAsync((char*)save + k * bytes, h->buf[4 * par + k], bytes, cudaMemcpyDeviceToDevice, h->stream) !=
            cudaSuccess)
            st = LAT_ECUDA;
    const bool was_dirty = h->dirty;
    auto restore = [&]() {
        for (int k = 0; k < 4; k++)
            if (cudaMemcpyAsync(h->buf[4 * par + k], (char*)save + k * bytes, bytes, cudaMemcpyDeviceToDevice,
                                h->stream) != cudaSuccess)
                return LAT_ECUDA;
        if (cudaMemcpyAsync(h->sc, &s0, sizeof(s0), cudaMemcpyHostToDevice, h->stream) != cudaSuccess) return LAT_ECUDA;
        h->dirty = was_dirty;
        return LAT_OK;
    };
    const int prev[4] = {h->variant, h->ty, h->zr, h->mcfg.depth};
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (st == LAT_OK && (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)) st = LAT_ECUDA;
    TuneShape best{0, 0, 0, 0};
    float best_ms = 0.0f, worst_ms = 0.0f;
    int tried = 0;
    for (const TuneShape& c : tune_candidates(h)) {
        if (st != LAT_OK) break;
        if (configure_kernel(h, c.variant, c.ty, c.zr, c.depth) != LAT_OK) continue;
        // the geometry the kernel was configured with (an automatic zr, the depth taken)
        const TuneShape got{h->variant, h->ty, 0, h->mcfg.depth};
        if ((st = restore()) != LAT_OK) break;
        // a warm-up that also captures the graph, then the timed steps
        if ((st = lat_evolve(h, kGraphChunk)) != LAT_OK) break;
        cudaEventRecord(e0, h->stream);
        if ((st = lat_evolve(h, steps)) != LAT_OK) break;
        cudaEventRecord(e1, h->stream);
        if (cudaEventSynchronize(e1) != cudaSuccess) { st = LAT_ECUDA; break; }
        DevScalars sn;
        if ((st = read_scalars(h, &sn)) != LAT_OK) break;
        if (sn.status != LAT_OK) { st = (lat_status)sn.status; break; }
        float ms = 0.0f;
        cudaEventElapsedTime(&ms, e0, e1);
        ms /= (float)steps;
        tried++;
        if (!best.variant || ms < best_ms) { best = got; best_ms = ms; }
        worst_ms = std::max(worst_ms, ms);
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    lat_status rs = restore();
    if (st == LAT_OK) st = rs;
    if (cudaStreamSynchronize(h->stream) != cudaSuccess && st == LAT_OK) st = LAT_ECUDA;
    cudaFree(save);
    if (st == LAT_OK && !best.variant) st = LAT_EUNSUPPORTED;
    if (st != LAT_OK) {
        configure_kernel(h, prev[0], prev[1], prev[2], prev[3]);
        return st;
    }
    LAT_TRY(configure_kernel(h, best.variant, best.ty, 0, best.depth));
    {
        std::lock_guard<std::mutex> lock(g_tune_mx);
        g_tuned[tune_key(h)] = TuneShape{best.variant, best.ty, 0, best.depth};
    }
    if (out) {
        out[0] = h->variant; out[1] = h->ty; out[2] = h->zr; out[3] = h->mcfg.depth;
        out[4] = tried;
        out[5] = (int64_t)std::llround(best_ms * 1e6);   // nanoseconds per step
        out[6] = (int64_t)std::llround(worst_ms * 1e6);
        out[7] = h->mcfg.blocks;
    }
    return LAT_OK;
}

lat_status lat_evolve(lat_handle* h, int64_t n_steps)
{
    if (!h || n_steps < 0) return LAT_EINVAL;
    if (h->slab) return LAT_ESTATE;
    LAT_TRY(ensure_prepared(h));
    int64_t left = n_steps;
    // Chunks of kGraphChunk steps replay one captured graph; the step kernels read
    // the ping-pong parity and the coefficients from device memory, so the same
    // graph is valid at any step. The legacy default stream cannot be captured.
    if (h->stream != nullptr && left >= kGraphChunk) {
        if (!h->graph) {
            cudaGraph_t g;
            LAT_CUDA(cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal));
            lat_status st = LAT_OK;
            for (int i = 0; i < kGraphChunk && st == LAT_OK; i++) st = launch_one_step(h);
            cudaError_t e = cudaStreamEndCapture(h->stream, &g);
            if (st != LAT_OK) return st;
            if (e != cudaSuccess) return LAT_ECUDA;
            e = cudaGraphInstantiate(&h->graph, g, 0);
            cudaGraphDestroy(g);
            if (e != cudaSuccess) { h->graph = nullptr; return LAT_ECUDA; }
            h->graph_steps = kGraphChunk;
        }
        while (left >= h->graph_steps) {
            LAT_CUDA(cudaGraphLaunch(h->graph, h->stream));
            left -= h->graph_steps;
        }
    }
    for (; left > 0; left--) LAT_TRY(launch_one_step(h));
    return LAT_OK;
}

lat_status lat_get_scalars(lat_handle* h, double out[8])
{
    if (!h || !out) return LAT_EINVAL;
    LAT_TRY(ensure_prepared(h));
    DevScalars s;
    LAT_TRY(read_scalars(h, &s));
    out[0] = s.t; out[1] = s.a; out[2] = s.ad; out[3] = (double)s.step;
    for (int k = 0; k < 4; k++) out[4 + k] = s.S[k];
    return (lat_status)s.status;
}

lat_status lat_set_scalars(lat_handle* h, const double in[4])
{
    if (!h || !in) return LAT_EINVAL;
    if (!std::isfinite(in[0]) || !(in[1] > 0.0) || !std::isfinite(in[2]) || !(in[3] >= 0.0)) return LAT_EINVAL;
    DevScalars s;
    LAT_TRY(read_scalars(h, &s));
    if (h->M.expansion == 2 && in[2] == 0.0) return LAT_EINVAL;   // l = a/a' undefined
    s.t = in[0];
    s.a = h->M.expansion ? in[1] : 1.0;
    s.ad = h->M.expansion ? in[2] : 0.0;
    s.ell = h->M.expansion == 2 ? ell_at_momentum_time(s.a, s.ad, h->M.dt) : 0.0;
    s.step = (long long)in[3];
    s.ticket = 0;
    s.ticket2 = 0;
    LAT_CUDA(cudaMemcpyAsync(h->sc, &s, sizeof(s), cudaMemcpyHostToDevice, h->stream));
    LAT_CUDA(cudaStreamSynchronize(h->stream));
    h->dirty = true;
    return LAT_OK;
}

lat_status lat_get_hubble_length(lat_handle* h, double* ell)
{
    if (!h || !ell) return LAT_EINVAL;
    if (h->M.expansion != 2) return LAT_ESTATE;
    DevScalars s;
    LAT_TRY(read_scalars(h, &s));
    *ell = s.ell;
    return (lat_status)s.status;
}

lat_status lat_set_hubble_length(lat_handle* h, double ell)
{
    if (!h) return LAT_EINVAL;
    if (h->M.expansion != 2) return LAT_ESTATE;
    if (!std::isfinite(ell) || ell == 0.0) return LAT_EINVAL;
    DevScalars s;
    LAT_TRY(read_scalars(h, &s));
    s.ell = ell;
    s.ticket = 0;
    s.ticket2 = 0;
    LAT_CUDA(cudaMemcpyAsync(h->sc, &s, sizeof(s), cudaMemcpyHostToDevice, h->stream));
    LAT_CUDA(cudaStreamSynchronize(h->stream));
    h->dirty = true;   // the next step's coefficients follow l
    return LAT_OK;
}

// The homogeneous mode that whole-field array `what` (0 = f, 1 = f') of `field`
// differs from its stored array by: P or Pi for phi of a split lattice, else 0.
double whole_offset(const lat_handle* h, const DevScalars& s, int field, int what)
{
    if (!h->M.split || field != 0) return 0.0;
    return what == 0 ? s.bgf : s.bgp;
}

lat_status lat_get_state(lat_handle* h, int field, int what, void* dst, int dst_is_device)
{
    if (!h || !dst || field < 0 || field > 1 || what < 0 || what > 3) return LAT_EINVAL;
    DevScalars s;
    LAT_TRY(read_scalars(h, &s));
    const int par = (int)(s.step & 1);
    const void* src = h->buf[4 * par + 2 * (what & 1) + field];
    LAT_CUDA(cudaMemcpyAsync(dst, src, h->nsites * h->esize,
                             dst_is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, h->stream));
    const double off = what < 2 ? whole_offset(h, s, field, what) : 0.0;
    if (off != 0.0 && dst_is_device) {
        cudaError_t e = h->prec == 32 ? launch_shift<float>((float*)dst, h->nsites, off, h->stream)
                                      : launch_shift<double>((double*)dst, h->nsites, off, h->stream);
        LAT_CUDA(e);
    }
    LAT_CUDA(cudaStreamSynchronize(h->stream));
    if (off != 0.0 && !dst_is_device) {   // whole values on the host: stored + P in FP64, rounded once
        if (h->prec == 32) {
            float* d = (float*)dst;
            for (size_t i = 0; i < h->nsites; i++) d[i] = (float)((double)d[i] + off);
        } else {
            double* d = (double*)dst;
            for (size_t i = 0; i < h->nsites; i++) d[i] += off;
        }
    }
    return (lat_status)s.status;
}

lat_status lat_set_state(lat_handle* h, int field, int what, const void* src, int src_is_device)
{
    if (!h || !src || field < 0 || field > 1 || what < 0 || what > 3) return LAT_EINVAL;
    DevScalars s;
    LAT_TRY(read_scalars(h, &s));
    const int par = (int)(s.step & 1);
    void* dst = h->buf[4 * par + 2 * (what & 1) + field];
    LAT_CUDA(cudaMemcpyAsync(dst, src, h->nsites * h->esize,
                             src_is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, h->stream));
    const double off = what < 2 ? whole_offset(h, s, field, what) : 0.0;
    if (off != 0.0) {   // whole values in: the stored array is measured from the homogeneous mode
        cudaError_t e = h->prec == 32 ? launch_shift<float>((float*)dst, h->nsites, -off, h->stream)
                                      : launch_shift<double>((double*)dst, h->nsites, -off, h->stream);
        LAT_CUDA(e);
    }
    LAT_CUDA(cudaStreamSynchronize(h->stream));
    h->dirty = true;
    return LAT_OK;
}

lat_status lat_upload_state(lat_handle* h, const void* const src[4], int src_is_device)
{
    if (!h || !src) return LAT_EINVAL;
    for (int k = 0; k < 4; k++)
        if (!src[k]) return LAT_EINVAL;
    DevScalars s;
    LAT_TRY(read_scalars(h, &s));
    const int par = (int)(s.step & 1);
    for (int k = 0; k < 4; k++)   // f_phi, f_chi, pi_phi, pi_chi of the current set
        LAT_CUDA(cudaMemcpyAsync(h->buf[4 * par + k], src[k], h->nsites * h->esize,
                                 src_is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, h->stream));
    h->dirty = true;
    return LAT_OK;
}

lat_status lat_download_state(lat_handle* h, void* const dst[4], int dst_is_device)
{
    if (!h || !dst) return LAT_EINVAL;
    for (int k = 0; k < 4; k++)
        if (!dst[k]) return LAT_EINVAL;
    LAT_TRY(ensure_prepared(h));
    // the parity of the state the queued work leaves: read after that work
    DevScalars s;
    LAT_TRY(read_scalars(h, &s));
    if (s.status != LAT_OK) return (lat_status)s.status;
    const int par = (int)(s.step & 1);
    for (int k = 0; k < 4; k++)
        LAT_CUDA(cudaMemcpyAsync(dst[k], h->buf[4 * par + k], h->nsites * h->esize,
                                 dst_is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, h->stream));
    LAT_CUDA(cudaStreamSynchronize(h->stream));
    return LAT_OK;
}

lat_status lat_buffer_layout(uint64_t array_bytes, uint64_t offsets[8], uint64_t* total_bytes)
{
    if (!offsets || !total_bytes || array_bytes == 0 || array_bytes > (1ull << 40)) return LAT_EINVAL;
    buffer_layout((size_t)array_bytes, offsets, total_bytes);
    return LAT_OK;
}

lat_status lat_evolve_host(lat_handle* h, void* const host[4], int64_t n_steps, int chunks, double* scalars_out)
{
    if (!h || !host || n_steps < 0) return LAT_EINVAL;
    if (h->slab) return LAT_ESTATE;
    for (int k = 0; k < 4; k++) {
        if (!host[k]) return LAT_EINVAL;
        cudaPointerAttributes at;
        if (cudaPointerGetAttributes(&at, host[k]) != cudaSuccess || at.type != cudaMemoryTypeHost) {
            cudaGetLastError();
            return LAT_EINVAL;   // not page-locked: the copies could not run asynchronously
        }
    }
    if (chunks == 0) chunks = 16;
    if (chunks < 1 || chunks > 64) return LAT_EINVAL;
    const int n = h->p.n;
    chunks = std::min(chunks, n);
    if (n_steps == 0) return LAT_OK;
    DevScalars s0;
    LAT_TRY(read_scalars(h, &s0));
    if (s0.status != LAT_OK) return (lat_status)s0.status;
    int par = (int)(s0.step & 1);
    const size_t plane = (size_t)n * n * h->esize;

    lat_status st = LAT_OK;
    auto ok = [&](cudaError_t e) {
        if (e != cudaSuccess && st == LAT_OK) st = LAT_ECUDA;
        return st == LAT_OK;
    };
    // streams, events and the scalar log live with the handle (lat_destroy)
    if (!h->host_up) ok(cudaStreamCreateWithFlags(&h->host_up, cudaStreamNonBlocking));
    if (!h->host_down && st == LAT_OK) ok(cudaStreamCreateWithFlags(&h->host_down, cudaStreamNonBlocking));
    if (!h->host_up_done && st == LAT_OK) ok(cudaEventCreateWithFlags(&h->host_up_done, cudaEventDisableTiming));
    if (!h->host_comp_done && st == LAT_OK) ok(cudaEventCreateWithFlags(&h->host_comp_done, cudaEventDisableTiming));
    for (int c = 0; c < chunks && st == LAT_OK; c++)
        if (!h->host_down_ev[c]) ok(cudaEventCreateWithFlags(&h->host_down_ev[c], cudaEventDisableTiming));
    if (st != LAT_OK) return st;
    if (scalars_out && h->host_log_cap < (size_t)n_steps) {
        if (h->host_log) cudaFree(h->host_log);
        h->host_log = nullptr;
        h->host_log_cap = 0;
        if (cudaMalloc((void**)&h->host_log, sizeof(DevScalars) * (size_t)n_steps) != cudaSuccess) return LAT_ENOMEM;
        h->host_log_cap = (size_t)n_steps;
    }
    cudaStream_t up = h->host_up, down = h->host_down;
    cudaEvent_t up_done = h->host_up_done, comp_done = h->host_comp_done;
    cudaEvent_t* down_ev = h->host_down_ev;
    DevScalars* dlog = scalars_out ? h->host_log : nullptr;
    // the upload of the first step follows the work already queued on the handle
    if (st == LAT_OK) ok(cudaEventRecord(comp_done, h->stream)) && ok(cudaStreamWaitEvent(up, comp_done, 0));
    for (int64_t k = 0; k < n_steps && st == LAT_OK; k++) {
        // up: chunk c of the four arrays into the current set, once the previous
        // step's download of the same chunk (the same host bytes) has landed
        for (int c = 0; c < chunks && st == LAT_OK; c++) {
            const size_t z0 = (size_t)c * n / chunks, z1 = (size_t)(c + 1) * n / chunks;
            if (k > 0) ok(cudaStreamWaitEvent(up, down_ev[c], 0));
            for (int a = 0; a < 4 && st == LAT_OK; a++)
                ok(cudaMemcpyAsync((char*)h->buf[4 * par + a] + z0 * plane, (const char*)host[a] + z0 * plane,
                                   (z1 - z0) * plane, cudaMemcpyHostToDevice, up));
        }
        if (st != LAT_OK) break;
        ok(cudaEventRecord(up_done, up)) && ok(cudaStreamWaitEvent(h->stream, up_done, 0));
        if (st != LAT_OK) break;
        // the step: the sums of the uploaded fields, then the fused step
        h->dirty = true;
        if ((st = ensure_prepared(h)) != LAT_OK || (st = launch_one_step(h)) != LAT_OK) break;
        if (dlog) ok(cudaMemcpyAsync(dlog + k, h->sc, sizeof(DevScalars), cudaMemcpyDeviceToDevice, h->stream));
        ok(cudaEventRecord(comp_done, h->stream)) && ok(cudaStreamWaitEvent(down, comp_done, 0));
        // down: the evolved set, chunk by chunk
        for (int c = 0; c < chunks && st == LAT_OK; c++) {
            const size_t z0 = (size_t)c * n / chunks, z1 = (size_t)(c + 1) * n / chunks;
            for (int a = 0; a < 4 && st == LAT_OK; a++)
                ok(cudaMemcpyAsync((char*)host[a] + z0 * plane, (const char*)h->buf[4 * (1 - par) + a] + z0 * plane,
                                   (z1 - z0) * plane, cudaMemcpyDeviceToHost, down));
            ok(cudaEventRecord(down_ev[c], down));
        }
        par ^= 1;
    }
    // the handle's stream continues after the last download (its next work may
    // overwrite the set being read)
    if (cudaStreamSynchronize(down) != cudaSuccess && st == LAT_OK) st = LAT_ECUDA;
    if (cudaStreamSynchronize(up) != cudaSuccess && st == LAT_OK) st = LAT_ECUDA;
    if (cudaStreamSynchronize(h->stream) != cudaSuccess && st == LAT_OK) st = LAT_ECUDA;
    if (st == LAT_OK && dlog) {
        std::vector<DevScalars> log((size_t)n_steps);
        if (cudaMemcpy(log.data(), dlog, sizeof(DevScalars) * (size_t)n_steps, cudaMemcpyDeviceToHost) != cudaSuccess)
            st = LAT_ECUDA;
        for (int64_t k = 0; k < n_steps && st == LAT_OK; k++) {
            const DevScalars& q = log[(size_t)k];
            double* o = scalars_out + 8 * k;
            o[0] = q.t; o[1] = q.a; o[2] = q.ad; o[3] = (double)q.step;
            for (int j = 0; j < 4; j++) o[4 + j] = q.S[j];
        }
    }
    if (st != LAT_OK) return st;
    DevScalars s1;
    LAT_TRY(read_scalars(h, &s1));
    return (lat_status)s1.status;
}

lat_status lat_get_background(lat_handle* h, double out[2])
{
    if (!h || !out) return LAT_EINVAL;
    DevScalars s;
    LAT_TRY(read_scalars(h, &s));
    out[0] = s.bgf;
    out[1] = s.bgp;
    return (lat_status)s.status;
}

lat_status lat_set_background(lat_handle* h, const double in[2])
{
    if (!h || !in) return LAT_EINVAL;
    if (!h->M.split) return LAT_ESTATE;
    if (!std::isfinite(in[0]) || !std::isfinite(in[1])) return LAT_EINVAL;
    DevScalars s;
    LAT_TRY(read_scalars(h, &s));
    const int par = (int)(s.step & 1);
    // phi = P + d unchanged: d += P_old - P_new, and the same for the momentum
    const double df = s.bgf - in[0], dp = s.bgp - in[1];
    void* f = h->buf[4 * par + 0];
    void* p = h->buf[4 * par + 2];
    cudaError_t e = h->prec == 32 ? launch_shift<float>((float*)f, h->nsites, df, h->stream)
                                  : launch_shift<double>((double*)f, h->nsites, df, h->stream);
    LAT_CUDA(e);
    e = h->prec == 32 ? launch_shift<float>((float*)p, h->nsites, dp, h->stream)
                      : launch_shift<double>((double*)p, h->nsites, dp, h->stream);
    LAT_CUDA(e);
    s.bgf = in[0];
    s.bgp = in[1];
    s.ticket = 0;
    s.ticket2 = 0;
    LAT_CUDA(cudaMemcpyAsync(h->sc, &s, sizeof(s), cudaMemcpyHostToDevice, h->stream));
    LAT_CUDA(cudaStreamSynchronize(h->stream));
    h->dirty = true;
    return LAT_OK;
}

lat_status lat_recenter(lat_handle* h)
{
    if (!h) return LAT_EINVAL;
    if (!h->M.split || h->slab) return LAT_ESTATE;   // a slab holds part of the volume only
    if ((size_t)2 * kSum2Blocks > h->partials_cap) return LAT_EUNSUPPORTED;
    DevScalars s;
    LAT_TRY(read_scalars(h, &s));
    const int par = (int)(s.step & 1);
    int nb = 0;
    cudaError_t e = h->prec == 32
                        ? launch_sum2<float>((const float*)h->buf[4 * par + 0], (const float*)h->buf[4 * par + 2],
                                             h->nsites, h->partials, &nb, h->stream)
                        : launch_sum2<double>((const double*)h->buf[4 * par + 0], (const double*)h->buf[4 * par + 2],
                                              h->nsites, h->partials, &nb, h->stream);
    LAT_CUDA(e);
    std::vector<double> part(2 * (size_t)nb);
    LAT_CUDA(cudaMemcpyAsync(part.data(), h->partials, part.size() * sizeof(double), cudaMemcpyDeviceToHost,
                             h->stream));
    LAT_CUDA(cudaStreamSynchronize(h->stream));
    double mf = 0.0, mp = 0.0;
    for (int b = 0; b < nb; b++) {
        mf += part[2 * (size_t)b];
        mp += part[2 * (size_t)b + 1];
    }
    const double in[2] = {s.bgf + mf / (double)h->nsites, s.bgp + mp / (double)h->nsites};
    return lat_set_background(h, in);
}

lat_status lat_init_fields(lat_handle* h)
{
    if (!h) return LAT_EINVAL;
    if (h->slab) return LAT_ESTATE;
    const lat_params& p = h->p;
    const Model& M = h->M;
    const int n = p.n;
    // homogeneous state at t = 0, a = 1 (Sec. II.B): H from the homogeneous energy
    const double cpl = p.model == LAT_MODEL_LPHI4 ? p.lambda : p.m * p.m;
    const double beta = (double)M.beta;
    const double V0 = cpl / beta * std::pow(p.phi0[0], beta) + 0.5 * p.g2 * p.phi0[0] * p.phi0[0] * p.phi0[1] * p.phi0[1];
    const double rho0 = 0.5 * (p.dphi0[0] * p.dphi0[0] + p.dphi0[1] * p.dphi0[1]) + V0;
    double ad = 0.0;
    if (p.expansion) {
        if (!(rho0 > 0.0)) return LAT_EINVAL;
        ad = std::sqrt(p.eight_pi_G * rho0 / 3.0) / M.B;   // a' = a^(1-s) H / B at a = 1
    }
    const double h0 = ad;
    double fh[2], ph[2], m2[2];
    for (int i = 0; i < 2; i++) {
        fh[i] = M.A * p.phi0[i];
        ph[i] = M.A / M.B * p.dphi0[i] + M.r * h0 * fh[i];
    }
    meff2_initial(p, M, m2);
    const double amp = p.fluct * M.A * M.B * std::pow(M.dx, -1.5);
    const double kcut = p.kcut > 0.0 ? p.kcut : n / 4.0;

    lat_status st = LAT_OK;
    double *re = nullptr, *df = nullptr, *dp = nullptr;
    void* spec = nullptr;
    cufftHandle fwd = 0, inv = 0;
    bool have_fwd = false, have_inv = false;
    const size_t nspec = (size_t)n * n * (n / 2 + 1);
    if (p.fluct != 0.0) {
        if (cudaMalloc((void**)&re, h->nsites * sizeof(double)) != cudaSuccess ||
            cudaMalloc((void**)&df, h->nsites * sizeof(double)) != cudaSuccess ||
            cudaMalloc((void**)&dp, h->nsites * sizeof(double)) != cudaSuccess ||
            cudaMalloc(&spec, nspec * sizeof(cufftDoubleComplex)) != cudaSuccess)
            st = LAT_ENOMEM;
        if (st == LAT_OK) {
            if (cufftPlan3d(&fwd, n, n, n, CUFFT_D2Z) != CUFFT_SUCCESS) st = LAT_ECUDA;
            else have_fwd = true;
        }
        if (st == LAT_OK) {
            if (cufftPlan3d(&inv, n, n, n, CUFFT_Z2D) != CUFFT_SUCCESS) st = LAT_ECUDA;
            else have_inv = true;
        }
        if (st == LAT_OK && (cufftSetStream(fwd, h->stream) != CUFFT_SUCCESS ||
                             cufftSetStream(inv, h->stream) != CUFFT_SUCCESS))
            st = LAT_ECUDA;
    }
    for (int field = 0; field < 2 && st == LAT_OK; field++) {
        if (p.fluct != 0.0) {
            for (int q = 0; q < 2 && st == LAT_OK; q++) {
                double* outq = q == 0 ? df : dp;
                if (launch_white_noise(re, n, p.seed, (uint32_t)field, (uint32_t)q, h->stream) != cudaSuccess) st = LAT_ECUDA;
                else if (cufftExecD2Z(fwd, re, (cufftDoubleComplex*)spec) != CUFFT_SUCCESS) st = LAT_ECUDA;
                else if (launch_spectral_scale(spec, n, M.dx, m2[field], amp, kcut, q, M.stencil, h->stream) != cudaSuccess) st = LAT_ECUDA;
                else if (cufftExecZ2D(inv, (cufftDoubleComplex*)spec, outq) != CUFFT_SUCCESS) st = LAT_ECUDA;
            }
        }
        if (st != LAT_OK) break;
        // split storage: the homogeneous part of phi goes to the scalar block and
        // the arrays hold the fluctuations alone
        const bool bg = M.split && field == 0;
        const double fhs = bg ? 0.0 : fh[field], phs = bg ? 0.0 : ph[field];
        cudaError_t e = h->prec == 32
                            ? launch_init_combine<float>(bufs_of<float>(h), field, df, dp, fhs, phs, M.r * h0,
                                                         0.5 * p.dt, n, h->stream)
                            : launch_init_combine<double>(bufs_of<double>(h), field, df, dp, fhs, phs, M.r * h0,
                                                          0.5 * p.dt, n, h->stream);
        if (e != cudaSuccess) st = LAT_ECUDA;
    }
    if (st == LAT_OK) {
        DevScalars s;
        std::memset(&s, 0, sizeof(s));
        s.t = 0.0;
        s.ad = ad;
        s.a = 1.0 + (p.expansion ? 0.5 * p.dt * ad : 0.0);
        s.ell = p.expansion == 2 ? ell_at_momentum_time(s.a, s.ad, p.dt) : 0.0;
        s.step = 0;
        if (M.split) {   // the homogeneous mode, advanced by dt/2 like the fields
            s.bgp = ph[0];
            s.bgf = fh[0] + 0.5 * p.dt * ph[0];
        }
        if (cudaMemcpyAsync(h->sc, &s, sizeof(s), cudaMemcpyHostToDevice, h->stream) != cudaSuccess) st = LAT_ECUDA;
    }
    if (st == LAT_OK) {
        h->dirty = true;
        st = ensure_prepared(h);
    }
    if (cudaStreamSynchronize(h->stream) != cudaSuccess && st == LAT_OK) st = LAT_ECUDA;
    if (have_fwd) cufftDestroy(fwd);
    if (have_inv) cufftDestroy(inv);
    cudaFree(re); cudaFree(df); cudaFree(dp); cudaFree(spec);
    return st;
}

lat_status lat_energies(lat_handle* h, lat_energy_report* out)
{
    if (!h || !out) return LAT_EINVAL;
    if (h->slab) return LAT_ESTATE;
    LAT_TRY(ensure_prepared(h));
    const Model& M = h->M;
    const int nb = energies_grid_blocks(M.n);
    std::vector<double> part((size_t)nb * kEnergySums);
    double tot[kEnergySums];
    for (int pass = 0; pass < 2; pass++) {
        cudaError_t e = h->prec == 32 ? launch_energies<float>(bufs_of<float>(h), M, h->sc, h->partials, h->means, pass, h->stream)
                                      : launch_energies<double>(bufs_of<double>(h), M, h->sc, h->partials, h->means, pass, h->stream);
        LAT_CUDA(e);
        LAT_CUDA(cudaMemcpyAsync(part.data(), h->partials, part.size() * sizeof(double), cudaMemcpyDeviceToHost,
                                 h->stream));
        LAT_CUDA(cudaStreamSynchronize(h->stream));
        double acc[kEnergySums] = {0, 0, 0, 0, 0, 0, 0};
        for (int b = 0; b < nb; b++)
            for (int k = 0; k < kEnergySums; k++) acc[k] += part[(size_t)b * kEnergySums + k];
        if (pass == 0) {
            for (int k = 0; k < kEnergySums; k++) tot[k] = acc[k] * M.inv_sites;
            LAT_CUDA(cudaMemcpyAsync(h->means, &tot[5], 2 * sizeof(double), cudaMemcpyHostToDevice, h->stream));
        } else {
            out->var[0] = acc[5] * M.inv_sites;
            out->var[1] = acc[6] * M.inv_sites;
        }
    }
    DevScalars s;
    LAT_TRY(read_scalars(h, &s));
    const double a = s.a;
    const double hh = M.expansion ? s.ad_half / a : 0.0;
    const double cg = std::pow(a, -2.0 * M.s - 2.0);
    const double conv = M.B * M.B / (M.A * M.A) * std::pow(a, 2.0 * M.s - 2.0 * M.r);
    const double kin0 = tot[0], kin1 = tot[1], pot = tot[4];
    const double gr0 = 0.5 * cg * tot[2] * M.lap_scale, gr1 = 0.5 * cg * tot[3] * M.lap_scale;
    out->t = s.t + 0.5 * M.dt;
    out->a = a;
    out->ad = M.expansion ? s.ad_half : 0.0;
    out->H = M.B * std::pow(a, M.s) * hh;
    out->rho = conv * (kin0 + kin1 + gr0 + gr1 + pot);
    out->p = conv * (kin0 + kin1 - (gr0 + gr1) / 3.0 - pot);
    out->w = out->p / out->rho;
    out->curv_resid = out->H != 0.0 ? M.eight_pi_G * out->rho / (3.0 * out->H * out->H) - 1.0 : NAN;
    out->kin[0] = conv * kin0; out->kin[1] = conv * kin1;
    out->grad[0] = conv * gr0; out->grad[1] = conv * gr1;
    out->pot = conv * pot;
    out->mean[0] = tot[5]; out->mean[1] = tot[6];
    return (lat_status)s.status;
}

lat_status lat_energy_field(lat_handle* h, void* rho_dev, void* p_dev)
{
    if (!h || !rho_dev || !p_dev) return LAT_EINVAL;
    if (((uintptr_t)rho_dev | (uintptr_t)p_dev) % h->esize != 0) return LAT_EINVAL;
    if (h->slab) return LAT_ESTATE;
    LAT_TRY(ensure_prepared(h));
    cudaError_t e = h->prec == 32
                        ? launch_energy_field<float>(bufs_of<float>(h), h->M, h->sc, (float*)rho_dev, (float*)p_dev,
                                                     h->stream)
                        : launch_energy_field<double>(bufs_of<double>(h), h->M, h->sc, (double*)rho_dev,
                                                      (double*)p_dev, h->stream);
    return cuda_status(e);
}

lat_status lat_spectrum(lat_handle* h, int field, int nbins, double* k_out, double* p_out, int64_t* count_out)
{
    if (!h || field < 0 || field > 1 || nbins < 1 || nbins > 4096 || !k_out || !p_out || !count_out)
        return LAT_EINVAL;
    if (h->slab) return LAT_ESTATE;
    const int n = h->p.n;
    DevScalars s;
    LAT_TRY(read_scalars(h, &s));
    const int par = (int)(s.step & 1);
    const size_t nspec = (size_t)n * n * (n / 2 + 1);
    const int nb = spectrum_grid_blocks(n);
    double* re = nullptr;
    void* spec = nullptr;
    double* part = nullptr;
    lat_status st = LAT_OK;
    cufftHandle fwd = 0;
    bool have = false;
    if (cudaMalloc((void**)&re, h->nsites * sizeof(double)) != cudaSuccess ||
        cudaMalloc(&spec, nspec * sizeof(cufftDoubleComplex)) != cudaSuccess ||
        cudaMalloc((void**)&part, (size_t)nb * 3 * nbins * sizeof(double)) != cudaSuccess)
        st = LAT_ENOMEM;
    if (st == LAT_OK) {
        const void* src = h->buf[4 * par + field];
        cudaError_t e = h->prec == 32 ? launch_to_double<float>((const float*)src, re, h->nsites, h->stream)
                                      : launch_to_double<double>((const double*)src, re, h->nsites, h->stream);
        if (e == cudaSuccess) e = launch_shift<double>(re, h->nsites, whole_offset(h, s, field, 0), h->stream);
        if (e != cudaSuccess) st = LAT_ECUDA;
    }
    if (st == LAT_OK) {
        if (cufftPlan3d(&fwd, n, n, n, CUFFT_D2Z) != CUFFT_SUCCESS) st = LAT_ECUDA;
        else have = true;
    }
    if (st == LAT_OK && cufftSetStream(fwd, h->stream) != CUFFT_SUCCESS) st = LAT_ECUDA;
    if (st == LAT_OK && cufftExecD2Z(fwd, re, (cufftDoubleComplex*)spec) != CUFFT_SUCCESS) st = LAT_ECUDA;
    if (st == LAT_OK && launch_spectrum_bins(spec, n, h->p.L, nbins, part, h->stream) != cudaSuccess) st = LAT_ECUDA;
    std::vector<double> hp;
    if (st == LAT_OK) {
        hp.resize((size_t)nb * 3 * nbins);
        if (cudaMemcpyAsync(hp.data(), part, hp.size() * sizeof(double), cudaMemcpyDeviceToHost, h->stream) != cudaSuccess ||
            cudaStreamSynchronize(h->stream) != cudaSuccess)
            st = LAT_ECUDA;
    }
    if (st == LAT_OK) {
        for (int b = 0; b < nbins; b++) {
            double pp = 0.0, kk = 0.0, cc = 0.0;
            for (int blk = 0; blk < nb; blk++) {
                const double* row = hp.data() + (size_t)blk * 3 * nbins;
                pp += row[b]; kk += row[nbins + b]; cc += row[2 * nbins + b];
            }
            count_out[b] = (int64_t)std::llround(cc);
            p_out[b] = cc > 0.0 ? pp / cc : 0.0;
            k_out[b] = cc > 0.0 ? kk / cc : 0.0;
        }
    }
    if (have) cufftDestroy(fwd);
    cudaFree(re); cudaFree(spec); cudaFree(part);
    if (st != LAT_OK) return st;
    return (lat_status)s.status;
}

} // extern "C"

namespace {

struct CkptHeader {
    char magic[8];       // "LATCKPT4"
    uint64_t bytes;      // whole blob
    uint32_t scalars_bytes;
    uint32_t esize;
    lat_params params;
};

uint64_t ckpt_bytes(const lat_handle* h)
{
    return sizeof(CkptHeader) + sizeof(DevScalars) + 4 * h->nsites * h->esize;
}

} // namespace

extern "C" {

lat_status lat_checkpoint_bytes(lat_handle* h, uint64_t* bytes)
{
    if (!h || !bytes) return LAT_EINVAL;
    *bytes = ckpt_bytes(h);
    return LAT_OK;
}

lat_status lat_save_checkpoint(lat_handle* h, void* dst, uint64_t bytes)
{
    if (!h || !dst || bytes != ckpt_bytes(h)) return LAT_EINVAL;
    if (h->slab) return LAT_ESTATE;
    LAT_TRY(ensure_prepared(h));
    DevScalars s;
    LAT_TRY(read_scalars(h, &s));
    if (s.status != LAT_OK) return (lat_status)s.status;
    CkptHeader hd;
    std::memset(&hd, 0, sizeof(hd));
    std::memcpy(hd.magic, "LATCKPT4", 8);
    hd.bytes = bytes;
    hd.scalars_bytes = sizeof(DevScalars);
    hd.esize = (uint32_t)h->esize;
    hd.params = h->p;
    unsigned char* out = (unsigned char*)dst;
    s.log = nullptr;
    s.log_base = 0;
    std::memcpy(out, &hd, sizeof(hd));
    std::memcpy(out + sizeof(hd), &s, sizeof(s));
    unsigned char* arr = out + sizeof(hd) + sizeof(s);
    const int par = (int)(s.step & 1);
    for (int k = 0; k < 4; k++)
        LAT_CUDA(cudaMemcpyAsync(arr + k * h->nsites * h->esize, h->buf[4 * par + k], h->nsites * h->esize,
                                 cudaMemcpyDeviceToHost, h->stream));
    LAT_CUDA(cudaStreamSynchronize(h->stream));
    return LAT_OK;
}

lat_status lat_load_checkpoint(lat_handle* h, const void* src, uint64_t bytes)
{
    if (!h || !src || bytes != ckpt_bytes(h)) return LAT_EINVAL;
    if (h->slab) return LAT_ESTATE;
    CkptHeader hd;
    std::memcpy(&hd, src, sizeof(hd));
    if (std::memcmp(hd.magic, "LATCKPT4", 8) != 0 || hd.bytes != bytes || hd.scalars_bytes != sizeof(DevScalars) ||
        hd.esize != h->esize || std::memcmp(&hd.params, &h->p, sizeof(lat_params)) != 0)
        return LAT_EINVAL;
    DevScalars s;
    std::memcpy(&s, (const unsigned char*)src + sizeof(hd), sizeof(s));
    s.ticket = 0;
    s.ticket2 = 0;
    s.log = nullptr;   // a device pointer is never taken from a blob
    s.log_base = 0;
    const unsigned char* arr = (const unsigned char*)src + sizeof(hd) + sizeof(s);
    const int par = (int)(s.step & 1);
    LAT_CUDA(cudaStreamSynchronize(h->stream));
    for (int k = 0; k < 4; k++)
        LAT_CUDA(cudaMemcpyAsync(h->buf[4 * par + k], arr + k * h->nsites * h->esize, h->nsites * h->esize,
                                 cudaMemcpyHostToDevice, h->stream));
    LAT_CUDA(cudaMemcpyAsync(h->sc, &s, sizeof(s), cudaMemcpyHostToDevice, h->stream));
    LAT_CUDA(cudaStreamSynchronize(h->stream));
    h->dirty = false;
    return LAT_OK;
}

} // extern "C"
