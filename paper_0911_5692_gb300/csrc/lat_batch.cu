// lat_batch.cu -- ensembles of independent lattices of uneven size and coupling
// stepped together by one persistent launch (Sec. II.B, eq. evo with eq.
// scalar-evo and eq. scale for every member; the paper runs one lattice at a
// time and returns to the host every step).
//
// All (lattice, y tile, z plane) work of one step is laid out in one list,
// weighted by sites, and cut into one contiguous range per resident block, so
// every block does the same amount of work whatever the member sizes. A block
// marches its ranges with the plane-ring segment of lat_march.cuh, writes one
// partial sum per range, and waits at a grid barrier: a counter and a generation
// word in device memory, with a wait bounded by the global timer (a block that
// gives up sets LAT_ETIMEOUT and every block leaves at its next barrier, so a
// broken launch returns an error instead of hanging). After the barrier every
// block that works on a member folds that member's partials in a fixed order
// and advances its FP64 scalars itself (identical results in every block), so
// one barrier per step suffices; one block per member stores them, into the
// scalar slot of the next step (two slots, alternating).
//
// The launch is cooperative (the runtime refuses it unless every block is
// resident, which the barrier needs) and is captured in a CUDA graph per step
// count. The block size and the largest tile height a member may take come from
// a small autotuner that times candidate shapes on the ensemble itself and
// caches the choice per (sizes, precision) for the process.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "lat_internal.h"
#include "lat_march.cuh"

namespace lat {

namespace {

struct BatchCtl {
    unsigned int count;   // blocks arrived at the current barrier
    unsigned int gen;     // barrier generation
    int status;           // LAT_ETIMEOUT if a wait ran out
    int pad;
};

template <typename T>
struct BatchLat {
    Model M;
    T* buf[8];            // f0, f1, p0, p1 of set 0, then of set 1
    int ty, depth;
    int seg_begin, seg_end;   // this member's ranges in the range table
    int owner;            // block that stores the member's scalars
    int pad;
};

struct BatchSeg {
    int l, yt, z0, nz;    // member, y tile, first plane, planes
};

constexpr unsigned long long kBarrierTimeoutNs = 2000000000ull;   // 2 s

__device__ __forceinline__ unsigned long long gtime()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Grid-wide barrier with a bounded wait. Returns false (in every thread) if
// this or another block gave up.
__device__ bool grid_barrier(BatchCtl* ctl, unsigned int nblocks, unsigned long long timeout_ns)
{
    __shared__ int ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        volatile unsigned int* vgen = &ctl->gen;
        volatile int* vst = &ctl->status;
        const unsigned int g = *vgen;
        __threadfence();
        int res = 1;
        if (atomicAdd(&ctl->count, 1u) == nblocks - 1u) {
            ctl->count = 0u;
            __threadfence();
            atomicExch(&ctl->gen, g + 1u);
        } else {
            const unsigned long long t0 = gtime();
            while (*vgen == g) {
                if (*vst != LAT_OK || gtime() - t0 > timeout_ns) {
                    atomicExch(&ctl->status, LAT_ETIMEOUT);
                    res = 0;
                    break;
                }
                __nanosleep(64);
            }
        }
        if (*vst != LAT_OK) res = 0;
        __threadfence();
        ok = res;
    }
    __syncthreads();
    return ok != 0;
}

// A scalar block written by another block earlier in this launch, read through
// L2 (a plain load could return a line this SM cached before it was rewritten).
__device__ inline void load_scalars_cg(const DevScalars* src, DevScalars& dst)
{
    static_assert(sizeof(DevScalars) % 8 == 0, "scalar block is copied in 8-byte words");
    const unsigned long long* s = reinterpret_cast<const unsigned long long*>(src);
    unsigned long long* d = reinterpret_cast<unsigned long long*>(&dst);
    for (int i = 0; i < (int)(sizeof(DevScalars) / 8); i++) d[i] = __ldcg(s + i);
}

// Fold member l's range partials of one step (fixed order, warp 0) and advance
// its scalars from `before`; result in `after` (thread 0).
template <typename T>
__device__ __noinline__ void member_scalars(const BatchLat<T>& BL, const double* part, const DevScalars& before,
                               DevScalars& after)
{
    if (threadIdx.x >= 32) return;
    double v[kSums] = {0.0, 0.0, 0.0, 0.0};
    for (int s = BL.seg_begin + (int)threadIdx.x; s < BL.seg_end; s += 32)
#pragma unroll
        for (int k = 0; k < kSums; k++) v[k] += __ldcg(part + (size_t)s * kSums + k);
#pragma unroll
    for (int k = 0; k < kSums; k++)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_down_sync(0xffffffffu, v[k], o);
    if (threadIdx.x == 0) {
        const Model& M = BL.M;
        const double S[kSums] = {v[0] * M.inv_dx2 * M.inv_sites, v[1] * M.inv_dx2 * M.inv_sites, v[2] * M.inv_sites,
                                 v[3] * M.inv_sites};
        load_scalars_cg(&before, after);
        advance_scalars(M, after, S, true);
    }
}

// sc: two scalar slots per member ([2 l + slot]); slot 0 holds the scalars at
// the start of the launch, slot (k & 1) those at the start of step k.
// part: [2][nsegs][kSums]; cta: range table offsets per block.
template <typename T, int MAXT, bool SPLIT>
__global__ void __launch_bounds__(MAXT, MAXT <= 256 ? 3 : (MAXT <= 512 ? 2 : 1)) batch_kernel(const BatchLat<T>* __restrict__ lats,
                                                     const BatchSeg* __restrict__ segs, const int* __restrict__ cta,
                                                     int nsegs, DevScalars* sc, double* part, BatchCtl* ctl, int nsteps,
                                                     int nlat, unsigned int extra, unsigned long long timeout_ns)
{
    __shared__ double red[32 * kSums];
    __shared__ DevScalars cur;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* const S = reinterpret_cast<T*>(smem_raw);
    const int sb = cta[blockIdx.x], se = cta[blockIdx.x + 1];
    // `extra` > 0 only for the barrier self-test: the barrier then waits for
    // arrivals that never come and every block leaves when its wait runs out
    const unsigned int nblocks = gridDim.x + extra;
    if (extra) {
        grid_barrier(ctl, nblocks, timeout_ns);
        return;
    }
    for (int k = 0; k < nsteps; k++) {
        double* pk = part + (size_t)(k & 1) * nsegs * kSums;
        const double* pprev = part + (size_t)((k + 1) & 1) * nsegs * kSums;
        int last_l = -1;
        for (int s = sb; s < se; s++) {
            const BatchSeg g = segs[s];
            const BatchLat<T>& BL = lats[g.l];
            if (g.l != last_l) {
                __syncthreads();   // every thread is done with the previous member's scalars
                if (k == 0) {
                    if (threadIdx.x == 0) cur = sc[2 * g.l];
                } else {
                    DevScalars after;
                    member_scalars(BL, pprev, sc[2 * g.l + ((k - 1) & 1)], after);
                    if (threadIdx.x == 0) {
                        cur = after;
                        if ((int)blockIdx.x == BL.owner) sc[2 * g.l + (k & 1)] = after;
                    }
                }
                __syncthreads();
                last_l = g.l;
            }
            double bs[kSums] = {0.0, 0.0, 0.0, 0.0};
            if (cur.status == LAT_OK) {
                const bool par = (cur.step & 1) != 0;
                MarchLattice<T> L;
                L.f0 = BL.buf[par ? 4 : 0];
                L.f1 = BL.buf[par ? 5 : 1];
                L.p0 = BL.buf[par ? 6 : 2];
                L.p1 = BL.buf[par ? 7 : 3];
                L.of0 = BL.buf[par ? 0 : 4];
                L.of1 = BL.buf[par ? 1 : 5];
                L.op0 = BL.buf[par ? 2 : 6];
                L.op1 = BL.buf[par ? 3 : 7];
                L.n = BL.M.n;
                L.ty = BL.ty;
                L.depth = BL.depth;
                L.K = site_coefs<T>(&cur, BL.M.beta);
                L.periodic = true;
                L.zbase = 0;
                MarchSums<T> A;
                A.zero();
                march_segment<T, SPLIT>(L, g.yt, g.z0, g.nz, S, A, s == sb);
                T v[kSums];
                A.totals(L.K.quartic, v);
                block_reduce(v, red, bs);
            }
            if (threadIdx.x == 0)
                for (int q = 0; q < kSums; q++) pk[(size_t)s * kSums + q] = bs[q];
        }
        __threadfence();
        if (!grid_barrier(ctl, nblocks, timeout_ns)) return;
    }
    // scalars after the last step, stored by each member's owner
    if (nsteps > 0) {
        const double* plast = part + (size_t)((nsteps - 1) & 1) * nsegs * kSums;
        for (int l = 0; l < nlat; l++) {
            const BatchLat<T>& BL = lats[l];
            if (BL.owner != (int)blockIdx.x) continue;
            DevScalars after;
            member_scalars(BL, plast, sc[2 * l + ((nsteps - 1) & 1)], after);
            if (threadIdx.x == 0) sc[2 * l + (nsteps & 1)] = after;
            __syncthreads();
        }
    }
}

// Copy the scalar blocks between the members' handles and the batch slots:
// dir 0: handle -> slot 0; dir 1: slot `slot` -> handle.
__global__ void scalars_copy_kernel(DevScalars* const* hsc, DevScalars* sc, int nlat, int dir, int slot)
{
    const int l = blockIdx.x * blockDim.x + threadIdx.x;
    if (l >= nlat) return;
    if (dir == 0) {
        DevScalars s = *hsc[l];
        s.ticket = 0u;
        sc[2 * l] = s;
    } else {
        *hsc[l] = sc[2 * l + slot];
    }
}

// the instance for a launch shape; `split`: some member stores phi split
template <typename T>
const void* batch_fn(int maxt, bool split)
{
    switch (maxt) {
    case 256: return split ? (const void*)batch_kernel<T, 256, true> : (const void*)batch_kernel<T, 256, false>;
    case 512: return split ? (const void*)batch_kernel<T, 512, true> : (const void*)batch_kernel<T, 512, false>;
    default: return split ? (const void*)batch_kernel<T, 1024, true> : (const void*)batch_kernel<T, 1024, false>;
    }
}

int maxt_of(int threads) { return threads <= 256 ? 256 : threads <= 512 ? 512 : 1024; }

// Shape of one launch.
struct BatchShape {
    int threads = 0;
    int tycap = 32;       // largest tile height a member takes
    int depth = 1;        // planes in flight ahead of the one computed
    int maxt = 0;
    size_t smem = 0;
    int blocks = 0;
    std::vector<int> ty;
};

std::mutex g_tune_mutex;
struct TunedShape {
    int threads, tycap, depth;
};
std::map<std::string, TunedShape> g_tuned;   // (sizes, precision) -> the fastest shape timed

} // namespace

} // namespace lat

using namespace lat;

struct lat_batch {
    int count = 0;
    int prec = 32;
    size_t esize = 4;
    cudaStream_t stream = nullptr;
    std::vector<lat_handle*> h;
    BatchShape shape;
    int nsegs = 0;
    void* dlats = nullptr;
    BatchSeg* dsegs = nullptr;
    int* dcta = nullptr;
    DevScalars* dsc = nullptr;
    DevScalars** dhsc = nullptr;
    double* dpart = nullptr;
    BatchCtl* dctl = nullptr;
    std::map<int64_t, cudaGraphExec_t> graphs;
    bool captured = false;
    bool split = false;   // some member stores phi split
};

namespace {

void free_tables(lat_batch* b)
{
    for (auto& kv : b->graphs) cudaGraphExecDestroy(kv.second);
    b->graphs.clear();
    cudaFree(b->dlats); cudaFree(b->dsegs); cudaFree(b->dcta); cudaFree(b->dpart);
    b->dlats = nullptr; b->dsegs = nullptr; b->dcta = nullptr; b->dpart = nullptr;
}

std::string tune_key(const lat_batch* b)
{
    std::vector<int> ns;
    for (lat_handle* h : b->h) ns.push_back(h->p.n);
    std::sort(ns.begin(), ns.end());
    std::string k = std::to_string(b->prec) + ":";
    for (int n : ns) k += std::to_string(n) + ",";
    return k;
}

// Tile heights (each member the largest of 32, 16, ... 1 that divides its side,
// is at most tycap and fits the block), ring size for the prefetch depth and
// resident blocks for a block size; false if some member does not fit.
bool shape_for(const lat_batch* b, int threads, int tycap, int depth, BatchShape* out)
{
    BatchShape s;
    s.threads = threads;
    s.tycap = tycap;
    s.depth = depth;
    s.maxt = maxt_of(threads);
    const int vw = (int)(16 / b->esize);
    size_t smem = 0;
    for (lat_handle* h : b->h) {
        const int n = h->p.n;
        int best = 0;
        for (int ty : {32, 16, 8, 4, 2, 1}) {
            if (ty > n || ty > tycap || n % ty != 0) continue;
            if ((ty + 3) * (n / vw) > threads) continue;
            if (ring_elems(n, ty, depth) * b->esize > 200 * 1024) continue;
            best = ty;
            break;
        }
        if (!best) return false;
        s.ty.push_back(best);
        smem = std::max(smem, ring_elems(n, best, depth) * b->esize);
    }
    s.smem = smem;
    const void* fn = b->prec == 32 ? batch_fn<float>(s.maxt, b->split) : batch_fn<double>(s.maxt, b->split);
    if (allow_dynamic_smem(fn, smem) != cudaSuccess) return false;
    int occ = 0, dev = 0, sms = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, threads, smem) != cudaSuccess || occ < 1) return false;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return false;
    s.blocks = occ * sms;
    *out = s;
    return true;
}

// Lay out the (member, y tile, z plane) work, weighted by sites, in one
// contiguous range per block, and upload the tables.
template <typename T>
lat_status build_tables(lat_batch* b, const BatchShape& s)
{
    const int nl = b->count;
    std::vector<double> w;          // weight of each (member, y tile) column of planes
    long long total = 0;
    for (int l = 0; l < nl; l++) total += (long long)b->h[l]->nsites;
    const int G = std::max(1, std::min<int>(s.blocks, (int)(total / 512 + 1)));
    std::vector<BatchSeg> segs;
    std::vector<int> cta(G + 1, 0);
    std::vector<BatchLat<T>> lats(nl);
    // walk the planes in order, cutting at multiples of total / G sites
    long long acc = 0;
    int blk = 0;
    for (int l = 0; l < nl; l++) {
        lat_handle* h = b->h[l];
        const int n = h->p.n, ty = s.ty[l];
        lats[l].M = h->M;
        for (int i = 0; i < 8; i++) lats[l].buf[i] = (T*)h->buf[i];
        lats[l].ty = ty;
        lats[l].depth = s.depth;
        lats[l].seg_begin = (int)segs.size();
        const long long per_plane = (long long)n * ty;
        for (int yt = 0; yt < n / ty; yt++) {
            int z = 0;
            while (z < n) {
                // planes this block can still take before its share is full
                const long long bound = (long long)((double)total * (blk + 1) / G);
                long long room = (bound - acc + per_plane - 1) / per_plane;
                if (blk == G - 1) room = n;
                if (room < 1) room = 1;
                const int nz = (int)std::min<long long>(room, n - z);
                segs.push_back(BatchSeg{l, yt, z, nz});
                acc += per_plane * nz;
                z += nz;
                while (blk < G - 1 && acc >= (long long)((double)total * (blk + 1) / G)) {
                    blk++;
                    cta[blk] = (int)segs.size();
                }
            }
        }
        lats[l].seg_end = (int)segs.size();
    }
    for (int i = blk + 1; i <= G; i++) cta[i] = (int)segs.size();
    // owner: the block holding the member's first range
    for (int l = 0; l < nl; l++) {
        int o = 0;
        while (o + 1 <= G && cta[o + 1] <= lats[l].seg_begin) o++;
        lats[l].owner = o;
    }
    free_tables(b);
    b->nsegs = (int)segs.size();
    b->shape = s;
    b->shape.blocks = G;
    if (cudaMalloc(&b->dlats, sizeof(BatchLat<T>) * nl) != cudaSuccess ||
        cudaMalloc((void**)&b->dsegs, sizeof(BatchSeg) * segs.size()) != cudaSuccess ||
        cudaMalloc((void**)&b->dcta, sizeof(int) * (G + 1)) != cudaSuccess ||
        cudaMalloc((void**)&b->dpart, sizeof(double) * 2 * kSums * segs.size()) != cudaSuccess)
        return LAT_ENOMEM;
    LAT_CUDA(cudaMemcpy(b->dlats, lats.data(), sizeof(BatchLat<T>) * nl, cudaMemcpyHostToDevice));
    LAT_CUDA(cudaMemcpy(b->dsegs, segs.data(), sizeof(BatchSeg) * segs.size(), cudaMemcpyHostToDevice));
    LAT_CUDA(cudaMemcpy(b->dcta, cta.data(), sizeof(int) * (G + 1), cudaMemcpyHostToDevice));
    return LAT_OK;
}

lat_status configure(lat_batch* b, int threads, int tycap, int depth)
{
    BatchShape s;
    if (!shape_for(b, threads, tycap, depth, &s)) return LAT_EUNSUPPORTED;
    return b->prec == 32 ? build_tables<float>(b, s) : build_tables<double>(b, s);
}

template <typename T>
cudaError_t launch_batch(lat_batch* b, int64_t nsteps, unsigned int extra = 0,
                         unsigned long long timeout_ns = kBarrierTimeoutNs)
{
    const int nl = b->count;
    scalars_copy_kernel<<<(nl + 127) / 128, 128, 0, b->stream>>>(b->dhsc, b->dsc, nl, 0, 0);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    e = cudaMemsetAsync(b->dctl, 0, sizeof(BatchCtl), b->stream);
    if (e != cudaSuccess) return e;
    const void* fn = batch_fn<T>(b->shape.maxt, b->split);
    const BatchLat<T>* lats = (const BatchLat<T>*)b->dlats;
    int nsegs = b->nsegs, ns = (int)nsteps, nlat = nl;
    void* args[] = {(void*)&lats, (void*)&b->dsegs, (void*)&b->dcta, (void*)&nsegs, (void*)&b->dsc,
                    (void*)&b->dpart, (void*)&b->dctl, (void*)&ns, (void*)&nlat, (void*)&extra, (void*)&timeout_ns};
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(b->shape.blocks);
    cfg.blockDim = dim3(b->shape.threads);
    cfg.dynamicSmemBytes = b->shape.smem;
    cfg.stream = b->stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    e = cudaLaunchKernelExC(&cfg, fn, args);
    if (e != cudaSuccess || extra) return e;
    scalars_copy_kernel<<<(nl + 127) / 128, 128, 0, b->stream>>>(b->dhsc, b->dsc, nl, 1, (int)(nsteps & 1));
    return cudaGetLastError();
}

lat_status run_steps(lat_batch* b, int64_t nsteps)
{
    if (nsteps <= 0) return LAT_OK;
    for (lat_handle* h : b->h) {
        LAT_TRY(ensure_prepared(h));
        drop_graph(h);
    }
    // one graph per step count (the count is a kernel argument)
    auto it = b->graphs.find(nsteps);
    if (it == b->graphs.end() && b->stream != nullptr) {
        cudaGraph_t g;
        cudaGraphExec_t ge = nullptr;
        if (cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
            cudaError_t e = b->prec == 32 ? launch_batch<float>(b, nsteps) : launch_batch<double>(b, nsteps);
            cudaError_t e2 = cudaStreamEndCapture(b->stream, &g);
            if (e == cudaSuccess && e2 == cudaSuccess) {
                if (cudaGraphInstantiate(&ge, g, 0) == cudaSuccess) it = b->graphs.emplace(nsteps, ge).first;
                cudaGraphDestroy(g);
            }
        }
        cudaGetLastError();   // a refused capture leaves no error behind; launch directly below
    }
    if (it != b->graphs.end()) {
        b->captured = true;
        LAT_CUDA(cudaGraphLaunch(it->second, b->stream));
    } else {
        b->captured = false;
        LAT_CUDA(b->prec == 32 ? launch_batch<float>(b, nsteps) : launch_batch<double>(b, nsteps));
    }
    return LAT_OK;
}

// Time candidate shapes (block size, tile cap, prefetch depth) on the ensemble
// itself (state saved and restored) and keep the fastest. Caps that give every
// member the same tile heights as one already listed, at the same block size
// and depth, are one candidate.
lat_status autotune(lat_batch* b, int steps)
{
    const std::string key = tune_key(b);
    std::vector<TunedShape> cands;
    for (int depth : {1, 2})
        for (int t : {128, 192, 256, 320, 384, 448, 512, 640, 768, 1024}) {
            std::vector<std::vector<int>> seen;
            for (int cap : {32, 16, 8, 4}) {
                BatchShape s;
                if (!shape_for(b, t, cap, depth, &s)) continue;
                if (std::find(seen.begin(), seen.end(), s.ty) != seen.end()) continue;
                seen.push_back(s.ty);
                cands.push_back({t, cap, depth});
            }
        }
    if (cands.empty()) return LAT_EUNSUPPORTED;
    // save the current state of every member
    const int nl = b->count;
    std::vector<void*> save(nl, nullptr);
    std::vector<DevScalars> ssave(nl);
    lat_status st = LAT_OK;
    for (int l = 0; l < nl && st == LAT_OK; l++) {
        lat_handle* h = b->h[l];
        st = ensure_prepared(h);
        if (st != LAT_OK) break;
        if (cudaMalloc(&save[l], 8 * h->nsites * h->esize) != cudaSuccess) { st = LAT_ENOMEM; break; }
        for (int i = 0; i < 8; i++)
            if (cudaMemcpyAsync((char*)save[l] + i * h->nsites * h->esize, h->buf[i], h->nsites * h->esize,
                                cudaMemcpyDeviceToDevice, b->stream) != cudaSuccess)
                st = LAT_ECUDA;
        if (cudaMemcpyAsync(&ssave[l], h->sc, sizeof(DevScalars), cudaMemcpyDeviceToHost, b->stream) != cudaSuccess)
            st = LAT_ECUDA;
    }
    if (cudaStreamSynchronize(b->stream) != cudaSuccess && st == LAT_OK) st = LAT_ECUDA;
    TunedShape best{0, 32, 1};
    float best_ms = 0.0f;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (st == LAT_OK && (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)) st = LAT_ECUDA;
    for (size_t c = 0; c < cands.size() && st == LAT_OK; c++) {
        if (configure(b, cands[c].threads, cands[c].tycap, cands[c].depth) != LAT_OK) continue;
        if (run_steps(b, 2) != LAT_OK) continue;   // warm-up and graph
        cudaEventRecord(e0, b->stream);
        lat_status rs = run_steps(b, steps);
        cudaEventRecord(e1, b->stream);
        if (rs != LAT_OK || cudaEventSynchronize(e1) != cudaSuccess) { st = LAT_ECUDA; break; }
        BatchCtl ctl;
        cudaMemcpy(&ctl, b->dctl, sizeof(ctl), cudaMemcpyDeviceToHost);
        if (ctl.status != LAT_OK) { st = (lat_status)ctl.status; break; }
        float ms = 0.0f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (!best.threads || ms < best_ms) {
            best = cands[c];
            best_ms = ms;
        }
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    // restore
    for (int l = 0; l < nl; l++) {
        lat_handle* h = b->h[l];
        if (!save[l]) continue;
        for (int i = 0; i < 8; i++)
            cudaMemcpyAsync(h->buf[i], (char*)save[l] + i * h->nsites * h->esize, h->nsites * h->esize,
                            cudaMemcpyDeviceToDevice, b->stream);
        cudaMemcpyAsync(h->sc, &ssave[l], sizeof(DevScalars), cudaMemcpyHostToDevice, b->stream);
    }
    if (cudaStreamSynchronize(b->stream) != cudaSuccess && st == LAT_OK) st = LAT_ECUDA;
    for (void* p : save) cudaFree(p);
    if (st != LAT_OK) return st;
    if (!best.threads) return LAT_EUNSUPPORTED;
    {
        std::lock_guard<std::mutex> lock(g_tune_mutex);
        g_tuned[key] = best;
    }
    return configure(b, best.threads, best.tycap, best.depth);
}

} // namespace

extern "C" {

lat_status lat_batch_create(const lat_params* params, int count, void* cuda_stream, lat_batch** out)
{
    if (!out) return LAT_EINVAL;
    *out = nullptr;
    if (!params || count < 1) return LAT_EINVAL;
    for (int i = 1; i < count; i++)
        if (params[i].precision != params[0].precision) return LAT_EINVAL;
    for (int i = 0; i < count; i++)   // the ensemble kernel is written for 7 points and eq. scale
        if (params[i].stencil == 27 || params[i].expansion == 2) return LAT_EUNSUPPORTED;
    lat_batch* b = new (std::nothrow) lat_batch();
    if (!b) return LAT_ENOMEM;
    b->count = count;
    b->prec = params[0].precision;
    b->esize = b->prec == 32 ? 4 : 8;
    b->stream = (cudaStream_t)cuda_stream;
    for (int i = 0; i < count; i++) b->split = b->split || params[i].split != 0;
    lat_status st = LAT_OK;
    for (int i = 0; i < count && st == LAT_OK; i++) {
        lat_handle* h = nullptr;
        st = lat_create(&params[i], cuda_stream, &h);
        if (st == LAT_OK) b->h.push_back(h);
    }
    std::vector<DevScalars*> hsc;
    for (lat_handle* h : b->h) hsc.push_back(h->sc);
    if (st == LAT_OK && (cudaMalloc((void**)&b->dsc, sizeof(DevScalars) * 2 * count) != cudaSuccess ||
                         cudaMalloc((void**)&b->dhsc, sizeof(DevScalars*) * count) != cudaSuccess ||
                         cudaMalloc((void**)&b->dctl, sizeof(BatchCtl)) != cudaSuccess))
        st = LAT_ENOMEM;
    if (st == LAT_OK && (cudaMemcpy(b->dhsc, hsc.data(), sizeof(DevScalars*) * count, cudaMemcpyHostToDevice) != cudaSuccess ||
                         cudaMemset(b->dsc, 0, sizeof(DevScalars) * 2 * count) != cudaSuccess ||
                         cudaMemset(b->dctl, 0, sizeof(BatchCtl)) != cudaSuccess))
        st = LAT_ECUDA;
    if (st == LAT_OK) {
        TunedShape tuned{0, 32, 1};
        {
            std::lock_guard<std::mutex> lock(g_tune_mutex);
            auto it = g_tuned.find(tune_key(b));
            if (it != g_tuned.end()) tuned = it->second;
        }
        if (tuned.threads) st = configure(b, tuned.threads, tuned.tycap, tuned.depth);
        else {
            st = LAT_EUNSUPPORTED;
            for (int t : {256, 512, 384, 640, 768, 1024, 128})
                if ((st = configure(b, t, 32, 1)) == LAT_OK) break;
        }
    }
    if (st != LAT_OK) {
        lat_batch_destroy(b);
        return st;
    }
    *out = b;
    return LAT_OK;
}

lat_status lat_batch_init_fields(lat_batch* b)
{
    if (!b) return LAT_EINVAL;
    for (lat_handle* h : b->h) LAT_TRY(lat_init_fields(h));
    return LAT_OK;
}

lat_status lat_batch_evolve(lat_batch* b, int64_t n_steps)
{
    if (!b || n_steps < 0 || n_steps > 0x7fffffff) return LAT_EINVAL;
    return run_steps(b, n_steps);
}

lat_status lat_batch_sync(lat_batch* b)
{
    if (!b) return LAT_EINVAL;
    LAT_CUDA(cudaStreamSynchronize(b->stream));
    BatchCtl ctl;
    LAT_CUDA(cudaMemcpy(&ctl, b->dctl, sizeof(ctl), cudaMemcpyDeviceToHost));
    if (ctl.status != LAT_OK) return (lat_status)ctl.status;
    for (lat_handle* h : b->h) LAT_TRY(lat_sync(h));
    return LAT_OK;
}

lat_status lat_batch_tune(lat_batch* b, int steps)
{
    if (!b || steps < 1) return LAT_EINVAL;
    return autotune(b, steps);
}

lat_status lat_batch_check_barrier(lat_batch* b, int64_t timeout_ns)
{
    if (!b || timeout_ns < 1000000 || timeout_ns > 2000000000) return LAT_EINVAL;
    LAT_CUDA(cudaStreamSynchronize(b->stream));
    LAT_CUDA(b->prec == 32 ? launch_batch<float>(b, 0, 1u, (unsigned long long)timeout_ns)
                           : launch_batch<double>(b, 0, 1u, (unsigned long long)timeout_ns));
    LAT_CUDA(cudaStreamSynchronize(b->stream));
    BatchCtl ctl;
    LAT_CUDA(cudaMemcpy(&ctl, b->dctl, sizeof(ctl), cudaMemcpyDeviceToHost));
    // the next launch starts from a cleared control word
    LAT_CUDA(cudaMemset(b->dctl, 0, sizeof(BatchCtl)));
    return (lat_status)ctl.status;
}

lat_status lat_batch_tile_heights(lat_batch* b, int32_t* ty)
{
    if (!b || !ty) return LAT_EINVAL;
    for (int i = 0; i < b->count; i++) ty[i] = b->shape.ty[i];
    return LAT_OK;
}

lat_status lat_batch_set_shape(lat_batch* b, int threads, int tycap, int depth)
{
    if (!b || threads < 32 || threads > 1024 || tycap < 1 || tycap > 32 || depth < 1 || depth > 2) return LAT_EINVAL;
    LAT_CUDA(cudaStreamSynchronize(b->stream));
    BatchShape s;
    if (!shape_for(b, threads, tycap, depth, &s)) return LAT_EUNSUPPORTED;
    return configure(b, threads, tycap, depth);
}

lat_status lat_batch_shape(lat_batch* b, int64_t out[4])
{
    if (!b || !out) return LAT_EINVAL;
    out[0] = b->shape.threads;
    out[1] = b->shape.tycap;
    out[2] = b->shape.depth;
    out[3] = b->shape.blocks;
    return LAT_OK;
}

lat_status lat_batch_member(lat_batch* b, int i, lat_handle** out)
{
    if (!b || !out || i < 0 || i >= b->count) return LAT_EINVAL;
    *out = b->h[i];
    return LAT_OK;
}

lat_status lat_batch_info(lat_batch* b, int64_t out[8])
{
    if (!b || !out) return LAT_EINVAL;
    out[0] = b->shape.blocks;
    out[1] = b->shape.threads;
    out[2] = (int64_t)b->shape.smem;
    out[3] = b->nsegs;
    out[4] = b->captured ? 1 : 0;
    int64_t sites = 0;
    for (lat_handle* h : b->h) sites += (int64_t)h->nsites;
    out[5] = sites;
    out[6] = b->count;
    out[7] = 1;
    return LAT_OK;
}

void lat_batch_destroy(lat_batch* b)
{
    if (!b) return;
    if (b->stream) cudaStreamSynchronize(b->stream);
    else cudaDeviceSynchronize();
    free_tables(b);
    cudaFree(b->dsc); cudaFree(b->dhsc); cudaFree(b->dctl);
    for (lat_handle* h : b->h) lat_destroy(h);
    delete b;
}

} // extern "C"
