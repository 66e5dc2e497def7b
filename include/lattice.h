/*
 * lattice.h -- C ABI of the GB300 lattice library: staggered-leapfrog evolution
 * of two interacting scalar fields (phi, chi) on a periodic N^3 lattice in an
 * expanding FRW universe, after J. Sainio, "CUDAEASY - a GPU Accelerated
 * Cosmological Lattice Program" (arXiv:0911.5692).
 *
 * Conventions for every entry point:
 *   - Every call returns lat_status; nothing is thrown across the ABI.
 *   - A handle is bound to the CUDA stream given at creation and is not
 *     thread-safe. Calls that launch work are asynchronous on that stream
 *     unless they say they synchronise.
 *   - Errors detected on the device (non-finite sums, a failed scale-factor
 *     solve, a wait that ran out of time) are sticky: the step kernels turn
 *     into no-ops and the error is returned by the next synchronising call
 *     (lat_energies, lat_sync, lat_get_scalars, lat_get_state).
 *   - Arrays are SoA, one array per field and per quantity, x fastest:
 *     element (x, y, z) is at ((z * n) + y) * n + x. Element type is float for
 *     precision 32 and double for precision 64.
 *   - Storage times follow the staggered leapfrog (Sec. II.B, eq. evo and the
 *     half-step desynchronisation after initialisation): fields f and the scale
 *     factor a live at t + dt/2, momenta f' and a' at t.
 *   - All quantities are in program units (Sec. II.B): f = A a^r phi,
 *     x_pr = B x, dt_pr = B a^s dt, with s - 2r + 3 = 0.
 */
#ifndef LATTICE_H
#define LATTICE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lat_handle lat_handle;

typedef enum {
    LAT_OK = 0,
    LAT_EINVAL = 1,       /* bad argument or parameter set */
    LAT_ECFL = 2,         /* dt too large for the stencil and masses */
    LAT_ENOMEM = 3,       /* device or host allocation failed */
    LAT_ECUDA = 4,        /* a CUDA runtime or library call failed */
    LAT_ENONFINITE = 5,   /* non-finite sums or no real root for a' (sticky) */
    LAT_ETIMEOUT = 6,     /* a bounded device wait ran out (sticky) */
    LAT_EUNSUPPORTED = 7, /* valid request the library does not serve */
    LAT_ESTATE = 8        /* call not valid in the handle's current state */
} lat_status;

/* Potentials, Sec. III and the lambda phi^4 lineage it compares with. */
enum {
    LAT_MODEL_LPHI4 = 0,  /* V = lambda/4 phi^4 + g2/2 phi^2 chi^2 */
    LAT_MODEL_M2PHI2 = 1  /* V = m^2/2 phi^2   + g2/2 phi^2 chi^2 */
};

typedef struct {
    int32_t n;            /* lattice side N (N^3 sites); 4 <= N <= 1024, N % 4 == 0 */
    int32_t precision;    /* 32 or 64: storage and arithmetic of fields and momenta */
    int32_t model;        /* LAT_MODEL_* */
    int32_t expansion;    /* 0: static space (a = 1, a' = 0); 1: FRW, eq. scale;
                             2: FRW through L = 1/H (lat_get_hubble_length) */
    double L;             /* box side, program units; dx = L / N */
    double dt;            /* time step, program units */
    double lambda, m, g2; /* physical couplings (Planck units fixed by eight_pi_G) */
    double phi0[2];       /* homogeneous phi, chi at t = 0 (physical) */
    double dphi0[2];      /* their physical-time derivatives */
    double eight_pi_G;    /* 1: reduced Planck units; 8 pi: non-reduced */
    double A, B, r, s;    /* rescaling; all four zero: derived from the dominant
                             term as in Sec. II.B (A = 1/phi0, B = sqrt(cpl)
                             phi0^(beta/2-1), r = 6/(2+beta), s = 3(2-beta)/(2+beta)) */
    double kcut;          /* initial fluctuations cut above |n| > kcut (units of
                             2 pi / L); 0: N/4 */
    double fluct;         /* multiplier on the vacuum fluctuation amplitude (1 = vacuum) */
    uint64_t seed;        /* seed of the counter-based generator for the initial state */
    int32_t stencil;      /* Laplacian (Sec. II.C): 0 or 7 = 7-point (LATTICEEASY);
                             27 = the 27-point stencil of Patra and Karttunen over
                             the 3x3x3 cube, weights 14/30 (6 faces), 3/30 (12
                             edges), 1/30 (8 corners), -128/30 (centre), in 1/dx^2 */
    int32_t split;        /* 0: every array holds its field whole. 1: the inflaton phi
                             (field 0) is stored as an FP64 homogeneous mode (its value
                             at the field time and momentum at the momentum time,
                             lat_get_background) plus arrays of the fluctuation about
                             it, the homogeneous initial values of Sec. II.B's initial
                             conditions evolved in FP64 and the vacuum fluctuations in
                             the arrays, so that FP32 arrays resolve fluctuations far
                             below FP32 precision of phi itself. The leapfrog is the
                             same step in exact arithmetic. chi is always stored whole.
                             The derivative (lat_vjp, lat_adjoint) returns
                             LAT_EUNSUPPORTED on a split lattice. */
} lat_params;

/* Volume averages at the field time, in physical units (Sec. II.B, eq. rho-pres;
 * residual curvature and w as in Sec. III). kin, grad and pot are the kinetic,
 * gradient and potential parts of rho (rho = sum kin + sum grad + pot); mean and
 * var are of the program-unit fields. */
typedef struct {
    double t, a, ad, H, rho, p, w, curv_resid;
    double kin[2], grad[2], pot, mean[2], var[2];
} lat_energy_report;

/* Create a lattice on `cuda_stream` (a cudaStream_t; NULL = legacy default
 * stream) with library-owned device buffers (8 arrays of N^3 elements: f and
 * f' of both fields, twice for the leapfrog's ping-pong). Validates the
 * parameters and the stability bound of the leapfrog (LAT_ECFL when
 * dt^2 (k_max^2 + m_eff^2) > 4 at the initial state, with k_max^2 the
 * stencil's largest lattice frequency squared: 12/dx^2 for 7 points, 92/(15 dx^2)
 * for 27). The fields start at zero; call lat_init_fields or lat_set_state.
 * A 27-point lattice runs on the plane-ring step kernel only (variant 2 of
 * lat_set_kernel). On error *out is NULL. */
lat_status lat_create(const lat_params* params, void* cuda_stream, lat_handle** out);

/* As lat_create, with caller-owned device buffers (e.g. torch tensors):
 * dev_bufs[0..7] = f_phi, f_chi, pi_phi, pi_chi of ping-pong set 0, then the
 * same four of set 1. Each holds N^3 elements of the chosen precision, 16-byte
 * aligned. They must outlive the handle; lat_destroy does not free them. */
lat_status lat_create_with_buffers(const lat_params* params, void* cuda_stream,
                                   void* const dev_bufs[8], lat_handle** out);

/* DEFROST-style initial conditions (Sec. II.B, last paragraph): homogeneous
 * values from params plus Gaussian vacuum fluctuations of every field and
 * momentum (white noise from Philox-4x32-10 keyed by the seed, filtered in
 * Fourier space to |f_k|^2 = 1/(2 w_k), |f'_k|^2 = w_k/2, w_k^2 = k_lat^2 +
 * m_eff^2, k_lat^2 = -L(k) the symbol of the configured stencil), converted to program units (f = A a^r phi, f' = (A/B) a^(r-s) phidot
 * + r (a'/a) f), then the fields and a advanced by dt/2. Runs on the device with
 * temporary buffers; synchronises the stream. */
lat_status lat_init_fields(lat_handle* h);

/* Advance n_steps leapfrog steps (Sec. II.B, eq. evo with eq. scalar-evo and
 * eq. scale). Each step is one fused kernel: the configured Laplacian (7- or
 * 27-point), potential derivative, kick and drift of both fields, the
 * <|grad f|^2> and <V> sums of
 * the new fields, and (in its last block) the FP64 scale-factor update that sets
 * the coefficients of the next step. Asynchronous; no host synchronisation.
 * n_steps >= 0. */
lat_status lat_evolve(lat_handle* h, int64_t n_steps);

/* Energy density, pressure, w, H, residual curvature, per-field kinetic /
 * gradient / potential parts, means and variances at the field time (Sec. II.B,
 * eq. rho-pres; Sec. III). Momenta at the field time are the average of those
 * at t and t + dt. Synchronises; returns a sticky device error if one is set. */
lat_status lat_energies(lat_handle* h, lat_energy_report* out);

/* Energy density and pressure at every site: eq. rho-pres of Sec. II.B evaluated
 * per site, the quantities of the paper's second kernel (Sec. II.C), which it
 * writes out every few hundred steps for visualisation.
 *   rho_dev, p_dev: device arrays of N^3 elements of the handle's precision,
 *     layout of lat_get_state, caller-owned; written with rho(x) and p(x) in the
 *     units of lat_energies (physical), at the field time.
 * Per site: the kinetic terms with the momenta at the field time, the potential,
 * and a gradient energy equal to half the weighted squared differences to all
 * the site's stencil neighbours (each neighbour pair shared evenly by its two
 * sites), so that the volume means of rho_dev and p_dev are lat_energies' rho
 * and p. Arithmetic in the handle's precision. Asynchronous on the handle's
 * stream (no host synchronisation). LAT_EINVAL for null or misaligned pointers,
 * LAT_ESTATE on a slab. */
lat_status lat_energy_field(lat_handle* h, void* rho_dev, void* p_dev);

/* Shell-binned power spectrum of field `field` (0 = phi, 1 = chi), the
 * diagnostic Sec. IV names as future work: bin b = round(|n|), n the integer
 * wave vector; p_out[b] = shell mean of |F_k|^2 / N^3 (F the forward DFT),
 * k_out[b] = shell mean of 2 pi |n| / L, count_out[b] = modes in the shell.
 * Host arrays of nbins entries, 1 <= nbins <= 4096. Synchronises. */
lat_status lat_spectrum(lat_handle* h, int field, int nbins, double* k_out, double* p_out,
                        int64_t* count_out);

/* Copy one array out: field 0/1, what 0 = f (at t + dt/2), 1 = f' (at t), each
 * whole (for phi of a split lattice: the homogeneous mode plus the stored
 * fluctuation, rounded to the handle's precision); what 2 = f, 3 = f' as stored
 * (for phi of a split lattice the fluctuation about lat_get_background's values,
 * else the same as 0 and 1). dst holds N^3 elements of the handle's precision, on
 * the device if dst_is_device, else host memory (pinned or pageable).
 * Synchronises. */
lat_status lat_get_state(lat_handle* h, int field, int what, void* dst, int dst_is_device);

/* Copy one array in (layout and `what` as lat_get_state: 0, 1 whole, from which
 * the current homogeneous mode is subtracted on a split lattice; 2, 3 as stored).
 * The sums and scale-factor coefficients are recomputed before the next step or
 * diagnostic. */
lat_status lat_set_state(lat_handle* h, int field, int what, const void* src, int src_is_device);

/* Upload the whole state in one call: src[0..3] = f_phi, f_chi, pi_phi, pi_chi
 * as stored (lat_get_state's what 2 and 3: on a split lattice phi and its
 * momentum are the fluctuations about lat_get_background's values; device memory
 * if src_is_device, else host memory). The step parity is read from the device
 * first (one small synchronous read); then the four copies are queued on the
 * handle's stream after the work already there, and the call returns without
 * waiting for them. Host sources should be page-locked for the copies to run
 * asynchronously and must stay unchanged until the stream has passed them (the
 * next synchronising call or lat_sync). The sums and coefficients are recomputed
 * before the next step or diagnostic. LAT_EINVAL for a null pointer. */
lat_status lat_upload_state(lat_handle* h, const void* const src[4], int src_is_device);

/* The counterpart of lat_upload_state: the four stored arrays of the current
 * state into dst[0..3] (f_phi, f_chi, pi_phi, pi_chi as stored; device memory if
 * dst_is_device, else host memory, page-locked for the copies to overlap),
 * queued on the handle's stream after the work already there; then waits for
 * them. Returns a sticky device error if one is set. LAT_EINVAL for a null
 * pointer. */
lat_status lat_download_state(lat_handle* h, void* const dst[4], int dst_is_device);

/* No counterpart in the paper: where the state that the step of Sec. II.B
 * reads and writes lies in memory. Where to put the eight state arrays
 * (f_phi, f_chi, pi_phi, pi_chi of set 0,
 * then of set 1; array_bytes each) in one allocation of *total_bytes bytes:
 * offsets[k] (host, bytes from its start, multiples of 128; the allocation
 * itself 16-byte aligned at least). The library lays out the buffers it
 * allocates itself this way, and lat_create_with_buffers callers should too:
 * the arrays are read and written at the same site index at once, and starts
 * that are equal modulo 2 KB (power-of-two arrays placed one after another)
 * make those accesses meet in the same memory partitions (the 512^3 FP32 step:
 * 0.79 against 0.73 ms). LAT_EINVAL for null pointers or array_bytes of 0 or
 * above 2^40. */
lat_status lat_buffer_layout(uint64_t array_bytes, uint64_t offsets[8], uint64_t* total_bytes);

/* Evolve a state held in host memory: n_steps times, upload host[0..3] (the
 * four stored arrays, as lat_upload_state takes them), take one step (the sums
 * of the uploaded fields, then the fused step of Sec. II.B) and download the
 * evolved arrays back into host[0..3] (as lat_download_state gives them). The
 * copies run in `chunks` z-ranges of planes (0: 16; at most 64 and N) on two
 * streams of the call's own, one per direction: chunk c of a step's upload
 * waits only for chunk c of the previous step's download (the same host
 * bytes), so a step's download and the next step's upload share the host link
 * in both directions. host[k] must be page-locked (LAT_EINVAL otherwise:
 * cudaHostAlloc or cudaHostRegister memory) and must not be touched until the
 * call returns. scalars_out (host, may be NULL): n_steps rows of the eight
 * values of lat_get_scalars after each step. Queued after the work already on
 * the handle's stream; waits for everything it queued before returning the
 * first error, or a sticky device error. LAT_EINVAL for null pointers, n_steps
 * < 0 or chunks out of range; LAT_ESTATE on a slab. */
lat_status lat_evolve_host(lat_handle* h, void* const host[4], int64_t n_steps, int chunks, double* scalars_out);

/* The homogeneous inflaton mode of split storage (lat_params.split = 1), in
 * program units: out[0] = its value P at the field time t + dt/2, out[1] = its
 * momentum at t. Zero on a lattice that stores phi whole. Synchronises. */
lat_status lat_get_background(lat_handle* h, double out[2]);

/* Move the homogeneous mode of a split lattice to in[0] (field time) and in[1]
 * (momentum time) without changing the state: the stored fluctuation arrays of
 * phi and its momentum are shifted by the differences (in FP64, rounded once).
 * LAT_ESTATE unless split = 1; LAT_EINVAL for non-finite values. */
lat_status lat_set_background(lat_handle* h, const double in[2]);

/* Move the homogeneous mode of a split lattice to the volume means of phi and of
 * its momentum (FP64 reductions on the device), so that the stored fluctuations
 * have zero mean; used after loading whole fields with lat_set_state.
 * Synchronises. LAT_ESTATE unless split = 1. */
lat_status lat_recenter(lat_handle* h);

/* Scalars: out[0] = t (time of the momenta), out[1] = a (at t + dt/2),
 * out[2] = a' (at t), out[3] = step count, out[4..7] = the volume averages
 * <|grad f_phi|^2>, <|grad f_chi|^2>, <f_phi^beta/beta>, <f_phi^2 f_chi^2/2> at the
 * field time, where <|grad f|^2> = -<f L f> for the configured Laplacian L (the
 * forward-difference sum for 7 points; the weighted sum over the 13 neighbour
 * pairs of each site for 27). Synchronises; returns a sticky device error if one
 * is set. */
lat_status lat_get_scalars(lat_handle* h, double out[8]);

/* Set t, a (at t + dt/2), a' (at t) and the step count from in[0..3]; the sums
 * and coefficients are recomputed before the next step. With expansion = 2 the
 * Hubble length l at t is set to a_t / a' with a_t = a - (dt/2) a'; LAT_EINVAL
 * there for a' = 0. */
lat_status lat_set_scalars(lat_handle* h, const double in[4]);

/* The L = 1/H form of the scale-factor update (expansion = 2; Sec. II.B notes
 * that DEFROST evolves L = 1/H first and a from it, so that no gradient average
 * enters, and prints no equation for it). In program time, with h = a'/a and
 * the Hubble length l = 1/h (physical L = a^(-s) l / B), the acceleration
 * equation a-double-dot/a = -(4 pi G/3)(rho + 3p), rho + 3p = 2 sum phidot^2 - 2V,
 * gives
 *   l' = (s + 1) + Gamma l^2,   a' = a / l,   a''/a = -s h^2 - Gamma,
 *   Gamma = (8 pi G / (3 A^2)) a^(-2r) (sum_i <(f_i' - r h f_i)^2> - <V_pr>),
 * and the f coefficient of eq. scalar-evo becomes r(2 - r) h^2 - r Gamma. l is
 * stored at the momentum time t (with a'), a at the field time. A step solves
 * the implicit midpoint equations for l_{n+1} and that coefficient, with the
 * momenta at the field time taken as the mean of the kick's two ends, then sets
 * a_{n+3/2} = a_{n+1/2} exp(dt / l_{n+1}); the a' reported after it is
 * (a_{n+3/2} - a_{n+1/2}) / dt. The L form does not impose the Friedmann
 * constraint: an initial mismatch is carried as spatial curvature
 * K = a^2 (H^2 - 8 pi G rho / 3), which it conserves. It cannot pass a = const
 * (H = 0, l infinite): a recollapsing lattice raises LAT_ENONFINITE there. Each
 * step takes one extra read-only pass over the four state arrays (its sums
 * need the Laplacian of the fields at the field time).
 * lat_get_hubble_length writes l at t (Synchronises); lat_set_hubble_length
 * sets it (after lat_set_scalars, which derives it from a and a'). Both return
 * LAT_ESTATE unless expansion = 2; set: LAT_EINVAL for l = 0 or not finite. */
lat_status lat_get_hubble_length(lat_handle* h, double* ell);
lat_status lat_set_hubble_length(lat_handle* h, double ell);

/* Wait for the handle's stream; return a sticky device error if one is set. */
lat_status lat_sync(lat_handle* h);

/* Checkpoint and resume (the paper has none; LATTICEEASY-style runs are long).
 * A checkpoint is a host blob: a header with the parameters, the FP64 scalar
 * block exactly as the device holds it (t, a, a', the sums and coefficients of
 * the next step) and the four state arrays. Loading it into a handle created
 * with the same parameters continues bit-identically to an uninterrupted run.
 * lat_checkpoint_bytes gives the blob size; save and load synchronise and
 * return LAT_EINVAL on a size or parameter mismatch. */
lat_status lat_checkpoint_bytes(lat_handle* h, uint64_t* bytes);
lat_status lat_save_checkpoint(lat_handle* h, void* dst, uint64_t bytes);
lat_status lat_load_checkpoint(lat_handle* h, const void* src, uint64_t bytes);

/* Choose the step kernel (all compute the same step): variant 0 = automatic
 * (FP32 lattices with N = 256, 512 or 1024: 5; otherwise 4 where a row is 128 or
 * more 16-byte vectors, FP32 N >= 512 or FP64 N >= 256, else 2 where it fits,
 * else 4), 2 = z-march through a shared-memory plane ring over full x rows,
 * filled by per-thread asynchronous copies, 4 = the same ring over x tiles of
 * at most 32 (or 16) 16-byte vectors with taller y tiles, 5 = x tiles exactly
 * 32 vectors wide (one warp per row) with N, ty and depth compiled in (FP32 N =
 * 256, 512, 1024 with ty 16; FP64 N = 256, 512 with ty 16 and depth 1) and one
 * warp that handles the tile's x neighbours (4 and 5: 7-point only);
 * ty = owned rows per tile, zr = planes per z-chunk, depth = planes prefetched
 * ahead, 0 = automatic. LAT_EINVAL for another variant; LAT_EUNSUPPORTED if the
 * variant cannot run this lattice (a 27-point lattice runs on variant 2 only;
 * ty, zr and depth apply to it as above). */
lat_status lat_set_kernel(lat_handle* h, int variant, int ty, int zr, int depth);

/* Autotune the step kernel (the paper finds its block size by trial and error,
 * Sec. II.C, keeping 256 computing threads after trying 64, 128 and 256,
 * Sec. III):
 * time `steps` steps (1 <= steps <= 100000, after a warm-up of 32 that also
 * captures the graph) for every kernel shape that can run this lattice --
 * variants 2, 4 and 5 over tile heights and prefetch depths (the 27-point
 * stencil: variant 2 over tile heights and depths) -- on the lattice's own
 * state, which is saved before and put back after every candidate and at the
 * end; keep the fastest, and remember it for the process per (N, precision,
 * stencil, split storage, expansion), so that handles created later with the
 * same key start with it. out (host, 8 entries, may be NULL): the chosen
 * variant, ty, zr, depth, the number of candidates timed, the best and the
 * slowest time per step in ns, and the blocks per step. Synchronises. Returns
 * a sticky device error if a candidate raised one (the previous kernel is kept). */
lat_status lat_tune(lat_handle* h, int steps, int64_t out[8]);

/* Launch geometry of the current step kernel: out[0] = variant, out[1] = blocks
 * per step, out[2] = threads per block, out[3] = dynamic shared memory bytes,
 * out[4] = kernels launched per step, out[5] = ty, out[6] = zr, out[7] = depth. */
lat_status lat_kernel_info(lat_handle* h, int64_t out[8]);

/* Volume sums of two field arrays without allocating device memory. The paper
 * has no counterpart; this is for callers that cannot call cudaMalloc (device
 * memory already reserved by another allocator such as a framework's caching
 * pool, a fixed memory budget, or code that cannot take cudaMalloc's implicit
 * device-wide synchronisation).
 * f_phi, f_chi: device arrays of n^3 elements (float for precision 32, double
 * for 64), layout as in lat_get_state, holding the fields whole; model:
 * LAT_MODEL_*; L: box side. Writes to out_dev (device, 4 doubles, caller-owned)
 * the averages <|grad f_phi|^2>, <|grad f_chi|^2> (forward differences / dx^2),
 * <f_phi^beta/beta> and <f_phi^2 f_chi^2 / 2> in FP64 arithmetic: the averages
 * lat_get_scalars reports in out[4..7] for a handle holding these fields with the
 * 7-point stencil (equal to FP64 rounding for FP64 fields; a handle with FP32
 * fields forms them in FP32 with compensated per-thread sums, within about 1e-7
 * relative). The gradient average of the 27-point stencil is not served here.
 * Asynchronous on cuda_stream (a cudaStream_t; NULL = legacy default stream).
 * Scratch: one static device array per GPU (about 33 KB, the same for every n,
 * held by every GPU that loads the library until the process exits); it calls no
 * cudaMalloc, cudaFree or allocating library routine. The first call on a device
 * looks the array up with cudaGetSymbolAddress and clears it, synchronously; make
 * that first call before any stream capture. The address is kept for the life of
 * the process, so do not use this entry point across a device reset
 * (cudaDeviceReset). Every call shares the array, so calls that overlap on the
 * GPU (different streams or threads without ordering) race: they may give wrong
 * sums or leave out_dev unwritten. Errors: LAT_EINVAL for null pointers, n < 4,
 * precision other than 32 or 64, an unknown model or L <= 0; LAT_EUNSUPPORTED for
 * n > 1024 (the lattice sides the library serves, the range this entry point is
 * tested over); LAT_ECUDA if the set-up or launch fails. */
lat_status lat_field_sums_static(const void* f_phi, const void* f_chi, int n, int precision, int model, double L,
                                 double* out_dev, void* cuda_stream);

/* Change the coupling g^2 of an existing handle (Sec. II.B: it enters the
 * program-unit potential as kappa0 = g^2 / (A^2 B^2)); the state is kept and the
 * next step's coefficients are recomputed. LAT_EINVAL for g2 < 0 or not finite,
 * LAT_ECFL if the new effective mass breaks the leapfrog stability bound. */
lat_status lat_set_g2(lat_handle* h, double g2);

/* Reverse-mode derivative (vector-Jacobian product) of n_steps leapfrog steps
 * (Sec. II.B, eq. evo with eq. scalar-evo and eq. scale) from the handle's
 * current state, exact for the discrete scheme: it includes the dependence of
 * a'', the field-equation coefficients and every later step on the volume sums
 * of gradient and potential energy (eq. scale). The paper has no derivative;
 * this is the differentiation the reference method is extended with.
 *   fbar_dev, pibar_dev: device arrays of 2 n^3 elements each (phi block then
 *     chi block, layout of lat_get_state, element type of the handle), caller-
 *     owned. In: the adjoint of f and pi after n_steps. Out: the adjoint of f and
 *     pi of the starting state.
 *   sbar[4]: in: sbar[0], sbar[1] = adjoint of a and a' after n_steps; out:
 *     sbar[0], sbar[1] = adjoint of the starting a and a', sbar[2] = derivative
 *     with respect to kappa0, sbar[3] = with respect to g^2.
 *   ckpt_every: steps between stored checkpoints; 0 = ceil(sqrt(n_steps)). The
 *     forward pass stores one checkpoint (three field pairs) per ckpt_every
 *     steps, the reverse pass recomputes each segment into ckpt_every field
 *     pairs; device memory grows as (3 n_steps / ckpt_every + 2 ckpt_every + 8)
 *     arrays.
 * The handle ends at the state after n_steps (as after lat_evolve).
 * Synchronises. LAT_ENOMEM if the checkpoints do not fit; LAT_EUNSUPPORTED for
 * a 27-point lattice, expansion = 2 or split storage; sticky device errors of the
 * forward or reverse pass are returned. */
lat_status lat_vjp(lat_handle* h, int64_t n_steps, int64_t ckpt_every, void* fbar_dev, void* pibar_dev,
                   double sbar[4]);

/* Value and gradient of an observable of the state after n_steps with respect
 * to the starting f, pi and g^2, by lat_vjp. observable 0: J = <chi^2>, the
 * volume mean of the squared program-unit chi (f_1). observable 1: the fraction
 * of the energy density in chi, eq. rho-pres's terms at the momentum time t of
 * the final state (fields and a taken back half a step: f_t = f - (dt/2) pi,
 * a_t = a - (dt/2) a', h = a'/a_t): J = (K_chi + G_chi) / (K_phi + K_chi + G_phi +
 * G_chi + <V_pr>) with K_i = <(pi_i - r h f_t,i)^2>/2 and G_i = a_t^(-2s-2)
 * <|grad+ f_t,i|^2>/2 (the physical factor cancels; the interaction energy counts
 * in the total only, so J also depends on g^2 directly, which dJ/dg^2 includes).
 * J_out (host, may be NULL)
 * gets J; dJ_dg2 (host, may be NULL) gets dJ/dg^2; dJ_df_dev and dJ_dpi_dev
 * (device, 2 n^3 elements each, as in lat_vjp) get dJ/df and dJ/dpi of the
 * starting state. n_steps = 0 gives J and its gradient at the current state.
 * LAT_EUNSUPPORTED for any other observable. Synchronises. */
lat_status lat_adjoint(lat_handle* h, int64_t n_steps, int observable, int64_t ckpt_every, double* J_out,
                       double* dJ_dg2, void* dJ_df_dev, void* dJ_dpi_dev);

/* ---- One lattice split into z-slabs (one slab per GPU; the paper leaves
 * multi-GPU runs as future work, Sec. IV). A slab handle owns planes
 * [z0, z0 + nzl) of the N^3 lattice described by params (n = N). Its eight
 * caller-owned device arrays (same order as lat_create_with_buffers) hold
 * nzl + 3 planes of N^2 elements each: stored plane p is global plane
 * z0 - 1 + p (mod N), so p = 0 is the halo below, 1..nzl the owned planes,
 * nzl + 1 and nzl + 2 the halos above. One step of the whole lattice is, on
 * every slab: (1) the caller fills the halos of the current ping-pong set
 * (set = step & 1): f_phi and f_chi planes 0, nzl + 1, nzl + 2 and pi_phi,
 * pi_chi plane nzl + 1 from the neighbouring slabs; (2) lat_slab_step; (3) the
 * caller adds the four shares of every slab (an allreduce); (4)
 * lat_slab_advance(advance = 1) with the total. Before the first step (and
 * after any state upload): halos, lat_slab_sums, allreduce,
 * lat_slab_advance(advance = 0). lat_get_state / lat_set_state /
 * lat_get_scalars / lat_set_scalars act on the slab's stored arrays; the
 * whole-lattice calls (evolve, init, energies, spectrum, checkpoints,
 * derivative, set_kernel) return LAT_ESTATE on a slab. nzl >= 2.
 * LAT_EUNSUPPORTED for a 27-point lattice or expansion = 2. */
lat_status lat_slab_create(const lat_params* params, int z0, int nzl, void* cuda_stream, void* const dev_bufs[8],
                           lat_handle** out);

/* Shares of the four volume averages of the slab's current fields (sums over
 * its owned sites / N^3, in the order of lat_get_scalars out[4..7]) into
 * sums_dev (device, 4 doubles). Needs the halos above. Asynchronous. */
lat_status lat_slab_sums(lat_handle* h, double* sums_dev);

/* The fused step on the owned planes (reads the current set including its
 * halos, writes the other set) and the shares of the averages of the new
 * fields into sums_dev (device, 4 doubles). Asynchronous. */
lat_status lat_slab_step(lat_handle* h, double* sums_dev);

/* The fused step on owned planes [zfirst, zfirst + zcount) only (0 <= zfirst,
 * 1 <= zcount, zfirst + zcount <= nzl), with the shares of those planes'
 * averages into sums_dev (device, 4 doubles); lat_slab_step is the range
 * [0, nzl). The step of a range reads the current set's planes zfirst - 1 ..
 * zfirst + zcount + 1 (owned z, stored z + 1) and the momenta of zfirst ..
 * zfirst + zcount: planes 2 .. nzl - 3 touch no halo plane, so the caller can
 * step them while the halo exchange is in flight and planes 0, 1, nzl - 2,
 * nzl - 1 after it. Ranges of one step run one after another on the slab's
 * stream (they share its block partials); the caller adds their shares.
 * Asynchronous. */
lat_status lat_slab_step_range(lat_handle* h, int zfirst, int zcount, double* sums_dev);

/* The FP64 scale-factor update (eq. scale) from the total of all slabs'
 * shares (sums_dev: device, 4 doubles): advance = 1 after a step (a, a', t and
 * the step count advance), 0 to set the coefficients of the first step.
 * Asynchronous. */
lat_status lat_slab_advance(lat_handle* h, const double* sums_dev, int advance);

/* Step (2) -- the fused step of Sec. II.B, eq. evo with eq. scalar-evo, and the
 * sums of the new fields for eq. scale -- for slabs of one lattice held by one
 * process (one GPU), in one
 * launch on the stream of slabs[0]: `ranges` holds nranges triples (slab
 * index into slabs[], first owned plane, plane count) of owned-plane ranges,
 * each under the conditions of lat_slab_step_range (the halos it reads are in
 * place), and sums_dev (device, 4 doubles) receives the sum of their shares.
 * The slabs' scalar blocks must agree (they do when every step ends with
 * lat_slab_advance_local); the coefficients are read from slabs[0]'s. The
 * caller orders the other slabs' streams against slabs[0]'s. 1 <= nslabs <= 8,
 * 1 <= nranges <= 16. LAT_EINVAL for null pointers, counts out of range, a
 * range outside its slab or slabs of different lattices; LAT_ESTATE for a
 * handle that is not a slab; LAT_EUNSUPPORTED for lattice sides without a
 * compiled warp-tile slab kernel (N = 256 or 512 in FP32, 256 in FP64), where
 * each range is stepped by lat_slab_step_range instead. Asynchronous. */
lat_status lat_slab_step_ranges(lat_handle* const* slabs, int nslabs, const int32_t* ranges, int nranges,
                                double* sums_dev);

/* Steps (3) and (4) above (the volume averages of Sec. II.B and the
 * scale-factor update of eq. scale) for slabs of one lattice held by one process (one
 * GPU), in one launch on the stream of slabs[0]: the nshares share vectors
 * (device pointers, 4 doubles each; a slab's whole-step share or its range
 * shares) are added in the order given, and every slab's scalars advance
 * with that total, as lat_slab_advance would. The caller orders the other
 * slabs' streams against slabs[0]'s (the shares written before the call, the
 * next step after it). 1 <= nslabs <= 64, 1 <= nshares <= 192. LAT_EINVAL for
 * null pointers, counts out of range or slabs of different lattices (side,
 * precision, model, expansion, dt or L differ), LAT_ESTATE for a handle that
 * is not a slab. Asynchronous. */
lat_status lat_slab_advance_local(lat_handle* const* slabs, int nslabs, const double* const* shares, int nshares,
                                  int advance);

/* No counterpart in the paper, whose program runs one lattice on one GPU
 * (Sec. II.C; several GPUs are its future work, Sec. IV). Copy `count` device
 * regions of `bytes` bytes each (src[i] to dst[i]; the
 * regions must not overlap) in one launch per 64 regions on cuda_stream: the
 * halo exchange of slabs that one process holds. Every pointer and `bytes`
 * must be multiples of 16 bytes (a plane of an even-sided lattice is), else
 * LAT_EINVAL; null arrays or pointers and count < 0 are LAT_EINVAL too.
 * count = 0 or bytes = 0 copies nothing. Asynchronous. */
lat_status lat_copy_regions(void* const* dst, const void* const* src, int count, uint64_t bytes, void* cuda_stream);

/* ---- Ensembles: independent lattices of uneven size and coupling stepped
 * together by one persistent launch. The paper evolves one lattice at a time
 * (Sec. II.C); every member here follows the same step (Sec. II.B, eq. evo with
 * eq. scalar-evo and eq. scale) with its own N, dt, couplings and a(t). */
typedef struct lat_batch lat_batch;

/* Create `count` members from params[0..count-1] (all of one precision; each
 * member owns its buffers), bound to cuda_stream. The launch shape comes from
 * the process's autotuner cache for this set of sizes and precision, else a
 * default. LAT_EINVAL for mixed precisions or a bad member (its lat_create
 * status is returned), LAT_EUNSUPPORTED if a member size fits no block shape or
 * a member has the 27-point stencil or expansion = 2. */
lat_status lat_batch_create(const lat_params* params, int count, void* cuda_stream, lat_batch** out);

/* lat_init_fields on every member (each with its own seed). Synchronises. */
lat_status lat_batch_init_fields(lat_batch* b);

/* Advance every member by n_steps (0 <= n_steps < 2^31) in one cooperative
 * launch (every block resident; the runtime refuses the launch otherwise),
 * captured in a CUDA graph per step count. Between steps the blocks meet at a
 * grid barrier whose waits are bounded by the global timer: a wait that runs out
 * makes every block leave and lat_batch_sync return LAT_ETIMEOUT. Asynchronous. */
lat_status lat_batch_evolve(lat_batch* b, int64_t n_steps);

/* Wait for the stream; return the first sticky error of the launch or of a
 * member. */
lat_status lat_batch_sync(lat_batch* b);

/* Autotune the launch shape: time `steps` steps for each candidate of block
 * size (128 .. 1024), tile-height cap (32, 16, 8, 4; each member takes the
 * largest tile height up to the cap that divides its side and fits the block)
 * and prefetch depth (1 or 2 planes in flight ahead of the computed one) on the
 * ensemble itself, keep the fastest and cache it for this process per (sizes,
 * precision); ensembles created later with the same sizes and precision start
 * with it. Member states are saved before and restored after. Synchronises. */
lat_status lat_batch_tune(lat_batch* b, int steps);

/* The tile height (y rows per work unit) each member is stepped with:
 * ty (host, one int32 per member, in creation order). */
lat_status lat_batch_tile_heights(lat_batch* b, int32_t* ty);

/* The launch shape in use (the block shape the paper picks by trial, Sec. II.C
 * and Sec. III, here chosen by lat_batch_tune): out (host) = threads per
 * block, tile-height cap, prefetch depth, blocks. */
lat_status lat_batch_shape(lat_batch* b, int64_t out[4]);

/* Step with the given shape from now on (the paper fixes its block shape by
 * hand, Sec. II.C): threads per block (32 .. 1024),
 * tile-height cap (1 .. 32) and prefetch depth (1 or 2); the values are those
 * lat_batch_tune sweeps. LAT_EINVAL out of those ranges, LAT_EUNSUPPORTED if
 * some member's tile does not fit the block or the shared memory. Waits for the
 * stream first; the member states are not touched. */
lat_status lat_batch_set_shape(lat_batch* b, int threads, int tycap, int depth);

/* Self-test of the bounded grid barrier (failure detection without a fault):
 * launches the ensemble kernel so that its barrier waits for one block more
 * than the launch has; every block's wait runs out after timeout_ns
 * (1 ms .. 2 s) and the call returns LAT_ETIMEOUT with the context still
 * usable. Member states are not touched. Synchronises. */
lat_status lat_batch_check_barrier(lat_batch* b, int64_t timeout_ns);

/* Borrow member i's handle (owned by the batch; do not destroy it) for state
 * access, energies, spectra or checkpoints. Do not evolve it on its own while
 * batch work is in flight. */
lat_status lat_batch_member(lat_batch* b, int i, lat_handle** out);

/* Launch shape: out[0] = blocks, out[1] = threads per block, out[2] = dynamic
 * shared memory bytes, out[3] = work ranges, out[4] = 1 if the last evolve ran
 * as a captured graph, out[5] = total sites, out[6] = members, out[7] = launches
 * per evolve call. */
lat_status lat_batch_info(lat_batch* b, int64_t out[8]);

/* Release the ensemble and its members. NULL is accepted. */
void lat_batch_destroy(lat_batch* b);

/* Release the handle and the buffers it owns. NULL is accepted. */
void lat_destroy(lat_handle* h);

/* Static description of a status code. */
const char* lat_status_string(lat_status st);

#ifdef __cplusplus
}
#endif

#endif /* LATTICE_H */
