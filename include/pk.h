/*
 * pk.h -- C ABI of the GB300 FFT power-spectrum library (libpk.so).
 *
 * The library computes the FFTPower estimator of nbodykit (Hand, Feng et al.,
 * arXiv:1712.05834) on one GPU:
 *
 *   paint     objects -> mesh with a CIC / TSC / PCS window, optionally a
 *             second mesh shifted by half a cell (interlacing)      Sec. 3.3.1-3.3.2
 *   r2c FFT   real mesh -> complex half grid (cuFFT)                Sec. 3.3.1
 *   compensate + interlace: divide by prod_i sinc^p(pi k_i / 2 k_N),
 *             average the two meshes with the half-cell phase       Eq. window-deconvolution
 *   bin       |delta(k)|^2 into k bins, (k, mu) bins about the z axis,
 *             Legendre multipoles l = 0, 2, 4, shot noise removed   Sec. 3.4.1
 *
 * Plain C types only.  Every call returns a pk_status; no call aborts or
 * throws.  A failed call leaves a message retrievable with pk_last_error().
 *
 * Conventions (fixed here because the paper leaves them open):
 *   - mesh node c sits at c * H, H = L / N; positions are wrapped into [0, L);
 *   - axis order (x, y, z) with z fastest in memory; the r2c axis and the line
 *     of sight are both z;
 *   - the interlaced mesh is painted at x + H/2 on all three axes and its
 *     transform multiplied by exp(+i (kx + ky + kz) H / 2) before averaging;
 *   - delta(k) = F~(k) / sum(w); P = L^3 |delta(k)|^2;
 *   - shot noise P_shot = L^3 sum(w^2) / sum(w)^2 (= 1 / nbar for unit weights),
 *     subtracted from P(k), P(k, mu) and P_0 only;
 *   - the DC mode is never binned; the stored half grid carries weight h = 1 on
 *     the l = 0 and l = N/2 planes and h = 2 elsewhere; x, y indices follow
 *     numpy fftfreq;
 *   - k bin b = floor((kF sqrt(m) - kmin) / dk), FP64, kF = (2 pi) / L,
 *     m = i'^2 + j'^2 + l^2; nk = floor((kmax - kmin) / dk); a mode is binned
 *     iff 0 <= b < nk; kmax <= 0 selects k_N = (pi N) / L;
 *   - mu = l / sqrt(m); mu bin q = largest q with q^2 m <= nmu^2 l^2, clamped
 *     to nmu - 1 (edges linspace(0, 1, nmu + 1), lower edge inclusive);
 *   - P_l(k) = (2l + 1) sum h P L_l(mu) / sum h, taken over the 1D k bins.
 */
#ifndef PK_H
#define PK_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct pk_plan_s *pk_plan_t;

typedef enum {
    PK_OK = 0,
    PK_EINVAL = 1,     /* an argument is out of range; nothing was launched    */
    PK_ENOMEM = 2,     /* a device or pinned host allocation failed            */
    PK_ECUDA = 3,      /* a CUDA runtime call failed (message has the string)  */
    PK_ECUFFT = 4,     /* a cuFFT call failed                                  */
    PK_EOVERFLOW = 5,  /* fixed-point paint headroom exceeded: lower the scale */
    PK_ETIMEOUT = 6,   /* a bounded device wait gave up                        */
    PK_ESTATE = 7      /* call out of order (e.g. compute before paint)        */
} pk_status;

typedef enum { PK_CIC = 2, PK_TSC = 3, PK_PCS = 4 } pk_window;   /* value = p */

/* Position layouts accepted by pk_paint. */
typedef enum {
    PK_F32 = 0,    /* n x 3 float, xyz packed (12 bytes per object)             */
    PK_F64 = 1,    /* n x 3 double, xyz packed (24 bytes per object)            */
    PK_F32X4 = 2   /* n x 4 float, xyzw with w the weight; 16-byte aligned      */
} pk_dtype;

/* Mesh / transform precision.  Both paint into int64 fixed point (so the
 * mesh is bit-identical run to run) and form the catalog weight sums in FP64
 * in a fixed order (also bit-identical run to run).
 * PK_MESH_F32: the library's own r2c transform at nmesh 128, 192, 256, 512
 * and 2048 (cuFFT R2C otherwise; see pk_use_own_fft); bins summed per CTA in
 * FP32 with shared-memory atomics, whose order (and so the last bits of
 * P(k)) can vary between runs, then across CTAs in FP64.
 * PK_MESH_F64: cuFFT D2Z; bins summed in FP64. */
typedef enum {
    PK_MESH_F32 = 0,   /* FP32 mesh, FP32 per-mode arithmetic                   */
    PK_MESH_F64 = 1    /* FP64 mesh, cuFFT D2Z, FP64 per-mode arithmetic        */
} pk_precision;

/* How pk_paint deposits the window weights.  Both give int64 fixed-point
 * cells (order-free, bit-identical run to run); they differ only in speed. */
typedef enum {
    PK_PAINT_SORT = 0,     /* tile sort + shared-memory tiles (one global write
                              per cell): the default, fastest on large meshes   */
    PK_PAINT_ATOMIC = 1    /* no sort: 64-bit global atomics into a dense
                              N^3 int64 accumulator per mesh (8 bytes per cell
                              extra), then a conversion pass; can win when the
                              accumulators stay in L2 (small meshes)            */
} pk_paint_variant;

typedef struct {
    double box_size;        /* L > 0                                             */
    int nmesh;              /* N: even, 4 <= N <= 4096                           */
    int window;             /* pk_window                                         */
    int interlaced;         /* 0 / 1                                             */
    int compensated;        /* 0 / 1: divide by prod_i sinc^p                    */
    double kmin;            /* >= 0                                              */
    double kmax;            /* <= 0 selects k_N                                  */
    double dk;              /* > 0                                               */
    int nmu;                /* 0: 1D bins only; >= 1: (k, mu) bins too           */
    unsigned poles_mask;    /* bit0 l=0, bit1 l=2, bit2 l=4                      */
    int los_axis;           /* must be 2 (z)                                     */
    int precision;          /* pk_precision                                      */
    int subtract_shot;      /* 0 / 1                                             */
    int fixed_scale_log2;   /* S: one weight unit = 2^S; 0 selects 22 (FP32 mesh)
                               or 32 (FP64 mesh); 1..40                          */
    int batch;              /* catalogs per plan (separate meshes); 0 -> 1       */
    int tile;               /* paint tile edge in cells; 0 -> automatic          */
    int paint_variant;      /* pk_paint_variant                                  */
    int64_t capacity;       /* objects per paint call to reserve at plan time so
                               that pk_paint never allocates or waits (16 bytes
                               of device memory per object for the tile sort);
                               0 -> the first paint reserves what it needs       */
} pk_config;

/* Result of one catalog.  All pointers are host memory owned by the plan and
 * stay valid until the next pk_compute or pk_destroy on that plan.  Arrays
 * of length nk * nmu are row-major [k bin][mu bin].  Empty bins hold NaN. */
typedef struct {
    int nk, nmu, npoles;          /* npoles = 3: rows l = 0, 2, 4                 */
    const double *k_edges;        /* nk + 1                                       */
    const double *mu_edges;       /* nmu + 1 (NULL if nmu == 0)                   */
    const double *k_mean;         /* nk: mode-weighted mean |k| per k bin         */
    const double *pk;             /* nk: P(k), shot noise removed if requested    */
    const double *poles;          /* 3 * nk: P_0, P_2, P_4 (rows not in the mask
                                     are NaN)                                      */
    const uint64_t *modes;        /* nk: weighted mode counts (full-grid count)   */
    const double *k_mean2d;       /* nk * nmu                                     */
    const double *mu_mean2d;      /* nk * nmu                                     */
    const double *pkmu;           /* nk * nmu: P(k, mu)                           */
    const uint64_t *modes2d;      /* nk * nmu                                     */
    double shot_noise;            /* L^3 sum(w^2) / sum(w)^2                      */
    double wsum, w2sum;           /* sum(w), sum(w^2) of the painted objects      */
} pk_result_view;

/* Fill *cfg with defaults: L = 1000, N = 256, CIC, not interlaced, compensated,
 * kmin = 0, kmax = k_N, dk = 2 kF, nmu = 0, all poles, z line of sight, FP32
 * mesh, shot noise subtracted, S automatic, batch 1, automatic tile, the
 * sort paint variant, no reserved capacity. */
void pk_config_default(pk_config *cfg);

/* Create a plan: the setup of the paper's to_mesh(Nmesh, BoxSize, window,
 * interlaced, compensated) and FFTPower(mode, dk, kmin, Nmu, poles, los)
 * options (Sec. 3.3.2 "From Catalog to Mesh", Sec. 3.4.1 "Power Spectra");
 * the paper's algorithms run at construction and keep their
 * results as attributes (Sec. 2.3.3), which this split into plan / paint /
 * compute / result mirrors.  Validates cfg, allocates the meshes (in-place r2c layout,
 * N x N x 2(N/2+1) reals per mesh, (1 + interlaced) meshes per catalog), the
 * cuFFT plan, the bin tables and result buffers, and computes the geometry-only
 * bin data (mode counts, mean k, mean mu) on the device.  All work of the plan
 * is issued on `cuda_stream` (a cudaStream_t; NULL = legacy default stream).
 * The device is the one current at this call.  On success *out owns
 * everything; release it with pk_destroy.
 * Errors: PK_EINVAL (bad config, message says which field), PK_ENOMEM, PK_ECUDA,
 * PK_ECUFFT.  On error *out is NULL and nothing is leaked. */
pk_status pk_plan(const pk_config *cfg, void *cuda_stream, pk_plan_t *out);

/* Paint n objects onto the mesh(es) of catalog 0 (Sec. 3.3.1, Eq. painting:
 * F = [1 + delta'] V with V = 1 and per-object weights W).
 *   pos      n objects in layout `dtype`, device or host memory (host memory is
 *            copied to the device on the plan's stream inside the call);
 *   weights  n floats (device or host) or NULL for unit weights; must be NULL
 *            with PK_F32X4, whose 4th component is the weight;
 *   accumulate 0: the catalog replaces the mesh; 1: it is added (the mesh must
 *            not have been transformed since the last paint).
 * Caller keeps ownership of pos and weights; they are read on the plan's
 * stream and may be reused once the stream has passed this call.  The call
 * does not wait for the GPU unless the objects exceed the capacity reserved
 * so far (cfg->capacity, or the largest earlier call), in which case it
 * synchronizes the stream once and grows the sorted copy.  With device
 * pointers and enough capacity, pk_paint and pk_compute only enqueue work,
 * so a stream capture of them (cudaStreamCaptureModeThreadLocal) records a
 * replayable CUDA graph; the graph re-reads pos, weights and the results
 * buffers in place, so replays see new positions written to the same
 * memory, and pk_result then reads the results of the last replay once the
 * caller has synchronized the stream.
 * Errors: PK_EINVAL (n < 0, bad dtype, misaligned PK_F32X4), PK_ESTATE
 * (accumulate onto a transformed mesh), PK_ENOMEM, PK_ECUDA. */
pk_status pk_paint(pk_plan_t plan, const void *pos, int dtype,
                   const float *weights, int64_t n, int accumulate);

/* Batched paint: catalogs 0 .. nitems-1 of a plan created with batch >= nitems.
 * pos / weights hold the catalogs back to back; offsets (host memory, nitems+1
 * entries, offsets[0] = 0, non-decreasing) delimit them.  Same layout rules,
 * ownership and errors as pk_paint, with accumulate = 0. */
pk_status pk_paint_many(pk_plan_t plan, const void *pos, int dtype,
                        const float *weights, const int64_t *offsets, int nitems);

/* Batched paint of a field value carried by the objects: the painted field is
 * F = [1 + delta'] V (Sec. 3.3.1) with V a per-object value, e.g. a velocity
 * component for the momentum field.  Each object deposits W V (W its weight,
 * 1 if weights is NULL); the normalization keeps sum W, so P = L^3 |F~|^2 /
 * (sum W)^2, and the shot noise is L^3 sum (W V)^2 / (sum W)^2.  values: n
 * floats, device or host, in the order of pos.  Otherwise as pk_paint_many.
 * Errors: as pk_paint_many, and PK_EINVAL for NULL values with objects. */
pk_status pk_paint_values(pk_plan_t plan, const void *pos, int dtype, const float *weights,
                          const float *values, const int64_t *offsets, int nitems);

/* Transform, compensate, interlace and bin every painted catalog of the plan
 * (Sec. 3.4.1 with Eq. window-deconvolution).  Asynchronous on the plan's
 * stream; the results are copied to plan-owned host memory and become
 * readable through pk_result.  Errors: PK_ESTATE (a catalog is not painted),
 * PK_ECUFFT, PK_ECUDA. */
pk_status pk_compute(pk_plan_t plan);

/* Wait for the last pk_compute and describe catalog `item`'s result: the
 * FFTPower attributes of Sec. 3.4.1 (P(k), P(k, mu), multipoles P_l, the bin
 * edges, mean k and mu, mode counts) plus the shot noise that was
 * subtracted.  The view's pointers are plan-owned host memory, valid until
 * the next pk_compute or pk_destroy.
 * Errors: PK_ESTATE (no compute yet), PK_EINVAL (item out of range),
 * PK_EOVERFLOW (fixed-point headroom exceeded while painting), PK_ECUDA. */
pk_status pk_result(pk_plan_t plan, int item, pk_result_view *out);

/* Cross power spectrum of catalogs item_a and item_b of the last pk_compute
 * (their transforms are still held by the plan): each stored mode contributes
 * P = L^3 Re(delta_a conj(delta_b)), delta formed for each catalog as in
 * pk_compute (interlacing combine, compensation, division by its own sum of
 * weights), binned in the same k, (k, mu) bins and multipoles.  Cross powers of
 * two fields painted from the same volume -- two tracers, or a density and a
 * momentum field (Sec. 3.3.1, V(x) a velocity component) -- carry no shot
 * noise term; none is subtracted.  item_a == item_b gives the auto power
 * without shot-noise subtraction.  Asynchronous on the plan's stream; read the
 * result with pk_cross_result.  Valid until the next pk_paint.
 * Errors: PK_ESTATE (no pk_compute since the last paint), PK_EINVAL (item out
 * of range), PK_ECUDA. */
pk_status pk_cross(pk_plan_t plan, int item_a, int item_b);

/* Wait for the last pk_cross and describe its result (same layout as
 * pk_result; shot_noise = 0, wsum = sum of catalog a's weights, w2sum = sum of
 * catalog b's weights).  The pointers stay valid until the next pk_cross or
 * pk_destroy.  Errors: PK_ESTATE (no pk_cross yet), PK_EOVERFLOW, PK_ECUDA. */
pk_status pk_cross_result(pk_plan_t plan, pk_result_view *out);

/* Power spectrum of the field projected onto one or two axes (the
 * ProjectedFFTPower of Sec. 3.4.1, e.g. for Lyman-alpha or lensing-like
 * projected fields).  The painted field summed over the dropped axes has, by
 * the projection-slice theorem, the transform of the 3D field at index 0 along
 * them, so the plan's transform of catalog `item` (after pk_compute) already
 * holds it.  Each mode of that plane or line: interlacing combine and
 * compensation as in pk_compute, P = L^d |F~|^2 / (sum w)^2 with d the number
 * of kept axes, every mode of the full d-dimensional grid counted once, binned
 * in |k| with the plan's k bins; the shot noise L^d sum w^2 / (sum w)^2 is
 * subtracted if the plan's subtract_shot is set.  keep_axes: bit 0 x, bit 1 y,
 * bit 2 z; one or two bits.  The call waits for the result; the pointers in
 * *out stay valid until the next pk_projected or pk_destroy.
 * Errors: PK_EINVAL (keep_axes, item), PK_ESTATE (no pk_compute since the last
 * paint), PK_ECUDA. */
typedef struct {
    int nk, ndim;                 /* k bins; d = number of kept axes               */
    const double *k_edges;        /* nk + 1                                       */
    const double *k_mean;         /* nk: mean |k| of the bin's modes              */
    const double *pk;             /* nk: projected power                          */
    const uint64_t *modes;        /* nk: modes of the d-dimensional grid          */
    double shot_noise;            /* L^d sum(w^2) / sum(w)^2                      */
    double wsum;                  /* sum(w)                                       */
} pk_projected_view;

pk_status pk_projected(pk_plan_t plan, int item, unsigned keep_axes, pk_projected_view *out);

/* Copy painted mesh `mesh` (0, or 1 = the interlaced mesh) of catalog `item`
 * into dst as a dense N x N x N array (z fastest) of the plan's precision
 * (float for PK_MESH_F32, double for PK_MESH_F64): the painted field F of
 * Sec. 3.3.1, in units of the object weights.  dst may be host or device
 * memory of at least N^3 elements; the call waits for the copy.  Valid between
 * a paint and the next pk_compute.  Errors: PK_ESTATE (mesh already
 * transformed or never painted), PK_EINVAL (item / mesh out of range), PK_ECUDA. */
pk_status pk_mesh(pk_plan_t plan, int item, int mesh, void *dst);

/* Choose the 3D r2c transform of pk_compute (the Fourier transform of the
 * painted field, Sec. 3.3.1; the binning it feeds, Sec. 3.4.1).  on = 1: the
 * library's own FFT kernels -- length-N complex FFTs along y and x of the mesh
 * with each z row read as N/2 complex pairs (d[2n] + i d[2n+1], in place),
 * then one pass that takes the length-N/2 FFTs along z, splits the packed
 * transform into the r2c transform and bins it without writing it.  on = 0:
 * cuFFT's in-place R2C, then the bin pass.  Both give the same result within
 * FP32 rounding.  It applies to the FP32 mesh form with nmesh 128, 192, 256,
 * 512, 1024 or 2048 and is the default at all but 1024 (where cuFFT measured
 * faster).  After a compute with it, pk_cross
 * and pk_projected first write the r2c transform into the meshes (one extra
 * pass).  Takes effect at the next pk_compute.
 * Errors: PK_EINVAL (on = 1 where the own transform does not apply). */
pk_status pk_use_own_fft(pk_plan_t plan, int on);

/* Stages whose device time pk_stage_times reports. */
typedef enum {
    PK_STAGE_SORT = 0,    /* tile count + scan + scatter (pk_paint)             */
    PK_STAGE_PAINT = 1,   /* shared-memory tile paint (pk_paint)                */
    PK_STAGE_FFT = 2,     /* r2c of every mesh: cuFFT, or the own y and x passes */
    PK_STAGE_BIN = 3,     /* compensate + interlace + bin (own transform: with   */
                          /* the z FFTs and the r2c split)                       */
    PK_STAGE_FINAL = 4,   /* histogram reduce + normalize + multipoles          */
    PK_NSTAGES = 5
} pk_stage;

/* Turn per-stage timing on (1) or off (0).  When on, pk_paint and pk_compute
 * record CUDA events on the plan's stream around each stage.  No effect on
 * results. */
pk_status pk_enable_timing(pk_plan_t plan, int on);

/* Device milliseconds of each stage (PK_NSTAGES doubles) of the last pk_paint
 * and pk_compute with timing on; waits for those events.  Stages not run are
 * 0.  Errors: PK_ESTATE (timing off), PK_ECUDA. */
pk_status pk_stage_times(pk_plan_t plan, double *ms);

/* Number of the library's own kernels launched on this plan since pk_plan
 * (plan-time geometry kernels included; cuFFT's kernels and memsets not). */
long long pk_launch_count(pk_plan_t plan);

/* Binning with no device allocation.  The paper has no counterpart: this
 * entry point exists for callers that cannot call cudaMalloc (code running
 * while a framework captures a stream into a CUDA graph and owns all memory,
 * programs whose device memory is handed out by a pool they do not control,
 * hosts that forbid allocation after start-up).  It runs the same fused
 * compensate + interlace + bin kernel as pk_compute on transforms the caller
 * already holds, with every piece of scratch (per-CTA histograms and the
 * compensation, phase and k-edge tables) in one fixed array of about 5.4 MB
 * compiled into the library (so every GPU that loads the library holds it
 * until the process exits).
 *   cfg     geometry and binning as for pk_plan; precision must be PK_MESH_F32,
 *           nmesh <= 4096, and nk * max(nmu, 1) + 2 nk <= 8192 (else PK_EINVAL);
 *   mesh    device pointer, N x N x (N/2+1) complex64 (interleaved re, im),
 *           the r2c transform of the painted mesh, 16-byte aligned;
 *   mesh2   the same for the interlaced mesh (required iff cfg->interlaced);
 *   sums    device pointer to nh doubles, overwritten: for nmu > 0, slots
 *           [0, nk*nmu) hold sum h |d|^2 of (k, mu) bin b*nmu+q, else slots
 *           [0, nk) hold sum h |d|^2 of k bin b; if cfg->poles_mask asks for
 *           l = 2 or 4, the next nk slots hold sum h |d|^2 L_2(mu) and the
 *           nk after them sum h |d|^2 L_4(mu) (L_2 = (3 mu^2 - 1) / 2,
 *           L_4 = (35 mu^4 - 30 mu^2 + 3) / 8).  d is the compensated (and
 *           interlace-combined) transform, not yet divided by sum(w): the
 *           power of a bin is L^3 sum / (sum(w)^2 * mode count);
 *   cuda_stream  the stream to run on; the call only enqueues work;
 *   err, errlen  optional buffer for a message on failure (may be NULL).
 * The first call on a device looks up the scratch array's device address
 * (with that device current); make that first call before any stream capture.
 * All calls share the one array: calls that overlap on the GPU (other streams
 * or host threads) race and must be serialized by the caller.  Nothing in it
 * needs to start at zero: every call rewrites what it later reads.
 * Errors: PK_EINVAL (sizes beyond the limits above, NULL or misaligned
 * pointers), PK_ECUDA. */
pk_status pk_bin_static(const pk_config *cfg, const void *mesh, const void *mesh2, double *sums,
                        void *cuda_stream, char *err, size_t errlen);

/* ---- Log-normal mock catalogs on the device ----
 * The LogNormalCatalog source that the paper's tests and benchmarks paint
 * (Sec. 3.2), over its Gaussian linear field, so that mock -> P(k) runs
 * wholly on the GPU.  One draw with seed s:
 *   1. white noise W on the ngrid^3 grid: Philox4x64-10 (Salmon et al.,
 *      SC'11) with key (s, 0); cells 4b .. 4b+3 (flat index, z fastest) use the
 *      four words of counter (b, 0, 0, 0) as two Box-Muller pairs, each word
 *      mapped to the uniform ((w >> 40) + 1/2) 2^-24;
 *   2. G~ = FFT(W) sqrt(A k^slope ngrid^3 / L^3) (DC removed), G = IFFT(G~)
 *      normalized by 1 / ngrid^3: a Gaussian field of power A k^slope;
 *   3. 1 + delta = exp(G - sigma^2 / 2), sigma^2 the grid variance of G,
 *      held as integer cell weights round(2^30 (1 + delta));
 *   4. exactly n objects (key (s, 1), counter (i, 0, 0, 0) for object i): the
 *      cell by inverse CDF of t = floor(w0 total / 2^64) over the exact
 *      integer prefix sums, a uniform offset inside the cell from w1..w3;
 *   5. z += f_rsd psi_z(cell) with psi~_z = i k_z / k^2 G~ (the linear
 *      displacement; its DC and z-Nyquist plane set to zero), wrapped into
 *      [0, L).
 * A draw depends only on (cfg, seed, n), not on the launch configuration. */
typedef struct pk_lognormal_s *pk_lognormal_t;

typedef struct {
    double box_size;        /* L > 0                                              */
    int ngrid;              /* field grid: even, 4 <= ngrid <= 2048               */
    double slope;           /* P(k) = amp k^slope                                 */
    double amp;             /* > 0: the amplitude; <= 0: chosen so that the grid
                               variance (1 / L^3) sum_{k != 0} P(k) = variance   */
    double variance;        /* used when amp <= 0; > 0                            */
    double f_rsd;           /* z displacement factor (linear RSD); 0: none        */
} pk_lognormal_config;

/* Create a generator: validates cfg, allocates the grid buffers (about 16 +
 * 8 (f_rsd != 0) bytes per cell, 16 bytes per cell for the weights and their
 * prefix sums) and the cuFFT plans; all its work runs on `cuda_stream`.
 * Errors: PK_EINVAL (bad cfg; message through pk_plan_error), PK_ENOMEM,
 * PK_ECUDA, PK_ECUFFT.  On error *out is NULL. */
pk_status pk_lognormal_plan(const pk_lognormal_config *cfg, void *cuda_stream, pk_lognormal_t *out);

/* The Gaussian linear field G of seed `seed` (steps 1-2) into `field`: a dense
 * ngrid^3 float array (z fastest), device or host memory.  Asynchronous on the
 * generator's stream for device memory.  Errors: PK_EINVAL, PK_ECUDA, PK_ECUFFT. */
pk_status pk_lognormal_field(pk_lognormal_t gen, uint64_t seed, float *field);

/* Draw n objects of seed `seed` into `pos`: n x 3 float (x, y, z), device
 * memory, in [0, L) (the layout PK_F32 of pk_paint).  Asynchronous on the
 * generator's stream; `pos` is written when the stream passes the call.
 * Errors: PK_EINVAL (n < 0, NULL pos), PK_ECUDA, PK_ECUFFT. */
pk_status pk_lognormal_draw(pk_lognormal_t gen, uint64_t seed, int64_t n, float *pos);

/* The amplitude A in use (the given one, or the one set from `variance`). */
double pk_lognormal_amp(pk_lognormal_t gen);

/* Number of the library's own kernels this generator has launched. */
long long pk_lognormal_launch_count(pk_lognormal_t gen);

/* Message of the last failed call on this generator ("" if none). */
const char *pk_lognormal_error(pk_lognormal_t gen);

/* Free the generator (waits for its stream).  NULL is a no-op. */
pk_status pk_lognormal_destroy(pk_lognormal_t gen);

/* ---- Survey multipoles (ConvolvedFFTPower, Sec. 3.4.1) ----
 * Power-spectrum multipoles of survey data (positions as right ascension,
 * declination and redshift, or observer-frame Cartesian), with the line of
 * sight from the observer to each point.  The paper names the estimator by
 * reference (the FFT-based estimator of Hand et al. 2017, 2l + 1 FFTs for
 * multipole l, after Bianchi et al. 2015, Scoccimarro 2015, Feldman, Kaiser &
 * Peacock 1994 and Yamamoto et al. 2006).  What the library computes:
 *   w      = w_comp w_fkp per object; w_fkp = 1 / (1 + nbar P0) when the
 *            config's p0_fkp > 0, else the given column (NULL = 1);
 *   alpha  = sum_data w_comp / sum_randoms w_comp;
 *   F      = painted data - alpha painted randoms, on the mesh whose node c
 *            sits at box_origin + c H (observer frame, observer at 0); with
 *            interlacing the two meshes are combined in Fourier space as in
 *            pk_compute and transformed back to one real field;
 *   A_0    = FFT[F];  A_l(k) = (4 pi / (2l + 1)) sum_m Y_lm(k^) FFT[F Y_lm(x^)](k)
 *            with the real spherical harmonics Y_lm (pk_survey_ylm) and x^
 *            the unit vector of node c (a node at the observer contributes to
 *            A_0 only); by the addition theorem A_l is the sum over nodes of
 *            F exp(-i k.x) L_l(k^.x^) (the phase of box_origin dropped);
 *   P_l(k) = (2l + 1) / I < Re[A_l A_0^*] / W^2(k) >_bin - [l = 0] S, with the
 *            k bins, mode weights and window W(k) of pk_compute,
 *            I = alpha sum_randoms nbar w_comp w_fkp^2 and
 *            S = (sum_data w^2 + alpha^2 sum_randoms w^2) / I.
 * Distances for sky input: flat LambdaCDM without radiation,
 * chi(z) = (c / H0) int_0^z dz' / sqrt(Om (1 + z')^3 + 1 - Om) in Mpc/h with
 * c / H0 = 2997.92458 Mpc/h; x = chi (cos Dec cos RA, cos Dec sin RA, sin Dec),
 * RA and Dec in degrees.  The library tabulates chi and its derivative at
 * 8192 redshifts in [0, zmax] (FP64 on the host) and interpolates with cubic
 * Hermite polynomials in FP64 on the device. */
typedef struct pk_survey_s *pk_survey_t;

typedef enum {
    PK_COORD_CARTESIAN = 0,   /* x, y, z in Mpc/h, observer at the origin         */
    PK_COORD_SKY = 1          /* RA (deg), Dec (deg), redshift z                  */
} pk_coord;

typedef struct {
    double box_size;        /* L > 0: edge of the cubic mesh box (Mpc/h)         */
    double box_origin[3];   /* observer-frame position of mesh node (0, 0, 0)    */
    int nmesh;              /* N: even, 4 <= N <= 4096                           */
    int window;             /* pk_window                                         */
    int interlaced;         /* 0 / 1                                             */
    int compensated;        /* 0 / 1                                             */
    double kmin, kmax, dk;  /* k bins as in pk_config (kmax <= 0 selects k_N)    */
    unsigned poles_mask;    /* bit0 l=0, bit1 l=2, bit2 l=4 (l = 0 always runs)  */
    int precision;          /* pk_precision                                      */
    int subtract_shot;      /* 0 / 1: subtract S from P_0                        */
    double omega_m;         /* matter density for PK_COORD_SKY, in (0, 1]; 0 when
                               only Cartesian input is used                      */
    double zmax;            /* largest redshift of the distance table (sky input);
                               0 selects 5                                      */
    double p0_fkp;          /* > 0: w_fkp = 1 / (1 + nbar P0); 0: given w_fkp    */
    int max_batch;          /* Y_lm-weighted meshes held at once (one weighting
                               pass and one bin pass per batch); 0: as many as
                               fit in half the free device memory                */
    int64_t capacity;       /* data + randoms objects to reserve (0: on demand)  */
} pk_survey_config;

/* One catalog for pk_survey_paint.  pos: n x 3 in the layout of `dtype`
 * (PK_F32 or PK_F64): (x, y, z) for PK_COORD_CARTESIAN, (RA, Dec, z) for
 * PK_COORD_SKY.  Columns are float arrays of n (device or host memory, like
 * pos); NULL columns are 1.  nbar (the mean number density at the object) is
 * required for the randoms and, when p0_fkp > 0, for the data. */
typedef struct {
    const void *pos;
    int dtype;              /* pk_dtype: PK_F32 or PK_F64                        */
    int coord;              /* pk_coord                                          */
    const float *wcomp;     /* completeness weights                              */
    const float *wfkp;      /* FKP weights (ignored when p0_fkp > 0)             */
    const float *nbar;      /* n(z) at each object                               */
    int64_t n;              /* >= 0                                              */
} pk_survey_catalog;

/* Fill *cfg with defaults: L = 1000, origin (0, 0, 0), N = 256, CIC, not
 * interlaced, compensated, kmin = 0, kmax = k_N, dk = 2 kF, l = 0, 2, 4, FP32
 * mesh, shot noise subtracted, Om = 0.31, zmax = 5, given FKP weights,
 * automatic batch, no reserved capacity. */
void pk_survey_config_default(pk_survey_config *cfg);

/* Create a survey plan: validates cfg, allocates two catalogs' meshes, the
 * A_0 transform, the Y_lm-weighted meshes of one batch and the cuFFT plans,
 * tabulates chi(z) when omega_m > 0, and computes the mode counts and mean k
 * of the k bins.  All work runs on `cuda_stream`.  Errors: PK_EINVAL
 * (message through pk_plan_error), PK_ENOMEM, PK_ECUDA, PK_ECUFFT; on error
 * *out is NULL. */
pk_status pk_survey_plan(const pk_survey_config *cfg, void *cuda_stream, pk_survey_t *out);

/* Convert (sky input) and paint the data and randoms: each object becomes
 * box-frame (x - box_origin, w) (FP32; FP64 positions for FP64 meshes), the
 * catalog sums of alpha, I and S are taken in FP64, and both catalogs are
 * painted into their own meshes
 * (int64 fixed point, as pk_paint).  randoms == NULL keeps the randoms
 * painted by the previous call (mocks that share one random catalog).
 * With no data objects alpha and I are 0 and every P_l is NaN.
 * Objects outside the box wrap periodically and are counted in n_outside;
 * sky objects with z outside [0, zmax] (or NaN) get weight 0 and are counted
 * in n_rejected.  Asynchronous on the plan's stream; host arrays are copied
 * first.  Errors: PK_EINVAL (dtype, coord, missing nbar, sky input without
 * omega_m, NULL pos with n > 0), PK_ESTATE (randoms == NULL before any
 * randoms), PK_ENOMEM, PK_ECUDA. */
pk_status pk_survey_paint(pk_survey_t plan, const pk_survey_catalog *data, const pk_survey_catalog *randoms);

/* Run the estimator on the painted catalogs: the FKP combination, the
 * interlacing round trip (interlaced plans), 1 + 5 [l=2] + 9 [l=4] r2c
 * transforms, the binning of A_0 and of every Y_lm-weighted transform, and
 * the normalization.  Asynchronous; pk_survey_result waits.  Errors:
 * PK_ESTATE (nothing painted), PK_ECUDA, PK_ECUFFT. */
pk_status pk_survey_compute(pk_survey_t plan);

typedef struct {
    int nk, npoles;               /* npoles = 3: rows l = 0, 2, 4                 */
    const double *k_edges;        /* nk + 1                                       */
    const double *k_mean;         /* nk                                           */
    const double *poles;          /* 3 * nk: P_0, P_2, P_4 (rows not asked: NaN;
                                     empty bins: NaN)                              */
    const uint64_t *modes;        /* nk                                           */
    double alpha, norm, shot_noise;
    double data_wsum, randoms_wsum;        /* sum w_comp                          */
    double data_w2sum, randoms_w2sum;      /* sum (w_comp w_fkp)^2                */
    double randoms_nsum;                   /* sum nbar w_comp w_fkp^2             */
    int64_t n_data, n_randoms;
    int64_t n_outside;            /* objects outside the box (wrapped)            */
    int64_t n_rejected;           /* sky objects with z outside [0, zmax]         */
} pk_survey_result_view;

/* Wait for the last pk_survey_compute and describe its result; the pointers
 * stay valid until the next compute or destroy.  Errors: PK_ESTATE (no
 * compute), PK_ECUDA. */
pk_status pk_survey_result(pk_survey_t plan, pk_survey_result_view *out);

/* Real spherical harmonic Y_lm of the unit vector (x, y, z), l = 2 or 4,
 * |m| <= l, orthonormal on the sphere (the functions the survey path
 * evaluates on the device, here in FP64 on the host); NaN for other (l, m). */
double pk_survey_ylm(int l, int m, double x, double y, double z);

/* Bounding box of a catalog's observer-frame Cartesian positions (sky input
 * converted exactly as pk_survey_paint converts it; sky objects with z
 * outside [0, zmax] or NaN are skipped), so that the mesh box can be chosen
 * to enclose the randoms before a survey plan exists.  omega_m and zmax as in
 * pk_survey_config (used for PK_COORD_SKY only; zmax 0 selects 5).  Runs on
 * `cuda_stream` and waits for the result; lo / hi receive the minimum and
 * maximum per axis (+inf / -inf when no object counts).  Host arrays are
 * copied first.  Errors: PK_EINVAL (NULL cat / lo / hi, dtype, coord, sky
 * input without omega_m in (0, 1]), PK_ENOMEM, PK_ECUDA. */
pk_status pk_survey_bounds(const pk_survey_catalog *cat, double omega_m, double zmax, void *cuda_stream,
                           double *lo, double *hi);

/* Stages whose device time pk_survey_stage_times reports. */
typedef enum {
    PK_SURVEY_STAGE_PREP = 0,    /* catalog conversion + sums (pk_survey_paint)     */
    PK_SURVEY_STAGE_PAINT = 1,   /* tile sort + paint of both catalogs              */
    PK_SURVEY_STAGE_FFT = 2,     /* every cuFFT call of pk_survey_compute           */
    PK_SURVEY_STAGE_FIELD = 3,   /* FKP combine, interlacing, Y_lm weighting         */
    PK_SURVEY_STAGE_BIN = 4,     /* per-mode sums of A_0 and the Y_lm transforms     */
    PK_SURVEY_STAGE_FINAL = 5,   /* row reduce + normalization                      */
    PK_SURVEY_NSTAGES = 6
} pk_survey_stage;

/* Turn per-stage timing on (1) or off (0): CUDA events around each stage of
 * pk_survey_paint and pk_survey_compute on the plan's stream.  No effect on
 * results. */
pk_status pk_survey_enable_timing(pk_survey_t plan, int on);

/* Device milliseconds per stage (PK_SURVEY_NSTAGES doubles) of the last
 * timed paint and compute; waits for their events.  Errors: PK_ESTATE
 * (timing off), PK_ECUDA. */
pk_status pk_survey_stage_times(pk_survey_t plan, double *ms);

/* Number of the library's own kernels launched on this survey plan. */
long long pk_survey_launch_count(pk_survey_t plan);

/* Message of the last failed call on this survey plan ("" if none). */
const char *pk_survey_error(pk_survey_t plan);

/* Free the survey plan (waits for its stream).  NULL is a no-op. */
pk_status pk_survey_destroy(pk_survey_t plan);

/* Free everything the plan owns (waits for its stream): the end of the
 * algorithm object of Sec. 2.3.3, whose results the caller has read through
 * pk_result.  NULL is a no-op. */
pk_status pk_destroy(pk_plan_t plan);

/* Static string naming a status. */
const char *pk_status_string(pk_status status);

/* Message of the last failed call on this plan ("" if none).  Valid until the
 * next call on the plan. */
const char *pk_last_error(pk_plan_t plan);

/* Message of the last failed pk_plan on this thread ("" if none). */
const char *pk_plan_error(void);

#ifdef __cplusplus
}
#endif

#endif /* PK_H */
