// pk_internal.h -- declarations shared by the two translation units of
// libpk.so (host API in pk_api.cu, kernels in pk_kernels.cu).  Not installed.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/pk.h"

namespace pk {

// Message of the last failed plan creation on this thread (pk_plan_error).
void set_plan_error(const char *msg);

// Geometry of the tile-sorted paint (Sec. 3.3.1 painting, Sec. 3.3.2 windows).
// The mesh is cut into cubic tiles of T^3 cells.  Each object is sorted by
// (home tile, boundary class); the paint CTA of a tile gathers its own objects
// and the boundary classes of its 26 neighbours.  Cells [floor(s)+lo,
// floor(s)+hi] along each axis cover the window support on both meshes.
struct PaintGeom {
    float invH;         // N / L in FP32
    float invH_lo;      // N / L - invH (the FP32 rounding residual)
    double invHd;       // N / L in FP64
    int N;              // cells per side
    int T;              // tile edge (divides N, T >= hi - lo)
    int ntx;            // tiles per side = N / T
    int lo, hi;         // reach of the window support relative to floor(s)
    long long ntiles;   // ntx^3 tiles per catalog
};

// Geometry of the fused compensate + interlace + bin pass (Sec. 3.4.1).
struct BinGeom {
    int N, Nh;              // Nh = N/2 + 1 stored z modes
    int nk, nmu;            // k bins, mu bins (nmu = 0: 1D only)
    int twod, poles;        // accumulate (k, mu) sums / mu^2, mu^4 sums
    int hbase;              // first pole slot in the per-CTA histogram
    int nh;                 // histogram length
    float kscale, koff;     // bin estimate: sqrt(m) * kscale - koff
    int mlo, mhi;           // binned modes have mlo <= m < mhi (and m != 0)
    int mu32;               // nmu^2 * max m < 2^32: mu-bin checks in 32 bits
};

struct FinalGeom {
    int nk, nmu, twod, poles, hbase, nh;
    unsigned poles_mask;
    int subtract_shot;
    double L3;              // L^3
    double headroom;        // 2^(62 - S): largest sum |w| with int64 cells safe
    int RL;                 // doubles per item in the result block
};

// Offsets inside one item's FP64 result block.
struct ResultLayout {
    int pk, poles, pkmu, shot, wsum, w2sum, flags, total;
};
ResultLayout result_layout(int nk, int nmu);

// ---- launchers (pk_kernels.cu); all asynchronous on `st` ----
int paint_classes();                  // boundary classes per tile (27)
// dynamic shared memory of one tile-paint CTA painting nmesh meshes
size_t paint_smem_bytes(int T, int window, int nmesh = 2);
size_t scan_tmp_elems(int64_t n);
// dst[0 .. n) = src[0 .. n) for a host array src, through kernel parameters
// (the host array may be reused as soon as the call returns).
cudaError_t launch_upload_i64(int64_t *dst, const int64_t *src, int n, int *launches, cudaStream_t st);
// w: weights (normalization; NULL = 1), vals: painted values V (NULL = 1);
// each object deposits W V and the sums keep sum W, sum (W V)^2, sum |W V|.
cudaError_t launch_sort_count(const void *pos, int dtype, const float *w, const float *vals,
                              const int64_t *item_off, int nitems, int64_t max_n, const PaintGeom &g,
                              uint32_t *count, double *wsums, double *wpart, unsigned *wmax, cudaStream_t st);
// Doubles of the per-block weight-sum rows (wpart) for nitems catalogs.
size_t wsum_partial_elems(int nitems);
cudaError_t launch_scan(const uint32_t *in, int64_t n, uint32_t *out, uint32_t *tmp, int *launches,
                        cudaStream_t st);
cudaError_t launch_scan64(const unsigned long long *in, int64_t n, unsigned long long *out,
                          unsigned long long *tmp, int *launches, cudaStream_t st);
cudaError_t launch_sort_scatter(const void *pos, int dtype, const float *w, const float *vals,
                                const int64_t *item_off, int nitems, int64_t max_n, const PaintGeom &g,
                                const uint32_t *off, uint32_t *count, float4 *sorted, int *err,
                                cudaStream_t st);
cudaError_t launch_paint_tiles(const float4 *sorted, const uint32_t *off, int nitems,
                               const PaintGeom &g, int window, int nmesh, int S, int f64,
                               const unsigned *wmax, int unit_weights, void *mesh,
                               long long item_stride, long long mesh_stride, int accumulate,
                               cudaStream_t st);

// Direct atomic paint into dense int64 accumulators (nitems x nmesh x N^3,
// zero on entry), then conversion into the r2c mesh layout (clears them).
cudaError_t launch_paint_atomic(const void *pos, int dtype, const float *w, const float *vals,
                                const int64_t *item_off, int nitems, int64_t max_n, const PaintGeom &g,
                                int window, int nmesh, int S, unsigned long long *acc, double *wsums,
                                double *wpart, unsigned *wmax, cudaStream_t st);
cudaError_t launch_acc_to_mesh(unsigned long long *acc, int nitems, int nmesh, int N, int S, int f64,
                               void *mesh, long long item_stride, long long mesh_stride, int accumulate,
                               int nsm, cudaStream_t st);

cudaError_t launch_bin(const void *mesh, int f64, int interlaced, long long item_stride_c,
                       long long mesh_stride_c, int nitems, int ctas_per_item,
                       const BinGeom &g, const void *cw, const void *ph, const int *kedge,
                       void *partial, cudaStream_t st);
// Cross power of two catalogs: mesh_a / mesh_b point at each catalog's first
// mesh (the interlaced one follows at mesh_stride_c); one item, `ctas` CTAs.
cudaError_t launch_bin_cross(const void *mesh_a, const void *mesh_b, int f64, int interlaced,
                             long long mesh_stride_c, int ctas, const BinGeom &g, const void *cw,
                             const void *ph, const int *kedge, void *partial, cudaStream_t st);
size_t bin_smem_bytes(const BinGeom &g, int f64);
int bin_ctas_per_sm(const BinGeom &g, int f64);
int bin_threads();
int reduce_chunks(int G);
int reduce_launches(int G);           // k_bin_reduce launches per launch_bin_reduce
cudaError_t launch_bin_reduce(const void *partial, int f64, int G, int nh, int nitems,
                              double *sums2, cudaStream_t st);
cudaError_t launch_finalize(const double *sums2, int G, const unsigned long long *modes1d,
                            const unsigned long long *modes2d, const double *wsums, const int *err,
                            const FinalGeom &f, int nitems, double *res, cudaStream_t st);

cudaError_t launch_finalize_cross(const double *sums2, int G, const unsigned long long *modes1d,
                                  const unsigned long long *modes2d, const double *wsums, const int *err,
                                  const FinalGeom &f, int item_a, int item_b, double *res, cudaStream_t st);

// Projected power: bin the plane / line of one catalog's transform that keeps
// the axes in keep_mask (bit a: axis a); sums[3 b + {0,1,2}] += h, h k, h |F|^2 cw.
cudaError_t launch_plane_bin(const void *m1, const void *m2, int f64, int N, int keep_mask, const void *cw,
                             const void *ph, const int *kedge, int nk, double kF, double *sums, int nsm,
                             cudaStream_t st);

// ---- own FFT path (pk_fft.cu), FP32 meshes with N in {128, 192, 256, 512, 1024, 2048} ----
// The meshes' z rows are read as N/2 complex values (packed real pairs).
bool own_fft_supported(int N);
bool own_fft_default(int N);                      // pk_compute uses it unless told otherwise
void own_fft_twiddles(int N, float *tw);          // tw[2e], tw[2e+1] = W_N^e, e < N
// length-N FFTs along y, then along x, of nmesh packed meshes mesh_c complex apart
cudaError_t launch_fft_xy(void *mesh, int nmesh, long long mesh_c, int N, const void *tw, cudaStream_t st);
// z transform + r2c split + the bin pass of launch_bin (FP32 form), partial
// histograms as launch_bin writes them
cudaError_t launch_zbin(const void *mesh, int interlaced, long long item_stride_c, long long mesh_stride_c,
                        int nitems, int ctas_per_item, const BinGeom &g, const void *cw, const void *ph,
                        const void *tw, const int *kedge, void *partial, cudaStream_t st);
size_t zbin_smem_bytes(const BinGeom &g, int interlaced);
int zbin_ctas_per_sm(const BinGeom &g, int interlaced);
// z transform + r2c split written back in place (the meshes then hold the r2c transform)
cudaError_t launch_zfinish(void *mesh, int interlaced, long long item_stride_c, long long mesh_stride_c,
                           int nitems, int N, const void *tw, int nsm, cudaStream_t st);

cudaError_t launch_geom_hist(const BinGeom &g, unsigned long long *H, unsigned long long *HL,
                             cudaStream_t st);
cudaError_t launch_geom_finalize(const BinGeom &g, const int *kedge, double kF,
                                 const unsigned long long *H, const unsigned long long *HL,
                                 unsigned long long *modes2d, double *kmean2d, double *mumean2d,
                                 cudaStream_t st);

}  // namespace pk
