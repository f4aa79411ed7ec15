// pk_kernels.cu -- sm_103a kernels of the FFT power-spectrum path.
//
//   k_tile_count    pass 1 of the tile counting sort: wrap each object into the
//                   box, find the tiles its window support touches (on both
//                   interlaced meshes), count copies per tile; sum w, w^2, |w|.
//   k_scan_*        exclusive scan of the tile counts (int64 offsets).
//   k_tile_scatter  pass 2: write one float4 (tile-local x, y, z, w) per copy.
//   k_paint_tiles   one CTA per tile: accumulate the window deposits of every
//                   copy in shared memory as int64 fixed point (order-free, so
//                   the mesh is bit-identical run to run), then write the tile
//                   once, coalesced, into the in-place r2c layout.  No global
//                   atomics, no global int64 mesh, no separate convert pass.
//                   Windows: B-splines of order p = 2, 3, 4 (CIC, TSC, PCS),
//                   Sec. 3.3.2; interlacing: second mesh at x + H/2, Sec. 3.3.2.
//   k_bin           fused window compensation (Eq. window-deconvolution),
//                   interlacing combine, |delta|^2, k bin (exact integer edges
//                   in m = |n|^2), mu bin (exact integer rule), Legendre
//                   weights; per-CTA shared-memory histograms, Sec. 3.4.1.
//   k_bin_reduce    fixed-order FP64 sum of the per-CTA histograms.
//   k_finalize      normalization L^3 / (sum w)^2, shot noise, multipoles.
//   k_geom_*        plan-time, geometry-only: exact mode counts per bin and
//                   mean k, mean mu (integer histograms over m, FP64 sums).
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "pk_internal.h"

namespace pk {

namespace {

constexpr int kCountThreads = 256;
constexpr int kPaintThreads = 256;
constexpr int kBinThreads = 256;
constexpr int kBinVec = 4;            // consecutive modes per thread
constexpr int kScanThreads = 1024;
constexpr int kScanPer = 4;           // elements per thread in a scan block
constexpr int kScanTile = kScanThreads * kScanPer;

__device__ __forceinline__ int floordiv(int a, int b) {   // b > 0
    return a >= 0 ? a / b : -((-a + b - 1) / b);
}

__device__ __forceinline__ int wrapmod(int a, int n) {
    int r = a % n;
    return r < 0 ? r + n : r;
}

// Cell coordinate s = x * (N / L) wrapped periodically into [0, N).  Written
// with explicitly rounded intrinsics so that no FMA contraction can differ
// between the count and the scatter kernels: both must see the same s.
__device__ __forceinline__ float wrap_cells(float x, float invH, int N) {
    const float n = (float)N;
    float s = __fmul_rn(x, invH);
    s = __fsub_rn(s, __fmul_rn(n, floorf(__fdiv_rn(s, n))));
    if (s < 0.0f) s = __fadd_rn(s, n);
    if (s >= n) s = __fsub_rn(s, n);
    return s;
}
__device__ __forceinline__ double wrap_cells(double x, double invH, int N) {
    const double n = (double)N;
    double s = __dmul_rn(x, invH);
    s = __dsub_rn(s, __dmul_rn(n, floor(__ddiv_rn(s, n))));
    if (s < 0.0) s = __dadd_rn(s, n);
    if (s >= n) s = __dsub_rn(s, n);
    return s;
}

// One object: cell-unit coordinates in [0, N) and its weight.
template <typename R>
struct Obj {
    R s[3];
    float w;
};

template <int DT>
struct PosReal { using type = float; };
template <>
struct PosReal<PK_F64> { using type = double; };

template <int DT>
__device__ __forceinline__ Obj<typename PosReal<DT>::type> load_obj(const void *pos, const float *w,
                                                                    int64_t i, const PaintGeom &g) {
    using R = typename PosReal<DT>::type;
    Obj<R> o;
    if (DT == PK_F32X4) {
        const float4 v = __ldg(reinterpret_cast<const float4 *>(pos) + i);
        o.s[0] = wrap_cells(v.x, g.invH, g.N);
        o.s[1] = wrap_cells(v.y, g.invH, g.N);
        o.s[2] = wrap_cells(v.z, g.invH, g.N);
        o.w = v.w;
    } else if (DT == PK_F32) {
        const float *p = reinterpret_cast<const float *>(pos) + 3 * i;
        o.s[0] = wrap_cells(__ldg(p + 0), g.invH, g.N);
        o.s[1] = wrap_cells(__ldg(p + 1), g.invH, g.N);
        o.s[2] = wrap_cells(__ldg(p + 2), g.invH, g.N);
        o.w = w ? __ldg(w + i) : 1.0f;
    } else {
        const double *p = reinterpret_cast<const double *>(pos) + 3 * i;
        o.s[0] = (R)wrap_cells(__ldg(p + 0), g.invHd, g.N);
        o.s[1] = (R)wrap_cells(__ldg(p + 1), g.invHd, g.N);
        o.s[2] = (R)wrap_cells(__ldg(p + 2), g.invHd, g.N);
        o.w = w ? __ldg(w + i) : 1.0f;
    }
    return o;
}

// Unwrapped tile indices u0 .. u0 + nu - 1 that cells floor(s)+lo .. floor(s)+hi hit.
template <typename R>
__device__ __forceinline__ void tile_span(R s, const PaintGeom &g, int &u0, int &nu) {
    const int c = (int)floor(s);
    u0 = floordiv(c + g.lo, g.T);
    nu = floordiv(c + g.hi, g.T) - u0 + 1;
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

template <int DT>
__global__ void __launch_bounds__(kCountThreads)
k_tile_count(const void *__restrict__ pos, const float *__restrict__ w,
             const int64_t *__restrict__ item_off, PaintGeom g, uint32_t *__restrict__ count,
             double *__restrict__ wsums) {
    using R = typename PosReal<DT>::type;
    const int item = blockIdx.y;
    const int64_t beg = item_off[item], end = item_off[item + 1];
    uint32_t *cnt = count + (int64_t)item * g.ntiles;
    double sw = 0.0, sw2 = 0.0, swa = 0.0;
    for (int64_t i = beg + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < end;
         i += (int64_t)gridDim.x * blockDim.x) {
        const Obj<R> o = load_obj<DT>(pos, w, i, g);
        int u0[3], nu[3];
        tile_span<R>(o.s[0], g, u0[0], nu[0]);
        tile_span<R>(o.s[1], g, u0[1], nu[1]);
        tile_span<R>(o.s[2], g, u0[2], nu[2]);
        for (int a = 0; a < nu[0]; ++a) {
            const int tx = wrapmod(u0[0] + a, g.ntx);
            for (int b = 0; b < nu[1]; ++b) {
                const int ty = wrapmod(u0[1] + b, g.ntx);
                for (int c = 0; c < nu[2]; ++c) {
                    const int tz = wrapmod(u0[2] + c, g.ntx);
                    atomicAdd(cnt + ((int64_t)tx * g.ntx + ty) * g.ntx + tz, 1u);
                }
            }
        }
        const double wd = (double)o.w;
        sw += wd;
        sw2 += wd * wd;
        swa += fabs(wd);
    }
    __shared__ double red[3][kCountThreads / 32];
    sw = warp_sum(sw);
    sw2 = warp_sum(sw2);
    swa = warp_sum(swa);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) {
        red[0][wid] = sw;
        red[1][wid] = sw2;
        red[2][wid] = swa;
    }
    __syncthreads();
    if (threadIdx.x < 3) {
        double t = 0.0;
        for (int k = 0; k < kCountThreads / 32; ++k) t += red[threadIdx.x][k];
        if (t != 0.0) atomicAdd(wsums + 3 * item + threadIdx.x, t);
    }
}

template <int DT>
__global__ void __launch_bounds__(kCountThreads)
k_tile_scatter(const void *__restrict__ pos, const float *__restrict__ w,
               const int64_t *__restrict__ item_off, PaintGeom g, uint32_t *__restrict__ count,
               const int64_t *__restrict__ off, float4 *__restrict__ sorted, int *__restrict__ err) {
    using R = typename PosReal<DT>::type;
    const int item = blockIdx.y;
    const int64_t beg = item_off[item], end = item_off[item + 1];
    const int64_t tbase = (int64_t)item * g.ntiles;
    for (int64_t i = beg + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < end;
         i += (int64_t)gridDim.x * blockDim.x) {
        const Obj<R> o = load_obj<DT>(pos, w, i, g);
        int u0[3], nu[3];
        tile_span<R>(o.s[0], g, u0[0], nu[0]);
        tile_span<R>(o.s[1], g, u0[1], nu[1]);
        tile_span<R>(o.s[2], g, u0[2], nu[2]);
        for (int a = 0; a < nu[0]; ++a) {
            const int ux = u0[0] + a, tx = wrapmod(ux, g.ntx);
            const float lx = (float)(o.s[0] - (R)(ux * g.T));
            for (int b = 0; b < nu[1]; ++b) {
                const int uy = u0[1] + b, ty = wrapmod(uy, g.ntx);
                const float ly = (float)(o.s[1] - (R)(uy * g.T));
                for (int c = 0; c < nu[2]; ++c) {
                    const int uz = u0[2] + c, tz = wrapmod(uz, g.ntx);
                    const float lz = (float)(o.s[2] - (R)(uz * g.T));
                    const int64_t t = tbase + ((int64_t)tx * g.ntx + ty) * g.ntx + tz;
                    const uint32_t left = atomicSub(count + t, 1u);
                    if (left == 0u) {              // more copies than counted: never write
                        atomicOr(err, 2);
                        continue;
                    }
                    sorted[off[t] + (left - 1u)] = make_float4(lx, ly, lz, o.w);
                }
            }
        }
    }
}

// ---- exclusive scan of uint32 counts into int64 offsets ----
__device__ __forceinline__ int64_t block_exclusive_scan(int64_t v, int64_t *total) {
    __shared__ int64_t wsum[kScanThreads / 32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int64_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int64_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) wsum[wid] = x;
    __syncthreads();
    if (wid == 0) {
        int64_t s = lane < kScanThreads / 32 ? wsum[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int64_t y = __shfl_up_sync(0xffffffffu, s, o);
            if (lane >= o) s += y;
        }
        if (lane < kScanThreads / 32) wsum[lane] = s;    // inclusive warp prefix
    }
    __syncthreads();
    const int64_t before = (wid > 0 ? wsum[wid - 1] : 0) + x - v;
    *total = wsum[kScanThreads / 32 - 1];
    __syncthreads();
    return before;
}

__global__ void __launch_bounds__(kScanThreads)
k_scan_blocks(const uint32_t *__restrict__ cnt, int64_t n, int64_t *__restrict__ off,
              int64_t *__restrict__ bsum) {
    const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanPer;
    int64_t v[kScanPer];
    int64_t s = 0;
#pragma unroll
    for (int k = 0; k < kScanPer; ++k) {
        v[k] = base + k < n ? (int64_t)cnt[base + k] : 0;
        s += v[k];
    }
    int64_t total;
    int64_t run = block_exclusive_scan(s, &total);
#pragma unroll
    for (int k = 0; k < kScanPer; ++k) {
        if (base + k < n) off[base + k] = run;
        run += v[k];
    }
    if (threadIdx.x == 0) bsum[blockIdx.x] = total;
}

__global__ void __launch_bounds__(kScanThreads)
k_scan_sums(int64_t *__restrict__ bsum, int nb, int64_t *__restrict__ grand) {
    // one block; nb <= kScanTile
    const int base = threadIdx.x * kScanPer;
    int64_t v[kScanPer];
    int64_t s = 0;
#pragma unroll
    for (int k = 0; k < kScanPer; ++k) {
        v[k] = base + k < nb ? bsum[base + k] : 0;
        s += v[k];
    }
    int64_t total;
    int64_t run = block_exclusive_scan(s, &total);
#pragma unroll
    for (int k = 0; k < kScanPer; ++k) {
        if (base + k < nb) bsum[base + k] = run;
        run += v[k];
    }
    if (threadIdx.x == 0) *grand = total;
}

__global__ void __launch_bounds__(kScanThreads)
k_scan_add(int64_t *__restrict__ off, int64_t n, const int64_t *__restrict__ bsum) {
    const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanPer;
    const int64_t add = bsum[blockIdx.x];
#pragma unroll
    for (int k = 0; k < kScanPer; ++k)
        if (base + k < n) off[base + k] += add;
}

// ---- tile paint ----
// Per-axis B-spline weights of order P for a node-relative coordinate u
// (cells): nodes base .. base + P - 1.
template <int P>
__device__ __forceinline__ void spline_weights(float u, int &base, float *wt) {
    if (P == 2) {                       // CIC
        const float f0 = floorf(u);
        const float f = u - f0;
        base = (int)f0;
        wt[0] = 1.0f - f;
        wt[1] = f;
    } else if (P == 3) {                // TSC: nearest node base + 1
        const float f0 = floorf(u - 0.5f);
        const float g = u - (f0 + 1.0f);    // in [-1/2, 1/2)
        base = (int)f0;
        const float a = 0.5f - g, b = 0.5f + g;
        wt[0] = 0.5f * a * a;
        wt[1] = 0.75f - g * g;
        wt[2] = 0.5f * b * b;
    } else {                            // PCS
        const float f0 = floorf(u);
        const float f = u - f0, r = 1.0f - f;
        base = (int)f0 - 1;
        const float f2 = f * f, r2 = r * r;
        wt[0] = (1.0f / 6.0f) * r2 * r;
        wt[1] = (1.0f / 6.0f) * (4.0f - 6.0f * f2 + 3.0f * f2 * f);
        wt[2] = (1.0f / 6.0f) * (4.0f - 6.0f * r2 + 3.0f * r2 * r);
        wt[3] = (1.0f / 6.0f) * f2 * f;
    }
}

template <int P>
__device__ __forceinline__ void deposit(unsigned long long *acc, int T, float x, float y, float z,
                                        float ws) {
    int bx, by, bz;
    float wx[P], wy[P], wz[P];
    spline_weights<P>(x, bx, wx);
    spline_weights<P>(y, by, wy);
    spline_weights<P>(z, bz, wz);
#pragma unroll
    for (int a = 0; a < P; ++a) {
        const int cx = bx + a;
        if ((unsigned)cx >= (unsigned)T) continue;
        const float vx = ws * wx[a];
#pragma unroll
        for (int b = 0; b < P; ++b) {
            const int cy = by + b;
            if ((unsigned)cy >= (unsigned)T) continue;
            const float vxy = vx * wy[b];
            unsigned long long *row = acc + (cx * T + cy) * T;
#pragma unroll
            for (int c = 0; c < P; ++c) {
                const int cz = bz + c;
                if ((unsigned)cz >= (unsigned)T) continue;
                const long long q = __float2ll_rn(vxy * wz[c]);
                if (q != 0) atomicAdd(row + cz, (unsigned long long)q);
            }
        }
    }
}

template <typename M>
__device__ __forceinline__ M fixed_to_real(unsigned long long a, int S);
template <>
__device__ __forceinline__ float fixed_to_real<float>(unsigned long long a, int S) {
    return ldexpf(__ll2float_rn((long long)a), -S);
}
template <>
__device__ __forceinline__ double fixed_to_real<double>(unsigned long long a, int S) {
    return ldexp(__ll2double_rn((long long)a), -S);
}

template <int P, int NM, typename M>
__global__ void __launch_bounds__(kPaintThreads)
k_paint_tiles(const float4 *__restrict__ sorted, const int64_t *__restrict__ off, PaintGeom g,
              int S, M *__restrict__ mesh, long long item_stride, long long mesh_stride,
              int accumulate) {
    extern __shared__ unsigned long long acc[];       // NM * T^3 fixed-point cells
    const int T = g.T, T3 = T * T * T;
    const int64_t gt = blockIdx.x;                    // item * ntiles + tile
    const int64_t item = gt / g.ntiles;
    const int64_t t = gt - item * g.ntiles;
    const int tx = (int)(t / ((int64_t)g.ntx * g.ntx));
    const int ty = (int)((t / g.ntx) % g.ntx);
    const int tz = (int)(t % g.ntx);
    for (int c = threadIdx.x; c < NM * T3; c += blockDim.x) acc[c] = 0ull;
    __syncthreads();
    const float scale = ldexpf(1.0f, S);
    const int64_t q1 = off[gt + 1];
    for (int64_t q = off[gt] + threadIdx.x; q < q1; q += blockDim.x) {
        const float4 v = __ldcs(sorted + q);
        const float ws = v.w * scale;
        deposit<P>(acc, T, v.x, v.y, v.z, ws);
        if (NM == 2) deposit<P>(acc + T3, T, v.x + 0.5f, v.y + 0.5f, v.z + 0.5f, ws);
    }
    __syncthreads();
    const long long pitch = 2LL * (g.N / 2 + 1);
    M *base = mesh + item * item_stride;
    for (int m = 0; m < NM; ++m) {
        M *mb = base + m * mesh_stride;
        for (int c = threadIdx.x; c < T3; c += blockDim.x) {
            const int cz = c % T, cy = (c / T) % T, cx = c / (T * T);
            const long long gx = (long long)tx * T + cx, gy = (long long)ty * T + cy;
            const long long idx = (gx * g.N + gy) * pitch + (long long)tz * T + cz;
            const M val = fixed_to_real<M>(acc[m * T3 + c], S);
            if (accumulate) mb[idx] += val;
            else mb[idx] = val;
        }
    }
}

// ---- fused compensate + interlace + bin ----
template <typename C>
__device__ __forceinline__ C cmul(C a, C b) {
    C r;
    r.x = a.x * b.x - a.y * b.y;
    r.y = a.x * b.y + a.y * b.x;
    return r;
}

__device__ __forceinline__ void load4(const float2 *p, float2 *a) {
    const float4 u = __ldcs(reinterpret_cast<const float4 *>(p));
    const float4 v = __ldcs(reinterpret_cast<const float4 *>(p) + 1);
    a[0] = make_float2(u.x, u.y);
    a[1] = make_float2(u.z, u.w);
    a[2] = make_float2(v.x, v.y);
    a[3] = make_float2(v.z, v.w);
}
__device__ __forceinline__ void load4(const double2 *p, double2 *a) {
#pragma unroll
    for (int k = 0; k < 4; ++k) a[k] = __ldcs(p + k);
}

__host__ __device__ __forceinline__ size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

template <typename R, typename C, typename A>
struct BinSmem {
    // layout: hist[nh] (A), cw_l[Nh] (R), ph_l[Nh] (C), edge[nk+1] (int)
    __host__ __device__ static size_t off_cw(const BinGeom &g) { return align_up((size_t)g.nh * sizeof(A), 16); }
    __host__ __device__ static size_t off_ph(const BinGeom &g) { return align_up(off_cw(g) + (size_t)g.Nh * sizeof(R), 16); }
    __host__ __device__ static size_t off_edge(const BinGeom &g) { return align_up(off_ph(g) + (size_t)g.Nh * sizeof(C), 16); }
    __host__ __device__ static size_t bytes(const BinGeom &g) { return align_up(off_edge(g) + (size_t)(g.nk + 1) * sizeof(int), 16); }
};

template <bool IL, bool TWOD, bool POLES, typename R, typename C, typename A>
__global__ void __launch_bounds__(kBinThreads)
k_bin(const C *__restrict__ mesh, long long item_stride_c, long long mesh_stride_c, int nchunks,
      BinGeom g, const R *__restrict__ cw, const C *__restrict__ ph, const int *__restrict__ kedge,
      A *__restrict__ partial) {
    using SM = BinSmem<R, C, A>;
    extern __shared__ __align__(16) unsigned char smraw[];
    A *hist = reinterpret_cast<A *>(smraw);
    R *scw = reinterpret_cast<R *>(smraw + SM::off_cw(g));
    C *sph = reinterpret_cast<C *>(smraw + SM::off_ph(g));
    int *sedge = reinterpret_cast<int *>(smraw + SM::off_edge(g));
    for (int k = threadIdx.x; k < g.nh; k += blockDim.x) hist[k] = (A)0;
    for (int k = threadIdx.x; k < g.Nh; k += blockDim.x) {
        scw[k] = cw[k];
        sph[k] = ph[k + g.N / 2];
    }
    for (int k = threadIdx.x; k <= g.nk; k += blockDim.x) sedge[k] = kedge[k];
    __syncthreads();

    const int item = blockIdx.y;
    const C *m1 = mesh + (long long)item * item_stride_c;
    const C *m2 = m1 + mesh_stride_c;
    const long long CH = (long long)kBinThreads * kBinVec;
    const int half = g.N / 2;
    for (int chunk = blockIdx.x; chunk < nchunks; chunk += gridDim.x) {
        const long long f0 = (long long)chunk * CH + (long long)kBinVec * threadIdx.x;
        if (f0 >= g.modes) continue;
        C a[kBinVec], b2[kBinVec];
        load4(m1 + f0, a);
        if (IL) load4(m2 + f0, b2);
        const long long row = f0 / g.Nh;
        int l = (int)(f0 - row * g.Nh);
        int i = (int)(row / g.N);
        int j = (int)(row - (long long)i * g.N);
        int r2 = 0;
        R rowcw = (R)0;
        C rowph;
        rowph.x = (R)0;
        rowph.y = (R)0;
        auto row_terms = [&]() {
            const int ip = i < half ? i : i - g.N;
            const int jp = j < half ? j : j - g.N;
            r2 = ip * ip + jp * jp;
            rowcw = cw[i] * cw[j];
            if (IL) {
                rowcw *= (R)0.25;
                rowph = cmul(ph[ip + half], ph[jp + half]);
            }
        };
        row_terms();
#pragma unroll
        for (int v = 0; v < kBinVec; ++v) {
            if (l == g.Nh) {
                l = 0;
                if (++j == g.N) {
                    j = 0;
                    ++i;
                }
                row_terms();
            }
            const int m = r2 + l * l;
            if (m != 0 && m >= g.mlo && m < g.mhi) {
                int b = (int)(sqrtf((float)m) * g.kscale - g.koff);
                b = min(max(b, 0), g.nk - 1);
                while (b > 0 && m < sedge[b]) --b;
                while (b < g.nk - 1 && m >= sedge[b + 1]) ++b;
                C z = a[v];
                if (IL) {
                    const C t = cmul(rowph, sph[l]);
                    z.x += b2[v].x * t.x - b2[v].y * t.y;
                    z.y += b2[v].x * t.y + b2[v].y * t.x;
                }
                R pw = (z.x * z.x + z.y * z.y) * rowcw * scw[l];
                if (l != 0 && l != half) pw += pw;
                if (TWOD) {
                    const int nmu = g.nmu;
                    int q = (int)((float)(nmu * l) * rsqrtf((float)m));
                    q = min(max(q, 0), nmu - 1);
                    const long long rhs = (long long)nmu * nmu * l * l;
                    while (q > 0 && (long long)q * q * m > rhs) --q;
                    while (q < nmu - 1 && (long long)(q + 1) * (q + 1) * m <= rhs) ++q;
                    atomicAdd(hist + b * nmu + q, (A)pw);
                } else {
                    atomicAdd(hist + b, (A)pw);
                }
                if (POLES) {
                    const R mu2 = (R)(l * l) / (R)m;
                    const R t2 = pw * mu2;
                    atomicAdd(hist + g.hbase + b, (A)t2);
                    atomicAdd(hist + g.hbase + g.nk + b, (A)(t2 * mu2));
                }
            }
            ++l;
        }
    }
    __syncthreads();
    A *out = partial + ((long long)item * gridDim.x + blockIdx.x) * g.nh;
    for (int k = threadIdx.x; k < g.nh; k += blockDim.x) out[k] = hist[k];
}

template <typename A>
__global__ void k_bin_reduce(const A *__restrict__ partial, int G, int nh, double *__restrict__ sums) {
    const int item = blockIdx.y;
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nh) return;
    const A *p = partial + (long long)item * G * nh + k;
    double s = 0.0;
    for (int c = 0; c < G; ++c) s += (double)p[(long long)c * nh];   // fixed order
    sums[(long long)item * nh + k] = s;
}

__global__ void k_finalize(const double *__restrict__ sums, const unsigned long long *__restrict__ modes1d,
                           const unsigned long long *__restrict__ modes2d,
                           const double *__restrict__ wsums, const int *__restrict__ err,
                           FinalGeom f, ResultLayout rl, double *__restrict__ res) {
    const int item = blockIdx.x;
    const double *s = sums + (long long)item * f.nh;
    double *r = res + (long long)item * f.RL;
    const double wsum = wsums[3 * item], w2sum = wsums[3 * item + 1], wabs = wsums[3 * item + 2];
    const double norm = f.L3 / (wsum * wsum);
    const double shot = f.L3 * w2sum / (wsum * wsum);
    const double sub = f.subtract_shot ? shot : 0.0;
    const double nan = __longlong_as_double(0x7ff8000000000000LL);
    for (int b = threadIdx.x; b < f.nk; b += blockDim.x) {
        double S0 = 0.0;
        if (f.twod) {
            for (int q = 0; q < f.nmu; ++q) S0 += s[b * f.nmu + q];
        } else {
            S0 = s[b];
        }
        const double cnt = (double)modes1d[b];
        double p0 = nan, p2 = nan, p4 = nan;
        if (cnt > 0.0) {
            p0 = norm * S0 / cnt - sub;
            if (f.poles) {
                const double M2 = s[f.hbase + b], M4 = s[f.hbase + f.nk + b];
                p2 = 5.0 * norm * (1.5 * M2 - 0.5 * S0) / cnt;
                p4 = 9.0 * norm * (35.0 * M4 - 30.0 * M2 + 3.0 * S0) / (8.0 * cnt);
            }
        }
        r[rl.pk + b] = p0;
        r[rl.poles + b] = (f.poles_mask & 1u) ? p0 : nan;
        r[rl.poles + f.nk + b] = (f.poles_mask & 2u) ? p2 : nan;
        r[rl.poles + 2 * f.nk + b] = (f.poles_mask & 4u) ? p4 : nan;
    }
    if (f.twod) {
        for (int bq = threadIdx.x; bq < f.nk * f.nmu; bq += blockDim.x) {
            const double cnt = (double)modes2d[bq];
            r[rl.pkmu + bq] = cnt > 0.0 ? norm * s[bq] / cnt - sub : nan;
        }
    }
    if (threadIdx.x == 0) {
        r[rl.shot] = shot;
        r[rl.wsum] = wsum;
        r[rl.w2sum] = w2sum;
        r[rl.flags] = (double)(((wabs > f.headroom) ? 1 : 0) | (*err & 2));
    }
}

// ---- plan-time geometry: integer histograms over (m, q) ----
__global__ void k_geom_hist(BinGeom g, unsigned long long *__restrict__ H,
                            unsigned long long *__restrict__ HL) {
    const int nq = g.nmu > 0 ? g.nmu : 1;
    const int half = g.N / 2;
    for (long long row = blockIdx.x; row < (long long)g.N * g.N; row += gridDim.x) {
        const int i = (int)(row / g.N), j = (int)(row % g.N);
        const int ip = i < half ? i : i - g.N, jp = j < half ? j : j - g.N;
        const int r2 = ip * ip + jp * jp;
        for (int l = threadIdx.x; l < g.Nh; l += blockDim.x) {
            const int m = r2 + l * l;
            if (m == 0 || m < g.mlo || m >= g.mhi) continue;
            int q = 0;
            if (g.nmu > 0) {
                const long long rhs = (long long)g.nmu * g.nmu * l * l;
                while (q + 1 <= g.nmu - 1 && (long long)(q + 1) * (q + 1) * m <= rhs) ++q;
            }
            const unsigned long long h = (l == 0 || l == half) ? 1ull : 2ull;
            atomicAdd(H + (long long)m * nq + q, h);
            atomicAdd(HL + (long long)m * nq + q, h * (unsigned long long)l);
        }
    }
}

__global__ void k_geom_finalize(BinGeom g, const int *__restrict__ kedge, double kF,
                                const unsigned long long *__restrict__ H,
                                const unsigned long long *__restrict__ HL,
                                unsigned long long *__restrict__ modes2d,
                                double *__restrict__ kmean2d, double *__restrict__ mumean2d) {
    const int nq = g.nmu > 0 ? g.nmu : 1;
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= g.nk * nq) return;
    const int b = idx / nq, q = idx % nq;
    unsigned long long cnt = 0;
    double ks = 0.0, mus = 0.0;
    const int m0 = max(kedge[b], 1), m1 = kedge[b + 1];
    for (int m = m0; m < m1; ++m) {
        const unsigned long long c = H[(long long)m * nq + q];
        if (c == 0) continue;
        const double sm = sqrt((double)m);
        cnt += c;
        ks += (double)c * sm;
        mus += (double)HL[(long long)m * nq + q] / sm;
    }
    const double nan = __longlong_as_double(0x7ff8000000000000LL);
    modes2d[idx] = cnt;
    kmean2d[idx] = cnt ? kF * ks / (double)cnt : nan;
    mumean2d[idx] = cnt ? mus / (double)cnt : nan;
}

template <typename K>
cudaError_t set_smem(K kernel, size_t bytes) {
    if (bytes <= 48 * 1024) return cudaSuccess;
    return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

unsigned grid_for(int64_t n, int threads, unsigned cap) {
    int64_t b = (n + threads - 1) / threads;
    if (b < 1) b = 1;
    if (b > (int64_t)cap) b = cap;
    return (unsigned)b;
}

}  // namespace

ResultLayout result_layout(int nk, int nmu) {
    ResultLayout r;
    r.pk = 0;
    r.poles = nk;
    r.pkmu = 4 * nk;
    r.shot = 4 * nk + nk * nmu;
    r.wsum = r.shot + 1;
    r.w2sum = r.shot + 2;
    r.flags = r.shot + 3;
    r.total = r.shot + 4;
    return r;
}

cudaError_t launch_tile_count(const void *pos, int dtype, const float *w, const int64_t *item_off,
                              int nitems, int64_t max_n, const PaintGeom &g, uint32_t *count,
                              double *wsums, cudaStream_t st) {
    dim3 grid(grid_for(max_n, kCountThreads, 1u << 20), nitems);
    switch (dtype) {
    case PK_F32: k_tile_count<PK_F32><<<grid, kCountThreads, 0, st>>>(pos, w, item_off, g, count, wsums); break;
    case PK_F64: k_tile_count<PK_F64><<<grid, kCountThreads, 0, st>>>(pos, w, item_off, g, count, wsums); break;
    default: k_tile_count<PK_F32X4><<<grid, kCountThreads, 0, st>>>(pos, w, item_off, g, count, wsums); break;
    }
    return cudaGetLastError();
}

cudaError_t launch_tile_scatter(const void *pos, int dtype, const float *w,
                                const int64_t *item_off, int nitems, int64_t max_n,
                                const PaintGeom &g, uint32_t *count, const int64_t *off,
                                float4 *sorted, int *err, cudaStream_t st) {
    dim3 grid(grid_for(max_n, kCountThreads, 1u << 20), nitems);
    switch (dtype) {
    case PK_F32: k_tile_scatter<PK_F32><<<grid, kCountThreads, 0, st>>>(pos, w, item_off, g, count, off, sorted, err); break;
    case PK_F64: k_tile_scatter<PK_F64><<<grid, kCountThreads, 0, st>>>(pos, w, item_off, g, count, off, sorted, err); break;
    default: k_tile_scatter<PK_F32X4><<<grid, kCountThreads, 0, st>>>(pos, w, item_off, g, count, off, sorted, err); break;
    }
    return cudaGetLastError();
}

cudaError_t launch_scan(const uint32_t *count, int64_t n, int64_t *off, int64_t *block_tmp,
                        cudaStream_t st) {
    const int64_t nb = (n + kScanTile - 1) / kScanTile;
    if (nb > kScanTile) return cudaErrorInvalidValue;
    if (nb > 0) k_scan_blocks<<<(unsigned)nb, kScanThreads, 0, st>>>(count, n, off, block_tmp);
    k_scan_sums<<<1, kScanThreads, 0, st>>>(block_tmp, (int)nb, off + n);
    if (nb > 0) k_scan_add<<<(unsigned)nb, kScanThreads, 0, st>>>(off, n, block_tmp);
    return cudaGetLastError();
}

size_t paint_smem_bytes(int T, int nmesh) {
    return (size_t)nmesh * T * T * T * sizeof(unsigned long long);
}

template <int P, int NM, typename M>
static cudaError_t paint_inst(const float4 *sorted, const int64_t *off, int nitems,
                              const PaintGeom &g, int S, void *mesh, long long item_stride,
                              long long mesh_stride, int accumulate, cudaStream_t st) {
    const size_t smem = paint_smem_bytes(g.T, NM);
    cudaError_t e = set_smem(k_paint_tiles<P, NM, M>, smem);
    if (e != cudaSuccess) return e;
    const long long nblocks = (long long)nitems * g.ntiles;
    if (nblocks <= 0) return cudaSuccess;
    if (nblocks > 0x7fffffffLL) return cudaErrorInvalidValue;
    k_paint_tiles<P, NM, M><<<(unsigned)nblocks, kPaintThreads, smem, st>>>(
        sorted, off, g, S, reinterpret_cast<M *>(mesh), item_stride, mesh_stride, accumulate);
    return cudaGetLastError();
}

cudaError_t launch_paint_tiles(const float4 *sorted, const int64_t *off, int nitems,
                               const PaintGeom &g, int window, int nmesh, int S, int f64,
                               void *mesh, long long item_stride, long long mesh_stride,
                               int accumulate, cudaStream_t st) {
#define PK_PAINT_CASE(P)                                                                              \
    if (window == P) {                                                                                \
        if (f64) return nmesh == 2 ? paint_inst<P, 2, double>(sorted, off, nitems, g, S, mesh,        \
                                                              item_stride, mesh_stride, accumulate, st) \
                                   : paint_inst<P, 1, double>(sorted, off, nitems, g, S, mesh,        \
                                                              item_stride, mesh_stride, accumulate, st); \
        return nmesh == 2 ? paint_inst<P, 2, float>(sorted, off, nitems, g, S, mesh, item_stride,     \
                                                    mesh_stride, accumulate, st)                      \
                          : paint_inst<P, 1, float>(sorted, off, nitems, g, S, mesh, item_stride,     \
                                                    mesh_stride, accumulate, st);                     \
    }
    PK_PAINT_CASE(2)
    PK_PAINT_CASE(3)
    PK_PAINT_CASE(4)
#undef PK_PAINT_CASE
    return cudaErrorInvalidValue;
}

size_t bin_smem_bytes(const BinGeom &g, int f64) {
    return f64 ? BinSmem<double, double2, double>::bytes(g) : BinSmem<float, float2, float>::bytes(g);
}

int bin_threads() { return kBinThreads; }

template <bool IL, bool TWOD, bool POLES, typename R, typename C, typename A>
static cudaError_t bin_inst(const void *mesh, long long item_stride_c, long long mesh_stride_c,
                            int nitems, int G, const BinGeom &g, const void *cw, const void *ph,
                            const int *kedge, void *partial, cudaStream_t st) {
    const size_t smem = BinSmem<R, C, A>::bytes(g);
    auto kern = k_bin<IL, TWOD, POLES, R, C, A>;
    cudaError_t e = set_smem(kern, smem);
    if (e != cudaSuccess) return e;
    const long long CH = (long long)kBinThreads * kBinVec;
    const int nchunks = (int)((g.modes + CH - 1) / CH);
    dim3 grid(G, nitems);
    kern<<<grid, kBinThreads, smem, st>>>(reinterpret_cast<const C *>(mesh), item_stride_c,
                                          mesh_stride_c, nchunks, g, reinterpret_cast<const R *>(cw),
                                          reinterpret_cast<const C *>(ph), kedge,
                                          reinterpret_cast<A *>(partial));
    return cudaGetLastError();
}

template <typename R, typename C, typename A>
static cudaError_t bin_dispatch(const void *mesh, int il, long long is, long long ms, int nitems,
                                int G, const BinGeom &g, const void *cw, const void *ph,
                                const int *kedge, void *partial, cudaStream_t st) {
    const int key = (il ? 4 : 0) | (g.twod ? 2 : 0) | (g.poles ? 1 : 0);
    switch (key) {
    case 0: return bin_inst<false, false, false, R, C, A>(mesh, is, ms, nitems, G, g, cw, ph, kedge, partial, st);
    case 1: return bin_inst<false, false, true, R, C, A>(mesh, is, ms, nitems, G, g, cw, ph, kedge, partial, st);
    case 2: return bin_inst<false, true, false, R, C, A>(mesh, is, ms, nitems, G, g, cw, ph, kedge, partial, st);
    case 3: return bin_inst<false, true, true, R, C, A>(mesh, is, ms, nitems, G, g, cw, ph, kedge, partial, st);
    case 4: return bin_inst<true, false, false, R, C, A>(mesh, is, ms, nitems, G, g, cw, ph, kedge, partial, st);
    case 5: return bin_inst<true, false, true, R, C, A>(mesh, is, ms, nitems, G, g, cw, ph, kedge, partial, st);
    case 6: return bin_inst<true, true, false, R, C, A>(mesh, is, ms, nitems, G, g, cw, ph, kedge, partial, st);
    default: return bin_inst<true, true, true, R, C, A>(mesh, is, ms, nitems, G, g, cw, ph, kedge, partial, st);
    }
}

cudaError_t launch_bin(const void *mesh, int f64, int interlaced, long long item_stride_c,
                       long long mesh_stride_c, int nitems, int ctas_per_item,
                       const BinGeom &g, const void *cw, const void *ph, const int *kedge,
                       void *partial, cudaStream_t st) {
    if (f64)
        return bin_dispatch<double, double2, double>(mesh, interlaced, item_stride_c, mesh_stride_c,
                                                      nitems, ctas_per_item, g, cw, ph, kedge, partial, st);
    return bin_dispatch<float, float2, float>(mesh, interlaced, item_stride_c, mesh_stride_c, nitems,
                                              ctas_per_item, g, cw, ph, kedge, partial, st);
}

int bin_ctas_per_sm(const BinGeom &g, int f64, int interlaced) {
    int n = 0;
    const size_t smem = bin_smem_bytes(g, f64);
    cudaError_t e;
    if (f64) {
        auto k = k_bin<true, true, true, double, double2, double>;
        set_smem(k, smem);
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k, kBinThreads, smem);
    } else {
        auto k = k_bin<true, true, true, float, float2, float>;
        set_smem(k, smem);
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k, kBinThreads, smem);
    }
    (void)interlaced;
    if (e != cudaSuccess || n < 1) n = 1;
    return n;
}

cudaError_t launch_bin_reduce(const void *partial, int f64, int G, int nh, int nitems,
                              double *sums, cudaStream_t st) {
    dim3 grid((nh + 255) / 256, nitems);
    if (f64) k_bin_reduce<double><<<grid, 256, 0, st>>>(reinterpret_cast<const double *>(partial), G, nh, sums);
    else k_bin_reduce<float><<<grid, 256, 0, st>>>(reinterpret_cast<const float *>(partial), G, nh, sums);
    return cudaGetLastError();
}

cudaError_t launch_finalize(const double *sums, const unsigned long long *modes1d,
                            const unsigned long long *modes2d, const double *wsums, const int *err,
                            const FinalGeom &f, int nitems, double *res, cudaStream_t st) {
    const ResultLayout rl = result_layout(f.nk, f.nmu);
    k_finalize<<<nitems, 256, 0, st>>>(sums, modes1d, modes2d, wsums, err, f, rl, res);
    return cudaGetLastError();
}

cudaError_t launch_geom_hist(const BinGeom &g, unsigned long long *H, unsigned long long *HL,
                             cudaStream_t st) {
    const long long rows = (long long)g.N * g.N;
    const unsigned grid = (unsigned)(rows < 65536 ? rows : 65536);
    k_geom_hist<<<grid, 256, 0, st>>>(g, H, HL);
    return cudaGetLastError();
}

cudaError_t launch_geom_finalize(const BinGeom &g, const int *kedge, double kF,
                                 const unsigned long long *H, const unsigned long long *HL,
                                 unsigned long long *modes1d, double *kmean1d,
                                 unsigned long long *modes2d, double *kmean2d,
                                 double *mumean2d, cudaStream_t st) {
    (void)modes1d;
    (void)kmean1d;
    const int nq = g.nmu > 0 ? g.nmu : 1;
    const int n = g.nk * nq;
    k_geom_finalize<<<(n + 127) / 128, 128, 0, st>>>(g, kedge, kF, H, HL, modes2d, kmean2d, mumean2d);
    return cudaGetLastError();
}

}  // namespace pk
