// pk_kernels.cu -- sm_103a kernels of the FFT power-spectrum path.
//
// Paint (Sec. 3.3.1 painting; Sec. 3.3.2 CIC / TSC / PCS B-spline windows and
// interlacing with a second mesh shifted by half a cell):
//   k_sort_count    wrap each object into the box, find its home tile (T^3
//                   cells) and its boundary class (per axis: near the low
//                   face, interior, near the high face -- 27 classes) and
//                   count objects per (tile, class) key (reductions whose
//                   result nobody waits for); sum w, w^2, |w| and max |w|.
//   k_wsum_reduce   weighted catalogs: the paint blocks' rows of weight sums
//                   added in a fixed order (run-to-run identical sums).
//   k_scan_*        exclusive scan of the key counts (uint32).
//   k_sort_scatter  write one float4 (home-tile-local x, y, z, w) per object
//                   at offset[key] + (its key's count, decremented): the
//                   order inside a key is whatever order the decrements are
//                   served in, which the paint's integer deposits do not
//                   see; the counts end at zero.  No per-object rank array.
//   k_paint_tiles   one CTA per tile: gather the tile's own objects and the
//                   boundary classes of its 26 neighbours whose window reaches
//                   into it, deposit B-spline weights into shared memory as
//                   exact int64 fixed point held in two uint32 words per cell
//                   (the split point is chosen per tile so the low word can
//                   never carry; shared 32-bit atomics are ~5x faster than
//                   64-bit ones here), then write the tile once, coalesced,
//                   into the in-place r2c layout.  Unit weights: one sweep
//                   over the candidates deposits both interlaced meshes (one
//                   32-bit word per cell each), branch-free in sparse tiles;
//                   weighted objects: one mesh per pass over staged
//                   candidates.  Integer adds are order-free: the mesh is
//                   bit-identical run to run and for any object order.
//   k_paint_atomic  the variant without a sort: one thread per object adds
//                   each deposit with a 64-bit global atomic into a dense
//                   int64 accumulator per mesh (as order-free as the tiles);
//   k_acc_to_mesh   converts the accumulators into the r2c layout and clears
//                   them.  Cheaper than sorting for small meshes that stay in
//                   L2; the plan's paint_variant picks one of the two.
// Bin (Sec. 3.4.1, Eq. window-deconvolution):
//   k_bin           warps take whole rows of the stored half grid and visit
//                   only the binned l range; per mode: interlace combine,
//                   sinc^p compensation, |delta|^2, k bin (exact integer
//                   edges in m = |n|^2), mu bin (exact integer rule),
//                   Legendre L_2(mu) / L_4(mu) weights; runs of equal bins merged
//                   in registers, then per-CTA shared-memory histograms.
//   k_bin_reduce    fixed-order FP64 sums of the per-CTA histograms in 32-row
//                   chunks, then (in place) of the chunks.
//   k_finalize      normalization L^3 / (sum w)^2, shot noise, multipoles.
// Plan time (geometry only):
//   k_geom_*        exact mode counts per bin and mean k, mean mu from integer
//                   histograms over (m, mu bin), summed in FP64.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <algorithm>
#include <type_traits>

#include "pk_internal.h"

namespace pk {

namespace {

constexpr int kCountThreads = 256;
constexpr unsigned kWsumBlocks = 2048;  // blocks per catalog of the passes that sum the weights
constexpr int kPaintThreads = 256;
constexpr int kBinThreads = 256;
constexpr int kBinVec = 4;            // consecutive modes per thread
constexpr int kScanThreads = 1024;
constexpr int kScanPer = 4;           // elements per thread in a scan block
constexpr int kScanTile = kScanThreads * kScanPer;
constexpr int kClasses = 27;          // boundary classes per tile
constexpr int kSegments = 75;         // (neighbour, class range) segments per tile
constexpr int kReduceChunk = 32;      // per-CTA histograms summed per reduce block
constexpr int kStage = 256;           // candidates staged in shared memory per batch (small: 6 CTAs / SM)
constexpr int kUploadChunk = 256;     // int64 values per parameter upload (2 KB)
// Sweep paint: tiles with at most this many candidates use branch-free
// deposits; denser tiles (e.g. uniform lattices, ~900 candidates per 16^3
// tile) were measured faster with deposits that skip cells outside the tile.
constexpr int kFlatMaxCand = 640;

// Cell coordinate s = x * (N / L) wrapped periodically into [0, N).  Written
// with explicitly rounded intrinsics so that no FMA contraction can differ
// between the count and the scatter kernels: both must see the same s.
// FP32 positions: s is returned as s_hi + *e, where s_hi = fl(x * invH) and
// *e is the exact residual of that product plus x times the residual of
// invH = N / L; cells and tiles follow s_hi, and e is added back into the
// small tile-local coordinate (whose resolution is ~1e-6 cells), so large
// meshes do not lose the FP32 rounding of s (up to 1.2e-4 cells at N = 2048).
// Positions outside [0, L) are wrapped on s_hi with e = 0.
__device__ __forceinline__ float wrap_cells(float x, float invH, float invH_lo, int N, float *e) {
    const float n = (float)N;
    float s = __fmul_rn(x, invH);
    *e = __fadd_rn(__fmaf_rn(x, invH, -s), __fmul_rn(x, invH_lo));
    if (!(s >= 0.0f && s < n)) {
        *e = 0.0f;
        s = __fsub_rn(s, __fmul_rn(n, floorf(__fdiv_rn(s, n))));
        if (s < 0.0f) s = __fadd_rn(s, n);
        if (s >= n) s = __fsub_rn(s, n);
        if (!(s >= 0.0f && s < n)) s = 0.0f;            // NaN / inf positions
    }
    return s;
}
__device__ __forceinline__ double wrap_cells(double x, double invH, int N) {
    const double n = (double)N;
    double s = __dmul_rn(x, invH);
    if (!(s >= 0.0 && s < n)) {
        s = __dsub_rn(s, __dmul_rn(n, floor(__ddiv_rn(s, n))));
        if (s < 0.0) s = __dadd_rn(s, n);
        if (s >= n) s = __dsub_rn(s, n);
        if (!(s >= 0.0 && s < n)) s = 0.0;
    }
    return s;
}

template <typename R>
struct Obj {
    R s[3];
    float e[3];       // residual of s (FP32 positions), 0 for FP64 positions
    float w;          // weight W (normalization: sum W)
    float a;          // painted amplitude W V (V: the painted value, 1 by default)
};

template <int DT>
struct PosReal { using type = float; };
template <>
struct PosReal<PK_F64> { using type = double; };

template <int DT>
__device__ __forceinline__ Obj<typename PosReal<DT>::type> load_obj(const void *pos, const float *w,
                                                                    const float *vals, int64_t i,
                                                                    const PaintGeom &g) {
    using R = typename PosReal<DT>::type;
    Obj<R> o;
    if (DT == PK_F32X4) {
        const float4 v = __ldg(reinterpret_cast<const float4 *>(pos) + i);
        o.s[0] = wrap_cells(v.x, g.invH, g.invH_lo, g.N, &o.e[0]);
        o.s[1] = wrap_cells(v.y, g.invH, g.invH_lo, g.N, &o.e[1]);
        o.s[2] = wrap_cells(v.z, g.invH, g.invH_lo, g.N, &o.e[2]);
        o.w = v.w;
    } else if (DT == PK_F32) {
        const float *p = reinterpret_cast<const float *>(pos) + 3 * i;
        o.s[0] = wrap_cells(__ldg(p + 0), g.invH, g.invH_lo, g.N, &o.e[0]);
        o.s[1] = wrap_cells(__ldg(p + 1), g.invH, g.invH_lo, g.N, &o.e[1]);
        o.s[2] = wrap_cells(__ldg(p + 2), g.invH, g.invH_lo, g.N, &o.e[2]);
        o.w = w ? __ldg(w + i) : 1.0f;
    } else {
        const double *p = reinterpret_cast<const double *>(pos) + 3 * i;
        o.s[0] = (R)wrap_cells(__ldg(p + 0), g.invHd, g.N);
        o.s[1] = (R)wrap_cells(__ldg(p + 1), g.invHd, g.N);
        o.s[2] = (R)wrap_cells(__ldg(p + 2), g.invHd, g.N);
        o.e[0] = o.e[1] = o.e[2] = 0.0f;
        o.w = w ? __ldg(w + i) : 1.0f;
    }
    o.a = vals ? o.w * __ldg(vals + i) : o.w;
    return o;
}

// Home tile and boundary class of one object.  Along each axis the class is
// 0 if the window reaches the tile below (c + lo < 0), 2 if it reaches the
// tile above (c + hi >= T), else 1; T >= hi - lo keeps these disjoint.
template <typename R>
__device__ __forceinline__ void home_key(const Obj<R> &o, const PaintGeom &g, int *tile3, int *cls) {
    int c = 0;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const int cell = min((int)floor(o.s[a]), g.N - 1);
        const int t = cell / g.T;
        const int cl = cell - t * g.T;
        tile3[a] = t;
        c = c * 3 + (cl < -g.lo ? 0 : (cl >= g.T - g.hi ? 2 : 1));
    }
    *cls = c;
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ float warp_max(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_down_sync(0xffffffffu, v, o));
    return v;
}

// Block reduction of the weight sums: sum W, sum (W V)^2, sum |W V| of the
// block's objects into its row wpart[(item * gridDim.x + block) * 3 + k]
// (summed over the blocks in a fixed order by k_wsum_reduce, so the sums do
// not depend on which block finishes first); wmax[item] = max |W V| (float
// bits, order-free), with W the weight and W V the painted amplitude.
// Unweighted: wsums[4 * item + {0,1,2}] += n, wmax = 1.
__device__ __forceinline__ void flush_wsums(double sw, double sw2, double swa, float mw, bool weighted,
                                            int item, int64_t n_item, double *__restrict__ wsums,
                                            double *__restrict__ wpart, unsigned *__restrict__ wmax) {
    if (weighted) {
        __shared__ double red[3][kCountThreads / 32];
        __shared__ float redm[kCountThreads / 32];
        sw = warp_sum(sw);
        sw2 = warp_sum(sw2);
        swa = warp_sum(swa);
        mw = warp_max(mw);
        const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
        if (lane == 0) {
            red[0][wid] = sw;
            red[1][wid] = sw2;
            red[2][wid] = swa;
            redm[wid] = mw;
        }
        __syncthreads();
        if (threadIdx.x < 3) {
            double t = 0.0;
            for (int k = 0; k < kCountThreads / 32; ++k) t += red[threadIdx.x][k];
            wpart[((size_t)item * gridDim.x + blockIdx.x) * 3 + threadIdx.x] = t;
        } else if (threadIdx.x == 3) {
            float m = 0.0f;
            for (int k = 0; k < kCountThreads / 32; ++k) m = fmaxf(m, redm[k]);
            atomicMax(wmax + item, __float_as_uint(m));
        }
    } else if (blockIdx.x == 0 && threadIdx.x < 3) {
        atomicAdd(wsums + 4 * item + threadIdx.x, (double)n_item);   // exact below 2^53
        if (threadIdx.x == 0) atomicMax(wmax + item, __float_as_uint(1.0f));
    }
}

// Fixed-order sum of the blocks' weight-sum rows of catalog blockIdx.x:
// thread t adds rows t, t + 256, ... in turn, then a fixed tree; the result
// is added to wsums[4 * item + k] (one writer per value).
__global__ void __launch_bounds__(256)
k_wsum_reduce(const double *__restrict__ wpart, int nblk, double *__restrict__ wsums) {
    __shared__ double red[3][256];
    const int item = blockIdx.x, t = threadIdx.x;
    double a[3] = {0.0, 0.0, 0.0};
    for (int b = t; b < nblk; b += 256)
#pragma unroll
        for (int k = 0; k < 3; ++k) a[k] += wpart[((size_t)item * nblk + b) * 3 + k];
#pragma unroll
    for (int k = 0; k < 3; ++k) red[k][t] = a[k];
    __syncthreads();
    for (int h = 128; h > 0; h >>= 1) {
        if (t < h)
#pragma unroll
            for (int k = 0; k < 3; ++k) red[k][t] += red[k][t + h];
        __syncthreads();
    }
    if (t < 3) wsums[4 * item + t] += red[t][0];
}

// Key of an object: (catalog, home tile, boundary class).
template <typename R>
__device__ __forceinline__ int64_t sort_key(const Obj<R> &o, const PaintGeom &g, int64_t kbase, int *t3) {
    int cls;
    home_key<R>(o, g, t3, &cls);
    return kbase + (((int64_t)t3[0] * g.ntx + t3[1]) * g.ntx + t3[2]) * kClasses + cls;
}

// Tile sort, pass 1: key counts, plus the weight sums.
template <int DT, bool WEIGHTED>
__global__ void __launch_bounds__(kCountThreads)
k_sort_count(const void *__restrict__ pos, const float *__restrict__ w, const float *__restrict__ vals,
             const int64_t *__restrict__ item_off, PaintGeom g, uint32_t *__restrict__ count,
             double *__restrict__ wsums, double *__restrict__ wpart, unsigned *__restrict__ wmax) {
    using R = typename PosReal<DT>::type;
    const int item = blockIdx.y;
    const int64_t beg = item_off[item], end = item_off[item + 1];
    const int64_t kbase = (int64_t)item * g.ntiles * kClasses;
    double sw = 0.0, sw2 = 0.0, swa = 0.0;
    float mw = 0.0f;
    for (int64_t i = beg + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < end;
         i += (int64_t)gridDim.x * blockDim.x) {
        const Obj<R> o = load_obj<DT>(pos, w, vals, i, g);
        int t3[3];
        atomicAdd(count + sort_key<R>(o, g, kbase, t3), 1u);   // result unused: a reduction
        if (WEIGHTED) {
            const double ad = (double)o.a;
            sw += (double)o.w;
            sw2 += ad * ad;
            swa += fabs(ad);
            mw = fmaxf(mw, fabsf(o.a));
        }
    }
    flush_wsums(sw, sw2, swa, mw, WEIGHTED, item, end - beg, wsums, wpart, wmax);
}

// Tile sort, pass 2: each object takes the last free slot of its key's range
// (the key's count, decremented: objects of the key not yet placed, this one
// included).  Measured: both passes are bound by the L2's atomic rate, not by
// its latency (two, four or eight objects per thread with every load and
// atomic issued before the first use ran 4 %, 10 % and 23 % slower).
template <int DT>
__global__ void __launch_bounds__(kCountThreads)
k_sort_scatter(const void *__restrict__ pos, const float *__restrict__ w, const float *__restrict__ vals,
               const int64_t *__restrict__ item_off, PaintGeom g, const uint32_t *__restrict__ off,
               uint32_t *__restrict__ count, float4 *__restrict__ sorted, int *__restrict__ err) {
    using R = typename PosReal<DT>::type;
    const int item = blockIdx.y;
    const int64_t beg = item_off[item], end = item_off[item + 1];
    const int64_t kbase = (int64_t)item * g.ntiles * kClasses;
    for (int64_t i = beg + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < end;
         i += (int64_t)gridDim.x * blockDim.x) {
        const Obj<R> o = load_obj<DT>(pos, w, vals, i, g);
        int t3[3];
        const int64_t key = sort_key<R>(o, g, kbase, t3);
        const uint32_t left = atomicSub(count + key, 1u);
        const uint32_t first = off[key];
        if (left == 0 || left > off[key + 1] - first) {   // count and scatter disagree: never write
            atomicOr(err, 2);
            continue;
        }
        sorted[first + left - 1] = make_float4((float)(o.s[0] - (R)(t3[0] * g.T)) + o.e[0],
                                               (float)(o.s[1] - (R)(t3[1] * g.T)) + o.e[1],
                                               (float)(o.s[2] - (R)(t3[2] * g.T)) + o.e[2], o.a);
    }
}

// ---- exclusive scan of uint32 counts (totals < 2^32) or uint64 weights ----
template <typename T>
__device__ __forceinline__ T block_exclusive_scan(T v, T *total) {
    __shared__ T wsum[kScanThreads / 32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    T x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const T y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) wsum[wid] = x;
    __syncthreads();
    if (wid == 0) {
        T s = lane < kScanThreads / 32 ? wsum[lane] : (T)0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const T y = __shfl_up_sync(0xffffffffu, s, o);
            if (lane >= o) s += y;
        }
        if (lane < kScanThreads / 32) wsum[lane] = s;
    }
    __syncthreads();
    const T before = (wid > 0 ? wsum[wid - 1] : (T)0) + x - v;
    *total = wsum[kScanThreads / 32 - 1];
    __syncthreads();
    return before;
}

// out may alias in: every thread reads its own elements before writing them.
template <typename T>
__global__ void __launch_bounds__(kScanThreads)
k_scan_blocks(const T *in, int64_t n, T *out, T *bsum) {
    const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanPer;
    T v[kScanPer];
    T s = 0;
#pragma unroll
    for (int k = 0; k < kScanPer; ++k) {
        v[k] = base + k < n ? in[base + k] : (T)0;
        s += v[k];
    }
    T total;
    T run = block_exclusive_scan<T>(s, &total);
#pragma unroll
    for (int k = 0; k < kScanPer; ++k) {
        if (base + k < n) out[base + k] = run;
        run += v[k];
    }
    if (threadIdx.x == 0) bsum[blockIdx.x] = total;
}

template <typename T>
__global__ void __launch_bounds__(kScanThreads)
k_scan_add(T *__restrict__ out, int64_t n, const T *__restrict__ bsum, int nb) {
    const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanPer;
    const T add = bsum[blockIdx.x];
#pragma unroll
    for (int k = 0; k < kScanPer; ++k)
        if (base + k < n) out[base + k] += add;
    if (blockIdx.x == 0 && threadIdx.x == 0) out[n] = bsum[nb];
}

// ---- tile paint ----
// Per-axis B-spline weights of order P at node-relative coordinate u (cells):
// nodes base .. base + P - 1.
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

// Fixed-point split of one tile: deposit q = round(v) (v = w W 2^S) is held as
// hi * 2^B + lo with lo in [0, 2^B]; the cell keeps sum(lo) and sum(hi) in two
// uint32 words.  With at most `ncand` deposits per cell, sum(lo) <=
// ncand 2^B < 2^32 and |sum(hi)| <= ncand (hmax + 1) < 2^31 by construction.
struct Split {
    int B;            // split bit (1 .. 22)
    float twoB;       // 2^B
    unsigned twoB_u;  // 2^B as an integer
    float inv2B;      // 2^-B
    float hi_scale;   // 2^(B - S): weight units of one hi count
    int fast;         // 2: no deposit needs a split; 1: split when needed;
                      // 0: this tile uses 64-bit shared atomics instead
};

// MODE 2: every deposit is known to satisfy 0 <= round(v) < 2^B (unit
// weights): one FMA, one subtract, one 32-bit shared atomic per cell.
// MODE 1: as 2, with a split into hi * 2^B + lo for the rare large or
// negative deposit.  MODE 0: 64-bit shared atomics (dense tiles).
template <int P, int MODE, int TC = 0>
__device__ __forceinline__ void deposit(unsigned *lo, unsigned *hi, unsigned long long *acc64,
                                        const Split &sp, int T, float x, float y, float z, float ws) {
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
            const int row = (cx * T + cy) * T;
#pragma unroll
            for (int c = 0; c < P; ++c) {
                const int cz = bz + c;
                if ((unsigned)cz >= (unsigned)T) continue;
                if (MODE == 2) {
                    atomicAdd(lo + row + cz, __float_as_uint(fmaf(vxy, wz[c], 8388608.0f)) - 0x4B000000u);
                } else if (MODE == 1) {
                    // 2^23 + round(v) in one FMA; its bits minus 0x4B000000 are
                    // round(v) whenever 0 <= round(v) < 2^B (B <= 22): the
                    // common case, one 32-bit shared atomic.
                    const unsigned q = __float_as_uint(fmaf(vxy, wz[c], 8388608.0f)) - 0x4B000000u;
                    if (q < sp.twoB_u) {
                        atomicAdd(lo + row + cz, q);
                    } else {              // large or negative deposit: split hi * 2^B + lo
                        const float v = vxy * wz[c];
                        const float hf = floorf(v * sp.inv2B);
                        const float lf = fmaf(-hf, sp.twoB, v);          // exact, in [0, 2^B)
                        const unsigned ql = __float_as_uint(lf + 8388608.0f) - 0x4B000000u;
                        atomicAdd(lo + row + cz, ql);
                        if (hf != 0.0f)
                            atomicAdd(hi + row + cz, (unsigned)(__float_as_int(hf + 12582912.0f) - 0x4B400000));
                    }
                } else {
                    const long long q = __float2ll_rn(vxy * wz[c]);
                    if (q) atomicAdd(acc64 + row + cz, (unsigned long long)q);
                }
            }
        }
    }
}

// MODE 2 deposit without branches: every one of the P^3 cells gets its
// atomic on sm[idx].  Per axis, an offset outside the tile is a large negative
// sentinel, so the index sum of a cell outside the tile is negative and
// min((unsigned)sum, trash) sends it to the lane's scratch word sm[trash]
// (never read); the lanes of a warp never split on tile bounds.  cell0: the
// first word of the mesh's cells in sm.
template <int P, int TC>
__device__ __forceinline__ void deposit_flat(unsigned *sm, int cell0, unsigned trash, int T, float x, float y,
                                             float z, float ws) {
    int bx, by, bz;
    float wx[P], wy[P], wz[P];
    spline_weights<P>(x, bx, wx);
    spline_weights<P>(y, by, wy);
    spline_weights<P>(z, bz, wz);
    const int TT = TC > 0 ? TC : T;
    constexpr int kOut = -(1 << 24);
    int ox[P], oy[P], oz[P];
#pragma unroll
    for (int a = 0; a < P; ++a) {
        const int cx = bx + a, cy = by + a, cz = bz + a;
        ox[a] = (unsigned)cx < (unsigned)TT ? cell0 + cx * TT * TT : kOut;
        oy[a] = (unsigned)cy < (unsigned)TT ? cy * TT : kOut;
        oz[a] = (unsigned)cz < (unsigned)TT ? cz : kOut;
    }
#pragma unroll
    for (int a = 0; a < P; ++a) {
        // TSC: skip an x plane that lies wholly outside the tile (measured
        // faster for TSC, slower for PCS, whose lanes diverge more)
        if (P == 3 && ox[a] == kOut) continue;
        const float vxw = ws * wx[a];
#pragma unroll
        for (int b = 0; b < P; ++b) {
            const float vxy = vxw * wy[b];
            const int oab = ox[a] + oy[b];
#pragma unroll
            for (int c = 0; c < P; ++c) {
                const unsigned q = __float_as_uint(fmaf(vxy, wz[c], 8388608.0f)) - 0x4B000000u;
                atomicAdd(sm + min((unsigned)(oab + oz[c]), trash), q);
            }
        }
    }
}

// ---- one-sweep paint of 16^3 tiles into a padded layout (unit weights, TSC and PCS) ----
// Shared layout: cell (x, y, z) of the tile's mesh m at word
//   m * kWords + x * kXS + y * kYS + kZlo + z,
// where every row of z holds a halo [-kZlo, kYS - kZlo) wide enough for every
// deposit of every window that reaches the tile along z (objects of the tile
// and the boundary classes of its neighbours, both meshes), so a deposit
// needs no bounds test along z; a window wholly outside the tile along z (the
// other mesh of a boundary candidate) and a row outside the tile along x or
// y are skipped by predicates (a word shared by many lanes of one atomic
// instruction would serialize them).  Each deposit is then one FFMA, one
// IADD and one 32-bit shared atomic at an immediate offset from its row.
//
// The strides are odd: candidates arrive grouped by (tile, boundary class),
// and on a lattice-like catalog a warp's lanes share z offsets, so with even
// strides (plane 384 = 0 mod 32 words, rows 24) their deposits fell on a few
// banks (5.1 shared wavefronts per atomic instruction measured on a
// Zel'dovich lattice at 0.125 objects per cell); rows of 25 and planes of 401
// words spread them over all 32 banks (PCS + interlacing 1.93 -> 1.22 ms on
// that lattice at 512^3, 1.01 -> 0.92 ms on the log-normal catalog; TSC
// with rows of 21 and planes of 337: 1.02 -> 0.69 and 0.537 -> 0.526 ms).
template <int P>
struct SweepLayout {
    static constexpr int T = 16;
    static constexpr int Zlo = P == 4 ? 4 : P - 1;    // z halo below the tile
    static constexpr int YS = P == 4 ? 25 : (P == 3 ? 21 : 19);   // row stride
    static constexpr int XS = P == 4 ? 401 : (P == 3 ? 337 : 305);  // plane stride
    static constexpr int Words = T * XS;              // one mesh (a multiple of 4 words)
    // first nodes of the windows that reach the tile along z: any other
    // window lies wholly outside it and deposits nothing
    static constexpr int BzMin = -Zlo, BzMax = YS - Zlo - P;
    static_assert(Zlo >= P - 1 && BzMax >= T - 1, "the halo must hold every window that reaches the tile");
    static_assert(XS >= T * YS && Words % 4 == 0, "rows inside their plane; 16-byte zeroing");
};

// Deposits of one candidate (tile-frame coordinates x, y, z in cells, weight
// ws already scaled by 2^S) into the mesh whose first word is sm.  A first
// node bz outside [BzMin, BzMax] only occurs for a window lying wholly
// outside the tile along z: it deposits nothing.
template <int P, bool SKIP_PLANES>
__device__ __forceinline__ void sweep_deposit(unsigned *sm, float x, float y, float z, float ws) {
    using Lay = SweepLayout<P>;
    constexpr int kOut = 1 << 20;                     // > Words: marks a row outside the tile
    int bx, by, bz;
    float wx[P], wy[P], wz[P];
    spline_weights<P>(x, bx, wx);
    spline_weights<P>(y, by, wy);
    spline_weights<P>(z, bz, wz);
    if (bz < Lay::BzMin || bz > Lay::BzMax) return;
    bz += Lay::Zlo;
    int ox[P], oy[P];
#pragma unroll
    for (int a = 0; a < P; ++a) {
        ox[a] = (unsigned)(bx + a) < (unsigned)Lay::T ? (bx + a) * Lay::XS : kOut;
        oy[a] = (unsigned)(by + a) < (unsigned)Lay::T ? (by + a) * Lay::YS + bz : kOut;
    }
#pragma unroll
    for (int a = 0; a < P; ++a) {
        if (SKIP_PLANES && ox[a] == kOut) continue;
        const float vxw = ws * wx[a];
#pragma unroll
        for (int b = 0; b < P; ++b) {
            const float vxy = vxw * wy[b];
            const int ro = ox[a] + oy[b];
            if (ro < Lay::Words) {           // a row inside the tile (no deposit otherwise)
                unsigned *row = sm + ro;
#pragma unroll
                for (int c = 0; c < P; ++c)
                    atomicAdd(row + c, __float_as_uint(fmaf(vxy, wz[c], 8388608.0f)) - 0x4B000000u);
            }
        }
    }
}

// Write mesh words of the padded layout (cells of the tile only) to the r2c
// mesh: two cells per thread and store, as flush_tile (two 32-bit loads: the
// odd strides leave a pair of cells 4-byte aligned only).
template <typename M, int P>
__device__ __forceinline__ void sweep_flush(const unsigned *sm, float inv_scale, M *__restrict__ dst0, int N,
                                            long long pitch, int accumulate) {
    using Lay = SweepLayout<P>;
    using M2 = typename std::conditional<sizeof(M) == 4, float2, double2>::type;
    constexpr int T = Lay::T, hT = T / 2;
    constexpr int planes = kPaintThreads / (hT * T);          // x planes per pass
    static_assert(kPaintThreads % (hT * T) == 0 && T % planes == 0, "flush mapping");
    const int t = threadIdx.x;
    const int cz = 2 * (t % hT);
    const int cy = (t / hT) % T;
    const int cx0 = t / (hT * T);
    int w = cx0 * Lay::XS + cy * Lay::YS + Lay::Zlo + cz;
    M *dst = dst0 + ((long long)cx0 * N + cy) * pitch + cz;
    const long long gstep = (long long)planes * N * pitch;
#pragma unroll 2
    for (int k = 0; k < T / planes; ++k, w += planes * Lay::XS, dst += gstep) {
        const uint2 l2 = make_uint2(sm[w], sm[w + 1]);
        M2 v;
        v.x = (M)l2.x * (M)inv_scale;
        v.y = (M)l2.y * (M)inv_scale;
        M2 *d2 = reinterpret_cast<M2 *>(dst);
        if (accumulate) {
            const M2 o = *d2;
            v.x += o.x;
            v.y += o.y;
        }
        *d2 = v;
    }
}

// Correctly rounded int64 -> float without the 64-bit conversion instruction.
__device__ __forceinline__ float ll_to_float_rn(long long q) {
    if (q == 0) return 0.0f;
    const unsigned long long u = q < 0 ? 0ull - (unsigned long long)q : (unsigned long long)q;
    const int nb = 64 - __clzll((long long)u);
    float f;
    if (nb <= 24) {
        f = (float)(unsigned)u;
    } else {
        const int sh = nb - 24;
        unsigned long long m = u >> sh;
        const unsigned long long rem = u & ((1ull << sh) - 1ull);
        const unsigned long long half = 1ull << (sh - 1);
        if (rem > half || (rem == half && (m & 1ull))) ++m;
        f = (float)(unsigned)m * __uint_as_float((unsigned)(127 + sh) << 23);
    }
    return q < 0 ? -f : f;
}

// Cell value in weight units from its fixed-point words.  FP32: the fast path
// rounds hi 2^(B-S) + lo 2^-S within one ulp (a fixed function of the integer
// words, so still bit-reproducible); the 64-bit path is rounded exactly.
// FP64: exact in both paths (the cell integer has far fewer than 53 bits).
template <typename M>
__device__ __forceinline__ M cell_value(unsigned lo, unsigned hi, unsigned long long a64, const Split &sp,
                                        float inv_scale);
template <>
__device__ __forceinline__ float cell_value<float>(unsigned lo, unsigned hi, unsigned long long a64,
                                                   const Split &sp, float inv_scale) {
    if (sp.fast) return fmaf((float)(int)hi, sp.hi_scale, (float)lo * inv_scale);
    return ll_to_float_rn((long long)a64) * inv_scale;
}
template <>
__device__ __forceinline__ double cell_value<double>(unsigned lo, unsigned hi, unsigned long long a64,
                                                     const Split &sp, float inv_scale) {
    if (sp.fast) return fma((double)(int)hi, (double)sp.hi_scale, (double)lo * (double)inv_scale);
    return __ll2double_rn((long long)a64) * (double)inv_scale;
}

// 2^k for -126 <= k <= 127, exactly (the fixed-point scales: S <= 40, B <= 22).
__device__ __forceinline__ float pow2f(int k) { return __uint_as_float((unsigned)(127 + k) << 23); }

__device__ __forceinline__ int ceil_log2(unsigned x) {     // x >= 1
    return x <= 1u ? 0 : 32 - __clz(x - 1u);
}

// Neighbour offset (-1, 0, +1 per axis) of gather segment s: s = (ax * 5 + ay)
// * 3 + az with ax, ay over the 5 (offset, class) pairs -- offset -1, three
// classes at offset 0, offset +1 -- and az over the 3 z offsets.
__device__ __forceinline__ int seg_dx(int s) { const int ax = s / 15; return ax == 0 ? -1 : (ax == 4 ? 1 : 0); }
__device__ __forceinline__ int seg_dy(int s) { const int ay = (s / 3) % 5; return ay == 0 ? -1 : (ay == 4 ? 1 : 0); }
__device__ __forceinline__ int seg_dz(int s) { return s % 3 - 1; }

// Candidate k of the tile (k < s_pre[kSegments]) in this tile's frame
// (segment shift added), weight scaled by 2^S.
__device__ __forceinline__ float4 fetch_candidate(const float4 *__restrict__ sorted, const uint32_t *s_beg,
                                                  const uint32_t *s_pre, int T, uint32_t k, float scale) {
    int lo_s = 0, hi_s = kSegments;                   // s_pre[lo_s] <= k < s_pre[hi_s]
    while (hi_s - lo_s > 1) {
        const int mid = (lo_s + hi_s) >> 1;
        if (s_pre[mid] <= k) lo_s = mid;
        else hi_s = mid;
    }
    const float4 v = __ldg(sorted + s_beg[lo_s] + (k - s_pre[lo_s]));
    return make_float4(v.x + (float)(seg_dx(lo_s) * T), v.y + (float)(seg_dy(lo_s) * T),
                       v.z + (float)(seg_dz(lo_s) * T), v.w * scale);
}

// Copy candidates [k0, k0 + n) of the tile into shared memory.
__device__ __forceinline__ void stage_candidates(const float4 *__restrict__ sorted, const uint32_t *s_beg,
                                                 const uint32_t *s_pre, int T, uint32_t k0, uint32_t n,
                                                 float scale, float4 *cand) {
    for (uint32_t j = threadIdx.x; j < n; j += blockDim.x)
        cand[j] = fetch_candidate(sorted, s_beg, s_pre, T, k0 + j, scale);
}

template <int P, int MODE, int TC>
__device__ __forceinline__ void deposit_staged(const float4 *cand, uint32_t n, unsigned *lo, unsigned *hi,
                                               unsigned long long *acc64, const Split &sp, int T, float sh) {
    for (uint32_t j = threadIdx.x; j < n; j += blockDim.x) {
        const float4 v = cand[j];
        deposit<P, MODE, TC>(lo, hi, acc64, sp, T, v.x + sh, v.y + sh, v.z + sh, v.w);
    }
}

template <int P, int TC>
__device__ __forceinline__ void deposit_any(const float4 *cand, uint32_t n, unsigned *lo, unsigned *hi,
                                            unsigned long long *acc64, const Split &sp, int T, float sh) {
    if (sp.fast == 2) deposit_staged<P, 2, TC>(cand, n, lo, hi, acc64, sp, T, sh);
    else if (sp.fast == 1) deposit_staged<P, 1, TC>(cand, n, lo, hi, acc64, sp, T, sh);
    else deposit_staged<P, 0, TC>(cand, n, lo, hi, acc64, sp, T, sh);
}

// Write one tile's cells to the mesh (r2c layout, rows of T cells along z at
// the given pitch).  Sources: lo alone (no split), lo + hi (split), or acc64
// (64-bit cells).  Even T: two cells per thread with 8- (FP32) or 16-byte
// (FP64) stores; the row pitch and tile origin are even, so they are aligned.
template <typename M, int TC>
__device__ __forceinline__ void flush_tile(const unsigned *lo, const unsigned *hi, const unsigned long long *acc64,
                                           const Split &sp, float inv_scale, M *__restrict__ mb, int T, int N,
                                           long long pitch, int accumulate) {
    using M2 = typename std::conditional<sizeof(M) == 4, float2, double2>::type;
    constexpr int kPlane = TC > 0 ? (TC / 2) * TC : 1;                 // cell pairs per x-plane
    constexpr bool kFixed = TC > 0 && TC % 2 == 0 && kPaintThreads % kPlane == 0 &&
                            TC % (kPaintThreads / kPlane) == 0;
    if constexpr (kFixed) {
        // each pass of the CTA covers whole x-planes: a thread keeps its
        // (cy, cz) and steps cx by a fixed stride, in shared and global memory
        constexpr int hT = TC > 0 ? TC / 2 : 1;
        constexpr int planes = kFixed ? kPaintThreads / kPlane : 1;
        const int t = threadIdx.x;
        const int cz = 2 * (t % hT);
        const int cy = (t / hT) % TC;
        const int cx0 = t / (hT * TC);
        int c = (cx0 * TC + cy) * TC + cz;
        M *dst = mb + ((long long)cx0 * N + cy) * pitch + cz;
        const long long gstep = (long long)planes * N * pitch;
#pragma unroll 2
        for (int k = 0; k < TC / planes; ++k, c += planes * TC * TC, dst += gstep) {
            M2 v;
            if (acc64) {
                v.x = cell_value<M>(0u, 0u, acc64[c], sp, inv_scale);
                v.y = cell_value<M>(0u, 0u, acc64[c + 1], sp, inv_scale);
            } else {
                const uint2 l2 = *reinterpret_cast<const uint2 *>(lo + c);
                const uint2 h2 = hi ? *reinterpret_cast<const uint2 *>(hi + c) : make_uint2(0u, 0u);
                v.x = cell_value<M>(l2.x, h2.x, 0ull, sp, inv_scale);
                v.y = cell_value<M>(l2.y, h2.y, 0ull, sp, inv_scale);
            }
            M2 *d2 = reinterpret_cast<M2 *>(dst);
            if (accumulate) {
                const M2 o = *d2;
                v.x += o.x;
                v.y += o.y;
            }
            *d2 = v;
        }
    } else if ((T & 1) == 0) {
        const int hT = T >> 1;
        const int npairs = T * T * hT;
        for (int p = threadIdx.x; p < npairs; p += blockDim.x) {
            const int r = TC > 0 ? p / (TC / 2) : p / hT;           // row = cx T + cy
            const int cz = 2 * (p - r * hT);
            const int cx = TC > 0 ? r / TC : r / T;
            const int cy = r - cx * T;
            const int c = r * T + cz;
            M2 v;
            if (acc64) {
                v.x = cell_value<M>(0u, 0u, acc64[c], sp, inv_scale);
                v.y = cell_value<M>(0u, 0u, acc64[c + 1], sp, inv_scale);
            } else {
                const uint2 l2 = *reinterpret_cast<const uint2 *>(lo + c);
                const uint2 h2 = hi ? *reinterpret_cast<const uint2 *>(hi + c) : make_uint2(0u, 0u);
                v.x = cell_value<M>(l2.x, h2.x, 0ull, sp, inv_scale);
                v.y = cell_value<M>(l2.y, h2.y, 0ull, sp, inv_scale);
            }
            M2 *dst = reinterpret_cast<M2 *>(mb + ((long long)cx * N + cy) * pitch + cz);
            if (accumulate) {
                const M2 o = *dst;
                v.x += o.x;
                v.y += o.y;
            }
            *dst = v;
        }
    } else {
        const int n = T * T * T;
        for (int c = threadIdx.x; c < n; c += blockDim.x) {
            const int r = c / T, cz = c - r * T;
            const int cx = r / T, cy = r - cx * T;
            const M val = acc64 ? cell_value<M>(0u, 0u, acc64[c], sp, inv_scale)
                                : cell_value<M>(lo[c], hi ? hi[c] : 0u, 0ull, sp, inv_scale);
            M *dst = mb + ((long long)cx * N + cy) * pitch + cz;
            if (accumulate) *dst += val;
            else *dst = val;
        }
    }
}

// TC > 0: the tile edge is the compile-time constant TC (index math in shifts).
template <int P, int NM, typename M, int TC>
__global__ void __launch_bounds__(kPaintThreads)
k_paint_tiles(const float4 *__restrict__ sorted, const uint32_t *__restrict__ off, PaintGeom g,
              int S, const unsigned *__restrict__ wmax_bits, float wmax_deposit, M *__restrict__ mesh,
              long long item_stride, long long mesh_stride, int accumulate) {
    extern __shared__ __align__(16) unsigned smu[];   // lo[T^3], hi[T^3] or acc64[T^3]; cand[kStage]
    __shared__ uint32_t s_beg[kSegments];
    __shared__ uint32_t s_pre[kSegments + 1];
    const int T = TC > 0 ? TC : g.T, T3 = T * T * T;
    unsigned *lo = smu, *hi = smu + T3;
    unsigned long long *acc64 = reinterpret_cast<unsigned long long *>(smu);
    float4 *cand = reinterpret_cast<float4 *>(smu + 2 * T3);

    // item * ntiles + tile (the launch keeps the block count below 2^31, so
    // 32-bit unsigned division suffices: 64-bit division is a long software
    // sequence that every thread of every tile would run)
    const unsigned gt = blockIdx.x;
    const unsigned ntiles = (unsigned)g.ntiles, ntx = (unsigned)g.ntx;
    const unsigned item = gt / ntiles;
    const unsigned t = gt - item * ntiles;
    const unsigned tq = t / ntx;
    const int tz = (int)(t - tq * ntx);
    const int tx = (int)(tq / ntx);
    const int ty = (int)(tq - (unsigned)tx * ntx);

    // Segments: neighbour offset d (per axis -1, 0, +1) with the classes of
    // that neighbour whose window reaches this tile: d = -1 -> class 2,
    // d = 0 -> any class, d = +1 -> class 0.  Index s = (ax * 5 + ay) * 3 + az
    // with ax, ay over the 5 (d, class) pairs and az over the 3 z offsets
    // (whose class ranges are contiguous keys).
    if (threadIdx.x < kSegments) {
        const int s = threadIdx.x;
        const int ax = s / 15, ay = (s / 3) % 5, az = s % 3;
        const int dx = ax == 0 ? -1 : (ax == 4 ? 1 : 0), cx = ax == 0 ? 2 : (ax == 4 ? 0 : ax - 1);
        const int dy = ay == 0 ? -1 : (ay == 4 ? 1 : 0), cy = ay == 0 ? 2 : (ay == 4 ? 0 : ay - 1);
        const int dz = az - 1;
        const int cz0 = dz == -1 ? 2 : 0, cz1 = dz == 1 ? 0 : 2;
        const int n = g.ntx;
        const int wx = tx + dx < 0 ? tx + dx + n : (tx + dx >= n ? tx + dx - n : tx + dx);
        const int wy = ty + dy < 0 ? ty + dy + n : (ty + dy >= n ? ty + dy - n : ty + dy);
        const int wz = tz + dz < 0 ? tz + dz + n : (tz + dz >= n ? tz + dz - n : tz + dz);
        const int64_t nt = ((int64_t)wx * n + wy) * n + wz;
        const int64_t kb = ((int64_t)item * g.ntiles + nt) * kClasses + cx * 9 + cy * 3;
        const uint32_t b = off[kb + cz0], e = off[kb + cz1 + 1];
        s_beg[s] = b;
        s_pre[s + 1] = e - b;
    }
    __syncthreads();
    if (threadIdx.x < 32) {                          // warp scan of the 75 lengths
        const int lane = threadIdx.x;
        uint32_t v0 = 0, v1 = 0, v2 = 0;
        if (3 * lane < kSegments) v0 = s_pre[3 * lane + 1];
        if (3 * lane + 1 < kSegments) v1 = s_pre[3 * lane + 2];
        if (3 * lane + 2 < kSegments) v2 = s_pre[3 * lane + 3];
        uint32_t x = v0 + v1 + v2;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        const uint32_t before = x - (v0 + v1 + v2);
        __syncwarp();
        if (lane == 0) s_pre[0] = 0;
        if (3 * lane < kSegments) s_pre[3 * lane + 1] = before + v0;
        if (3 * lane + 1 < kSegments) s_pre[3 * lane + 2] = before + v0 + v1;
        if (3 * lane + 2 < kSegments) s_pre[3 * lane + 3] = before + v0 + v1 + v2;
    }
    __syncthreads();
    const uint32_t total = s_pre[kSegments];

    Split sp;
    {
        const unsigned nc = total > 0u ? total : 1u;
        sp.B = min(22, 31 - ceil_log2(nc));
        sp.twoB = __uint_as_float((unsigned)(127 + max(sp.B, 0)) << 23);
        sp.twoB_u = 1u << max(sp.B, 0);
        sp.inv2B = __uint_as_float((unsigned)(127 - max(sp.B, 0)) << 23);
        sp.hi_scale = pow2f(sp.B - S);
        const float wmax = __uint_as_float(wmax_bits[item]);
        const float hmax = wmax * pow2f(S - sp.B);
        sp.fast = sp.B >= 1 && hmax < 4194304.0f && (float)nc * (hmax + 1.0f) < 2.0e9f;
        // wmax_deposit > 0: all weights are in [0, wmax_deposit / max W]; then
        // no deposit reaches 2^B if wmax_deposit 2^S < 2^B - 1
        if (sp.fast && wmax_deposit > 0.0f && wmax_deposit * pow2f(S) < (float)(sp.twoB_u - 1u)) sp.fast = 2;
    }
    const float scale = pow2f(S);
    const float inv_scale = pow2f(-S);
    // With no split needed (unit weights, sparse tile) the tile is painted in
    // one sweep over its candidates, each read once straight from the sorted
    // copy (nothing to stage), with branch-free deposits; an interlaced pair
    // goes into lo (mesh 0) and hi (mesh 1) together.
    const bool sweep = sp.fast == 2;
    // TSC and PCS sweeps of 16^3 tiles deposit into the padded layout
    // (SweepLayout); CIC keeps the compact one (its padded layout with even
    // strides measured 0.69 against 0.54 ms)
    const bool kPadded = sweep && TC == 16 && (P == 4 || P == 3);
    const bool staged_once = total <= (uint32_t)kStage;
    if (staged_once && !sweep) stage_candidates(sorted, s_beg, s_pre, T, 0u, total, scale, cand);
    const long long pitch = 2LL * (g.N / 2 + 1);
    M *base = mesh + item * item_stride;

    const int passes = sweep ? 1 : NM;
    const long long tile_off = ((long long)tx * T * g.N + (long long)ty * T) * pitch + (long long)tz * T;
#pragma unroll 1
    for (int m = 0; m < passes; ++m) {
        {
            uint4 *z4 = reinterpret_cast<uint4 *>(smu);
            const int nw = kPadded ? NM * SweepLayout<P>::Words
                                   : ((sweep && NM == 1) ? T3 : 2 * T3);   // a single unsplit mesh uses lo only
            const int n4 = nw / 4;
            for (int c = threadIdx.x; c < n4; c += blockDim.x) z4[c] = make_uint4(0u, 0u, 0u, 0u);
            for (int c = 4 * n4 + threadIdx.x; c < nw; c += blockDim.x) smu[c] = 0u;
        }
        __syncthreads();
        const float sh = m ? 0.5f : 0.0f;
        if (kPadded) {
            // one-sweep deposits into the padded layout (SweepLayout), both meshes
            for (uint32_t k = threadIdx.x; k < total; k += blockDim.x) {
                const float4 v = fetch_candidate(sorted, s_beg, s_pre, T, k, scale);
                sweep_deposit<P, false>(smu, v.x, v.y, v.z, v.w);
                if (NM == 2)
                    sweep_deposit<P, false>(smu + SweepLayout<P>::Words, v.x + 0.5f, v.y + 0.5f, v.z + 0.5f,
                                             v.w);
            }
        } else if (sweep) {
            // the staging area is unused here: its first 32 words are the lanes' scratch
            const unsigned trash = (unsigned)(2 * T3) + (threadIdx.x & 31);
            const bool flat = total <= (uint32_t)kFlatMaxCand;
            for (uint32_t k = threadIdx.x; k < total; k += blockDim.x) {
                const float4 v = fetch_candidate(sorted, s_beg, s_pre, T, k, scale);
                if (flat) {
                    deposit_flat<P, TC>(smu, 0, trash, T, v.x, v.y, v.z, v.w);
                    if (NM == 2) deposit_flat<P, TC>(smu, T3, trash, T, v.x + 0.5f, v.y + 0.5f, v.z + 0.5f, v.w);
                } else {
                    deposit<P, 2, TC>(lo, nullptr, nullptr, sp, T, v.x, v.y, v.z, v.w);
                    if (NM == 2) deposit<P, 2, TC>(hi, nullptr, nullptr, sp, T, v.x + 0.5f, v.y + 0.5f, v.z + 0.5f, v.w);
                }
            }
        } else if (staged_once) {
            deposit_any<P, TC>(cand, total, lo, hi, acc64, sp, T, sh);
        } else {
            for (uint32_t k0 = 0; k0 < total; k0 += kStage) {     // dense tile: batches
                const uint32_t n = min((uint32_t)kStage, total - k0);
                __syncthreads();                                  // previous batch consumed
                stage_candidates(sorted, s_beg, s_pre, T, k0, n, scale, cand);
                __syncthreads();
                deposit_any<P, TC>(cand, n, lo, hi, acc64, sp, T, sh);
            }
        }
        __syncthreads();
        if (kPadded) {
            sweep_flush<M, P>(smu, inv_scale, base + tile_off, g.N, pitch, accumulate);
            if (NM == 2)
                sweep_flush<M, P>(smu + SweepLayout<P>::Words, inv_scale, base + mesh_stride + tile_off, g.N, pitch,
                                  accumulate);
        } else if (sweep) {
            flush_tile<M, TC>(lo, nullptr, nullptr, sp, inv_scale, base + tile_off, T, g.N, pitch, accumulate);
            if (NM == 2)
                flush_tile<M, TC>(hi, nullptr, nullptr, sp, inv_scale, base + mesh_stride + tile_off, T, g.N, pitch,
                                  accumulate);
        } else {
            flush_tile<M, TC>(sp.fast ? lo : nullptr, sp.fast == 1 ? hi : nullptr, sp.fast ? nullptr : acc64, sp,
                              inv_scale, base + m * mesh_stride + tile_off, T, g.N, pitch, accumulate);
        }
        __syncthreads();
    }
}

// ---- direct atomic paint (the variant without a sort) ----
// Per object: the same wrapped cell coordinate as the sort path, cell
// c0 = floor(s) and offset u = (s - c0) + e along each axis; every deposit
// round(w 2^S W) is added with a 64-bit global atomic (RED) into a dense
// N^3 int64 accumulator per mesh.  Integer adds keep the accumulator
// independent of object order.  The accumulator is converted and cleared by
// k_acc_to_mesh.
template <int P>
__device__ __forceinline__ void deposit_global(unsigned long long *__restrict__ acc, int N,
                                               const int *c0, const float *u, float sh, float ws) {
    int bx, by, bz;
    float wx[P], wy[P], wz[P];
    spline_weights<P>(u[0] + sh, bx, wx);
    spline_weights<P>(u[1] + sh, by, wy);
    spline_weights<P>(u[2] + sh, bz, wz);
    int cz[P];
#pragma unroll
    for (int c = 0; c < P; ++c) {
        int v = c0[2] + bz + c;
        v = v < 0 ? v + N : (v >= N ? v - N : v);
        cz[c] = v;
    }
#pragma unroll
    for (int a = 0; a < P; ++a) {
        int cx = c0[0] + bx + a;
        cx = cx < 0 ? cx + N : (cx >= N ? cx - N : cx);
        const float vx = ws * wx[a];
#pragma unroll
        for (int b = 0; b < P; ++b) {
            int cy = c0[1] + by + b;
            cy = cy < 0 ? cy + N : (cy >= N ? cy - N : cy);
            const float vxy = vx * wy[b];
            unsigned long long *row = acc + ((long long)cx * N + cy) * N;
#pragma unroll
            for (int c = 0; c < P; ++c) {
                // round(v) in one FMA when 0 <= round(v) < 2^22, else the
                // rounded product converted to int64
                const float t = fmaf(vxy, wz[c], 8388608.0f);
                long long q;
                if (t >= 8388608.0f && t < 12582912.0f) q = (long long)(__float_as_uint(t) - 0x4B000000u);
                else q = __float2ll_rn(vxy * wz[c]);
                if (q) atomicAdd(row + cz[c], (unsigned long long)q);
            }
        }
    }
}

template <int DT, int P, int NM>
__global__ void __launch_bounds__(kCountThreads)
k_paint_atomic(const void *__restrict__ pos, const float *__restrict__ w, const float *__restrict__ vals,
               const int64_t *__restrict__ item_off, PaintGeom g, int S, bool weighted,
               unsigned long long *__restrict__ acc, double *__restrict__ wsums,
               double *__restrict__ wpart, unsigned *__restrict__ wmax) {
    using R = typename PosReal<DT>::type;
    const int item = blockIdx.y;
    const int64_t beg = item_off[item], end = item_off[item + 1];
    const long long n3 = (long long)g.N * g.N * g.N;
    unsigned long long *ab = acc + (long long)item * NM * n3;
    const float scale = ldexpf(1.0f, S);
    double sw = 0.0, sw2 = 0.0, swa = 0.0;
    float mw = 0.0f;
    for (int64_t i = beg + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < end;
         i += (int64_t)gridDim.x * blockDim.x) {
        const Obj<R> o = load_obj<DT>(pos, w, vals, i, g);
        int c0[3];
        float u[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            c0[a] = min((int)floor(o.s[a]), g.N - 1);
            u[a] = (float)(o.s[a] - (R)c0[a]) + o.e[a];
        }
        const float ws = o.a * scale;
#pragma unroll
        for (int m = 0; m < NM; ++m) deposit_global<P>(ab + m * n3, g.N, c0, u, m ? 0.5f : 0.0f, ws);
        if (weighted) {
            const double ad = (double)o.a;
            sw += (double)o.w;
            sw2 += ad * ad;
            swa += fabs(ad);
            mw = fmaxf(mw, fabsf(o.a));
        }
    }
    flush_wsums(sw, sw2, swa, mw, weighted, item, end - beg, wsums, wpart, wmax);
}

template <typename M>
__device__ __forceinline__ M acc_value(unsigned long long q, float inv_scale);
template <>
__device__ __forceinline__ float acc_value<float>(unsigned long long q, float inv_scale) {
    return ll_to_float_rn((long long)q) * inv_scale;
}
template <>
__device__ __forceinline__ double acc_value<double>(unsigned long long q, float inv_scale) {
    return __ll2double_rn((long long)q) * (double)inv_scale;
}

// Dense int64 accumulators (nitems x nm x N^3, z fastest) -> the r2c padded
// mesh layout, two cells per thread; each accumulator pair is cleared after
// it is read so the next paint starts from zero.
template <typename M>
__global__ void __launch_bounds__(256)
k_acc_to_mesh(ulonglong2 *__restrict__ acc, long long npairs, int N, int nm, float inv_scale,
              M *__restrict__ mesh, long long item_stride, long long mesh_stride, int accumulate) {
    using M2 = typename std::conditional<sizeof(M) == 4, float2, double2>::type;
    const long long n3 = (long long)N * N * N;
    const long long pitch = 2LL * (N / 2 + 1);
    for (long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x; j < npairs;
         j += (long long)gridDim.x * blockDim.x) {
        const long long cell = 2 * j;
        const long long im = cell / n3;
        const long long r = cell - im * n3;
        const long long row = r / N;
        const int cz = (int)(r - row * N);
        const long long item = im / nm;
        const int m = (int)(im - item * nm);
        const ulonglong2 q = acc[j];
        acc[j] = make_ulonglong2(0ull, 0ull);
        M *dst = mesh + item * item_stride + m * mesh_stride + row * pitch + cz;
        M2 v;
        v.x = acc_value<M>(q.x, inv_scale);
        v.y = acc_value<M>(q.y, inv_scale);
        if (accumulate) {
            const M2 o = *reinterpret_cast<const M2 *>(dst);
            v.x += o.x;
            v.y += o.y;
        }
        *reinterpret_cast<M2 *>(dst) = v;
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

__host__ __device__ __forceinline__ size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

template <typename R, typename C, typename A>
struct BinSmem {
    // layout: hist[nh] (A), cw_l[Nh] (R), ph_l[Nh] (C), edge pairs[nk] (int2: m range of bin b)
    __host__ __device__ static size_t off_cw(const BinGeom &g) { return align_up((size_t)g.nh * sizeof(A), 16); }
    // the cw and ph tables hold Nh + Nh/4 + 1 entries: k_bin stores entry l at l + l/4
    __host__ __device__ static size_t tab(const BinGeom &g) { return (size_t)g.Nh + (size_t)(g.Nh >> 2) + 1; }
    __host__ __device__ static size_t off_ph(const BinGeom &g) { return align_up(off_cw(g) + tab(g) * sizeof(R), 16); }
    __host__ __device__ static size_t off_edge(const BinGeom &g) { return align_up(off_ph(g) + tab(g) * sizeof(C), 16); }
    __host__ __device__ static size_t bytes(const BinGeom &g) { return align_up(off_edge(g) + (size_t)g.nk * sizeof(int2), 16); }
};

// floor(sqrt(x)) for 0 <= x < 2^26, exact.
__device__ __forceinline__ int isqrt_floor(int x) {
    int s = (int)sqrtf((float)x);
    while (s > 0 && s * s > x) --s;
    while ((s + 1) * (s + 1) <= x) ++s;
    return s;
}

// Fused compensate + interlace + bin.  Rows are the unit of work: each warp
// takes whole rows (i, j) and visits only the l range whose modes fall in a k
// bin, mlo <= i'^2 + j'^2 + l^2 < mhi (and m != 0); each lane sums kBinVec
// consecutive modes of it in registers and flushes a run to the per-CTA
// shared histogram when its bin changes.  CROSS: the meshes of a second
// catalog at meshb; each mode contributes Re(delta_a conj(delta_b)) instead
// of |delta|^2.  MU32: the mu-bin test q^2 m <= nmu^2 l^2 fits in 32 bits.
template <bool IL, bool TWOD, bool POLES, typename R, typename C, typename A, bool CROSS = false, bool MU32 = true>
__global__ void __launch_bounds__(kBinThreads, sizeof(R) == 4 ? 5 : 1)
k_bin(const C *__restrict__ mesh, long long item_stride_c, long long mesh_stride_c, BinGeom g,
      const R *__restrict__ cw, const C *__restrict__ ph, const int *__restrict__ kedge, A *__restrict__ partial,
      const C *__restrict__ meshb) {
    using SM = BinSmem<R, C, A>;
    extern __shared__ __align__(16) unsigned char smraw[];
    A *hist = reinterpret_cast<A *>(smraw);
    R *scw = reinterpret_cast<R *>(smraw + SM::off_cw(g));
    C *sph = reinterpret_cast<C *>(smraw + SM::off_ph(g));
    int2 *sedge = reinterpret_cast<int2 *>(smraw + SM::off_edge(g));
    for (int k = threadIdx.x; k < g.nh; k += blockDim.x) hist[k] = (A)0;
    // entry l at l + l/4: lanes read l = l0 + 4 lane + v, which this skew
    // spreads over all banks (4-byte cw) or two wavefronts (8-byte ph)
    for (int k = threadIdx.x; k < g.Nh; k += blockDim.x) {
        scw[k + (k >> 2)] = cw[k];
        sph[k + (k >> 2)] = ph[k + g.N / 2];
    }
    for (int k = threadIdx.x; k < g.nk; k += blockDim.x) sedge[k] = make_int2(kedge[k], kedge[k + 1]);
    __syncthreads();

    const int item = blockIdx.y;
    const C *m1 = mesh + (long long)item * item_stride_c;
    const C *m2 = m1 + mesh_stride_c;
    const C *n1 = CROSS ? meshb : m1;
    const C *n2 = n1 + mesh_stride_c;
    const int half = g.N / 2, N = g.N, Nh = g.Nh;
    const int nk = g.nk, nmu = g.nmu, hbase = g.hbase;
    const float kscale = g.kscale, koff = g.koff;
    const int lane = threadIdx.x & 31;
    const int wpb = blockDim.x >> 5;
    const int rows = N * N;
    for (int row = blockIdx.x * wpb + (threadIdx.x >> 5); row < rows; row += gridDim.x * wpb) {
        const int i = row / N, j = row - i * N;
        const int ip = i < half ? i : i - N;
        const int jp = j < half ? j : j - N;
        const int r2 = ip * ip + jp * jp;
        if (r2 >= g.mhi) continue;
        const int lhi = min(Nh, isqrt_floor(g.mhi - 1 - r2) + 1);
        int llo = g.mlo > r2 ? isqrt_floor(g.mlo - r2 - 1) + 1 : 0;
        if (r2 == 0 && llo == 0) llo = 1;
        if (llo >= lhi) continue;
        R rowcw = cw[i] * cw[j];
        C rowph;
        rowph.x = (R)0;
        rowph.y = (R)0;
        if (IL) {
            rowcw *= (R)0.25;
            rowph = cmul(ph[ip + half], ph[jp + half]);
        }
        const long long base = (long long)row * Nh;
        for (int l0 = llo + kBinVec * lane; l0 < lhi; l0 += 32 * kBinVec) {
            const int cnt = lhi - l0;                   // modes of this run: min(cnt, kBinVec)
            C a[kBinVec], b2[kBinVec], ca[CROSS ? kBinVec : 1], cb2[CROSS && IL ? kBinVec : 1];
#pragma unroll
            for (int v = 0; v < kBinVec; ++v) {
                const long long at = base + l0 + min(v, cnt - 1);   // the tail re-reads the last mode
                a[v] = __ldcs(m1 + at);
                if (IL) b2[v] = __ldcs(m2 + at);
                if (CROSS) {
                    ca[CROSS ? v : 0] = __ldcs(n1 + at);
                    if (IL) cb2[CROSS && IL ? v : 0] = __ldcs(n2 + at);
                }
            }
            int cur2 = -1, cur1 = -1;                 // open register runs
            R run2 = (R)0, runm2 = (R)0, runm4 = (R)0;
#pragma unroll
            for (int v = 0; v < kBinVec; ++v) {
                const bool live = v < cnt;
                const int l = min(l0 + v, lhi - 1);
                const int m = r2 + l * l;
                // FP32 estimate of the k bin, then one exact step against the FP64
                // edges: the estimate's error (below 4e-7 kmax / dk + 0.1, the
                // plan requires kmax / dk < 2^20) puts it at most one bin off
                const float rsm = rsqrtf((float)m);
                int b = (int)((float)m * rsm * kscale - koff);
                b = min(max(b, 0), nk - 1);
                {
                    const int2 e = sedge[b];
                    b += (int)(m >= e.y) - (int)(m < e.x);
                }
                C z = a[v];
                C y;
                if (CROSS) y = ca[CROSS ? v : 0];
                if (IL) {
                    const C t = cmul(rowph, sph[l + (l >> 2)]);
                    z.x += b2[v].x * t.x - b2[v].y * t.y;
                    z.y += b2[v].x * t.y + b2[v].y * t.x;
                    if (CROSS) {
                        const C u = cb2[CROSS && IL ? v : 0];
                        y.x += u.x * t.x - u.y * t.y;
                        y.y += u.x * t.y + u.y * t.x;
                    }
                }
                R pw = (CROSS ? z.x * y.x + z.y * y.y : z.x * z.x + z.y * z.y) * rowcw * scw[l + (l >> 2)];
                pw *= (R)((l != 0 && l != half) ? 2 : 1) * (R)(live ? 1 : 0);
                int key = b;
                if (TWOD) {
                    // mu bin: FP32 estimate, then one exact integer step each way
                    int q = (int)((float)(nmu * l) * rsm);
                    q = min(max(q, 0), nmu - 1);
                    if (MU32) {
                        const unsigned rhs = (unsigned)(nmu * nmu) * (unsigned)(l * l);
                        q -= (int)(q > 0 && (unsigned)(q * q) * (unsigned)m > rhs);
                        q += (int)(q < nmu - 1 && (unsigned)((q + 1) * (q + 1)) * (unsigned)m <= rhs);
                    } else {
                        const long long rhs = (long long)nmu * nmu * l * l;
                        q -= (int)(q > 0 && (long long)q * q * m > rhs);
                        q += (int)(q < nmu - 1 && (long long)(q + 1) * (q + 1) * m <= rhs);
                    }
                    key = b * nmu + q;
                }
                // flush an open run when the key changes (predicated, no branch)
                const bool new2 = key != cur2;
                if (new2 && cur2 >= 0) atomicAdd(hist + cur2, (A)run2);
                run2 = new2 ? pw : run2 + pw;
                cur2 = key;
                if (POLES) {
                    // FP32: mu = l rsqrt(m) from the k-bin estimate (a few ulp);
                    // FP64: the exact quotient.  The sums are of P L_2(mu) and
                    // P L_4(mu) themselves, not of P mu^2 and P mu^4: forming
                    // P_4 from mu moments (35 M4 - 30 M2 + 3 S0) would amplify
                    // the FP32 partial sums' rounding about forty-fold.
                    R mu2;
                    if (sizeof(R) == 4) {
                        const float mu = (float)l * rsm;
                        mu2 = (R)(mu * mu);
                    } else {
                        mu2 = (R)(l * l) / (R)m;
                    }
                    const R t2 = pw * ((R)1.5 * mu2 - (R)0.5);
                    const R t4 = pw * (((R)4.375 * mu2 - (R)3.75) * mu2 + (R)0.375);
                    const bool new1 = b != cur1;
                    if (new1 && cur1 >= 0) {
                        atomicAdd(hist + hbase + cur1, (A)runm2);
                        atomicAdd(hist + hbase + nk + cur1, (A)runm4);
                    }
                    runm2 = new1 ? t2 : runm2 + t2;
                    runm4 = new1 ? t4 : runm4 + t4;
                    cur1 = b;
                }
            }
            atomicAdd(hist + cur2, (A)run2);
            if (POLES) {
                atomicAdd(hist + hbase + cur1, (A)runm2);
                atomicAdd(hist + hbase + nk + cur1, (A)runm4);
            }
        }
    }
    __syncthreads();
    A *out = partial + ((long long)item * gridDim.x + blockIdx.x) * g.nh;
    for (int k = threadIdx.x; k < g.nh; k += blockDim.x) out[k] = hist[k];
}

// sums2[(item * nchunk + chunk) * nh + k] = sum of the chunk's per-CTA histograms, in order.
// out_rows: rows per catalog in sums2 (a second pass over sums2 itself, with
// G = out_rows, sums each column of a catalog's rows into its row 0 in place:
// a thread reads and writes only its own column).
template <typename A>
__global__ void k_bin_reduce(const A *__restrict__ partial, int G, int nh, int out_rows,
                             double *__restrict__ sums2) {
    const int item = blockIdx.z, chunk = blockIdx.y;
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nh) return;
    const int c0 = chunk * kReduceChunk, c1 = min(G, c0 + kReduceChunk);
    const A *p = partial + ((long long)item * G) * nh + k;
    double s = 0.0;
    for (int c = c0; c < c1; ++c) s += (double)p[(long long)c * nh];
    sums2[((long long)item * out_rows + chunk) * nh + k] = s;
}

// Auto power of every catalog (cross_b < 0: block = catalog), or the cross
// power of catalogs cross_a and cross_b (one block): normalization
// L^3 / (sum w_a sum w_b), no shot noise; the result block then carries
// sum w_a and sum w_b in its wsum and w2sum slots.
__global__ void k_finalize(const double *__restrict__ sums2, int nchunk, int nsum,
                           const unsigned long long *__restrict__ modes1d,
                           const unsigned long long *__restrict__ modes2d,
                           const double *__restrict__ wsums, const int *__restrict__ err,
                           FinalGeom f, ResultLayout rl, double *__restrict__ res, int cross_a, int cross_b) {
    const bool cross = cross_b >= 0;
    const int item = blockIdx.x;
    const int ia = cross ? cross_a : item, ib = cross ? cross_b : item;
    const double *s0 = sums2 + (long long)item * nchunk * f.nh;
    double *r = res + (long long)item * f.RL;
    const double wsum = wsums[4 * ia], wsum_b = wsums[4 * ib];
    const double w2sum = cross ? wsum_b : wsums[4 * ia + 1];
    const double wabs = fmax(wsums[4 * ia + 2], wsums[4 * ib + 2]);
    const double norm = f.L3 / (wsum * wsum_b);
    const double shot = cross ? 0.0 : f.L3 * w2sum / (wsum * wsum);
    const double sub = f.subtract_shot ? shot : 0.0;
    const double nan = __longlong_as_double(0x7ff8000000000000LL);
    auto S = [&](int k) {
        double t = 0.0;
        for (int c = 0; c < nsum; ++c) t += s0[(long long)c * f.nh + k];
        return t;
    };
    // bins spread over the gridDim.y blocks of the catalog (FP64 divisions are
    // slow on this part: one block took ~30 us for 3500 bins)
    const int t0 = blockIdx.y * blockDim.x + threadIdx.x, tstride = gridDim.y * blockDim.x;
    for (int b = t0; b < f.nk; b += tstride) {
        double S0 = 0.0;
        if (f.twod) {
            for (int q = 0; q < f.nmu; ++q) S0 += S(b * f.nmu + q);
        } else {
            S0 = S(b);
        }
        const double cnt = (double)modes1d[b];
        double p0 = nan, p2 = nan, p4 = nan;
        if (cnt > 0.0) {
            p0 = norm * S0 / cnt - sub;
            if (f.poles) {               // slots: sum h P L_2(mu), sum h P L_4(mu)
                p2 = 5.0 * norm * S(f.hbase + b) / cnt;
                p4 = 9.0 * norm * S(f.hbase + f.nk + b) / cnt;
            }
        }
        r[rl.pk + b] = p0;
        r[rl.poles + b] = (f.poles_mask & 1u) ? p0 : nan;
        r[rl.poles + f.nk + b] = (f.poles_mask & 2u) ? p2 : nan;
        r[rl.poles + 2 * f.nk + b] = (f.poles_mask & 4u) ? p4 : nan;
    }
    if (f.twod) {
        for (int bq = t0; bq < f.nk * f.nmu; bq += tstride) {
            const double cnt = (double)modes2d[bq];
            r[rl.pkmu + bq] = cnt > 0.0 ? norm * S(bq) / cnt - sub : nan;
        }
    }
    if (blockIdx.y == 0 && threadIdx.x == 0) {
        r[rl.shot] = shot;
        r[rl.wsum] = wsum;
        r[rl.w2sum] = w2sum;
        r[rl.flags] = (double)(((wabs > f.headroom) ? 1 : 0) | (*err & 2));
    }
}

// ---- projected power (ProjectedFFTPower): one plane or line of the transform ----
// By the projection-slice theorem the d-dimensional transform of the field
// summed over the dropped axes is the 3D transform at index 0 along them, so
// the projected power needs only those modes.  Each mode of the plane: the
// usual interlacing combine and compensation, |delta|^2 (times the half-grid
// weight h when z is kept), exact k bin from the m-edge table, FP64 atomics
// into count / sum h k / sum h |F|^2 cw per bin.
template <typename R, typename C>
__global__ void k_plane_bin(const C *__restrict__ m1, const C *__restrict__ m2, int N, int keep_mask,
                            const R *__restrict__ cw, const C *__restrict__ ph, const int *__restrict__ kedge,
                            int nk, double kF, double *__restrict__ sums) {
    const int Nh = N / 2 + 1;
    const int nx = (keep_mask & 1) ? N : 1, ny = (keep_mask & 2) ? N : 1, nz = (keep_mask & 4) ? Nh : 1;
    const long long total = (long long)nx * ny * nz;
    const int half = N / 2;
    for (long long f = (long long)blockIdx.x * blockDim.x + threadIdx.x; f < total;
         f += (long long)gridDim.x * blockDim.x) {
        const int l = (int)(f % nz);
        const long long r = f / nz;
        const int j = (int)(r % ny);
        const int i = (int)(r / ny);
        const int ip = i < half ? i : i - N, jp = j < half ? j : j - N;
        const long long m = (long long)ip * ip + (long long)jp * jp + (long long)l * l;
        if (m == 0 || m < kedge[0] || m >= kedge[nk]) continue;
        int a = 0, b = nk;                               // kedge[a] <= m < kedge[b]
        while (b - a > 1) {
            const int mid = (a + b) >> 1;
            if (kedge[mid] <= m) a = mid;
            else b = mid;
        }
        const long long idx = ((long long)i * N + j) * Nh + l;
        double zr = (double)m1[idx].x, zi = (double)m1[idx].y;
        double wgt = (double)cw[i] * (double)cw[j] * (double)cw[l];
        if (m2) {
            // e^{+i pi (i' + j' + l) / N} as the product of the per-axis phase table entries
            const C pa = ph[ip + half], pb = ph[jp + half], pc = ph[l + half];
            const double tr = (double)pa.x * pb.x - (double)pa.y * pb.y;
            const double ti = (double)pa.x * pb.y + (double)pa.y * pb.x;
            const double er = tr * pc.x - ti * pc.y, ei = tr * pc.y + ti * pc.x;
            const double br = (double)m2[idx].x, bi = (double)m2[idx].y;
            zr += br * er - bi * ei;
            zi += br * ei + bi * er;
            wgt *= 0.25;
        }
        const double h = ((keep_mask & 4) && l != 0 && l != half) ? 2.0 : 1.0;
        atomicAdd(sums + 3 * a, h);
        atomicAdd(sums + 3 * a + 1, h * kF * sqrt((double)m));
        atomicAdd(sums + 3 * a + 2, h * (zr * zr + zi * zi) * wgt);
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
// Raise a kernel's dynamic shared-memory limit when the launch may pass the
// 48 KB default together with the kernel's static shared arrays (a few KB at
// most here), so an exactly-48 KB dynamic request is covered too.
cudaError_t set_smem(K kernel, size_t bytes) {
    if (bytes <= 40 * 1024) return cudaSuccess;
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

int paint_classes() { return kClasses; }

cudaError_t launch_sort_count(const void *pos, int dtype, const float *w, const float *vals,
                              const int64_t *item_off, int nitems, int64_t max_n, const PaintGeom &g,
                              uint32_t *count, double *wsums, double *wpart, unsigned *wmax, cudaStream_t st) {
    const bool weighted = w != nullptr || vals != nullptr || dtype == PK_F32X4;
    dim3 grid(grid_for(max_n, kCountThreads, weighted ? kWsumBlocks : 1u << 20), nitems);
#define PK_COUNT(DT)                                                                                    \
    if (weighted) k_sort_count<DT, true><<<grid, kCountThreads, 0, st>>>(pos, w, vals, item_off, g, count, wsums, wpart, wmax); \
    else k_sort_count<DT, false><<<grid, kCountThreads, 0, st>>>(pos, w, vals, item_off, g, count, wsums, wpart, wmax);
    switch (dtype) {
    case PK_F32: PK_COUNT(PK_F32) break;
    case PK_F64: PK_COUNT(PK_F64) break;
    default: PK_COUNT(PK_F32X4) break;
    }
#undef PK_COUNT
    if (weighted) {
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        k_wsum_reduce<<<nitems, 256, 0, st>>>(wpart, (int)grid.x, wsums);
    }
    return cudaGetLastError();
}

size_t wsum_partial_elems(int nitems) { return (size_t)nitems * kWsumBlocks * 3; }

cudaError_t launch_sort_scatter(const void *pos, int dtype, const float *w, const float *vals,
                                const int64_t *item_off, int nitems, int64_t max_n, const PaintGeom &g,
                                const uint32_t *off, uint32_t *count, float4 *sorted, int *err,
                                cudaStream_t st) {
    dim3 grid(grid_for(max_n, kCountThreads, 1u << 20), nitems);
    switch (dtype) {
    case PK_F32: k_sort_scatter<PK_F32><<<grid, kCountThreads, 0, st>>>(pos, w, vals, item_off, g, off, count, sorted, err); break;
    case PK_F64: k_sort_scatter<PK_F64><<<grid, kCountThreads, 0, st>>>(pos, w, vals, item_off, g, off, count, sorted, err); break;
    default: k_sort_scatter<PK_F32X4><<<grid, kCountThreads, 0, st>>>(pos, w, vals, item_off, g, off, count, sorted, err); break;
    }
    return cudaGetLastError();
}

// Small host arrays travel as kernel parameters (copied at launch, so the
// host may reuse its array at once and a captured graph keeps the values).
struct I64Chunk {
    int64_t v[kUploadChunk];
};

__global__ void k_upload_i64(int64_t *__restrict__ dst, I64Chunk c, int n) {
    if ((int)threadIdx.x < n) dst[threadIdx.x] = c.v[threadIdx.x];
}

cudaError_t launch_upload_i64(int64_t *dst, const int64_t *src, int n, int *launches, cudaStream_t st) {
    for (int b = 0; b < n; b += kUploadChunk) {
        const int m = n - b < kUploadChunk ? n - b : kUploadChunk;
        I64Chunk c;
        for (int k = 0; k < m; ++k) c.v[k] = src[b + k];
        k_upload_i64<<<1, kUploadChunk, 0, st>>>(dst + b, c, m);
        *launches += 1;
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

size_t scan_tmp_elems(int64_t n) {
    size_t t = 0;
    while (n > 1) {
        const int64_t nb = (n + kScanTile - 1) / kScanTile;
        t += (size_t)nb + 1;
        n = nb;
    }
    return t + 2;
}

template <typename T>
static cudaError_t scan_impl(const T *in, int64_t n, T *out, T *tmp, int *launches, cudaStream_t st) {
    const int64_t nb = (n + kScanTile - 1) / kScanTile;
    if (nb <= 1) {
        k_scan_blocks<T><<<1, kScanThreads, 0, st>>>(in, n, out, out + n);
        *launches += 1;
        return cudaGetLastError();
    }
    if (nb > 0x7fffffffLL) return cudaErrorInvalidValue;
    k_scan_blocks<T><<<(unsigned)nb, kScanThreads, 0, st>>>(in, n, out, tmp);
    *launches += 1;
    cudaError_t e = scan_impl<T>(tmp, nb, tmp, tmp + nb + 1, launches, st);
    if (e != cudaSuccess) return e;
    k_scan_add<T><<<(unsigned)nb, kScanThreads, 0, st>>>(out, n, tmp, (int)nb);
    *launches += 1;
    return cudaGetLastError();
}

// out[0 .. n) = exclusive scan of in, out[n] = total.  tmp: scan_tmp_elems(n).
cudaError_t launch_scan(const uint32_t *in, int64_t n, uint32_t *out, uint32_t *tmp, int *launches,
                        cudaStream_t st) {
    return scan_impl<uint32_t>(in, n, out, tmp, launches, st);
}

cudaError_t launch_scan64(const unsigned long long *in, int64_t n, unsigned long long *out,
                          unsigned long long *tmp, int *launches, cudaStream_t st) {
    return scan_impl<unsigned long long>(in, n, out, tmp, launches, st);
}

size_t paint_smem_bytes(int T, int window, int nmesh) {
    const size_t general = (size_t)2 * T * T * T * sizeof(unsigned) + (size_t)kStage * sizeof(float4);
    const size_t padded = T != 16 ? 0
                          : window == 4 ? (size_t)nmesh * SweepLayout<4>::Words * sizeof(unsigned)
                          : window == 3 ? (size_t)nmesh * SweepLayout<3>::Words * sizeof(unsigned) : 0;
    return general > padded ? general : padded;
}

template <int P, int NM, typename M>
static cudaError_t paint_inst(const float4 *sorted, const uint32_t *off, int nitems,
                              const PaintGeom &g, int S, const unsigned *wmax, float wmax_deposit,
                              void *mesh, long long item_stride, long long mesh_stride, int accumulate,
                              cudaStream_t st) {
    const size_t smem = paint_smem_bytes(g.T, P, NM);   // one padded mesh fits the general area
    const long long nblocks = (long long)nitems * g.ntiles;
    if (nblocks <= 0) return cudaSuccess;
    if (nblocks > 0x7fffffffLL) return cudaErrorInvalidValue;
    auto kern = g.T == 16 ? k_paint_tiles<P, NM, M, 16> : k_paint_tiles<P, NM, M, 0>;
    cudaError_t e = set_smem(kern, smem);
    if (e != cudaSuccess) return e;
    kern<<<(unsigned)nblocks, kPaintThreads, smem, st>>>(sorted, off, g, S, wmax, wmax_deposit,
                                                         reinterpret_cast<M *>(mesh), item_stride,
                                                         mesh_stride, accumulate);
    return cudaGetLastError();
}

cudaError_t launch_paint_tiles(const float4 *sorted, const uint32_t *off, int nitems,
                               const PaintGeom &g, int window, int nmesh, int S, int f64,
                               const unsigned *wmax, int unit_weights, void *mesh,
                               long long item_stride, long long mesh_stride, int accumulate,
                               cudaStream_t st) {
    // Largest single deposit w W with unit weights: max W = (max per-axis weight)^3.
    const float wdep = !unit_weights ? 0.0f : (window == 2 ? 1.0f : window == 3 ? 0.421875f : 0.2962963f);
#define PK_PAINT_CASE(P)                                                                              \
    if (window == P) {                                                                                \
        if (f64) return nmesh == 2 ? paint_inst<P, 2, double>(sorted, off, nitems, g, S, wmax, wdep, mesh, \
                                                              item_stride, mesh_stride, accumulate, st) \
                                   : paint_inst<P, 1, double>(sorted, off, nitems, g, S, wmax, wdep, mesh, \
                                                              item_stride, mesh_stride, accumulate, st); \
        return nmesh == 2 ? paint_inst<P, 2, float>(sorted, off, nitems, g, S, wmax, wdep, mesh,     \
                                                    item_stride, mesh_stride, accumulate, st)         \
                          : paint_inst<P, 1, float>(sorted, off, nitems, g, S, wmax, wdep, mesh,     \
                                                    item_stride, mesh_stride, accumulate, st);        \
    }
    PK_PAINT_CASE(2)
    PK_PAINT_CASE(3)
    PK_PAINT_CASE(4)
#undef PK_PAINT_CASE
    return cudaErrorInvalidValue;
}

template <int DT, int P, int NM>
static cudaError_t atomic_inst(const void *pos, const float *w, const float *vals, const int64_t *item_off, int nitems,
                               int64_t max_n, const PaintGeom &g, int S, bool weighted,
                               unsigned long long *acc, double *wsums, double *wpart, unsigned *wmax,
                               cudaStream_t st) {
    dim3 grid(grid_for(max_n, kCountThreads, weighted ? kWsumBlocks : 1u << 20), nitems);
    k_paint_atomic<DT, P, NM><<<grid, kCountThreads, 0, st>>>(pos, w, vals, item_off, g, S, weighted, acc,
                                                             wsums, wpart, wmax);
    if (weighted) {
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        k_wsum_reduce<<<nitems, 256, 0, st>>>(wpart, (int)grid.x, wsums);
    }
    return cudaGetLastError();
}

template <int DT>
static cudaError_t atomic_dispatch(const void *pos, const float *w, const float *vals, const int64_t *item_off, int nitems,
                                   int64_t max_n, const PaintGeom &g, int window, int nmesh, int S,
                                   bool weighted, unsigned long long *acc, double *wsums, double *wpart,
                                   unsigned *wmax, cudaStream_t st) {
#define PK_ATOMIC_CASE(P)                                                                              \
    if (window == P)                                                                                   \
        return nmesh == 2 ? atomic_inst<DT, P, 2>(pos, w, vals, item_off, nitems, max_n, g, S, weighted, acc, \
                                                  wsums, wpart, wmax, st)                             \
                          : atomic_inst<DT, P, 1>(pos, w, vals, item_off, nitems, max_n, g, S, weighted, acc, \
                                                  wsums, wpart, wmax, st);
    PK_ATOMIC_CASE(2)
    PK_ATOMIC_CASE(3)
    PK_ATOMIC_CASE(4)
#undef PK_ATOMIC_CASE
    return cudaErrorInvalidValue;
}

cudaError_t launch_paint_atomic(const void *pos, int dtype, const float *w, const float *vals,
                                const int64_t *item_off, int nitems, int64_t max_n, const PaintGeom &g,
                                int window, int nmesh, int S, unsigned long long *acc, double *wsums,
                                double *wpart, unsigned *wmax, cudaStream_t st) {
    const bool weighted = w != nullptr || vals != nullptr || dtype == PK_F32X4;
    switch (dtype) {
    case PK_F32:
        return atomic_dispatch<PK_F32>(pos, w, vals, item_off, nitems, max_n, g, window, nmesh, S, weighted, acc,
                                       wsums, wpart, wmax, st);
    case PK_F64:
        return atomic_dispatch<PK_F64>(pos, w, vals, item_off, nitems, max_n, g, window, nmesh, S, weighted, acc,
                                       wsums, wpart, wmax, st);
    default:
        return atomic_dispatch<PK_F32X4>(pos, w, vals, item_off, nitems, max_n, g, window, nmesh, S, weighted,
                                         acc, wsums, wpart, wmax, st);
    }
}

cudaError_t launch_acc_to_mesh(unsigned long long *acc, int nitems, int nmesh, int N, int S, int f64,
                               void *mesh, long long item_stride, long long mesh_stride, int accumulate,
                               int nsm, cudaStream_t st) {
    const long long npairs = (long long)nitems * nmesh * N * N * N / 2;
    if (npairs <= 0) return cudaSuccess;
    const unsigned grid = grid_for(npairs, 256, (unsigned)(nsm > 0 ? nsm * 8 : 1024));
    const float inv_scale = ldexpf(1.0f, -S);
    ulonglong2 *a2 = reinterpret_cast<ulonglong2 *>(acc);
    if (f64)
        k_acc_to_mesh<double><<<grid, 256, 0, st>>>(a2, npairs, N, nmesh, inv_scale,
                                                    reinterpret_cast<double *>(mesh), item_stride,
                                                    mesh_stride, accumulate);
    else
        k_acc_to_mesh<float><<<grid, 256, 0, st>>>(a2, npairs, N, nmesh, inv_scale,
                                                   reinterpret_cast<float *>(mesh), item_stride,
                                                   mesh_stride, accumulate);
    return cudaGetLastError();
}

size_t bin_smem_bytes(const BinGeom &g, int f64) {
    return f64 ? BinSmem<double, double2, double>::bytes(g) : BinSmem<float, float2, float>::bytes(g);
}

int bin_threads() { return kBinThreads; }

template <bool IL, bool TWOD, bool POLES, typename R, typename C, typename A, bool CROSS>
static cudaError_t bin_inst(const void *mesh, long long item_stride_c, long long mesh_stride_c,
                            int nitems, int G, const BinGeom &g, const void *cw, const void *ph,
                            const int *kedge, void *partial, const void *meshb, cudaStream_t st) {
    const size_t smem = BinSmem<R, C, A>::bytes(g);
    auto kern = (g.mu32 || !TWOD) ? k_bin<IL, TWOD, POLES, R, C, A, CROSS, true>
                                  : k_bin<IL, TWOD, POLES, R, C, A, CROSS, false>;
    cudaError_t e = set_smem(kern, smem);
    if (e != cudaSuccess) return e;
    dim3 grid(G, nitems);
    kern<<<grid, kBinThreads, smem, st>>>(reinterpret_cast<const C *>(mesh), item_stride_c,
                                          mesh_stride_c, g, reinterpret_cast<const R *>(cw),
                                          reinterpret_cast<const C *>(ph), kedge,
                                          reinterpret_cast<A *>(partial), reinterpret_cast<const C *>(meshb));
    return cudaGetLastError();
}

template <typename R, typename C, typename A, bool CROSS>
static cudaError_t bin_dispatch(const void *mesh, int il, long long is, long long ms, int nitems,
                                int G, const BinGeom &g, const void *cw, const void *ph,
                                const int *kedge, void *partial, const void *meshb, cudaStream_t st) {
    const int key = (il ? 4 : 0) | (g.twod ? 2 : 0) | (g.poles ? 1 : 0);
#define PK_BIN(a, b, c) bin_inst<a, b, c, R, C, A, CROSS>(mesh, is, ms, nitems, G, g, cw, ph, kedge, partial, meshb, st)
    switch (key) {
    case 0: return PK_BIN(false, false, false);
    case 1: return PK_BIN(false, false, true);
    case 2: return PK_BIN(false, true, false);
    case 3: return PK_BIN(false, true, true);
    case 4: return PK_BIN(true, false, false);
    case 5: return PK_BIN(true, false, true);
    case 6: return PK_BIN(true, true, false);
    default: return PK_BIN(true, true, true);
    }
#undef PK_BIN
}

cudaError_t launch_bin(const void *mesh, int f64, int interlaced, long long item_stride_c,
                       long long mesh_stride_c, int nitems, int ctas_per_item,
                       const BinGeom &g, const void *cw, const void *ph, const int *kedge,
                       void *partial, cudaStream_t st) {
    if (f64)
        return bin_dispatch<double, double2, double, false>(mesh, interlaced, item_stride_c, mesh_stride_c,
                                                             nitems, ctas_per_item, g, cw, ph, kedge, partial,
                                                             nullptr, st);
    return bin_dispatch<float, float2, float, false>(mesh, interlaced, item_stride_c, mesh_stride_c, nitems,
                                                     ctas_per_item, g, cw, ph, kedge, partial, nullptr, st);
}

cudaError_t launch_bin_cross(const void *mesh_a, const void *mesh_b, int f64, int interlaced,
                             long long mesh_stride_c, int ctas, const BinGeom &g, const void *cw,
                             const void *ph, const int *kedge, void *partial, cudaStream_t st) {
    if (f64)
        return bin_dispatch<double, double2, double, true>(mesh_a, interlaced, 0, mesh_stride_c, 1, ctas, g, cw,
                                                            ph, kedge, partial, mesh_b, st);
    return bin_dispatch<float, float2, float, true>(mesh_a, interlaced, 0, mesh_stride_c, 1, ctas, g, cw, ph,
                                                    kedge, partial, mesh_b, st);
}

int bin_ctas_per_sm(const BinGeom &g, int f64) {
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
    if (e != cudaSuccess || n < 1) n = 1;
    return n;
}

int reduce_chunks(int G) { return (G + kReduceChunk - 1) / kReduceChunk; }
int reduce_launches(int G) { return reduce_chunks(G) > 1 ? 2 : 1; }

cudaError_t launch_bin_reduce(const void *partial, int f64, int G, int nh, int nitems,
                              double *sums2, cudaStream_t st) {
    const int nchunk = reduce_chunks(G);
    if (nchunk > kReduceChunk) return cudaErrorInvalidValue;    // the second pass is one chunk
    dim3 grid((nh + 127) / 128, nchunk, nitems);
    if (f64) k_bin_reduce<double><<<grid, 128, 0, st>>>(reinterpret_cast<const double *>(partial), G, nh, nchunk, sums2);
    else k_bin_reduce<float><<<grid, 128, 0, st>>>(reinterpret_cast<const float *>(partial), G, nh, nchunk, sums2);
    if (nchunk > 1) {       // the chunk rows of each catalog into its row 0 (kReduceChunk >= nchunk)
        dim3 g2((nh + 127) / 128, 1, nitems);
        k_bin_reduce<double><<<g2, 128, 0, st>>>(sums2, nchunk, nh, nchunk, sums2);
    }
    return cudaGetLastError();
}

// Blocks per catalog for k_finalize: one per 256 bins of the larger table.
static unsigned finalize_blocks(const FinalGeom &f) {
    const int bins = f.twod && f.nk * f.nmu > f.nk ? f.nk * f.nmu : f.nk;
    return (unsigned)std::min(64, std::max(1, (bins + 255) / 256));
}

cudaError_t launch_finalize(const double *sums2, int G, const unsigned long long *modes1d,
                            const unsigned long long *modes2d, const double *wsums, const int *err,
                            const FinalGeom &f, int nitems, double *res, cudaStream_t st) {
    const ResultLayout rl = result_layout(f.nk, f.nmu);
    k_finalize<<<dim3(nitems, finalize_blocks(f)), 256, 0, st>>>(sums2, reduce_chunks(G), 1, modes1d, modes2d, wsums, err, f, rl, res, -1, -1);
    return cudaGetLastError();
}

cudaError_t launch_finalize_cross(const double *sums2, int G, const unsigned long long *modes1d,
                                  const unsigned long long *modes2d, const double *wsums, const int *err,
                                  const FinalGeom &f, int item_a, int item_b, double *res, cudaStream_t st) {
    const ResultLayout rl = result_layout(f.nk, f.nmu);
    k_finalize<<<dim3(1, finalize_blocks(f)), 256, 0, st>>>(sums2, reduce_chunks(G), 1, modes1d, modes2d, wsums, err, f, rl, res, item_a,
                                  item_b);
    return cudaGetLastError();
}

cudaError_t launch_plane_bin(const void *m1, const void *m2, int f64, int N, int keep_mask, const void *cw,
                             const void *ph, const int *kedge, int nk, double kF, double *sums, int nsm,
                             cudaStream_t st) {
    const int Nh = N / 2 + 1;
    const long long total = (long long)((keep_mask & 1) ? N : 1) * ((keep_mask & 2) ? N : 1) * ((keep_mask & 4) ? Nh : 1);
    const unsigned grid = grid_for(total, 256, (unsigned)(nsm > 0 ? nsm * 8 : 1024));
    if (f64)
        k_plane_bin<double, double2><<<grid, 256, 0, st>>>(
            reinterpret_cast<const double2 *>(m1), reinterpret_cast<const double2 *>(m2), N, keep_mask,
            reinterpret_cast<const double *>(cw), reinterpret_cast<const double2 *>(ph), kedge, nk, kF, sums);
    else
        k_plane_bin<float, float2><<<grid, 256, 0, st>>>(
            reinterpret_cast<const float2 *>(m1), reinterpret_cast<const float2 *>(m2), N, keep_mask,
            reinterpret_cast<const float *>(cw), reinterpret_cast<const float2 *>(ph), kedge, nk, kF, sums);
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
                                 unsigned long long *modes2d, double *kmean2d, double *mumean2d,
                                 cudaStream_t st) {
    const int nq = g.nmu > 0 ? g.nmu : 1;
    const int n = g.nk * nq;
    k_geom_finalize<<<(n + 127) / 128, 128, 0, st>>>(g, kedge, kF, H, HL, modes2d, kmean2d, mumean2d);
    return cudaGetLastError();
}

}  // namespace pk
