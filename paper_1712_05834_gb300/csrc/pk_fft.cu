// pk_fft.cu -- the library's own 3D r2c transform of FP32 meshes, with its
// last axis fused into the bin pass (the transform of Sec. 3.3.1; the
// binning of Sec. 3.4.1, Eq. window-deconvolution).
//
// Each real mesh row d[0..N) along z is read as M = N/2 complex values
// c[n] = d[2n] + i d[2n+1]; the padded r2c layout (rows of 2(N/2+1) reals)
// holds them in place, so nothing is copied.  The 3D transform of d is then
// made of three steps:
//   k_fft_axis (y)   length-N complex FFTs along y of the packed array;
//   k_fft_axis (x)   the same along x;
//   k_zbin           one warp per pair of rows (kx, ky) and (-kx, -ky):
//                    length-M FFTs along z of both rows of both meshes, the
//                    split of the packed transform C into the r2c transform
//                      D[l] = (C[l] + conj C'[M-l]) / 2
//                             - (i/2) W_N^l (C[l] - conj C'[M-l]),  l = 0..M
//                    (C' the partner row, indices mod M; the x and y
//                    transforms of a real array pair (kx, ky) with
//                    (-kx, -ky)), then the bin pass of k_bin on both rows:
//                    interlace combine, sinc^p compensation, k bin, mu bin,
//                    Legendre sums, register runs flushed into a per-CTA
//                    histogram.  The r2c transform itself is never written.
//   k_zfinish        the z step and the split without binning: D written
//                    into the rows in place, for the passes that read the
//                    transform after a compute (cross and projected power).
// All transforms are forward (e^{-2 pi i jk/n}), unnormalized, radix-8
// decimation in frequency with radix-4 and radix-3 steps where the length
// needs them (N = 2^k, 128 <= N <= 2048, and N = 192);
// twiddles come from one table W_N^e (e < N) computed in FP64 on the host
// (the x and y passes read W^n and W^{4n} of a butterfly from it and form
// its other twiddles as products, a few ulp each).
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "pk_internal.h"

namespace pk {

namespace {

constexpr int kZVec = 4;              // consecutive modes per lane in the bin step

__device__ __forceinline__ float2 c_add(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 c_sub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 c_mul(float2 a, float2 b) {
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ float2 c_mi(float2 a) { return make_float2(a.y, -a.x); }   // a * (-i)

// In-register DFT of R points: v[k] <- sum_j v[j] W_R^{jk}.
template <int R>
__device__ __forceinline__ void dft(float2 *v);

template <>
__device__ __forceinline__ void dft<4>(float2 *v) {
    const float2 a = c_add(v[0], v[2]), b = c_sub(v[0], v[2]);
    const float2 c = c_add(v[1], v[3]), d = c_mi(c_sub(v[1], v[3]));
    v[0] = c_add(a, c);
    v[2] = c_sub(a, c);
    v[1] = c_add(b, d);
    v[3] = c_sub(b, d);
}

template <>
__device__ __forceinline__ void dft<3>(float2 *v) {
    const float h = 0.86602540378443865f;                      // sqrt(3) / 2
    const float2 s = c_add(v[1], v[2]), d = c_sub(v[1], v[2]);
    const float2 m = make_float2(v[0].x - 0.5f * s.x, v[0].y - 0.5f * s.y);
    v[0] = c_add(v[0], s);
    v[1] = make_float2(m.x + h * d.y, m.y - h * d.x);          // W_3 = -1/2 - i sqrt(3)/2
    v[2] = make_float2(m.x - h * d.y, m.y + h * d.x);
}

// Split into the even and odd outputs: X[2k] = DFT4(v[j] + v[j+4]),
// X[2k+1] = DFT4((v[j] - v[j+4]) W_8^j).
template <>
__device__ __forceinline__ void dft<8>(float2 *v) {
    const float h = 0.70710678118654752f;
    float2 u[4], w[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        u[j] = c_add(v[j], v[j + 4]);
        w[j] = c_sub(v[j], v[j + 4]);
    }
    w[1] = make_float2(h * (w[1].x + w[1].y), h * (w[1].y - w[1].x));    // * W_8 = (1 - i)/sqrt 2
    w[2] = c_mi(w[2]);                                                   // * W_8^2 = -i
    w[3] = make_float2(h * (w[3].y - w[3].x), -h * (w[3].x + w[3].y));   // * W_8^3 = -(1 + i)/sqrt 2
    dft<4>(u);
    dft<4>(w);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        v[2 * k] = u[k];
        v[2 * k + 1] = w[k];
    }
}

// Radix of the decimation-in-frequency step over blocks of S points: 8, with
// 4 for the blocks of 16, 12 and 4 points and 3 for a block of 3 (lengths
// 2^k >= 4 and 3 * 2^k: 192 runs 8, 8, 3 and 96 runs 8, 4, 3).
__host__ __device__ constexpr int radix_of(int S) {
    return S == 3 ? 3 : (S == 4 || S == 12 || S == 16) ? 4 : 8;
}

// Radix order of the z FFTs: as radix_of, but 4 for the blocks of 32 (a
// length-256 transform runs 8, 4, 8).
__host__ __device__ constexpr int zradix_of(int S) { return S == 32 ? 4 : radix_of(S); }

// Frequency at position p (< S) after all steps over a block of S points:
// a step of radix R puts output k of the butterfly at n + (S/R) k, so the
// digits of p, most significant first, are the frequency's digits from the
// least significant up.
template <int S, int MUL, bool Z = false>
__device__ __forceinline__ int dif_freq(int p) {
    if constexpr (S == 1) {
        return 0;
    } else {
        constexpr int R = Z ? zradix_of(S) : radix_of(S), Q = S / R;
        return (p / Q) * MUL + dif_freq<Q, MUL * R, Z>(p % Q);
    }
}

// ---------------------------------------------------------------------------
// x and y passes: one CTA per tile of NB adjacent packed columns (n) of one
// line set; element a (along the transformed axis) of column c sits at
// g + a * astride + c.  The tile is read from global memory straight into
// the first step's registers, kept in shared memory between steps
// (buf[a * NB + c]: NB threads cover one row of buf) and written back from
// the last step's registers in natural order.  Tile shapes per line length:
// 16 columns (128-byte runs of each line) where the tile fits twice per SM
// (N <= 512: 512 threads, two CTAs per SM); 16 columns in one CTA of 1024
// threads at N = 1024 (136 KB); 8 columns at N = 2048 (144 KB: 16 would not
// fit).  Measured: at N = 2048 the x lines' 64-byte runs stream at 2.9 TB/s
// where 128-byte ones reach 5 TB/s.
template <int LEN>
struct AxisCfg {
    static constexpr int NB = LEN >= 2048 ? 8 : 16;        // columns per tile
    // threads per CTA (for 192 lines: 8 butterfly groups divide 24 and 64)
    static constexpr int T = LEN >= 1024 ? 1024 : (LEN >= 256 ? 512 : (LEN == 192 ? 128 : 256));
    static constexpr int MINB = LEN >= 1024 ? 1 : (LEN >= 256 ? 2 : (LEN == 192 ? 8 : 4));   // CTAs per SM
};

template <int LEN, int NB, int S, bool FIRST>
__device__ __forceinline__ void axis_step(float2 *buf, float2 *g, long long astride, const float2 *tw, int c,
                                          int grp) {
    constexpr int R = radix_of(S), Q = S / R;
    constexpr int NG = AxisCfg<LEN>::T / NB;    // thread groups (one per butterfly index)
    constexpr int PER = (LEN / R) / NG;       // butterflies per thread
    static_assert((LEN / R) % NG == 0 && PER >= 1, "butterflies must split evenly over the threads");
    if constexpr (Q == 1) {
        static_assert(!FIRST, "a single-step transform is not used");
#pragma unroll
        for (int s = 0; s < PER; ++s) {
            const int blk = grp + NG * s;
            float2 v[R];
#pragma unroll
            for (int j = 0; j < R; ++j) v[j] = buf[(blk * R + j) * NB + c];
            dft<R>(v);
#pragma unroll
            for (int k = 0; k < R; ++k) g[(long long)dif_freq<LEN, 1>(blk * R + k) * astride + c] = v[k];
        }
    } else {
        float2 v[PER][R];
#pragma unroll
        for (int s = 0; s < PER; ++s) {
            const int beta = grp + NG * s;
            const int base = (beta / Q) * S + beta % Q;
#pragma unroll
            for (int j = 0; j < R; ++j)
                v[s][j] = FIRST ? g[(long long)(base + Q * j) * astride + c] : buf[(base + Q * j) * NB + c];
        }
#pragma unroll
        for (int s = 0; s < PER; ++s) {
            const int beta = grp + NG * s;
            const int n = beta % Q, base = (beta / Q) * S + n;
            dft<R>(v[s]);
            {
                constexpr int E = LEN / S;
                float2 ww[R];
                ww[1] = tw[n * E];
                if constexpr (R == 8) {
                    ww[4] = tw[4 * n * E];
                    ww[2] = c_mul(ww[1], ww[1]);
                    ww[3] = c_mul(ww[2], ww[1]);
                    ww[5] = c_mul(ww[4], ww[1]);
                    ww[6] = c_mul(ww[4], ww[2]);
                    ww[7] = c_mul(ww[4], ww[3]);
                } else if constexpr (R == 4) {
                    ww[2] = tw[2 * n * E];
                    ww[3] = c_mul(ww[2], ww[1]);
                } else {
#pragma unroll
                    for (int k = 2; k < R; ++k) ww[k] = tw[k * n * E];
                }
#pragma unroll
                for (int k = 1; k < R; ++k) v[s][k] = c_mul(v[s][k], ww[k]);
            }
#pragma unroll
            for (int k = 0; k < R; ++k) buf[(base + Q * k) * NB + c] = v[s][k];
        }
        __syncthreads();
        axis_step<LEN, NB, Q, false>(buf, g, astride, tw, c, grp);
    }
}

template <int LEN, int NB>
__global__ void __launch_bounds__(AxisCfg<LEN>::T, AxisCfg<LEN>::MINB)
k_fft_axis(float2 *__restrict__ mesh, long long mesh_c, long long outer_stride, long long astride,
           const float2 *__restrict__ twg) {
    extern __shared__ __align__(16) unsigned char smraw[];
    float2 *tw = reinterpret_cast<float2 *>(smraw);
    float2 *buf = tw + LEN;
    for (int e = threadIdx.x; e < LEN; e += AxisCfg<LEN>::T) tw[e] = twg[e];
    constexpr unsigned NBL = (LEN / 2) / NB;   // column tiles per line
    const unsigned t = blockIdx.x;
    const unsigned nb = t % NBL, rest = t / NBL;
    const unsigned outer = rest % LEN, m = rest / LEN;
    float2 *g = mesh + (long long)m * mesh_c + (long long)outer * outer_stride + (long long)nb * NB;
    __syncthreads();
    axis_step<LEN, NB, LEN, true>(buf, g, astride, tw, threadIdx.x % NB, threadIdx.x / NB);
}


template <int LEN>
cudaError_t axis_inst(float2 *mesh, int nmesh, long long mesh_c, const float2 *tw, cudaStream_t st) {
    constexpr int NB = AxisCfg<LEN>::NB, T = AxisCfg<LEN>::T;
    const size_t smem = sizeof(float2) * (size_t)LEN * (NB + 1);
    auto kern = k_fft_axis<LEN, NB>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const long long Nh = LEN / 2 + 1;
    const unsigned grid = (unsigned)nmesh * LEN * ((LEN / 2) / NB);
    // y: lines (x, n) with stride Nh; then x: lines (y, n) with stride N Nh
    kern<<<grid, T, smem, st>>>(mesh, mesh_c, (long long)LEN * Nh, Nh, tw);
    kern<<<grid, T, smem, st>>>(mesh, mesh_c, Nh, (long long)LEN * Nh, tw);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// z step: one warp transforms the rows of a pair.  Rows live in the warp's
// shared buffer, RS slots each; position p sits in slot p ^ ((p >> 2) & 15),
// a bijection on [0, M] that keeps the FFT steps, the natural-order write and
// the bin loop's lane patterns (kZVec consecutive modes per lane, ascending
// and mirrored) free of bank conflicts, except the reads of the last step of
// the length-256 FFT (two-way; radix order 8, 4, 8 -- the order 8, 8, 4 had
// its middle step's reads and writes two-way).  Tables indexed by l use the
// same slots.
__device__ __forceinline__ int zslot(int p) { return p ^ ((p >> 2) & 15); }

// A pair is handled by one warp up to M = 256 (eight pairs per CTA at a
// time), by the whole CTA above (its four rows of M complex are 16 or 32 KB).
template <int M>
struct ZRows {
    // slots per row: positions 0..M, even (zslot(M) = M for M = 2^k >= 64;
    // up to M + 15 otherwise)
    static constexpr int RS = (M & (M - 1)) == 0 ? M + 2 : M + 16;
    static constexpr int WPB = 8;                 // warps per CTA
    static constexpr int NT = M >= 512 ? 256 : 32;   // threads per pair
    static constexpr int PPC = 256 / NT;          // pairs in flight per CTA
};

// Twiddles of the z FFT steps, one table per step with block size S (from M
// down): entry (k - 1) Q + n = W_S^{nk} (Q = S/R, n < Q, 1 <= k < R), so the
// lanes of a step read consecutive or equal entries.
__host__ __device__ constexpr int ztw_offset(int M, int S) {
    int off = 0;
    for (int s = M; s > S; s /= zradix_of(s)) {
        const int q = s / zradix_of(s);
        off += q > 1 ? (zradix_of(s) - 1) * q : 0;
    }
    return off;
}

__device__ __forceinline__ void fill_ztw(float2 *ztw, const float2 *__restrict__ twg, int M) {
    for (int s = M; s > 1; s /= zradix_of(s)) {
        const int R = zradix_of(s), Q = s / R, off = ztw_offset(M, s);
        if (Q == 1) continue;
        for (int e = threadIdx.x; e < (R - 1) * Q; e += blockDim.x) {
            const int k = e / Q + 1, n = e % Q;
            ztw[off + e] = twg[2 * n * k * (M / s)];     // W_N^{2nk M/S} = W_S^{nk}
        }
    }
}

// Row r of a pair: r = 2 q + s, mesh q (interlaced second mesh for q = 1),
// s = 0 for the row (kx, ky), 1 for its partner (-kx, -ky).
__device__ __forceinline__ const float2 *pair_row(const float2 *m1, const float2 *m2, long long offA,
                                                  long long offB, int r) {
    return ((r >> 1) ? m2 : m1) + ((r & 1) ? offB : offA);
}

// Barrier of the NT threads that share a pair: the warp, or the whole CTA.
template <int NT>
__device__ __forceinline__ void pair_sync() {
    if constexpr (NT == 32) __syncwarp();
    else __syncthreads();
}

// One step over blocks of S points of the length-M FFTs of the NR rows of a
// pair, by NT threads (FIRST: read from the mesh).  The last step writes the
// outputs in natural order.
template <int M, int NR, int S, bool FIRST, int NT = 32>
__device__ __forceinline__ void zfft_step(float2 *rows, const float2 *m1, const float2 *m2, long long offA,
                                          long long offB, const float2 *ztw, int lane) {
    constexpr int RS = ZRows<M>::RS;
    constexpr int R = zradix_of(S), Q = S / R;
    constexpr int BPR = M / R;                    // butterflies per row
    constexpr int TOT = NR * BPR;
    constexpr int PER = (TOT + NT - 1) / NT;
    constexpr int TW = ztw_offset(M, S);
    float2 v[PER][R];
#pragma unroll
    for (int s = 0; s < PER; ++s) {
        const int beta = lane + NT * s;
        if (TOT % NT == 0 || beta < TOT) {
            const int r = beta / BPR, b = beta % BPR;
            const int base = (b / Q) * S + b % Q;
            if (FIRST) {
                const float2 *src = pair_row(m1, m2, offA, offB, r);
#pragma unroll
                for (int j = 0; j < R; ++j) v[s][j] = __ldcs(src + base + Q * j);
            } else {
#pragma unroll
                for (int j = 0; j < R; ++j) v[s][j] = rows[r * RS + zslot(base + Q * j)];
            }
        }
    }
    // the last step writes other positions than it reads: all reads first
    if constexpr (Q == 1) pair_sync<NT>();
#pragma unroll
    for (int s = 0; s < PER; ++s) {
        const int beta = lane + NT * s;
        if (TOT % NT == 0 || beta < TOT) {
            const int r = beta / BPR, b = beta % BPR;
            const int n = b % Q, base = (b / Q) * S + n;
            dft<R>(v[s]);
            if constexpr (Q > 1) {
#pragma unroll
                for (int k = 1; k < R; ++k) v[s][k] = c_mul(v[s][k], ztw[TW + (k - 1) * Q + n]);   // W_S^{nk}
#pragma unroll
                for (int k = 0; k < R; ++k) rows[r * RS + zslot(base + Q * k)] = v[s][k];
            } else {
#pragma unroll
                for (int k = 0; k < R; ++k) rows[r * RS + zslot(dif_freq<M, 1, true>(base + k))] = v[s][k];
            }
        }
    }
    pair_sync<NT>();
    if constexpr (Q > 1) zfft_step<M, NR, Q, false, NT>(rows, m1, m2, offA, offB, ztw, lane);
}

// 2 D[l] from u = C[l] and v = C'[M-l] (w = W_N^l):
// (u + conj v) - i w (u - conj v).
__device__ __forceinline__ float2 split2(float2 u, float2 v, float2 w) {
    const float ox = u.x - v.x, oy = u.y + v.y;
    const float wx = w.x * ox - w.y * oy, wy = w.x * oy + w.y * ox;
    return make_float2(u.x + v.x + wy, u.y - v.y - wx);
}

// Pair p of the N^2/2 + 2 row pairs {(i, j), (-i, -j)}: rows with 0 < i < M
// (partners have i > M), then i = 0 and i = M with 0 <= j <= M.
__device__ __forceinline__ void pair_rows(int p, int N, int *i, int *j) {
    const int M = N / 2;
    if (p < (M - 1) * N) {
        *i = 1 + p / N;
        *j = p % N;
    } else {
        const int q = p - (M - 1) * N;
        *i = q <= M ? 0 : M;
        *j = q <= M ? q : q - (M + 1);
    }
}

__device__ __forceinline__ int isqrt_floor_z(int x) {     // floor(sqrt(x)), 0 <= x < 2^26, exact
    int s = (int)sqrtf((float)x);
    while (s > 0 && s * s > x) --s;
    while ((s + 1) * (s + 1) <= x) ++s;
    return s;
}

// Shared memory of k_zbin / k_zfinish: the z-step twiddles, W_N^l (l <= M,
// swizzled like the rows), the warps' row buffers, then (k_zbin only) the
// histogram, the cw and phase tables (swizzled) and the k-bin edges.
template <int M, int NR>
struct ZSmem {
    __host__ __device__ static constexpr size_t al(size_t x) { return (x + 15) / 16 * 16; }
    __host__ __device__ static size_t off_wl() { return al(sizeof(float2) * ztw_offset(M, 1)); }
    __host__ __device__ static size_t off_rows() { return off_wl() + al(sizeof(float2) * ZRows<M>::RS); }
    __host__ __device__ static size_t off_hist() {
        return off_rows() + al(sizeof(float2) * (size_t)ZRows<M>::PPC * NR * ZRows<M>::RS);
    }
    __host__ __device__ static size_t off_cw(const BinGeom &g) { return off_hist() + al(sizeof(float) * g.nh); }
    __host__ __device__ static size_t off_ph(const BinGeom &g) {
        return off_cw(g) + al(sizeof(float) * ZRows<M>::RS);
    }
    __host__ __device__ static size_t off_edge(const BinGeom &g) {
        return off_ph(g) + al(sizeof(float2) * ZRows<M>::RS);
    }
    __host__ __device__ static size_t bytes(const BinGeom &g) { return off_edge(g) + al(sizeof(int2) * g.nk); }
};

// Fill the z-step twiddles and the swizzled W_N^l, l = 0..M.
template <int M, int NR>
__device__ __forceinline__ void fill_z_tables(unsigned char *smraw, const float2 *__restrict__ twg) {
    using SM = ZSmem<M, NR>;
    fill_ztw(reinterpret_cast<float2 *>(smraw), twg, M);
    float2 *wl = reinterpret_cast<float2 *>(smraw + SM::off_wl());
    for (int l = threadIdx.x; l <= M; l += blockDim.x) wl[zslot(l)] = twg[l];
}

// Bin the modes llo <= l < lhi of the pair's two rows, (i, j) and its partner
// (pi, pj), straight from the z transforms C of the pair (rows a1, b1 of the
// first mesh, a2, b2 of the interlaced one): D of each row from the split,
// then the per-mode arithmetic of k_bin (FP32 form).  Both rows have the
// same r2 = kx'^2 + ky'^2 and so, mode by mode, the same m, k bin, mu bin and
// Legendre weights: each key is computed once and takes the sum of both
// rows' powers (the partner's is left out for a row that is its own partner).
template <bool IL, bool TWOD, bool POLES, bool MU32, int M, int NT = 32>
__device__ __forceinline__ void bin_pair(const float2 *rows, int i, int j, int pi, int pj, int r2, int llo,
                                         int lhi, const BinGeom &g, const float *__restrict__ cw,
                                         const float2 *__restrict__ ph, const float *scw, const float2 *sph,
                                         const float2 *swl, const int2 *sedge, float *hist, int lane) {
    constexpr int RS = ZRows<M>::RS, N = 2 * M;
    const float2 *a1 = rows, *b1 = rows + RS, *a2 = rows + 2 * RS, *b2 = rows + 3 * RS;
    const int nk = g.nk, nmu = g.nmu, hbase = g.hbase;
    const float kscale = g.kscale, koff = g.koff;
    const bool self = pi == i && pj == j;
    // 1/4 undoes the factor 2 of the split; the interlaced mean (F1 + F2 t)/2 another 1/4
    const float scale = IL ? 0.0625f : 0.25f;
    const float cwA = cw[i] * cw[j] * scale;
    const float cwB = self ? 0.0f : cw[pi] * cw[pj] * scale;
    float2 phA = make_float2(0.0f, 0.0f), phB = phA;
    if (IL) {
        const int ip = i < M ? i : i - N, jp = j < M ? j : j - N;
        const int pip = pi < M ? pi : pi - N, pjp = pj < M ? pj : pj - N;
        phA = c_mul(ph[ip + M], ph[jp + M]);
        phB = c_mul(ph[pip + M], ph[pjp + M]);
    }
    for (int l0 = llo + kZVec * lane; l0 < lhi; l0 += NT * kZVec) {
        const int cnt = lhi - l0;
        int cur2 = -1, cur1 = -1;
        float run2 = 0.0f, runm2 = 0.0f, runm4 = 0.0f;
#pragma unroll
        for (int v = 0; v < kZVec; ++v) {
            const bool live = v < cnt;
            const int l = min(l0 + v, lhi - 1);
            const int m = r2 + l * l;
            const float rsm = rsqrtf((float)m);
            int b = (int)((float)m * rsm * kscale - koff);
            b = min(max(b, 0), nk - 1);
            {
                const int2 e = sedge[b];
                b += (int)(m >= e.y) - (int)(m < e.x);
            }
            const int sl = zslot(l), la = zslot(l == M ? 0 : l), lb = zslot(l == 0 ? 0 : M - l);
            const float2 w = swl[sl];
            float2 dA = split2(a1[la], b1[lb], w);
            float2 dB = split2(b1[la], a1[lb], w);
            if (IL) {
                const float2 t = sph[sl];
                const float2 tA = c_mul(phA, t), tB = c_mul(phB, t);
                const float2 eA = split2(a2[la], b2[lb], w), eB = split2(b2[la], a2[lb], w);
                dA.x += eA.x * tA.x - eA.y * tA.y;
                dA.y += eA.x * tA.y + eA.y * tA.x;
                dB.x += eB.x * tB.x - eB.y * tB.y;
                dB.y += eB.x * tB.y + eB.y * tB.x;
            }
            float pw = ((dA.x * dA.x + dA.y * dA.y) * cwA + (dB.x * dB.x + dB.y * dB.y) * cwB) * scw[sl];
            pw *= (float)((l != 0 && l != M) ? 2 : 1) * (float)(live ? 1 : 0);
            int key = b;
            if (TWOD) {
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
            const bool new2 = key != cur2;
            if (new2 && cur2 >= 0) atomicAdd(hist + cur2, run2);
            run2 = new2 ? pw : run2 + pw;
            cur2 = key;
            if (POLES) {
                const float mu = (float)l * rsm;
                const float mu2 = mu * mu;
                const float t2 = pw * (1.5f * mu2 - 0.5f);
                const float t4 = pw * ((4.375f * mu2 - 3.75f) * mu2 + 0.375f);
                const bool new1 = b != cur1;
                if (new1 && cur1 >= 0) {
                    atomicAdd(hist + hbase + cur1, runm2);
                    atomicAdd(hist + hbase + nk + cur1, runm4);
                }
                runm2 = new1 ? t2 : runm2 + t2;
                runm4 = new1 ? t4 : runm4 + t4;
                cur1 = b;
            }
        }
        atomicAdd(hist + cur2, run2);
        if (POLES) {
            atomicAdd(hist + hbase + cur1, runm2);
            atomicAdd(hist + hbase + nk + cur1, runm4);
        }
    }
}

// Fused z transform + split + bin over the row pairs of one catalog per
// blockIdx.y; warps take pairs in a grid-strided loop and skip pairs whose
// r2 = kx'^2 + ky'^2 puts no mode into a bin (their rows are not read).
template <bool IL, bool TWOD, bool POLES, bool MU32, int M>
__global__ void __launch_bounds__(32 * ZRows<M>::WPB)
k_zbin(const float2 *__restrict__ mesh, long long item_stride_c, long long mesh_stride_c, BinGeom g,
       const float *__restrict__ cw, const float2 *__restrict__ ph, const float2 *__restrict__ twg,
       const int *__restrict__ kedge, float *__restrict__ partial) {
    constexpr int NR = IL ? 4 : 2, RS = ZRows<M>::RS, NT = ZRows<M>::NT, PPC = ZRows<M>::PPC, N = 2 * M,
                  Nh = M + 1;
    using SM = ZSmem<M, NR>;
    extern __shared__ __align__(16) unsigned char smraw[];
    const float2 *ztw = reinterpret_cast<const float2 *>(smraw);
    const float2 *swl = reinterpret_cast<const float2 *>(smraw + SM::off_wl());
    float *hist = reinterpret_cast<float *>(smraw + SM::off_hist());
    float *scw = reinterpret_cast<float *>(smraw + SM::off_cw(g));
    float2 *sph = reinterpret_cast<float2 *>(smraw + SM::off_ph(g));
    int2 *sedge = reinterpret_cast<int2 *>(smraw + SM::off_edge(g));
    const int lane = threadIdx.x % NT, grp = threadIdx.x / NT;
    float2 *rows = reinterpret_cast<float2 *>(smraw + SM::off_rows()) + (size_t)grp * NR * RS;
    fill_z_tables<M, NR>(smraw, twg);
    for (int k = threadIdx.x; k < g.nh; k += blockDim.x) hist[k] = 0.0f;
    for (int k = threadIdx.x; k < Nh; k += blockDim.x) {
        scw[zslot(k)] = cw[k];
        sph[zslot(k)] = ph[k + M];
    }
    for (int k = threadIdx.x; k < g.nk; k += blockDim.x) sedge[k] = make_int2(kedge[k], kedge[k + 1]);
    __syncthreads();

    const float2 *m1 = mesh + (long long)blockIdx.y * item_stride_c;
    const float2 *m2 = m1 + mesh_stride_c;
    const int npairs = (M - 1) * N + 2 * (M + 1);
    for (int p = blockIdx.x * PPC + grp; p < npairs; p += gridDim.x * PPC) {
        int i, j;
        pair_rows(p, N, &i, &j);
        const int ip = i < M ? i : i - N, jp = j < M ? j : j - N;
        const int r2 = ip * ip + jp * jp;
        if (r2 >= g.mhi) continue;
        const int lhi = min(Nh, isqrt_floor_z(g.mhi - 1 - r2) + 1);
        int llo = g.mlo > r2 ? isqrt_floor_z(g.mlo - r2 - 1) + 1 : 0;
        if (r2 == 0 && llo == 0) llo = 1;
        if (llo >= lhi) continue;
        const int pi = i == 0 ? 0 : N - i, pj = j == 0 ? 0 : N - j;
        const long long offA = ((long long)i * N + j) * Nh, offB = ((long long)pi * N + pj) * Nh;
        pair_sync<NT>();    // the previous pair's bin reads are done
        zfft_step<M, NR, M, true, NT>(rows, m1, m2, offA, offB, ztw, lane);
        bin_pair<IL, TWOD, POLES, MU32, M, NT>(rows, i, j, pi, pj, r2, llo, lhi, g, cw, ph, scw, sph, swl, sedge,
                                               hist, lane);
    }
    __syncthreads();
    float *out = partial + ((long long)blockIdx.y * gridDim.x + blockIdx.x) * g.nh;
    for (int k = threadIdx.x; k < g.nh; k += blockDim.x) out[k] = hist[k];
}

// The z transform and split of every row pair, written back in place: the
// meshes then hold the r2c transform, as after cuFFT's R2C.
template <int M, int NR>
__global__ void __launch_bounds__(32 * ZRows<M>::WPB)
k_zfinish(float2 *__restrict__ mesh, long long item_stride_c, long long mesh_stride_c,
          const float2 *__restrict__ twg) {
    constexpr int RS = ZRows<M>::RS, NT = ZRows<M>::NT, PPC = ZRows<M>::PPC, N = 2 * M, Nh = M + 1;
    using SM = ZSmem<M, NR>;
    extern __shared__ __align__(16) unsigned char smraw[];
    const float2 *ztw = reinterpret_cast<const float2 *>(smraw);
    const float2 *swl = reinterpret_cast<const float2 *>(smraw + SM::off_wl());
    const int lane = threadIdx.x % NT, grp = threadIdx.x / NT;
    float2 *rows = reinterpret_cast<float2 *>(smraw + SM::off_rows()) + (size_t)grp * NR * RS;
    fill_z_tables<M, NR>(smraw, twg);
    __syncthreads();
    float2 *m1 = mesh + (long long)blockIdx.y * item_stride_c;
    float2 *m2 = m1 + mesh_stride_c;
    const int npairs = (M - 1) * N + 2 * (M + 1);
    for (int p = blockIdx.x * PPC + grp; p < npairs; p += gridDim.x * PPC) {
        int i, j;
        pair_rows(p, N, &i, &j);
        const int pi = i == 0 ? 0 : N - i, pj = j == 0 ? 0 : N - j;
        const long long offA = ((long long)i * N + j) * Nh, offB = ((long long)pi * N + pj) * Nh;
        pair_sync<NT>();
        zfft_step<M, NR, M, true, NT>(rows, m1, m2, offA, offB, ztw, lane);
        // every row pair's transform is in shared memory before any store:
        // the stores below overwrite only this pair's rows
        const bool self = pi == i && pj == j;
#pragma unroll
        for (int q = 0; q < NR / 2; ++q) {
            float2 *dst = q ? m2 : m1;
            const float2 *ra = rows + (2 * q) * RS, *rb = ra + RS;
            for (int l = lane; l < Nh; l += NT) {
                const int sl = zslot(l), la = zslot(l == M ? 0 : l), lb = zslot(l == 0 ? 0 : M - l);
                const float2 w = swl[sl];
                const float2 dA = split2(ra[la], rb[lb], w);
                dst[offA + l] = make_float2(0.5f * dA.x, 0.5f * dA.y);
                if (!self) {
                    const float2 dB = split2(rb[la], ra[lb], w);
                    dst[offB + l] = make_float2(0.5f * dB.x, 0.5f * dB.y);
                }
            }
        }
    }
}

template <int M, bool IL, bool TWOD, bool POLES>
cudaError_t zbin_inst(const void *mesh, long long is, long long ms, int nitems, int G, const BinGeom &g,
                      const void *cw, const void *ph, const void *tw, const int *kedge, void *partial,
                      cudaStream_t st) {
    constexpr int NR = IL ? 4 : 2;
    const size_t smem = ZSmem<M, NR>::bytes(g);
    auto kern = (g.mu32 || !TWOD) ? k_zbin<IL, TWOD, POLES, true, M> : k_zbin<IL, TWOD, POLES, false, M>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    dim3 grid(G, nitems);
    kern<<<grid, 32 * ZRows<M>::WPB, smem, st>>>(
        reinterpret_cast<const float2 *>(mesh), is, ms, g, reinterpret_cast<const float *>(cw),
        reinterpret_cast<const float2 *>(ph), reinterpret_cast<const float2 *>(tw), kedge,
        reinterpret_cast<float *>(partial));
    return cudaGetLastError();
}

template <int M>
cudaError_t zbin_dispatch(const void *mesh, int il, long long is, long long ms, int nitems, int G,
                          const BinGeom &g, const void *cw, const void *ph, const void *tw, const int *kedge,
                          void *partial, cudaStream_t st) {
    const int key = (il ? 4 : 0) | (g.twod ? 2 : 0) | (g.poles ? 1 : 0);
#define PK_ZBIN(a, b, c) zbin_inst<M, a, b, c>(mesh, is, ms, nitems, G, g, cw, ph, tw, kedge, partial, st)
    switch (key) {
    case 0: return PK_ZBIN(false, false, false);
    case 1: return PK_ZBIN(false, false, true);
    case 2: return PK_ZBIN(false, true, false);
    case 3: return PK_ZBIN(false, true, true);
    case 4: return PK_ZBIN(true, false, false);
    case 5: return PK_ZBIN(true, false, true);
    case 6: return PK_ZBIN(true, true, false);
    default: return PK_ZBIN(true, true, true);
    }
#undef PK_ZBIN
}

template <int M, int NR>
cudaError_t zfinish_inst(void *mesh, long long is, long long ms, int nitems, int nsm, const void *tw,
                         cudaStream_t st) {
    const size_t smem = ZSmem<M, NR>::off_hist();
    auto kern = k_zfinish<M, NR>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int occ = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, 32 * ZRows<M>::WPB, smem) != cudaSuccess ||
        occ < 1) {
        cudaGetLastError();
        occ = 1;
    }
    dim3 grid((unsigned)(nsm > 0 ? nsm : 1) * occ, nitems);
    kern<<<grid, 32 * ZRows<M>::WPB, smem, st>>>(reinterpret_cast<float2 *>(mesh), is, ms,
                                                 reinterpret_cast<const float2 *>(tw));
    return cudaGetLastError();
}

}  // namespace

bool own_fft_supported(int N) { return N == 128 || N == 192 || N == 256 || N == 512 || N == 1024 || N == 2048; }

// Measured on a GB300 (FFT + bin): 32 catalogs of 128^3 0.40 against 0.56 ms
// with cuFFT, 24 of 192^3 1.07 against 1.35 ms, 512^3 1.25 against 1.84 ms,
// 2048^3 121 against 234 ms; at 1024^3 13.4 against 12.7 ms (the CTA-per-pair
// z pass is latency-bound at 16 warps per SM), so 1024 keeps cuFFT unless the
// caller asks for the own transform.
bool own_fft_default(int N) { return N == 128 || N == 192 || N == 256 || N == 512 || N == 2048; }

void own_fft_twiddles(int N, float *tw) {
    for (int e = 0; e < N; ++e) {
        double c = cos(2.0 * M_PI * e / N), s = -sin(2.0 * M_PI * e / N);
        if (4 * e % N == 0) {            // the quarter turns exactly
            const int q = 4 * e / N;
            c = q == 0 ? 1.0 : q == 2 ? -1.0 : 0.0;
            s = q == 1 ? -1.0 : q == 3 ? 1.0 : 0.0;
        }
        tw[2 * e] = (float)c;
        tw[2 * e + 1] = (float)s;
    }
}

cudaError_t launch_fft_xy(void *mesh, int nmesh, long long mesh_c, int N, const void *tw, cudaStream_t st) {
    float2 *m = reinterpret_cast<float2 *>(mesh);
    const float2 *t = reinterpret_cast<const float2 *>(tw);
    switch (N) {
    case 128: return axis_inst<128>(m, nmesh, mesh_c, t, st);
    case 192: return axis_inst<192>(m, nmesh, mesh_c, t, st);
    case 256: return axis_inst<256>(m, nmesh, mesh_c, t, st);
    case 512: return axis_inst<512>(m, nmesh, mesh_c, t, st);
    case 1024: return axis_inst<1024>(m, nmesh, mesh_c, t, st);
    case 2048: return axis_inst<2048>(m, nmesh, mesh_c, t, st);
    default: return cudaErrorInvalidValue;
    }
}

size_t zbin_smem_bytes(const BinGeom &g, int interlaced) {
    switch (g.N) {
    case 128: return interlaced ? ZSmem<64, 4>::bytes(g) : ZSmem<64, 2>::bytes(g);
    case 192: return interlaced ? ZSmem<96, 4>::bytes(g) : ZSmem<96, 2>::bytes(g);
    case 256: return interlaced ? ZSmem<128, 4>::bytes(g) : ZSmem<128, 2>::bytes(g);
    case 512: return interlaced ? ZSmem<256, 4>::bytes(g) : ZSmem<256, 2>::bytes(g);
    case 1024: return interlaced ? ZSmem<512, 4>::bytes(g) : ZSmem<512, 2>::bytes(g);
    case 2048: return interlaced ? ZSmem<1024, 4>::bytes(g) : ZSmem<1024, 2>::bytes(g);
    default: return 0;
    }
}

int zbin_ctas_per_sm(const BinGeom &g, int interlaced) {
    const size_t smem = zbin_smem_bytes(g, interlaced);
    if (smem == 0) return 1;
    int threads = 0;
    const void *kern = nullptr;
#define PK_ZK(M)                                                                                            \
    threads = 32 * ZRows<M>::WPB;                                                                           \
    kern = interlaced ? reinterpret_cast<const void *>(k_zbin<true, true, true, true, M>)                   \
                      : reinterpret_cast<const void *>(k_zbin<false, true, true, true, M>);
    if (g.N == 128) {
        PK_ZK(64)
    } else if (g.N == 192) {
        PK_ZK(96)
    } else if (g.N == 256) {
        PK_ZK(128)
    } else if (g.N == 512) {
        PK_ZK(256)
    } else if (g.N == 1024) {
        PK_ZK(512)
    } else {
        PK_ZK(1024)
    }
#undef PK_ZK
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) {
        cudaGetLastError();
        return 1;
    }
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kern, threads, smem) != cudaSuccess || n < 1) {
        cudaGetLastError();
        n = 1;
    }
    return n;
}

cudaError_t launch_zbin(const void *mesh, int interlaced, long long item_stride_c, long long mesh_stride_c,
                        int nitems, int ctas_per_item, const BinGeom &g, const void *cw, const void *ph,
                        const void *tw, const int *kedge, void *partial, cudaStream_t st) {
    switch (g.N) {
    case 128:
        return zbin_dispatch<64>(mesh, interlaced, item_stride_c, mesh_stride_c, nitems, ctas_per_item, g, cw,
                                 ph, tw, kedge, partial, st);
    case 192:
        return zbin_dispatch<96>(mesh, interlaced, item_stride_c, mesh_stride_c, nitems, ctas_per_item, g, cw,
                                 ph, tw, kedge, partial, st);
    case 256:
        return zbin_dispatch<128>(mesh, interlaced, item_stride_c, mesh_stride_c, nitems, ctas_per_item, g, cw,
                                  ph, tw, kedge, partial, st);
    case 512:
        return zbin_dispatch<256>(mesh, interlaced, item_stride_c, mesh_stride_c, nitems, ctas_per_item, g, cw,
                                  ph, tw, kedge, partial, st);
    case 1024:
        return zbin_dispatch<512>(mesh, interlaced, item_stride_c, mesh_stride_c, nitems, ctas_per_item, g, cw,
                                  ph, tw, kedge, partial, st);
    case 2048:
        return zbin_dispatch<1024>(mesh, interlaced, item_stride_c, mesh_stride_c, nitems, ctas_per_item, g, cw,
                                   ph, tw, kedge, partial, st);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_zfinish(void *mesh, int interlaced, long long item_stride_c, long long mesh_stride_c,
                           int nitems, int N, const void *tw, int nsm, cudaStream_t st) {
    switch (N) {
    case 128:
        return interlaced ? zfinish_inst<64, 4>(mesh, item_stride_c, mesh_stride_c, nitems, nsm, tw, st)
                          : zfinish_inst<64, 2>(mesh, item_stride_c, mesh_stride_c, nitems, nsm, tw, st);
    case 192:
        return interlaced ? zfinish_inst<96, 4>(mesh, item_stride_c, mesh_stride_c, nitems, nsm, tw, st)
                          : zfinish_inst<96, 2>(mesh, item_stride_c, mesh_stride_c, nitems, nsm, tw, st);
    case 256:
        return interlaced ? zfinish_inst<128, 4>(mesh, item_stride_c, mesh_stride_c, nitems, nsm, tw, st)
                          : zfinish_inst<128, 2>(mesh, item_stride_c, mesh_stride_c, nitems, nsm, tw, st);
    case 512:
        return interlaced ? zfinish_inst<256, 4>(mesh, item_stride_c, mesh_stride_c, nitems, nsm, tw, st)
                          : zfinish_inst<256, 2>(mesh, item_stride_c, mesh_stride_c, nitems, nsm, tw, st);
    case 1024:
        return interlaced ? zfinish_inst<512, 4>(mesh, item_stride_c, mesh_stride_c, nitems, nsm, tw, st)
                          : zfinish_inst<512, 2>(mesh, item_stride_c, mesh_stride_c, nitems, nsm, tw, st);
    case 2048:
        return interlaced ? zfinish_inst<1024, 4>(mesh, item_stride_c, mesh_stride_c, nitems, nsm, tw, st)
                          : zfinish_inst<1024, 2>(mesh, item_stride_c, mesh_stride_c, nitems, nsm, tw, st);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace pk
