// pk_survey.cu -- survey power-spectrum multipoles (the ConvolvedFFTPower of
// Sec. 3.4.1): FKP field of data and randoms, local line of sight through the
// real spherical harmonics (2l + 1 transforms for multipole l), FKP
// normalization and shot noise.  The estimator, its readings and the sky ->
// Cartesian convention are stated in include/pk.h.
//
// Pipeline on the plan's stream (one GPU):
//   paint    k_survey_prep converts each catalog (sky or Cartesian) into
//            box-frame positions + w_comp w_fkp and takes its FP64 sums;
//            the tile-sort paint of an internal pk plan (batch 2) paints data
//            into catalog 0's meshes and randoms into catalog 1's;
//            k_survey_const reduces the sums to alpha, I and S.
//   compute  interlaced: k_fkp_combine (F = D - alpha R on both meshes), r2c
//            of both, k_survey_interlace (A_0 = the combination, and the
//            same / N^3 for the inverse), c2r -> the real field F.
//            For each batch of Y_lm slots: k_survey_ylm writes F Y_lm(x^)
//            (non-interlaced: F = D - alpha R on the fly, and the first batch
//            also copies F for A_0), one r2c per mesh, k_survey_bin adds
//            h cw Y_lm(k^) Re[A_lm A_0^*] (and h cw |A_0|^2 once) into
//            per-CTA FP64 rows; k_survey_final reduces the rows in a fixed
//            order and normalizes.
//   bounds   k_survey_bounds + k_survey_bounds_final: a catalog's observer-
//            frame bounding box (pk_survey_bounds), for choosing the box.
#include <cuda_runtime.h>
#include <cufft.h>

#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <string>
#include <vector>

#include "pk_internal.h"
#include "pk_plan.h"

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

namespace {

constexpr int kSlots = 14;              // Y_lm slots: 0..4 -> l = 2, m = s - 2; 5..13 -> l = 4, m = s - 9
constexpr int kPrepThreads = 256;
constexpr int kPrepCtasPerSm = 4;
constexpr int kSums = 5;                // per catalog: sum wc, sum w^2, sum nbar wc wf^2, outside, rejected
constexpr int kRowThreads = 256;        // warp-per-row kernels
constexpr int kChiNodes = 8192;
constexpr double kCOverH0 = 2997.92458;
constexpr int kConst = 16;              // constants block: see k_survey_const

// Real spherical harmonics of the unit vector (x, y, z), orthonormal on the
// sphere: Y_lm = N_lm P_l^|m|(z) (cos m phi or sin |m| phi) written as
// polynomials in x, y, z, with N_lm from (2l + 1)/(4 pi) (l - |m|)!/(l + |m|)!
// (times 2 for m != 0).  Slot s: 0..4 -> l = 2, m = s - 2; 5..13 -> l = 4,
// m = s - 9.
constexpr double kYa = 1.0925484305920792;    // (1/2) sqrt(15/pi)
constexpr double kYb = 0.31539156525252005;   // (1/4) sqrt(5/pi)
constexpr double kYc = 0.5462742152960396;    // (1/4) sqrt(15/pi)
constexpr double kYd = 2.5033429417967046;    // (3/4) sqrt(35/pi)
constexpr double kYe = 1.7701307697799304;    // (3/4) sqrt(35/(2 pi))
constexpr double kYf = 0.9461746957575601;    // (3/4) sqrt(5/pi)
constexpr double kYg = 0.6690465435572892;    // (3/4) sqrt(5/(2 pi))
constexpr double kYh = 0.10578554691520431;   // (3/16) sqrt(1/pi)
constexpr double kYi = 0.47308734787878004;   // (3/8) sqrt(5/pi)
constexpr double kYj = 0.6258357354491761;    // (3/16) sqrt(35/pi)

template <typename T>
__host__ __device__ __forceinline__ T ylm_slot(int s, T x, T y, T z) {
    switch (s) {
    case 0: return T(kYa) * x * y;
    case 1: return T(kYa) * y * z;
    case 2: return T(kYb) * (T(3) * z * z - T(1));
    case 3: return T(kYa) * x * z;
    case 4: return T(kYc) * (x * x - y * y);
    case 5: return T(kYd) * x * y * (x * x - y * y);
    case 6: return T(kYe) * y * z * (T(3) * x * x - y * y);
    case 7: return T(kYf) * x * y * (T(7) * z * z - T(1));
    case 8: return T(kYg) * y * z * (T(7) * z * z - T(3));
    case 9: return T(kYh) * ((T(35) * z * z - T(30)) * z * z + T(3));
    case 10: return T(kYg) * x * z * (T(7) * z * z - T(3));
    case 11: return T(kYi) * (x * x - y * y) * (T(7) * z * z - T(1));
    case 12: return T(kYe) * x * z * (x * x - T(3) * y * y);
    case 13: return T(kYj) * (x * x * (x * x - T(3) * y * y) - y * y * (T(3) * x * x - y * y));
    }
    return T(0);
}

// All 14 slots at once, sharing the products (the same polynomials).
template <typename T>
__device__ __forceinline__ void ylm_all(T x, T y, T z, T *Y) {
    const T x2 = x * x, y2 = y * y, z2 = z * z, xy = x * y, yz = y * z, xz = x * z, d = x2 - y2;
    const T t7 = T(7) * z2 - T(1), t3 = T(7) * z2 - T(3);
    Y[0] = T(kYa) * xy;
    Y[1] = T(kYa) * yz;
    Y[2] = T(kYb) * (T(3) * z2 - T(1));
    Y[3] = T(kYa) * xz;
    Y[4] = T(kYc) * d;
    Y[5] = T(kYd) * xy * d;
    Y[6] = T(kYe) * yz * (T(3) * x2 - y2);
    Y[7] = T(kYf) * xy * t7;
    Y[8] = T(kYg) * yz * t3;
    Y[9] = T(kYh) * ((T(35) * z2 - T(30)) * z2 + T(3));
    Y[10] = T(kYg) * xz * t3;
    Y[11] = T(kYi) * d * t7;
    Y[12] = T(kYe) * xz * (x2 - T(3) * y2);
    Y[13] = T(kYj) * (x2 * (x2 - T(3) * y2) - y2 * (T(3) * x2 - y2));
}

// ---------------------------------------------------------------- prep --

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

// Cubic Hermite interpolation of chi(z) from nodes k dz carrying (chi, dchi/dz).
__device__ __forceinline__ double chi_of_z(const double2 *__restrict__ tab, int n, double inv_dz, double dz,
                                           double z) {
    double t = z * inv_dz;
    int k = (int)t;
    if (k > n - 2) k = n - 2;
    if (k < 0) k = 0;
    const double u = t - (double)k;
    const double2 a = tab[k], b = tab[k + 1];
    const double u2 = u * u, u3 = u2 * u;
    const double h00 = 2.0 * u3 - 3.0 * u2 + 1.0, h10 = u3 - 2.0 * u2 + u;
    const double h01 = -2.0 * u3 + 3.0 * u2, h11 = u3 - u2;
    return h00 * a.x + h10 * dz * a.y + h01 * b.x + h11 * dz * b.y;
}

struct PrepArgs {
    double ox, oy, oz, L;       // box origin (observer frame), box edge
    double p0;                  // > 0: w_fkp = 1 / (1 + nbar p0)
    const double2 *chi;         // sky input: (chi, dchi/dz) at k dz
    int nchi;
    double dz, inv_dz, zmax;
};

// Observer-frame position of object i: Cartesian input as given; sky input
// (RA, Dec in degrees, z) through chi(z).  False (and the box origin) for a
// sky object with z outside [0, zmax] or NaN.
template <typename P, bool SKY>
__device__ __forceinline__ bool observer_xyz(const P *__restrict__ pos, long long i, const PrepArgs &a, double *x,
                                             double *y, double *z) {
    const double c0 = (double)pos[3 * i], c1 = (double)pos[3 * i + 1], c2 = (double)pos[3 * i + 2];
    if (!SKY) {
        *x = c0;
        *y = c1;
        *z = c2;
        return true;
    }
    if (!(c2 >= 0.0 && c2 <= a.zmax)) {
        *x = a.ox;
        *y = a.oy;
        *z = a.oz;
        return false;
    }
    const double r = chi_of_z(a.chi, a.nchi, a.inv_dz, a.dz, c2);
    double sr, cr, sd, cd;
    sincospi(c0 / 180.0, &sr, &cr);
    sincospi(c1 / 180.0, &sd, &cd);
    *x = r * cd * cr;
    *y = r * cd * sr;
    *z = r * sd;
    return true;
}

// Per-CTA minimum and maximum of the observer-frame positions that count
// (partial[6 b + {0,1,2}] = min x, y, z; + {3,4,5} = max).
template <typename P, bool SKY>
__global__ void __launch_bounds__(kPrepThreads)
k_survey_bounds(const P *__restrict__ pos, long long n, PrepArgs a, double *__restrict__ partial) {
    const double inf = __longlong_as_double(0x7ff0000000000000LL);
    double v[6] = {inf, inf, inf, -inf, -inf, -inf};
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        double x, y, z;
        if (!observer_xyz<P, SKY>(pos, i, a, &x, &y, &z)) continue;
        v[0] = fmin(v[0], x);
        v[1] = fmin(v[1], y);
        v[2] = fmin(v[2], z);
        v[3] = fmax(v[3], x);
        v[4] = fmax(v[4], y);
        v[5] = fmax(v[5], z);
    }
    __shared__ double red[kPrepThreads / 32][6];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
    for (int k = 0; k < 6; ++k) {
        double t = v[k];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const double u = __shfl_down_sync(0xffffffffu, t, o);
            t = k < 3 ? fmin(t, u) : fmax(t, u);
        }
        if (lane == 0) red[warp][k] = t;
    }
    __syncthreads();
    if (threadIdx.x < 6) {
        const int k = threadIdx.x;
        double t = red[0][k];
        for (int w = 1; w < kPrepThreads / 32; ++w) t = k < 3 ? fmin(t, red[w][k]) : fmax(t, red[w][k]);
        partial[6LL * blockIdx.x + k] = t;
    }
}

__global__ void k_survey_bounds_final(const double *__restrict__ partial, int G, double *__restrict__ out) {
    const int k = threadIdx.x;
    if (k >= 6) return;
    double t = partial[k];
    for (int b = 1; b < G; ++b) t = k < 3 ? fmin(t, partial[6LL * b + k]) : fmax(t, partial[6LL * b + k]);
    out[k] = t;
}

// One catalog -> box-frame positions + weights, and its FP64 sums.
// F64OUT: positions as double xyz (FP64 meshes) and weights in wout;
// otherwise float4 xyzw in out4.
template <typename P, bool SKY, bool F64OUT>
__global__ void __launch_bounds__(kPrepThreads)
k_survey_prep(const P *__restrict__ pos, long long n, const float *__restrict__ wcomp,
              const float *__restrict__ wfkp, const float *__restrict__ nbar, PrepArgs a,
              float4 *__restrict__ out4, double *__restrict__ out3, float *__restrict__ wout,
              double *__restrict__ partial) {
    double s_wc = 0.0, s_w2 = 0.0, s_n = 0.0, s_out = 0.0, s_rej = 0.0;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        double wc = wcomp ? (double)wcomp[i] : 1.0;
        const double nb = nbar ? (double)nbar[i] : 0.0;
        double wf = a.p0 > 0.0 ? 1.0 / (1.0 + nb * a.p0) : (wfkp ? (double)wfkp[i] : 1.0);
        double x, y, z;
        const bool ok = observer_xyz<P, SKY>(pos, i, a, &x, &y, &z);
        if (!ok) {
            wc = 0.0;
            wf = 0.0;
            s_rej += 1.0;
        }
        const double bx = x - a.ox, by = y - a.oy, bz = z - a.oz;
        if (ok && !(bx >= 0.0 && bx < a.L && by >= 0.0 && by < a.L && bz >= 0.0 && bz < a.L)) s_out += 1.0;
        const double w = wc * wf;
        if (F64OUT) {
            out3[3 * i] = bx;
            out3[3 * i + 1] = by;
            out3[3 * i + 2] = bz;
            wout[i] = (float)w;
        } else {
            out4[i] = make_float4((float)bx, (float)by, (float)bz, (float)w);
        }
        s_wc += wc;
        s_w2 += w * w;
        s_n += nb * wc * wf * wf;
    }
    __shared__ double red[kPrepThreads / 32][kSums];
    const double v[kSums] = {s_wc, s_w2, s_n, s_out, s_rej};
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
    for (int k = 0; k < kSums; ++k) {
        const double t = warp_sum(v[k]);
        if (lane == 0) red[warp][k] = t;
    }
    __syncthreads();
    if (threadIdx.x < kSums) {
        double t = 0.0;
        for (int w = 0; w < kPrepThreads / 32; ++w) t += red[w][threadIdx.x];
        partial[(long long)blockIdx.x * kSums + threadIdx.x] = t;
    }
}

// Constants block c[kConst]: 0 alpha, 1 norm I, 2 shot S, 3 wsum_d, 4 wsum_r,
// 5 w2_d, 6 w2_r, 7 nsum_r, 8 nsum_d, 9 outside_d, 10 outside_r,
// 11 rejected_d, 12 rejected_r.  Fixed-order sums of the per-CTA rows.
__global__ void k_survey_const(const double *__restrict__ pd, int gd, const double *__restrict__ pr, int gr,
                               double *__restrict__ c) {
    __shared__ double s[2][kSums];
    const int t = threadIdx.x;
    if (t < 2 * kSums) {
        const int cat = t / kSums, k = t % kSums;
        const double *p = cat == 0 ? pd : pr;
        const int g = cat == 0 ? gd : gr;
        double acc = 0.0;
        for (int b = 0; b < g; ++b) acc += p[(long long)b * kSums + k];
        s[cat][k] = acc;
    }
    __syncthreads();
    if (t == 0) {
        const double alpha = s[0][0] / s[1][0];
        const double norm = alpha * s[1][2];
        c[0] = alpha;
        c[1] = norm;
        c[2] = (s[0][1] + alpha * alpha * s[1][1]) / norm;
        c[3] = s[0][0];
        c[4] = s[1][0];
        c[5] = s[0][1];
        c[6] = s[1][1];
        c[7] = s[1][2];
        c[8] = s[0][2];
        c[9] = s[0][3];
        c[10] = s[1][3];
        c[11] = s[0][4];
        c[12] = s[1][4];
        for (int k = 13; k < kConst; ++k) c[k] = 0.0;
    }
}

// ------------------------------------------------------------- compute --

template <typename T> struct VecOf;
template <> struct VecOf<float> { using type = float4; };     // 4 reals per load
template <> struct VecOf<double> { using type = double2; };   // 2 reals per load

// d[i] -= alpha r[i] over n reals (n a multiple of the vector width).
template <typename T>
__global__ void __launch_bounds__(256)
k_fkp_combine(T *__restrict__ d, const T *__restrict__ r, long long n, const double *__restrict__ c) {
    using V = typename VecOf<T>::type;
    constexpr int W = sizeof(V) / sizeof(T);
    const T alpha = (T)c[0];
    V *dv = reinterpret_cast<V *>(d);
    const V *rv = reinterpret_cast<const V *>(r);
    const long long nv = n / W;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < nv;
         i += (long long)gridDim.x * blockDim.x) {
        V a = dv[i];
        const V b = __ldcs(rv + i);
        if constexpr (W == 4) {
            a.x -= alpha * b.x;
            a.y -= alpha * b.y;
            a.z -= alpha * b.z;
            a.w -= alpha * b.w;
        } else {
            a.x -= alpha * b.x;
            a.y -= alpha * b.y;
        }
        dv[i] = a;
    }
}

template <typename C>
__device__ __forceinline__ C cmulc(C a, C b) {
    C r;
    r.x = a.x * b.x - a.y * b.y;
    r.y = a.x * b.y + a.y * b.x;
    return r;
}

// A_0 = (F~1 + F~2 e^{i pi (i' + j' + l) / N}) / 2 on every mode with no
// index at N/2 (zero there); F~1 <- A_0 / N^3 for the inverse transform.
template <typename R, typename C>
__global__ void __launch_bounds__(kRowThreads)
k_survey_interlace(C *__restrict__ f1, const C *__restrict__ f2, C *__restrict__ a0, const C *__restrict__ ph,
                   int N, int Nh, R inv_n3) {
    const int half = N / 2;
    const long long rows = (long long)N * N;
    const int lane = threadIdx.x & 31;
    const long long w0 = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
    for (long long row = w0; row < rows; row += nw) {
        const int i = (int)(row / N), j = (int)(row - (long long)i * N);
        const int ip = i < half ? i : i - N, jp = j < half ? j : j - N;
        const bool nyq_row = i == half || j == half;
        const C rp = cmulc(ph[ip + half], ph[jp + half]);
        const long long base = row * Nh;
        for (int l = lane; l < Nh; l += 32) {
            C z;
            z.x = (R)0;
            z.y = (R)0;
            if (!nyq_row && l != half) {
                const C a = f1[base + l], b = f2[base + l];
                const C t = cmulc(rp, ph[l + half]);
                z.x = (R)0.5 * (a.x + b.x * t.x - b.y * t.y);
                z.y = (R)0.5 * (a.y + b.x * t.y + b.y * t.x);
            }
            a0[base + l] = z;
            C s;
            s.x = z.x * inv_n3;
            s.y = z.y * inv_n3;
            f1[base + l] = s;
        }
    }
}

template <typename T> struct PairOf;
template <> struct PairOf<float> { using type = float2; };
template <> struct PairOf<double> { using type = double2; };

// Y_lm-weighted copies of the real field: out[s][cell] = F(cell) Y_{s0+s}(x^).
// FKP: F = D - alpha R read from the two catalogs' meshes (else F = D).
// a0: if not NULL, F is also copied there (real layout) for A_0.  Two cells
// per lane and two such pairs per step, loads first; rows are written whole,
// padding pair included (as zeros), so the stores stream without partial
// sectors.  NB > 0: the slots [S0, S0 + NB) fixed at compile time; NB = 0:
// s0, nb.
template <typename T, bool FKP, int S0, int NB>
__global__ void __launch_bounds__(kRowThreads)
k_survey_ylm(const T *__restrict__ D, const T *__restrict__ Rm, const double *__restrict__ c, T *__restrict__ a0,
             T *__restrict__ out, long long stride, int s0, int nb, int N, int rowlen, T ox, T oy, T oz, T H) {
    using T2 = typename PairOf<T>::type;
    const T alpha = FKP ? (T)c[0] : (T)0;
    const long long rows = (long long)N * N;
    const int lane = threadIdx.x & 31;
    const int npair = N / 2, nrow = rowlen / 2;     // pairs with cells, pairs per stored row
    const long long w0 = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
    for (long long row = w0; row < rows; row += nw) {
        const int i = (int)(row / N), j = (int)(row - (long long)i * N);
        const T x = ox + (T)i * H, y = oy + (T)j * H;
        const T rxy = x * x + y * y;
        const long long base = row * rowlen;
        for (int q0 = lane; q0 < nrow; q0 += 64) {
            T2 f[2];
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int q = q0 + 32 * h;
                f[h].x = (T)0;
                f[h].y = (T)0;
                if (q < npair) {
                    f[h] = __ldcs(reinterpret_cast<const T2 *>(D + base + 2 * q));
                    if (FKP) {
                        const T2 r = __ldcs(reinterpret_cast<const T2 *>(Rm + base + 2 * q));
                        f[h].x -= alpha * r.x;
                        f[h].y -= alpha * r.y;
                    }
                }
            }
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int q = q0 + 32 * h;
                if (q >= nrow) break;
                const long long idx = base + 2 * q;
                if (a0) *reinterpret_cast<T2 *>(a0 + idx) = f[h];
                T u[2][3], g[2];
#pragma unroll
                for (int e = 0; e < 2; ++e) {
                    const T z = oz + (T)(2 * q + e) * H;
                    const T r2 = rxy + z * z;
                    u[e][0] = u[e][1] = u[e][2] = (T)0;
                    g[e] = (T)0;
                    if (q < npair && r2 > (T)0) {
                        T inv;
                        if constexpr (sizeof(T) == 4) inv = rsqrtf(r2);
                        else inv = (T)1 / sqrt(r2);
                        u[e][0] = x * inv;
                        u[e][1] = y * inv;
                        u[e][2] = z * inv;
                        g[e] = e == 0 ? f[h].x : f[h].y;
                    }
                }
                if constexpr (NB > 0) {
                    T Y0[kSlots], Y1[kSlots];
                    ylm_all<T>(u[0][0], u[0][1], u[0][2], Y0);
                    ylm_all<T>(u[1][0], u[1][1], u[1][2], Y1);
#pragma unroll
                    for (int s = 0; s < NB; ++s) {
                        T2 o;
                        o.x = g[0] * Y0[S0 + s];
                        o.y = g[1] * Y1[S0 + s];
                        __stcs(reinterpret_cast<T2 *>(out + (long long)s * stride + idx), o);
                    }
                } else {
                    for (int s = 0; s < nb; ++s) {
                        T2 o;
                        o.x = g[0] * ylm_slot<T>(s0 + s, u[0][0], u[0][1], u[0][2]);
                        o.y = g[1] * ylm_slot<T>(s0 + s, u[1][0], u[1][1], u[1][2]);
                        __stcs(reinterpret_cast<T2 *>(out + (long long)s * stride + idx), o);
                    }
                }
            }
        }
    }
}

// Per-mode sums of one batch: hist[b] += h cw |A_0|^2 (first batch only),
// hist[nk + b] / hist[2 nk + b] += h cw sum_s Y_s(k^) Re[A_s A_0^*] over the
// batch's l = 2 / l = 4 slots.  Each CTA adds its histogram into its own FP64
// row of `partial` (the first batch overwrites).  NB > 0: slots [S0, S0 + NB)
// fixed at compile time; NB = 0: s0, nb.
template <typename R, typename C, int S0, int NB>
__global__ void __launch_bounds__(kRowThreads, sizeof(R) == 4 ? 6 : 1)
k_survey_bin(const C *__restrict__ A0, const C *__restrict__ S, long long stride_c, int s0, int nb, int first,
             pk::BinGeom g, const R *__restrict__ cw, const int *__restrict__ kedge, double *__restrict__ partial) {
    extern __shared__ __align__(16) unsigned char smraw[];
    const int nk = g.nk;
    R *hist = reinterpret_cast<R *>(smraw);
    int2 *sedge = reinterpret_cast<int2 *>(smraw + ((3 * nk * sizeof(R) + 15) / 16) * 16);
    for (int k = threadIdx.x; k < 3 * nk; k += blockDim.x) hist[k] = (R)0;
    for (int k = threadIdx.x; k < nk; k += blockDim.x) sedge[k] = make_int2(kedge[k], kedge[k + 1]);
    __syncthreads();
    const int N = g.N, Nh = g.Nh, half = N / 2;
    const long long rows = (long long)N * N;
    const int lane = threadIdx.x & 31;
    const long long w0 = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
    const int sb = NB > 0 ? S0 : s0, ne = NB > 0 ? NB : nb;
    const bool has2 = ne > 0 && sb < 5, has4 = ne > 0 && sb + ne > 5;
    for (long long row = w0; row < rows; row += nw) {
        const int i = (int)(row / N), j = (int)(row - (long long)i * N);
        const int ip = i < half ? i : i - N, jp = j < half ? j : j - N;
        const int r2 = ip * ip + jp * jp;
        if (r2 >= g.mhi) continue;
        const R rowcw = cw[i] * cw[j];
        const long long base = row * Nh;
        for (int l = lane; l < Nh; l += 32) {
            const int m = r2 + l * l;
            if (m >= g.mhi) break;
            if (m == 0 || m < g.mlo) continue;
            R rs;
            if constexpr (sizeof(R) == 4) rs = rsqrtf((float)m);
            else rs = (R)1 / sqrt((R)m);
            int b = (int)((float)m * (float)rs * g.kscale - g.koff);
            b = min(max(b, 0), nk - 1);
            int2 e = sedge[b];
            while (b > 0 && m < e.x) e = sedge[--b];
            while (b < nk - 1 && m >= e.y) e = sedge[++b];
            R w = rowcw * cw[l];
            if (l != 0 && l != half) w += w;
            const C a = __ldcs(A0 + base + l);
            if (first) atomicAdd(hist + b, w * (a.x * a.x + a.y * a.y));
            if (ne == 0) continue;
            const R kx = (R)ip * rs, ky = (R)jp * rs, kz = (R)l * rs;
            R t2 = (R)0, t4 = (R)0;
            if constexpr (NB > 0) {
                R Y[kSlots];
                ylm_all<R>(kx, ky, kz, Y);
#pragma unroll
                for (int s = 0; s < NB; ++s) {
                    const C v = __ldcs(S + (long long)s * stride_c + base + l);
                    const R re = v.x * a.x + v.y * a.y;
                    if (S0 + s < 5) t2 += Y[S0 + s] * re;
                    else t4 += Y[S0 + s] * re;
                }
            } else {
                for (int s = 0; s < nb; ++s) {
                    const C v = __ldcs(S + (long long)s * stride_c + base + l);
                    const R re = v.x * a.x + v.y * a.y;
                    const R y = ylm_slot<R>(s0 + s, kx, ky, kz);
                    if (s0 + s < 5) t2 += y * re;
                    else t4 += y * re;
                }
            }
            if (has2) atomicAdd(hist + nk + b, w * t2);
            if (has4) atomicAdd(hist + 2 * nk + b, w * t4);
        }
    }
    __syncthreads();
    double *out = partial + (long long)blockIdx.x * 3 * nk;
    for (int k = threadIdx.x; k < 3 * nk; k += blockDim.x) out[k] = (first ? 0.0 : out[k]) + (double)hist[k];
}

// res[l_row * nk + b]: P_0 = T0 / (modes I) - S, P_l = 4 pi T_l / (modes I);
// rows not in the mask and empty bins NaN; res[3 nk ..] = the constants block.
__global__ void k_survey_final(const double *__restrict__ partial, int G, int nk,
                               const unsigned long long *__restrict__ modes, const double *__restrict__ c,
                               unsigned mask, int subtract_shot, double *__restrict__ res) {
    const double nan = __longlong_as_double(0x7ff8000000000000LL);
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < 3 * nk; k += gridDim.x * blockDim.x) {
        const int row = k / nk, b = k - row * nk;
        double t = 0.0;
        for (int q = 0; q < G; ++q) t += partial[(long long)q * 3 * nk + k];
        const double md = (double)modes[b];
        double p = nan;
        if ((mask >> row) & 1u) {
            if (md > 0.0) {
                const double norm = c[1];
                if (row == 0) p = t / (md * norm) - (subtract_shot ? c[2] : 0.0);
                else p = 4.0 * M_PI * t / (md * norm);
            }
        }
        res[k] = p;
    }
    if (blockIdx.x == 0 && threadIdx.x < kConst) res[3 * nk + threadIdx.x] = c[threadIdx.x];
}

}  // namespace

// ==================================================================== host

struct pk_survey_s {
    pk_survey_config cfg{};
    pk_plan_t P = nullptr;          // paint machinery, tables and geometry (batch 2)
    cudaStream_t st = nullptr;
    int N = 0, Nh = 0, nm = 1, f64 = 0, nsm = 0;
    size_t esz = 4;
    long long mesh_reals = 0;
    int sa = 0, sb = 0;             // active Y_lm slots [sa, sb)
    int batch = 0;                  // Y_lm-weighted meshes resident per pass
    void *a0 = nullptr;             // A_0: one mesh (complex half grid)
    void *slots = nullptr;          // batch meshes
    cufftHandle fft_b = 0, fft_inv = 0;   // single-mesh r2c, single-mesh c2r
    int have_b = 0, have_inv = 0;
    void *fft_work = nullptr;
    void *obj = nullptr;            // staged box-frame objects (data then randoms)
    int64_t obj_cap = 0;
    void *stage = nullptr;          // host inputs copied here
    size_t stage_cap = 0;
    double2 *chi = nullptr;         // (chi, dchi/dz) at k dz
    double dz = 0.0;
    int G = 0;                      // prep CTAs per catalog
    double *psum = nullptr;         // [2][G][kSums]
    double *cst = nullptr;          // kConst
    int Gb = 0;                     // bin CTAs
    double *partial = nullptr;      // [Gb][3 nk]
    double *res = nullptr, *h_res = nullptr;
    cudaEvent_t done = nullptr;
    int painted = 0, have_rand = 0, computed = 0;
    int64_t nd = 0, nr = 0;
    long long launches = 0;
    int timing = 0;
    std::vector<cudaEvent_t> ev;                  // timing events, reused
    std::vector<int> seg_paint, seg_compute;      // stage of segment i (event i .. i + 1)
    int ev_paint0 = 0, ev_compute0 = 0;           // first event of each list
    std::string err;
};

namespace {

pk_status sfail(pk_survey_s *S, pk_status s, const std::string &msg) {
    if (S) S->err = msg;
    else pk::set_plan_error(msg.c_str());
    return s;
}

#define SV_CUDA(S, call)                                                                       \
    do {                                                                                       \
        cudaError_t e_ = (call);                                                               \
        if (e_ != cudaSuccess)                                                                 \
            return sfail(S, e_ == cudaErrorMemoryAllocation ? PK_ENOMEM : PK_ECUDA,            \
                         std::string(#call) + ": " + cudaGetErrorString(e_));                  \
    } while (0)

#define SV_CUFFT(S, call)                                                                      \
    do {                                                                                       \
        cufftResult r_ = (call);                                                               \
        if (r_ != CUFFT_SUCCESS)                                                               \
            return sfail(S, r_ == CUFFT_ALLOC_FAILED ? PK_ENOMEM : PK_ECUFFT,                  \
                         std::string(#call) + ": cufftResult " + std::to_string((int)r_));    \
    } while (0)

bool dev_ptr(const void *p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// Start a timed segment of `stage` (list 0: paint, 1: compute); stage < 0
// closes the list.  Events come from a pool: paint uses the front, compute
// the rest.
cudaError_t tmark(pk_survey_s *S, int list, int stage) {
    if (!S->timing) return cudaSuccess;
    std::vector<int> &seg = list == 0 ? S->seg_paint : S->seg_compute;
    const int base = list == 0 ? 0 : 16;
    const int idx = base + (int)seg.size();
    if (idx >= (list == 0 ? 16 : 16 + 256)) return cudaSuccess;
    while ((int)S->ev.size() <= idx) {
        cudaEvent_t e;
        cudaError_t r = cudaEventCreate(&e);
        if (r != cudaSuccess) return r;
        S->ev.push_back(e);
    }
    cudaError_t r = cudaEventRecord(S->ev[idx], S->st);
    if (r == cudaSuccess) seg.push_back(stage);
    return r;
}

void free_survey(pk_survey_s *S) {
    if (!S) return;
    if (S->st || S->P) cudaStreamSynchronize(S->st);
    if (S->have_b) cufftDestroy(S->fft_b);
    if (S->have_inv) cufftDestroy(S->fft_inv);
    void *dev[] = {S->a0, S->slots, S->fft_work, S->obj, S->stage, S->chi, S->psum, S->cst, S->partial, S->res};
    for (void *d : dev)
        if (d) cudaFree(d);
    if (S->h_res) cudaFreeHost(S->h_res);
    if (S->done) cudaEventDestroy(S->done);
    for (cudaEvent_t e : S->ev) cudaEventDestroy(e);
    if (S->P) pk_destroy(S->P);
    delete S;
}

double inv_E(double z, double om) { return 1.0 / sqrt(om * (1.0 + z) * (1.0 + z) * (1.0 + z) + 1.0 - om); }

// chi at nodes k dz by composite 8-point Gauss-Legendre quadrature, FP64.
void chi_table(double om, double zmax, std::vector<double> &tab, double *dz_out) {
    static const double gx[4] = {0.1834346424956498, 0.5255324099163290, 0.7966664774136267,
                                 0.9602898564975363};
    static const double gw[4] = {0.3626837833783620, 0.3137066458778873, 0.2223810344533745,
                                 0.1012285362903763};
    const double dz = zmax / (kChiNodes - 1);
    tab.assign(2 * kChiNodes, 0.0);
    double chi = 0.0;
    for (int k = 0; k < kChiNodes; ++k) {
        const double z = k * dz;
        if (k > 0) {
            const double a = (k - 1) * dz, mid = a + 0.5 * dz, hw = 0.5 * dz;
            double acc = 0.0;
            for (int q = 0; q < 4; ++q)
                acc += gw[q] * (inv_E(mid - hw * gx[q], om) + inv_E(mid + hw * gx[q], om));
            chi += kCOverH0 * hw * acc;
        }
        tab[2 * k] = chi;
        tab[2 * k + 1] = kCOverH0 * inv_E(z, om);
    }
    *dz_out = dz;
}

// Copy a host array into the staging buffer at byte offset `at` (device
// arrays pass through).
const void *stage_in(pk_survey_s *S, const void *p, size_t bytes, size_t *at, bool dev) {
    if (!p || dev) return p;
    char *dst = reinterpret_cast<char *>(S->stage) + *at;
    if (cudaMemcpyAsync(dst, p, bytes, cudaMemcpyHostToDevice, S->st) != cudaSuccess) return nullptr;
    *at += (bytes + 255) / 256 * 256;
    return dst;
}

}  // namespace

extern "C" {

void pk_survey_config_default(pk_survey_config *c) {
    if (!c) return;
    memset(c, 0, sizeof(*c));
    c->box_size = 1000.0;
    c->nmesh = 256;
    c->window = PK_CIC;
    c->interlaced = 0;
    c->compensated = 1;
    c->dk = 2.0 * (2.0 * M_PI) / c->box_size;
    c->poles_mask = 7u;
    c->precision = PK_MESH_F32;
    c->subtract_shot = 1;
    c->omega_m = 0.31;
    c->zmax = 5.0;
}

double pk_survey_ylm(int l, int m, double x, double y, double z) {
    if ((l != 2 && l != 4) || m < -l || m > l) return NAN;
    const int s = l == 2 ? m + 2 : 5 + m + 4;
    return ylm_slot<double>(s, x, y, z);
}

static pk_status survey_build(pk_survey_s *S, const pk_survey_config *cfg, void *stream) {
    const pk_survey_config &c = *cfg;
    if (!(c.box_size > 0.0) || !isfinite(c.box_size)) return sfail(S, PK_EINVAL, "box_size must be > 0");
    for (int a = 0; a < 3; ++a)
        if (!isfinite(c.box_origin[a])) return sfail(S, PK_EINVAL, "box_origin must be finite");
    if (c.poles_mask == 0 || (c.poles_mask & ~7u) != 0)
        return sfail(S, PK_EINVAL, "poles_mask must be a nonzero subset of bits 0..2");
    if (c.omega_m < 0.0 || c.omega_m > 1.0 || !isfinite(c.omega_m))
        return sfail(S, PK_EINVAL, "omega_m must be in [0, 1] (0: no sky input)");
    if (c.zmax < 0.0 || c.zmax > 1100.0 || !isfinite(c.zmax)) return sfail(S, PK_EINVAL, "zmax must be in [0, 1100]");
    if (!(c.p0_fkp >= 0.0) || !isfinite(c.p0_fkp)) return sfail(S, PK_EINVAL, "p0_fkp must be >= 0");
    if (c.max_batch < 0) return sfail(S, PK_EINVAL, "max_batch must be >= 0");
    if (c.capacity < 0) return sfail(S, PK_EINVAL, "capacity must be >= 0");
    S->cfg = c;
    if (S->cfg.zmax == 0.0) S->cfg.zmax = 5.0;

    pk_config pc;
    pk_config_default(&pc);
    pc.box_size = c.box_size;
    pc.nmesh = c.nmesh;
    pc.window = c.window;
    pc.interlaced = c.interlaced;
    pc.compensated = c.compensated;
    pc.kmin = c.kmin;
    pc.kmax = c.kmax;
    pc.dk = c.dk;
    pc.nmu = 0;
    pc.poles_mask = 1u;
    pc.precision = c.precision;
    pc.batch = 2;
    pc.capacity = c.capacity;
    pk_status s = pk_plan(&pc, stream, &S->P);
    if (s != PK_OK) return sfail(S, s, pk_plan_error());
    pk_plan_s *P = S->P;
    S->st = P->st;
    S->N = P->N;
    S->Nh = P->Nh;
    S->nm = P->nm;
    S->f64 = P->f64;
    S->esz = P->esz;
    S->nsm = P->nsm;
    S->mesh_reals = P->mesh_reals;
    S->sa = (c.poles_mask & 2u) ? 0 : 5;
    S->sb = (c.poles_mask & 4u) ? kSlots : 5;
    if (S->sb < S->sa) S->sb = S->sa;
    const int nslot = S->sb - S->sa;
    const size_t mesh_bytes = (size_t)S->mesh_reals * S->esz;

    SV_CUDA(S, cudaEventCreateWithFlags(&S->done, cudaEventDisableTiming));
    SV_CUDA(S, cudaMalloc(&S->a0, mesh_bytes));
    S->G = S->nsm * kPrepCtasPerSm;
    SV_CUDA(S, cudaMalloc(reinterpret_cast<void **>(&S->psum), sizeof(double) * 2 * S->G * kSums));
    SV_CUDA(S, cudaMemset(S->psum, 0, sizeof(double) * 2 * S->G * kSums));
    SV_CUDA(S, cudaMalloc(reinterpret_cast<void **>(&S->cst), sizeof(double) * kConst));
    const int nk = P->bg.nk;
    S->Gb = S->nsm * 6;                // six 256-thread bin CTAs per SM (registers capped to fit)
    SV_CUDA(S, cudaMalloc(reinterpret_cast<void **>(&S->partial), sizeof(double) * (size_t)S->Gb * 3 * nk));
    SV_CUDA(S, cudaMalloc(reinterpret_cast<void **>(&S->res), sizeof(double) * (3 * (size_t)nk + kConst)));
    SV_CUDA(S, cudaMallocHost(reinterpret_cast<void **>(&S->h_res), sizeof(double) * (3 * (size_t)nk + kConst)));
    if (c.capacity > 0) {
        const size_t per = S->f64 ? 3 * sizeof(double) + sizeof(float) : sizeof(float4);
        SV_CUDA(S, cudaMalloc(&S->obj, per * (size_t)c.capacity + 256));
        S->obj_cap = c.capacity;
    }
    if (c.omega_m > 0.0) {
        std::vector<double> tab;
        chi_table(c.omega_m, S->cfg.zmax, tab, &S->dz);
        SV_CUDA(S, cudaMalloc(reinterpret_cast<void **>(&S->chi), sizeof(double) * tab.size()));
        SV_CUDA(S, cudaMemcpy(S->chi, tab.data(), sizeof(double) * tab.size(), cudaMemcpyHostToDevice));
    }

    // Y_lm-weighted meshes resident per pass (written by one field pass, read
    // by one bin pass); each is transformed by its own single-mesh cuFFT call
    // (at 1024^3 a batched plan over 14 meshes measured 2x slower per mesh).
    if (nslot > 0) {
        int batch = nslot;
        if (c.max_batch > 0) batch = std::min(batch, c.max_batch);
        else {
            size_t fr = 0, tot = 0;
            SV_CUDA(S, cudaMemGetInfo(&fr, &tot));
            const size_t fit = fr / 2 / mesh_bytes;
            batch = (int)std::max<size_t>(1, std::min<size_t>((size_t)batch, fit));
        }
        S->batch = batch;
        SV_CUDA(S, cudaMalloc(&S->slots, mesh_bytes * (size_t)batch));
        long long n[3] = {S->N, S->N, S->N};
        long long inembed[3] = {S->N, S->N, 2LL * S->Nh};
        long long onembed[3] = {S->N, S->N, (long long)S->Nh};
        size_t work = 0, w1 = 0;
        SV_CUFFT(S, cufftCreate(&S->fft_b));
        S->have_b = 1;
        SV_CUFFT(S, cufftSetAutoAllocation(S->fft_b, 0));
        SV_CUFFT(S, cufftMakePlanMany64(S->fft_b, 3, n, inembed, 1, S->mesh_reals, onembed, 1, S->mesh_reals / 2,
                                        S->f64 ? CUFFT_D2Z : CUFFT_R2C, 1, &w1));
        work = std::max(work, w1);
        if (c.interlaced) {
            SV_CUFFT(S, cufftCreate(&S->fft_inv));
            S->have_inv = 1;
            SV_CUFFT(S, cufftSetAutoAllocation(S->fft_inv, 0));
            SV_CUFFT(S, cufftMakePlanMany64(S->fft_inv, 3, n, onembed, 1, S->mesh_reals / 2, inembed, 1,
                                            S->mesh_reals, S->f64 ? CUFFT_Z2D : CUFFT_C2R, 1, &w1));
            work = std::max(work, w1);
        }
        SV_CUDA(S, cudaMalloc(&S->fft_work, std::max<size_t>(work, 16)));
        cufftHandle hs[2] = {S->fft_b, S->fft_inv};
        int have[2] = {S->have_b, S->have_inv};
        for (int k = 0; k < 2; ++k) {
            if (!have[k]) continue;
            SV_CUFFT(S, cufftSetWorkArea(hs[k], S->fft_work));
            SV_CUFFT(S, cufftSetStream(hs[k], S->st));
        }
    }
    return PK_OK;
}

pk_status pk_survey_plan(const pk_survey_config *cfg, void *cuda_stream, pk_survey_t *out) {
    pk::set_plan_error("");
    if (!out) return sfail(nullptr, PK_EINVAL, "out is NULL");
    *out = nullptr;
    if (!cfg) return sfail(nullptr, PK_EINVAL, "cfg is NULL");
    pk_survey_s *S = new (std::nothrow) pk_survey_s();
    if (!S) return sfail(nullptr, PK_ENOMEM, "host allocation failed");
    S->st = reinterpret_cast<cudaStream_t>(cuda_stream);
    pk_status s = survey_build(S, cfg, cuda_stream);
    if (s != PK_OK) {
        pk::set_plan_error(S->err.c_str());
        free_survey(S);
        return s;
    }
    *out = S;
    return PK_OK;
}

static pk_status check_catalog(pk_survey_s *S, const pk_survey_catalog *c, bool randoms) {
    if (c->n < 0) return sfail(S, PK_EINVAL, "catalog n must be >= 0");
    if (c->dtype != PK_F32 && c->dtype != PK_F64) return sfail(S, PK_EINVAL, "catalog dtype must be PK_F32 or PK_F64");
    if (c->coord != PK_COORD_CARTESIAN && c->coord != PK_COORD_SKY)
        return sfail(S, PK_EINVAL, "catalog coord must be PK_COORD_CARTESIAN or PK_COORD_SKY");
    if (c->coord == PK_COORD_SKY && !S->chi)
        return sfail(S, PK_EINVAL, "sky coordinates need omega_m > 0 in the survey config");
    if (c->n > 0 && !c->pos) return sfail(S, PK_EINVAL, "catalog pos is NULL");
    if (randoms && c->n < 1) return sfail(S, PK_EINVAL, "the randoms need at least one object");
    if (c->n > 0 && !c->nbar && (randoms || S->cfg.p0_fkp > 0.0))
        return sfail(S, PK_EINVAL, randoms ? "the randoms need nbar (normalization)"
                                           : "p0_fkp > 0 needs the data's nbar");
    return PK_OK;
}

// Prep one catalog into the object buffer at object offset `at`.
static pk_status prep_catalog(pk_survey_s *S, const pk_survey_catalog *c, int64_t at, int cat) {
    const int64_t n = c->n;
    const bool pdev = n == 0 || dev_ptr(c->pos);
    const bool wdev = !c->wcomp || n == 0 || dev_ptr(c->wcomp);
    const bool fdev = !c->wfkp || n == 0 || dev_ptr(c->wfkp);
    const bool ndev = !c->nbar || n == 0 || dev_ptr(c->nbar);
    const size_t rb = c->dtype == PK_F64 ? 24 : 12;
    if (!pdev || !wdev || !fdev || !ndev) {
        const size_t need = ((size_t)n * rb + 255) / 256 * 256 + 3 * (((size_t)n * 4 + 255) / 256 * 256);
        if (need > S->stage_cap) {
            SV_CUDA(S, cudaStreamSynchronize(S->st));
            if (S->stage) cudaFree(S->stage);
            S->stage = nullptr;
            S->stage_cap = 0;
            SV_CUDA(S, cudaMalloc(&S->stage, need));
            S->stage_cap = need;
        } else {
            SV_CUDA(S, cudaStreamSynchronize(S->st));   // the previous catalog's copies may still read it
        }
    }
    size_t off = 0;
    const void *pos = stage_in(S, c->pos, (size_t)n * rb, &off, pdev);
    const float *wc = reinterpret_cast<const float *>(stage_in(S, c->wcomp, (size_t)n * 4, &off, wdev));
    const float *wf = reinterpret_cast<const float *>(stage_in(S, c->wfkp, (size_t)n * 4, &off, fdev));
    const float *nb = reinterpret_cast<const float *>(stage_in(S, c->nbar, (size_t)n * 4, &off, ndev));
    if ((n > 0 && !pos) || (c->wcomp && !wc) || (c->wfkp && !wf) || (c->nbar && !nb))
        return sfail(S, PK_ECUDA, "copying a host catalog to the device failed");
    PrepArgs a;
    a.ox = S->cfg.box_origin[0];
    a.oy = S->cfg.box_origin[1];
    a.oz = S->cfg.box_origin[2];
    a.L = S->cfg.box_size;
    a.p0 = S->cfg.p0_fkp;
    a.chi = S->chi;
    a.nchi = kChiNodes;
    a.dz = S->dz;
    a.inv_dz = S->dz > 0.0 ? 1.0 / S->dz : 0.0;
    a.zmax = S->cfg.zmax;
    const int64_t cap = S->obj_cap;
    float4 *o4 = S->f64 ? nullptr : reinterpret_cast<float4 *>(S->obj) + at;
    double *o3 = S->f64 ? reinterpret_cast<double *>(S->obj) + 3 * at : nullptr;
    float *ow = S->f64 ? reinterpret_cast<float *>(reinterpret_cast<double *>(S->obj) + 3 * cap) + at : nullptr;
    double *ps = S->psum + (size_t)cat * S->G * kSums;
    const bool sky = c->coord == PK_COORD_SKY;
    const bool f64in = c->dtype == PK_F64;
#define SV_PREP(PT, SK, FO)                                                                                  \
    k_survey_prep<PT, SK, FO><<<S->G, kPrepThreads, 0, S->st>>>(reinterpret_cast<const PT *>(pos), n, wc, wf, \
                                                                nb, a, o4, o3, ow, ps)
    if (S->f64) {
        if (f64in) { if (sky) SV_PREP(double, true, true); else SV_PREP(double, false, true); }
        else { if (sky) SV_PREP(float, true, true); else SV_PREP(float, false, true); }
    } else {
        if (f64in) { if (sky) SV_PREP(double, true, false); else SV_PREP(double, false, false); }
        else { if (sky) SV_PREP(float, true, false); else SV_PREP(float, false, false); }
    }
#undef SV_PREP
    SV_CUDA(S, cudaGetLastError());
    S->launches += 1;
    return PK_OK;
}

pk_status pk_survey_paint(pk_survey_t S, const pk_survey_catalog *data, const pk_survey_catalog *randoms) {
    if (!S) return PK_EINVAL;
    S->err.clear();
    if (!data) return sfail(S, PK_EINVAL, "data is NULL");
    pk_status s = check_catalog(S, data, false);
    if (s != PK_OK) return s;
    if (randoms) {
        s = check_catalog(S, randoms, true);
        if (s != PK_OK) return s;
    } else if (!S->have_rand) {
        return sfail(S, PK_ESTATE, "randoms == NULL before any randoms were painted");
    }
    const int64_t nd = data->n, nr = randoms ? randoms->n : 0;
    const int64_t ntot = nd + nr;
    if (ntot >= (int64_t)0xffffffffLL) return sfail(S, PK_EINVAL, "at most 2^32 - 2 objects per paint");
    if (ntot > S->obj_cap) {
        SV_CUDA(S, cudaStreamSynchronize(S->st));
        if (S->obj) cudaFree(S->obj);
        S->obj = nullptr;
        S->obj_cap = 0;
        const size_t per = S->f64 ? 3 * sizeof(double) + sizeof(float) : sizeof(float4);
        SV_CUDA(S, cudaMalloc(&S->obj, per * (size_t)ntot + 256));
        S->obj_cap = ntot;
    }
    S->seg_paint.clear();
    SV_CUDA(S, tmark(S, 0, PK_SURVEY_STAGE_PREP));
    s = prep_catalog(S, data, 0, 0);
    if (s != PK_OK) return s;
    if (randoms) {
        s = prep_catalog(S, randoms, nd, 1);
        if (s != PK_OK) return s;
    }
    k_survey_const<<<1, 32, 0, S->st>>>(S->psum, S->G, S->psum + (size_t)S->G * kSums, S->G, S->cst);
    SV_CUDA(S, cudaGetLastError());
    S->launches += 1;
    SV_CUDA(S, tmark(S, 0, PK_SURVEY_STAGE_PAINT));
    const int64_t off[3] = {0, nd, nd + nr};
    const int nitems = randoms ? 2 : 1;
    const long long before = pk_launch_count(S->P);
    if (S->f64) {
        const double *p3 = reinterpret_cast<const double *>(S->obj);
        const float *w = reinterpret_cast<const float *>(p3 + 3 * S->obj_cap);
        s = pk_paint_many(S->P, p3, PK_F64, w, off, nitems);
    } else {
        s = pk_paint_many(S->P, S->obj, PK_F32X4, nullptr, off, nitems);
    }
    S->launches += pk_launch_count(S->P) - before;
    if (s != PK_OK) return sfail(S, s, std::string("paint: ") + pk_last_error(S->P));
    SV_CUDA(S, tmark(S, 0, -1));
    S->nd = nd;
    if (randoms) {
        S->nr = nr;
        S->have_rand = 1;
    }
    S->painted = 1;
    S->computed = 0;
    return PK_OK;
}

}  // extern "C"

template <typename R, typename C>
static pk_status survey_compute_t(pk_survey_s *S) {
    pk_plan_s *P = S->P;
    const cudaStream_t st = S->st;
    const int N = S->N, Nh = S->Nh;
    const long long mr = S->mesh_reals;
    R *D = reinterpret_cast<R *>(P->mesh);                 // catalog 0, mesh 0
    R *Rm = D + (long long)S->nm * mr;                      // catalog 1, mesh 0
    R *A0r = reinterpret_cast<R *>(S->a0);
    C *A0 = reinterpret_cast<C *>(S->a0);
    R *SL = reinterpret_cast<R *>(S->slots);
    const int nslot = S->sb - S->sa;
    const int rowblocks = S->nsm * 8;
    const R H = (R)(S->cfg.box_size / N);
    const R ox = (R)S->cfg.box_origin[0], oy = (R)S->cfg.box_origin[1], oz = (R)S->cfg.box_origin[2];
    const bool il = S->cfg.interlaced != 0;

    S->seg_compute.clear();
    if (il) {
        // F = D - alpha R on both meshes, both transformed, combined into A_0
        SV_CUDA(S, tmark(S, 1, PK_SURVEY_STAGE_FIELD));
        k_fkp_combine<R><<<S->nsm * 8, 256, 0, st>>>(D, Rm, (long long)S->nm * mr, S->cst);
        SV_CUDA(S, cudaGetLastError());
        SV_CUDA(S, tmark(S, 1, PK_SURVEY_STAGE_FFT));
        SV_CUFFT(S, pk::transform_meshes(P, D, S->nm));
        C *f1 = reinterpret_cast<C *>(D);
        const R inv_n3 = (R)(1.0 / ((double)N * N * N));
        SV_CUDA(S, tmark(S, 1, PK_SURVEY_STAGE_FIELD));
        k_survey_interlace<R, C><<<rowblocks, kRowThreads, 0, st>>>(f1, f1 + mr / 2, A0,
                                                                    reinterpret_cast<const C *>(P->d_ph), N, Nh,
                                                                    inv_n3);
        SV_CUDA(S, cudaGetLastError());
        S->launches += 2;
        if (nslot > 0) {
            SV_CUDA(S, tmark(S, 1, PK_SURVEY_STAGE_FFT));
            if (S->f64) {
                SV_CUFFT(S, cufftExecZ2D(S->fft_inv, reinterpret_cast<cufftDoubleComplex *>(D),
                                         reinterpret_cast<cufftDoubleReal *>(D)));
            } else {
                SV_CUFFT(S, cufftExecC2R(S->fft_inv, reinterpret_cast<cufftComplex *>(D),
                                         reinterpret_cast<cufftReal *>(D)));
            }
        }
    }

    const pk::BinGeom &g = P->bg;
    const size_t smem = ((3 * (size_t)g.nk * sizeof(R) + 15) / 16) * 16 + (size_t)g.nk * sizeof(int2);
    if (smem > 200 * 1024) return sfail(S, PK_EINVAL, "too many k bins for the per-CTA histogram");
    {
        void (*bins[4])(const C *, const C *, long long, int, int, int, pk::BinGeom, const R *, const int *,
                        double *) = {k_survey_bin<R, C, 0, 0>, k_survey_bin<R, C, 0, 14>, k_survey_bin<R, C, 0, 5>,
                                     k_survey_bin<R, C, 5, 9>};
        for (auto f : bins)
            SV_CUDA(S, cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    }
    const int nbatches = nslot > 0 ? (nslot + S->batch - 1) / S->batch : 1;
    for (int bi = 0; bi < nbatches; ++bi) {
        const int s0 = S->sa + bi * S->batch;
        const int nb = nslot > 0 ? std::min(S->batch, S->sb - s0) : 0;
        const bool first = bi == 0;
        R *a0copy = (!il && first) ? A0r : nullptr;
        // compile-time slot ranges for the usual batches, else the generic kernel
        const int spec = (s0 == 0 && nb == 14) ? 1 : (s0 == 0 && nb == 5) ? 2 : (s0 == 5 && nb == 9) ? 3 : 0;
        if (nb > 0 || a0copy) {
            SV_CUDA(S, tmark(S, 1, PK_SURVEY_STAGE_FIELD));
            const R *Rsrc = il ? nullptr : Rm;
            R *a0dst = il ? nullptr : a0copy;
#define SV_YLM(FKP, S0_, NB_)                                                                                   \
    k_survey_ylm<R, FKP, S0_, NB_><<<rowblocks, kRowThreads, 0, st>>>(D, Rsrc, S->cst, a0dst, SL, mr, s0, nb, N, \
                                                                      2 * Nh, ox, oy, oz, H)
            if (il) {
                if (spec == 1) SV_YLM(false, 0, 14);
                else if (spec == 2) SV_YLM(false, 0, 5);
                else if (spec == 3) SV_YLM(false, 5, 9);
                else SV_YLM(false, 0, 0);
            } else {
                if (spec == 1) SV_YLM(true, 0, 14);
                else if (spec == 2) SV_YLM(true, 0, 5);
                else if (spec == 3) SV_YLM(true, 5, 9);
                else SV_YLM(true, 0, 0);
            }
#undef SV_YLM
            SV_CUDA(S, cudaGetLastError());
            S->launches += 1;
        }
        SV_CUDA(S, tmark(S, 1, PK_SURVEY_STAGE_FFT));
        if (a0copy) SV_CUFFT(S, pk::transform_meshes(P, A0r, 1));
        for (int k = 0; k < nb; ++k) {
            R *mk = SL + (long long)k * mr;
            if (S->f64) {
                SV_CUFFT(S, cufftExecD2Z(S->fft_b, reinterpret_cast<cufftDoubleReal *>(mk),
                                         reinterpret_cast<cufftDoubleComplex *>(mk)));
            } else {
                SV_CUFFT(S, cufftExecR2C(S->fft_b, reinterpret_cast<cufftReal *>(mk), reinterpret_cast<cufftComplex *>(mk)));
            }
        }
        SV_CUDA(S, tmark(S, 1, PK_SURVEY_STAGE_BIN));
#define SV_BIN(S0_, NB_)                                                                                        \
    k_survey_bin<R, C, S0_, NB_><<<S->Gb, kRowThreads, smem, st>>>(A0, reinterpret_cast<const C *>(SL), mr / 2, s0, \
                                                                   nb, first ? 1 : 0, g,                            \
                                                                   reinterpret_cast<const R *>(P->d_cw), P->d_kedge, \
                                                                   S->partial)
        if (spec == 1) SV_BIN(0, 14);
        else if (spec == 2) SV_BIN(0, 5);
        else if (spec == 3) SV_BIN(5, 9);
        else SV_BIN(0, 0);
#undef SV_BIN
        SV_CUDA(S, cudaGetLastError());
        S->launches += 1;
    }
    const int nk = g.nk;
    SV_CUDA(S, tmark(S, 1, PK_SURVEY_STAGE_FINAL));
    k_survey_final<<<(3 * nk + 127) / 128, 128, 0, st>>>(S->partial, S->Gb, nk, P->d_modes1d, S->cst,
                                                         S->cfg.poles_mask | 1u, S->cfg.subtract_shot, S->res);
    SV_CUDA(S, cudaGetLastError());
    S->launches += 1;
    SV_CUDA(S, tmark(S, 1, -1));
    SV_CUDA(S, cudaMemcpyAsync(S->h_res, S->res, sizeof(double) * (3 * (size_t)nk + kConst), cudaMemcpyDeviceToHost,
                               st));
    SV_CUDA(S, cudaEventRecord(S->done, st));
    return PK_OK;
}

extern "C" {

pk_status pk_survey_compute(pk_survey_t S) {
    if (!S) return PK_EINVAL;
    S->err.clear();
    if (!S->painted) return sfail(S, PK_ESTATE, "nothing painted since the last compute");
    pk_status s = S->f64 ? survey_compute_t<double, double2>(S) : survey_compute_t<float, float2>(S);
    if (s != PK_OK) return s;
    S->painted = 0;
    S->computed = 1;
    return PK_OK;
}

pk_status pk_survey_result(pk_survey_t S, pk_survey_result_view *out) {
    if (!S) return PK_EINVAL;
    S->err.clear();
    if (!out) return sfail(S, PK_EINVAL, "out is NULL");
    if (!S->computed) return sfail(S, PK_ESTATE, "no compute yet");
    SV_CUDA(S, cudaEventSynchronize(S->done));
    pk_plan_s *P = S->P;
    const int nk = P->bg.nk;
    const double *c = S->h_res + 3 * (size_t)nk;
    memset(out, 0, sizeof(*out));
    out->nk = nk;
    out->npoles = 3;
    out->k_edges = P->k_edges.data();
    out->k_mean = P->kmean1d.data();
    out->modes = P->modes1d.data();
    out->poles = S->h_res;
    out->alpha = c[0];
    out->norm = c[1];
    out->shot_noise = c[2];
    out->data_wsum = c[3];
    out->randoms_wsum = c[4];
    out->data_w2sum = c[5];
    out->randoms_w2sum = c[6];
    out->randoms_nsum = c[7];
    out->n_data = S->nd;
    out->n_randoms = S->nr;
    out->n_outside = (int64_t)llround(c[9] + c[10]);
    out->n_rejected = (int64_t)llround(c[11] + c[12]);
    return PK_OK;
}

pk_status pk_survey_bounds(const pk_survey_catalog *cat, double omega_m, double zmax, void *cuda_stream,
                           double *lo, double *hi) {
    if (!cat || !lo || !hi) return sfail(nullptr, PK_EINVAL, "cat, lo and hi must not be NULL");
    if (cat->dtype != PK_F32 && cat->dtype != PK_F64)
        return sfail(nullptr, PK_EINVAL, "catalog dtype must be PK_F32 or PK_F64");
    if (cat->coord != PK_COORD_CARTESIAN && cat->coord != PK_COORD_SKY)
        return sfail(nullptr, PK_EINVAL, "catalog coord must be PK_COORD_CARTESIAN or PK_COORD_SKY");
    const bool sky = cat->coord == PK_COORD_SKY;
    if (sky && !(omega_m > 0.0 && omega_m <= 1.0))
        return sfail(nullptr, PK_EINVAL, "sky input needs omega_m in (0, 1]");
    if (!(zmax >= 0.0 && zmax <= 1100.0)) return sfail(nullptr, PK_EINVAL, "zmax must be in [0, 1100]");
    if (cat->n < 0 || (cat->n > 0 && !cat->pos)) return sfail(nullptr, PK_EINVAL, "catalog pos / n invalid");
    for (int k = 0; k < 3; ++k) {
        lo[k] = INFINITY;
        hi[k] = -INFINITY;
    }
    if (cat->n == 0) return PK_OK;
    const cudaStream_t st = reinterpret_cast<cudaStream_t>(cuda_stream);
    const size_t pbytes = (size_t)cat->n * (cat->dtype == PK_F64 ? 24 : 12);
    int dev = 0, nsm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        cudaGetLastError();
        return sfail(nullptr, PK_ECUDA, "no CUDA device");
    }
    const int G = nsm * kPrepCtasPerSm;
    std::vector<double> tab;
    PrepArgs a{};
    a.nchi = kChiNodes;
    a.zmax = zmax > 0.0 ? zmax : 5.0;
    if (sky) chi_table(omega_m, a.zmax, tab, &a.dz);
    a.inv_dz = a.dz > 0.0 ? 1.0 / a.dz : 0.0;
    const bool pdev = dev_ptr(cat->pos);
    // one device block: 6 results | G x 6 per-CTA partials | chi table | positions (host input)
    const size_t off_part = 64, off_tab = off_part + 48 * (size_t)G;
    const size_t off_pos = (off_tab + 8 * tab.size() + 255) / 256 * 256;
    char *buf = nullptr;
    if (cudaMalloc(reinterpret_cast<void **>(&buf), off_pos + (pdev ? 0 : pbytes)) != cudaSuccess) {
        cudaGetLastError();
        return sfail(nullptr, PK_ENOMEM, "device allocation failed");
    }
    double *res = reinterpret_cast<double *>(buf);
    double *part = reinterpret_cast<double *>(buf + off_part);
    a.chi = sky ? reinterpret_cast<const double2 *>(buf + off_tab) : nullptr;
    const void *pos = pdev ? cat->pos : buf + off_pos;
    cudaError_t e = cudaSuccess;
    if (sky) e = cudaMemcpyAsync(buf + off_tab, tab.data(), 8 * tab.size(), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess && !pdev) e = cudaMemcpyAsync(buf + off_pos, cat->pos, pbytes, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) {
        const long long n = cat->n;
        if (cat->dtype == PK_F64) {
            const double *pp = reinterpret_cast<const double *>(pos);
            if (sky) k_survey_bounds<double, true><<<G, kPrepThreads, 0, st>>>(pp, n, a, part);
            else k_survey_bounds<double, false><<<G, kPrepThreads, 0, st>>>(pp, n, a, part);
        } else {
            const float *pp = reinterpret_cast<const float *>(pos);
            if (sky) k_survey_bounds<float, true><<<G, kPrepThreads, 0, st>>>(pp, n, a, part);
            else k_survey_bounds<float, false><<<G, kPrepThreads, 0, st>>>(pp, n, a, part);
        }
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) {
        k_survey_bounds_final<<<1, 32, 0, st>>>(part, G, res);
        e = cudaGetLastError();
    }
    double out[6];
    if (e == cudaSuccess) e = cudaMemcpyAsync(out, res, sizeof(out), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    cudaFree(buf);
    if (e != cudaSuccess) return sfail(nullptr, PK_ECUDA, std::string("survey bounds: ") + cudaGetErrorString(e));
    for (int k = 0; k < 3; ++k) {
        lo[k] = out[k];
        hi[k] = out[3 + k];
    }
    return PK_OK;
}

pk_status pk_survey_enable_timing(pk_survey_t S, int on) {
    if (!S) return PK_EINVAL;
    S->err.clear();
    S->timing = on ? 1 : 0;
    S->seg_paint.clear();
    S->seg_compute.clear();
    return PK_OK;
}

pk_status pk_survey_stage_times(pk_survey_t S, double *ms) {
    if (!S) return PK_EINVAL;
    S->err.clear();
    if (!ms) return sfail(S, PK_EINVAL, "ms is NULL");
    if (!S->timing) return sfail(S, PK_ESTATE, "timing is off");
    for (int k = 0; k < PK_SURVEY_NSTAGES; ++k) ms[k] = 0.0;
    for (int list = 0; list < 2; ++list) {
        const std::vector<int> &seg = list == 0 ? S->seg_paint : S->seg_compute;
        const int base = list == 0 ? 0 : 16;
        if (seg.empty()) continue;
        SV_CUDA(S, cudaEventSynchronize(S->ev[base + (int)seg.size() - 1]));
        for (size_t i = 0; i + 1 < seg.size(); ++i) {
            if (seg[i] < 0) continue;
            float t = 0.0f;
            SV_CUDA(S, cudaEventElapsedTime(&t, S->ev[base + i], S->ev[base + i + 1]));
            ms[seg[i]] += t;
        }
    }
    return PK_OK;
}

long long pk_survey_launch_count(pk_survey_t S) { return S ? S->launches : 0; }

const char *pk_survey_error(pk_survey_t S) { return S ? S->err.c_str() : ""; }

pk_status pk_survey_destroy(pk_survey_t S) {
    free_survey(S);
    return PK_OK;
}

}  // extern "C"
