// pk_lognormal.cu -- log-normal mock catalogs generated on the device: the
// LogNormalCatalog source that the paper's tests and benchmarks paint
// (Sec. 3.2), over its Gaussian linear field.
//
// One draw (seed, n):
//   k_ln_noise    ng^3 unit Gaussians: Philox4x64-10 (Salmon et al., SC'11)
//                 with key (seed, 0); cells 4b .. 4b+3 (flat index, z fastest)
//                 take the words of counter (b, 0, 0, 0), two Box-Muller pairs.
//   cuFFT R2C
//   k_ln_shape    G~ = W~ sqrt(A k^slope ng^3 / L^3) / ng^3 (the 1 / ng^3 of the
//                 inverse transform folded in), DC = 0; psi_z~ = i k_z / k^2 G~
//                 with DC and the z-Nyquist plane set to zero.
//   cuFFT C2R     G and psi_z on the grid.
//   k_ln_moments  sum G, sum G^2 (FP64) -> sigma^2.
//   k_ln_weights  q = round(2^30 exp(G - sigma^2 / 2)) as uint64 cell weights.
//   scan          exact exclusive prefix sums of q (uint64).
//   k_ln_place    object i (key (seed, 1), counter (i, 0, 0, 0)): cell by inverse
//                 CDF of t = floor(w0 total / 2^64), uniform offset in the cell
//                 from w1..w3, z + f_rsd psi_z(cell), wrapped into [0, L).
// The counters depend only on the cell or object index, so a catalog is the
// same for any launch configuration.
#include <cuda_runtime.h>
#include <cufft.h>

#include <math.h>
#include <string.h>

#include <string>
#include <vector>

#include "pk_internal.h"

namespace pk {
namespace {

constexpr int kLnThreads = 256;
constexpr int kCoarse = 1024;         // cells per block of the coarse CDF index

struct Philox4x64 {
    unsigned long long w[4];
};

__device__ __forceinline__ Philox4x64 philox4x64(unsigned long long c0, unsigned long long key0,
                                                 unsigned long long key1) {
    unsigned long long x0 = c0, x1 = 0ull, x2 = 0ull, x3 = 0ull;
    unsigned long long k0 = key0, k1 = key1;
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const unsigned long long hi0 = __umul64hi(0xD2E7470EE14C6C93ull, x0), lo0 = 0xD2E7470EE14C6C93ull * x0;
        const unsigned long long hi1 = __umul64hi(0xCA5A826395121157ull, x2), lo1 = 0xCA5A826395121157ull * x2;
        x0 = hi1 ^ x1 ^ k0;
        x1 = lo1;
        x2 = hi0 ^ x3 ^ k1;
        x3 = lo0;
        k0 += 0x9E3779B97F4A7C15ull;
        k1 += 0xBB67AE8584CAA73Bull;
    }
    Philox4x64 o;
    o.w[0] = x0;
    o.w[1] = x1;
    o.w[2] = x2;
    o.w[3] = x3;
    return o;
}

// (row, col) of a flat index in rows of width w, advanced by a fixed stride
// with one division at the start instead of one per step.
struct Walk {
    long long row, drow;
    int col, dcol, w;
    __device__ __forceinline__ Walk(long long f, long long stride, int width) : w(width) {
        row = f / w;
        col = (int)(f - row * w);
        drow = stride / w;
        dcol = (int)(stride - drow * w);
    }
    __device__ __forceinline__ void step() {
        row += drow;
        col += dcol;
        if (col >= w) {
            col -= w;
            ++row;
        }
    }
};

// ((x >> 40) + 1/2) 2^-24: exact in FP32, strictly inside (0, 1).
__device__ __forceinline__ float uniform24(unsigned long long x) {
    return ((float)(unsigned)(x >> 40) + 0.5f) * 5.9604644775390625e-8f;
}

__global__ void __launch_bounds__(kLnThreads)
k_ln_noise(float *__restrict__ g, int ng, long long pitch, unsigned long long seed) {
    const long long ncell = (long long)ng * ng * ng;
    const long long b0 = (long long)blockIdx.x * blockDim.x + threadIdx.x, stride = (long long)gridDim.x * blockDim.x;
    Walk w(4 * b0, 4 * stride, ng);                   // cell 4b
    for (long long b = b0; 4 * b < ncell; b += stride, w.step()) {
        const Philox4x64 r = philox4x64((unsigned long long)b, seed, 0ull);
#pragma unroll
        for (int pair = 0; pair < 2; ++pair) {
            const float u1 = uniform24(r.w[2 * pair]), u2 = uniform24(r.w[2 * pair + 1]);
            const float rad = sqrtf(-2.0f * logf(u1));
            float sn, cs;
            sincospif(2.0f * u2, &sn, &cs);
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                int l = w.col + 2 * pair + h;              // the 4 cells may cross into the next row
                long long row = w.row;
                if (l >= ng) {
                    l -= ng;
                    ++row;
                }
                g[row * pitch + l] = h ? rad * sn : rad * cs;
            }
        }
    }
}

__global__ void __launch_bounds__(kLnThreads)
k_ln_shape(float2 *__restrict__ gk, float2 *__restrict__ psik, int ng, float kf2, float amp_scale,
           float quarter_slope, float inv_n3, float kf) {
    const int nh = ng / 2 + 1;
    const long long nmodes = (long long)ng * ng * nh;
    const long long f0 = (long long)blockIdx.x * blockDim.x + threadIdx.x, stride = (long long)gridDim.x * blockDim.x;
    Walk w(f0, stride, nh);
    for (long long f = f0; f < nmodes; f += stride, w.step()) {
        const int l = w.col;
        const int irow = (int)w.row;                    // < ng^2 <= 2^22
        const int i = irow / ng, j = irow - i * ng;
        const int ip = i < ng / 2 ? i : i - ng, jp = j < ng / 2 ? j : j - ng;
        const float m = (float)(ip * ip + jp * jp + l * l);
        float2 v = gk[f];
        if (m == 0.0f) {
            gk[f] = make_float2(0.0f, 0.0f);
            if (psik) psik[f] = make_float2(0.0f, 0.0f);
            continue;
        }
        // sqrt(A (kF^2 m)^(slope/2) ng^3 / L^3) / ng^3
        const float fac = sqrtf(amp_scale) * powf(kf2 * m, quarter_slope) * inv_n3;
        v.x *= fac;
        v.y *= fac;
        gk[f] = v;
        if (psik) {
            if (l == ng / 2) {
                psik[f] = make_float2(0.0f, 0.0f);
            } else {
                const float a = (kf * (float)l) / (kf2 * m);        // k_z / k^2
                psik[f] = make_float2(-a * v.y, a * v.x);           // i k_z / k^2 G~
            }
        }
    }
}

__global__ void __launch_bounds__(kLnThreads)
k_ln_moments(const float *__restrict__ g, int ng, long long pitch, double *__restrict__ stats) {
    const long long ncell = (long long)ng * ng * ng;
    double s1 = 0.0, s2 = 0.0;
    const long long c0 = (long long)blockIdx.x * blockDim.x + threadIdx.x, stride = (long long)gridDim.x * blockDim.x;
    Walk w(c0, stride, ng);
    for (long long c = c0; c < ncell; c += stride, w.step()) {
        const double v = (double)g[w.row * pitch + w.col];
        s1 += v;
        s2 += v * v;
    }
    __shared__ double r1[kLnThreads / 32], r2[kLnThreads / 32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        s1 += __shfl_down_sync(0xffffffffu, s1, o);
        s2 += __shfl_down_sync(0xffffffffu, s2, o);
    }
    if ((threadIdx.x & 31) == 0) {
        r1[threadIdx.x >> 5] = s1;
        r2[threadIdx.x >> 5] = s2;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0.0, b = 0.0;
        for (int k = 0; k < kLnThreads / 32; ++k) {
            a += r1[k];
            b += r2[k];
        }
        atomicAdd(stats + 0, a);
        atomicAdd(stats + 1, b);
    }
}

__global__ void __launch_bounds__(kLnThreads)
k_ln_weights(const float *__restrict__ g, int ng, long long pitch, const double *__restrict__ stats,
             unsigned long long *__restrict__ q) {
    const long long ncell = (long long)ng * ng * ng;
    const double mean = stats[0] / (double)ncell;
    const float half_var = (float)(0.5 * (stats[1] / (double)ncell - mean * mean));
    const long long c0 = (long long)blockIdx.x * blockDim.x + threadIdx.x, stride = (long long)gridDim.x * blockDim.x;
    Walk w(c0, stride, ng);
    for (long long c = c0; c < ncell; c += stride, w.step()) {
        const float x = g[w.row * pitch + w.col] - half_var;
        q[c] = (unsigned long long)__float2ll_rn(expf(x) * 1073741824.0f);
    }
}

// coarse[k] = excl[min(k kCoarse, ncell)], k = 0 .. nblk: a small index that
// stays in cache, so each object's search touches one 8 KB block of excl.
__global__ void k_ln_coarse(const unsigned long long *__restrict__ excl, long long ncell, long long nblk,
                            unsigned long long *__restrict__ coarse) {
    for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k <= nblk;
         k += (long long)gridDim.x * blockDim.x) {
        const long long c = k * kCoarse;
        coarse[k] = excl[c < ncell ? c : ncell];
    }
}

__global__ void __launch_bounds__(kLnThreads)
k_ln_place(const unsigned long long *__restrict__ excl, const unsigned long long *__restrict__ coarse,
           long long nblk, int ng, double L, const float *__restrict__ psi, long long pitch, float f_rsd,
           unsigned long long seed, long long n, float *__restrict__ pos) {
    const long long ncell = (long long)ng * ng * ng;
    const unsigned long long total = excl[ncell];
    const double H = L / ng;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const Philox4x64 r = philox4x64((unsigned long long)i, seed, 1ull);
        const unsigned long long t = __umul64hi(r.w[0], total);
        long long ka = 0, kb = nblk;                      // coarse[ka] <= t < coarse[kb]
        while (kb - ka > 1) {
            const long long mid = ka + ((kb - ka) >> 1);
            if (coarse[mid] <= t) ka = mid;
            else kb = mid;
        }
        long long a = ka * kCoarse, b = kb * kCoarse < ncell ? kb * kCoarse : ncell;   // excl[a] <= t < excl[b]
        while (b - a > 1) {
            const long long mid = a + ((b - a) >> 1);
            if (excl[mid] <= t) a = mid;
            else b = mid;
        }
        const long long c = a;
        const long long ix = c / ((long long)ng * ng), iy = (c / ng) % ng, iz = c % ng;
        double z = ((double)iz + (double)uniform24(r.w[3])) * H;
        if (psi) z += (double)f_rsd * (double)psi[(c / ng) * pitch + iz];
        z = z - L * floor(z / L);
        if (z >= L) z -= L;
        // FP32 rounding can reach L exactly: that point is 0 on the periodic box
        float xf = (float)(((double)ix + (double)uniform24(r.w[1])) * H);
        float yf = (float)(((double)iy + (double)uniform24(r.w[2])) * H);
        float zf = (float)z;
        const float Lf = (float)L;
        pos[3 * i + 0] = xf >= Lf ? 0.0f : xf;
        pos[3 * i + 1] = yf >= Lf ? 0.0f : yf;
        pos[3 * i + 2] = zf >= Lf ? 0.0f : zf;
    }
}

unsigned grid_of(long long n, int nsm) {
    long long b = (n + kLnThreads - 1) / kLnThreads;
    const long long cap = (long long)(nsm > 0 ? nsm : 132) * 16;
    if (b > cap) b = cap;
    return (unsigned)(b < 1 ? 1 : b);
}

}  // namespace
}  // namespace pk

using namespace pk;

struct pk_lognormal_s {
    pk_lognormal_config cfg;
    cudaStream_t st = nullptr;
    int ng = 0, nsm = 0;
    long long pitch = 0;             // reals per grid row (2 (ng/2 + 1))
    double amp = 0.0;
    float *g = nullptr;              // G (in-place r2c / c2r layout)
    float *psi = nullptr;            // psi_z (same layout), if f_rsd != 0
    unsigned long long *q = nullptr;     // cell weights
    unsigned long long *excl = nullptr;  // exclusive prefix sums, excl[ncell] = total
    unsigned long long *coarse = nullptr;  // excl at every kCoarse-th cell (and at ncell)
    long long nblk = 0;
    unsigned long long *scan_tmp = nullptr;
    double *stats = nullptr;
    cufftHandle fwd = 0, inv = 0;
    bool fwd_made = false, inv_made = false;
    long long launches = 0;
    std::string err;
};

namespace {

pk_status ln_fail(pk_lognormal_s *G, pk_status s, const std::string &msg) {
    if (G) G->err = msg;
    else pk::set_plan_error(msg.c_str());
    return s;
}

#define LN_CUDA(gen, call)                                                                    \
    do {                                                                                      \
        cudaError_t e_ = (call);                                                              \
        if (e_ != cudaSuccess)                                                                \
            return ln_fail(gen, e_ == cudaErrorMemoryAllocation ? PK_ENOMEM : PK_ECUDA,       \
                           std::string(#call) + ": " + cudaGetErrorString(e_));              \
    } while (0)

#define LN_CUFFT(gen, call)                                                                   \
    do {                                                                                      \
        cufftResult r_ = (call);                                                              \
        if (r_ != CUFFT_SUCCESS)                                                              \
            return ln_fail(gen, r_ == CUFFT_ALLOC_FAILED ? PK_ENOMEM : PK_ECUFFT,             \
                           std::string(#call) + ": cufftResult " + std::to_string((int)r_)); \
    } while (0)

void ln_free(pk_lognormal_s *G) {
    if (!G) return;
    if (G->st || G->g) cudaStreamSynchronize(G->st);
    if (G->fwd_made) cufftDestroy(G->fwd);
    if (G->inv_made) cufftDestroy(G->inv);
    void *dev[] = {G->g, G->psi, G->q, G->excl, G->coarse, G->scan_tmp, G->stats};
    for (void *d : dev)
        if (d) cudaFree(d);
    delete G;
}

// A with (1 / L^3) sum_{k != 0} A k^slope = variance over the full ng^3 grid:
// counts of each m = i'^2 + j'^2 + l'^2 (exact integers; |i'| = a occurs once
// for a = 0 and a = ng/2, twice otherwise), then one power per m.
double ln_amplitude(int ng, double L, double slope, double variance) {
    const int h = ng / 2;
    const long long mmax = 3LL * h * h;
    std::vector<long long> cnt(mmax + 1, 0);
    auto mult = [h](int a) { return (a == 0 || a == h) ? 1LL : 2LL; };
    for (int a = 0; a <= h; ++a)
        for (int b = 0; b <= h; ++b) {
            const long long mab = mult(a) * mult(b), sab = (long long)a * a + (long long)b * b;
            for (int c = 0; c <= h; ++c) cnt[sab + (long long)c * c] += mab * mult(c);
        }
    const double kf = 2.0 * M_PI / L;
    double total = 0.0;
    for (long long m = 1; m <= mmax; ++m)
        if (cnt[m]) total += (double)cnt[m] * pow(kf * kf * (double)m, 0.5 * slope);
    return variance * L * L * L / total;
}

}  // namespace

extern "C" {

pk_status pk_lognormal_plan(const pk_lognormal_config *cfg, void *cuda_stream, pk_lognormal_t *out) {
    pk::set_plan_error("");
    if (!out) return ln_fail(nullptr, PK_EINVAL, "out is NULL");
    *out = nullptr;
    if (!cfg) return ln_fail(nullptr, PK_EINVAL, "cfg is NULL");
    const pk_lognormal_config &c = *cfg;
    if (!(c.box_size > 0.0) || !isfinite(c.box_size)) return ln_fail(nullptr, PK_EINVAL, "box_size must be > 0");
    if (c.ngrid < 4 || c.ngrid > 2048 || (c.ngrid % 2) != 0)
        return ln_fail(nullptr, PK_EINVAL, "ngrid must be even and in [4, 2048]");
    if (!isfinite(c.slope)) return ln_fail(nullptr, PK_EINVAL, "slope must be finite");
    if (!(c.amp > 0.0) && !(c.variance > 0.0))
        return ln_fail(nullptr, PK_EINVAL, "variance must be > 0 when amp <= 0");
    if (!isfinite(c.f_rsd)) return ln_fail(nullptr, PK_EINVAL, "f_rsd must be finite");
    pk_lognormal_s *G = new (std::nothrow) pk_lognormal_s();
    if (!G) return ln_fail(nullptr, PK_ENOMEM, "host allocation failed");
    G->cfg = c;
    G->st = reinterpret_cast<cudaStream_t>(cuda_stream);
    G->ng = c.ngrid;
    G->pitch = 2LL * (c.ngrid / 2 + 1);
    G->amp = c.amp > 0.0 ? c.amp : ln_amplitude(c.ngrid, c.box_size, c.slope, c.variance);
    auto bail = [&](pk_status s) {
        pk::set_plan_error(G->err.c_str());
        ln_free(G);
        return s;
    };
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&G->nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        G->err = "cannot query the CUDA device";
        return bail(PK_ECUDA);
    }
    const long long ng = c.ngrid, ncell = ng * ng * ng;
    const size_t grid_bytes = sizeof(float) * (size_t)(ng * ng * G->pitch);
    cudaError_t e = cudaMalloc(reinterpret_cast<void **>(&G->g), grid_bytes);
    if (e == cudaSuccess && c.f_rsd != 0.0) e = cudaMalloc(reinterpret_cast<void **>(&G->psi), grid_bytes);
    if (e == cudaSuccess) e = cudaMalloc(reinterpret_cast<void **>(&G->q), sizeof(unsigned long long) * ncell);
    if (e == cudaSuccess)
        e = cudaMalloc(reinterpret_cast<void **>(&G->excl), sizeof(unsigned long long) * (ncell + 1));
    if (e == cudaSuccess)
        e = cudaMalloc(reinterpret_cast<void **>(&G->scan_tmp), sizeof(unsigned long long) * scan_tmp_elems(ncell));
    if (e == cudaSuccess) e = cudaMalloc(reinterpret_cast<void **>(&G->stats), 2 * sizeof(double));
    G->nblk = (ncell + kCoarse - 1) / kCoarse;
    if (e == cudaSuccess)
        e = cudaMalloc(reinterpret_cast<void **>(&G->coarse), sizeof(unsigned long long) * (G->nblk + 1));
    if (e != cudaSuccess) {
        G->err = std::string("device allocation: ") + cudaGetErrorString(e);
        return bail(e == cudaErrorMemoryAllocation ? PK_ENOMEM : PK_ECUDA);
    }
    // in-place transforms on the padded layout: real rows of 2 (ng/2 + 1), complex rows of ng/2 + 1
    long long n3[3] = {ng, ng, ng};
    long long real_emb[3] = {ng, ng, G->pitch};
    long long cplx_emb[3] = {ng, ng, G->pitch / 2};
    size_t work = 0;
    if (cufftCreate(&G->fwd) != CUFFT_SUCCESS) {
        G->err = "cufftCreate failed";
        return bail(PK_ECUFFT);
    }
    G->fwd_made = true;
    if (cufftMakePlanMany64(G->fwd, 3, n3, real_emb, 1, ng * ng * G->pitch, cplx_emb, 1, ng * ng * G->pitch / 2,
                            CUFFT_R2C, 1, &work) != CUFFT_SUCCESS) {
        G->err = "cuFFT R2C plan failed";
        return bail(PK_ECUFFT);
    }
    if (cufftCreate(&G->inv) != CUFFT_SUCCESS) {
        G->err = "cufftCreate failed";
        return bail(PK_ECUFFT);
    }
    G->inv_made = true;
    if (cufftMakePlanMany64(G->inv, 3, n3, cplx_emb, 1, ng * ng * G->pitch / 2, real_emb, 1, ng * ng * G->pitch,
                            CUFFT_C2R, 1, &work) != CUFFT_SUCCESS) {
        G->err = "cuFFT C2R plan failed";
        return bail(PK_ECUFFT);
    }
    if (cufftSetStream(G->fwd, G->st) != CUFFT_SUCCESS || cufftSetStream(G->inv, G->st) != CUFFT_SUCCESS) {
        G->err = "cufftSetStream failed";
        return bail(PK_ECUFFT);
    }
    *out = G;
    return PK_OK;
}

// Noise -> G (and psi_z) on the grid; returns the status.
static pk_status ln_field(pk_lognormal_s *G, unsigned long long seed) {
    const int ng = G->ng;
    const long long ncell = (long long)ng * ng * ng;
    const long long nmodes = (long long)ng * ng * (ng / 2 + 1);
    const double L = G->cfg.box_size;
    k_ln_noise<<<grid_of(ncell / 4, G->nsm), kLnThreads, 0, G->st>>>(G->g, ng, G->pitch, seed);
    LN_CUDA(G, cudaGetLastError());
    LN_CUFFT(G, cufftExecR2C(G->fwd, G->g, reinterpret_cast<cufftComplex *>(G->g)));
    const double kf = 2.0 * M_PI / L;
    k_ln_shape<<<grid_of(nmodes, G->nsm), kLnThreads, 0, G->st>>>(
        reinterpret_cast<float2 *>(G->g), reinterpret_cast<float2 *>(G->psi), ng, (float)(kf * kf),
        (float)(G->amp * (double)ncell / (L * L * L)), (float)(0.25 * G->cfg.slope), (float)(1.0 / (double)ncell),
        (float)kf);
    LN_CUDA(G, cudaGetLastError());
    LN_CUFFT(G, cufftExecC2R(G->inv, reinterpret_cast<cufftComplex *>(G->g), G->g));
    if (G->psi)
        LN_CUFFT(G, cufftExecC2R(G->inv, reinterpret_cast<cufftComplex *>(G->psi), G->psi));
    G->launches += 2;
    return PK_OK;
}

pk_status pk_lognormal_field(pk_lognormal_t G, uint64_t seed, float *field) {
    if (!G) return PK_EINVAL;
    G->err.clear();
    if (!field) return ln_fail(G, PK_EINVAL, "field is NULL");
    pk_status s = ln_field(G, seed);
    if (s != PK_OK) return s;
    const size_t row = sizeof(float) * G->ng;
    LN_CUDA(G, cudaMemcpy2DAsync(field, row, G->g, sizeof(float) * G->pitch, row, (size_t)G->ng * G->ng,
                                 cudaMemcpyDefault, G->st));
    return PK_OK;
}

pk_status pk_lognormal_draw(pk_lognormal_t G, uint64_t seed, int64_t n, float *pos) {
    if (!G) return PK_EINVAL;
    G->err.clear();
    if (n < 0) return ln_fail(G, PK_EINVAL, "n must be >= 0");
    if (n > 0 && !pos) return ln_fail(G, PK_EINVAL, "pos is NULL");
    pk_status s = ln_field(G, seed);
    if (s != PK_OK) return s;
    const int ng = G->ng;
    const long long ncell = (long long)ng * ng * ng;
    LN_CUDA(G, cudaMemsetAsync(G->stats, 0, 2 * sizeof(double), G->st));
    k_ln_moments<<<grid_of(ncell, G->nsm), kLnThreads, 0, G->st>>>(G->g, ng, G->pitch, G->stats);
    LN_CUDA(G, cudaGetLastError());
    k_ln_weights<<<grid_of(ncell, G->nsm), kLnThreads, 0, G->st>>>(G->g, ng, G->pitch, G->stats, G->q);
    LN_CUDA(G, cudaGetLastError());
    int launches = 0;
    LN_CUDA(G, launch_scan64(G->q, ncell, G->excl, G->scan_tmp, &launches, G->st));
    k_ln_coarse<<<grid_of(G->nblk + 1, G->nsm), kLnThreads, 0, G->st>>>(G->excl, ncell, G->nblk, G->coarse);
    LN_CUDA(G, cudaGetLastError());
    if (n > 0) {
        k_ln_place<<<grid_of(n, G->nsm), kLnThreads, 0, G->st>>>(G->excl, G->coarse, G->nblk, ng, G->cfg.box_size,
                                                                  G->psi, G->pitch, (float)G->cfg.f_rsd, seed,
                                                                  (long long)n, pos);
        LN_CUDA(G, cudaGetLastError());
    }
    G->launches += 4 + launches + (n > 0);
    return PK_OK;
}

double pk_lognormal_amp(pk_lognormal_t G) { return G ? G->amp : 0.0; }

long long pk_lognormal_launch_count(pk_lognormal_t G) { return G ? G->launches : 0; }

const char *pk_lognormal_error(pk_lognormal_t G) { return G ? G->err.c_str() : ""; }

pk_status pk_lognormal_destroy(pk_lognormal_t G) {
    ln_free(G);
    return PK_OK;
}

}  // extern "C"
