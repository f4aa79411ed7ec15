// pk_static.cu -- pk_bin_static: the binning pass with no device allocation.
//
// Some callers cannot call cudaMalloc: code that runs while a stream is being
// captured into a CUDA graph by a framework that owns all memory, programs
// whose device memory is carved up by a custom pool allocator they do not
// control, or embedded hosts that forbid allocation after start-up.  For them
// this file offers one entry point that bins caller-provided transforms using
// a fixed scratch array compiled into the library instead of allocating.
//
// The scratch array is a file-scope static __device__ array, so every GPU
// that loads the library holds kScratchBytes of it until the process exits.
// In host code its name is only a host-side stand-in: the device address is
// obtained once per device with cudaGetSymbolAddress (with that device
// current) and passed to the kernels.  All calls share the array: calls that
// overlap on the GPU (different streams, or different host threads) race.
#include <cuda_runtime.h>
#include <math.h>
#include <string.h>

#include <mutex>

#include "pk_internal.h"

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

namespace {

constexpr int kMaxCtas = 160;             // per-CTA histograms kept in the scratch
constexpr int kMaxBins = 8192;            // histogram length nh (all sums)
constexpr int kMaxMesh = 4096;            // N
constexpr size_t kPartialBytes = (size_t)kMaxCtas * kMaxBins * sizeof(float);
constexpr size_t kCwOff = kPartialBytes;                                  // float[kMaxMesh]
constexpr size_t kPhOff = kCwOff + (size_t)kMaxMesh * sizeof(float);      // float2[kMaxMesh + 1]
constexpr size_t kEdgeOff = kPhOff + (size_t)(kMaxMesh + 2) * sizeof(float2);   // int[kMaxBins + 1]
constexpr size_t kScratchBytes = kEdgeOff + (size_t)(kMaxBins + 8) * sizeof(int);

static __device__ __align__(256) unsigned char g_bin_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
unsigned char *g_scratch_ptr[kMaxDevices] = {};

// Copies msg into the caller's buffer (if any) and returns s.
struct ErrOut {
    char *buf;
    size_t len;
    pk_status operator()(pk_status s, const char *msg) const {
        if (buf && len > 0) {
            strncpy(buf, msg, len - 1);
            buf[len - 1] = '\0';
        }
        return s;
    }
};

// k bin of squared index m, the same FP64 expression as the plan path, with
// every operation explicitly rounded.
__host__ __device__ inline long long static_kbin(long long m, double kF, double kmin, double dk) {
#ifdef __CUDA_ARCH__
    return (long long)floor(__ddiv_rn(__dsub_rn(__dmul_rn(kF, __dsqrt_rn((double)m)), kmin), dk));
#else
    return (long long)floor((kF * sqrt((double)m) - kmin) / dk);
#endif
}

// Smallest m in [0, mcap + 1] with kbin(m) >= b (kbin is monotone in m).
__host__ __device__ inline int static_edge(int b, double kF, double kmin, double dk, int mcap) {
    int lo = 0, hi = mcap + 1;
    if (static_kbin(hi, kF, kmin, dk) < b) return mcap + 1;
    while (lo < hi) {
        const int mid = lo + (hi - lo) / 2;
        if (static_kbin(mid, kF, kmin, dk) >= b) hi = mid;
        else lo = mid + 1;
    }
    return lo;
}

// Compensation, interlace-phase and k-edge tables, written into the scratch.
__global__ void k_static_tables(int N, int p, int compensated, double kF, double kmin, double dk,
                                int nk, int mcap, float *cw, float2 *ph, int *kedge) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < N) {
        const int ip = t < N / 2 ? t : t - N;
        const double x = M_PI * (double)ip / (double)N;
        const double s = x == 0.0 ? 1.0 : sin(x) / x;
        cw[t] = compensated ? (float)(1.0 / pow(s, 2 * p)) : 1.0f;
    }
    if (t <= N) {
        const double a = M_PI * (double)(t - N / 2) / (double)N;
        ph[t] = make_float2((float)cos(a), (float)sin(a));
    }
    if (t <= nk) kedge[t] = static_edge(t, kF, kmin, dk, mcap);
}

// sums[k] = sum over the G per-CTA histograms, in CTA order.
__global__ void k_static_reduce(const float *__restrict__ partial, int G, int nh, double *__restrict__ sums) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nh) return;
    double s = 0.0;
    for (int c = 0; c < G; ++c) s += (double)partial[(size_t)c * nh + k];
    sums[k] = s;
}

}  // namespace

extern "C" pk_status pk_bin_static(const pk_config *cfg, const void *mesh, const void *mesh2,
                                   double *sums, void *cuda_stream, char *err, size_t errlen) {
    const ErrOut static_fail{err, errlen};
    if (err && errlen > 0) err[0] = '\0';
    if (!cfg || !mesh || !sums) return static_fail(PK_EINVAL, "cfg, mesh and sums must not be NULL");
    const pk_config &c = *cfg;
    if (c.precision != PK_MESH_F32) return static_fail(PK_EINVAL, "only PK_MESH_F32 (complex64 transforms)");
    if (!(c.box_size > 0.0) || c.nmesh < 4 || c.nmesh > kMaxMesh || (c.nmesh % 2) != 0)
        return static_fail(PK_EINVAL, "box_size must be > 0 and nmesh even in [4, 4096]");
    if (c.window != PK_CIC && c.window != PK_TSC && c.window != PK_PCS)
        return static_fail(PK_EINVAL, "window must be PK_CIC, PK_TSC or PK_PCS");
    if (!(c.dk > 0.0) || !(c.kmin >= 0.0) || c.nmu < 0 || c.los_axis != 2 || (c.poles_mask & ~7u))
        return static_fail(PK_EINVAL, "need dk > 0, kmin >= 0, nmu >= 0, los_axis 2, poles_mask in 0..7");
    if (c.interlaced && !mesh2) return static_fail(PK_EINVAL, "interlaced needs mesh2");
    if ((reinterpret_cast<uintptr_t>(mesh) % 16) || (mesh2 && (reinterpret_cast<uintptr_t>(mesh2) % 16)))
        return static_fail(PK_EINVAL, "meshes must be 16-byte aligned");
    const int N = c.nmesh, Nh = N / 2 + 1;
    const double L = c.box_size;
    const double kF = (2.0 * M_PI) / L;
    const double kmax = c.kmax > 0.0 ? c.kmax : (M_PI * N) / L;
    const double nkd = floor((kmax - c.kmin) / c.dk);
    if (!(nkd >= 1.0) || nkd > kMaxBins) return static_fail(PK_EINVAL, "k binning gives no bins or more than 8192");
    if (kmax / c.dk >= 1048576.0) return static_fail(PK_EINVAL, "k binning too fine: kmax / dk must be below 2^20");
    const int nk = (int)nkd;
    const int mcap = 3 * (N / 2) * (N / 2) + 1;

    pk::BinGeom bg;
    memset(&bg, 0, sizeof(bg));
    bg.N = N;
    bg.Nh = Nh;
    bg.nk = nk;
    bg.nmu = c.nmu;
    bg.twod = c.nmu > 0;
    bg.poles = (c.poles_mask & 6u) != 0;
    bg.hbase = bg.twod ? nk * c.nmu : nk;
    bg.nh = bg.hbase + (bg.poles ? 2 * nk : 0);
    if (bg.nh > kMaxBins) return static_fail(PK_EINVAL, "more than 8192 histogram slots (nk * nmu + 2 nk)");
    bg.kscale = (float)(kF / c.dk);
    bg.koff = (float)(c.kmin / c.dk);
    bg.mlo = static_edge(0, kF, c.kmin, c.dk, mcap);
    bg.mhi = static_edge(nk, kF, c.kmin, c.dk, mcap);
    bg.mu32 = (double)(c.nmu + 1) * (c.nmu + 1) * (double)(bg.mhi + 1) < 4294967295.0 &&
              (double)c.nmu * c.nmu * (double)(N / 2) * (N / 2) < 4294967295.0;
    if (pk::bin_smem_bytes(bg, 0) > 200 * 1024) return static_fail(PK_EINVAL, "histogram too large for shared memory");

    int dev = 0, nsm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return static_fail(PK_ECUDA, cudaGetErrorString(e));
    if (dev < 0 || dev >= kMaxDevices) return static_fail(PK_EINVAL, "device index above 63");
    unsigned char *scratch = nullptr;
    {
        // Set-up, once per device, with that device current.
        std::lock_guard<std::mutex> lock(g_setup_mutex);
        if (!g_scratch_ptr[dev]) {
            void *p = nullptr;
            e = cudaGetSymbolAddress(&p, g_bin_scratch);
            if (e != cudaSuccess) return static_fail(PK_ECUDA, cudaGetErrorString(e));
            g_scratch_ptr[dev] = reinterpret_cast<unsigned char *>(p);
        }
        scratch = g_scratch_ptr[dev];
    }
    float *partial = reinterpret_cast<float *>(scratch);
    float *cw = reinterpret_cast<float *>(scratch + kCwOff);
    float2 *ph = reinterpret_cast<float2 *>(scratch + kPhOff);
    int *kedge = reinterpret_cast<int *>(scratch + kEdgeOff);
    const cudaStream_t st = reinterpret_cast<cudaStream_t>(cuda_stream);

    k_static_tables<<<(N + 1 + nk + 1 + 255) / 256, 256, 0, st>>>(N, c.window, c.compensated, kF, c.kmin,
                                                                     c.dk, nk, mcap, cw, ph, kedge);
    e = cudaGetLastError();
    if (e != cudaSuccess) return static_fail(PK_ECUDA, cudaGetErrorString(e));
    // As many CTAs as the plan path runs (bin_ctas_per_sm per SM), as far as
    // their per-CTA histograms fit in the scratch (G * nh <= kMaxCtas * kMaxBins).
    const long long fit = (long long)kMaxCtas * kMaxBins / bg.nh;
    long long Gw = (long long)nsm * pk::bin_ctas_per_sm(bg, 0);
    if (Gw > fit) Gw = fit;
    if (Gw < 1) Gw = 1;
    const int G = (int)Gw;
    const long long mesh_stride_c =
        mesh2 ? (long long)((reinterpret_cast<intptr_t>(mesh2) - reinterpret_cast<intptr_t>(mesh)) / 8) : 0;
    e = pk::launch_bin(mesh, 0, c.interlaced ? 1 : 0, 0, mesh_stride_c, 1, G, bg, cw, ph, kedge, partial, st);
    if (e != cudaSuccess) return static_fail(PK_ECUDA, cudaGetErrorString(e));
    k_static_reduce<<<(bg.nh + 255) / 256, 256, 0, st>>>(partial, G, bg.nh, sums);
    e = cudaGetLastError();
    if (e != cudaSuccess) return static_fail(PK_ECUDA, cudaGetErrorString(e));
    return PK_OK;
}
