// pk_api.cu -- host side of the C ABI declared in include/pk.h.
//
// A plan owns everything a power-spectrum evaluation needs on the device: the
// meshes (in-place r2c layout), the cuFFT plan, the compensation / phase
// tables, the exact k-bin edges in m = |n|^2 space, the geometry-only bin data
// (mode counts, mean k and mu), the tile-sort buffers and the result blocks.
// All device work of a plan runs on the stream given to pk_plan.
//
// Build this file with -ffp-contract=off: the k-bin edges are computed here in
// FP64 with the expression floor((kF sqrt(m) - kmin) / dk) and must round
// exactly as written.
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

using namespace pk;


namespace {

thread_local std::string g_plan_error;

pk_status fail(pk_plan_s *p, pk_status s, const std::string &msg) {
    if (p) p->err = msg;
    else g_plan_error = msg;
    return s;
}

#define PK_CUDA(plan, call)                                                                   \
    do {                                                                                      \
        cudaError_t e_ = (call);                                                              \
        if (e_ != cudaSuccess)                                                                \
            return fail(plan, e_ == cudaErrorMemoryAllocation ? PK_ENOMEM : PK_ECUDA,         \
                        std::string(#call) + ": " + cudaGetErrorString(e_));                 \
    } while (0)

#define PK_CUFFT(plan, call)                                                                  \
    do {                                                                                      \
        cufftResult r_ = (call);                                                              \
        if (r_ != CUFFT_SUCCESS)                                                              \
            return fail(plan, r_ == CUFFT_ALLOC_FAILED ? PK_ENOMEM : PK_ECUFFT,               \
                        std::string(#call) + ": cufftResult " + std::to_string((int)r_));    \
    } while (0)

template <typename T>
cudaError_t dev_alloc(T **ptr, size_t bytes) {
    *ptr = nullptr;
    if (bytes == 0) bytes = 16;
    return cudaMalloc(reinterpret_cast<void **>(ptr), bytes);
}

void free_plan(pk_plan_s *p) {
    if (!p) return;
    cudaStreamSynchronize(p->st);
    for (cufftHandle h : p->fft) cufftDestroy(h);
    void *dev[] = {p->mesh, p->d_count, p->d_off, p->d_scan_tmp, p->d_sorted,
                   p->d_stage, p->d_item_off, p->d_wsums, p->d_wpart, p->d_wmax, p->d_cw, p->d_ph,
                   p->d_kedge, p->d_partial, p->d_sums2, p->d_res, p->d_modes1d, p->d_modes2d,
                   p->d_err, p->d_acc, p->fft_work, p->d_xres, p->d_proj, p->d_tw};
    for (void *d : dev)
        if (d) cudaFree(d);
    if (p->h_res) cudaFreeHost(p->h_res);
    if (p->h_xres) cudaFreeHost(p->h_xres);
    if (p->xdone) cudaEventDestroy(p->xdone);
    if (p->done) cudaEventDestroy(p->done);
    for (cudaEvent_t e : p->tev)
        if (e) cudaEventDestroy(e);
    delete p;
}

// k bin of squared index m, exactly as the header states it.
long long kbin_of(long long m, double kF, double kmin, double dk) {
    return (long long)floor((kF * sqrt((double)m) - kmin) / dk);
}

// Reach of the window support (both meshes) relative to floor(s), in cells.
void window_reach(int p, int interlaced, int *lo, int *hi) {
    if (p == 2) {
        *lo = 0;
        *hi = interlaced ? 2 : 1;
    } else if (p == 3) {
        *lo = -1;
        *hi = 2;
    } else {
        *lo = -1;
        *hi = interlaced ? 3 : 2;
    }
}

// Tile edge: a divisor of N with T >= hi - lo (so an object's window reaches at
// most one neighbour per axis) and 2 T^3 uint32 of shared memory.  Prefers the
// largest divisor <= 16, else the smallest in [17, 28].
int choose_tile(int N, int span, int requested) {
    const int tmin = span > 1 ? span : 1;
    auto ok = [&](int T) { return T >= tmin && N % T == 0 && paint_smem_bytes(T, 4) <= 200 * 1024; };
    if (requested > 0) return ok(requested) ? requested : -1;
    int best = -1;
    for (int T = tmin; T <= 16 && T <= N; ++T)
        if (ok(T)) best = T;
    if (best < 8) {
        for (int T = 17; T <= 28 && T <= N; ++T)
            if (ok(T)) return T;
    }
    return best;
}

bool is_device_pointer(const void *ptr) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, ptr) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// True while `st` is being captured into a CUDA graph.
int capturing(cudaStream_t st) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st, &cs) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return cs == cudaStreamCaptureStatusActive;
}

size_t record_bytes(int dtype) {
    return dtype == PK_F32 ? 12 : dtype == PK_F64 ? 24 : 16;
}

double sinc(double x) { return x == 0.0 ? 1.0 : sin(x) / x; }

}  // namespace

void pk::set_plan_error(const char *msg) { g_plan_error = msg ? msg : ""; }

// r2c of `count` consecutive meshes from `first`: one call per mesh on a
// single-mesh plan, else one call of the plan over one catalog's meshes
// (count must then be nm).
cufftResult pk::transform_meshes(pk_plan_s *P, void *first, int count) {
    if (ensure_cufft(P) != PK_OK) return CUFFT_ALLOC_FAILED;
    if (!P->fft_single && count != P->nm) return CUFFT_INVALID_VALUE;
    const int calls = P->fft_single ? count : 1;
    for (int k = 0; k < calls; ++k) {
        cufftResult r;
        if (P->f64) {
            cufftDoubleReal *m = reinterpret_cast<cufftDoubleReal *>(first) + (size_t)k * P->mesh_reals;
            r = cufftExecD2Z(P->fft[0], m, reinterpret_cast<cufftDoubleComplex *>(m));
        } else {
            cufftReal *m = reinterpret_cast<cufftReal *>(first) + (size_t)k * P->mesh_reals;
            r = cufftExecR2C(P->fft[0], m, reinterpret_cast<cufftComplex *>(m));
        }
        if (r != CUFFT_SUCCESS) return r;
    }
    return CUFFT_SUCCESS;
}

// cuFFT plans of a plan's meshes (in-place r2c): over 1, 2, 4, ... catalogs and
// all B, or one single-mesh plan; one shared work area, the plan's stream.
// Made when the plan is built unless the own transform serves it, else on
// first use (pk_use_own_fft(plan, 0), or transform_meshes for the survey
// passes), so a 2048^3 plan on the own transform holds no cuFFT work area.
pk_status pk::ensure_cufft(pk_plan_s *P) {
    if (!P->fft.empty()) return PK_OK;
    if (capturing(P->st)) return fail(P, PK_ESTATE, "cuFFT plans cannot be made under stream capture");
    {
        // Meshes above 512^3 are transformed one per call: at 1024^3 a plan
        // batched over two meshes took 18.4 ms against 10.9 ms for two
        // single-mesh calls (equal at 512^3, where batching helps small meshes).
        P->fft_single = P->N > kSingleFftAbove;
        P->fft_items.clear();
        if (P->fft_single) {
            P->fft_items.push_back(1);
        } else {
            for (int c = 1; c < P->B; c <<= 1) P->fft_items.push_back(c);
            P->fft_items.push_back(P->B);
        }
        long long n[3] = {P->N, P->N, P->N};
        long long inembed[3] = {P->N, P->N, 2LL * P->Nh};
        long long onembed[3] = {P->N, P->N, (long long)P->Nh};
        size_t work_max = 0;
        for (int c : P->fft_items) {
            cufftHandle h;
            PK_CUFFT(P, cufftCreate(&h));
            P->fft.push_back(h);
            PK_CUFFT(P, cufftSetAutoAllocation(h, 0));
            size_t work = 0;
            PK_CUFFT(P, cufftMakePlanMany64(h, 3, n, inembed, 1, P->mesh_reals, onembed, 1, P->mesh_reals / 2,
                                            P->f64 ? CUFFT_D2Z : CUFFT_R2C,
                                            P->fft_single ? 1LL : (long long)c * P->nm, &work));
            work_max = std::max(work_max, work);
        }
        PK_CUDA(P, dev_alloc(&P->fft_work, work_max));
        for (cufftHandle h : P->fft) PK_CUFFT(P, cufftSetWorkArea(h, P->fft_work));
        for (cufftHandle h : P->fft) PK_CUFFT(P, cufftSetStream(h, P->st));
    }
    return PK_OK;
}

extern "C" {

void pk_config_default(pk_config *c) {
    if (!c) return;
    memset(c, 0, sizeof(*c));
    c->box_size = 1000.0;
    c->nmesh = 256;
    c->window = PK_CIC;
    c->interlaced = 0;
    c->compensated = 1;
    c->kmin = 0.0;
    c->kmax = 0.0;
    c->dk = 2.0 * (2.0 * M_PI) / c->box_size;
    c->nmu = 0;
    c->poles_mask = 7u;
    c->los_axis = 2;
    c->precision = PK_MESH_F32;
    c->subtract_shot = 1;
    c->fixed_scale_log2 = 0;
    c->batch = 1;
    c->tile = 0;
}

const char *pk_status_string(pk_status s) {
    switch (s) {
    case PK_OK: return "PK_OK";
    case PK_EINVAL: return "PK_EINVAL: invalid argument";
    case PK_ENOMEM: return "PK_ENOMEM: out of memory";
    case PK_ECUDA: return "PK_ECUDA: CUDA runtime error";
    case PK_ECUFFT: return "PK_ECUFFT: cuFFT error";
    case PK_EOVERFLOW: return "PK_EOVERFLOW: fixed-point paint headroom exceeded";
    case PK_ETIMEOUT: return "PK_ETIMEOUT: bounded device wait gave up";
    case PK_ESTATE: return "PK_ESTATE: call out of order";
    }
    return "unknown pk_status";
}

const char *pk_last_error(pk_plan_t plan) { return plan ? plan->err.c_str() : ""; }

const char *pk_plan_error(void) { return g_plan_error.c_str(); }

static pk_status plan_build(pk_plan_s *P, const pk_config *cfg) {
    const pk_config &c = *cfg;
    // ---- validate ----
    if (!(c.box_size > 0.0) || !isfinite(c.box_size)) return fail(P, PK_EINVAL, "box_size must be > 0");
    if (c.nmesh < 4 || c.nmesh > 4096 || (c.nmesh % 2) != 0)
        return fail(P, PK_EINVAL, "nmesh must be even and in [4, 4096]");
    if (c.window != PK_CIC && c.window != PK_TSC && c.window != PK_PCS)
        return fail(P, PK_EINVAL, "window must be PK_CIC, PK_TSC or PK_PCS");
    if (!(c.dk > 0.0) || !isfinite(c.dk)) return fail(P, PK_EINVAL, "dk must be > 0");
    if (!(c.kmin >= 0.0) || !isfinite(c.kmin)) return fail(P, PK_EINVAL, "kmin must be >= 0");
    if (c.nmu < 0 || c.nmu > 1000) return fail(P, PK_EINVAL, "nmu must be in [0, 1000]");
    if (c.los_axis != 2) return fail(P, PK_EINVAL, "los_axis must be 2 (z, the r2c axis)");
    if (c.precision != PK_MESH_F32 && c.precision != PK_MESH_F64)
        return fail(P, PK_EINVAL, "precision must be PK_MESH_F32 or PK_MESH_F64");
    if (c.fixed_scale_log2 < 0 || c.fixed_scale_log2 > 40)
        return fail(P, PK_EINVAL, "fixed_scale_log2 must be in [0, 40]");
    if (c.batch < 0 || c.batch > 65535) return fail(P, PK_EINVAL, "batch must be in [0, 65535]");
    if ((c.poles_mask & ~7u) != 0) return fail(P, PK_EINVAL, "poles_mask uses bits 0..2 only");
    if (c.paint_variant != PK_PAINT_SORT && c.paint_variant != PK_PAINT_ATOMIC)
        return fail(P, PK_EINVAL, "paint_variant must be PK_PAINT_SORT or PK_PAINT_ATOMIC");
    if (c.capacity < 0 || c.capacity >= (int64_t)0xffffffffLL)
        return fail(P, PK_EINVAL, "capacity must be in [0, 2^32 - 2]");

    P->cfg = c;
    P->N = c.nmesh;
    P->Nh = c.nmesh / 2 + 1;
    P->p = c.window;
    P->nm = c.interlaced ? 2 : 1;
    P->B = c.batch > 0 ? c.batch : 1;
    P->f64 = c.precision == PK_MESH_F64;
    P->esz = P->f64 ? 8 : 4;
    P->S = c.fixed_scale_log2 > 0 ? c.fixed_scale_log2 : (P->f64 ? 32 : 22);
    P->mesh_reals = (long long)P->N * P->N * 2 * P->Nh;

    int rlo, rhi;
    window_reach(P->p, c.interlaced, &rlo, &rhi);
    const int T = choose_tile(P->N, rhi - rlo, c.tile);
    if (T <= 0)
        return fail(P, PK_EINVAL, "tile must divide nmesh, be >= the window reach and fit in shared memory");
    const double L = c.box_size;
    P->kF = (2.0 * M_PI) / L;
    const double kmax = c.kmax > 0.0 ? c.kmax : (M_PI * P->N) / L;
    const double nkd = floor((kmax - c.kmin) / c.dk);
    if (!(nkd >= 1.0) || nkd > 1e6) return fail(P, PK_EINVAL, "k binning gives no bins (or more than 1e6)");
    // The bin kernel's FP32 estimate of the k bin must stay within one bin of
    // the exact FP64 bin (its absolute error is below 4e-7 kmax / dk + 0.1).
    if (kmax / c.dk >= 1048576.0) return fail(P, PK_EINVAL, "k binning too fine: kmax / dk must be below 2^20");
    const int nk = (int)nkd;
    PK_CUDA(P, cudaGetDevice(&P->device));
    PK_CUDA(P, cudaDeviceGetAttribute(&P->nsm, cudaDevAttrMultiProcessorCount, P->device));

    // ---- paint geometry ----
    PaintGeom &pg = P->pg;
    pg.invH = (float)((double)P->N / c.box_size);
    pg.invH_lo = (float)((double)P->N / c.box_size - (double)pg.invH);
    pg.invHd = (double)P->N / c.box_size;
    pg.N = P->N;
    pg.T = T;
    pg.ntx = P->N / T;
    pg.lo = rlo;
    pg.hi = rhi;
    pg.ntiles = (long long)pg.ntx * pg.ntx * pg.ntx;
    P->nkeys = pg.ntiles * paint_classes();

    // ---- k bins: exact edges in m space ----
    const long long mcap = 3LL * (P->N / 2) * (P->N / 2) + 1;
    P->kedge.assign(nk + 1, 0);
    {
        int bnext = 0;
        for (long long m = 0; m <= mcap && bnext <= nk; ++m) {
            const long long bm = kbin_of(m, P->kF, c.kmin, c.dk);
            while (bnext <= nk && bm >= bnext) P->kedge[bnext++] = (int)m;
        }
        for (; bnext <= nk; ++bnext) P->kedge[bnext] = (int)(mcap + 1);
    }
    P->k_edges.resize(nk + 1);
    for (int b = 0; b <= nk; ++b) P->k_edges[b] = c.kmin + b * c.dk;
    const int nmu = c.nmu;
    P->mu_edges.resize(nmu > 0 ? nmu + 1 : 0);
    for (int q = 0; q <= nmu && nmu > 0; ++q) P->mu_edges[q] = (double)q / nmu;

    BinGeom &bg = P->bg;
    bg.N = P->N;
    bg.Nh = P->Nh;
    bg.nk = nk;
    bg.nmu = nmu;
    bg.twod = nmu > 0;
    bg.poles = (c.poles_mask & 6u) != 0;
    bg.hbase = bg.twod ? nk * nmu : nk;
    bg.nh = bg.hbase + (bg.poles ? 2 * nk : 0);
    bg.kscale = (float)(P->kF / c.dk);
    bg.koff = (float)(c.kmin / c.dk);
    bg.mlo = P->kedge[0];
    bg.mhi = P->kedge[nk];
    bg.mu32 = (double)(nmu + 1) * (nmu + 1) * (double)(bg.mhi + 1) < 4294967295.0 &&
              (double)nmu * nmu * (double)(P->N / 2) * (P->N / 2) < 4294967295.0;
    if (bin_smem_bytes(bg, P->f64) > 200 * 1024)
        return fail(P, PK_EINVAL, "too many (k, mu) bins for the per-CTA histogram");

    FinalGeom &fg = P->fg;
    fg.nk = nk;
    fg.nmu = nmu;
    fg.twod = bg.twod;
    fg.poles = bg.poles;
    fg.hbase = bg.hbase;
    fg.nh = bg.nh;
    fg.poles_mask = c.poles_mask;
    fg.subtract_shot = c.subtract_shot;
    fg.L3 = L * L * L;
    fg.headroom = ldexp(1.0, 62 - P->S);
    P->rl = result_layout(nk, nmu);
    fg.RL = P->rl.total;

    // ---- stream, events, memory ----
    P->st = nullptr;
    PK_CUDA(P, cudaEventCreateWithFlags(&P->done, cudaEventDisableTiming));
    const size_t mesh_bytes = (size_t)P->B * P->nm * P->mesh_reals * P->esz;
    PK_CUDA(P, dev_alloc(&P->mesh, mesh_bytes));
    const long long keys_all = (long long)P->B * P->nkeys;
    PK_CUDA(P, dev_alloc(&P->d_count, sizeof(uint32_t) * keys_all));
    PK_CUDA(P, dev_alloc(&P->d_off, sizeof(uint32_t) * (keys_all + 1)));
    PK_CUDA(P, dev_alloc(&P->d_scan_tmp, sizeof(uint32_t) * scan_tmp_elems(keys_all)));
    PK_CUDA(P, dev_alloc(&P->d_item_off, sizeof(int64_t) * (P->B + 1)));
    PK_CUDA(P, dev_alloc(&P->d_wsums, sizeof(double) * 4 * P->B));
    PK_CUDA(P, dev_alloc(&P->d_wpart, sizeof(double) * wsum_partial_elems(P->B)));
    PK_CUDA(P, dev_alloc(&P->d_wmax, sizeof(unsigned) * P->B));
    PK_CUDA(P, dev_alloc(&P->d_err, sizeof(int)));
    PK_CUDA(P, cudaMemset(P->d_err, 0, sizeof(int)));
    PK_CUDA(P, dev_alloc(&P->d_cw, P->esz * P->N));
    PK_CUDA(P, dev_alloc(&P->d_ph, 2 * P->esz * (P->N + 1)));
    PK_CUDA(P, dev_alloc(&P->d_kedge, sizeof(int) * (nk + 1)));
    const int occ = bin_ctas_per_sm(bg, P->f64);
    P->G_total = P->nsm * occ;
    PK_CUDA(P, dev_alloc(&P->d_partial, (size_t)(P->G_total + P->B) * bg.nh * (P->f64 ? 8 : 4)));
    PK_CUDA(P, dev_alloc(&P->d_sums2, sizeof(double) * (size_t)(reduce_chunks(P->G_total) + P->B) * bg.nh));
    PK_CUDA(P, dev_alloc(&P->d_res, sizeof(double) * (size_t)P->B * fg.RL));
    PK_CUDA(P, cudaMallocHost(reinterpret_cast<void **>(&P->h_res), sizeof(double) * (size_t)P->B * fg.RL));
    PK_CUDA(P, dev_alloc(&P->d_xres, sizeof(double) * (size_t)fg.RL));
    PK_CUDA(P, dev_alloc(&P->d_proj, sizeof(double) * 3 * (size_t)nk));
    PK_CUDA(P, cudaMallocHost(reinterpret_cast<void **>(&P->h_xres), sizeof(double) * (size_t)fg.RL));
    PK_CUDA(P, cudaEventCreateWithFlags(&P->xdone, cudaEventDisableTiming));
    const int nq = nmu > 0 ? nmu : 1;
    if (c.paint_variant == PK_PAINT_ATOMIC) {
        const size_t acc_bytes = sizeof(unsigned long long) * (size_t)P->B * P->nm * P->N * P->N * P->N;
        PK_CUDA(P, dev_alloc(&P->d_acc, acc_bytes));
        PK_CUDA(P, cudaMemset(P->d_acc, 0, acc_bytes));
    } else if (c.capacity > 0) {
        PK_CUDA(P, dev_alloc(&P->d_sorted, sizeof(float4) * (size_t)c.capacity));
        P->sorted_cap = c.capacity;
    }
    PK_CUDA(P, dev_alloc(&P->d_modes1d, sizeof(unsigned long long) * nk));
    PK_CUDA(P, dev_alloc(&P->d_modes2d, sizeof(unsigned long long) * (size_t)nk * nq));

    // ---- tables (FP64 on the host, stored in the mesh precision) ----
    {
        std::vector<double> cw(P->N), ph(2 * (P->N + 1));
        for (int i = 0; i < P->N; ++i) {
            const int ip = i < P->N / 2 ? i : i - P->N;
            const double s = sinc(M_PI * ip / P->N);
            cw[i] = c.compensated ? 1.0 / pow(s, 2 * P->p) : 1.0;
        }
        for (int k = 0; k <= P->N; ++k) {
            const double a = M_PI * (double)(k - P->N / 2) / P->N;
            ph[2 * k] = cos(a);
            ph[2 * k + 1] = sin(a);
        }
        if (P->f64) {
            PK_CUDA(P, cudaMemcpy(P->d_cw, cw.data(), 8 * cw.size(), cudaMemcpyHostToDevice));
            PK_CUDA(P, cudaMemcpy(P->d_ph, ph.data(), 8 * ph.size(), cudaMemcpyHostToDevice));
        } else {
            std::vector<float> cwf(cw.begin(), cw.end()), phf(ph.begin(), ph.end());
            PK_CUDA(P, cudaMemcpy(P->d_cw, cwf.data(), 4 * cwf.size(), cudaMemcpyHostToDevice));
            PK_CUDA(P, cudaMemcpy(P->d_ph, phf.data(), 4 * phf.size(), cudaMemcpyHostToDevice));
        }
        PK_CUDA(P, cudaMemcpy(P->d_kedge, P->kedge.data(), sizeof(int) * (nk + 1), cudaMemcpyHostToDevice));
    }

    // ---- own transform: FP32 meshes of the supported sizes (the default at all but 1024) ----
    if (!P->f64 && own_fft_supported(P->N)) {
        std::vector<float> tw(2 * (size_t)P->N);
        own_fft_twiddles(P->N, tw.data());
        PK_CUDA(P, dev_alloc(&P->d_tw, sizeof(float) * tw.size()));
        PK_CUDA(P, cudaMemcpy(P->d_tw, tw.data(), sizeof(float) * tw.size(), cudaMemcpyHostToDevice));
        // one wave of k_zbin CTAs, within the partial histograms k_bin's grid sized
        P->G_own = std::min(P->G_total, P->nsm * zbin_ctas_per_sm(bg, c.interlaced));
        P->own_fft = own_fft_default(P->N) ? 1 : 0;
    }

    // ---- geometry-only bin data: exact counts, mean k, mean mu ----
    {
        const size_t hn = (size_t)bg.mhi * nq + 1;
        if (hn > ((size_t)1 << 28))
            return fail(P, PK_EINVAL, "nmu too large for this nmesh / kmax (geometry histogram > 2^28)");
        unsigned long long *H = nullptr, *HL = nullptr;
        PK_CUDA(P, dev_alloc(&H, sizeof(unsigned long long) * hn));
        cudaError_t e = dev_alloc(&HL, sizeof(unsigned long long) * hn);
        if (e != cudaSuccess) {
            cudaFree(H);
            return fail(P, PK_ENOMEM, "geometry histogram allocation failed");
        }
        double *kmean2d = nullptr, *mumean2d = nullptr;
        e = dev_alloc(&kmean2d, sizeof(double) * (size_t)nk * nq);
        if (e == cudaSuccess) e = dev_alloc(&mumean2d, sizeof(double) * (size_t)nk * nq);
        if (e == cudaSuccess) e = cudaMemset(H, 0, sizeof(unsigned long long) * hn);
        if (e == cudaSuccess) e = cudaMemset(HL, 0, sizeof(unsigned long long) * hn);
        if (e == cudaSuccess) e = launch_geom_hist(bg, H, HL, nullptr);
        if (e == cudaSuccess)
            e = launch_geom_finalize(bg, P->d_kedge, P->kF, H, HL, P->d_modes2d, kmean2d, mumean2d,
                                     nullptr);
        if (e == cudaSuccess) e = cudaDeviceSynchronize();
        P->launches += 2;
        P->modes2d.resize((size_t)nk * nq);
        P->kmean2d.resize((size_t)nk * nq);
        P->mumean2d.resize((size_t)nk * nq);
        if (e == cudaSuccess)
            e = cudaMemcpy(P->modes2d.data(), P->d_modes2d, 8 * P->modes2d.size(), cudaMemcpyDeviceToHost);
        if (e == cudaSuccess)
            e = cudaMemcpy(P->kmean2d.data(), kmean2d, 8 * P->kmean2d.size(), cudaMemcpyDeviceToHost);
        if (e == cudaSuccess)
            e = cudaMemcpy(P->mumean2d.data(), mumean2d, 8 * P->mumean2d.size(), cudaMemcpyDeviceToHost);
        cudaFree(H);
        cudaFree(HL);
        if (kmean2d) cudaFree(kmean2d);
        if (mumean2d) cudaFree(mumean2d);
        if (e != cudaSuccess)
            return fail(P, e == cudaErrorMemoryAllocation ? PK_ENOMEM : PK_ECUDA,
                        std::string("geometry pass: ") + cudaGetErrorString(e));
        P->modes1d.assign(nk, 0);
        P->kmean1d.assign(nk, NAN);
        for (int b = 0; b < nk; ++b) {
            unsigned long long cnt = 0;
            double ks = 0.0;
            for (int q = 0; q < nq; ++q) {
                const unsigned long long cq = P->modes2d[(size_t)b * nq + q];
                cnt += cq;
                if (cq) ks += P->kmean2d[(size_t)b * nq + q] * (double)cq;
            }
            P->modes1d[b] = cnt;
            if (cnt) P->kmean1d[b] = ks / (double)cnt;
        }
        PK_CUDA(P, cudaMemcpy(P->d_modes1d, P->modes1d.data(), 8 * nk, cudaMemcpyHostToDevice));
    }

    return PK_OK;
}

pk_status pk_plan(const pk_config *cfg, void *cuda_stream, pk_plan_t *out) {
    g_plan_error.clear();
    if (!out) return fail(nullptr, PK_EINVAL, "out is NULL");
    *out = nullptr;
    if (!cfg) return fail(nullptr, PK_EINVAL, "cfg is NULL");
    pk_plan_s *P = new (std::nothrow) pk_plan_s();
    if (!P) return fail(nullptr, PK_ENOMEM, "host allocation failed");
    pk_status s = plan_build(P, cfg);
    if (s != PK_OK) {
        g_plan_error = P->err;
        free_plan(P);
        return s;
    }
    P->st = reinterpret_cast<cudaStream_t>(cuda_stream);
    if (!P->own_fft) {
        s = ensure_cufft(P);
        if (s != PK_OK) {
            g_plan_error = P->err;
            free_plan(P);
            return s;
        }
    }
    *out = P;
    return PK_OK;
}

// The atomic variant: weight sums and deposits in one pass, then conversion.
static pk_status paint_atomic(pk_plan_s *P, const void *dpos, int dtype, const float *dw, const float *dv,
                              const int64_t *offsets, int nitems, int64_t max_n, int accumulate) {
    const cudaStream_t st = P->st;
    const int tm = P->timing && !capturing(st);
    if (tm) PK_CUDA(P, cudaEventRecord(P->tev[0], st));
    int launches = 2;
    PK_CUDA(P, launch_upload_i64(P->d_item_off, offsets, nitems + 1, &launches, st));
    if (!accumulate) {
        PK_CUDA(P, cudaMemsetAsync(P->d_wsums, 0, sizeof(double) * 4 * nitems, st));
        PK_CUDA(P, cudaMemsetAsync(P->d_wmax, 0, sizeof(unsigned) * nitems, st));
    }
    if (tm) PK_CUDA(P, cudaEventRecord(P->tev[1], st));   // no sort stage
    PK_CUDA(P, launch_paint_atomic(dpos, dtype, dw, dv, P->d_item_off, nitems, max_n, P->pg, P->p, P->nm, P->S,
                                   P->d_acc, P->d_wsums, P->d_wpart, P->d_wmax, st));
    if (dw != nullptr || dv != nullptr || dtype == PK_F32X4) launches += 1;   // the weight sums' reduce
    PK_CUDA(P, launch_acc_to_mesh(P->d_acc, nitems, P->nm, P->N, P->S, P->f64, P->mesh,
                                  P->nm * P->mesh_reals, P->mesh_reals, accumulate, P->nsm, st));
    if (tm) PK_CUDA(P, cudaEventRecord(P->tev[2], st));
    P->tev_paint = tm;
    P->launches += launches;
    P->npainted = nitems;
    P->transformed = 0;
    P->zpacked = 0;
    return PK_OK;
}

static pk_status paint_impl(pk_plan_s *P, const void *pos, int dtype, const float *weights,
                            const float *values, const int64_t *offsets, int nitems, int accumulate) {
    if (dtype != PK_F32 && dtype != PK_F64 && dtype != PK_F32X4)
        return fail(P, PK_EINVAL, "dtype must be PK_F32, PK_F64 or PK_F32X4");
    if (dtype == PK_F32X4 && weights)
        return fail(P, PK_EINVAL, "weights must be NULL with PK_F32X4 (the 4th component is the weight)");
    if (nitems < 1 || nitems > P->B) return fail(P, PK_EINVAL, "item count exceeds the plan's batch");
    if (accumulate && (P->transformed || P->npainted < nitems))
        return fail(P, PK_ESTATE, "accumulate needs an untransformed, painted mesh");
    if (offsets[0] != 0) return fail(P, PK_EINVAL, "offsets[0] must be 0");
    int64_t max_n = 0;
    for (int k = 0; k < nitems; ++k) {
        const int64_t nk = offsets[k + 1] - offsets[k];
        if (nk < 0) return fail(P, PK_EINVAL, "offsets must be non-decreasing (n >= 0)");
        max_n = std::max(max_n, nk);
    }
    const int64_t ntot = offsets[nitems];
    if (ntot > 0 && !pos) return fail(P, PK_EINVAL, "pos is NULL");
    const cudaStream_t st = P->st;
    const size_t rb = record_bytes(dtype);

    // stage host inputs on the device
    const void *dpos = pos;
    const float *dw = weights;
    const float *dv = values;
    const bool pos_dev = ntot == 0 || is_device_pointer(pos);
    const bool w_dev = !weights || ntot == 0 || is_device_pointer(weights);
    const bool v_dev = !values || ntot == 0 || is_device_pointer(values);
    if (pos_dev && dtype == PK_F32X4 && (reinterpret_cast<uintptr_t>(pos) % 16) != 0)
        return fail(P, PK_EINVAL, "PK_F32X4 positions must be 16-byte aligned");
    if (pos_dev && dtype == PK_F64 && (reinterpret_cast<uintptr_t>(pos) % 8) != 0)
        return fail(P, PK_EINVAL, "PK_F64 positions must be 8-byte aligned");
    if ((!pos_dev || !w_dev || !v_dev) && capturing(st))
        return fail(P, PK_EINVAL, "host positions, weights or values cannot be painted under stream capture");
    if (!pos_dev || !w_dev || !v_dev) {
        const size_t pbytes = pos_dev ? 0 : (size_t)ntot * rb;
        const size_t pad = (pbytes + 255) / 256 * 256;
        const size_t wbytes = w_dev ? 0 : (size_t)ntot * sizeof(float);
        const size_t wpad = (wbytes + 255) / 256 * 256;
        const size_t vbytes = v_dev ? 0 : (size_t)ntot * sizeof(float);
        const size_t need = pad + wpad + vbytes;
        if (need > P->stage_cap) {
            PK_CUDA(P, cudaStreamSynchronize(st));
            if (P->d_stage) cudaFree(P->d_stage);
            P->d_stage = nullptr;
            P->stage_cap = 0;
            PK_CUDA(P, cudaMalloc(&P->d_stage, need));
            P->stage_cap = need;
        }
        char *sb = reinterpret_cast<char *>(P->d_stage);
        if (!pos_dev) {
            PK_CUDA(P, cudaMemcpyAsync(sb, pos, pbytes, cudaMemcpyHostToDevice, st));
            dpos = sb;
        }
        if (!w_dev) {
            PK_CUDA(P, cudaMemcpyAsync(sb + pad, weights, wbytes, cudaMemcpyHostToDevice, st));
            dw = reinterpret_cast<const float *>(sb + pad);
        }
        if (!v_dev) {
            PK_CUDA(P, cudaMemcpyAsync(sb + pad + wpad, values, vbytes, cudaMemcpyHostToDevice, st));
            dv = reinterpret_cast<const float *>(sb + pad + wpad);
        }
    }

    if (ntot >= (int64_t)0xffffffffLL)
        return fail(P, PK_EINVAL, "at most 2^32 - 2 objects per paint call");
    if (P->cfg.paint_variant == PK_PAINT_ATOMIC)
        return paint_atomic(P, dpos, dtype, dw, dv, offsets, nitems, max_n, accumulate);
    if (ntot > P->sorted_cap && capturing(st))
        return fail(P, PK_EINVAL, "objects exceed the plan's capacity under stream capture");
    if (ntot > P->sorted_cap) {                 // grow the key-ordered copy (rare)
        PK_CUDA(P, cudaStreamSynchronize(st));
        if (P->d_sorted) cudaFree(P->d_sorted);
        P->d_sorted = nullptr;
        P->sorted_cap = 0;
        PK_CUDA(P, cudaMalloc(reinterpret_cast<void **>(&P->d_sorted), sizeof(float4) * (size_t)ntot));
        P->sorted_cap = ntot;
    }
    const long long nkeys = (long long)nitems * P->nkeys;
    const int tm = P->timing && !capturing(st);
    if (tm) PK_CUDA(P, cudaEventRecord(P->tev[0], st));
    int launches = 2;   // count, scatter
    PK_CUDA(P, launch_upload_i64(P->d_item_off, offsets, nitems + 1, &launches, st));
    PK_CUDA(P, cudaMemsetAsync(P->d_count, 0, sizeof(uint32_t) * nkeys, st));
    if (!accumulate) {
        PK_CUDA(P, cudaMemsetAsync(P->d_wsums, 0, sizeof(double) * 4 * nitems, st));
        PK_CUDA(P, cudaMemsetAsync(P->d_wmax, 0, sizeof(unsigned) * nitems, st));
    }
    PK_CUDA(P, launch_sort_count(dpos, dtype, dw, dv, P->d_item_off, nitems, max_n, P->pg, P->d_count,
                                 P->d_wsums, P->d_wpart, P->d_wmax, st));
    if (dw != nullptr || dv != nullptr || dtype == PK_F32X4) launches += 1;   // the weight sums' reduce
    PK_CUDA(P, launch_scan(P->d_count, nkeys, P->d_off, P->d_scan_tmp, &launches, st));
    PK_CUDA(P, launch_sort_scatter(dpos, dtype, dw, dv, P->d_item_off, nitems, max_n, P->pg, P->d_off,
                                   P->d_count, P->d_sorted, P->d_err, st));
    if (tm) PK_CUDA(P, cudaEventRecord(P->tev[1], st));
    const int unit_weights = dw == nullptr && dv == nullptr && dtype != PK_F32X4;
    PK_CUDA(P, launch_paint_tiles(P->d_sorted, P->d_off, nitems, P->pg, P->p, P->nm, P->S, P->f64,
                                  P->d_wmax, unit_weights, P->mesh, P->nm * P->mesh_reals,
                                  P->mesh_reals, accumulate, st));
    launches += 1;
    if (tm) PK_CUDA(P, cudaEventRecord(P->tev[2], st));
    P->tev_paint = tm;
    P->launches += launches;
    P->npainted = nitems;
    P->transformed = 0;
    P->zpacked = 0;
    return PK_OK;
}

pk_status pk_paint(pk_plan_t P, const void *pos, int dtype, const float *weights, int64_t n,
                   int accumulate) {
    if (!P) return PK_EINVAL;
    P->err.clear();
    if (n < 0) return fail(P, PK_EINVAL, "n must be >= 0");
    const int64_t off[2] = {0, n};
    return paint_impl(P, pos, dtype, weights, nullptr, off, 1, accumulate ? 1 : 0);
}

pk_status pk_paint_many(pk_plan_t P, const void *pos, int dtype, const float *weights,
                        const int64_t *offsets, int nitems) {
    if (!P) return PK_EINVAL;
    P->err.clear();
    if (!offsets) return fail(P, PK_EINVAL, "offsets is NULL");
    return paint_impl(P, pos, dtype, weights, nullptr, offsets, nitems, 0);
}

pk_status pk_paint_values(pk_plan_t P, const void *pos, int dtype, const float *weights, const float *values,
                          const int64_t *offsets, int nitems) {
    if (!P) return PK_EINVAL;
    P->err.clear();
    if (!offsets) return fail(P, PK_EINVAL, "offsets is NULL");
    if (!values && offsets[nitems > 0 ? nitems : 0] > 0) return fail(P, PK_EINVAL, "values is NULL");
    return paint_impl(P, pos, dtype, weights, values, offsets, nitems, 0);
}

pk_status pk_compute(pk_plan_t P) {
    if (!P) return PK_EINVAL;
    P->err.clear();
    if (P->npainted < 1 || P->transformed) return fail(P, PK_ESTATE, "nothing painted since the last compute");
    const cudaStream_t st = P->st;
    const int cap = capturing(st);
    const int tm = P->timing && !cap;
    if (tm) PK_CUDA(P, cudaEventRecord(P->tev[3], st));
    const int nitems = P->npainted;
    const long long item_c = (long long)P->nm * P->mesh_reals / 2;   // complex elements
    const long long mesh_c = P->mesh_reals / 2;
    int G = std::max(1, P->G_total / nitems);
    pk_status s_ = PK_OK;
    if (P->own_fft) {
        // x and y passes, then z fused into the bin pass: the meshes end up
        // holding the x/y transforms of the packed z rows (zpacked)
        G = std::max(1, P->G_own / nitems);
        PK_CUDA(P, launch_fft_xy(P->mesh, nitems * P->nm, mesh_c, P->N, P->d_tw, st));
        P->transformed = 1;
        P->zpacked = 1;
        if (tm) PK_CUDA(P, cudaEventRecord(P->tev[4], st));
        PK_CUDA(P, launch_zbin(P->mesh, P->cfg.interlaced, item_c, mesh_c, nitems, G, P->bg, P->d_cw, P->d_ph,
                               P->d_tw, P->d_kedge, P->d_partial, st));
        P->launches += 2;   // the two axis passes
    } else if ((s_ = ensure_cufft(P)) != PK_OK) {
        return s_;
    } else if (P->fft_single) {
        PK_CUFFT(P, transform_meshes(P, P->mesh, P->npainted * P->nm));
    } else {
        // the painted catalogs: the whole-batch plan, else the binary digits of
        // the count (every power of two below B has a plan, and count < B)
        const int nplans = (int)P->fft.size();
        int left = P->npainted, at = 0;
        for (int k = nplans - 1; k >= 0 && left > 0; --k) {
            const int c = P->fft_items[k];
            const bool whole = k == nplans - 1;
            if (whole ? c != left : c > left) continue;
            const size_t off = (size_t)at * P->nm * P->mesh_reals;
            if (P->f64) {
                cufftDoubleReal *r = reinterpret_cast<cufftDoubleReal *>(P->mesh) + off;
                PK_CUFFT(P, cufftExecD2Z(P->fft[k], r, reinterpret_cast<cufftDoubleComplex *>(r)));
            } else {
                cufftReal *r = reinterpret_cast<cufftReal *>(P->mesh) + off;
                PK_CUFFT(P, cufftExecR2C(P->fft[k], r, reinterpret_cast<cufftComplex *>(r)));
            }
            at += c;
            left -= c;
        }
        if (left != 0) return fail(P, PK_ECUFFT, "internal: catalog count not covered by the FFT plans");
    }
    if (!P->own_fft) {
        P->transformed = 1;
        P->zpacked = 0;
        if (tm) PK_CUDA(P, cudaEventRecord(P->tev[4], st));
        PK_CUDA(P, launch_bin(P->mesh, P->f64, P->cfg.interlaced, item_c, mesh_c, nitems, G, P->bg,
                              P->d_cw, P->d_ph, P->d_kedge, P->d_partial, st));
    }
    if (tm) PK_CUDA(P, cudaEventRecord(P->tev[5], st));
    PK_CUDA(P, launch_bin_reduce(P->d_partial, P->f64, G, P->bg.nh, nitems, P->d_sums2, st));
    PK_CUDA(P, launch_finalize(P->d_sums2, G, P->d_modes1d, P->d_modes2d, P->d_wsums, P->d_err, P->fg,
                               nitems, P->d_res, st));
    if (tm) PK_CUDA(P, cudaEventRecord(P->tev[6], st));
    P->tev_compute = tm;
    P->launches += 2 + reduce_launches(G);   // bin, reduce (one or two passes), finalize
    PK_CUDA(P, cudaMemcpyAsync(P->h_res, P->d_res, sizeof(double) * (size_t)nitems * P->fg.RL,
                               cudaMemcpyDeviceToHost, st));
    // Under stream capture the results come from a later graph replay, which
    // the caller synchronizes; an event recorded into the capture could not
    // be waited on outside it.
    if (!cap) PK_CUDA(P, cudaEventRecord(P->done, st));
    P->done_valid = !cap;
    P->computed = nitems;
    P->npainted = 0;
    return PK_OK;
}

static pk_status fill_view(pk_plan_s *P, const double *r, pk_result_view *out);

// After a compute on the own transform the meshes hold the x/y transforms of
// the packed z rows; the passes that read the r2c transform itself get it
// written in place first (once per compute).
static pk_status finish_transform(pk_plan_s *P) {
    if (!P->zpacked) return PK_OK;
    const long long item_c = (long long)P->nm * P->mesh_reals / 2;
    PK_CUDA(P, launch_zfinish(P->mesh, P->cfg.interlaced, item_c, P->mesh_reals / 2, P->computed, P->N, P->d_tw,
                              P->nsm, P->st));
    P->launches += 1;
    P->zpacked = 0;
    return PK_OK;
}

pk_status pk_use_own_fft(pk_plan_t P, int on) {
    if (!P) return PK_EINVAL;
    P->err.clear();
    if (on && !P->d_tw)
        return fail(P, PK_EINVAL, "the own transform needs the FP32 mesh form and nmesh 128, 192, 256, 512, 1024 or 2048");
    if (!on) {
        if (pk_status s = ensure_cufft(P); s != PK_OK) return s;
    }
    P->own_fft = on ? 1 : 0;
    return PK_OK;
}

pk_status pk_result(pk_plan_t P, int item, pk_result_view *out) {
    if (!P) return PK_EINVAL;
    P->err.clear();
    if (!out) return fail(P, PK_EINVAL, "out is NULL");
    if (P->computed < 1) return fail(P, PK_ESTATE, "no compute yet");
    if (item < 0 || item >= P->computed) return fail(P, PK_EINVAL, "item out of range");
    if (P->done_valid) PK_CUDA(P, cudaEventSynchronize(P->done));
    return fill_view(P, P->h_res + (size_t)item * P->fg.RL, out);
}

pk_status pk_cross(pk_plan_t P, int item_a, int item_b) {
    if (!P) return PK_EINVAL;
    P->err.clear();
    if (!P->transformed || P->computed < 1) return fail(P, PK_ESTATE, "pk_cross needs a pk_compute first");
    if (item_a < 0 || item_a >= P->computed || item_b < 0 || item_b >= P->computed)
        return fail(P, PK_EINVAL, "item out of range");
    const cudaStream_t st = P->st;
    if (pk_status s = finish_transform(P); s != PK_OK) return s;
    const long long item_c = (long long)P->nm * P->mesh_reals / 2;   // complex elements per catalog
    const long long mesh_c = P->mesh_reals / 2;
    const size_t csz = 2 * P->esz;
    const char *base = reinterpret_cast<const char *>(P->mesh);
    PK_CUDA(P, launch_bin_cross(base + (size_t)item_a * item_c * csz, base + (size_t)item_b * item_c * csz, P->f64,
                                P->cfg.interlaced, mesh_c, P->G_total, P->bg, P->d_cw, P->d_ph, P->d_kedge,
                                P->d_partial, st));
    PK_CUDA(P, launch_bin_reduce(P->d_partial, P->f64, P->G_total, P->bg.nh, 1, P->d_sums2, st));
    PK_CUDA(P, launch_finalize_cross(P->d_sums2, P->G_total, P->d_modes1d, P->d_modes2d, P->d_wsums, P->d_err,
                                     P->fg, item_a, item_b, P->d_xres, st));
    P->launches += 2 + reduce_launches(P->G_total);
    PK_CUDA(P, cudaMemcpyAsync(P->h_xres, P->d_xres, sizeof(double) * (size_t)P->fg.RL, cudaMemcpyDeviceToHost,
                               st));
    const int cap = capturing(st);
    if (!cap) PK_CUDA(P, cudaEventRecord(P->xdone, st));
    P->xdone_valid = !cap;
    P->xcomputed = 1;
    return PK_OK;
}

pk_status pk_cross_result(pk_plan_t P, pk_result_view *out) {
    if (!P) return PK_EINVAL;
    P->err.clear();
    if (!out) return fail(P, PK_EINVAL, "out is NULL");
    if (!P->xcomputed) return fail(P, PK_ESTATE, "no pk_cross yet");
    if (P->xdone_valid) PK_CUDA(P, cudaEventSynchronize(P->xdone));
    return fill_view(P, P->h_xres, out);
}

pk_status pk_projected(pk_plan_t P, int item, unsigned keep_axes, pk_projected_view *out) {
    if (!P) return PK_EINVAL;
    P->err.clear();
    if (!out) return fail(P, PK_EINVAL, "out is NULL");
    const int d = (int)((keep_axes & 1u) + ((keep_axes >> 1) & 1u) + ((keep_axes >> 2) & 1u));
    if ((keep_axes & ~7u) != 0 || d < 1 || d > 2)
        return fail(P, PK_EINVAL, "keep_axes must name one or two of the axes x (1), y (2), z (4)");
    if (!P->transformed || P->computed < 1) return fail(P, PK_ESTATE, "pk_projected needs a pk_compute first");
    if (item < 0 || item >= P->computed) return fail(P, PK_EINVAL, "item out of range");
    const cudaStream_t st = P->st;
    if (pk_status s = finish_transform(P); s != PK_OK) return s;
    const int nk = P->bg.nk;
    const size_t csz = 2 * P->esz;
    const size_t item_bytes = (size_t)P->nm * P->mesh_reals * P->esz;
    const char *m1 = reinterpret_cast<const char *>(P->mesh) + (size_t)item * item_bytes;
    const char *m2 = P->cfg.interlaced ? m1 + (size_t)(P->mesh_reals / 2) * csz : nullptr;
    PK_CUDA(P, cudaMemsetAsync(P->d_proj, 0, sizeof(double) * 3 * (size_t)nk, st));
    PK_CUDA(P, launch_plane_bin(m1, m2, P->f64, P->N, (int)keep_axes, P->d_cw, P->d_ph, P->d_kedge, nk, P->kF,
                                P->d_proj, P->nsm, st));
    P->launches += 1;
    std::vector<double> sums(3 * (size_t)nk);
    double ws[4];
    PK_CUDA(P, cudaMemcpyAsync(sums.data(), P->d_proj, sizeof(double) * sums.size(), cudaMemcpyDeviceToHost, st));
    PK_CUDA(P, cudaMemcpyAsync(ws, P->d_wsums + 4 * item, sizeof(ws), cudaMemcpyDeviceToHost, st));
    PK_CUDA(P, cudaStreamSynchronize(st));
    const double L = P->cfg.box_size;
    const double Ld = d == 1 ? L : L * L;
    const double wsum = ws[0], w2sum = ws[1];
    const double norm = Ld / (wsum * wsum);
    const double shot = Ld * w2sum / (wsum * wsum);
    P->proj_k.assign(nk, NAN);
    P->proj_pk.assign(nk, NAN);
    P->proj_modes.assign(nk, 0);
    for (int b = 0; b < nk; ++b) {
        const double cnt = sums[3 * b];
        P->proj_modes[b] = (uint64_t)cnt;
        if (cnt > 0.0) {
            P->proj_k[b] = sums[3 * b + 1] / cnt;
            P->proj_pk[b] = norm * sums[3 * b + 2] / cnt - (P->cfg.subtract_shot ? shot : 0.0);
        }
    }
    memset(out, 0, sizeof(*out));
    out->nk = nk;
    out->ndim = d;
    out->k_edges = P->k_edges.data();
    out->k_mean = P->proj_k.data();
    out->pk = P->proj_pk.data();
    out->modes = P->proj_modes.data();
    out->shot_noise = shot;
    out->wsum = wsum;
    return PK_OK;
}

static pk_status fill_view(pk_plan_s *P, const double *r, pk_result_view *out) {
    const ResultLayout &rl = P->rl;
    const int nk = P->bg.nk, nmu = P->bg.nmu;
    memset(out, 0, sizeof(*out));
    out->nk = nk;
    out->nmu = nmu;
    out->npoles = 3;
    out->k_edges = P->k_edges.data();
    out->mu_edges = nmu > 0 ? P->mu_edges.data() : nullptr;
    out->k_mean = P->kmean1d.data();
    out->pk = r + rl.pk;
    out->poles = r + rl.poles;
    out->modes = P->modes1d.data();
    out->k_mean2d = nmu > 0 ? P->kmean2d.data() : nullptr;
    out->mu_mean2d = nmu > 0 ? P->mumean2d.data() : nullptr;
    out->pkmu = nmu > 0 ? r + rl.pkmu : nullptr;
    out->modes2d = nmu > 0 ? P->modes2d.data() : nullptr;
    out->shot_noise = r[rl.shot];
    out->wsum = r[rl.wsum];
    out->w2sum = r[rl.w2sum];
    const int flags = (int)r[rl.flags];
    if (flags & 2) return fail(P, PK_ECUDA, "internal: tile sort saw more copies than it counted");
    if (flags & 1) return fail(P, PK_EOVERFLOW, "sum |w| * 2^S exceeded 2^62: lower fixed_scale_log2");
    return PK_OK;
}

pk_status pk_mesh(pk_plan_t P, int item, int mesh, void *dst) {
    if (!P) return PK_EINVAL;
    P->err.clear();
    if (!dst) return fail(P, PK_EINVAL, "dst is NULL");
    if (P->transformed || P->npainted < 1) return fail(P, PK_ESTATE, "no painted, untransformed mesh");
    if (item < 0 || item >= P->npainted) return fail(P, PK_EINVAL, "item out of range");
    if (mesh < 0 || mesh >= P->nm) return fail(P, PK_EINVAL, "mesh out of range");
    const char *src = reinterpret_cast<const char *>(P->mesh) +
                      ((size_t)item * P->nm + mesh) * P->mesh_reals * P->esz;
    const size_t row = (size_t)P->N * P->esz;
    PK_CUDA(P, cudaMemcpy2DAsync(dst, row, src, (size_t)2 * P->Nh * P->esz, row,
                                 (size_t)P->N * P->N, cudaMemcpyDefault, P->st));
    PK_CUDA(P, cudaStreamSynchronize(P->st));
    return PK_OK;
}

pk_status pk_enable_timing(pk_plan_t P, int on) {
    if (!P) return PK_EINVAL;
    P->err.clear();
    if (on && !P->tev[0]) {
        for (cudaEvent_t &e : P->tev) PK_CUDA(P, cudaEventCreate(&e));
    }
    P->timing = on ? 1 : 0;
    P->tev_paint = P->tev_compute = 0;
    return PK_OK;
}

pk_status pk_stage_times(pk_plan_t P, double *ms) {
    if (!P) return PK_EINVAL;
    P->err.clear();
    if (!ms) return fail(P, PK_EINVAL, "ms is NULL");
    if (!P->timing) return fail(P, PK_ESTATE, "timing is off");
    for (int k = 0; k < PK_NSTAGES; ++k) ms[k] = 0.0;
    float t = 0.0f;
    if (P->tev_paint) {
        PK_CUDA(P, cudaEventSynchronize(P->tev[2]));
        PK_CUDA(P, cudaEventElapsedTime(&t, P->tev[0], P->tev[1]));
        ms[PK_STAGE_SORT] = t;
        PK_CUDA(P, cudaEventElapsedTime(&t, P->tev[1], P->tev[2]));
        ms[PK_STAGE_PAINT] = t;
    }
    if (P->tev_compute) {
        PK_CUDA(P, cudaEventSynchronize(P->tev[6]));
        PK_CUDA(P, cudaEventElapsedTime(&t, P->tev[3], P->tev[4]));
        ms[PK_STAGE_FFT] = t;
        PK_CUDA(P, cudaEventElapsedTime(&t, P->tev[4], P->tev[5]));
        ms[PK_STAGE_BIN] = t;
        PK_CUDA(P, cudaEventElapsedTime(&t, P->tev[5], P->tev[6]));
        ms[PK_STAGE_FINAL] = t;
    }
    return PK_OK;
}

long long pk_launch_count(pk_plan_t P) { return P ? P->launches : 0; }

pk_status pk_destroy(pk_plan_t P) {
    if (!P) return PK_OK;
    free_plan(P);
    return PK_OK;
}

}  // extern "C"
