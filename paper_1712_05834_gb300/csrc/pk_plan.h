// pk_plan.h -- the plan object behind pk_plan_t, shared by the host-side
// translation units of libpk.so (pk_api.cu builds and runs it; the survey
// path in pk_survey.cu paints through it and reads its tables).  Not installed.
#pragma once

#include <cuda_runtime.h>
#include <cufft.h>

#include <string>
#include <vector>

#include "pk_internal.h"

struct pk_plan_s {
    pk_config cfg;
    cudaStream_t st = nullptr;
    int device = 0, nsm = 0;
    int N = 0, Nh = 0, p = 0, nm = 1, B = 1, f64 = 0, S = 32;
    size_t esz = 4;                  // bytes per mesh real
    long long mesh_reals = 0;        // N * N * 2 * Nh
    pk::PaintGeom pg{};
    pk::BinGeom bg{};
    pk::FinalGeom fg{};
    pk::ResultLayout rl{};
    double kF = 0.0;

    void *mesh = nullptr;
    // cuFFT plans over 2^k catalogs (k = 0, 1, ...) and over the whole batch,
    // so a compute of n < batch catalogs transforms only their meshes; one
    // shared work area.
    std::vector<int> fft_items;
    std::vector<cufftHandle> fft;
    int fft_single = 0;              // one single-mesh plan, one call per mesh (large meshes)
    void *fft_work = nullptr;
    // Own transform (pk_fft.cu): y and x passes, then z fused into the bin.
    int own_fft = 0;                 // pk_compute uses it (FP32 form, supported N)
    int zpacked = 0;                 // meshes hold the x/y transforms of packed z rows
    int G_own = 0;                   // k_zbin CTAs for one catalog
    void *d_tw = nullptr;            // W_N^e, e < N (float2)

    uint32_t *d_count = nullptr;     // objects per (tile, class) key
    uint32_t *d_off = nullptr;       // exclusive scan of d_count (+ total)
    uint32_t *d_scan_tmp = nullptr;
    float4 *d_sorted = nullptr;      // objects in key order, home-tile-local xyz + w
    int64_t sorted_cap = 0;
    long long nkeys = 0;             // keys per catalog
    void *d_stage = nullptr;
    size_t stage_cap = 0;
    int64_t *d_item_off = nullptr;   // catalog offsets of the last paint call
    double *d_wsums = nullptr;       // per catalog: sum w, sum w^2, sum |w|, spare
    double *d_wpart = nullptr;       // per catalog and paint block: its three weight sums
    unsigned *d_wmax = nullptr;      // per catalog: max |w| as float bits
    int *d_err = nullptr;           // bit 1: tile sort inconsistency (never expected)
    unsigned long long *d_acc = nullptr;   // atomic variant: B * nm * N^3 int64 cells

    void *d_cw = nullptr, *d_ph = nullptr;
    int *d_kedge = nullptr;
    int G_total = 0;
    void *d_partial = nullptr;
    double *d_sums2 = nullptr, *d_res = nullptr, *h_res = nullptr;
    double *d_xres = nullptr, *h_xres = nullptr;   // cross-power result block
    double *d_proj = nullptr;                      // projected power: 3 sums per k bin
    std::vector<double> proj_k, proj_pk;
    std::vector<uint64_t> proj_modes;
    cudaEvent_t xdone = nullptr;
    int xdone_valid = 0, xcomputed = 0;
    unsigned long long *d_modes1d = nullptr, *d_modes2d = nullptr;

    std::vector<int> kedge;
    std::vector<double> k_edges, mu_edges, kmean1d, kmean2d, mumean2d;
    std::vector<uint64_t> modes1d, modes2d;

    int npainted = 0;       // catalogs painted since the last compute
    int transformed = 0;    // meshes hold transforms
    int computed = 0;       // catalogs with results
    cudaEvent_t done = nullptr;
    int done_valid = 0;             // `done` marks the last pk_compute (not captured)
    int timing = 0;
    cudaEvent_t tev[7] = {};        // stage boundaries: sort | paint || fft | bin | final
    int tev_paint = 0, tev_compute = 0;
    long long launches = 0;         // library kernels launched on this plan
    std::string err;
};

// Meshes with N above this are transformed one per cuFFT call.
constexpr int kSingleFftAbove = 512;

namespace pk {
// r2c of `count` consecutive meshes of the plan's layout starting at `first`
// (batched plans: count must equal the meshes of one catalog).
cufftResult transform_meshes(pk_plan_s *P, void *first, int count);
// Make the plan's cuFFT plans if they do not exist yet (not under stream capture).
pk_status ensure_cufft(pk_plan_s *P);
}  // namespace pk
