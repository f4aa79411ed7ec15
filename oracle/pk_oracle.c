/*
 * pk_oracle.c -- plain FP64 CPU oracle for the FFT power-spectrum path of
 * nbodykit (Hand, Feng et al., arXiv:1712.05834).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the correctness reference that the
 * CUDA path is compared against.  Only tests/, __graft_entry__.smoke() and
 * bench.py's cpu_baseline / reference leg may load it.  It shares no code,
 * header, table or constant with the CUDA library, and the CUDA library never
 * loads it.
 *
 * Everything is FP64 and written as the plainest loop that states the
 * definition:
 *
 *   oracle_window_weight  B-spline mass-assignment windows of order p = 2, 3, 4
 *                         (CIC, TSC, PCS), Sec. 3.3.2 "From Catalog to Mesh",
 *                         windows cited there to Hockney & Eastwood.
 *   oracle_paint          the painted field F(x) = [1 + delta'(x)] V(x) with
 *                         V = 1 and per-object weights, Sec. 3.3.1 (painting
 *                         equation); one mesh per call, optionally displaced by
 *                         a fraction of a cell (the interlaced second mesh,
 *                         Sec. 3.3.2, "separated by half of a cell size").
 *   oracle_paint_block    the same painted field, evaluated only on one B^3
 *                         block of cells (for meshes too large to hold).
 *   oracle_mode_counts    the weighted mode counts of every k and (k, mu) bin
 *                         (the h-weighted stored half grid, Sec. 3.4.1).
 *   oracle_bin            the FFTPower mode loop, Sec. 3.4.1: window
 *                         compensation by prod_i sinc^p(pi k_i / 2 k_N)
 *                         (Eq. window-deconvolution), the interlacing combine,
 *                         |delta(k)|^2 averaged in k bins, (k, mu) bins and
 *                         Legendre multipoles l = 0, 2, 4.
 *   oracle_bin_pair       the same loop for the cross power of two catalogs,
 *                         P = L^3 Re(delta_a conj(delta_b)) (the cross-correlation
 *                         of two painted fields, e.g. two tracers or a density
 *                         and a momentum field, Sec. 3.3.1).
 *   oracle_r2c            the forward transform between painting and binning
 *                         (Sec. 3.3.1: the real field and its complex Fourier
 *                         field), F~(n) = sum_c F[c] exp(-2 pi i c.n / N), as
 *                         three passes of a plain mixed-radix Cooley-Tukey FFT
 *                         (decimation in time by the smallest prime factor; a
 *                         prime length is summed directly), last axis halved.
 *
 * Parallel loops (OpenMP) never change a result with the thread count: the
 * paint gives each thread a fixed range of x planes and adds every object's
 * deposits in object order; the mode loop sums fixed blocks of x rows and
 * adds the blocks in order; the FFT works on independent lines.
 *
 * Conventions the paper leaves open (each one also used by the CUDA path and
 * listed with its reasoning in the design notes):
 *   - mesh node c sits at position c * H, H = L / N; s = x N / L in cell units;
 *   - positions are wrapped periodically into [0, L);
 *   - the interlaced mesh is painted at x + H/2 on every axis and its
 *     transform is multiplied by exp(+i (kx + ky + kz) H / 2) before averaging;
 *   - k index of axes x, y follows numpy fftfreq (i' = i for i < N/2, else
 *     i - N); the r2c axis z stores l = 0 .. N/2 (l = N/2 taken as +N/2);
 *   - the stored half grid is walked with weight h = 1 on the l = 0 and
 *     l = N/2 planes and h = 2 elsewhere; the DC mode is never binned;
 *   - k bin b = floor((kF * sqrt(m) - kmin) / dk) in IEEE FP64, in exactly
 *     that order, kF = (2 pi) / L, m = i'^2 + j'^2 + l^2; kept iff 0 <= b < nk;
 *   - mu = l / sqrt(m) in [0, 1]; mu bin q = largest integer with
 *     q^2 m <= nmu^2 l^2, clamped to nmu - 1 (edges linspace(0,1,nmu+1),
 *     lower edge inclusive), evaluated in exact integer arithmetic;
 *   - P(mode) = L^3 |delta(k)|^2 with delta(k) = F~(k) / sum(w).
 *
 * Build with -ffp-contract=off: the k-bin expression must round exactly as
 * written.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

/* B-spline mass-assignment window of order p evaluated at distance d (cells)
 * from a mesh node.  Sec. 3.3.2: CIC, TSC, PCS with p = 2, 3, 4. */
double oracle_window_weight(int p, double d)
{
    d = fabs(d);
    if (p == 2) {
        return d < 1.0 ? 1.0 - d : 0.0;
    }
    if (p == 3) {
        if (d < 0.5) return 0.75 - d * d;
        if (d < 1.5) return 0.5 * (1.5 - d) * (1.5 - d);
        return 0.0;
    }
    if (p == 4) {
        if (d < 1.0) return (4.0 - 6.0 * d * d + 3.0 * d * d * d) / 6.0;
        if (d < 2.0) return (2.0 - d) * (2.0 - d) * (2.0 - d) / 6.0;
        return 0.0;
    }
    return NAN;
}

int64_t oracle_kbin(int64_t m, double L, double kmin, double dk);
int64_t oracle_mubin(int64_t m, int64_t l, int64_t nmu);

static int64_t mod_n(int64_t c, int64_t n)
{
    int64_t r = c % n;
    return r < 0 ? r + n : r;
}

/* Paint n objects onto mesh[N][N][N] (C order, z fastest), adding
 *   F[c] += w_q * prod_a W_p(s_a - c_a)
 * for every node c within the window support, with s = wrap(x) N / L + shift.
 * pos is n x 3 FP64, w is n FP64 or NULL (unit weights).  The mesh is not
 * cleared.  Each OpenMP thread owns a fixed range of x planes and walks all
 * objects in order, adding only the deposits that land in its planes, so every
 * cell receives its deposits in object order whatever the thread count.
 * Returns 0, or -1 on bad arguments. */
int oracle_paint(const double *pos, const double *w, int64_t n, double L, int N,
                 int p, double shift, double *mesh)
{
    if (N < 1 || L <= 0.0 || (p < 2 || p > 4)) return -1;
    const int64_t NN = (int64_t)N;
#pragma omp parallel
    {
        int nt = 1, t = 0;
#ifdef _OPENMP
        nt = omp_get_num_threads();
        t = omp_get_thread_num();
#endif
        const int64_t x0 = NN * t / nt, x1 = NN * (t + 1) / nt;   /* this thread's x planes */
        for (int64_t q = 0; q < n && x0 < x1; ++q) {
            double wa[3][8];
            int64_t ia[3][8];
            int mine = 0;
            if (NN >= 2 * (p + 2)) {
                /* skip at once an object whose nodes c0 .. c0 + p + 1 along x
                 * (periodic) miss the planes [x0, x1) */
                double x = pos[3 * q];
                x = x - L * floor(x / L);
                const int64_t d = mod_n((int64_t)floor(x * (double)N / L + shift - 0.5 * p) - x0, NN);
                if (d >= x1 - x0 && d + p + 1 < NN) continue;
            }
            for (int a = 0; a < 3; ++a) {
                double x = pos[3 * q + a];
                x = x - L * floor(x / L);              /* periodic wrap into [0, L) */
                double s = x * (double)N / L + shift;  /* cell units */
                int64_t c0 = (int64_t)floor(s - 0.5 * p);
                for (int k = 0; k < p + 2; ++k) {      /* every node within p/2 */
                    int64_t c = c0 + k;
                    wa[a][k] = oracle_window_weight(p, s - (double)c);
                    ia[a][k] = mod_n(c, NN);
                    if (a == 0 && ia[0][k] >= x0 && ia[0][k] < x1) mine = 1;
                }
                if (a == 0 && !mine) break;            /* no deposit in this thread's planes */
            }
            if (!mine) continue;
            double wq = w ? w[q] : 1.0;
            for (int kx = 0; kx < p + 2; ++kx) {
                if (ia[0][kx] < x0 || ia[0][kx] >= x1) continue;
                for (int ky = 0; ky < p + 2; ++ky)
                    for (int kz = 0; kz < p + 2; ++kz) {
                        double v = wq * wa[0][kx] * wa[1][ky] * wa[2][kz];
                        if (v == 0.0) continue;
                        mesh[(ia[0][kx] * NN + ia[1][ky]) * NN + ia[2][kz]] += v;
                    }
            }
        }
    }
    return 0;
}

/* The painted field F of oracle_paint, evaluated only on the cells
 * c0 + (a, b, c), 0 <= a, b, c < B (indices taken periodically), into
 * out[B][B][B].  Objects whose window misses the block contribute nothing.
 * Independent objects are split over OpenMP threads, each with its own block,
 * summed at the end.  Returns 0, or -1 on bad arguments. */
int oracle_paint_block(const double *pos, const double *w, int64_t n, double L, int N, int p,
                       double shift, const int64_t *c0, int B, double *out)
{
    if (N < 1 || L <= 0.0 || p < 2 || p > 4 || B < 1 || B > N) return -1;
    const int64_t NN = N, BB = B, B3 = BB * BB * BB;
    memset(out, 0, sizeof(double) * (size_t)B3);
#pragma omp parallel
    {
        double *acc = (double *)calloc((size_t)B3, sizeof(double));
#pragma omp for schedule(static)
        for (int64_t q = 0; q < n; ++q) {
            double wa[3][8];
            int64_t ia[3][8];     /* offset of the node inside the block, or -1 */
            int any = 1;
            for (int a = 0; a < 3 && any; ++a) {
                double x = pos[3 * q + a];
                x = x - L * floor(x / L);
                double s = x * (double)N / L + shift;
                int64_t cfirst = (int64_t)floor(s - 0.5 * p);
                any = 0;
                for (int k = 0; k < p + 2; ++k) {
                    int64_t c = cfirst + k;
                    wa[a][k] = oracle_window_weight(p, s - (double)c);
                    int64_t off = mod_n(c - c0[a], NN);
                    ia[a][k] = off < BB ? off : -1;
                    if (ia[a][k] >= 0 && wa[a][k] != 0.0) any = 1;
                }
            }
            if (!any) continue;
            double wq = w ? w[q] : 1.0;
            for (int kx = 0; kx < p + 2; ++kx) {
                if (ia[0][kx] < 0) continue;
                for (int ky = 0; ky < p + 2; ++ky) {
                    if (ia[1][ky] < 0) continue;
                    for (int kz = 0; kz < p + 2; ++kz) {
                        if (ia[2][kz] < 0) continue;
                        acc[(ia[0][kx] * BB + ia[1][ky]) * BB + ia[2][kz]] +=
                            wq * wa[0][kx] * wa[1][ky] * wa[2][kz];
                    }
                }
            }
        }
#pragma omp critical
        for (int64_t k = 0; k < B3; ++k) out[k] += acc[k];
        free(acc);
    }
    return 0;
}

/* Weighted mode counts of the k bins (modes1d[nk]) and, if nmu > 0, of the
 * (k, mu) bins (modes2d[nk * nmu]): the stored half grid with h = 1 on the
 * l = 0 and l = N/2 planes and 2 elsewhere, DC excluded, bins as in
 * oracle_kbin / oracle_mubin.  Outputs are overwritten.  Rows i are split over
 * OpenMP threads with private counters.  Returns 0, or -1 on bad arguments. */
int oracle_mode_counts(int N, double L, double kmin, double dk, int nk, int nmu,
                       int64_t *modes1d, int64_t *modes2d)
{
    if (N < 2 || (N % 2) != 0 || L <= 0.0 || dk <= 0.0 || nk < 0 || nmu < 0) return -1;
    const int64_t NN = N, Nh = N / 2 + 1, nq = nmu > 0 ? nmu : 1;
    memset(modes1d, 0, sizeof(int64_t) * (size_t)nk);
    if (nmu > 0) memset(modes2d, 0, sizeof(int64_t) * (size_t)(nk * nmu));
#pragma omp parallel
    {
        int64_t *c1 = (int64_t *)calloc((size_t)nk, sizeof(int64_t));
        int64_t *c2 = (int64_t *)calloc((size_t)(nk * nq), sizeof(int64_t));
#pragma omp for schedule(dynamic, 4)
        for (int64_t i = 0; i < NN; ++i) {
            int64_t ip = i < NN / 2 ? i : i - NN;
            for (int64_t j = 0; j < NN; ++j) {
                int64_t jp = j < NN / 2 ? j : j - NN;
                for (int64_t l = 0; l < Nh; ++l) {
                    int64_t m = ip * ip + jp * jp + l * l;
                    if (m == 0) continue;
                    int64_t b = oracle_kbin(m, L, kmin, dk);
                    if (b < 0 || b >= nk) continue;
                    int64_t h = (l == 0 || l == NN / 2) ? 1 : 2;
                    c1[b] += h;
                    if (nmu > 0) c2[b * nmu + oracle_mubin(m, l, nmu)] += h;
                }
            }
        }
#pragma omp critical
        {
            for (int k = 0; k < nk; ++k) modes1d[k] += c1[k];
            if (nmu > 0)
                for (int k = 0; k < nk * nmu; ++k) modes2d[k] += c2[k];
        }
        free(c1);
        free(c2);
    }
    return 0;
}

static double sinc(double x)
{
    return x == 0.0 ? 1.0 : sin(x) / x;
}

/* k bin of integer squared index m: floor((kF sqrt(m) - kmin) / dk), FP64,
 * evaluated in exactly this order. */
int64_t oracle_kbin(int64_t m, double L, double kmin, double dk)
{
    double kF = (2.0 * M_PI) / L;
    return (int64_t)floor((kF * sqrt((double)m) - kmin) / dk);
}

/* mu bin of a mode: largest q with q^2 m <= nmu^2 l^2, clamped to nmu - 1. */
int64_t oracle_mubin(int64_t m, int64_t l, int64_t nmu)
{
    int64_t q = 0;
    while (q + 1 <= nmu && (q + 1) * (q + 1) * m <= nmu * nmu * l * l) ++q;
    return q < nmu - 1 ? q : nmu - 1;
}

/* FFTPower mode loop over the stored half grid of one (or two, interlaced)
 * r2c transforms F1, F2 of shape [N][N][N/2+1] complex (interleaved re, im).
 *
 * For every stored mode except DC:
 *   delta = F1                                   (not interlaced), or
 *   delta = (F1 + F2 exp(+i pi (i' + j' + l) / N)) / 2   (interlaced),
 *   delta /= prod_a sinc(pi n_a / N)^p           (if compensated),
 *   delta /= wsum;  P = L^3 |delta|^2,
 * and with weight h the sums below are accumulated into the bins.  All output
 * arrays must be zeroed by the caller:
 *   1D  (nk):      modes1d, ksum1d, psum1d, p2sum1d (P L2(mu)), p4sum1d (P L4(mu))
 *   2D  (nk*nmu):  modes2d, ksum2d, musum2d, psum2d   (only if nmu > 0)
 * Returns 0, or -1 on bad arguments. */
/* delta(k) of one stored mode: the interlacing combine, the compensation and
 * the division by the total weight, as listed above. */
static void mode_delta(const double *F1, const double *F2, int64_t idx, int64_t ip, int64_t jp, int64_t l,
                       int N, int p, int compensated, double wsum, double *re_out, double *im_out)
{
    double re = F1[2 * idx], im = F1[2 * idx + 1];
    if (F2) {
        double ph = M_PI * (double)(ip + jp + l) / (double)N;
        double c = cos(ph), s = sin(ph);
        double re2 = F2[2 * idx], im2 = F2[2 * idx + 1];
        re = 0.5 * (re + (re2 * c - im2 * s));
        im = 0.5 * (im + (re2 * s + im2 * c));
    }
    if (compensated) {
        double W = pow(sinc(M_PI * (double)ip / N), p) *
                   pow(sinc(M_PI * (double)jp / N), p) *
                   pow(sinc(M_PI * (double)l / N), p);
        re /= W;
        im /= W;
    }
    *re_out = re / wsum;
    *im_out = im / wsum;
}

/* The mode loop over the x rows i0 <= i < i1, adding into the given sums. */
static void bin_rows(const double *F1, const double *F2, const double *G1, const double *G2, int N,
                     double L, int p, int compensated, double wsum, double wsum_b, double kmin, double dk,
                     int nk, int nmu, int64_t i0, int64_t i1, int64_t *modes1d, double *ksum1d, double *psum1d,
                     double *p2sum1d, double *p4sum1d, int64_t *modes2d, double *ksum2d, double *musum2d,
                     double *psum2d)
{
    const int64_t NN = N, Nh = N / 2 + 1;
    const double kF = (2.0 * M_PI) / L;
    const double L3 = L * L * L;
    for (int64_t i = i0; i < i1; ++i) {
        int64_t ip = i < NN / 2 ? i : i - NN;       /* fftfreq */
        for (int64_t j = 0; j < NN; ++j) {
            int64_t jp = j < NN / 2 ? j : j - NN;
            for (int64_t l = 0; l < Nh; ++l) {
                int64_t m = ip * ip + jp * jp + l * l;
                if (m == 0) continue;                /* DC is never binned */
                int64_t b = oracle_kbin(m, L, kmin, dk);
                if (b < 0 || b >= nk) continue;
                double h = (l == 0 || l == NN / 2) ? 1.0 : 2.0;
                int64_t idx = ((i * NN) + j) * Nh + l;
                double re, im;
                mode_delta(F1, F2, idx, ip, jp, l, N, p, compensated, wsum, &re, &im);
                double P;
                if (G1) {                            /* cross power with the second catalog */
                    double reb, imb;
                    mode_delta(G1, G2, idx, ip, jp, l, N, p, compensated, wsum_b, &reb, &imb);
                    P = L3 * (re * reb + im * imb);
                } else {
                    P = L3 * (re * re + im * im);
                }
                double k = kF * sqrt((double)m);
                double mu = (double)l / sqrt((double)m);
                double mu2 = mu * mu;
                double L2 = 0.5 * (3.0 * mu2 - 1.0);
                double L4 = (35.0 * mu2 * mu2 - 30.0 * mu2 + 3.0) / 8.0;
                modes1d[b] += (int64_t)h;
                ksum1d[b] += h * k;
                psum1d[b] += h * P;
                p2sum1d[b] += h * P * L2;
                p4sum1d[b] += h * P * L4;
                if (nmu > 0) {
                    int64_t q = oracle_mubin(m, l, nmu);
                    int64_t bq = b * nmu + q;
                    modes2d[bq] += (int64_t)h;
                    ksum2d[bq] += h * k;
                    musum2d[bq] += h * mu;
                    psum2d[bq] += h * P;
                }
            }
        }
    }
}

/* The same loop for the cross power of two catalogs painted on equal meshes:
 * P = L^3 Re(delta_a conj(delta_b)) with each delta formed as above from its
 * own transforms (G1, G2) and total weight (wsum_b).  G1 = NULL gives the
 * auto power of the first catalog.  The x rows are cut into at most 64 fixed
 * blocks, each summed on its own (in parallel), and the blocks are added into
 * the outputs in row order, so the sums do not depend on the thread count. */
int oracle_bin_pair(const double *F1, const double *F2, const double *G1, const double *G2, int N,
                    double L, int p, int compensated, double wsum, double wsum_b, double kmin, double dk,
                    int nk, int nmu, int64_t *modes1d, double *ksum1d, double *psum1d, double *p2sum1d,
                    double *p4sum1d, int64_t *modes2d, double *ksum2d, double *musum2d, double *psum2d)
{
    if (N < 2 || (N % 2) != 0 || L <= 0.0 || dk <= 0.0 || nk < 0 || nmu < 0)
        return -1;
    const int64_t NN = N;
    const int64_t nblk = NN < 64 ? NN : 64;
    const size_t n1 = (size_t)nk, n2 = nmu > 0 ? (size_t)nk * (size_t)nmu : 1;
    const size_t per = 5 * n1 + 4 * n2;           /* one block's sums */
    double *blk = (double *)calloc((size_t)nblk * per, sizeof(double));
    if (!blk) return -2;
    int64_t *cnt = (int64_t *)calloc((size_t)nblk * (n1 + n2), sizeof(int64_t));
    if (!cnt) {
        free(blk);
        return -2;
    }
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t b = 0; b < nblk; ++b) {
        double *s = blk + (size_t)b * per;
        int64_t *c = cnt + (size_t)b * (n1 + n2);
        bin_rows(F1, F2, G1, G2, N, L, p, compensated, wsum, wsum_b, kmin, dk, nk, nmu,
                 NN * b / nblk, NN * (b + 1) / nblk, c, s, s + n1, s + 2 * n1, s + 3 * n1,
                 c + n1, s + 5 * n1, s + 5 * n1 + n2, s + 5 * n1 + 2 * n2);
    }
    for (int64_t b = 0; b < nblk; ++b) {
        const double *s = blk + (size_t)b * per;
        const int64_t *c = cnt + (size_t)b * (n1 + n2);
        for (size_t k = 0; k < n1; ++k) {
            modes1d[k] += c[k];
            ksum1d[k] += s[k];
            psum1d[k] += s[n1 + k];
            p2sum1d[k] += s[2 * n1 + k];
            p4sum1d[k] += s[3 * n1 + k];
        }
        if (nmu > 0) {
            for (size_t k = 0; k < n2; ++k) {
                modes2d[k] += c[n1 + k];
                ksum2d[k] += s[5 * n1 + k];
                musum2d[k] += s[5 * n1 + n2 + k];
                psum2d[k] += s[5 * n1 + 2 * n2 + k];
            }
        }
    }
    free(blk);
    free(cnt);
    return 0;
}

int oracle_bin(const double *F1, const double *F2, int N, double L, int p,
               int compensated, double wsum, double kmin, double dk, int nk,
               int nmu, int64_t *modes1d, double *ksum1d, double *psum1d,
               double *p2sum1d, double *p4sum1d, int64_t *modes2d,
               double *ksum2d, double *musum2d, double *psum2d)
{
    return oracle_bin_pair(F1, F2, NULL, NULL, N, L, p, compensated, wsum, 1.0, kmin, dk, nk, nmu,
                           modes1d, ksum1d, psum1d, p2sum1d, p4sum1d, modes2d, ksum2d, musum2d, psum2d);
}

/* ---- the forward transform (Sec. 3.3.1: real field -> complex field) ----
 *
 * One-dimensional DFT X[k] = sum_{j<n} x[j] w_n^{j k}, w_n = exp(-2 pi i / n),
 * by mixed-radix Cooley-Tukey decimation in time: with p the smallest prime
 * factor of n and m = n / p, Y_r = DFT_m(x[r], x[r + p], x[r + 2p], ...) for
 * r < p, and X[k] = sum_{r<p} w_n^{r k} Y_r[k mod m].  A prime n (m = 1) is
 * therefore the direct sum.  Complex numbers are interleaved (re, im) doubles;
 * tw[2e], tw[2e + 1] = cos, -sin (2 pi e / Ntw) for 0 <= e < Ntw, and n
 * divides Ntw, so w_n^e = tw entry (e mod n) Ntw / n.  scratch holds 2 n
 * doubles; the result goes to out[0 .. 2n). */
static int smallest_prime_factor(int n)
{
    for (int p = 2; p * p <= n; ++p)
        if (n % p == 0) return p;
    return n;
}

static void dft_rec(const double *in, int64_t stride, int n, double *out, const double *tw, int Ntw,
                    double *scratch)
{
    if (n == 1) {
        out[0] = in[0];
        out[1] = in[1];
        return;
    }
    const int p = smallest_prime_factor(n), m = n / p;
    for (int r = 0; r < p; ++r)                     /* the p decimated sub-transforms */
        dft_rec(in + 2 * (int64_t)r * stride, stride * p, m, out + 2 * (int64_t)r * m, tw, Ntw, scratch);
    const int64_t step = Ntw / n;
    for (int k = 0; k < n; ++k) {
        const int km = k % m;
        double sr = 0.0, si = 0.0;
        int64_t e = 0;                              /* e = r k mod n */
        for (int r = 0; r < p; ++r) {
            const double wr = tw[2 * e * step], wi = tw[2 * e * step + 1];
            const double yr = out[2 * ((int64_t)r * m + km)], yi = out[2 * ((int64_t)r * m + km) + 1];
            sr += wr * yr - wi * yi;
            si += wr * yi + wi * yr;
            e += k;
            if (e >= n) e -= n;
        }
        scratch[2 * k] = sr;
        scratch[2 * k + 1] = si;
    }
    memcpy(out, scratch, sizeof(double) * 2 * (size_t)n);
}

/* 1D transform of n complex values, in place in line[0 .. 2n); work holds 4 n doubles. */
void oracle_dft_line(double *line, int n, const double *tw, double *work)
{
    dft_rec(line, 1, n, work, tw, n, work + 2 * (size_t)n);
    memcpy(line, work, sizeof(double) * 2 * (size_t)n);
}

/* The twiddle table of length n (see above): tw[2n]. */
void oracle_twiddles(int n, double *tw)
{
    for (int e = 0; e < n; ++e) {
        const double a = 2.0 * M_PI * (double)e / (double)n;
        tw[2 * e] = cos(a);
        tw[2 * e + 1] = -sin(a);
    }
}

/* r2c transform of mesh[N][N][N] (real, C order) into out[N][N][N/2+1]
 * (complex interleaved): F~(i, j, l) = sum_c F[c] exp(-2 pi i (c_x i + c_y j
 * + c_z l) / N), computed as 1D transforms along z (keeping l <= N/2), then
 * y, then x.  Lines are independent and split over OpenMP threads.  Returns
 * 0, or -1 on bad arguments, -2 if memory runs out. */
int oracle_r2c(const double *mesh, int N, double *out)
{
    if (N < 1) return -1;
    const int64_t NN = N, Nh = N / 2 + 1;
    double *tw = (double *)malloc(sizeof(double) * 2 * (size_t)N);
    if (!tw) return -2;
    oracle_twiddles(N, tw);
    int fail = 0;
#pragma omp parallel
    {
        double *line = (double *)malloc(sizeof(double) * 6 * (size_t)N);
        if (!line) {
#pragma omp atomic write
            fail = 1;
        }
        double *work = line ? line + 2 * (size_t)N : NULL;
        /* z: real input lines, keep l = 0 .. N/2 */
#pragma omp for schedule(static)
        for (int64_t r = 0; r < NN * NN; ++r) {
            if (!line) continue;
            for (int64_t c = 0; c < NN; ++c) {
                line[2 * c] = mesh[r * NN + c];
                line[2 * c + 1] = 0.0;
            }
            oracle_dft_line(line, N, tw, work);
            memcpy(out + 2 * r * Nh, line, sizeof(double) * 2 * (size_t)Nh);
        }
        /* y: lines (i, *, l) */
#pragma omp for schedule(static)
        for (int64_t r = 0; r < NN * Nh; ++r) {
            if (!line) continue;
            const int64_t i = r / Nh, l = r % Nh;
            for (int64_t j = 0; j < NN; ++j) {
                line[2 * j] = out[2 * ((i * NN + j) * Nh + l)];
                line[2 * j + 1] = out[2 * ((i * NN + j) * Nh + l) + 1];
            }
            oracle_dft_line(line, N, tw, work);
            for (int64_t j = 0; j < NN; ++j) {
                out[2 * ((i * NN + j) * Nh + l)] = line[2 * j];
                out[2 * ((i * NN + j) * Nh + l) + 1] = line[2 * j + 1];
            }
        }
        /* x: lines (*, j, l) */
#pragma omp for schedule(static)
        for (int64_t r = 0; r < NN * Nh; ++r) {
            if (!line) continue;
            const int64_t j = r / Nh, l = r % Nh;
            for (int64_t i = 0; i < NN; ++i) {
                line[2 * i] = out[2 * ((i * NN + j) * Nh + l)];
                line[2 * i + 1] = out[2 * ((i * NN + j) * Nh + l) + 1];
            }
            oracle_dft_line(line, N, tw, work);
            for (int64_t i = 0; i < NN; ++i) {
                out[2 * ((i * NN + j) * Nh + l)] = line[2 * i];
                out[2 * ((i * NN + j) * Nh + l) + 1] = line[2 * i + 1];
            }
        }
        free(line);
    }
    free(tw);
    return fail ? -2 : 0;
}

/* Threads the OpenMP loops above run on (1 without OpenMP). */
int oracle_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* Run the OpenMP loops above on n threads from now on (n >= 1). */
void oracle_set_threads(int n)
{
#ifdef _OPENMP
    if (n >= 1) omp_set_num_threads(n);
#else
    (void)n;
#endif
}
