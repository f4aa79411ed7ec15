/*
 * lognormal_oracle.c -- plain FP64 CPU oracle of the log-normal mock
 * generator (the LogNormalCatalog source that the paper's tests and
 * benchmarks paint, Sec. 3.2; nbodykit's Gaussian LinearMesh underneath it).
 *
 * TEST INFRASTRUCTURE ONLY, like pk_oracle.c: only tests/,
 * __graft_entry__.smoke() and bench.py's CPU legs load it; it shares no code
 * with the CUDA library.
 *
 * The random numbers follow one counter-based definition that both sides
 * implement on their own:
 *   Philox4x64-10 (Salmon, Moraes, Dror & Shaw, "Parallel random numbers: as
 *   easy as 1, 2, 3", SC'11): a 4 x 64-bit counter and a 2 x 64-bit key; each
 *   of 10 rounds multiplies counter words 0 and 2 by the two round constants,
 *   mixes the high halves with the other words and the key, and bumps the key
 *   by the two Weyl constants.
 *   uniform(x) = ((x >> 40) + 1/2) 2^-24, strictly inside (0, 1).
 *   White noise (key = (seed, 0)): cells 4b .. 4b+3 (flat index, z fastest)
 *   take the four words of counter (b, 0, 0, 0); the pairs (w0, w1) and
 *   (w2, w3) give two Gaussians each by the Box-Muller transform,
 *   r = sqrt(-2 ln u1), (r cos 2 pi u2, r sin 2 pi u2).
 *   Objects (key = (seed, 1)): object i takes counter (i, 0, 0, 0); word 0
 *   picks its cell by inverse CDF (t = floor(w0 total / 2^64) against the
 *   exact integer cumulative cell weights), words 1..3 its offset inside the
 *   cell.
 *
 *   oracle_philox4x64   one Philox4x64-10 block.
 *   oracle_white_noise  the ng^3 white-noise grid.
 *   oracle_place        exactly n objects from integer cell weights: cell by
 *                       inverse CDF, uniform offset in the cell, z displaced
 *                       by f psi_z(cell) and wrapped into [0, L).
 */
#include <math.h>
#include <stdint.h>

static const uint64_t PHILOX_M0 = 0xD2E7470EE14C6C93ULL;
static const uint64_t PHILOX_M1 = 0xCA5A826395121157ULL;
static const uint64_t PHILOX_W0 = 0x9E3779B97F4A7C15ULL;
static const uint64_t PHILOX_W1 = 0xBB67AE8584CAA73BULL;

static void mulhilo64(uint64_t a, uint64_t b, uint64_t *hi, uint64_t *lo)
{
    unsigned __int128 p = (unsigned __int128)a * b;
    *hi = (uint64_t)(p >> 64);
    *lo = (uint64_t)p;
}

void oracle_philox4x64(const uint64_t *ctr, const uint64_t *key, uint64_t *out)
{
    uint64_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
    uint64_t k0 = key[0], k1 = key[1];
    for (int r = 0; r < 10; ++r) {
        uint64_t hi0, lo0, hi1, lo1;
        mulhilo64(PHILOX_M0, x0, &hi0, &lo0);
        mulhilo64(PHILOX_M1, x2, &hi1, &lo1);
        uint64_t y0 = hi1 ^ x1 ^ k0, y1 = lo1, y2 = hi0 ^ x3 ^ k1, y3 = lo0;
        x0 = y0;
        x1 = y1;
        x2 = y2;
        x3 = y3;
        k0 += PHILOX_W0;
        k1 += PHILOX_W1;
    }
    out[0] = x0;
    out[1] = x1;
    out[2] = x2;
    out[3] = x3;
}

static double uniform24(uint64_t x)
{
    return ((double)(x >> 40) + 0.5) * (1.0 / 16777216.0);
}

int oracle_white_noise(int ng, uint64_t seed, double *out)
{
    if (ng < 2 || (ng % 2) != 0 || !out) return 1;
    const int64_t ncell = (int64_t)ng * ng * ng;
    const uint64_t key[2] = {seed, 0};
    const double two_pi = 6.283185307179586476925286766559;
    for (int64_t b = 0; 4 * b < ncell; ++b) {
        const uint64_t ctr[4] = {(uint64_t)b, 0, 0, 0};
        uint64_t w[4];
        oracle_philox4x64(ctr, key, w);
        for (int pair = 0; pair < 2; ++pair) {
            const double u1 = uniform24(w[2 * pair]), u2 = uniform24(w[2 * pair + 1]);
            const double r = sqrt(-2.0 * log(u1));
            out[4 * b + 2 * pair] = r * cos(two_pi * u2);
            out[4 * b + 2 * pair + 1] = r * sin(two_pi * u2);
        }
    }
    return 0;
}

int oracle_place(const int64_t *excl, int ng, double L, const double *psi_z, double f_rsd, uint64_t seed,
                 int64_t n, double *pos)
{
    if (ng < 2 || !excl || n < 0 || (n > 0 && !pos)) return 1;
    const int64_t ncell = (int64_t)ng * ng * ng;
    const uint64_t total = (uint64_t)excl[ncell];
    if (n > 0 && total == 0) return 2;
    const uint64_t key[2] = {seed, 1};
    const double H = L / ng;
    for (int64_t i = 0; i < n; ++i) {
        const uint64_t ctr[4] = {(uint64_t)i, 0, 0, 0};
        uint64_t w[4];
        oracle_philox4x64(ctr, key, w);
        uint64_t t, lo;
        mulhilo64(w[0], total, &t, &lo);            /* t uniform in [0, total) */
        /* the cell c with excl[c] <= t < excl[c + 1] */
        int64_t a = 0, b = ncell;                    /* excl[a] <= t < excl[b] */
        while (b - a > 1) {
            const int64_t mid = a + (b - a) / 2;
            if ((uint64_t)excl[mid] <= t) a = mid;
            else b = mid;
        }
        const int64_t c = a;
        const int64_t ix = c / ((int64_t)ng * ng), iy = (c / ng) % ng, iz = c % ng;
        double z = ((double)iz + uniform24(w[3])) * H;
        if (psi_z) z += f_rsd * psi_z[c];
        z = z - L * floor(z / L);
        if (z >= L) z -= L;
        pos[3 * i + 0] = ((double)ix + uniform24(w[1])) * H;
        pos[3 * i + 1] = ((double)iy + uniform24(w[2])) * H;
        pos[3 * i + 2] = z;
    }
    return 0;
}
