/*
 * hd_oracle.c -- sequential CPU oracle for massively parallel local Monte
 * Carlo (MPMC) of hard disks, the checkerboard method of Engel et al.,
 * "Hard-disk equation of state" (arXiv:1211.1645), Sec. II.B, with the
 * static pressure estimator of Sec. II.C.1 (Eqs. 2-4) and the orientational
 * order of Sec. III (Eq. 8).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, obviously sequential
 * statement of what the GPU path computes.  Only the test-suite, the smoke
 * check and the benchmark's CPU-baseline leg may load it.  It shares no code,
 * header, table or constant generator with the CUDA library.
 *
 * Units: lengths are in units of the disk radius sigma, so a disk has radius 1
 * and two disks overlap when their centre distance is below 2.
 *
 * Two number forms follow the same chain:
 *   HDO_FP64  - IEEE double, every expression evaluated in the order written
 *               here; compile with -ffp-contract=off so no FMA is formed.
 *   HDO_FIXED - cell-relative integer coordinates in units of 2^-24 sigma,
 *               exact integer overlap test (d^2 < (2 sigma)^2 = 2^50).
 *
 * Parity notes (pinned by tests/test_oracle_*.py):
 *   philox4x32_10        pinned by published known-answer vectors
 *   chain (sweep)        pinned by the never-overlap invariant, the exact
 *                        two-disk separation law, the hard-disk virial series
 *                        and frame-change invariance of global positions
 *   histogram            pinned by brute-force pair enumeration from global
 *                        coordinates (exact in the fixed-point form)
 *   psi6                 pinned by hand-built hexagonal shells, rotation and
 *                        reflection covariance and brute-force neighbour search
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define HDO_FP64 0
#define HDO_FIXED 1
#define HDO_LATTICE_SQUARE 0
#define HDO_LATTICE_TRIANGULAR 1

#define HDO_OK 0
#define HDO_ERR_ARG 1
#define HDO_ERR_REACH 2
#define HDO_ERR_MEM 3

/* 2^24: fixed-point units per sigma */
#define FX_SCALE 16777216.0
#define HDO_PI 3.14159265358979323846
/* (2 sigma)^2 in fixed-point units squared: (2^25)^2 */
#define FX_DIAM2 ((int64_t)1 << 50)

/* ------------------------------------------------------------------------- */
/* Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11).  Ten rounds of the      */
/* 4x32 multiply-xor bijection; the two-word key is bumped by the Weyl        */
/* constants between rounds.                                                  */
/* ------------------------------------------------------------------------- */
void hdo_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)x0;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)x2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t y0 = hi1 ^ x1 ^ k0;
        uint32_t y1 = lo1;
        uint32_t y2 = hi0 ^ x3 ^ k1;
        uint32_t y3 = lo0;
        x0 = y0; x1 = y1; x2 = y2; x3 = y3;
    }
    out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

/* Integer in [0, n) from one 32-bit word: floor(word * n / 2^32). */
static uint32_t bounded(uint32_t word, uint32_t n)
{
    return (uint32_t)(((uint64_t)word * (uint64_t)n) >> 32);
}

/* Counter tags (fourth counter word) keep the draw streams disjoint. */
#define TAG_SWEEP 1u
#define TAG_SHUFFLE 2u
#define TAG_TRIAL 3u

/* ------------------------------------------------------------------------- */
/* State                                                                      */
/* ------------------------------------------------------------------------- */
typedef struct hdo_state {
    int64_t N;
    int m;            /* cells per side (even, >= 4) */
    int form;         /* HDO_FP64 / HDO_FIXED */
    int nt;           /* trial moves per occupied active cell per pass */
    double eta_in;    /* requested packing fraction */
    double L, w, w_below, delta; /* FP64 geometry, sigma units */
    int64_t W, LF, D; /* fixed-point cell side, box side, max step */
    uint32_t key[2];
    uint64_t sweep;   /* sweeps done so far */
    /* per-disk state, indexed by disk id */
    int32_t *cx, *cy;
    double *ux, *uy;   /* FP64 offsets inside the cell, in [0, w) */
    int32_t *fx, *fy;  /* fixed offsets inside the cell, in [0, W) */
    /* shift of the current cell frame */
    double sx, sy;
    int64_t Sx, Sy;
    /* cell lists of the current frame: ids ascending inside each cell */
    int64_t *cstart;   /* m*m + 1 */
    int64_t *cids;     /* N */
    uint64_t attempts, accepts;
    int max_occupancy;
} hdo_state;

static int wrap(int c, int m)
{
    c %= m;
    if (c < 0) c += m;
    return c;
}

/* Rebuild the cell lists: counting sort by cell, ids ascending in a cell. */
static void build_lists(hdo_state *s)
{
    int64_t ncell = (int64_t)s->m * s->m;
    memset(s->cstart, 0, sizeof(int64_t) * (size_t)(ncell + 1));
    for (int64_t i = 0; i < s->N; ++i)
        s->cstart[(int64_t)s->cy[i] * s->m + s->cx[i] + 1]++;
    for (int64_t c = 0; c < ncell; ++c) {
        int64_t occ = s->cstart[c + 1];
        if (occ > s->max_occupancy) s->max_occupancy = (int)occ;
        s->cstart[c + 1] += s->cstart[c];
    }
    int64_t *fill = (int64_t *)malloc(sizeof(int64_t) * (size_t)ncell);
    for (int64_t c = 0; c < ncell; ++c) fill[c] = s->cstart[c];
    for (int64_t i = 0; i < s->N; ++i) {
        int64_t c = (int64_t)s->cy[i] * s->m + s->cx[i];
        s->cids[fill[c]++] = i;
    }
    free(fill);
}

/* Place global coordinate t in [0, L) into cell index and offset (FP64). */
static void bin_fp64(const hdo_state *s, double t, int32_t *c_out, double *u_out)
{
    int c = (int)(t / s->w);
    if (c > s->m - 1) c = s->m - 1;
    if (c < 0) c = 0;
    double u = t - (double)c * s->w;
    if (u < 0.0 && c > 0) {
        c -= 1;
        u = t - (double)c * s->w;
    }
    if (u >= s->w && c < s->m - 1) {
        c += 1;
        u = t - (double)c * s->w;
    }
    if (u < 0.0) u = 0.0;
    if (u >= s->w) u = s->w_below;
    *c_out = c;
    *u_out = u;
}

/* Load global positions (sigma units, any real value, periodic) into the
 * state; the cell frame is reset to shift zero. */
int hdo_set_positions(hdo_state *s, const double *xy)
{
    s->sx = 0.0; s->sy = 0.0; s->Sx = 0; s->Sy = 0;
    for (int64_t i = 0; i < s->N; ++i) {
        double px = xy[2 * i], py = xy[2 * i + 1];
        if (s->form == HDO_FP64) {
            double tx = fmod(px, s->L), ty = fmod(py, s->L);
            if (tx < 0.0) tx += s->L;
            if (ty < 0.0) ty += s->L;
            if (tx >= s->L) tx = 0.0;
            if (ty >= s->L) ty = 0.0;
            bin_fp64(s, tx, &s->cx[i], &s->ux[i]);
            bin_fp64(s, ty, &s->cy[i], &s->uy[i]);
        } else {
            int64_t X = llround(px * FX_SCALE) % s->LF;
            int64_t Y = llround(py * FX_SCALE) % s->LF;
            if (X < 0) X += s->LF;
            if (Y < 0) Y += s->LF;
            s->cx[i] = (int32_t)(X / s->W);
            s->fx[i] = (int32_t)(X % s->W);
            s->cy[i] = (int32_t)(Y / s->W);
            s->fy[i] = (int32_t)(Y % s->W);
        }
    }
    s->max_occupancy = 0;
    build_lists(s);
    return HDO_OK;
}

/* Global positions of all disks (sigma units, in [0, L)), by disk id. */
void hdo_positions(const hdo_state *s, double *xy)
{
    for (int64_t i = 0; i < s->N; ++i) {
        if (s->form == HDO_FP64) {
            double X = ((double)s->cx[i] * s->w + s->ux[i]) + s->sx;
            double Y = ((double)s->cy[i] * s->w + s->uy[i]) + s->sy;
            if (X >= s->L) X -= s->L;
            if (Y >= s->L) Y -= s->L;
            xy[2 * i] = X;
            xy[2 * i + 1] = Y;
        } else {
            int64_t X = (int64_t)s->cx[i] * s->W + s->fx[i] + s->Sx;
            int64_t Y = (int64_t)s->cy[i] * s->W + s->fy[i] + s->Sy;
            if (X >= s->LF) X -= s->LF;
            if (Y >= s->LF) Y -= s->LF;
            xy[2 * i] = (double)X / FX_SCALE;
            xy[2 * i + 1] = (double)Y / FX_SCALE;
        }
    }
}

void hdo_destroy(hdo_state *s)
{
    if (!s) return;
    free(s->cx); free(s->cy); free(s->ux); free(s->uy);
    free(s->fx); free(s->fy); free(s->cstart); free(s->cids);
    free(s);
}

/*
 * Geometry (Sec. II.A): L = sqrt(N pi / eta) for unit radius.  Cells have
 * side w = L/m with m the largest even integer such that w >= cell_min
 * (cell_min >= 2 sigma, Sec. II.B).  The initial square lattice has
 * n = ceil(sqrt(N)) columns of spacing L/n; the "triangular" variant shifts
 * odd rows by half a spacing.
 */
hdo_state *hdo_create(int64_t N, double eta, double delta, uint64_t seed, int form,
                      int lattice, int nt, double cell_min, int *status)
{
    *status = HDO_ERR_ARG;
    if (N < 2 || !(eta > 0.0) || !(delta >= 0.0) || (form != HDO_FP64 && form != HDO_FIXED))
        return NULL;
    if (lattice != HDO_LATTICE_SQUARE && lattice != HDO_LATTICE_TRIANGULAR) return NULL;
    if (!(cell_min >= 2.0)) return NULL;
    double L = sqrt((double)N * HDO_PI / eta);
    int m = 2 * (int)floor(L / (2.0 * cell_min));
    if (m < 4) return NULL;
    if (!(L / (double)m < 8.0)) return NULL; /* cells hold at most 36 disks */
    int64_t n = (int64_t)ceil(sqrt((double)N));
    while (n * n < N) ++n;
    while ((n - 1) * (n - 1) >= N) --n;
    if (L / (double)n < 2.0) return NULL; /* lattice would overlap */

    hdo_state *s = (hdo_state *)calloc(1, sizeof(hdo_state));
    if (!s) { *status = HDO_ERR_MEM; return NULL; }
    s->N = N; s->m = m; s->form = form; s->eta_in = eta;
    s->L = L;
    s->w = L / (double)m;
    s->w_below = nextafter(s->w, 0.0);
    s->delta = delta;
    s->W = llround(s->w * FX_SCALE);
    s->LF = (int64_t)m * s->W;
    s->D = llround(delta * FX_SCALE);
    if (form == HDO_FIXED && (s->W >= ((int64_t)1 << 29) || 2 * s->D + 1 >= ((int64_t)1 << 32) || s->D >= s->W)) {
        free(s);
        return NULL;
    }
    if (form == HDO_FP64 && !(delta < s->w)) { free(s); return NULL; }
    s->key[0] = (uint32_t)(seed & 0xffffffffu);
    s->key[1] = (uint32_t)(seed >> 32);
    int64_t ncell = (int64_t)m * m;
    if (nt <= 0) nt = (int)((N + ncell - 1) / ncell);
    s->nt = nt;
    s->cx = (int32_t *)calloc((size_t)N, sizeof(int32_t));
    s->cy = (int32_t *)calloc((size_t)N, sizeof(int32_t));
    s->ux = (double *)calloc((size_t)N, sizeof(double));
    s->uy = (double *)calloc((size_t)N, sizeof(double));
    s->fx = (int32_t *)calloc((size_t)N, sizeof(int32_t));
    s->fy = (int32_t *)calloc((size_t)N, sizeof(int32_t));
    s->cstart = (int64_t *)calloc((size_t)(ncell + 1), sizeof(int64_t));
    s->cids = (int64_t *)calloc((size_t)N, sizeof(int64_t));
    if (!s->cx || !s->cy || !s->ux || !s->uy || !s->fx || !s->fy || !s->cstart || !s->cids) {
        hdo_destroy(s);
        *status = HDO_ERR_MEM;
        return NULL;
    }
    /* lattice: disk k sits in row k / n, column k % n */
    double *xy = (double *)malloc(sizeof(double) * 2 * (size_t)N);
    for (int64_t k = 0; k < N; ++k) {
        int64_t row = k / n, col = k % n;
        int64_t numx = 2 * col + 1 + ((lattice == HDO_LATTICE_TRIANGULAR && (row & 1)) ? 1 : 0);
        if (numx >= 2 * n) numx -= 2 * n;
        int64_t numy = 2 * row + 1;
        if (form == HDO_FP64) {
            xy[2 * k] = ((double)numx * s->L) / (double)(2 * n);
            xy[2 * k + 1] = ((double)numy * s->L) / (double)(2 * n);
        } else {
            xy[2 * k] = (double)((numx * s->LF) / (2 * n)) / FX_SCALE;
            xy[2 * k + 1] = (double)((numy * s->LF) / (2 * n)) / FX_SCALE;
        }
    }
    hdo_set_positions(s, xy);
    free(xy);
    *status = HDO_OK;
    return s;
}

/* Per-sweep draws: new frame shift and the order of the four colours. */
static void sweep_draws(const hdo_state *s, uint64_t sweep, double *sx, double *sy,
                        int64_t *Sx, int64_t *Sy, int perm[4])
{
    uint32_t ctr[4] = {(uint32_t)sweep, 0u, 0u, TAG_SWEEP};
    uint32_t a[4];
    hdo_philox4x32_10(ctr, s->key, a);
    *sx = ((double)a[0] * 0x1p-32) * s->w;
    *sy = ((double)a[1] * 0x1p-32) * s->w;
    *Sx = (int64_t)(((uint64_t)a[0] * (uint64_t)s->W) >> 32);
    *Sy = (int64_t)(((uint64_t)a[1] * (uint64_t)s->W) >> 32);
    /* rank r in [0, 24) decoded as a permutation in lexicographic order */
    uint32_t r = bounded(a[2], 24u);
    int avail[4] = {0, 1, 2, 3};
    int navail = 4;
    uint32_t radix[3] = {6u, 2u, 1u};
    for (int p = 0; p < 3; ++p) {
        uint32_t d = r / radix[p];
        r = r % radix[p];
        perm[p] = avail[d];
        for (int q = (int)d; q < navail - 1; ++q) avail[q] = avail[q + 1];
        navail--;
    }
    perm[3] = avail[0];
}

/* Move one coordinate of one disk into the new frame (FP64). */
static void frame_change_fp64(const hdo_state *s, double d, int32_t *c, double *u)
{
    double t = *u + d;
    int cc = *c;
    if (t < 0.0) {
        double v = t + s->w;
        if (v < s->w) {
            cc -= 1;
            t = v;
        } else {
            t = 0.0;
        }
    } else if (t >= s->w) {
        t = t - s->w;
        cc += 1;
        if (t >= s->w) t = s->w_below;
    }
    *c = wrap(cc, s->m);
    *u = t;
}

static void frame_change_fixed(const hdo_state *s, int64_t d, int32_t *c, int32_t *u)
{
    int64_t t = (int64_t)(*u) + d;
    int cc = *c;
    if (t < 0) {
        t += s->W;
        cc -= 1;
    } else if (t >= s->W) {
        t -= s->W;
        cc += 1;
    }
    *c = wrap(cc, s->m);
    *u = (int32_t)t;
}

/* Offsets of the three cells of a stencil row or column, FP64 / fixed. */
static double cell_off_fp64(const hdo_state *s, int o)
{
    return o < 0 ? -s->w : (o > 0 ? s->w : 0.0);
}

/* One active cell: shuffle its occupants, then nt serial trial moves; the
 * trials are added to *attempts, the accepted ones to *accepts. */
static void update_cell(hdo_state *s, uint32_t sweep32, int ccx, int ccy, uint64_t *attempts, uint64_t *accepts)
{
    int m = s->m;
    int64_t c = (int64_t)ccy * m + ccx;
    int64_t n = s->cstart[c + 1] - s->cstart[c];
    if (n == 0) return;
    const int64_t *ids = &s->cids[s->cstart[c]];

    /* Fisher-Yates shuffle of the occupants (ascending ids).  The swap words
     * come from the shuffle stream; in the fixed-point form, whose step uses
     * only two words of a trial block, the first two swap words are the
     * unused words 2 and 3 of trial 0's block and the shuffle stream supplies
     * the rest. */
    int64_t perm[64];
    uint32_t words[72];
    for (int64_t k = 0; k < n; ++k) perm[k] = k;
    uint32_t lead = 0;
    if (s->form == HDO_FIXED && n > 1) {
        uint32_t ctr[4] = {sweep32, 0u, (uint32_t)c, TAG_TRIAL};
        uint32_t a[4];
        hdo_philox4x32_10(ctr, s->key, a);
        words[0] = a[2];
        words[1] = a[3];
        lead = 2;
    }
    for (uint32_t blk = 0; lead + 4 * blk < (uint32_t)(n - 1); ++blk) {
        uint32_t ctr[4] = {sweep32, blk, (uint32_t)c, TAG_SHUFFLE};
        hdo_philox4x32_10(ctr, s->key, &words[lead + 4 * blk]);
    }
    for (int64_t k = n - 1; k >= 1; --k) {
        uint32_t j = bounded(words[n - 1 - k], (uint32_t)(k + 1));
        int64_t tmp = perm[k];
        perm[k] = perm[j];
        perm[j] = tmp;
    }

    for (int t = 0; t < s->nt; ++t) {
        uint32_t ctr[4] = {sweep32, (uint32_t)t, (uint32_t)c, TAG_TRIAL};
        uint32_t a[4];
        hdo_philox4x32_10(ctr, s->key, a);
        int64_t i = ids[perm[t % n]];
        (*attempts)++;
        int overlap = 0;
        if (s->form == HDO_FP64) {
            uint64_t kx = ((uint64_t)(a[0] >> 6) << 27) | (uint64_t)(a[1] >> 5);
            uint64_t ky = ((uint64_t)(a[2] >> 6) << 27) | (uint64_t)(a[3] >> 5);
            int64_t vx = (int64_t)(2 * kx + 1) - ((int64_t)1 << 53);
            int64_t vy = (int64_t)(2 * ky + 1) - ((int64_t)1 << 53);
            double dx = (s->delta * (double)vx) * 0x1p-53;
            double dy = (s->delta * (double)vy) * 0x1p-53;
            double nx = s->ux[i] + dx;
            double ny = s->uy[i] + dy;
            if (!(nx >= 0.0 && nx < s->w && ny >= 0.0 && ny < s->w)) continue;
            for (int oy = -1; oy <= 1 && !overlap; ++oy) {
                for (int ox = -1; ox <= 1 && !overlap; ++ox) {
                    int64_t nc = (int64_t)wrap(ccy + oy, m) * m + wrap(ccx + ox, m);
                    double offx = cell_off_fp64(s, ox), offy = cell_off_fp64(s, oy);
                    for (int64_t q = s->cstart[nc]; q < s->cstart[nc + 1]; ++q) {
                        int64_t j = s->cids[q];
                        if (j == i) continue;
                        double rx = (s->ux[j] + offx) - nx;
                        double ry = (s->uy[j] + offy) - ny;
                        double d2 = rx * rx + ry * ry;
                        if (d2 < 4.0) { overlap = 1; break; }
                    }
                }
            }
            if (!overlap) {
                s->ux[i] = nx;
                s->uy[i] = ny;
                (*accepts)++;
            }
        } else {
            int64_t dX = (int64_t)bounded(a[0], (uint32_t)(2 * s->D + 1)) - s->D;
            int64_t dY = (int64_t)bounded(a[1], (uint32_t)(2 * s->D + 1)) - s->D;
            int64_t nx = (int64_t)s->fx[i] + dX;
            int64_t ny = (int64_t)s->fy[i] + dY;
            if (!(nx >= 0 && nx < s->W && ny >= 0 && ny < s->W)) continue;
            for (int oy = -1; oy <= 1 && !overlap; ++oy) {
                for (int ox = -1; ox <= 1 && !overlap; ++ox) {
                    int64_t nc = (int64_t)wrap(ccy + oy, m) * m + wrap(ccx + ox, m);
                    for (int64_t q = s->cstart[nc]; q < s->cstart[nc + 1]; ++q) {
                        int64_t j = s->cids[q];
                        if (j == i) continue;
                        int64_t rx = ((int64_t)s->fx[j] + ox * s->W) - nx;
                        int64_t ry = ((int64_t)s->fy[j] + oy * s->W) - ny;
                        if (rx * rx + ry * ry < FX_DIAM2) { overlap = 1; break; }
                    }
                }
            }
            if (!overlap) {
                s->fx[i] = (int32_t)nx;
                s->fy[i] = (int32_t)ny;
                (*accepts)++;
            }
        }
    }
}

/*
 * n checkerboard sweeps (Sec. II.B).  Each sweep: draw a new random grid
 * shift and move every disk into the shifted frame, rebuild the cell lists,
 * then visit the four colours in a random order; the cells of one colour are
 * independent, so visiting them in row-major order is the sequential
 * statement of the parallel pass.
 */
void hdo_sweep(hdo_state *s, int64_t nsweeps)
{
    int m = s->m;
    for (int64_t it = 0; it < nsweeps; ++it) {
        uint64_t sweep = s->sweep;
        double sx, sy;
        int64_t Sx, Sy;
        int perm[4];
        sweep_draws(s, sweep, &sx, &sy, &Sx, &Sy, perm);
        if (s->form == HDO_FP64) {
            double dsx = s->sx - sx, dsy = s->sy - sy;
            for (int64_t i = 0; i < s->N; ++i) {
                frame_change_fp64(s, dsx, &s->cx[i], &s->ux[i]);
                frame_change_fp64(s, dsy, &s->cy[i], &s->uy[i]);
            }
            s->sx = sx;
            s->sy = sy;
        } else {
            int64_t dSx = s->Sx - Sx, dSy = s->Sy - Sy;
            for (int64_t i = 0; i < s->N; ++i) {
                frame_change_fixed(s, dSx, &s->cx[i], &s->fx[i]);
                frame_change_fixed(s, dSy, &s->cy[i], &s->fy[i]);
            }
            s->Sx = Sx;
            s->Sy = Sy;
        }
        build_lists(s);
        for (int p = 0; p < 4; ++p) {
            int col = perm[p];
            for (int ccy = (col >> 1); ccy < m; ccy += 2)
                for (int ccx = (col & 1); ccx < m; ccx += 2)
                    update_cell(s, (uint32_t)sweep, ccx, ccy, &s->attempts, &s->accepts);
        }
        s->sweep = sweep + 1;
    }
}

/* ------------------------------------------------------------------------- */
/* Measurements                                                               */
/* ------------------------------------------------------------------------- */

/* Relative vector from disk i to disk j whose cell lies (dcx, dcy) cells
 * away, expressed in i's cell frame. */
static void rel_fp64(const hdo_state *s, int64_t i, int64_t j, int dcx, int dcy, double *rx, double *ry)
{
    *rx = (s->ux[j] + (double)dcx * s->w) - s->ux[i];
    *ry = (s->uy[j] + (double)dcy * s->w) - s->uy[i];
}

static void rel_fixed(const hdo_state *s, int64_t i, int64_t j, int dcx, int dcy, int64_t *rx, int64_t *ry)
{
    *rx = ((int64_t)s->fx[j] + (int64_t)dcx * s->W) - s->fx[i];
    *ry = ((int64_t)s->fy[j] + (int64_t)dcy * s->W) - s->fy[i];
}

/* Minimum-image cell difference of j relative to i, in (-m/2, m/2]. */
static int cell_diff(int a, int b, int m)
{
    int d = b - a;
    while (d > m / 2) d -= m;
    while (d <= -m / 2) d += m;
    return d;
}

/*
 * Contact-shell pair histogram (Eq. 2 numerator): counts of unordered pairs
 * whose centre distance r lies in [2 + k dr, 2 + (k+1) dr), k = 0..K-1.  The
 * pair vector is taken in the frame of the lower disk id.  FP64: bin edges
 * (2 + k dr)^2 compared with r^2.  Fixed point: dr is rounded to the 2^-24
 * grid and the comparison is exact in integers.  brute != 0 enumerates all
 * pairs instead of the cell stencil.
 */
int hdo_histogram(const hdo_state *s, int K, double dr, int brute, uint64_t *counts)
{
    if (K <= 0 || !(dr > 0.0)) return HDO_ERR_ARG;
    int m = s->m;
    for (int k = 0; k < K; ++k) counts[k] = 0;
    double *E = (double *)malloc(sizeof(double) * (size_t)(K + 1));
    int64_t *EF = (int64_t *)malloc(sizeof(int64_t) * (size_t)(K + 1));
    int64_t DR = llround(dr * FX_SCALE);
    for (int k = 0; k <= K; ++k) {
        double e = 2.0 + (double)k * dr;
        E[k] = e * e;
        int64_t ef = ((int64_t)1 << 25) + (int64_t)k * DR;
        EF[k] = ef * ef;
    }
    int R;
    if (s->form == HDO_FP64) R = (int)floor((2.0 + (double)K * dr) / s->w) + 1;
    else R = (int)((((int64_t)1 << 25) + (int64_t)K * DR) / s->W) + 1;
    if (2 * R + 1 > m) { free(E); free(EF); return HDO_ERR_REACH; }

    for (int64_t i = 0; i < s->N; ++i) {
        /* candidate partners: either every disk, or the (2R+1)^2 cell stencil */
        int ncand_cells = brute ? 1 : (2 * R + 1) * (2 * R + 1);
        for (int cidx = 0; cidx < ncand_cells; ++cidx) {
            int64_t jlo, jhi;
            int sdx = 0, sdy = 0;
            if (brute) {
                jlo = 0; jhi = s->N;
            } else {
                sdx = cidx % (2 * R + 1) - R;
                sdy = cidx / (2 * R + 1) - R;
                int64_t nc = (int64_t)wrap(s->cy[i] + sdy, m) * m + wrap(s->cx[i] + sdx, m);
                jlo = s->cstart[nc]; jhi = s->cstart[nc + 1];
            }
            for (int64_t q = jlo; q < jhi; ++q) {
                int64_t j = brute ? q : s->cids[q];
                if (j <= i) continue; /* each unordered pair once, seen from the lower id */
                int ex = sdx, ey = sdy;
                if (brute) {
                    ex = cell_diff(s->cx[i], s->cx[j], m);
                    ey = cell_diff(s->cy[i], s->cy[j], m);
                    if (ex < -R || ex > R || ey < -R || ey > R) continue;
                }
                int bin = -1;
                if (s->form == HDO_FP64) {
                    double rx, ry;
                    rel_fp64(s, i, j, ex, ey, &rx, &ry);
                    double r2 = rx * rx + ry * ry;
                    for (int k = 0; k < K; ++k)
                        if (r2 >= E[k] && r2 < E[k + 1]) { bin = k; break; }
                } else {
                    int64_t rx, ry;
                    rel_fixed(s, i, j, ex, ey, &rx, &ry);
                    int64_t r2 = rx * rx + ry * ry;
                    for (int k = 0; k < K; ++k)
                        if (r2 >= EF[k] && r2 < EF[k + 1]) { bin = k; break; }
                }
                if (bin >= 0) counts[bin]++;
            }
        }
    }
    free(E);
    free(EF);
    return HDO_OK;
}

/* Six nearest neighbours kept sorted by (r^2, id).  The FP64 form keys on
 * the double r^2; the fixed form on the exact integer r^2 (128-bit, so that a
 * brute-force scan across the whole box cannot overflow). */
typedef __int128 i128;
typedef struct { double d2; i128 d2i; int64_t id; int dcx, dcy; } nbr_t;

static int nbr_less(int form, const nbr_t *a, const nbr_t *b)
{
    if (form == HDO_FP64)
        return a->d2 < b->d2 || (a->d2 == b->d2 && a->id < b->id);
    return a->d2i < b->d2i || (a->d2i == b->d2i && a->id < b->id);
}

static void nbr_insert(int form, nbr_t *best, int *nb, const nbr_t *cand)
{
    if (*nb == 6 && !nbr_less(form, cand, &best[5])) return;
    int p = (*nb < 6) ? (*nb)++ : 5;
    while (p > 0 && nbr_less(form, cand, &best[p - 1])) {
        best[p] = best[p - 1];
        --p;
    }
    best[p] = *cand;
}

static void make_cand(const hdo_state *s, int64_t i, int64_t j, int dcx, int dcy, nbr_t *c)
{
    c->id = j; c->dcx = dcx; c->dcy = dcy;
    c->d2 = 0.0; c->d2i = 0;
    if (s->form == HDO_FP64) {
        double rx, ry;
        rel_fp64(s, i, j, dcx, dcy, &rx, &ry);
        c->d2 = rx * rx + ry * ry;
    } else {
        i128 rx = (i128)s->fx[j] + (i128)dcx * s->W - s->fx[i];
        i128 ry = (i128)s->fy[j] + (i128)dcy * s->W - s->fy[i];
        c->d2i = rx * rx + ry * ry;
    }
}

/*
 * Local bond-orientational order (Eq. 8): psi_j = (1/6) sum over the six
 * nearest neighbours k of exp(6 i phi_jk), phi measured from the +x axis on
 * the minimum-image vector.  exp(6 i phi) is evaluated as z^6 / |z|^6 with
 * z = rx + i ry, so no trigonometric function enters.  Neighbours are summed
 * in ascending (r^2, id).  The FP64 form computes in double; the fixed form
 * takes the exact integer vector, scales it by 2^-24 into float and computes
 * in float.  The global Psi_6 = (1/N) sum_j psi_j is formed from this field
 * by the Python layer (an exactly rounded sum, then one division by N).
 * brute != 0 scans all disks instead of expanding cell rings.
 */
int hdo_psi6(const hdo_state *s, int brute, double *local)
{
    int m = s->m;
    if (s->N < 7) return HDO_ERR_REACH;
    for (int64_t i = 0; i < s->N; ++i) {
        nbr_t best[6], cand;
        int nb = 0;
        if (brute) {
            for (int64_t j = 0; j < s->N; ++j) {
                if (j == i) continue;
                make_cand(s, i, j, cell_diff(s->cx[i], s->cx[j], m), cell_diff(s->cy[i], s->cy[j], m), &cand);
                nbr_insert(s->form, best, &nb, &cand);
            }
        } else {
            int R = 2;
            for (;;) {
                if (2 * R + 1 > m) return HDO_ERR_REACH;
                nb = 0;
                for (int dcy = -R; dcy <= R; ++dcy) {
                    for (int dcx = -R; dcx <= R; ++dcx) {
                        int64_t nc = (int64_t)wrap(s->cy[i] + dcy, m) * m + wrap(s->cx[i] + dcx, m);
                        for (int64_t q = s->cstart[nc]; q < s->cstart[nc + 1]; ++q) {
                            int64_t j = s->cids[q];
                            if (j == i) continue;
                            make_cand(s, i, j, dcx, dcy, &cand);
                            nbr_insert(s->form, best, &nb, &cand);
                        }
                    }
                }
                /* the ring search is certain once the sixth neighbour is
                 * strictly closer than the nearest point outside the stencil */
                int ok = 0;
                if (nb == 6) {
                    if (s->form == HDO_FP64) {
                        double c = s->ux[i] + (double)R * s->w;
                        double c2 = (double)(R + 1) * s->w - s->ux[i];
                        double c3 = s->uy[i] + (double)R * s->w;
                        double c4 = (double)(R + 1) * s->w - s->uy[i];
                        if (c2 < c) c = c2;
                        if (c3 < c) c = c3;
                        if (c4 < c) c = c4;
                        ok = best[5].d2 < c * c;
                    } else {
                        i128 c = (i128)s->fx[i] + (i128)R * s->W;
                        i128 c2 = (i128)(R + 1) * s->W - s->fx[i];
                        i128 c3 = (i128)s->fy[i] + (i128)R * s->W;
                        i128 c4 = (i128)(R + 1) * s->W - s->fy[i];
                        if (c2 < c) c = c2;
                        if (c3 < c) c = c3;
                        if (c4 < c) c = c4;
                        ok = best[5].d2i < c * c;
                    }
                }
                if (ok) break;
                ++R;
            }
        }
        if (nb < 6) return HDO_ERR_REACH;
        double pre, pim;
        if (s->form == HDO_FP64) {
            double sr = 0.0, si = 0.0;
            for (int k = 0; k < 6; ++k) {
                double x, y;
                rel_fp64(s, i, best[k].id, best[k].dcx, best[k].dcy, &x, &y);
                double xx = x * x, yy = y * y;
                double r2 = xx + yy;
                double c2 = xx - yy, s2 = (x * y) * 2.0;
                double c4 = c2 * c2 - s2 * s2, s4 = (c2 * s2) * 2.0;
                double c6 = c4 * c2 - s4 * s2, s6 = c4 * s2 + s4 * c2;
                double r6 = (r2 * r2) * r2;
                sr += c6 / r6;
                si += s6 / r6;
            }
            pre = sr / 6.0;
            pim = si / 6.0;
        } else {
            float sr = 0.0f, si = 0.0f;
            for (int k = 0; k < 6; ++k) {
                int64_t ix, iy;
                rel_fixed(s, i, best[k].id, best[k].dcx, best[k].dcy, &ix, &iy);
                float x = (float)ix * 0x1p-24f, y = (float)iy * 0x1p-24f;
                float xx = x * x, yy = y * y;
                float r2 = xx + yy;
                float c2 = xx - yy, s2 = (x * y) * 2.0f;
                float c4 = c2 * c2 - s2 * s2, s4 = (c2 * s2) * 2.0f;
                float c6 = c4 * c2 - s4 * s2, s6 = c4 * s2 + s4 * c2;
                float r6 = (r2 * r2) * r2;
                sr += c6 / r6;
                si += s6 / r6;
            }
            pre = (double)(sr / 6.0f);
            pim = (double)(si / 6.0f);
        }
        local[2 * i] = pre;
        local[2 * i + 1] = pim;
    }
    return HDO_OK;
}

/* ------------------------------------------------------------------------- */
/* Accessors                                                                  */
/* ------------------------------------------------------------------------- */
void hdo_stats(const hdo_state *s, uint64_t *attempts, uint64_t *accepts)
{
    *attempts = s->attempts;
    *accepts = s->accepts;
}

/* geom[0..9] = L, w, delta, m, W, LF, D, nt, max_occupancy, sweeps */
void hdo_geometry(const hdo_state *s, double *geom)
{
    geom[0] = s->form == HDO_FP64 ? s->L : (double)s->LF / FX_SCALE;
    geom[1] = s->form == HDO_FP64 ? s->w : (double)s->W / FX_SCALE;
    geom[2] = s->form == HDO_FP64 ? s->delta : (double)s->D / FX_SCALE;
    geom[3] = (double)s->m;
    geom[4] = (double)s->W;
    geom[5] = (double)s->LF;
    geom[6] = (double)s->D;
    geom[7] = (double)s->nt;
    geom[8] = (double)s->max_occupancy;
    geom[9] = (double)s->sweep;
}

/* Raw per-disk frame state, for tests: cell indices and offsets (sigma). */
void hdo_frame(const hdo_state *s, int32_t *cell_xy, double *off_xy, double *shift)
{
    for (int64_t i = 0; i < s->N; ++i) {
        cell_xy[2 * i] = s->cx[i];
        cell_xy[2 * i + 1] = s->cy[i];
        if (s->form == HDO_FP64) {
            off_xy[2 * i] = s->ux[i];
            off_xy[2 * i + 1] = s->uy[i];
        } else {
            off_xy[2 * i] = (double)s->fx[i] / FX_SCALE;
            off_xy[2 * i + 1] = (double)s->fy[i] / FX_SCALE;
        }
    }
    shift[0] = s->form == HDO_FP64 ? s->sx : (double)s->Sx / FX_SCALE;
    shift[1] = s->form == HDO_FP64 ? s->sy : (double)s->Sy / FX_SCALE;
}
