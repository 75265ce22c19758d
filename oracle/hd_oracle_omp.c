/*
 * hd_oracle_omp.c -- TEST INFRASTRUCTURE: the oracle's sweep spread over the
 * host's cores, for the all-cores CPU baseline of the benchmark.  Only
 * tests/ and the benchmark's CPU-baseline leg use it.
 *
 * It is the same program as hd_oracle.c (included below, so every step of
 * the chain is the oracle's own code): per sweep the frame change of every
 * disk, the cell lists, then the four colours in the sweep's order.  Only
 * the loops change: the frame change runs over disks on all threads (each
 * disk's is independent), the cell lists are built sequentially, and the
 * active cells of one colour are shared out between threads (cells of one
 * colour are never neighbours and every draw is keyed by its cell, so the
 * order of the cells does not matter, Sec. II.B).  Trial counts are summed
 * per thread.  The chain is bit-identical to hdo_sweep's (tested).
 */
#include "hd_oracle.c"

#include <omp.h>

void hdo_sweep_omp(hdo_state *s, int64_t nsweeps, int threads)
{
    int m = s->m;
    if (threads < 1) threads = omp_get_max_threads();
    for (int64_t it = 0; it < nsweeps; ++it) {
        uint64_t sweep = s->sweep;
        double sx, sy;
        int64_t Sx, Sy;
        int perm[4];
        sweep_draws(s, sweep, &sx, &sy, &Sx, &Sy, perm);
        if (s->form == HDO_FP64) {
            double dsx = s->sx - sx, dsy = s->sy - sy;
#pragma omp parallel for num_threads(threads) schedule(static)
            for (int64_t i = 0; i < s->N; ++i) {
                frame_change_fp64(s, dsx, &s->cx[i], &s->ux[i]);
                frame_change_fp64(s, dsy, &s->cy[i], &s->uy[i]);
            }
            s->sx = sx;
            s->sy = sy;
        } else {
            int64_t dSx = s->Sx - Sx, dSy = s->Sy - Sy;
#pragma omp parallel for num_threads(threads) schedule(static)
            for (int64_t i = 0; i < s->N; ++i) {
                frame_change_fixed(s, dSx, &s->cx[i], &s->fx[i]);
                frame_change_fixed(s, dSy, &s->cy[i], &s->fy[i]);
            }
            s->Sx = Sx;
            s->Sy = Sy;
        }
        build_lists(s);
        uint64_t att = 0, acc = 0;
        for (int p = 0; p < 4; ++p) {
            int col = perm[p];
#pragma omp parallel for num_threads(threads) schedule(static) reduction(+ : att, acc)
            for (int ccy = (col >> 1); ccy < m; ccy += 2) {
                uint64_t a = 0, c = 0;
                for (int ccx = (col & 1); ccx < m; ccx += 2) update_cell(s, (uint32_t)sweep, ccx, ccy, &a, &c);
                att += a;
                acc += c;
            }
        }
        s->attempts += att;
        s->accepts += acc;
        s->sweep = sweep + 1;
    }
}
