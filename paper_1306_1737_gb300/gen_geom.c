/*
 * Geometry helpers for the synthetic input generator (workloads.py): random
 * sequential addition of points with a minimum separation, and a search for
 * close point pairs, both under periodic boundaries with a linked-cell list.
 * Input generation only: nothing here is part of the pair-interaction method.
 * Random numbers come from the caller (numpy PCG64), so results are seeded.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>

static inline double min_image1(double d, double L) { return d - L * nearbyint(d / L); }

/* Consume candidates cand[0..ncand) in order; accept one when no accepted
 * point lies within dmin (minimum image).  State: pts/npts (accepted points),
 * head[ncell] / next[nmax] linked cells of side >= dmin (nc[3] cells).
 * Stops when npts reaches nmax.  Returns the number of candidates consumed. */
int64_t gen_rsa_fill(const double* L, double dmin, const int* nc, int* head, int* next,
                     double* pts, int64_t* npts, int64_t nmax, const double* cand, int64_t ncand) {
    const double d2 = dmin * dmin;
    const double w[3] = {L[0] / nc[0], L[1] / nc[1], L[2] / nc[2]};
    int64_t k = 0;
    for (; k < ncand && *npts < nmax; ++k) {
        const double* c = cand + 3 * k;
        int ci[3];
        for (int a = 0; a < 3; ++a) {
            ci[a] = (int)(c[a] / w[a]);
            if (ci[a] >= nc[a]) ci[a] = nc[a] - 1;
            if (ci[a] < 0) ci[a] = 0;
        }
        int ok = 1;
        for (int ox = -1; ox <= 1 && ok; ++ox)
            for (int oy = -1; oy <= 1 && ok; ++oy)
                for (int oz = -1; oz <= 1 && ok; ++oz) {
                    const int gx = (ci[0] + ox + nc[0]) % nc[0];
                    const int gy = (ci[1] + oy + nc[1]) % nc[1];
                    const int gz = (ci[2] + oz + nc[2]) % nc[2];
                    for (int p = head[(gx * nc[1] + gy) * nc[2] + gz]; p >= 0; p = next[p]) {
                        const double dx = min_image1(pts[3 * p] - c[0], L[0]);
                        const double dy = min_image1(pts[3 * p + 1] - c[1], L[1]);
                        const double dz = min_image1(pts[3 * p + 2] - c[2], L[2]);
                        if (dx * dx + dy * dy + dz * dz < d2) { ok = 0; break; }
                    }
                }
        if (!ok) continue;
        const int64_t p = *npts;
        pts[3 * p] = c[0];
        pts[3 * p + 1] = c[1];
        pts[3 * p + 2] = c[2];
        const int cell = (ci[0] * nc[1] + ci[1]) * nc[2] + ci[2];
        next[p] = head[cell];
        head[cell] = (int)p;
        *npts = p + 1;
    }
    return k;
}

/* Pairs (i < j) of points closer than r (minimum image), cells of side >= r
 * (needs at least 3 cells per dimension).  Writes up to cap pairs; returns
 * the total number found. */
int64_t gen_close_pairs(const double* L, double r, int64_t n, const double* pts, int64_t cap,
                        int64_t* out_i, int64_t* out_j) {
    int nc[3];
    for (int a = 0; a < 3; ++a) {
        nc[a] = (int)floor(L[a] / r);
        if (nc[a] < 3) return -1;
    }
    const int64_t ncell = (int64_t)nc[0] * nc[1] * nc[2];
    int* head = (int*)malloc(sizeof(int) * ncell);
    int* next = (int*)malloc(sizeof(int) * (n > 0 ? n : 1));
    for (int64_t c = 0; c < ncell; ++c) head[c] = -1;
    const double w[3] = {L[0] / nc[0], L[1] / nc[1], L[2] / nc[2]};
    int* cellof = (int*)malloc(sizeof(int) * 3 * (n > 0 ? n : 1));
    for (int64_t p = n - 1; p >= 0; --p) {
        int ci[3];
        for (int a = 0; a < 3; ++a) {
            double x = pts[3 * p + a] - L[a] * floor(pts[3 * p + a] / L[a]);
            ci[a] = (int)(x / w[a]);
            if (ci[a] >= nc[a]) ci[a] = nc[a] - 1;
            cellof[3 * p + a] = ci[a];
        }
        const int cell = (ci[0] * nc[1] + ci[1]) * nc[2] + ci[2];
        next[p] = head[cell];
        head[cell] = (int)p;
    }
    int64_t found = 0;
    for (int64_t p = 0; p < n; ++p) {
        for (int ox = -1; ox <= 1; ++ox)
            for (int oy = -1; oy <= 1; ++oy)
                for (int oz = -1; oz <= 1; ++oz) {
                    const int gx = (cellof[3 * p] + ox + nc[0]) % nc[0];
                    const int gy = (cellof[3 * p + 1] + oy + nc[1]) % nc[1];
                    const int gz = (cellof[3 * p + 2] + oz + nc[2]) % nc[2];
                    for (int q = head[(gx * nc[1] + gy) * nc[2] + gz]; q >= 0; q = next[q]) {
                        if (q <= p) continue;
                        const double dx = min_image1(pts[3 * p] - pts[3 * q], L[0]);
                        const double dy = min_image1(pts[3 * p + 1] - pts[3 * q + 1], L[1]);
                        const double dz = min_image1(pts[3 * p + 2] - pts[3 * q + 2], L[2]);
                        if (dx * dx + dy * dy + dz * dz < r * r) {
                            if (found < cap) {
                                out_i[found] = p;
                                out_j[found] = q;
                            }
                            ++found;
                        }
                    }
                }
    }
    free(head);
    free(next);
    free(cellof);
    return found;
}
