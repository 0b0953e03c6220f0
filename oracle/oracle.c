/*
 * FP64 CPU oracle for the cluster-pair non-bonded method of Pall & Hess,
 * "A flexible algorithm for calculating pair interactions on SIMD
 * architectures".
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may call, link or
 * load this file; only the tests, the smoke check and the benchmark's CPU
 * baseline leg use it.  It shares no code with the CUDA library.
 *
 * Everything here is plain and slow on purpose:
 *   - or_forces_brute: the O(N^2) minimum-image double loop over all particle
 *     pairs (Sec. 1 and Sec. 3.2, Eqs. for the LJ and Coulomb forces).
 *   - or_grid: the spatial clustering of Sec. 2.3 (x/y grid of spacing
 *     (max(M,N)/rho)^(1/3), columns sorted on z, consecutive groups of C,
 *     dummy padding of the last cluster, bounding boxes).
 *   - or_pairlist: the cluster-pair search of Sec. 2.3 / Fig. 3 evaluated by
 *     brute force over every cluster pair and every periodic shift, plus the
 *     exclusion bitmask of Sec. 2.4.
 *   - or_prune: the particle-pair distance pruning of Sec. 2.3.
 *   - or_pair: one pair interaction (Sec. 3.2).
 *
 * Floating point: FP64 everywhere except where a floating-point value decides
 * an integer (the grid cell of a particle, the z order, the wrap into the
 * box): there the decision is taken in FP32, the precision of the inputs and
 * of the kernels, with every operation rounded separately (compile with
 * -ffp-contract=off).
 *
 * Parity status of each function is stated beside it.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_ELEC_RF 0
#define OR_ELEC_EWALD 1

#define OR_COMB_LB 0        /* Lorentz-Berthelot: sigma arithmetic, eps geometric */
#define OR_COMB_GEOM 1      /* geometric on C6 and C12 */

/* Coulomb prefactor 1/(4 pi eps0) in kJ mol^-1 nm e^-2; the paper writes the
 * force with 1/(4 pi eps0) (Sec. 3.2) without a numerical value. */
#define OR_FCOUL 138.935458

typedef struct {
    int elec;        /* OR_ELEC_RF or OR_ELEC_EWALD */
    int comb;        /* OR_COMB_LB or OR_COMB_GEOM */
    double rc;       /* interaction cut-off (nm), LJ and Coulomb */
    double eps_rf;   /* reaction-field dielectric constant; <= 0 means infinity */
    double beta;     /* Ewald splitting parameter (nm^-1) */
} or_params;

int or_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ------------------------------------------------------------------------ */
/* Pair interaction (Sec. 3.2).
 *
 * Lennard-Jones: F = e_ij (12 C12 / r^13 - 6 C6 / r^7) r_hat,
 *                V = e_ij (C12 / r^12 - C6 / r^6)   (plain cut-off).
 * Coulomb:       F = f q_i q_j (e_ij / r^2 + g(r)) r_hat
 *   reaction field g(r) = -2 k r with k = (eps_rf - 1) / ((2 eps_rf + 1) rc^3)
 *     (eps_r = 1; eps_rf -> infinity gives k = 1/(2 rc^3)),
 *     V = f q_i q_j (e_ij / r + k r^2 - c_rf), c_rf = 1/rc + k rc^2, so that
 *     V(rc) = 0 for a non-excluded pair;
 *   Ewald real space g(r) = d/dr [erf(beta r) / r], i.e.
 *     F = f q_i q_j (e_ij - erf(beta r) + (2 beta r / sqrt(pi)) exp(-beta^2 r^2)) / r^2,
 *     V = f q_i q_j (e_ij - erf(beta r)) / r.
 * e_ij = 1 for a normal pair, 0 for a force-field-excluded pair: the LJ and
 * the plain Coulomb term vanish while the correction g(r) stays (Sec. 2.4).
 *
 * Outputs the scalar F/r (so the force vector on i is fscal * r_vec with
 * r_vec = x_i - x_j) and the two energies.  Pairs with r >= rc give zero.
 * Parity: pinned (LJ minimum, RF zero at rc, Ewald against an independent
 * erfc and the beta -> 0 limit, exclusion difference = plain Coulomb).
 */
void or_pair(const or_params* p, double r, double qq, double c6, double c12, int excluded,
             double* fscal, double* vlj, double* vc) {
    *fscal = 0.0; *vlj = 0.0; *vc = 0.0;
    if (!(r < p->rc)) return;
    const double e = excluded ? 0.0 : 1.0;
    const double rinv = 1.0 / r;
    const double rinv2 = rinv * rinv;
    const double rinv6 = rinv2 * rinv2 * rinv2;
    /* LJ */
    const double flj = e * (12.0 * c12 * rinv6 * rinv6 - 6.0 * c6 * rinv6);  /* = F_LJ * r */
    *vlj = e * (c12 * rinv6 * rinv6 - c6 * rinv6);
    double fc, vcc;
    if (p->elec == OR_ELEC_RF) {
        double k;
        if (p->eps_rf <= 0.0 || isinf(p->eps_rf))
            k = 1.0 / (2.0 * p->rc * p->rc * p->rc);
        else
            k = (p->eps_rf - 1.0) / ((2.0 * p->eps_rf + 1.0) * p->rc * p->rc * p->rc);
        const double crf = 1.0 / p->rc + k * p->rc * p->rc;
        /* F * r = f qq (e / r - 2 k r^2) */
        fc = OR_FCOUL * qq * (e * rinv - 2.0 * k * r * r);
        vcc = OR_FCOUL * qq * (e * rinv + k * r * r - crf);
    } else {
        const double br = p->beta * r;
        const double erfv = erf(br);
        const double gauss = 2.0 * br / sqrt(M_PI) * exp(-br * br);
        /* F * r = f qq (e - erf(br) + gauss) / r */
        fc = OR_FCOUL * qq * (e - erfv + gauss) * rinv;
        vcc = OR_FCOUL * qq * (e - erfv) * rinv;
    }
    *fscal = (flj + fc) * rinv2;   /* (F * r) / r^2 = F / r */
    *vc = vcc;
}

/* LJ pair parameters from per-type sigma/epsilon (Sec. 3.2: combination
 * rules, geometric or Lorentz-Berthelot).  C6 = 4 eps sigma^6,
 * C12 = 4 eps sigma^12. */
void or_lj_pair_params(int comb, double si, double ei, double sj, double ej,
                       double* c6, double* c12) {
    if (comb == OR_COMB_LB) {
        const double s = 0.5 * (si + sj);
        const double e = sqrt(ei * ej);
        const double s6 = s * s * s * s * s * s;
        *c6 = 4.0 * e * s6;
        *c12 = 4.0 * e * s6 * s6;
    } else {
        const double si6 = si * si * si * si * si * si;
        const double sj6 = sj * sj * sj * sj * sj * sj;
        const double c6i = 4.0 * ei * si6, c12i = 4.0 * ei * si6 * si6;
        const double c6j = 4.0 * ej * sj6, c12j = 4.0 * ej * sj6 * sj6;
        *c6 = sqrt(c6i * c6j);
        *c12 = sqrt(c12i * c12j);
    }
}

static int is_excluded(const int* excl_off, const int* excl_idx, int i, int j) {
    if (!excl_off) return 0;
    for (int k = excl_off[i]; k < excl_off[i + 1]; ++k)
        if (excl_idx[k] == j) return 1;
    return 0;
}

/* Minimum-image displacement x_i - x_j (FP64) for a rectangular box. */
static void min_image(const double L[3], const double xi[3], const double xj[3], double d[3]) {
    for (int k = 0; k < 3; ++k) {
        double v = xi[k] - xj[k];
        v -= L[k] * nearbyint(v / L[k]);
        d[k] = v;
    }
}

/* ------------------------------------------------------------------------ */
/* Tier A: brute-force forces, energies and virial.
 *
 * For every ordered pair (i, j), i != j, with minimum-image displacement
 * r_ij = x_i - x_j (valid because rc < L/2), the force on i from j is the
 * pair force above.  Energies count each unordered pair once (Newton's third
 * law, Sec. 2.3) and the virial is W = sum_{i<j} r_ij (x) F_ij.
 *
 * xyz: [n][3] in any periodic image; box: edge lengths (the callers pass
 * the FP32 inputs promoted to FP64; finite-difference checks pass FP64); sel: if
 * n_sel > 0, forces are computed only for atoms sel[0..n_sel) (each against
 * all n atoms) and energies/virial are not produced.
 * f: [n_sel or n][3]; e: [2] (LJ, Coulomb); vir: [9] row-major W[a][b].
 * Returns 0, or -1 when rc >= L/2.
 * Parity: pinned (Newton, finite-difference gradient, virial against an
 * affine-deformation derivative, translation invariance, pair counts).
 */
int or_forces_brute(int n, const double* xyz, const float* q, const int* type,
                    int ntypes, const double* sigma, const double* eps,
                    const int* excl_off, const int* excl_idx, const double* box,
                    const or_params* p, int n_sel, const int* sel,
                    double* f, double* e, double* vir) {
    double L[3] = {box[0], box[1], box[2]};
    for (int k = 0; k < 3; ++k)
        if (!(p->rc < 0.5 * L[k])) return -1;
    double* c6t = (double*)malloc(sizeof(double) * ntypes * ntypes);
    double* c12t = (double*)malloc(sizeof(double) * ntypes * ntypes);
    for (int a = 0; a < ntypes; ++a)
        for (int b = 0; b < ntypes; ++b)
            or_lj_pair_params(p->comb, sigma[a], eps[a], sigma[b], eps[b],
                              &c6t[a * ntypes + b], &c12t[a * ntypes + b]);
    const int full = (n_sel <= 0);
    const int ni = full ? n : n_sel;
    double elj = 0.0, ec = 0.0;
    double w[9] = {0};
#pragma omp parallel for schedule(dynamic, 16) reduction(+ : elj, ec) reduction(+ : w[:9])
    for (int ii = 0; ii < ni; ++ii) {
        const int i = full ? ii : sel[ii];
        const double xi[3] = {xyz[3 * i], xyz[3 * i + 1], xyz[3 * i + 2]};
        double fi[3] = {0, 0, 0};
        for (int j = 0; j < n; ++j) {
            if (j == i) continue;
            const double xj[3] = {xyz[3 * j], xyz[3 * j + 1], xyz[3 * j + 2]};
            double d[3];
            min_image(L, xi, xj, d);
            const double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
            if (!(r2 < p->rc * p->rc)) continue;
            const double r = sqrt(r2);
            const int ex = is_excluded(excl_off, excl_idx, i, j);
            const int tt = type[i] * ntypes + type[j];
            double fs, vlj, vc;
            or_pair(p, r, (double)q[i] * (double)q[j], c6t[tt], c12t[tt], ex, &fs, &vlj, &vc);
            for (int k = 0; k < 3; ++k) fi[k] += fs * d[k];
            if (full) {
                /* each unordered pair is visited twice */
                elj += 0.5 * vlj;
                ec += 0.5 * vc;
                for (int a = 0; a < 3; ++a)
                    for (int b = 0; b < 3; ++b) w[3 * a + b] += 0.5 * d[a] * fs * d[b];
            }
        }
        for (int k = 0; k < 3; ++k) f[3 * ii + k] = fi[k];
    }
    if (full) {
        if (e) { e[0] = elj; e[1] = ec; }
        if (vir) memcpy(vir, w, sizeof(w));
    }
    free(c6t);
    free(c12t);
    return 0;
}

/* Number of unordered pairs with minimum-image distance < r (brute force). */
int64_t or_count_pairs_within(int n, const double* xyz, const double* box, double r) {
    double L[3] = {box[0], box[1], box[2]};
    int64_t cnt = 0;
#pragma omp parallel for schedule(dynamic, 16) reduction(+ : cnt)
    for (int i = 0; i < n; ++i) {
        const double xi[3] = {xyz[3 * i], xyz[3 * i + 1], xyz[3 * i + 2]};
        for (int j = i + 1; j < n; ++j) {
            const double xj[3] = {xyz[3 * j], xyz[3 * j + 1], xyz[3 * j + 2]};
            double d[3];
            min_image(L, xi, xj, d);
            if (d[0] * d[0] + d[1] * d[1] + d[2] * d[2] < r * r) ++cnt;
        }
    }
    return cnt;
}

/* ------------------------------------------------------------------------ */
/* Spatial clustering (Sec. 2.3, Fig. 2).
 *
 * Reading of the paper's steps, all decisions in FP32:
 *  1. wrap: x' = x; if x' < 0 then x' = x' + L; if x' >= L then x' = x' - L
 *     (FP32 ops; requires -L <= x < 2L, else error);
 *  2. grid along x and y of spacing s = (C / rho)^(1/3), rho = n / V (FP64):
 *     n_x = max(1, floor(L_x / s)), same for y;
 *  3. cell of a particle: inv = (float)(n_x / L_x); ix = min(n_x - 1,
 *     (int)(x' * inv)) with one FP32 rounded product; same for y;
 *     column = ix * n_y + iy;
 *  4. particles sorted into columns (column order), within a column on
 *     (z', original index) ascending;
 *  5. clusters are consecutive groups of C in a column; the last cluster of a
 *     column is padded with dummy slots;
 *  6. dummy slot k (global slot index) sits at x = -G (1 + k mod 4096),
 *     y = -G (1 + k div 4096), z = -G with G the smallest power of two
 *     >= 4 max(L); charge 0, type 0.  No dummy is ever within any cut-off of
 *     a particle or of another dummy, under any periodic shift;
 *  7. bounding box of a cluster: min/max over its real particles.
 * Outputs are sized by the caller from or_grid_dims (n_pad_max).
 * Parity: pinned (permutation, z order, column bounds, dummy fraction).
 */
static float wrap_f32(float x, float Lf, int* bad) {
    volatile float v = x;
    if (v < 0.0f) v = v + Lf;
    if (v >= Lf) v = v - Lf;
    if (!(v >= 0.0f && v < Lf)) *bad = 1;
    return v;
}

void or_grid_dims(int n, const float* box, int C, int* nx, int* ny, int64_t* n_pad_max) {
    const double Lx = box[0], Ly = box[1], Lz = box[2];
    int gx = 1, gy = 1;
    if (n > 0) {
        const double rho = (double)n / (Lx * Ly * Lz);
        const double s = cbrt((double)C / rho);
        gx = (int)floor(Lx / s);
        gy = (int)floor(Ly / s);
        if (gx < 1) gx = 1;
        if (gy < 1) gy = 1;
    }
    *nx = gx;
    *ny = gy;
    *n_pad_max = (int64_t)n + (int64_t)gx * gy * (C - 1);
}

typedef struct { int col; uint32_t zbits; int idx; } grid_key;

static int cmp_grid_key(const void* a, const void* b) {
    const grid_key* x = (const grid_key*)a;
    const grid_key* y = (const grid_key*)b;
    if (x->col != y->col) return x->col < y->col ? -1 : 1;
    if (x->zbits != y->zbits) return x->zbits < y->zbits ? -1 : 1;
    return x->idx < y->idx ? -1 : (x->idx > y->idx ? 1 : 0);
}

float or_dummy_spacing(const float* box) {
    float m = box[0];
    if (box[1] > m) m = box[1];
    if (box[2] > m) m = box[2];
    float g = 1.0f;
    while (g < 4.0f * m) g *= 2.0f;
    return g;
}

/* Returns the number of clusters, or -1 on a coordinate outside [-L, 2L). */
int64_t or_grid(int n, const float* xyz, const float* q, const int* type, const float* box, int C,
                float* wrapped /* [n][3] */, int* col_of_atom /* [n] */,
                int* col_clu_start /* [nx*ny+1] */, int* atom_of_slot /* [n_pad_max] */,
                int* slot_of_atom /* [n] */, float* xyzq_slot /* [n_pad_max][4] */,
                int* type_slot /* [n_pad_max] */, float* bb /* [n_clu][6] */) {
    int nx, ny;
    int64_t npm;
    or_grid_dims(n, box, C, &nx, &ny, &npm);
    const float Lx = box[0], Ly = box[1], Lz = box[2];
    const float invx = (float)((double)nx / (double)Lx);
    const float invy = (float)((double)ny / (double)Ly);
    const int ncol = nx * ny;
    int bad = 0;
    grid_key* keys = (grid_key*)malloc(sizeof(grid_key) * (n > 0 ? n : 1));
    for (int i = 0; i < n; ++i) {
        const float x = wrap_f32(xyz[3 * i], Lx, &bad);
        const float y = wrap_f32(xyz[3 * i + 1], Ly, &bad);
        const float z = wrap_f32(xyz[3 * i + 2], Lz, &bad);
        wrapped[3 * i] = x;
        wrapped[3 * i + 1] = y;
        wrapped[3 * i + 2] = z;
        volatile float px = x * invx;
        volatile float py = y * invy;
        int ix = (int)px, iy = (int)py;
        if (ix > nx - 1) ix = nx - 1;
        if (iy > ny - 1) iy = ny - 1;
        const int col = ix * ny + iy;
        col_of_atom[i] = col;
        uint32_t zb;
        memcpy(&zb, &z, 4);
        keys[i].col = col;
        keys[i].zbits = zb;   /* z >= 0: IEEE bits are monotonic */
        keys[i].idx = i;
    }
    if (bad) { free(keys); return -1; }
    qsort(keys, (size_t)n, sizeof(grid_key), cmp_grid_key);
    /* column sizes and cluster offsets */
    int* cnt = (int*)calloc((size_t)ncol, sizeof(int));
    for (int i = 0; i < n; ++i) cnt[keys[i].col]++;
    col_clu_start[0] = 0;
    for (int c = 0; c < ncol; ++c) col_clu_start[c + 1] = col_clu_start[c] + (cnt[c] + C - 1) / C;
    const int64_t nclu = col_clu_start[ncol];
    const float G = or_dummy_spacing(box);
    /* fill slots */
    int pos = 0;
    for (int c = 0; c < ncol; ++c) {
        const int64_t s0 = (int64_t)col_clu_start[c] * C;
        const int64_t s1 = (int64_t)col_clu_start[c + 1] * C;
        for (int64_t s = s0; s < s1; ++s) {
            const int t = (int)(s - s0);
            if (t < cnt[c]) {
                const int a = keys[pos + t].idx;
                atom_of_slot[s] = a;
                slot_of_atom[a] = (int)s;
                xyzq_slot[4 * s + 0] = wrapped[3 * a];
                xyzq_slot[4 * s + 1] = wrapped[3 * a + 1];
                xyzq_slot[4 * s + 2] = wrapped[3 * a + 2];
                xyzq_slot[4 * s + 3] = q[a];
                type_slot[s] = type[a];
            } else {
                atom_of_slot[s] = -1;
                xyzq_slot[4 * s + 0] = -G * (float)(1 + (s % 4096));
                xyzq_slot[4 * s + 1] = -G * (float)(1 + (s / 4096));
                xyzq_slot[4 * s + 2] = -G;
                xyzq_slot[4 * s + 3] = 0.0f;
                type_slot[s] = 0;
            }
        }
        pos += cnt[c];
    }
    /* bounding boxes over real particles */
    for (int64_t g = 0; g < nclu; ++g) {
        float lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
        for (int t = 0; t < C; ++t) {
            const int64_t s = g * C + t;
            if (atom_of_slot[s] < 0) continue;
            for (int k = 0; k < 3; ++k) {
                const float v = xyzq_slot[4 * s + k];
                if (v < lo[k]) lo[k] = v;
                if (v > hi[k]) hi[k] = v;
            }
        }
        for (int k = 0; k < 3; ++k) { bb[6 * g + k] = lo[k]; bb[6 * g + 3 + k] = hi[k]; }
    }
    free(cnt);
    free(keys);
    return nclu;
}

/* Slot coordinates for a later frame: the particle's current coordinates plus
 * the wrap offset applied at gridding (wrapped - original, FP32), so that a
 * particle keeps its periodic image for the lifetime of the list. */
void or_slot_coords(int64_t n_slots, const int* atom_of_slot, const float* xyz_new,
                    const float* xyz_grid, const float* wrapped, const float* xyzq_grid,
                    float* xyzq_out) {
    for (int64_t s = 0; s < n_slots; ++s) {
        const int a = atom_of_slot[s];
        if (a < 0) {
            for (int k = 0; k < 4; ++k) xyzq_out[4 * s + k] = xyzq_grid[4 * s + k];
            continue;
        }
        for (int k = 0; k < 3; ++k) {
            volatile float off = wrapped[3 * a + k] - xyz_grid[3 * a + k];
            volatile float v = xyz_new[3 * a + k] + off;
            xyzq_out[4 * s + k] = v;
        }
        xyzq_out[4 * s + 3] = xyzq_grid[4 * s + 3];
    }
}

/* ------------------------------------------------------------------------ */
/* Cluster-pair search (Sec. 2.3, Fig. 3) and exclusion masks (Sec. 2.4).
 *
 * Canonical list: keys (a, b, s) with cluster indices a <= b and s the
 * periodic shift applied to cluster a, s = (sx, sy, sz) in {-1,0,1}^3 encoded
 * as (sx+1)*9 + (sy+1)*3 + (sz+1) (13 = no shift).  For a == b only s = 13
 * and the lexicographically positive half (s > 13) are kept (each pair once,
 * Newton's third law).  A key is in the list iff
 *     d_BB(a + s, b) < rlist  and  (d_BB(a + s, b) < rBB  or
 *                                    min atom distance(a + s, b) < rlist)
 * with d_BB the FP64 distance between the exact FP32 bounding boxes and the
 * atom distance the FP64 distance between real particles of a and b (slots of
 * dummies never take part).
 * Mask bit (i*C + j) = 1 iff slot i of a and slot j of b hold real, distinct
 * particles that are not force-field excluded and (a != b or s != 13 or
 * j > i): the pair gets the full LJ + Coulomb interaction.
 * Parity: pinned (every particle pair within rlist covered exactly once by the
 * keys; mask bits against the exclusion list; list size ratio).
 */
static double bb_dist2(const float* bba, const float* bbb, const double sh[3]) {
    double d2 = 0.0;
    for (int k = 0; k < 3; ++k) {
        const double alo = (double)bba[k] + sh[k], ahi = (double)bba[3 + k] + sh[k];
        const double blo = bbb[k], bhi = bbb[3 + k];
        double g = 0.0;
        if (blo > ahi) g = blo - ahi;
        else if (alo > bhi) g = alo - bhi;
        d2 += g * g;
    }
    return d2;
}

static double atom_min_dist2(int C, const float* xyzq, const int* atom_of_slot, int64_t a, int64_t b,
                             const double sh[3]) {
    double m = INFINITY;
    for (int i = 0; i < C; ++i) {
        const int64_t si = a * C + i;
        if (atom_of_slot[si] < 0) continue;
        for (int j = 0; j < C; ++j) {
            const int64_t sj = b * C + j;
            if (atom_of_slot[sj] < 0) continue;
            double d2 = 0.0;
            for (int k = 0; k < 3; ++k) {
                const double v = (double)xyzq[4 * si + k] + sh[k] - (double)xyzq[4 * sj + k];
                d2 += v * v;
            }
            if (d2 < m) m = d2;
        }
    }
    return m;
}

static void shift_vec(int s, const float* box, double sh[3]) {
    sh[0] = (double)(s / 9 - 1) * (double)box[0];
    sh[1] = (double)((s / 3) % 3 - 1) * (double)box[1];
    sh[2] = (double)(s % 3 - 1) * (double)box[2];
}

static int key_in_list(int C, const float* xyzq, const int* atom_of_slot, const float* bb,
                       const float* box, double rlist, double rbb, int64_t a, int64_t b, int s) {
    if (a == b && s < 13) return 0;
    double sh[3];
    shift_vec(s, box, sh);
    const double d2 = bb_dist2(bb + 6 * a, bb + 6 * b, sh);
    if (!(d2 < rlist * rlist)) return 0;
    if (d2 < rbb * rbb) return 1;
    return atom_min_dist2(C, xyzq, atom_of_slot, a, b, sh) < rlist * rlist;
}

uint64_t or_mask(int C, const int* atom_of_slot, const int* excl_off, const int* excl_idx,
                 int64_t a, int64_t b, int s) {
    uint64_t m = 0;
    for (int i = 0; i < C; ++i) {
        const int pi = atom_of_slot[a * C + i];
        if (pi < 0) continue;
        for (int j = 0; j < C; ++j) {
            const int pj = atom_of_slot[b * C + j];
            if (pj < 0 || pj == pi) continue;
            if (a == b && s == 13 && !(j > i)) continue;
            if (is_excluded(excl_off, excl_idx, pi, pj)) continue;
            m |= (uint64_t)1 << (i * C + j);
        }
    }
    return m;
}

/* Full canonical list: every key (a <= b, s), sorted by (a, b, s).
 * Writes up to cap keys; returns the total count (or -1 if rlist >= L/2). */
int64_t or_pairlist(int64_t nclu, int C, const float* xyzq, const int* atom_of_slot,
                    const float* bb, const float* box, double rlist, double rbb,
                    const int* excl_off, const int* excl_idx, int64_t cap,
                    int* out_a, int* out_b, int* out_s, uint64_t* out_mask) {
    for (int k = 0; k < 3; ++k)
        if (!(rlist < 0.5 * (double)box[k])) return -1;
    int64_t* cnt = (int64_t*)calloc((size_t)nclu + 1, sizeof(int64_t));
#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t a = 0; a < nclu; ++a) {
        int64_t c = 0;
        for (int64_t b = a; b < nclu; ++b)
            for (int s = 0; s < 27; ++s)
                c += key_in_list(C, xyzq, atom_of_slot, bb, box, rlist, rbb, a, b, s);
        cnt[a + 1] = c;
    }
    for (int64_t a = 0; a < nclu; ++a) cnt[a + 1] += cnt[a];
    const int64_t total = cnt[nclu];
#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t a = 0; a < nclu; ++a) {
        int64_t o = cnt[a];
        for (int64_t b = a; b < nclu; ++b)
            for (int s = 0; s < 27; ++s)
                if (key_in_list(C, xyzq, atom_of_slot, bb, box, rlist, rbb, a, b, s)) {
                    if (o < cap) {
                        out_a[o] = (int)a;
                        out_b[o] = (int)b;
                        out_s[o] = s;
                        out_mask[o] = or_mask(C, atom_of_slot, excl_off, excl_idx, a, b, s);
                    }
                    ++o;
                }
    }
    free(cnt);
    return total;
}

/* Keys of the canonical list that involve cluster c (as a or as b), for
 * sampled checks on large boxes; sorted by (a, b, s). */
int64_t or_pairlist_cluster(int64_t nclu, int C, const float* xyzq, const int* atom_of_slot,
                            const float* bb, const float* box, double rlist, double rbb,
                            const int* excl_off, const int* excl_idx, int64_t c, int64_t cap,
                            int* out_a, int* out_b, int* out_s, uint64_t* out_mask) {
    int64_t o = 0;
    for (int64_t x = 0; x < nclu; ++x) {
        const int64_t a = x < c ? x : c;
        const int64_t b = x < c ? c : x;
        for (int s = 0; s < 27; ++s)
            if (key_in_list(C, xyzq, atom_of_slot, bb, box, rlist, rbb, a, b, s)) {
                if (o < cap) {
                    out_a[o] = (int)a;
                    out_b[o] = (int)b;
                    out_s[o] = s;
                    out_mask[o] = or_mask(C, atom_of_slot, excl_off, excl_idx, a, b, s);
                }
                ++o;
            }
    }
    return o;
}

/* Minimum FP64 distance between the particles of key (a, b, s) counted by the
 * interaction (real, distinct, and j > i on the unshifted diagonal), and the
 * FP64 bounding-box distance; used to exempt keys near a threshold. */
void or_key_distances(int C, const float* xyzq, const int* atom_of_slot, const float* bb,
                      const float* box, int64_t nkeys, const int* ka, const int* kb, const int* ks,
                      double* dmin_atom, double* d_bb) {
#pragma omp parallel for schedule(static)
    for (int64_t k = 0; k < nkeys; ++k) {
        double sh[3];
        shift_vec(ks[k], box, sh);
        d_bb[k] = sqrt(bb_dist2(bb + 6 * (int64_t)ka[k], bb + 6 * (int64_t)kb[k], sh));
        dmin_atom[k] = sqrt(atom_min_dist2(C, xyzq, atom_of_slot, ka[k], kb[k], sh));
    }
}

/* ------------------------------------------------------------------------ */
/* Pruning (Sec. 2.3): a key is kept iff at least one particle pair that the
 * interaction counts -- real, distinct, and on the unshifted diagonal only
 * j > i; full-interaction and force-field-excluded pairs alike, since the
 * latter still get the RF/Ewald correction -- is closer than r_prune under
 * the current slot coordinates.  keep[k] = 1/0; dmin[k] = that minimum
 * distance (FP64), for threshold exemptions.
 * Parity: pinned (no pair within r_prune is lost; brute-force pair cover). */
void or_prune(int C, const float* xyzq, const int* atom_of_slot, const float* box,
              double r_prune, int64_t nkeys, const int* ka, const int* kb, const int* ks,
              unsigned char* keep, double* dmin) {
#pragma omp parallel for schedule(static)
    for (int64_t k = 0; k < nkeys; ++k) {
        double sh[3];
        shift_vec(ks[k], box, sh);
        const int64_t a = ka[k], b = kb[k];
        double m = INFINITY;
        for (int i = 0; i < C; ++i) {
            const int64_t si = a * C + i;
            if (atom_of_slot[si] < 0) continue;
            for (int j = 0; j < C; ++j) {
                const int64_t sj = b * C + j;
                if (atom_of_slot[sj] < 0) continue;
                if (atom_of_slot[si] == atom_of_slot[sj]) continue;
                if (a == b && ks[k] == 13 && !(j > i)) continue;
                double d2 = 0.0;
                for (int x = 0; x < 3; ++x) {
                    const double v = (double)xyzq[4 * si + x] + sh[x] - (double)xyzq[4 * sj + x];
                    d2 += v * v;
                }
                if (d2 < m) m = d2;
            }
        }
        dmin[k] = sqrt(m);
        keep[k] = m < r_prune * r_prune;
    }
}

/* For each unordered particle pair within r (minimum image), count how many
 * list keys cover it (with its image shift): cover[0] = pairs covered exactly
 * once, cover[1] = pairs not covered, cover[2] = pairs covered more than once.
 * Independent of the list construction: expands keys to particle pairs.
 * Brute force, small boxes only. */
void or_pair_cover(int n, const float* xyz_wrapped, const float* box, double r, int C,
                   const int* atom_of_slot, const int* slot_of_atom, int64_t nkeys,
                   const int* ka, const int* kb, const int* ks, int64_t* cover) {
    /* count[i*n + j] for i < j, restricted to pairs within r */
    int* hits = (int*)calloc((size_t)n * (size_t)n, sizeof(int));
    const double L[3] = {box[0], box[1], box[2]};
    for (int64_t k = 0; k < nkeys; ++k) {
        double sh[3];
        shift_vec(ks[k], box, sh);
        for (int i = 0; i < C; ++i) {
            const int pi = atom_of_slot[(int64_t)ka[k] * C + i];
            if (pi < 0) continue;
            for (int j = 0; j < C; ++j) {
                const int pj = atom_of_slot[(int64_t)kb[k] * C + j];
                if (pj < 0 || pj == pi) continue;
                if (ka[k] == kb[k] && ks[k] == 13 && !(j > i)) continue;
                double d2 = 0.0;
                for (int x = 0; x < 3; ++x) {
                    const double v = (double)xyz_wrapped[3 * pi + x] + sh[x] - (double)xyz_wrapped[3 * pj + x];
                    d2 += v * v;
                }
                if (d2 < r * r) {
                    const int lo = pi < pj ? pi : pj, hi = pi < pj ? pj : pi;
                    hits[(size_t)lo * n + hi]++;
                }
            }
        }
    }
    int64_t once = 0, none = 0, many = 0;
    for (int i = 0; i < n; ++i) {
        const double xi[3] = {xyz_wrapped[3 * i], xyz_wrapped[3 * i + 1], xyz_wrapped[3 * i + 2]};
        for (int j = i + 1; j < n; ++j) {
            const double xj[3] = {xyz_wrapped[3 * j], xyz_wrapped[3 * j + 1], xyz_wrapped[3 * j + 2]};
            double d[3];
            min_image(L, xi, xj, d);
            const int h = hits[(size_t)i * n + j];
            if (d[0] * d[0] + d[1] * d[1] + d[2] * d[2] < r * r) {
                if (h == 1) ++once;
                else if (h == 0) ++none;
                else ++many;
            } else if (h > 0) {
                ++many;  /* covered although not within r: impossible */
            }
        }
    }
    (void)slot_of_atom;
    cover[0] = once;
    cover[1] = none;
    cover[2] = many;
    free(hits);
}

/* ------------------------------------------------------------------------ */
/* Ewald real-space force factor (Sec. 3.2) and the small network that may
 * stand in for it.
 *
 * c(r) = erfc(beta r) + (2 beta r / sqrt(pi)) exp(-beta^2 r^2): the force of
 * a non-excluded Ewald real-space pair is f qq c(r) / r^2 (g(r) = d/dr
 * [erf(beta r)/r] added to the plain 1/r^2).  Parity: pinned by erfc values
 * and the beta -> 0 limit c = 1.
 */
void or_ewald_factor(int64_t n, const double* r, double beta, double* out) {
    for (int64_t i = 0; i < n; ++i) {
        const double br = beta * r[i];
        out[i] = erfc(br) + 2.0 * br / sqrt(M_PI) * exp(-br * br);
    }
}

#define OR_MLP_H 32
#define OR_MLP_NP (OR_MLP_H + OR_MLP_H + OR_MLP_H * OR_MLP_H + OR_MLP_H + OR_MLP_H + 1)

static double or_silu(double z) { return z / (1.0 + exp(-z)); }

/* d/dz [z s(z)] with s the logistic function: s + z s (1 - s). */
static double or_silu_d(double z) {
    const double s = 1.0 / (1.0 + exp(-z));
    return s + z * s * (1.0 - s);
}

/* One sample through the network, keeping the pre-activations. */
static double or_mlp_one(const double* p, double x, double* z1, double* h1, double* z2, double* h2) {
    const double* W1 = p;
    const double* b1 = p + OR_MLP_H;
    const double* W2 = p + 2 * OR_MLP_H;
    const double* b2 = W2 + OR_MLP_H * OR_MLP_H;
    const double* W3 = b2 + OR_MLP_H;
    const double b3 = W3[OR_MLP_H];
    for (int j = 0; j < OR_MLP_H; ++j) {
        z1[j] = W1[j] * x + b1[j];
        h1[j] = or_silu(z1[j]);
    }
    double y = b3;
    for (int k = 0; k < OR_MLP_H; ++k) {
        double s = b2[k];
        for (int j = 0; j < OR_MLP_H; ++j) s += W2[k * OR_MLP_H + j] * h1[j];
        z2[k] = s;
        h2[k] = or_silu(s);
        y += W3[k] * h2[k];
    }
    return y;
}

/* Multilayer perceptron 1 -> 32 -> 32 -> 1 with SiLU hidden layers (the
 * learned stand-in for c(r)).  Input x = (r - (r_min + r_max) / 2) * 2 /
 * (r_max - r_min); h1 = SiLU(W1 x + b1), h2 = SiLU(W2 h1 + b2),
 * y = W3 . h2 + b3.  Parameters (1153): W1[32], b1[32], W2[32][32] (row =
 * output unit), b2[32], W3[32], b3.
 * Parity: pinned by a closed form (weights reducing the network to
 * SiLU(SiLU(ln 3)) = (3/4) SiLU(ln 3) ... at chosen inputs) and by its
 * linearity in the last layer. */
void or_mlp_forward(const double* p, double rmin, double rmax, int64_t n, const double* r, double* y) {
    const double c0 = 0.5 * (rmin + rmax), c1 = 2.0 / (rmax - rmin);
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
        double z1[OR_MLP_H], h1[OR_MLP_H], z2[OR_MLP_H], h2[OR_MLP_H];
        y[i] = or_mlp_one(p, (r[i] - c0) * c1, z1, h1, z2, h2);
    }
}

/* Loss L = (1/n) sum_i w_i (y(r_i) - t_i)^2 (w may be NULL: all ones) and its
 * gradient with respect to the 1153 parameters, by the chain rule layer by
 * layer from the output back.  Parity: pinned by central finite differences
 * of the loss (forward pinned separately). */
double or_mlp_loss_grad(const double* p, double rmin, double rmax, int64_t n, const double* r,
                        const double* t, const double* w, double* grad) {
    const double c0 = 0.5 * (rmin + rmax), c1 = 2.0 / (rmax - rmin);
    const double* W2 = p + 2 * OR_MLP_H;
    const double* W3 = W2 + OR_MLP_H * OR_MLP_H + OR_MLP_H;
    double* gW1 = grad;
    double* gb1 = grad + OR_MLP_H;
    double* gW2 = grad + 2 * OR_MLP_H;
    double* gb2 = gW2 + OR_MLP_H * OR_MLP_H;
    double* gW3 = gb2 + OR_MLP_H;
    double* gb3 = gW3 + OR_MLP_H;
    memset(grad, 0, sizeof(double) * OR_MLP_NP);
    double loss = 0.0;
    for (int64_t i = 0; i < n; ++i) {
        double z1[OR_MLP_H], h1[OR_MLP_H], z2[OR_MLP_H], h2[OR_MLP_H], dz2[OR_MLP_H];
        const double x = (r[i] - c0) * c1;
        const double y = or_mlp_one(p, x, z1, h1, z2, h2);
        const double wi = w ? w[i] : 1.0;
        const double e = y - t[i];
        loss += wi * e * e / (double)n;
        const double dy = 2.0 * wi * e / (double)n;   /* dL/dy */
        *gb3 += dy;
        for (int k = 0; k < OR_MLP_H; ++k) {
            gW3[k] += dy * h2[k];
            dz2[k] = dy * W3[k] * or_silu_d(z2[k]);
            gb2[k] += dz2[k];
            for (int j = 0; j < OR_MLP_H; ++j) gW2[k * OR_MLP_H + j] += dz2[k] * h1[j];
        }
        for (int j = 0; j < OR_MLP_H; ++j) {
            double dh = 0.0;
            for (int k = 0; k < OR_MLP_H; ++k) dh += W2[k * OR_MLP_H + j] * dz2[k];
            const double dz1 = dh * or_silu_d(z1[j]);
            gW1[j] += dz1 * x;
            gb1[j] += dz1;
        }
    }
    return loss;
}

/* ------------------------------------------------------------------------ */
/* Tier B: the same forces, energies and virial as or_forces_brute through a
 * cell list (cells of edge >= rc along each axis; every particle meets the
 * particles of its own and its neighbouring cells, each neighbouring cell
 * counted once even where fewer than three cells span an axis), so its cost
 * grows linearly with n.  Pairs use the same pair function and minimum
 * image as Tier A, so the two agree to rounding; the cell enumeration is
 * independent code and is pinned against Tier A on small boxes.
 * Arguments and outputs as or_forces_brute (sel: forces of the selected
 * particles only).  Returns 0, or -1 when rc >= L/2.
 */
int or_forces_cells(int n, const double* xyz, const float* q, const int* type,
                    int ntypes, const double* sigma, const double* eps,
                    const int* excl_off, const int* excl_idx, const double* box,
                    const or_params* p, int n_sel, const int* sel,
                    double* f, double* e, double* vir) {
    const double L[3] = {box[0], box[1], box[2]};
    for (int k = 0; k < 3; ++k)
        if (!(p->rc < 0.5 * L[k])) return -1;
    int nc[3];
    for (int k = 0; k < 3; ++k) {
        nc[k] = (int)floor(L[k] / p->rc);
        if (nc[k] < 1) nc[k] = 1;
    }
    const int64_t ncell = (int64_t)nc[0] * nc[1] * nc[2];
    int* cell_of = (int*)malloc(sizeof(int) * (n > 0 ? n : 1));
    int64_t* start = (int64_t*)calloc((size_t)ncell + 1, sizeof(int64_t));
    int* members = (int*)malloc(sizeof(int) * (n > 0 ? n : 1));
    for (int i = 0; i < n; ++i) {
        int c[3];
        for (int k = 0; k < 3; ++k) {
            double x = xyz[3 * i + k] - L[k] * floor(xyz[3 * i + k] / L[k]);
            int v = (int)(x / L[k] * nc[k]);
            if (v < 0) v = 0;
            if (v >= nc[k]) v = nc[k] - 1;
            c[k] = v;
        }
        cell_of[i] = (c[0] * nc[1] + c[1]) * nc[2] + c[2];
        start[cell_of[i] + 1]++;
    }
    for (int64_t c = 0; c < ncell; ++c) start[c + 1] += start[c];
    {
        int64_t* fill = (int64_t*)malloc(sizeof(int64_t) * (size_t)(ncell > 0 ? ncell : 1));
        memcpy(fill, start, sizeof(int64_t) * (size_t)ncell);
        for (int i = 0; i < n; ++i) members[fill[cell_of[i]]++] = i;
        free(fill);
    }
    double* c6t = (double*)malloc(sizeof(double) * ntypes * ntypes);
    double* c12t = (double*)malloc(sizeof(double) * ntypes * ntypes);
    for (int a = 0; a < ntypes; ++a)
        for (int b = 0; b < ntypes; ++b)
            or_lj_pair_params(p->comb, sigma[a], eps[a], sigma[b], eps[b],
                              &c6t[a * ntypes + b], &c12t[a * ntypes + b]);
    const int full = (n_sel <= 0);
    const int ni = full ? n : n_sel;
    const double rc2 = p->rc * p->rc;
    double elj = 0.0, ec = 0.0;
    double w[9] = {0};
#pragma omp parallel for schedule(dynamic, 64) reduction(+ : elj, ec) reduction(+ : w[:9])
    for (int ii = 0; ii < ni; ++ii) {
        const int i = full ? ii : sel[ii];
        const int ci = cell_of[i];
        const int cz = ci % nc[2], cy = (ci / nc[2]) % nc[1], cx = ci / (nc[2] * nc[1]);
        /* distinct neighbouring cells along each axis */
        int nb[3][3], nn[3];
        const int cc[3] = {cx, cy, cz};
        for (int k = 0; k < 3; ++k) {
            nn[k] = 0;
            for (int o = -1; o <= 1; ++o) {
                const int v = ((cc[k] + o) % nc[k] + nc[k]) % nc[k];
                int seen = 0;
                for (int m = 0; m < nn[k]; ++m) seen |= (nb[k][m] == v);
                if (!seen) nb[k][nn[k]++] = v;
            }
        }
        double fi[3] = {0, 0, 0};
        for (int a = 0; a < nn[0]; ++a)
            for (int b = 0; b < nn[1]; ++b)
                for (int c = 0; c < nn[2]; ++c) {
                    const int64_t cell = ((int64_t)nb[0][a] * nc[1] + nb[1][b]) * nc[2] + nb[2][c];
                    for (int64_t m = start[cell]; m < start[cell + 1]; ++m) {
                        const int j = members[m];
                        if (j == i) continue;
                        double d[3];
                        for (int k = 0; k < 3; ++k) {
                            double v = xyz[3 * i + k] - xyz[3 * j + k];
                            v -= L[k] * nearbyint(v / L[k]);
                            d[k] = v;
                        }
                        const double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
                        if (!(r2 < rc2)) continue;
                        int ex = 0;
                        if (excl_off)
                            for (int k = excl_off[i]; k < excl_off[i + 1]; ++k) ex |= (excl_idx[k] == j);
                        const int tt = type[i] * ntypes + type[j];
                        double fs, vlj, vc;
                        or_pair(p, sqrt(r2), (double)q[i] * (double)q[j], c6t[tt], c12t[tt], ex, &fs, &vlj, &vc);
                        for (int k = 0; k < 3; ++k) fi[k] += fs * d[k];
                        if (full) {
                            elj += 0.5 * vlj;
                            ec += 0.5 * vc;
                            for (int x = 0; x < 3; ++x)
                                for (int y = 0; y < 3; ++y) w[3 * x + y] += 0.5 * d[x] * fs * d[y];
                        }
                    }
                }
        for (int k = 0; k < 3; ++k) f[3 * ii + k] = fi[k];
    }
    if (full) {
        if (e) { e[0] = elj; e[1] = ec; }
        if (vir) memcpy(vir, w, sizeof(w));
    }
    free(c6t);
    free(c12t);
    free(cell_of);
    free(start);
    free(members);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Verlet-buffer energy drift (Appendix): for a pair whose distance moves
 * from r0 > rl = rc + rb (outside the list) to rt < rc during a list
 * lifetime, with the pair potential expanded to second order at rc,
 *   I = int_{rt < rc} int_{r0 > rl} [V1 (rt - rc) + V2/2 (rt - rc)^2]
 *           phi((rt - r0)/sigma)/sigma dr0 drt,
 * phi the standard normal density.  Evaluated here by plain 2-D quadrature
 * (midpoint rule on u = rt - rc in [-L, 0], w = r0 - rl in [0, L],
 * L = rb + 12 sigma), with no use of the closed form.
 * Parity: pinned by the exact value at rb = 0 and by symbolic integration. */
double or_buffer_drift_integral(double V1, double V2, double rb, double sigma) {
    const int n = 1500;
    const double L = rb + 12.0 * sigma;
    const double h = L / n;
    double sum = 0.0;
    for (int a = 0; a < n; ++a) {
        const double u = -L + (a + 0.5) * h;           /* rt - rc <= 0 */
        const double f = V1 * u + 0.5 * V2 * u * u;
        double inner = 0.0;
        for (int b = 0; b < n; ++b) {
            const double w = (b + 0.5) * h;             /* r0 - rl >= 0 */
            const double z = (u - w - rb) / sigma;      /* (rt - r0) / sigma */
            inner += exp(-0.5 * z * z);
        }
        sum += f * inner;
    }
    return sum * h * h / (sigma * sqrt(2.0 * M_PI));
}

/* ------------------------------------------------------------------------ */
/* Pair-distance histogram: the pair correlation function, the analysis the
 * paper lists beside force calculation as limited-range pair work (Sec. 1)
 * and for which it advises a list rebuilt every time and no cut-off
 * conditional in the kernel (Sec. 2.3).
 *
 * Every unordered pair {i, j} of distinct particles that is not force-field
 * excluded, whose types match the selection (type_a < 0: every pair; else
 * {type_i, type_j} = {type_a, type_b}) and whose minimum-image FP64 distance
 * r is below r_max adds one to bin floor(r / dr), dr = r_max / nbins.
 * near[k] (k = 0..nbins) counts the selected pairs with |r - k dr| < delta,
 * the pairs whose bin a computation of r in lower precision may put on the
 * other side of edge k (near[nbins] includes pairs just beyond r_max).
 * brute != 0: the O(n^2) double loop; else a cell list (cells of edge >=
 * r_max + delta, each distinct neighbouring cell visited once, a pair counted
 * from its lower index).
 * Returns 0, or -1 when r_max + delta >= L/2, nbins < 1 or delta >= dr/2.
 * Parity: pinned by a cubic lattice's exact shell counts and by brute force. */
static int rdf_selected(const int* type, int type_a, int type_b, int i, int j) {
    if (type_a < 0) return 1;
    return (type[i] == type_a && type[j] == type_b) || (type[i] == type_b && type[j] == type_a);
}

static void rdf_add(double r2, double r_max, double dr, double delta, int nbins, int64_t* hist,
                    int64_t* near) {
    const double r = sqrt(r2);
    if (r < r_max) {
        int k = (int)floor(r / dr);
        if (k > nbins - 1) k = nbins - 1;
        hist[k]++;
    }
    const int e = (int)nearbyint(r / dr);
    if (e >= 0 && e <= nbins && fabs(r - e * dr) < delta) near[e]++;
}

int or_rdf(int n, const double* xyz, const int* type, const int* excl_off, const int* excl_idx,
           const double* box, double r_max, int nbins, int type_a, int type_b, double delta, int brute,
           int64_t* hist, int64_t* near) {
    const double L[3] = {box[0], box[1], box[2]};
    const double dr = r_max / nbins;
    const double rr = r_max + delta;
    if (nbins < 1 || !(r_max > 0.0) || !(delta >= 0.0) || !(delta < 0.5 * dr)) return -1;
    for (int k = 0; k < 3; ++k)
        if (!(rr < 0.5 * L[k])) return -1;
    memset(hist, 0, sizeof(int64_t) * (size_t)nbins);
    memset(near, 0, sizeof(int64_t) * (size_t)(nbins + 1));
    if (brute) {
#pragma omp parallel for schedule(dynamic, 16) reduction(+ : hist[:nbins], near[:nbins + 1])
        for (int i = 0; i < n; ++i) {
            const double xi[3] = {xyz[3 * i], xyz[3 * i + 1], xyz[3 * i + 2]};
            for (int j = i + 1; j < n; ++j) {
                if (!rdf_selected(type, type_a, type_b, i, j) || is_excluded(excl_off, excl_idx, i, j)) continue;
                const double xj[3] = {xyz[3 * j], xyz[3 * j + 1], xyz[3 * j + 2]};
                double d[3];
                min_image(L, xi, xj, d);
                const double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
                if (r2 < rr * rr) rdf_add(r2, r_max, dr, delta, nbins, hist, near);
            }
        }
        return 0;
    }
    int nc[3];
    for (int k = 0; k < 3; ++k) {
        nc[k] = (int)floor(L[k] / rr);
        if (nc[k] < 1) nc[k] = 1;
    }
    const int64_t ncell = (int64_t)nc[0] * nc[1] * nc[2];
    int* cell_of = (int*)malloc(sizeof(int) * (n > 0 ? n : 1));
    int64_t* start = (int64_t*)calloc((size_t)ncell + 1, sizeof(int64_t));
    int* members = (int*)malloc(sizeof(int) * (n > 0 ? n : 1));
    for (int i = 0; i < n; ++i) {
        int c[3];
        for (int k = 0; k < 3; ++k) {
            const double x = xyz[3 * i + k] - L[k] * floor(xyz[3 * i + k] / L[k]);
            int v = (int)(x / L[k] * nc[k]);
            if (v < 0) v = 0;
            if (v >= nc[k]) v = nc[k] - 1;
            c[k] = v;
        }
        cell_of[i] = (c[0] * nc[1] + c[1]) * nc[2] + c[2];
        start[cell_of[i] + 1]++;
    }
    for (int64_t c = 0; c < ncell; ++c) start[c + 1] += start[c];
    {
        int64_t* fill = (int64_t*)malloc(sizeof(int64_t) * (size_t)(ncell > 0 ? ncell : 1));
        memcpy(fill, start, sizeof(int64_t) * (size_t)ncell);
        for (int i = 0; i < n; ++i) members[fill[cell_of[i]]++] = i;
        free(fill);
    }
#pragma omp parallel for schedule(dynamic, 64) reduction(+ : hist[:nbins], near[:nbins + 1])
    for (int i = 0; i < n; ++i) {
        const int ci = cell_of[i];
        const int cc[3] = {ci / (nc[2] * nc[1]), (ci / nc[2]) % nc[1], ci % nc[2]};
        int nb[3][3], nn[3];
        for (int k = 0; k < 3; ++k) {
            nn[k] = 0;
            for (int o = -1; o <= 1; ++o) {
                const int v = ((cc[k] + o) % nc[k] + nc[k]) % nc[k];
                int seen = 0;
                for (int m = 0; m < nn[k]; ++m) seen |= (nb[k][m] == v);
                if (!seen) nb[k][nn[k]++] = v;
            }
        }
        const double xi[3] = {xyz[3 * i], xyz[3 * i + 1], xyz[3 * i + 2]};
        for (int a = 0; a < nn[0]; ++a)
            for (int b = 0; b < nn[1]; ++b)
                for (int c = 0; c < nn[2]; ++c) {
                    const int64_t cell = ((int64_t)nb[0][a] * nc[1] + nb[1][b]) * nc[2] + nb[2][c];
                    for (int64_t m = start[cell]; m < start[cell + 1]; ++m) {
                        const int j = members[m];
                        if (j <= i) continue;
                        if (!rdf_selected(type, type_a, type_b, i, j) || is_excluded(excl_off, excl_idx, i, j))
                            continue;
                        const double xj[3] = {xyz[3 * j], xyz[3 * j + 1], xyz[3 * j + 2]};
                        double d[3];
                        min_image(L, xi, xj, d);
                        const double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
                        if (r2 < rr * rr) rdf_add(r2, r_max, dr, delta, nbins, hist, near);
                    }
                }
    }
    free(cell_of);
    free(start);
    free(members);
    return 0;
}
