/*
 * misa_oracle.c -- plain FP64 CPU oracle for the EAM lattice-list MD hot path
 * of MISA-MD (Chu et al., "MISA-MD: an efficient parallel molecular dynamics
 * simulation for cascade collision", arXiv:2107.07866).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link, load or
 * call this file: only tests/, __graft_entry__.smoke() and the cpu_baseline /
 * reference leg of bench.py use it.  It shares no code, header, table or
 * constant generator with the CUDA library under paper_2107_07866_gb300/.
 *
 * What it computes, and where each piece comes from:
 *   - Spline tables (Sec. 4.1): one cubic polynomial per segment of an
 *     equidistant knot grid.  The paper does not name the spline type; its
 *     coefficients are rebuilt on the fly from a local window of raw knots,
 *     so this oracle reads it as the local cubic Hermite spline with knot
 *     slopes from central differences (4th order inside, 2nd order at the
 *     two outermost knots of each end).  The spline is written out in the
 *     Hermite basis straight from the knots; no power-form coefficients.
 *   - EAM energy (Eq. eam_base) and pair force (Eq. eam_force_ij), computed
 *     in the five steps listed after Eq. eam_force_ij (Sec. 2.2): density,
 *     embedding derivative, pair derivative, density derivative, force sum.
 *     The method reaches exactly this plain result (Sec. 3, end), so the
 *     oracle enumerates pairs by brute force over periodic images, or by a
 *     plain cell list, not by the lattice list.
 *   - Lattice id (Sec. 3, Eq. for index = 2 bx by z + 2 bx y + x), nearest
 *     lattice site (the hash function of Sec. 3), the lattice list with its
 *     neighbour offset index and run-away ("hash clash") atoms (Alg. 1,
 *     Alg. 2), as a second, independent pair enumeration used only to check
 *     that the lattice-list pair set equals the brute-force pair set.
 *   - Velocity Verlet (Fig. 1, read as kick-drift-kick), adaptive timestep
 *     (Sec. 1 feature list), PKA insertion (Sec. 5.1).
 *   - Gradient of a force-matching + energy loss with respect to the knot
 *     values (no counterpart in the paper; used to fit potentials).
 *
 * Units: Angstrom, eV, fs, amu.  a = F/m * MISA_O_ACC, with
 * MISA_O_ACC = 1 eV/(Angstrom amu) in Angstrom/fs^2 (CODATA 2018).
 *
 * Parity pins live in tests/test_oracle_*.py.  "parity unpinned" items:
 * none of the functions below; cascade physics (Frenkel-pair counts vs the
 * paper's figures) is not attempted.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define MISA_O_ACC 9.6485332123310018e-3 /* (1.602176634e-19 J) / (1.66053906660e-27 kg) in A/fs^2 */

/* ------------------------------------------------------------------------ */
/* Spline tables (Sec. 4.1)                                                  */
/* ------------------------------------------------------------------------ */

/* Knot slopes dy/dx of the local Hermite reading of the Sec. 4.1 spline. */
int or_spline_slopes(const double *y, int n, double h, double *m)
{
    if (n < 5 || h <= 0.0) return -1;
    for (int k = 0; k < n; ++k) {
        if (k == 0)
            m[k] = (-3.0 * y[0] + 4.0 * y[1] - y[2]) / (2.0 * h);
        else if (k == n - 1)
            m[k] = (3.0 * y[n - 1] - 4.0 * y[n - 2] + y[n - 3]) / (2.0 * h);
        else if (k == 1 || k == n - 2)
            m[k] = (y[k + 1] - y[k - 1]) / (2.0 * h);
        else
            m[k] = (y[k - 2] - 8.0 * y[k - 1] + 8.0 * y[k + 1] - y[k + 2]) / (12.0 * h);
    }
    return 0;
}

/* Segment and local coordinate of x on the grid x_k = k h, k = 0..n-1. */
static void seg_of(double x, int n, double h, int *s, double *t)
{
    double u = x / h;
    int k = (int)floor(u);
    if (k < 0) k = 0;
    if (k > n - 2) k = n - 2;
    *s = k;
    *t = u - (double)k;
}

/* Value and derivative of the Hermite spline at x.  Inside [0, x_{n-1}]
 * this is the cubic of segment s written in the Hermite basis. */
double or_spline_eval(const double *y, const double *m, int n, double h, double x, double *deriv)
{
    int s;
    double t;
    seg_of(x, n, h, &s, &t);
    double t2 = t * t, t3 = t2 * t;
    double h00 = 2.0 * t3 - 3.0 * t2 + 1.0;
    double h10 = t3 - 2.0 * t2 + t;
    double h01 = -2.0 * t3 + 3.0 * t2;
    double h11 = t3 - t2;
    double d00 = 6.0 * t2 - 6.0 * t;
    double d10 = 3.0 * t2 - 4.0 * t + 1.0;
    double d01 = -6.0 * t2 + 6.0 * t;
    double d11 = 3.0 * t2 - 2.0 * t;
    double y0 = y[s], y1 = y[s + 1], m0 = m[s] * h, m1 = m[s + 1] * h;
    if (deriv) *deriv = (d00 * y0 + d10 * m0 + d01 * y1 + d11 * m1) / h;
    return h00 * y0 + h10 * m0 + h01 * y1 + h11 * m1;
}

/* Weights w_k with S(x) = sum_k w_k y_k (and dS/dx = sum_k dw_k y_k): the
 * spline is linear in its knot values.  Writes up to 8 (index, w, dw)
 * triples; returns their count.  Used by the knot-gradient oracle. */
int or_spline_weights(int n, double h, double x, int *idx, double *w, double *dw)
{
    int s;
    double t;
    seg_of(x, n, h, &s, &t);
    double t2 = t * t, t3 = t2 * t;
    double c[4] = {2.0 * t3 - 3.0 * t2 + 1.0, (t3 - 2.0 * t2 + t) * h, -2.0 * t3 + 3.0 * t2, (t3 - t2) * h};
    double dc[4] = {(6.0 * t2 - 6.0 * t) / h, 3.0 * t2 - 4.0 * t + 1.0, (-6.0 * t2 + 6.0 * t) / h, 3.0 * t2 - 2.0 * t};
    /* local accumulation over knots s-2 .. s+3 */
    double acc[6] = {0}, dacc[6] = {0};
    int base = s - 2;
    acc[2] += c[0];
    dacc[2] += dc[0];
    acc[3] += c[2];
    dacc[3] += dc[2];
    for (int e = 0; e < 2; ++e) {
        int k = s + e;
        double cm = e == 0 ? c[1] : c[3];
        double dcm = e == 0 ? dc[1] : dc[3];
        /* slope stencil of knot k (matches or_spline_slopes) */
        int ks[5];
        double kw[5];
        int ns = 0;
        if (k == 0) {
            ks[0] = 0; kw[0] = -3.0 / (2.0 * h);
            ks[1] = 1; kw[1] = 4.0 / (2.0 * h);
            ks[2] = 2; kw[2] = -1.0 / (2.0 * h);
            ns = 3;
        } else if (k == n - 1) {
            ks[0] = n - 1; kw[0] = 3.0 / (2.0 * h);
            ks[1] = n - 2; kw[1] = -4.0 / (2.0 * h);
            ks[2] = n - 3; kw[2] = 1.0 / (2.0 * h);
            ns = 3;
        } else if (k == 1 || k == n - 2) {
            ks[0] = k + 1; kw[0] = 1.0 / (2.0 * h);
            ks[1] = k - 1; kw[1] = -1.0 / (2.0 * h);
            ns = 2;
        } else {
            ks[0] = k - 2; kw[0] = 1.0 / (12.0 * h);
            ks[1] = k - 1; kw[1] = -8.0 / (12.0 * h);
            ks[2] = k + 1; kw[2] = 8.0 / (12.0 * h);
            ks[3] = k + 2; kw[3] = -1.0 / (12.0 * h);
            ns = 4;
        }
        for (int q = 0; q < ns; ++q) {
            int j = ks[q] - base; /* always within 0..5 for the stencils above */
            acc[j] += cm * kw[q];
            dacc[j] += dcm * kw[q];
        }
    }
    int cnt = 0;
    for (int j = 0; j < 6; ++j) {
        int k = base + j;
        if (k < 0 || k >= n) continue;
        if (acc[j] == 0.0 && dacc[j] == 0.0) continue;
        idx[cnt] = k;
        w[cnt] = acc[j];
        dw[cnt] = dacc[j];
        ++cnt;
    }
    return cnt;
}

/* ------------------------------------------------------------------------ */
/* EAM potential from three tables (Sec. 2.2, Sec. 4.1)                      */
/* ------------------------------------------------------------------------ */

typedef struct or_pot {
    int n;
    double rc, rho_max, hr, hrho, r_floor;
    double *f, *phi, *F;    /* knot values (owned copies) */
    double *mf, *mphi, *mF; /* knot slopes */
} or_pot;

or_pot *or_pot_new(int n, double rc, double rho_max, const double *f, const double *phi, const double *F)
{
    if (n < 5 || rc <= 0.0 || rho_max <= 0.0) return NULL;
    or_pot *p = (or_pot *)calloc(1, sizeof(or_pot));
    p->n = n;
    p->rc = rc;
    p->rho_max = rho_max;
    p->hr = rc / (double)(n - 1);
    p->hrho = rho_max / (double)(n - 1);
    p->r_floor = 1e-4;
    p->f = (double *)malloc(sizeof(double) * n);
    p->phi = (double *)malloc(sizeof(double) * n);
    p->F = (double *)malloc(sizeof(double) * n);
    p->mf = (double *)malloc(sizeof(double) * n);
    p->mphi = (double *)malloc(sizeof(double) * n);
    p->mF = (double *)malloc(sizeof(double) * n);
    memcpy(p->f, f, sizeof(double) * n);
    memcpy(p->phi, phi, sizeof(double) * n);
    memcpy(p->F, F, sizeof(double) * n);
    or_spline_slopes(p->f, n, p->hr, p->mf);
    or_spline_slopes(p->phi, n, p->hr, p->mphi);
    or_spline_slopes(p->F, n, p->hrho, p->mF);
    return p;
}

void or_pot_free(or_pot *p)
{
    if (!p) return;
    free(p->f); free(p->phi); free(p->F);
    free(p->mf); free(p->mphi); free(p->mF);
    free(p);
}

/* f(r) or phi(r) (which = 0 / 1): zero at and beyond rc. */
static double pair_fn(const or_pot *p, int which, double r, double *d)
{
    if (r >= p->rc) {
        *d = 0.0;
        return 0.0;
    }
    if (r < p->r_floor) r = p->r_floor;
    const double *y = which == 0 ? p->f : p->phi;
    const double *m = which == 0 ? p->mf : p->mphi;
    return or_spline_eval(y, m, p->n, p->hr, r, d);
}

/* Embedding F(rho); linear continuation beyond rho_max. */
static double embed_fn(const or_pot *p, double rho, double *d)
{
    if (rho > p->rho_max) {
        double slope = p->mF[p->n - 1];
        *d = slope;
        return p->F[p->n - 1] + slope * (rho - p->rho_max);
    }
    if (rho < 0.0) rho = 0.0;
    return or_spline_eval(p->F, p->mF, p->n, p->hrho, rho, d);
}

/* which: 0 f(r), 1 phi(r), 2 F(rho). */
double or_pot_eval(const or_pot *p, int which, double x, double *deriv)
{
    double d = 0.0, v;
    if (which == 2) v = embed_fn(p, x, &d);
    else v = pair_fn(p, which, x, &d);
    if (deriv) *deriv = d;
    return v;
}

/* ------------------------------------------------------------------------ */
/* BCC lattice and lattice id (Sec. 3)                                       */
/* ------------------------------------------------------------------------ */

/* Lattice id of site (x, y, z), x in [0, 2 bx): index = 2 bx by z + 2 bx y + x. */
int64_t or_site_index(int bx, int by, int x, int y, int z)
{
    return 2 * (int64_t)bx * by * z + 2 * (int64_t)bx * y + x;
}

/* Inverse of or_site_index plus the Cartesian position of the site: even x
 * is the cube corner of cell (x/2, y, z), odd x the body centre of it. */
void or_site_coords(int bx, int by, int64_t id, int *x, int *y, int *z)
{
    int64_t row = 2 * (int64_t)bx;
    *x = (int)(id % row);
    *y = (int)((id / row) % by);
    *z = (int)(id / (row * by));
}

void or_site_position(int bx, int by, double a0, int64_t id, double r[3])
{
    int x, y, z;
    or_site_coords(bx, by, id, &x, &y, &z);
    double half = (x & 1) ? 0.5 : 0.0;
    r[0] = a0 * ((double)(x / 2) + half);
    r[1] = a0 * ((double)y + half);
    r[2] = a0 * ((double)z + half);
}

static double wrap1(double v, double L)
{
    double w = fmod(v, L);
    if (w < 0.0) w += L;
    if (w >= L) w -= L;
    return w;
}

static int imod(int a, int n)
{
    int r = a % n;
    return r < 0 ? r + n : r;
}

/* The hash function of Sec. 3: the nearest lattice site of a position.
 * Candidates are the nearest cube corner and the nearest body centre; the
 * closer wins, an exact tie goes to the lower lattice id. */
int64_t or_nearest_site(int bx, int by, int bz, double a0, const double p[3])
{
    double s[3], dc = 0.0, de = 0.0;
    int c[3], e[3];
    int nb[3] = {bx, by, bz};
    for (int d = 0; d < 3; ++d) {
        s[d] = p[d] / a0;
        double cr = floor(s[d] + 0.5);
        double ef = floor(s[d]);
        dc += (s[d] - cr) * (s[d] - cr);
        de += (s[d] - ef - 0.5) * (s[d] - ef - 0.5);
        c[d] = imod((int)cr, nb[d]);
        e[d] = imod((int)ef, nb[d]);
    }
    int64_t idc = or_site_index(bx, by, 2 * c[0], c[1], c[2]);
    int64_t ide = or_site_index(bx, by, 2 * e[0] + 1, e[1], e[2]);
    if (dc < de) return idc;
    if (de < dc) return ide;
    return idc < ide ? idc : ide;
}

/* Wigner-Seitz defect count of a configuration (the vacancy / interstitial
 * counts behind the Frenkel-pair curves of Sec. 5.1): every atom belongs to
 * the cell of its nearest lattice site; a site whose cell holds no atom is a
 * vacancy, every atom beyond the first in a cell an interstitial. */
void or_ws_defects(int bx, int by, int bz, double a0, int64_t N, const double *x, int64_t *n_vac, int64_t *n_int)
{
    int64_t ns = 2 * (int64_t)bx * by * bz;
    int64_t *occ = (int64_t *)calloc((size_t)(ns > 0 ? ns : 1), sizeof(int64_t));
    for (int64_t i = 0; i < N; ++i) occ[or_nearest_site(bx, by, bz, a0, x + 3 * i)]++;
    int64_t v = 0, e = 0;
    for (int64_t s = 0; s < ns; ++s) {
        if (occ[s] == 0) ++v;
        if (occ[s] > 1) e += occ[s] - 1;
    }
    free(occ);
    *n_vac = v;
    *n_int = e;
}

/* PKA site of Sec. 5.1: the atom at the box centre, i.e. the cube corner of
 * cell (bx/2, by/2, bz/2). */
int64_t or_pka_site(int bx, int by, int bz)
{
    return or_site_index(bx, by, 2 * (bx / 2), by / 2, bz / 2);
}

/* ------------------------------------------------------------------------ */
/* Pair enumeration: brute force over periodic images, or a cell list        */
/* ------------------------------------------------------------------------ */

typedef struct {
    int64_t N;
    const double *x; /* N*3, wrapped into [0, L) */
    double L[3];
    double rc;
    int mode; /* 0 brute force, 1 cell list */
    /* cell list */
    int nc[3];
    int64_t *cell_start; /* nc0*nc1*nc2 + 1 */
    int64_t *cell_atoms; /* N */
} or_nbr;

static void nbr_init(or_nbr *nb, int64_t N, const double *x, const double L[3], double rc, int mode)
{
    memset(nb, 0, sizeof(*nb));
    nb->N = N;
    nb->x = x;
    nb->rc = rc;
    for (int d = 0; d < 3; ++d) nb->L[d] = L[d];
    nb->mode = mode;
    if (mode == 1) {
        for (int d = 0; d < 3; ++d) {
            nb->nc[d] = (int)floor(L[d] / rc);
            if (nb->nc[d] < 3) nb->mode = 0; /* 27 distinct neighbour cells needed */
        }
    }
    if (nb->mode == 1) {
        int64_t ncell = (int64_t)nb->nc[0] * nb->nc[1] * nb->nc[2];
        nb->cell_start = (int64_t *)calloc((size_t)ncell + 1, sizeof(int64_t));
        nb->cell_atoms = (int64_t *)malloc(sizeof(int64_t) * (size_t)(N > 0 ? N : 1));
        int64_t *cell_of = (int64_t *)malloc(sizeof(int64_t) * (size_t)(N > 0 ? N : 1));
        for (int64_t i = 0; i < N; ++i) {
            int c[3];
            for (int d = 0; d < 3; ++d) {
                c[d] = (int)(x[3 * i + d] / L[d] * nb->nc[d]);
                if (c[d] >= nb->nc[d]) c[d] = nb->nc[d] - 1;
                if (c[d] < 0) c[d] = 0;
            }
            cell_of[i] = ((int64_t)c[2] * nb->nc[1] + c[1]) * nb->nc[0] + c[0];
            nb->cell_start[cell_of[i] + 1]++;
        }
        for (int64_t c = 0; c < ncell; ++c) nb->cell_start[c + 1] += nb->cell_start[c];
        int64_t *fill = (int64_t *)malloc(sizeof(int64_t) * (size_t)ncell);
        memcpy(fill, nb->cell_start, sizeof(int64_t) * (size_t)ncell);
        for (int64_t i = 0; i < N; ++i) nb->cell_atoms[fill[cell_of[i]]++] = i;
        free(fill);
        free(cell_of);
    }
}

static void nbr_free(or_nbr *nb)
{
    free(nb->cell_start);
    free(nb->cell_atoms);
}

/* Calls visit(ctx, j, dvec = x_i - x_j (image), r) for every j != i (or a
 * periodic image of i itself) with r < rc. */
typedef void (*visit_fn)(void *ctx, int64_t j, const double dv[3], double r);

static void nbr_visit(const or_nbr *nb, int64_t i, visit_fn visit, void *ctx)
{
    const double *xi = nb->x + 3 * i;
    double rc2 = nb->rc * nb->rc;
    if (nb->mode == 1) {
        int c[3];
        for (int d = 0; d < 3; ++d) {
            c[d] = (int)(xi[d] / nb->L[d] * nb->nc[d]);
            if (c[d] >= nb->nc[d]) c[d] = nb->nc[d] - 1;
            if (c[d] < 0) c[d] = 0;
        }
        for (int dz = -1; dz <= 1; ++dz)
            for (int dy = -1; dy <= 1; ++dy)
                for (int dx = -1; dx <= 1; ++dx) {
                    int cx = imod(c[0] + dx, nb->nc[0]);
                    int cy = imod(c[1] + dy, nb->nc[1]);
                    int cz = imod(c[2] + dz, nb->nc[2]);
                    int64_t cell = ((int64_t)cz * nb->nc[1] + cy) * nb->nc[0] + cx;
                    for (int64_t q = nb->cell_start[cell]; q < nb->cell_start[cell + 1]; ++q) {
                        int64_t j = nb->cell_atoms[q];
                        if (j == i) continue;
                        double dv[3], r2 = 0.0;
                        for (int d = 0; d < 3; ++d) {
                            double t = xi[d] - nb->x[3 * j + d];
                            t -= nb->L[d] * floor(t / nb->L[d] + 0.5); /* minimum image */
                            dv[d] = t;
                            r2 += t * t;
                        }
                        if (r2 < rc2) visit(ctx, j, dv, sqrt(r2));
                    }
                }
        return;
    }
    /* brute force: every atom, every periodic image within reach */
    int m[3];
    for (int d = 0; d < 3; ++d) m[d] = (int)ceil(nb->rc / nb->L[d]);
    for (int64_t j = 0; j < nb->N; ++j) {
        for (int iz = -m[2]; iz <= m[2]; ++iz)
            for (int iy = -m[1]; iy <= m[1]; ++iy)
                for (int ix = -m[0]; ix <= m[0]; ++ix) {
                    if (j == i && ix == 0 && iy == 0 && iz == 0) continue;
                    double sh[3] = {ix * nb->L[0], iy * nb->L[1], iz * nb->L[2]};
                    double dv[3], r2 = 0.0;
                    for (int d = 0; d < 3; ++d) {
                        dv[d] = xi[d] - (nb->x[3 * j + d] + sh[d]);
                        r2 += dv[d] * dv[d];
                    }
                    if (r2 < rc2) visit(ctx, j, dv, sqrt(r2));
                }
    }
}

/* ------------------------------------------------------------------------ */
/* EAM evaluation: the five steps of Sec. 2.2                                */
/* ------------------------------------------------------------------------ */

typedef struct {
    const or_pot *p;
    const double *Fp;
    double Fpi;
    double rho, ephi, F[3];
} eam_ctx;

static void visit_rho(void *c, int64_t j, const double dv[3], double r)
{
    (void)j; (void)dv;
    eam_ctx *e = (eam_ctx *)c;
    double d;
    e->rho += pair_fn(e->p, 0, r, &d); /* step 1: rho_i = sum_j f(r_ij) */
}

static void visit_force(void *c, int64_t j, const double dv[3], double r)
{
    eam_ctx *e = (eam_ctx *)c;
    double dfr, dphi;
    pair_fn(e->p, 0, r, &dfr);                 /* step 4: f'(r_ij) */
    e->ephi += 0.5 * pair_fn(e->p, 1, r, &dphi); /* step 3: phi'(r_ij); half pair energy */
    if (r < e->p->r_floor) return;             /* direction undefined: no force */
    /* step 5, Eq. eam_force_ij: F_ij = -[F'_i f'(r) + F'_j f'(r) + phi'(r)] (x_i - x_j)/r */
    double s = -((e->Fpi + e->Fp[j]) * dfr + dphi) / r;
    for (int d = 0; d < 3; ++d) e->F[d] += s * dv[d];
}

static void wrap_positions(int64_t N, const double *x, const double L[3], double *out)
{
    for (int64_t i = 0; i < N; ++i)
        for (int d = 0; d < 3; ++d) out[3 * i + d] = wrap1(x[3 * i + d], L[d]);
}

/* Density, embedding derivative, per-atom energy E_i (Eq. eam_base) and force
 * F_i (Eq. eam_force_ij summed over j) of every atom.  Any output may be
 * NULL.  mode 0: brute force over periodic images, 1: cell list. */
int or_eam(const or_pot *p, int64_t N, const double *x, const double L[3], int mode, int nthreads,
           double *rho, double *Fp, double *E, double *F)
{
    if (!p || N < 0) return -1;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
    double *xw = (double *)malloc(sizeof(double) * 3 * (size_t)(N > 0 ? N : 1));
    double *rh = (double *)malloc(sizeof(double) * (size_t)(N > 0 ? N : 1));
    double *fp = (double *)malloc(sizeof(double) * (size_t)(N > 0 ? N : 1));
    double *fe = (double *)malloc(sizeof(double) * (size_t)(N > 0 ? N : 1));
    wrap_positions(N, x, L, xw);
    or_nbr nb;
    nbr_init(&nb, N, xw, L, p->rc, mode);
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t i = 0; i < N; ++i) {
        eam_ctx e = {p, NULL, 0.0, 0.0, 0.0, {0, 0, 0}};
        nbr_visit(&nb, i, visit_rho, &e);
        double d;
        rh[i] = e.rho;
        fe[i] = embed_fn(p, e.rho, &d); /* F(rho_i) */
        fp[i] = d;                      /* step 2: F'(rho_i) */
    }
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t i = 0; i < N; ++i) {
        eam_ctx e = {p, fp, fp[i], 0.0, 0.0, {0, 0, 0}};
        nbr_visit(&nb, i, visit_force, &e);
        if (E) E[i] = fe[i] + e.ephi;
        if (F)
            for (int d = 0; d < 3; ++d) F[3 * i + d] = e.F[d];
    }
    if (rho) memcpy(rho, rh, sizeof(double) * (size_t)N);
    if (Fp) memcpy(Fp, fp, sizeof(double) * (size_t)N);
    nbr_free(&nb);
    free(xw); free(rh); free(fp); free(fe);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Alloys (Sec. 2.2, Eq. eam_base and eam_force_ij with atom types)          */
/* ------------------------------------------------------------------------ */
/* Species a has a density function rho_a(r) and an embedding function
 * F_a(rho); each unordered pair (a, b) a pair function phi_ab(r).  Each is
 * held in an or_pot on the same grids: spec[a] keeps rho_a in f and F_a in F,
 * pair[ab] keeps phi_ab in phi, ab = a n - a (a - 1)/2 + (b - a) for a <= b. */
typedef struct or_alloy {
    int nsp;
    or_pot **spec, **pair;
} or_alloy;

static int pair_slot(int a, int b, int nsp)
{
    if (a > b) {
        int t = a;
        a = b;
        b = t;
    }
    return a * nsp - a * (a - 1) / 2 + (b - a);
}

or_alloy *or_alloy_new(int n, int nsp, double rc, double rho_max, const double *f, const double *F,
                       const double *phi)
{
    if (nsp < 1 || nsp > 8) return NULL;
    int npair = nsp * (nsp + 1) / 2;
    or_alloy *a = (or_alloy *)calloc(1, sizeof(or_alloy));
    a->nsp = nsp;
    a->spec = (or_pot **)calloc((size_t)nsp, sizeof(or_pot *));
    a->pair = (or_pot **)calloc((size_t)npair, sizeof(or_pot *));
    double *zero = (double *)calloc((size_t)n, sizeof(double));
    for (int s = 0; s < nsp; ++s) a->spec[s] = or_pot_new(n, rc, rho_max, f + (size_t)s * n, zero, F + (size_t)s * n);
    for (int q = 0; q < npair; ++q) a->pair[q] = or_pot_new(n, rc, rho_max, zero, phi + (size_t)q * n, zero);
    free(zero);
    return a;
}

void or_alloy_free(or_alloy *a)
{
    if (!a) return;
    for (int s = 0; s < a->nsp; ++s) or_pot_free(a->spec[s]);
    for (int q = 0; q < a->nsp * (a->nsp + 1) / 2; ++q) or_pot_free(a->pair[q]);
    free(a->spec);
    free(a->pair);
    free(a);
}

typedef struct {
    const or_alloy *al;
    const int8_t *type;
    const double *Fp;
    int ti;
    double Fpi;
    double rho, ephi, F[3];
} alloy_ctx;

static void visit_rho_alloy(void *c, int64_t j, const double dv[3], double r)
{
    (void)dv;
    alloy_ctx *e = (alloy_ctx *)c;
    double d;
    e->rho += pair_fn(e->al->spec[e->type[j]], 0, r, &d); /* step 1: rho_i = sum_j rho_{t_j}(r_ij) */
}

static void visit_force_alloy(void *c, int64_t j, const double dv[3], double r)
{
    alloy_ctx *e = (alloy_ctx *)c;
    const int tj = e->type[j];
    double dfj, dfi, dphi;
    pair_fn(e->al->spec[tj], 0, r, &dfj);   /* rho_{t_j}'(r) */
    pair_fn(e->al->spec[e->ti], 0, r, &dfi); /* rho_{t_i}'(r) */
    e->ephi += 0.5 * pair_fn(e->al->pair[pair_slot(e->ti, tj, e->al->nsp)], 1, r, &dphi);
    if (r < e->al->spec[0]->r_floor) return;
    /* Eq. eam_force_ij: -[F'_i rho_j'(r) + F'_j rho_i'(r) + phi_ij'(r)] (x_i - x_j)/r */
    double s = -(e->Fpi * dfj + e->Fp[j] * dfi + dphi) / r;
    for (int d = 0; d < 3; ++d) e->F[d] += s * dv[d];
}

/* or_eam for an alloy: type[i] in [0, nsp) is the species of atom i. */
int or_eam_alloy(const or_alloy *al, int64_t N, const double *x, const int8_t *type, const double L[3], int mode,
                 int nthreads, double *rho, double *Fp, double *E, double *F)
{
    if (!al || N < 0) return -1;
    for (int64_t i = 0; i < N; ++i)
        if (type[i] < 0 || type[i] >= al->nsp) return -2;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
    const size_t n1 = (size_t)(N > 0 ? N : 1);
    double *xw = (double *)malloc(sizeof(double) * 3 * n1);
    double *rh = (double *)malloc(sizeof(double) * n1);
    double *fp = (double *)malloc(sizeof(double) * n1);
    double *fe = (double *)malloc(sizeof(double) * n1);
    wrap_positions(N, x, L, xw);
    or_nbr nb;
    nbr_init(&nb, N, xw, L, al->spec[0]->rc, mode);
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t i = 0; i < N; ++i) {
        alloy_ctx e = {al, type, NULL, type[i], 0.0, 0.0, 0.0, {0, 0, 0}};
        nbr_visit(&nb, i, visit_rho_alloy, &e);
        double d;
        rh[i] = e.rho;
        fe[i] = embed_fn(al->spec[type[i]], e.rho, &d); /* F_{t_i}(rho_i) */
        fp[i] = d;                                       /* step 2 */
    }
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t i = 0; i < N; ++i) {
        alloy_ctx e = {al, type, fp, type[i], fp[i], 0.0, 0.0, {0, 0, 0}};
        nbr_visit(&nb, i, visit_force_alloy, &e);
        if (E) E[i] = fe[i] + e.ephi;
        if (F)
            for (int d = 0; d < 3; ++d) F[3 * i + d] = e.F[d];
    }
    if (rho) memcpy(rho, rh, sizeof(double) * (size_t)N);
    if (Fp) memcpy(Fp, fp, sizeof(double) * (size_t)N);
    nbr_free(&nb);
    free(xw); free(rh); free(fp); free(fe);
    return 0;
}

/* Same quantities for a sample of atoms only (for systems too large for a
 * full oracle pass): each target's density, energy and force, with the
 * embedding derivatives of its neighbours computed on demand.  Cell list. */
typedef struct {
    const or_nbr *nb;
    const or_pot *p;
    double Fpi;
    double ephi, F[3];
} sample_ctx;

static double rho_of(const or_nbr *nb, const or_pot *p, int64_t i)
{
    eam_ctx e = {p, NULL, 0.0, 0.0, 0.0, {0, 0, 0}};
    nbr_visit(nb, i, visit_rho, &e);
    return e.rho;
}

static void visit_sample_force(void *c, int64_t j, const double dv[3], double r)
{
    sample_ctx *s = (sample_ctx *)c;
    double dfr, dphi, dFj;
    embed_fn(s->p, rho_of(s->nb, s->p, j), &dFj);
    pair_fn(s->p, 0, r, &dfr);
    s->ephi += 0.5 * pair_fn(s->p, 1, r, &dphi);
    if (r < s->p->r_floor) return;
    double k = -((s->Fpi + dFj) * dfr + dphi) / r;
    for (int d = 0; d < 3; ++d) s->F[d] += k * dv[d];
}

int or_eam_sample(const or_pot *p, int64_t N, const double *x, const double L[3], int nthreads,
                  int64_t nt, const int64_t *targets, double *rho_t, double *E_t, double *F_t)
{
    if (!p) return -1;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
    double *xw = (double *)malloc(sizeof(double) * 3 * (size_t)(N > 0 ? N : 1));
    wrap_positions(N, x, L, xw);
    or_nbr nb;
    nbr_init(&nb, N, xw, L, p->rc, 1);
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t q = 0; q < nt; ++q) {
        int64_t i = targets[q];
        double rho = rho_of(&nb, p, i), dF;
        double Fi = embed_fn(p, rho, &dF);
        sample_ctx s = {&nb, p, dF, 0.0, {0, 0, 0}};
        nbr_visit(&nb, i, visit_sample_force, &s);
        if (rho_t) rho_t[q] = rho;
        if (E_t) E_t[q] = Fi + s.ephi;
        if (F_t)
            for (int d = 0; d < 3; ++d) F_t[3 * q + d] = s.F[d];
    }
    nbr_free(&nb);
    free(xw);
    return 0;
}

/* Pair list (i < j, image-resolved r) within rc, for pair-set comparisons.
 * Writes up to cap (i, j) pairs and their distances; returns the count. */
typedef struct {
    int64_t i, cap, cnt;
    int64_t *pi, *pj;
    double *pr;
} plist_ctx;

static void visit_plist(void *c, int64_t j, const double dv[3], double r)
{
    (void)dv;
    plist_ctx *pl = (plist_ctx *)c;
    if (j < pl->i) return;
    if (pl->cnt < pl->cap) {
        pl->pi[pl->cnt] = pl->i;
        pl->pj[pl->cnt] = j;
        pl->pr[pl->cnt] = r;
    }
    pl->cnt++;
}

int64_t or_pair_list(int64_t N, const double *x, const double L[3], double rc, int mode, int64_t cap,
                     int64_t *pi, int64_t *pj, double *pr)
{
    double *xw = (double *)malloc(sizeof(double) * 3 * (size_t)(N > 0 ? N : 1));
    wrap_positions(N, x, L, xw);
    or_nbr nb;
    nbr_init(&nb, N, xw, L, rc, mode);
    plist_ctx pl = {0, cap, 0, pi, pj, pr};
    for (int64_t i = 0; i < N; ++i) {
        pl.i = i;
        nbr_visit(&nb, i, visit_plist, &pl);
    }
    nbr_free(&nb);
    free(xw);
    return pl.cnt;
}

/* ------------------------------------------------------------------------ */
/* Molecular dynamics (Fig. 1): velocity Verlet, adaptive timestep, PKA      */
/* ------------------------------------------------------------------------ */

/* Timestep of the next step: dt_max, or the step that moves the fastest atom
 * by dx_max if that is shorter (adaptive timestep, Sec. 1). */
double or_next_dt(int64_t N, const double *v, double dt_max, double dx_max)
{
    if (dx_max <= 0.0) return dt_max;
    double vmax = 0.0;
    for (int64_t i = 0; i < N; ++i) {
        double s = sqrt(v[3 * i] * v[3 * i] + v[3 * i + 1] * v[3 * i + 1] + v[3 * i + 2] * v[3 * i + 2]);
        if (s > vmax) vmax = s;
    }
    if (vmax <= 0.0) return dt_max;
    double dt = dx_max / vmax;
    return dt < dt_max ? dt : dt_max;
}

/* PKA insertion (Sec. 5.1): the atom gets kinetic energy E (eV) along dir. */
void or_insert_pka(double *v, int64_t atom, double mass, double energy, const double dir[3])
{
    double nrm = sqrt(dir[0] * dir[0] + dir[1] * dir[1] + dir[2] * dir[2]);
    double speed = sqrt(2.0 * energy / mass * MISA_O_ACC); /* |v| in A/fs */
    for (int d = 0; d < 3; ++d) v[3 * atom + d] = speed * dir[d] / nrm;
}

/* Kinetic energy in eV. */
double or_kinetic(int64_t N, const double *v, double mass)
{
    double ke = 0.0;
    for (int64_t i = 0; i < N; ++i)
        ke += v[3 * i] * v[3 * i] + v[3 * i + 1] * v[3 * i + 1] + v[3 * i + 2] * v[3 * i + 2];
    return 0.5 * mass * ke / MISA_O_ACC;
}

/* Runs n steps of kick-drift-kick velocity Verlet in the NVE ensemble.
 * x, v (N*3) are updated in place; a (N*3) holds the acceleration of the
 * current positions on entry (computed here if acc_valid == 0) and of the
 * final positions on return.  Per step s (0-based) it may record the
 * timestep, potential and kinetic energy after the step (log: n*3, or NULL).
 * Returns the simulated time. */
double or_md_run(const or_pot *p, int64_t N, double *x, double *v, double *a, int acc_valid,
                 const double L[3], double mass, double dt_max, double dx_max, int nsteps, int mode,
                 int nthreads, double *log)
{
    double *F = (double *)malloc(sizeof(double) * 3 * (size_t)(N > 0 ? N : 1));
    double *E = log ? (double *)malloc(sizeof(double) * (size_t)(N > 0 ? N : 1)) : NULL;
    double conv = MISA_O_ACC / mass;
    if (!acc_valid) {
        or_eam(p, N, x, L, mode, nthreads, NULL, NULL, NULL, F);
        for (int64_t q = 0; q < 3 * N; ++q) a[q] = F[q] * conv;
    }
    double t = 0.0;
    for (int s = 0; s < nsteps; ++s) {
        double dt = or_next_dt(N, v, dt_max, dx_max);
        for (int64_t i = 0; i < N; ++i)
            for (int d = 0; d < 3; ++d) {
                v[3 * i + d] += 0.5 * dt * a[3 * i + d];
                x[3 * i + d] = wrap1(x[3 * i + d] + dt * v[3 * i + d], L[d]);
            }
        or_eam(p, N, x, L, mode, nthreads, NULL, NULL, E, F);
        for (int64_t q = 0; q < 3 * N; ++q) {
            a[q] = F[q] * conv;
            v[q] += 0.5 * dt * a[q];
        }
        t += dt;
        if (log) {
            double pe = 0.0;
            for (int64_t i = 0; i < N; ++i) pe += E[i];
            log[3 * s] = dt;
            log[3 * s + 1] = pe;
            log[3 * s + 2] = or_kinetic(N, v, mass);
        }
    }
    free(F);
    free(E);
    return t;
}

/* ------------------------------------------------------------------------ */
/* Lattice list: hash array + run-away ("hash clash") atoms (Sec. 3)         */
/* ------------------------------------------------------------------------ */
/* Storage only: it never changes physics.  Reading of Alg. 2 used here: an
 * array atom whose displacement from its own site exceeds the skin delta is
 * moved to the run-away list (stricter than "its nearest site changed",
 * which it implies for delta below half the nearest-neighbour distance); a
 * run-away atom whose nearest site is empty and which lies within delta of
 * it is moved back into the array, lowest atom id first.  Assignment from
 * scratch follows the same rules, lowest atom id first. */

typedef struct or_lattice {
    int bx, by, bz;
    double a0, skin;
    int64_t ns;          /* 2 bx by bz sites */
    int64_t *site_atom;  /* atom id or -1 */
    int64_t nra;         /* run-away count */
    int64_t *ra;         /* run-away atom ids, ascending */
} or_lattice;

static double disp2_to_site(const or_lattice *lt, int64_t site, const double p[3])
{
    double r[3], L[3] = {lt->bx * lt->a0, lt->by * lt->a0, lt->bz * lt->a0}, s = 0.0;
    or_site_position(lt->bx, lt->by, lt->a0, site, r);
    for (int d = 0; d < 3; ++d) {
        double t = p[d] - r[d];
        t -= L[d] * floor(t / L[d] + 0.5);
        s += t * t;
    }
    return s;
}

or_lattice *or_lattice_new(int bx, int by, int bz, double a0, double skin)
{
    or_lattice *lt = (or_lattice *)calloc(1, sizeof(or_lattice));
    lt->bx = bx; lt->by = by; lt->bz = bz;
    lt->a0 = a0; lt->skin = skin;
    lt->ns = 2 * (int64_t)bx * by * bz;
    lt->site_atom = (int64_t *)malloc(sizeof(int64_t) * (size_t)lt->ns);
    lt->ra = (int64_t *)malloc(sizeof(int64_t) * (size_t)lt->ns);
    for (int64_t s = 0; s < lt->ns; ++s) lt->site_atom[s] = -1;
    lt->nra = 0;
    return lt;
}

void or_lattice_free(or_lattice *lt)
{
    if (!lt) return;
    free(lt->site_atom);
    free(lt->ra);
    free(lt);
}

/* Assign N atoms (positions x) from scratch. */
void or_lattice_assign(or_lattice *lt, int64_t N, const double *x)
{
    double L[3] = {lt->bx * lt->a0, lt->by * lt->a0, lt->bz * lt->a0};
    for (int64_t s = 0; s < lt->ns; ++s) lt->site_atom[s] = -1;
    lt->nra = 0;
    for (int64_t i = 0; i < N; ++i) {
        double p[3] = {wrap1(x[3 * i], L[0]), wrap1(x[3 * i + 1], L[1]), wrap1(x[3 * i + 2], L[2])};
        int64_t s = or_nearest_site(lt->bx, lt->by, lt->bz, lt->a0, p);
        if (lt->site_atom[s] < 0 && disp2_to_site(lt, s, p) <= lt->skin * lt->skin) lt->site_atom[s] = i;
        else lt->ra[lt->nra++] = i;
    }
}

/* Alg. 2 (hash update) under the reading above. */
void or_lattice_update(or_lattice *lt, int64_t N, const double *x)
{
    (void)N;
    double L[3] = {lt->bx * lt->a0, lt->by * lt->a0, lt->bz * lt->a0};
    /* part 1: demote */
    for (int64_t s = 0; s < lt->ns; ++s) {
        int64_t i = lt->site_atom[s];
        if (i < 0) continue;
        double p[3] = {wrap1(x[3 * i], L[0]), wrap1(x[3 * i + 1], L[1]), wrap1(x[3 * i + 2], L[2])};
        if (disp2_to_site(lt, s, p) > lt->skin * lt->skin) {
            lt->site_atom[s] = -1;
            lt->ra[lt->nra++] = i;
        }
    }
    /* keep the run-away list ordered by atom id (lowest id promoted first) */
    for (int64_t a = 1; a < lt->nra; ++a) {
        int64_t v = lt->ra[a], b = a - 1;
        while (b >= 0 && lt->ra[b] > v) {
            lt->ra[b + 1] = lt->ra[b];
            --b;
        }
        lt->ra[b + 1] = v;
    }
    /* part 2: promote */
    int64_t keep = 0;
    for (int64_t q = 0; q < lt->nra; ++q) {
        int64_t i = lt->ra[q];
        double p[3] = {wrap1(x[3 * i], L[0]), wrap1(x[3 * i + 1], L[1]), wrap1(x[3 * i + 2], L[2])};
        int64_t s = or_nearest_site(lt->bx, lt->by, lt->bz, lt->a0, p);
        if (lt->site_atom[s] < 0 && disp2_to_site(lt, s, p) <= lt->skin * lt->skin) lt->site_atom[s] = i;
        else lt->ra[keep++] = i;
    }
    lt->nra = keep;
}

int64_t or_lattice_site_atom(const or_lattice *lt, int64_t *out)
{
    memcpy(out, lt->site_atom, sizeof(int64_t) * (size_t)lt->ns);
    return lt->ns;
}

int64_t or_lattice_runaways(const or_lattice *lt, int64_t *out)
{
    memcpy(out, lt->ra, sizeof(int64_t) * (size_t)lt->nra);
    return lt->nra;
}

/* Neighbour offset index (Sec. 3): all lattice-id displacements from a site
 * of parity par (0 corner, 1 body centre) to the sites whose lattice vector
 * is at most R long, as (dx, dy, dz) in lattice coordinates (x counts
 * half-cells, y and z whole cells).  Returns the count (<= cap). */
int or_offsets(double a0, double R, int par, int cap, int *dxyz)
{
    int cnt = 0;
    int m = (int)ceil(R / a0) + 1;
    for (int z = -m; z <= m; ++z)
        for (int y = -m; y <= m; ++y)
            for (int x2 = -2 * m - 1; x2 <= 2 * m + 1; ++x2) {
                /* target parity = (par + x2) & 1; its cell = site cell + (x, y, z) */
                int tp = (par + x2) & 1;
                int tcx = (par + x2 - tp) / 2; /* cell shift in x */
                double dxr = (tcx + 0.5 * tp) - 0.5 * par;
                double dyr = (y + 0.5 * tp) - 0.5 * par;
                double dzr = (z + 0.5 * tp) - 0.5 * par;
                double d = a0 * sqrt(dxr * dxr + dyr * dyr + dzr * dzr);
                if (d == 0.0 || d > R) continue;
                if (cnt < cap) {
                    dxyz[3 * cnt] = x2;
                    dxyz[3 * cnt + 1] = y;
                    dxyz[3 * cnt + 2] = z;
                }
                ++cnt;
            }
    return cnt;
}

/* Pair set of the lattice list (Alg. 1, all three parts), with the reading
 * that run-away interactions are symmetric: array atom i gets run-aways too.
 *   part 1: array atom i x array atoms at sites site(i) + offset, offsets
 *           within rc + 2 skin (both displacements are at most skin);
 *   part 2: run-away j x array atoms at sites nearest(j) + offset, offsets
 *           within rc + skin + R_ws (R_ws = sqrt(5)/4 a0 bounds the distance
 *           of any point to its nearest bcc site), and the array atom at
 *           nearest(j) itself;
 *   part 3: run-away x run-away, every pair tested directly.
 * Lists each unordered pair (i < j) within rc once.  Returns the count. */
int64_t or_lattice_pairs(const or_lattice *lt, const double *x, double rc, int64_t cap, int64_t *pi,
                         int64_t *pj, double *pr)
{
    double L[3] = {lt->bx * lt->a0, lt->by * lt->a0, lt->bz * lt->a0};
    int bx = lt->bx, by = lt->by, bz = lt->bz;
    int64_t cnt = 0;
    int off[2][3 * 1024], noff[2], off2[2][3 * 2048], noff2[2];
    double R1 = rc + 2.0 * lt->skin, R2 = rc + lt->skin + sqrt(5.0) / 4.0 * lt->a0;
    for (int par = 0; par < 2; ++par) {
        noff[par] = or_offsets(lt->a0, R1, par, 1024, off[par]);
        noff2[par] = or_offsets(lt->a0, R2, par, 2048, off2[par]);
    }
#define EMIT(I, J)                                                                      \
    do {                                                                                \
        int64_t a_ = (I), b_ = (J);                                                     \
        double r2_ = 0.0;                                                               \
        for (int d = 0; d < 3; ++d) {                                                   \
            double t = wrap1(x[3 * a_ + d], L[d]) - wrap1(x[3 * b_ + d], L[d]);          \
            t -= L[d] * floor(t / L[d] + 0.5);                                          \
            r2_ += t * t;                                                               \
        }                                                                               \
        if (r2_ < rc * rc) {                                                            \
            if (cnt < cap) {                                                            \
                pi[cnt] = a_ < b_ ? a_ : b_;                                            \
                pj[cnt] = a_ < b_ ? b_ : a_;                                            \
                pr[cnt] = sqrt(r2_);                                                    \
            }                                                                           \
            ++cnt;                                                                      \
        }                                                                               \
    } while (0)
    /* part 1 */
    for (int64_t s = 0; s < lt->ns; ++s) {
        int64_t i = lt->site_atom[s];
        if (i < 0) continue;
        int sx, sy, sz;
        or_site_coords(bx, by, s, &sx, &sy, &sz);
        int par = sx & 1;
        for (int k = 0; k < noff[par]; ++k) {
            int tx = imod(sx + off[par][3 * k], 2 * bx);
            int ty = imod(sy + off[par][3 * k + 1], by);
            int tz = imod(sz + off[par][3 * k + 2], bz);
            int64_t t = or_site_index(bx, by, tx, ty, tz);
            int64_t j = lt->site_atom[t];
            if (j < 0 || t <= s) continue; /* each array pair once */
            EMIT(i, j);
        }
    }
    /* part 2 */
    for (int64_t q = 0; q < lt->nra; ++q) {
        int64_t j = lt->ra[q];
        double p[3] = {wrap1(x[3 * j], L[0]), wrap1(x[3 * j + 1], L[1]), wrap1(x[3 * j + 2], L[2])};
        int64_t s = or_nearest_site(bx, by, bz, lt->a0, p);
        if (lt->site_atom[s] >= 0) EMIT(j, lt->site_atom[s]);
        int sx, sy, sz;
        or_site_coords(bx, by, s, &sx, &sy, &sz);
        int par = sx & 1;
        int64_t seen[2048];
        int nseen = 0;
        for (int k = 0; k < noff2[par]; ++k) {
            int tx = imod(sx + off2[par][3 * k], 2 * bx);
            int ty = imod(sy + off2[par][3 * k + 1], by);
            int tz = imod(sz + off2[par][3 * k + 2], bz);
            int64_t t = or_site_index(bx, by, tx, ty, tz);
            /* small boxes: two offsets may wrap onto the same site; visit it once */
            int dup = (t == s);
            for (int u = 0; u < nseen && !dup; ++u) dup = (seen[u] == t);
            if (dup) continue;
            seen[nseen++] = t;
            int64_t i = lt->site_atom[t];
            if (i >= 0) EMIT(j, i);
        }
    }
    /* part 3 */
    for (int64_t q = 0; q < lt->nra; ++q)
        for (int64_t w = q + 1; w < lt->nra; ++w) EMIT(lt->ra[q], lt->ra[w]);
#undef EMIT
    return cnt;
}

/* ------------------------------------------------------------------------ */
/* Knot gradient of a force-matching + energy loss (no paper counterpart)    */
/* ------------------------------------------------------------------------ */
/* Loss over one configuration of N atoms:
 *   L = (1/(3N)) sum_i |F_i - Fref_i|^2 + ((E - Eref)/N)^2
 * where E = sum_i E_i.  grad (3n: f knots, phi knots, F knots) receives
 * dL/d(knot) accumulated (+=).  Returns L.
 * With lambda_i = 2 (F_i - Fref_i)/(3N), sum_i lambda_i . F_i equals minus the
 * derivative of E along the displacement field lambda, so its knot gradient
 * is minus that directional derivative of dE/d(knot); the energy term
 * contributes 2 (E - Eref)/N^2 dE/d(knot).  Plain loops over the brute-force
 * pair enumeration (or the cell list, mode 1). */
typedef struct {
    const or_pot *p;
    const double *xw, *lam, *Fp, *Fpp, *dlrho;
    int64_t i;
    double ce;   /* energy weight 2 (E - Eref)/N^2 */
    double *gf, *gphi;
    double acc;  /* scratch accumulator */
} grad_ctx;

/* D_lambda rho_i = sum_j f'(r_ij) rhat_ij . (lambda_i - lambda_j) */
static void visit_dlrho(void *c, int64_t j, const double dv[3], double r)
{
    grad_ctx *g = (grad_ctx *)c;
    if (r < g->p->r_floor) return;
    double d;
    pair_fn(g->p, 0, r, &d);
    double proj = 0.0;
    for (int k = 0; k < 3; ++k) proj += dv[k] / r * (g->lam[3 * g->i + k] - g->lam[3 * j + k]);
    g->acc += d * proj;
}

static void visit_grad(void *c, int64_t j, const double dv[3], double r)
{
    grad_ctx *g = (grad_ctx *)c;
    const or_pot *p = g->p;
    int64_t i = g->i;
    double rr = r < p->r_floor ? p->r_floor : r;
    double proj = 0.0; /* d r_ij / d eps along lambda */
    if (r >= p->r_floor)
        for (int k = 0; k < 3; ++k) proj += dv[k] / r * (g->lam[3 * i + k] - g->lam[3 * j + k]);
    int idx[8];
    double w[8], dw[8];
    int cnt = or_spline_weights(p->n, p->hr, rr, idx, w, dw);
    for (int q = 0; q < cnt; ++q) {
        /* phi knots: dE/dphi_k = 1/2 sum_{i != j} B_k(r_ij); minus its lambda derivative */
        g->gphi[idx[q]] += 0.5 * g->ce * w[q] - 0.5 * dw[q] * proj;
        /* f knots: dE/df_k = sum_i F'(rho_i) sum_j B_k(r_ij) */
        g->gf[idx[q]] += g->ce * g->Fp[i] * w[q] - (g->Fpp[i] * g->dlrho[i] * w[q] + g->Fp[i] * dw[q] * proj);
    }
}

/* F''(rho) of the embedding spline (second derivative of the Hermite cubic). */
static double embed_dd(const or_pot *p, double rho)
{
    if (rho > p->rho_max) return 0.0;
    if (rho < 0.0) rho = 0.0;
    int s;
    double t;
    seg_of(rho, p->n, p->hrho, &s, &t);
    double h = p->hrho;
    double y0 = p->F[s], y1 = p->F[s + 1], m0 = p->mF[s] * h, m1 = p->mF[s + 1] * h;
    double dd = (12.0 * t - 6.0) * y0 + (6.0 * t - 4.0) * m0 + (-12.0 * t + 6.0) * y1 + (6.0 * t - 2.0) * m1;
    return dd / (h * h);
}

double or_loss_grad(const or_pot *p, int64_t N, const double *x, const double L[3], int mode,
                    const double *Fref, double Eref, double *grad, double *E_out, double *F_out)
{
    int n = p->n;
    double *rho = (double *)malloc(sizeof(double) * (size_t)N);
    double *Fp = (double *)malloc(sizeof(double) * (size_t)N);
    double *Fpp = (double *)malloc(sizeof(double) * (size_t)N);
    double *Ei = (double *)malloc(sizeof(double) * (size_t)N);
    double *F = (double *)malloc(sizeof(double) * 3 * (size_t)N);
    double *lam = (double *)malloc(sizeof(double) * 3 * (size_t)N);
    double *dl = (double *)malloc(sizeof(double) * (size_t)N);
    double *xw = (double *)malloc(sizeof(double) * 3 * (size_t)N);
    or_eam(p, N, x, L, mode, 1, rho, Fp, Ei, F);
    double E = 0.0, lf = 0.0;
    for (int64_t i = 0; i < N; ++i) E += Ei[i];
    for (int64_t q = 0; q < 3 * N; ++q) {
        double d = F[q] - Fref[q];
        lf += d * d;
        lam[q] = 2.0 * d / (3.0 * (double)N);
    }
    double loss = lf / (3.0 * (double)N) + ((E - Eref) / (double)N) * ((E - Eref) / (double)N);
    double ce = 2.0 * (E - Eref) / ((double)N * (double)N);
    for (int64_t i = 0; i < N; ++i) Fpp[i] = embed_dd(p, rho[i]);
    wrap_positions(N, x, L, xw);
    or_nbr nb;
    nbr_init(&nb, N, xw, L, p->rc, mode);
    grad_ctx g = {p, xw, lam, Fp, Fpp, dl, 0, ce, grad, grad + n, 0.0};
    for (int64_t i = 0; i < N; ++i) {
        g.i = i;
        g.acc = 0.0;
        nbr_visit(&nb, i, visit_dlrho, &g);
        dl[i] = g.acc;
    }
    for (int64_t i = 0; i < N; ++i) {
        g.i = i;
        nbr_visit(&nb, i, visit_grad, &g);
        /* F knots: dE/dF_k = sum_i B_k(rho_i); lambda derivative B'_k(rho_i) D rho_i */
        if (rho[i] > p->rho_max) {
            /* linear continuation: F = y_{n-1} + m_{n-1} (rho - rho_max) */
            int idx[8];
            double w[8], dw[8];
            int cnt = or_spline_weights(n, p->hrho, p->rho_max, idx, w, dw);
            double ex = rho[i] - p->rho_max;
            for (int q = 0; q < cnt; ++q)
                grad[2 * n + idx[q]] += ce * (w[q] + dw[q] * ex) - dw[q] * dl[i];
        } else {
            int idx[8];
            double w[8], dw[8];
            int cnt = or_spline_weights(n, p->hrho, rho[i] < 0.0 ? 0.0 : rho[i], idx, w, dw);
            for (int q = 0; q < cnt; ++q) grad[2 * n + idx[q]] += ce * w[q] - dw[q] * dl[i];
        }
    }
    nbr_free(&nb);
    if (E_out) *E_out = E;
    if (F_out) memcpy(F_out, F, sizeof(double) * 3 * (size_t)N);
    free(rho); free(Fp); free(Fpp); free(Ei); free(F); free(lam); free(dl); free(xw);
    return loss;
}

int or_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
