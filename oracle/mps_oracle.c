/*
 * mps_oracle.c -- plain, slow, FP64 CPU oracle of one MPS time step.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check and the bench's CPU
 * baseline may load this file's library.  It shares no code, header, table or constant
 * generator with the GB300 library; each side is written from the paper independently.
 *
 * Paper: Vieira-e-Silva et al., "A fluid simulation system based on the MPS method"
 * (arXiv 2105.01677).  Each function cites the passage it follows.  Where the paper is
 * silent or ambiguous, the reading adopted is stated beside the code.
 *
 * Compiled with -O2 -ffp-contract=off: no fused multiply-add anywhere, so every product
 * and sum is one IEEE-754 binary64 rounding.  The per-particle loops carry OpenMP pragmas
 * (each iteration writes only its own outputs, so results do not depend on thread count);
 * every reduction that feeds a result (dot products, sums over neighbours) is sequential
 * in ascending particle id.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_FLUID 0
#define ORC_WALL 1
#define ORC_DUMMY 2
#define ORC_GHOST 3

#define ORC_OK 0
#define ORC_EINVAL -1
#define ORC_ENOMEM -2
#define ORC_ECG_NOCONV -3
#define ORC_ENONFINITE -4
#define ORC_ESKIN -5
#define ORC_ECOINCIDENT -6
#define ORC_ECAP -7

typedef struct {
    int32_t dim;
    int32_t pressure_mode;   /* 0 = PPE (fully incompressible), 1 = equation of state (WC) */
    double l0, re_n, re_lap, rho, nu, dt, beta;
    double g[3];
    double c0, gamma;
    double alpha_c;          /* compressibility coefficient of the PPE diagonal term */
    double cg_tol;
    int32_t cg_max_iter;
    int32_t clamp_negative_p;
    double cell_skin;
    double box_min[3], box_max[3];
    /* Two-phase (multi-density, multi-viscosity) flow, Sec. 3.2.1: per-particle density  */
    /* and kinematic viscosity in particle order, or NULL for the uniform rho and nu.    */
    const double* rho_i;
    const double* nu_i;
    /* Numerical options of Sec. 3.1 / 3.3:                                               */
    int32_t kernel;          /* 0: w of Eq. 4 (re/r - 1); 1: the WC kernel (1 - r/re)^3     */
    int32_t grad_form;       /* 0: difference form with p_hat_i; 1: CMPS, Eq. 18           */
    int32_t source;          /* PPE source: 0 Eq. 13; 1 HS, Eq. 21; 2 HS + ECS, Eq. 24-25  */
    int32_t pad0;
} orc_params;

static double rho_of(const orc_params* p, int64_t i) { return p->rho_i ? p->rho_i[i] : p->rho; }
static double nu_of(const orc_params* p, int64_t i) { return p->nu_i ? p->nu_i[i] : p->nu; }

typedef struct {
    int32_t cg_iters;
    int32_t cg_restarts;
    double cg_resid;          /* true relative residual ||b - A x|| / ||b|| at exit */
    double n0_pnd, n0_lap, lambda;
    double max_disp;
    int64_t n_surface;
    int64_t n_ghost;
    int64_t n_ppe_rows;
} orc_report;

void orc_set_threads(int n) {
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

int orc_get_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ------------------------------------------------------------------------------------ */
/* Kernel weight, Eq. 4: w(r) = re/r - 1 for 0 <= r < re, else 0 (kernel 0); the       */
/* kernel the paper recommends with the equation of state (Sec. 3.1):                   */
/* w(r) = (1 - r/re)^3 for 0 <= r < re, else 0 (kernel 1).                              */
/* ------------------------------------------------------------------------------------ */
static double weight(double r, double re, int kernel) {
    if (r >= re) return 0.0;
    if (kernel == 1) {
        double t = 1.0 - r / re;
        return t * t * t;
    }
    return re / r - 1.0;
}

/* Squared distance of an offset, summed in the fixed order ((dx*dx)+(dy*dy))+(dz*dz).  */
static double dist2(double dx, double dy, double dz) {
    double s = dx * dx;
    s = s + dy * dy;
    s = s + dz * dz;
    return s;
}

/* ------------------------------------------------------------------------------------ */
/* Reference density n0 and lambda (Eq. 5 and the lambda of Eq. 7) on an ideal lattice. */
/* n0 = sum of w(|o| l0) over integer offsets o != 0 with |o| l0 < re (Eq. 5 evaluated  */
/* at an interior particle of an unjittered lattice of spacing l0);                     */
/* lambda = sum w r^2 / sum w over the same offsets (Eq. 7: weighted mean of r_ij^2).   */
/* ------------------------------------------------------------------------------------ */
int orc_lattice(int32_t dim, double l0, double re, double* n0_out, double* lambda_out,
                int32_t kernel) {
    if ((dim != 2 && dim != 3) || !(l0 > 0.0) || !(re > 0.0)) return ORC_EINVAL;
    int m = (int)ceil(re / l0) + 1;
    int mz = (dim == 3) ? m : 0;
    double sw = 0.0, swr2 = 0.0;
    for (int a = -m; a <= m; a++)
        for (int b = -m; b <= m; b++)
            for (int c = -mz; c <= mz; c++) {
                if (a == 0 && b == 0 && c == 0) continue;
                double r2 = dist2(a * l0, b * l0, c * l0);
                if (!(r2 < re * re)) continue;
                double w = weight(sqrt(r2), re, kernel);
                sw = sw + w;
                swr2 = swr2 + w * r2;
            }
    if (n0_out) *n0_out = sw;
    if (lambda_out) *lambda_out = (sw > 0.0) ? swr2 / sw : 0.0;
    return ORC_OK;
}

/* ------------------------------------------------------------------------------------ */
/* Background cell grid (Sec. 4.1, cell-linked list).  Side h = max(re_n, re_lap)(1+s). */
/* Cell coordinate per axis c = floor((x - box_min)/h); a particle whose coordinate is   */
/* outside [0, ncell) on any axis is outside the grid and becomes a GHOST.  The cell's   */
/* Morton key interleaves the bits of (cx, cy[, cz]) with x in the least-significant     */
/* position.                                                                             */
/* ------------------------------------------------------------------------------------ */
static double cell_side(const orc_params* p) {
    double re = p->re_n > p->re_lap ? p->re_n : p->re_lap;
    return re * (1.0 + p->cell_skin);
}

static int grid_dims(const orc_params* p, int32_t ncell[3], int32_t* bits) {
    double h = cell_side(p);
    int maxc = 1;
    for (int a = 0; a < 3; a++) {
        if (a >= p->dim) { ncell[a] = 1; continue; }
        double ext = p->box_max[a] - p->box_min[a];
        if (!(ext > 0.0)) return ORC_EINVAL;
        double q = floor(ext / h) + 1.0;
        if (q > 65536.0) return ORC_EINVAL;
        ncell[a] = (int32_t)q;
        if (ncell[a] > maxc) maxc = ncell[a];
    }
    int b = 0;
    while ((1 << b) < maxc) b++;
    if (b == 0) b = 1;
    if (b * p->dim > 32) return ORC_EINVAL;
    *bits = b;
    return ORC_OK;
}

static uint32_t morton(const int32_t c[3], int dim, int bits) {
    uint32_t key = 0;
    for (int k = 0; k < bits; k++)
        for (int a = 0; a < dim; a++)
            key |= (uint32_t)((c[a] >> k) & 1) << (k * dim + a);
    return key;
}

/* cell_key[i] = Morton key, or 0xFFFFFFFF for a particle outside the grid or a GHOST.   */
int orc_cell_keys(const orc_params* p, int64_t n, const double* pos, const int8_t* type,
                  uint32_t* cell_key, int32_t* cell_xyz) {
    int32_t ncell[3], bits;
    int rc = grid_dims(p, ncell, &bits);
    if (rc) return rc;
    double h = cell_side(p);
    for (int64_t i = 0; i < n; i++) {
        int32_t c[3] = {0, 0, 0};
        int inside = (type[i] != ORC_GHOST);
        for (int a = 0; a < p->dim && inside; a++) {
            double q = floor((pos[i * p->dim + a] - p->box_min[a]) / h);
            if (!(q >= 0.0 && q < (double)ncell[a])) inside = 0;
            else c[a] = (int32_t)q;
        }
        if (cell_xyz) for (int a = 0; a < 3; a++) cell_xyz[i * 3 + a] = inside ? c[a] : -1;
        cell_key[i] = inside ? morton(c, p->dim, bits) : 0xFFFFFFFFu;
    }
    return ORC_OK;
}

/* ------------------------------------------------------------------------------------ */
/* Neighbour sets (Sec. 4.1).  j is a neighbour of i iff j != i, neither is a GHOST and  */
/* ((dx*dx)+(dy*dy))+(dz*dz) < re*re with d = r_j - r_i, all in binary64 (w = 0 at      */
/* r >= re, Eq. 4).  Rows are returned in ascending id order.                            */
/* mode 0: brute force over all pairs.  mode 1: plain cell-linked list of side re.       */
/* ------------------------------------------------------------------------------------ */
typedef struct {
    int64_t* off;   /* n+1 */
    int32_t* ids;
} csr_t;

static void csr_free(csr_t* c) { free(c->off); free(c->ids); c->off = NULL; c->ids = NULL; }

static int cmp_i32(const void* a, const void* b) {
    int32_t x = *(const int32_t*)a, y = *(const int32_t*)b;
    return (x > y) - (x < y);
}

static void coords(const double* pos, int dim, int64_t i, double* x, double* y, double* z) {
    *x = pos[i * dim + 0];
    *y = pos[i * dim + 1];
    *z = (dim == 3) ? pos[i * dim + 2] : 0.0;
}

static int is_pair(const double* pos, int dim, int64_t i, int64_t j, double re2) {
    double xi, yi, zi, xj, yj, zj;
    coords(pos, dim, i, &xi, &yi, &zi);
    coords(pos, dim, j, &xj, &yj, &zj);
    return dist2(xj - xi, yj - yi, zj - zi) < re2;
}

static int neighbors_brute(int dim, int64_t n, const double* pos, const int8_t* type, double re,
                           csr_t* out) {
    double re2 = re * re;
    int64_t* cnt = calloc((size_t)n + 1, sizeof(int64_t));
    if (!cnt) return ORC_ENOMEM;
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t i = 0; i < n; i++) {
        if (type[i] == ORC_GHOST) continue;
        int64_t c = 0;
        for (int64_t j = 0; j < n; j++)
            if (j != i && type[j] != ORC_GHOST && is_pair(pos, dim, i, j, re2)) c++;
        cnt[i + 1] = c;
    }
    for (int64_t i = 0; i < n; i++) cnt[i + 1] += cnt[i];
    int32_t* ids = malloc(sizeof(int32_t) * (size_t)(cnt[n] > 0 ? cnt[n] : 1));
    if (!ids) { free(cnt); return ORC_ENOMEM; }
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t i = 0; i < n; i++) {
        if (type[i] == ORC_GHOST) continue;
        int64_t k = cnt[i];
        for (int64_t j = 0; j < n; j++)
            if (j != i && type[j] != ORC_GHOST && is_pair(pos, dim, i, j, re2)) ids[k++] = (int32_t)j;
    }
    out->off = cnt;
    out->ids = ids;
    return ORC_OK;
}

static int neighbors_cells(int dim, int64_t n, const double* pos, const int8_t* type, double re,
                           csr_t* out) {
    double re2 = re * re;
    double lo[3] = {0, 0, 0}, hi[3] = {0, 0, 0};
    int any = 0;
    for (int64_t i = 0; i < n; i++) {
        if (type[i] == ORC_GHOST) continue;
        double x[3];
        coords(pos, dim, i, &x[0], &x[1], &x[2]);
        for (int a = 0; a < 3; a++) {
            if (!any || x[a] < lo[a]) lo[a] = x[a];
            if (!any || x[a] > hi[a]) hi[a] = x[a];
        }
        any = 1;
    }
    int64_t nc[3];
    for (int a = 0; a < 3; a++) nc[a] = (int64_t)floor((hi[a] - lo[a]) / re) + 1;
    int64_t ncell = nc[0] * nc[1] * nc[2];
    int64_t* head = malloc(sizeof(int64_t) * (size_t)(ncell > 0 ? ncell : 1));
    int64_t* next = malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
    int64_t* cid = malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
    int64_t* cnt = calloc((size_t)n + 1, sizeof(int64_t));
    if (!head || !next || !cid || !cnt) { free(head); free(next); free(cid); free(cnt); return ORC_ENOMEM; }
    for (int64_t c = 0; c < ncell; c++) head[c] = -1;
    /* insert in descending id order so each cell's list runs in ascending id order */
    for (int64_t i = n - 1; i >= 0; i--) {
        cid[i] = -1;
        if (type[i] == ORC_GHOST) continue;
        double x[3];
        coords(pos, dim, i, &x[0], &x[1], &x[2]);
        int64_t c[3];
        for (int a = 0; a < 3; a++) {
            c[a] = (int64_t)floor((x[a] - lo[a]) / re);
            if (c[a] < 0) c[a] = 0;
            if (c[a] >= nc[a]) c[a] = nc[a] - 1;
        }
        cid[i] = c[0] + nc[0] * (c[1] + nc[1] * c[2]);
        next[i] = head[cid[i]];
        head[cid[i]] = i;
    }
    for (int pass = 0; pass < 2; pass++) {
        int32_t* ids = NULL;
        if (pass == 1) {
            for (int64_t i = 0; i < n; i++) cnt[i + 1] += cnt[i];
            ids = malloc(sizeof(int32_t) * (size_t)(cnt[n] > 0 ? cnt[n] : 1));
            if (!ids) { free(head); free(next); free(cid); free(cnt); return ORC_ENOMEM; }
            out->ids = ids;
        }
#pragma omp parallel for schedule(dynamic, 64)
        for (int64_t i = 0; i < n; i++) {
            if (cid[i] < 0) continue;
            int64_t cx = cid[i] % nc[0], cy = (cid[i] / nc[0]) % nc[1], cz = cid[i] / (nc[0] * nc[1]);
            int64_t k = (pass == 1) ? cnt[i] : 0;
            for (int64_t dz = -1; dz <= 1; dz++)
                for (int64_t dy = -1; dy <= 1; dy++)
                    for (int64_t dx = -1; dx <= 1; dx++) {
                        int64_t x = cx + dx, y = cy + dy, z = cz + dz;
                        if (x < 0 || y < 0 || z < 0 || x >= nc[0] || y >= nc[1] || z >= nc[2]) continue;
                        for (int64_t j = head[x + nc[0] * (y + nc[1] * z)]; j >= 0; j = next[j]) {
                            if (j == i || !is_pair(pos, dim, i, j, re2)) continue;
                            if (pass == 0) k++;
                            else out->ids[k++] = (int32_t)j;
                        }
                    }
            if (pass == 0) cnt[i + 1] = k;
            else qsort(out->ids + cnt[i], (size_t)(k - cnt[i]), sizeof(int32_t), cmp_i32);
        }
    }
    free(head); free(next); free(cid);
    out->off = cnt;
    return ORC_OK;
}

static int neighbors(int dim, int64_t n, const double* pos, const int8_t* type, double re,
                     int mode, csr_t* out) {
    return mode == 0 ? neighbors_brute(dim, n, pos, type, re, out)
                     : neighbors_cells(dim, n, pos, type, re, out);
}

/* Exported neighbour sets: offsets[n+1]; ids filled only if ids != NULL and cap fits.   */
int orc_neighbors(int32_t dim, int64_t n, const double* pos, const int8_t* type, double re,
                  int32_t mode, int64_t* offsets, int32_t* ids, int64_t cap) {
    csr_t c = {0, 0};
    int rc = neighbors(dim, n, pos, type, re, mode, &c);
    if (rc) return rc;
    memcpy(offsets, c.off, sizeof(int64_t) * (size_t)(n + 1));
    if (ids) {
        if (c.off[n] > cap) { csr_free(&c); return ORC_ECAP; }
        memcpy(ids, c.ids, sizeof(int32_t) * (size_t)c.off[n]);
    }
    csr_free(&c);
    return ORC_OK;
}

/* ------------------------------------------------------------------------------------ */
/* Particle number density, Eq. 5: n_i = sum_{j != i} w(|r_j - r_i|), every non-GHOST   */
/* neighbour counted (fluid, wall and dummy alike).                                     */
/* ------------------------------------------------------------------------------------ */
static void pnd_from(int dim, int64_t n, const double* pos, const int8_t* type, double re,
                     int kernel, const csr_t* nb, double* nd) {
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; i++) {
        double s = 0.0;
        if (type[i] != ORC_GHOST) {
            double xi, yi, zi;
            coords(pos, dim, i, &xi, &yi, &zi);
            for (int64_t k = nb->off[i]; k < nb->off[i + 1]; k++) {
                int64_t j = nb->ids[k];
                double xj, yj, zj;
                coords(pos, dim, j, &xj, &yj, &zj);
                s = s + weight(sqrt(dist2(xj - xi, yj - yi, zj - zi)), re, kernel);
            }
        }
        nd[i] = s;
    }
}

int orc_pnd(int32_t dim, int64_t n, const double* pos, const int8_t* type, double re,
            int32_t mode, double* nd, int32_t kernel) {
    csr_t nb = {0, 0};
    int rc = neighbors(dim, n, pos, type, re, mode, &nb);
    if (rc) return rc;
    pnd_from(dim, n, pos, type, re, kernel, &nb, nd);
    csr_free(&nb);
    return ORC_OK;
}

/* ------------------------------------------------------------------------------------ */
/* Laplacian model, Eq. 7: lap(phi)_i = 2d/(n0 lambda) sum_{j != i} (phi_j - phi_i) w.   */
/* Neighbours j of every non-GHOST kind enter (walls and dummies carry their own phi).  */
/* ------------------------------------------------------------------------------------ */
static void laplacian_from(int dim, int64_t n, const double* pos, const int8_t* type, double re,
                           int kernel, double n0, double lambda, const csr_t* nb,
                           const double* phi, int ncomp, double* out) {
    double coef = (2.0 * dim) / (n0 * lambda);
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; i++) {
        double xi, yi, zi;
        coords(pos, dim, i, &xi, &yi, &zi);
        for (int c = 0; c < ncomp; c++) {
            double s = 0.0;
            if (type[i] != ORC_GHOST) {
                for (int64_t k = nb->off[i]; k < nb->off[i + 1]; k++) {
                    int64_t j = nb->ids[k];
                    double xj, yj, zj;
                    coords(pos, dim, j, &xj, &yj, &zj);
                    double w = weight(sqrt(dist2(xj - xi, yj - yi, zj - zi)), re, kernel);
                    s = s + (phi[j * ncomp + c] - phi[i * ncomp + c]) * w;
                }
            }
            out[i * ncomp + c] = coef * s;
        }
    }
}

int orc_laplacian(int32_t dim, int64_t n, const double* pos, const int8_t* type, double re,
                  double n0, double lambda, const double* phi, int32_t ncomp, double* out,
                  int32_t kernel) {
    csr_t nb = {0, 0};
    int rc = neighbors(dim, n, pos, type, re, 1, &nb);
    if (rc) return rc;
    laplacian_from(dim, n, pos, type, re, kernel, n0, lambda, &nb, phi, ncomp, out);
    csr_free(&nb);
    return ORC_OK;
}

/* ------------------------------------------------------------------------------------ */
/* Pressure gradient, the difference form of Eq. (multi-density gradient, Sec. 3.2.1)   */
/* with a single density and the minimum-pressure stabilisation p_hat:                   */
/*   grad p_i = d/n0 sum_{j != i, j not DUMMY} (p_j - p_hat_i) / r_ij^2 * r_ij * w(r_ij) */
/* with r_ij = r_j - r_i (form 0), or the antisymmetric CMPS gradient of Eq. 18 (form   */
/* 1), whose pair term ((p_i + p_j) - (p_hat_i + p_hat_j)) w / r_ij^2 is symmetric in    */
/* i, j, so that the pair forces cancel and linear momentum is conserved.               */
/* ------------------------------------------------------------------------------------ */
static void gradient_from(int dim, int64_t n, const double* pos, const int8_t* type, double re,
                          int kernel, int form, double n0, const csr_t* nb, const double* p,
                          const double* phat, double* out) {
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; i++) {
        double s[3] = {0.0, 0.0, 0.0};
        if (type[i] != ORC_GHOST) {
            double xi, yi, zi;
            coords(pos, dim, i, &xi, &yi, &zi);
            for (int64_t k = nb->off[i]; k < nb->off[i + 1]; k++) {
                int64_t j = nb->ids[k];
                if (type[j] == ORC_DUMMY) continue;
                double xj, yj, zj;
                coords(pos, dim, j, &xj, &yj, &zj);
                double d[3] = {xj - xi, yj - yi, zj - zi};
                double r2 = dist2(d[0], d[1], d[2]);
                double w = weight(sqrt(r2), re, kernel);
                double f = (form == 1) ? ((p[i] + p[j]) - (phat[i] + phat[j])) / r2 * w
                                       : (p[j] - phat[i]) / r2 * w;
                for (int a = 0; a < 3; a++) s[a] = s[a] + f * d[a];
            }
        }
        for (int a = 0; a < dim; a++) out[i * dim + a] = ((double)dim / n0) * s[a];
    }
}

int orc_gradient(int32_t dim, int64_t n, const double* pos, const int8_t* type, double re,
                 double n0, const double* p, const double* phat, double* out, int32_t kernel,
                 int32_t form) {
    csr_t nb = {0, 0};
    int rc = neighbors(dim, n, pos, type, re, 1, &nb);
    if (rc) return rc;
    gradient_from(dim, n, pos, type, re, kernel, form, n0, &nb, p, phat, out);
    csr_free(&nb);
    return ORC_OK;
}

/* ------------------------------------------------------------------------------------ */
/* PPE assembly (Eq. 13 with the Laplacian of Eq. 7, the matrix layout of the CUDA PPE  */
/* listing of Sec. 4.3).  Rows P = FLUID/WALL particles not on the free surface.        */
/*   c_ij = 2d/(n0_lap lambda rho) w(r_ij), j a non-DUMMY neighbour within re_lap;      */
/*   A_ii = sum_j c_ij + alpha_c/dt^2;  A_ij = -c_ij when j is in P (p_j = 0 otherwise); */
/*   b_i  = (1/dt^2) (n*_i - n0)/n0.                                                    */
/* Rows outside P are identity rows with b = 0, so A is N x N, symmetric positive       */
/* definite for alpha_c > 0, and x = 0 there.                                            */
/* Column order inside a row: diagonal first, then ascending id.                        */
/* ------------------------------------------------------------------------------------ */
typedef struct {
    int64_t* off;
    int32_t* col;
    double* val;
} mat_t;

static void mat_free(mat_t* m) { free(m->off); free(m->col); free(m->val); }

static int in_ppe(const int8_t* type, const uint8_t* flags, int64_t i) {
    return (type[i] == ORC_FLUID || type[i] == ORC_WALL) && !(flags[i] & 1);
}

/* Two-phase (per-particle densities given): the 1/rho of the Laplacian becomes the pair */
/* factor 2/(rho_i + rho_j) (the reciprocal of the pair's mean density), which keeps A    */
/* symmetric:  c_ij = (2d/(n0_lap lambda)) (2/(rho_i + rho_j)) w(r_ij).                   */
static int assemble_ppe(const orc_params* p, int64_t n, const double* pos, const int8_t* type,
                        const uint8_t* flags, const csr_t* nb_lap, double n0_lap, double lambda,
                        mat_t* A) {
    int dim = p->dim;
    double coef = (2.0 * dim) / (n0_lap * lambda * p->rho);
    double coef0 = (2.0 * dim) / (n0_lap * lambda);
    A->off = calloc((size_t)n + 1, sizeof(int64_t));
    if (!A->off) return ORC_ENOMEM;
    for (int64_t i = 0; i < n; i++) {
        int64_t c = 1;
        if (in_ppe(type, flags, i))
            for (int64_t k = nb_lap->off[i]; k < nb_lap->off[i + 1]; k++)
                if (in_ppe(type, flags, nb_lap->ids[k])) c++;
        A->off[i + 1] = A->off[i] + c;
    }
    A->col = malloc(sizeof(int32_t) * (size_t)A->off[n]);
    A->val = malloc(sizeof(double) * (size_t)A->off[n]);
    if (!A->col || !A->val) { mat_free(A); return ORC_ENOMEM; }
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; i++) {
        int64_t k0 = A->off[i];
        A->col[k0] = (int32_t)i;
        if (!in_ppe(type, flags, i)) { A->val[k0] = 1.0; continue; }
        double xi, yi, zi;
        coords(pos, dim, i, &xi, &yi, &zi);
        double diag = 0.0;
        int64_t k = k0 + 1;
        for (int64_t q = nb_lap->off[i]; q < nb_lap->off[i + 1]; q++) {
            int64_t j = nb_lap->ids[q];
            if (type[j] == ORC_DUMMY) continue;
            double xj, yj, zj;
            coords(pos, dim, j, &xj, &yj, &zj);
            double w = weight(sqrt(dist2(xj - xi, yj - yi, zj - zi)), p->re_lap, p->kernel);
            double c = p->rho_i ? (coef0 * (2.0 / (p->rho_i[i] + p->rho_i[j]))) * w : coef * w;
            diag = diag + c;
            if (in_ppe(type, flags, j)) {
                A->col[k] = (int32_t)j;
                A->val[k] = -c;
                k++;
            }
        }
        A->val[k0] = diag + p->alpha_c / (p->dt * p->dt);
    }
    return ORC_OK;
}

static void spmv(int64_t n, const mat_t* A, const double* x, double* y) {
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; i++) {
        double s = 0.0;
        for (int64_t k = A->off[i]; k < A->off[i + 1]; k++) s = s + A->val[k] * x[A->col[k]];
        y[i] = s;
    }
}

static double dot(int64_t n, const double* a, const double* b) {
    double s = 0.0;
    for (int64_t i = 0; i < n; i++) s = s + a[i] * b[i];
    return s;
}

/* ------------------------------------------------------------------------------------ */
/* Conjugate gradients on A x = b (Sec. 3.1.2 solves the PPE by a CG method; the        */
/* incomplete-Cholesky preconditioner is not used here).  x0 = 0.  Stop when the        */
/* recurrence residual satisfies ||r||/||b|| <= tol; then the true residual b - A x is  */
/* recomputed; if it is still above tol, CG restarts from x with that residual.  At     */
/* most cg_max_iter iterations in total.                                                 */
/* ------------------------------------------------------------------------------------ */
static int cg_solve(int64_t n, const mat_t* A, const double* b, double* x, double tol, int max_iter,
                    int* iters_out, int* restarts_out, double* resid_out) {
    double* r = malloc(sizeof(double) * (size_t)n);
    double* d = malloc(sizeof(double) * (size_t)n);
    double* q = malloc(sizeof(double) * (size_t)n);
    if (!r || !d || !q) { free(r); free(d); free(q); return ORC_ENOMEM; }
    for (int64_t i = 0; i < n; i++) x[i] = 0.0;
    double bnorm = sqrt(dot(n, b, b));
    int it = 0, restarts = 0, rc = ORC_OK;
    double rel = 0.0;
    if (bnorm == 0.0) goto done;
    for (;;) {
        spmv(n, A, x, q);
        for (int64_t i = 0; i < n; i++) r[i] = b[i] - q[i];
        double rho = dot(n, r, r);
        rel = sqrt(rho) / bnorm;
        if (rel <= tol) break;
        if (it >= max_iter) { rc = ORC_ECG_NOCONV; break; }
        if (it > 0) restarts++;
        for (int64_t i = 0; i < n; i++) d[i] = r[i];
        while (it < max_iter) {
            spmv(n, A, d, q);
            double alpha = rho / dot(n, d, q);
            for (int64_t i = 0; i < n; i++) x[i] = x[i] + alpha * d[i];
            for (int64_t i = 0; i < n; i++) r[i] = r[i] - alpha * q[i];
            double rho_new = dot(n, r, r);
            it++;
            if (sqrt(rho_new) / bnorm <= tol) break;
            double beta = rho_new / rho;
            for (int64_t i = 0; i < n; i++) d[i] = r[i] + beta * d[i];
            rho = rho_new;
        }
    }
done:
    *iters_out = it;
    *restarts_out = restarts;
    *resid_out = rel;
    free(r); free(d); free(q);
    return rc;
}

/* Dense Cholesky solve for small SPD systems (cross-check of CG); -1 if not SPD.      */
int orc_dense_spd_solve(int64_t n, double* a, const double* b, double* x) {
    for (int64_t j = 0; j < n; j++) {
        double s = a[j * n + j];
        for (int64_t k = 0; k < j; k++) s = s - a[j * n + k] * a[j * n + k];
        if (!(s > 0.0)) return -1;
        double ljj = sqrt(s);
        a[j * n + j] = ljj;
        for (int64_t i = j + 1; i < n; i++) {
            double t = a[i * n + j];
            for (int64_t k = 0; k < j; k++) t = t - a[i * n + k] * a[j * n + k];
            a[i * n + j] = t / ljj;
        }
    }
    for (int64_t i = 0; i < n; i++) {
        double t = b[i];
        for (int64_t k = 0; k < i; k++) t = t - a[i * n + k] * x[k];
        x[i] = t / a[i * n + i];
    }
    for (int64_t i = n - 1; i >= 0; i--) {
        double t = x[i];
        for (int64_t k = i + 1; k < n; k++) t = t - a[k * n + i] * x[k];
        x[i] = t / a[i * n + i];
    }
    return 0;
}

/* ------------------------------------------------------------------------------------ */
/* Weakly-compressible pressure, Eq. 16: p = rho c0^2/gamma ((n* / n0)^gamma - 1) on    */
/* FLUID/WALL particles not on the free surface; 0 elsewhere.  Two-phase (Sec. 3.2.1):   */
/* p_i = rho_i alpha_i with alpha_i = c0^2/gamma ((n*_i/n0)^gamma - 1), the particle's  */
/* own density.                                                                          */
/* ------------------------------------------------------------------------------------ */
static double wc_pressure(const orc_params* p, double rho, double nstar, double n0) {
    return rho * p->c0 * p->c0 / p->gamma * (pow(nstar / n0, p->gamma) - 1.0);
}

/* ------------------------------------------------------------------------------------ */
/* One time step.  Order (Sec. 3: semi-implicit predictor-corrector, first-order Euler): */
/*  1. grid: particles outside the cell grid become GHOST (velocity zeroed);            */
/*  2. predict (Eq. 2 without pressure): FLUID u* = u + dt (nu lap(u) + g), Eq. 7 over  */
/*     re_lap at r^k; r* = r + dt u*.  Other kinds keep u and r;                        */
/*  3. number density n* at r* over re_n (Eq. 5); free surface n* < beta n0 (Eq. 15)    */
/*     for FLUID/WALL;                                                                   */
/*  4. pressure: PPE (Eq. 13, assembled as above, CG) or equation of state (Eq. 16);    */
/*  5. PPE: negative pressure clamped to 0 (optional); p_hat_i = min over i and its     */
/*     non-DUMMY neighbours within re_n.  Equation of state: p_hat_i = p_i;             */
/*  6. correction: FLUID u' = -(dt/rho) grad p (gradient above, re_n, at r*); two-phase */
/*     u' = -(dt/rho_i) grad p, the multi-density pressure term of Sec. 3.2.1 (with       */
/*     p_j = rho_j alpha_j the bracket (rho_j/rho_i) alpha_j - alpha_i is (p_j - p_i)/rho_i);*/
/*     the viscosity of step 2 is the particle's own nu_i.                                */
/*     u = u* + u', r = r* + dt u'.                                                      */
/* ------------------------------------------------------------------------------------ */

/* Any pair of a neighbour set at distance 0 makes w infinite (Eq. 4): an error.        */
static int check_coincident(int dim, int64_t n, const double* pos, const csr_t* nb) {
    for (int64_t i = 0; i < n; i++)
        for (int64_t k = nb->off[i]; k < nb->off[i + 1]; k++) {
            int64_t j = nb->ids[k];
            double xi, yi, zi, xj, yj, zj;
            coords(pos, dim, i, &xi, &yi, &zi);
            coords(pos, dim, j, &xj, &yj, &zj);
            if (!(dist2(xj - xi, yj - yi, zj - zi) > 0.0)) return ORC_ECOINCIDENT;
        }
    return ORC_OK;
}

static int stage_grid(const orc_params* p, int64_t n, const double* pos, double* vel,
                      int8_t* type, orc_report* R) {
    uint32_t* key = malloc(sizeof(uint32_t) * (size_t)n);
    if (!key) return ORC_ENOMEM;
    int rc = orc_cell_keys(p, n, pos, type, key, NULL);
    if (!rc)
        for (int64_t i = 0; i < n; i++) {
            if (key[i] == 0xFFFFFFFFu && type[i] != ORC_GHOST) {
                type[i] = ORC_GHOST;
                for (int a = 0; a < p->dim; a++) vel[i * p->dim + a] = 0.0;
            }
            if (type[i] == ORC_GHOST) R->n_ghost++;
        }
    free(key);
    return rc;
}

static int stage_predict(const orc_params* p, int64_t n, const double* pos, const double* vel,
                         const int8_t* type, int nb_mode, double* ps, double* us, orc_report* R) {
    int dim = p->dim;
    csr_t nb = {0, 0};
    double* lap = malloc(sizeof(double) * (size_t)(n * dim));
    if (!lap) return ORC_ENOMEM;
    int rc = neighbors(dim, n, pos, type, p->re_lap, nb_mode, &nb);
    if (!rc) rc = check_coincident(dim, n, pos, &nb);
    if (!rc) {
        laplacian_from(dim, n, pos, type, p->re_lap, p->kernel, R->n0_lap, R->lambda, &nb, vel,
                       dim, lap);
        for (int64_t i = 0; i < n; i++)
            for (int a = 0; a < dim; a++) {
                int64_t q = i * dim + a;
                if (type[i] == ORC_FLUID) {
                    us[q] = vel[q] + p->dt * (nu_of(p, i) * lap[q] + p->g[a]);
                    ps[q] = pos[q] + p->dt * us[q];
                } else {
                    us[q] = vel[q];
                    ps[q] = pos[q];
                }
            }
        /* The neighbour sets at r* below are searched afresh at r*, so they are exact     */
        /* whatever the motion.  The library's candidate lists, gathered at r^k, need a     */
        /* direct search for every particle that moves more than half the cell skin; it    */
        /* gives up (MPS_ESKIN) beyond max(64, n/256) such particles, and so does this.     */
        double re = p->re_n > p->re_lap ? p->re_n : p->re_lap;
        const double half = 0.5 * p->cell_skin * re;
        int64_t n_fast = 0;
        R->max_disp = 0.0;
        for (int64_t i = 0; i < n; i++) {
            if (type[i] != ORC_FLUID) continue;
            double d2 = 0.0;
            for (int a = 0; a < dim; a++) {
                double d = ps[i * dim + a] - pos[i * dim + a];
                d2 = d2 + d * d;
            }
            if (sqrt(d2) > R->max_disp) R->max_disp = sqrt(d2);
            if (sqrt(d2) > half) n_fast++;
        }
        if (n_fast > (n / 256 > 64 ? n / 256 : 64)) rc = ORC_ESKIN;
    }
    csr_free(&nb);
    free(lap);
    return rc;
}

static int stage_density(const orc_params* p, int64_t n, const double* ps, const int8_t* type,
                         int nb_mode, csr_t* nb_n, double* nstar, uint8_t* flags, orc_report* R) {
    int rc = neighbors(p->dim, n, ps, type, p->re_n, nb_mode, nb_n);
    if (!rc) rc = check_coincident(p->dim, n, ps, nb_n);
    if (rc) return rc;
    pnd_from(p->dim, n, ps, type, p->re_n, p->kernel, nb_n, nstar);
    R->n_surface = 0;
    R->n_ppe_rows = 0;
    for (int64_t i = 0; i < n; i++) {
        int surf = (type[i] == ORC_FLUID || type[i] == ORC_WALL) && nstar[i] < p->beta * R->n0_pnd;
        flags[i] = (uint8_t)(surf ? 1 : 0);
        if (surf) R->n_surface++;
        if (in_ppe(type, flags, i)) R->n_ppe_rows++;
    }
    return ORC_OK;
}

static void ppe_rhs(const orc_params* p, int64_t n, const int8_t* type, const uint8_t* flags,
                    const double* nstar, double n0, double* b) {
    double inv_dt2 = 1.0 / (p->dt * p->dt);
    for (int64_t i = 0; i < n; i++)
        b[i] = in_ppe(type, flags, i) ? inv_dt2 * ((nstar[i] - n0) / n0) : 0.0;
}

/* ------------------------------------------------------------------------------------ */
/* Time derivative of the number density along a velocity field (the Dn/Dt of Eq. 21    */
/* and Eq. 24), for the kernel of Eq. 4:                                                 */
/*   (Dn/Dt)_i = sum_{j != i} w'(r_ij) (r_ij . u_ij) / r_ij = -sum re/r_ij^3 (r_ij . u_ij) */
/* with r_ij = r_j - r_i, u_ij = u_j - u_i, over the number-density neighbours (re_n,   */
/* every non-GHOST kind).                                                                */
/* ------------------------------------------------------------------------------------ */
static void dn_dt(const orc_params* p, int64_t n, const double* x, const double* u,
                  const int8_t* type, const csr_t* nb, double* out) {
    int dim = p->dim;
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; i++) {
        double s = 0.0;
        if (type[i] != ORC_GHOST) {
            double xi, yi, zi, ui[3] = {0.0, 0.0, 0.0};
            coords(x, dim, i, &xi, &yi, &zi);
            for (int a = 0; a < dim; a++) ui[a] = u[i * dim + a];
            for (int64_t k = nb->off[i]; k < nb->off[i + 1]; k++) {
                int64_t j = nb->ids[k];
                double xj, yj, zj;
                coords(x, dim, j, &xj, &yj, &zj);
                double d[3] = {xj - xi, yj - yi, zj - zi};
                double du[3] = {0.0, 0.0, 0.0};
                for (int a = 0; a < dim; a++) du[a] = u[j * dim + a] - ui[a];
                double r2 = dist2(d[0], d[1], d[2]);
                double r = sqrt(r2);
                double dot = (d[0] * du[0] + d[1] * du[1]) + d[2] * du[2];
                s = s + p->re_n / (r2 * r) * dot;
            }
        }
        out[i] = -s;
    }
}

/* ------------------------------------------------------------------------------------ */
/* Higher-order source term (MPS-HS), Eq. 21, from the predicted motion r*, u*.  In the  */
/* scaling of the PPE here (A = -(1/rho) L + alpha_c/dt^2 I) the right-hand side is      */
/*   b_i = (Dn/Dt)*_i / (n0 dt),                                                         */
/* positive where the predicted flow compresses the fluid, like Eq. 13's source.         */
/* With the error-compensating source (Eq. 24-25, source 2) the right-hand side adds    */
/*   ECS_i / dt,  ECS_i = |eps_i| (Dn/Dt)^k_i / n0 + |dt (Dn/Dt)^k_i / n0| eps_i / dt,   */
/* eps_i = (n^k_i - n0)/n0, number density and its rate at the step's start r^k, u^k.   */
/* (Eq. 25 prints ECS beside rho/(n0 dt) (Dn/Dt)* without the factor rho/dt its units   */
/* need; it is taken with that factor, i.e. ECS / dt after the division by rho.)         */
/* ------------------------------------------------------------------------------------ */
static void hs_rhs(const orc_params* p, int64_t n, const int8_t* type, const uint8_t* flags,
                   const double* dstar, const double* nk, const double* dk, double n0,
                   double* b) {
    for (int64_t i = 0; i < n; i++) {
        if (!in_ppe(type, flags, i)) { b[i] = 0.0; continue; }
        double v = dstar[i] / (n0 * p->dt);
        if (p->source == 2) {
            double eps = (nk[i] - n0) / n0;
            double ecs = fabs(eps) * (dk[i] / n0) + fabs(p->dt * dk[i] / n0) * (eps / p->dt);
            v = v + ecs / p->dt;
        }
        b[i] = v;
    }
}

/* The HS / ECS source of every row (steps 3-4 of a step with source 1 or 2).           */
static int hs_source(const orc_params* p, int64_t n, const double* pos, const double* vel,
                     const double* ps, const double* us, const int8_t* type,
                     const uint8_t* flags, const csr_t* nb_n, int nb_mode, double n0,
                     double* b) {
    double* dstar = malloc(sizeof(double) * (size_t)n);
    double* nk = malloc(sizeof(double) * (size_t)n);
    double* dk = malloc(sizeof(double) * (size_t)n);
    csr_t nb_k = {0, 0};
    int rc = ORC_ENOMEM;
    if (!dstar || !nk || !dk) goto out;
    dn_dt(p, n, ps, us, type, nb_n, dstar);
    if (p->source == 2) {
        rc = neighbors(p->dim, n, pos, type, p->re_n, nb_mode, &nb_k);
        if (rc) goto out;
        pnd_from(p->dim, n, pos, type, p->re_n, p->kernel, &nb_k, nk);
        dn_dt(p, n, pos, vel, type, &nb_k, dk);
    }
    hs_rhs(p, n, type, flags, dstar, nk, dk, n0, b);
    rc = ORC_OK;
out:
    free(dstar); free(nk); free(dk);
    csr_free(&nb_k);
    return rc;
}

static int check_params(const orc_params* p, int64_t n) {
    int dim = p->dim;
    if ((dim != 2 && dim != 3) || n <= 0 || !(p->l0 > 0) || !(p->re_n > 0) || !(p->re_lap > 0) ||
        !(p->rho > 0) || !(p->dt > 0) || !(p->cell_skin >= 0))
        return ORC_EINVAL;
    if (p->kernel < 0 || p->kernel > 1 || p->grad_form < 0 || p->grad_form > 1 || p->source < 0 ||
        p->source > 2 || (p->source >= 1 && p->kernel != 0))
        return ORC_EINVAL;
    for (int64_t i = 0; i < n; i++) {
        if (p->rho_i && !(p->rho_i[i] > 0.0 && isfinite(p->rho_i[i]))) return ORC_EINVAL;
        if (p->nu_i && !(p->nu_i[i] >= 0.0 && isfinite(p->nu_i[i]))) return ORC_EINVAL;
    }
    return ORC_OK;
}

int orc_step(const orc_params* p, int64_t n, double* pos, double* vel, int8_t* type,
             double* pres, double* nstar, uint8_t* flags, orc_report* rep, int32_t solve_only,
             int32_t nb_mode) {
    int dim = p->dim;
    int rc = check_params(p, n);
    if (rc) return rc;
    for (int64_t i = 0; i < n * dim; i++)
        if (!isfinite(pos[i]) || !isfinite(vel[i])) return ORC_ENONFINITE;
    orc_report R;
    memset(&R, 0, sizeof R);
    rc = orc_lattice(dim, p->l0, p->re_n, &R.n0_pnd, NULL, p->kernel);
    if (!rc) rc = orc_lattice(dim, p->l0, p->re_lap, &R.n0_lap, &R.lambda, p->kernel);
    if (rc) return rc;
    double n0 = R.n0_pnd;

    double* ps = malloc(sizeof(double) * (size_t)(n * dim));   /* r* */
    double* us = malloc(sizeof(double) * (size_t)(n * dim));   /* u* */
    double* phat = malloc(sizeof(double) * (size_t)n);
    double* grad = malloc(sizeof(double) * (size_t)(n * dim));
    double* bvec = malloc(sizeof(double) * (size_t)n);
    csr_t nb_n = {0, 0}, nb_l = {0, 0};
    mat_t A = {0, 0, 0};
    if (!ps || !us || !phat || !grad || !bvec) { rc = ORC_ENOMEM; goto out; }

    rc = stage_grid(p, n, pos, vel, type, &R);                          /* 1 */
    if (!rc) rc = stage_predict(p, n, pos, vel, type, nb_mode, ps, us, &R);   /* 2 */
    if (!rc) rc = stage_density(p, n, ps, type, nb_mode, &nb_n, nstar, flags, &R);  /* 3 */
    if (rc) goto out;

    if (p->pressure_mode == 0) {                                        /* 4, 5: PPE */
        rc = neighbors(dim, n, ps, type, p->re_lap, nb_mode, &nb_l);
        if (!rc) rc = assemble_ppe(p, n, ps, type, flags, &nb_l, R.n0_lap, R.lambda, &A);
        if (rc) goto out;
        if (p->source >= 1) {
            rc = hs_source(p, n, pos, vel, ps, us, type, flags, &nb_n, nb_mode, n0, bvec);
            if (rc) goto out;
        } else {
            ppe_rhs(p, n, type, flags, nstar, n0, bvec);
        }
        rc = cg_solve(n, &A, bvec, pres, p->cg_tol, p->cg_max_iter, &R.cg_iters, &R.cg_restarts,
                      &R.cg_resid);
        if (rc) goto out;
        for (int64_t i = 0; i < n; i++)
            if (!in_ppe(type, flags, i)) pres[i] = 0.0;
        if (p->clamp_negative_p)
            for (int64_t i = 0; i < n; i++)
                if (pres[i] < 0.0) pres[i] = 0.0;
        for (int64_t i = 0; i < n; i++) {
            double m = pres[i];
            for (int64_t k = nb_n.off[i]; k < nb_n.off[i + 1]; k++) {
                int64_t j = nb_n.ids[k];
                if (type[j] != ORC_DUMMY && pres[j] < m) m = pres[j];
            }
            phat[i] = m;
        }
    } else {                                                            /* 4, 5: EOS */
        for (int64_t i = 0; i < n; i++) {
            pres[i] = in_ppe(type, flags, i) ? wc_pressure(p, rho_of(p, i), nstar[i], n0) : 0.0;
            phat[i] = pres[i];
        }
        /* The CMPS gradient needs p_hat as the neighbourhood minimum on this path too (with */
        /* p_hat = p its pair term vanishes identically).                                  */
        if (p->grad_form == 1)
            for (int64_t i = 0; i < n; i++) {
                double m = pres[i];
                for (int64_t k = nb_n.off[i]; k < nb_n.off[i + 1]; k++) {
                    int64_t j = nb_n.ids[k];
                    if (type[j] != ORC_DUMMY && pres[j] < m) m = pres[j];
                }
                phat[i] = m;
            }
    }
    if (solve_only) goto out;

    gradient_from(dim, n, ps, type, p->re_n, p->kernel, p->grad_form, n0, &nb_n, pres, phat,
                  grad);                                                /* 6 */
    for (int64_t i = 0; i < n; i++)
        for (int a = 0; a < dim; a++) {
            int64_t q = i * dim + a;
            if (type[i] == ORC_FLUID) {
                double du = -(p->dt / rho_of(p, i)) * grad[q];
                vel[q] = us[q] + du;
                pos[q] = ps[q] + p->dt * du;
            }
        }

out:
    if (rep) *rep = R;
    free(ps); free(us); free(phat); free(grad); free(bvec);
    csr_free(&nb_n); csr_free(&nb_l);
    mat_free(&A);
    return rc;
}

/* ------------------------------------------------------------------------------------ */
/* The PPE system a step would solve (steps 1-3 above, then the assembly), for the      */
/* matrix pins (symmetry, definiteness, dense-solve cross-check).  Two calls: first     */
/* with col/val NULL to get off[n+1]; then with buffers of off[n] entries.  Inputs are  */
/* not modified.                                                                         */
/* ------------------------------------------------------------------------------------ */
int orc_ppe_system(const orc_params* p, int64_t n, const double* pos, const double* vel,
                   const int8_t* type_in, int64_t* off, int32_t* col, double* val, double* b,
                   double* pstar, double* nstar_out, uint8_t* flags_out) {
    int dim = p->dim;
    int rc = check_params(p, n);
    if (rc) return rc;
    orc_report R;
    memset(&R, 0, sizeof R);
    rc = orc_lattice(dim, p->l0, p->re_n, &R.n0_pnd, NULL, p->kernel);
    if (!rc) rc = orc_lattice(dim, p->l0, p->re_lap, &R.n0_lap, &R.lambda, p->kernel);
    if (rc) return rc;
    double* vel_c = malloc(sizeof(double) * (size_t)(n * dim));
    double* ps = malloc(sizeof(double) * (size_t)(n * dim));
    double* us = malloc(sizeof(double) * (size_t)(n * dim));
    double* nstar = malloc(sizeof(double) * (size_t)n);
    int8_t* type = malloc((size_t)n);
    uint8_t* flags = malloc((size_t)n);
    csr_t nb_n = {0, 0}, nb_l = {0, 0};
    mat_t A = {0, 0, 0};
    rc = ORC_ENOMEM;
    if (!vel_c || !ps || !us || !nstar || !type || !flags) goto out;
    memcpy(vel_c, vel, sizeof(double) * (size_t)(n * dim));
    memcpy(type, type_in, (size_t)n);
    rc = stage_grid(p, n, pos, vel_c, type, &R);
    if (!rc) rc = stage_predict(p, n, pos, vel_c, type, 1, ps, us, &R);
    if (!rc) rc = stage_density(p, n, ps, type, 1, &nb_n, nstar, flags, &R);
    if (!rc) rc = neighbors(dim, n, ps, type, p->re_lap, 1, &nb_l);
    if (!rc) rc = assemble_ppe(p, n, ps, type, flags, &nb_l, R.n0_lap, R.lambda, &A);
    if (rc) goto out;
    memcpy(off, A.off, sizeof(int64_t) * (size_t)(n + 1));
    if (col && val) {
        memcpy(col, A.col, sizeof(int32_t) * (size_t)A.off[n]);
        memcpy(val, A.val, sizeof(double) * (size_t)A.off[n]);
    }
    if (b) {
        if (p->source >= 1) rc = hs_source(p, n, pos, vel_c, ps, us, type, flags, &nb_n, 1,
                                           R.n0_pnd, b);
        else ppe_rhs(p, n, type, flags, nstar, R.n0_pnd, b);
        if (rc) goto out;
    }
    if (pstar) memcpy(pstar, ps, sizeof(double) * (size_t)(n * dim));
    if (nstar_out) memcpy(nstar_out, nstar, sizeof(double) * (size_t)n);
    if (flags_out) memcpy(flags_out, flags, (size_t)n);
out:
    free(vel_c); free(ps); free(us); free(nstar); free(type); free(flags);
    csr_free(&nb_n); csr_free(&nb_l);
    mat_free(&A);
    return rc;
}

/* CG on a caller-supplied CSR system (used to pin the solver against a dense solve).   */
int orc_cg(int64_t n, const int64_t* off, const int32_t* col, const double* val, const double* b,
           double* x, double tol, int32_t max_iter, int32_t* iters, double* resid) {
    mat_t A = {(int64_t*)off, (int32_t*)col, (double*)val};
    int it = 0, rs = 0;
    int rc = cg_solve(n, &A, b, x, tol, max_iter, &it, &rs, resid);
    *iters = it;
    return rc;
}

/* ------------------------------------------------------------------------------------ */
/* Reverse (vector-Jacobian product) of one step, the adjoint of the step map           */
/*   (r^k, u^k, g) -> (r^{k+1}, u^{k+1})                                                  */
/* defined by orc_step (PPE or equation-of-state path; kernel of Eq. 4, difference-form */
/* gradient, source of Eq. 13; one or two phases).  Given the adjoints gr = dL/dr^{k+1}, */
/* gu = dL/du^{k+1} (n*dim each) it returns dL/dr^k, dL/du^k and dL/dg.                  */
/* The discrete choices of the step are held fixed: neighbour sets, the GHOST and free- */
/* surface sets, the clamp's active set and the particle giving p_hat_i (the strict     */
/* minimum in ascending neighbour order, p_i first).  Within them the step is smooth and */
/* this is its exact derivative (up to the CG tolerance of the adjoint solve).          */
/*                                                                                        */
/* Chain, from the last stage back (x_ij = r_j - r_i, s = |x_ij|, w(s) = re/s - 1,       */
/* w'(s) = -re/s^2; every pair term adds +X to particle j and -X to particle i):        */
/*  6. u = u* + u', r = r* + dt u', u' = -(dt/rho_i) G_i, FLUID:                          */
/*       gu* = gu, gr* = gr, gG_i = -(dt/rho_i)(gu_i + dt gr_i);                           */
/*     G_i = d/n0 sum_j (p_j - p_hat_i) x w/s^2 over non-dummy j within re_n at r*:      */
/*       gp_j += d/n0 (x . gG_i) w/s^2, gphat_i -= the same,                              */
/*       X = d/n0 (p_j - p_hat_i) [q gG_i + (q'/s)(x . gG_i) x],  q = w/s^2;               */
/*  5. p_hat_i = p_m(i): gp_m(i) += gphat_i; clamp: gp_i = 0 where p_i <= 0 was clamped;  */
/*     only rows of the PPE (or, for the equation of state, FLUID/WALL rows off the      */
/*     surface) carry a pressure that depends on the state;                               */
/*  4. PPE: A p = b with A symmetric, so A lam = gp gives gb = lam and, per coefficient  */
/*     c_ij (i a PPE row, j a non-dummy neighbour within re_lap; A_ii holds +c_ij and    */
/*     A_ij holds -c_ij when j is a row), gc_ij = -lam_i (p_i - p_j) with p_j = 0 off    */
/*     the rows; c_ij = K_ij w(s): X = gc_ij K_ij w'(s) x/s.  gn*_i = lam_i/(n0 dt^2).    */
/*     Equation of state: gn*_i = gp_i rho_i c0^2 (n*_i/n0)^(gamma-1) / n0;              */
/*  3. n*_i = sum_j w(s) over every non-GHOST j within re_n at r*: X = gn*_i w'(s) x/s;  */
/*  2. r* = r + dt u* (FLUID), so gr = gr*, gu* += dt gr*;                                */
/*     u* = u + dt (nu_i lap(u)_i + g): gu += gu*, gg += dt gu*, and per pair within     */
/*     re_lap at r^k (k = dt nu_i 2d/(n0_lap lambda)): gu_j += k w gu*_i, gu_i -= the     */
/*     same, X = k (gu*_i . (u_j - u_i)) w'(s) x/s;                                        */
/*     The viscosity nu_i enters only u*_i (FLUID), linearly: dL/dnu_i = dt gu*_i .       */
/*     lap(u)_i = dt 2d/(n0_lap lambda) sum_j w(s) (gu*_i . (u_j - u_i)) (out_nu, n      */
/*     values; 0 off FLUID; with one viscosity for all, dL/dnu is their sum);            */
/*  1. a particle that becomes a GHOST in this step has its velocity reset: gu = 0.      */
/* Other kinds: r^{k+1} = r^k, u^{k+1} = u^k (identity) plus their part in pair terms.   */
/* ------------------------------------------------------------------------------------ */
static void add_pair(double* out, int dim, int64_t i, int64_t j, const double X[3]) {
    for (int a = 0; a < dim; a++) {
        out[j * dim + a] = out[j * dim + a] + X[a];
        out[i * dim + a] = out[i * dim + a] - X[a];
    }
}

int orc_step_vjp(const orc_params* p, int64_t n, const double* pos, const double* vel,
                 const int8_t* type_in, const double* gr, const double* gu, double* out_r,
                 double* out_u, double* out_g, double* out_nu, orc_report* rep,
                 int32_t nb_mode) {
    int dim = p->dim;
    int rc = check_params(p, n);
    if (rc) return rc;
    if (p->kernel != 0 || p->grad_form != 0 || p->source != 0) return ORC_EINVAL;
    for (int64_t i = 0; i < n * dim; i++)
        if (!isfinite(pos[i]) || !isfinite(vel[i])) return ORC_ENONFINITE;
    orc_report R;
    memset(&R, 0, sizeof R);
    rc = orc_lattice(dim, p->l0, p->re_n, &R.n0_pnd, NULL, 0);
    if (!rc) rc = orc_lattice(dim, p->l0, p->re_lap, &R.n0_lap, &R.lambda, 0);
    if (rc) return rc;
    const double n0 = R.n0_pnd, dt = p->dt;
    const size_t nv = (size_t)(n * dim);

    double* x0 = malloc(sizeof(double) * nv);      /* r^k */
    double* u0 = malloc(sizeof(double) * nv);      /* u^k after the grid stage */
    double* ps = malloc(sizeof(double) * nv);      /* r* */
    double* us = malloc(sizeof(double) * nv);      /* u* */
    double* nstar = malloc(sizeof(double) * (size_t)n);
    double* bvec = malloc(sizeof(double) * (size_t)n);
    double* ppre = calloc((size_t)n, sizeof(double));   /* PPE solution before the clamp */
    double* pres = calloc((size_t)n, sizeof(double));
    int64_t* amin = malloc(sizeof(int64_t) * (size_t)n);
    double* gG = calloc(nv, sizeof(double));
    double* gp = calloc((size_t)n, sizeof(double));
    double* gphat = calloc((size_t)n, sizeof(double));
    double* lam = calloc((size_t)n, sizeof(double));
    double* gn = calloc((size_t)n, sizeof(double));
    double* grs = malloc(sizeof(double) * nv);     /* dL/dr* */
    double* gus = calloc(nv, sizeof(double));      /* dL/du* */
    int8_t* type = malloc((size_t)n);
    uint8_t* flags = calloc((size_t)n, 1);
    csr_t nb_n = {0, 0}, nb_l = {0, 0}, nb_k = {0, 0};
    mat_t A = {0, 0, 0};
    if (!x0 || !u0 || !ps || !us || !nstar || !bvec || !ppre || !pres || !amin || !gG || !gp ||
        !gphat || !lam || !gn || !grs || !gus || !type || !flags) {
        rc = ORC_ENOMEM;
        goto out;
    }
    memcpy(x0, pos, sizeof(double) * nv);
    memcpy(u0, vel, sizeof(double) * nv);
    memcpy(type, type_in, (size_t)n);

    /* ---- forward, keeping what the reverse needs */
    rc = stage_grid(p, n, x0, u0, type, &R);
    if (!rc) rc = stage_predict(p, n, x0, u0, type, nb_mode, ps, us, &R);
    if (!rc) rc = stage_density(p, n, ps, type, nb_mode, &nb_n, nstar, flags, &R);
    if (rc) goto out;
    for (int64_t i = 0; i < n; i++) amin[i] = i;
    if (p->pressure_mode == 0) {
        rc = neighbors(dim, n, ps, type, p->re_lap, nb_mode, &nb_l);
        if (!rc) rc = assemble_ppe(p, n, ps, type, flags, &nb_l, R.n0_lap, R.lambda, &A);
        if (rc) goto out;
        ppe_rhs(p, n, type, flags, nstar, n0, bvec);
        rc = cg_solve(n, &A, bvec, ppre, p->cg_tol, p->cg_max_iter, &R.cg_iters,
                      &R.cg_restarts, &R.cg_resid);
        if (rc) goto out;
        for (int64_t i = 0; i < n; i++) {
            if (!in_ppe(type, flags, i)) ppre[i] = 0.0;
            pres[i] = (p->clamp_negative_p && ppre[i] < 0.0) ? 0.0 : ppre[i];
        }
        for (int64_t i = 0; i < n; i++) {
            double m = pres[i];
            for (int64_t k = nb_n.off[i]; k < nb_n.off[i + 1]; k++) {
                int64_t j = nb_n.ids[k];
                if (type[j] != ORC_DUMMY && pres[j] < m) { m = pres[j]; amin[i] = j; }
            }
        }
    } else {
        for (int64_t i = 0; i < n; i++)
            pres[i] = in_ppe(type, flags, i) ? wc_pressure(p, rho_of(p, i), nstar[i], n0) : 0.0;
    }

    /* ---- 6: correction */
    memcpy(grs, gr, sizeof(double) * nv);
    for (int64_t i = 0; i < n; i++) {
        if (type[i] != ORC_FLUID) continue;
        double k = -(dt / rho_of(p, i));
        for (int a = 0; a < dim; a++) {
            int64_t q = i * dim + a;
            gG[q] = k * (gu[q] + dt * gr[q]);
            gus[q] = gu[q];
        }
    }
    /* gradient pairs (re_n, non-dummy j, at r*) */
    const double cg0 = (double)dim / n0;
    for (int64_t i = 0; i < n; i++) {
        if (type[i] != ORC_FLUID) continue;
        double xi, yi, zi;
        coords(ps, dim, i, &xi, &yi, &zi);
        double gi[3] = {0.0, 0.0, 0.0};
        for (int a = 0; a < dim; a++) gi[a] = gG[i * dim + a];
        for (int64_t k = nb_n.off[i]; k < nb_n.off[i + 1]; k++) {
            int64_t j = nb_n.ids[k];
            if (type[j] == ORC_DUMMY) continue;
            double xj, yj, zj;
            coords(ps, dim, j, &xj, &yj, &zj);
            double d[3] = {xj - xi, yj - yi, zj - zi};
            double s2 = dist2(d[0], d[1], d[2]);
            double s = sqrt(s2);
            double w = p->re_n / s - 1.0;
            double wd = -p->re_n / s2;
            double q = w / s2;
            double qd = wd / s2 - 2.0 * w / (s2 * s);
            double dg = (d[0] * gi[0] + d[1] * gi[1]) + d[2] * gi[2];
            gp[j] = gp[j] + cg0 * q * dg;
            gphat[i] = gphat[i] - cg0 * q * dg;
            double f = cg0 * (pres[j] - pres[amin[i]]);
            double X[3];
            for (int a = 0; a < 3; a++) X[a] = f * (q * gi[a] + (qd / s) * dg * d[a]);
            add_pair(grs, dim, i, j, X);
        }
    }
    /* ---- 5: p_hat, clamp (p_hat_i = p_i on the equation-of-state path: amin[i] = i) */
    for (int64_t i = 0; i < n; i++)
        if (type[i] == ORC_FLUID) gp[amin[i]] = gp[amin[i]] + gphat[i];
    for (int64_t i = 0; i < n; i++) {
        if (!in_ppe(type, flags, i)) gp[i] = 0.0;
        else if (p->pressure_mode == 0 && p->clamp_negative_p && !(ppre[i] > 0.0)) gp[i] = 0.0;
    }
    /* ---- 4: pressure */
    if (p->pressure_mode == 0) {
        int it = 0, rs = 0;
        double res = 0.0;
        rc = cg_solve(n, &A, gp, lam, p->cg_tol, p->cg_max_iter, &it, &rs, &res);
        if (rc) goto out;
        const double coef = (2.0 * dim) / (R.n0_lap * R.lambda * p->rho);
        const double coef0 = (2.0 * dim) / (R.n0_lap * R.lambda);
        for (int64_t i = 0; i < n; i++) {
            if (!in_ppe(type, flags, i)) continue;
            gn[i] = lam[i] / (n0 * dt * dt);
            double xi, yi, zi;
            coords(ps, dim, i, &xi, &yi, &zi);
            for (int64_t k = nb_l.off[i]; k < nb_l.off[i + 1]; k++) {
                int64_t j = nb_l.ids[k];
                if (type[j] == ORC_DUMMY) continue;
                double xj, yj, zj;
                coords(ps, dim, j, &xj, &yj, &zj);
                double d[3] = {xj - xi, yj - yi, zj - zi};
                double s2 = dist2(d[0], d[1], d[2]);
                double s = sqrt(s2);
                double K = p->rho_i ? coef0 * (2.0 / (p->rho_i[i] + p->rho_i[j])) : coef;
                double gc = -lam[i] * (ppre[i] - ppre[j]);
                double f = gc * K * (-p->re_lap / s2) / s;
                double X[3] = {f * d[0], f * d[1], f * d[2]};
                add_pair(grs, dim, i, j, X);
            }
        }
    } else {
        for (int64_t i = 0; i < n; i++)
            if (in_ppe(type, flags, i))
                gn[i] = gp[i] * rho_of(p, i) * p->c0 * p->c0 * pow(nstar[i] / n0, p->gamma - 1.0) / n0;
    }
    /* ---- 3: number density (re_n, every non-GHOST neighbour, at r*) */
    for (int64_t i = 0; i < n; i++) {
        if (gn[i] == 0.0) continue;
        double xi, yi, zi;
        coords(ps, dim, i, &xi, &yi, &zi);
        for (int64_t k = nb_n.off[i]; k < nb_n.off[i + 1]; k++) {
            int64_t j = nb_n.ids[k];
            double xj, yj, zj;
            coords(ps, dim, j, &xj, &yj, &zj);
            double d[3] = {xj - xi, yj - yi, zj - zi};
            double s2 = dist2(d[0], d[1], d[2]);
            double f = gn[i] * (-p->re_n / s2) / sqrt(s2);
            double X[3] = {f * d[0], f * d[1], f * d[2]};
            add_pair(grs, dim, i, j, X);
        }
    }
    /* ---- 2: r* = r + dt u*, u* = u + dt (nu lap(u) + g) */
    memcpy(out_r, grs, sizeof(double) * nv);
    for (int a = 0; a < 3; a++) out_g[a] = 0.0;
    for (int64_t i = 0; i < n; i++)
        for (int a = 0; a < dim; a++) {
            int64_t q = i * dim + a;
            if (type[i] == ORC_FLUID) {
                gus[q] = gus[q] + dt * grs[q];
                out_u[q] = gus[q];
                out_g[a] = out_g[a] + dt * gus[q];
            } else {
                out_u[q] = gu[q];
            }
        }
    rc = neighbors(dim, n, x0, type, p->re_lap, nb_mode, &nb_k);
    if (rc) goto out;
    const double clap = (2.0 * dim) / (R.n0_lap * R.lambda);
    if (out_nu)
        for (int64_t i = 0; i < n; i++) out_nu[i] = 0.0;
    for (int64_t i = 0; i < n; i++) {
        if (type[i] != ORC_FLUID) continue;
        double xi, yi, zi;
        coords(x0, dim, i, &xi, &yi, &zi);
        double k = dt * nu_of(p, i) * clap;
        double gnu = 0.0;   /* sum_j w (gu*_i . (u_j - u_i)) */
        for (int64_t kk = nb_k.off[i]; kk < nb_k.off[i + 1]; kk++) {
            int64_t j = nb_k.ids[kk];
            double xj, yj, zj;
            coords(x0, dim, j, &xj, &yj, &zj);
            double d[3] = {xj - xi, yj - yi, zj - zi};
            double s2 = dist2(d[0], d[1], d[2]);
            double s = sqrt(s2);
            double w = p->re_lap / s - 1.0;
            double gdu = 0.0;
            for (int a = 0; a < dim; a++) {
                double gsa = gus[i * dim + a];
                out_u[j * dim + a] = out_u[j * dim + a] + k * w * gsa;
                out_u[i * dim + a] = out_u[i * dim + a] - k * w * gsa;
                gdu = gdu + gsa * (u0[j * dim + a] - u0[i * dim + a]);
            }
            double f = k * gdu * (-p->re_lap / s2) / s;
            double X[3] = {f * d[0], f * d[1], f * d[2]};
            add_pair(out_r, dim, i, j, X);
            gnu = gnu + w * gdu;
        }
        if (out_nu) out_nu[i] = dt * clap * gnu;
    }
    /* ---- 1: a particle turned GHOST in this step had its velocity reset */
    for (int64_t i = 0; i < n; i++)
        if (type[i] == ORC_GHOST && type_in[i] != ORC_GHOST)
            for (int a = 0; a < dim; a++) out_u[i * dim + a] = 0.0;

out:
    if (rep) *rep = R;
    free(x0); free(u0); free(ps); free(us); free(nstar); free(bvec); free(ppre); free(pres);
    free(amin); free(gG); free(gp); free(gphat); free(lam); free(gn); free(grs); free(gus);
    free(type); free(flags);
    csr_free(&nb_n); csr_free(&nb_l); csr_free(&nb_k);
    mat_free(&A);
    return rc;
}
