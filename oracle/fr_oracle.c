/*
 * fr_oracle.c -- plain, slow, obviously-correct FP64 CPU reference for the
 * f(R) scalaron solver of Li, Zhao, Teyssier & Koyama, "ECOSMOG: An Efficient
 * Code for Simulating Modified Gravity" (arXiv:1110.1379).
 *
 * TEST INFRASTRUCTURE ONLY.  It is called by tests/, by the smoke check and by
 * the CPU-baseline leg of bench.py.  The GPU library never links, loads or
 * calls it, and it shares no code, header, table or constant with the CUDA
 * path.
 *
 * The unknown here is the paper's own variable  ut = ln(-a^2 f_R)  (Sec. III.C,
 * "f~_R = -e^{u~}").  The public entry points take and return the shifted
 * variable u = ut - ubar(a) = ln(f_R / fbar_R) and convert at the boundary.
 * Every equation is evaluated in the form it has in the paper:
 *   - operator: Eq. (discrete_fR) multiplied by c~^2, i.e. the left-hand side of
 *     Eq. (bc_modified_fR_op), written face by face as (b_i + b_j)(u_j - u_i);
 *   - ghost faces of refinement patches: Eq. (u_i-1jk) with r = m_ghost/m_i;
 *   - Newton derivative: Eq. (bc_modified_fR_dop);
 *   - relaxation: u <- u - L/(dL/du) (end of Sec. V.B.1), red-black order;
 *   - FAS coarse equation L^H(u^H) = L^H(R u^h) - R d^h, correction
 *     u^h += P(u^H - R u^h) (Sec. V.B.2 and V.B.3);
 *   - prolongation weights 27/9/3/1 over 64 (Sec. V.A.3).
 * Readings where the paper is silent (restriction operator, level count,
 * coarsest solve, Newton step cap, norm) are marked "Reading:" below.
 *
 * Pins (tests/test_oracle_pins.py; no function here is unpinned):
 *   model_init        test_minus_rbar_41, test_background_matches_paper_fields,
 *                     test_homogeneous_converges_to_background
 *   cell_op           test_algebraic_limit, test_linear_limit_fft,
 *                     test_point_mass_far_field_is_linear_yukawa,
 *                     test_sine_closed_form_second_order, test_gaussian_closed_form_converges,
 *                     test_flux_terms_telescope, test_newton_derivative_central_difference
 *   ngs_sweep         test_sweep_equals_cell_by_cell_red_then_black
 *   restrict_avg      test_restriction_identities
 *   restrict_faces    test_face_restriction_exact_for_linear_faces
 *   prolong_add       test_prolongation_weights_are_the_papers,
 *                     test_prolongation_exact_for_linear_fields,
 *                     test_prolongation_on_a_patch_drops_outside_cells
 *   count_levels      test_level_count_rule
 *   vcycle, coarsest  test_two_level_vcycle_by_hand, test_vcycle_beats_single_grid,
 *                     test_dense_newton_matches_fas_periodic / _patch
 *   orc_patch_bc      test_patch_bc_exact_for_linear_parent,
 *                     test_patch_bc_wraps_a_periodic_parent,
 *                     test_two_level_gaussian_patch, test_three_level_gaussian_patch,
 *                     test_patch_with_exact_boundary_reproduces_full_grid
 *   orc_cic           test_cic_mean_density_is_one,
 *                     test_cic_centred_particle_and_translation, test_cic_brute_force
 * oracle/mutation_check.py plants mistakes in this file and checks that a pin fails.
 *
 * Layout: every field is [n2][n1][n0], x (index 0) fastest.
 * Boundary values of a patch are six packed faces in the order
 * -x, +x, -y, +y, -z, +z; the face normal to axis `ax` is indexed by the two
 * other axes p < q as  c[q] * n[p] + c[p].
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#define ORC_OK 0
#define ORC_EINVAL 1
#define ORC_ENOMEM 2
#define ORC_ENOCONV 4

/* ------------------------------------------------------------------------- */
/* Model constants (Sec. II, Sec. III.A, Sec. III.C, Sec. VI.A.1)             */
/* ------------------------------------------------------------------------- */
typedef struct {
    double ct;    /* c~ = c / (B H0): c in km/s, H0 = 100 h km/s/Mpc, B in Mpc/h */
    double om, ol, a, nhs;
    double xi;    /* xi = c1 / c2^2 (Sec. II) */
    double src;   /* (1/3) Om a^4 (n a^2 xi)^{1/(n+1)}: coefficient of exp(-u/(n+1)) */
    double bkg;   /* Om a^4 (a^-3 + 4 OL/Om) */
    double dens;  /* Om a: coefficient of (rho - 1) */
    double ubar;  /* ln|fbar~_R(a)| from the homogeneous solution (Sec. VI.A.1) */
} OModel;

static void model_init(OModel *m, double box, double a, double om, double fr0, double nhs)
{
    m->ct = 299792.458 / (100.0 * box);
    m->om = om;
    m->ol = 1.0 - om; /* flat background */
    m->a = a;
    m->nhs = nhs;
    /* Homogeneous solution (Sec. VI.A.1) at a = 1 defines |f_R0|:
     *   |f_R0| = n xi / [3(1 + 4 OL/Om)]^{n+1}. */
    double k1 = 3.0 * (1.0 + 4.0 * m->ol / om);
    m->xi = fr0 * pow(k1, nhs + 1.0) / nhs;
    double ka = 3.0 * (pow(a, -3.0) + 4.0 * m->ol / om);
    m->src = om * pow(a, 4.0) * pow(nhs * a * a * m->xi, 1.0 / (nhs + 1.0)) / 3.0;
    m->bkg = om * pow(a, 4.0) * (pow(a, -3.0) + 4.0 * m->ol / om);
    m->dens = om * a;
    m->ubar = log(nhs * a * a * m->xi / pow(ka, nhs + 1.0));
}

/* ------------------------------------------------------------------------- */
/* One grid level                                                             */
/* ------------------------------------------------------------------------- */
typedef struct {
    int n[3];
    long ncell;
    double h;      /* cell size in code units (box side 1) */
    double pre;    /* c~^2 / (2 h^2), the prefactor in Eq. (bc_modified_fR_op) */
    int dirichlet; /* 0: periodic domain grid; 1: refinement patch with ghosts */
    double *u;     /* paper variable u~ */
    double *rho;   /* density rho~ (restricted on coarse levels) */
    double *f;     /* right-hand side (0 on the finest level) */
    double *uR;    /* R u^h saved for the FAS correction */
    double *d;     /* residual scratch */
    double *ub;    /* packed boundary values u_b (Dirichlet only), paper variable */
    long foff[6];  /* offsets of the six faces inside ub */
} OLevel;

static long idx3(const int n[3], int i, int j, int k)
{
    return ((long)k * n[1] + j) * n[0] + i;
}

static void face_axes(int ax, int *p, int *q)
{
    *p = (ax == 0) ? 1 : 0;
    *q = (ax == 2) ? 1 : 2;
}

static void face_offsets(const int n[3], long foff[6])
{
    long off = 0;
    for (int f = 0; f < 6; f++) {
        int p, q;
        face_axes(f / 2, &p, &q);
        foff[f] = off;
        off += (long)n[p] * n[q];
    }
}

static long face_size_total(const int n[3])
{
    long foff[6];
    face_offsets(n, foff);
    int p, q;
    face_axes(2, &p, &q);
    return foff[5] + (long)n[p] * n[q];
}

/* Boundary value u_b stored for the face `f` of the boundary cell c[3]. */
static double face_value(const OLevel *L, int f, const int c[3])
{
    int p, q;
    face_axes(f / 2, &p, &q);
    return L->ub[L->foff[f] + (long)c[q] * L->n[p] + c[p]];
}

/*
 * L(u) at one cell and dL/du at that cell.
 * Flux form of Eq. (discrete_fR) times c~^2, b = e^u, b_{i+1/2} = (b_i+b_{i+1})/2:
 *   c~^2/h^2 sum_faces b_{face} (u_j - u_i) = pre * sum_j (b_i + b_j)(u_j - u_i),
 * plus  -Om a (rho - 1) + (1/3) Om a^4 (n a^2 xi)^{1/(n+1)} e^{-u/(n+1)} - Om a^4 K(a).
 * A ghost neighbour (outside a patch) takes u_g = u_b - r u_b + r u_i with
 * r = m_{ghost}/m_i = -1 and b_g = exp(u_g) (Eq. u_i-1jk and the remark that
 * follows it); its face term is then (b_i + b_g)(u_g - u_i), which regrouped over
 * all faces is exactly Eq. (bc_modified_fR_op).  The derivative of each face term
 * with respect to u_i reproduces Eq. (bc_modified_fR_dop) term by term.
 */
static void cell_op(const OLevel *L, const OModel *m, int i, int j, int k,
                    double *Lval, double *dL)
{
    const int c[3] = {i, j, k};
    long ci = idx3(L->n, i, j, k);
    double ui = L->u[ci];
    double bi = exp(ui);
    double flux = 0.0, dflux = 0.0;
    for (int f = 0; f < 6; f++) {
        int ax = f / 2;
        int nb[3] = {i, j, k};
        nb[ax] += (f % 2) ? 1 : -1;
        int inside = nb[ax] >= 0 && nb[ax] < L->n[ax];
        if (inside || !L->dirichlet) {
            nb[ax] = (nb[ax] + L->n[ax]) % L->n[ax]; /* periodic wrap */
            double uj = L->u[idx3(L->n, nb[0], nb[1], nb[2])];
            double bj = exp(uj);
            flux += (bi + bj) * (uj - ui);
            dflux += bi * (uj - ui) - (bi + bj);
        } else {
            const double r = -1.0; /* mask -1 (ghost) over mask +1 (active) */
            double ubv = face_value(L, f, c);
            double ug = ubv - r * ubv + r * ui;
            double bg = exp(ug);
            flux += (bi + bg) * (ug - ui);
            dflux += (bi + r * bg) * (ug - ui) + (bi + bg) * (r - 1.0);
        }
    }
    double s = exp(-ui / (m->nhs + 1.0));
    *Lval = L->pre * flux - m->dens * (L->rho[ci] - 1.0) + m->src * s - m->bkg;
    *dL = L->pre * dflux - m->src * s / (m->nhs + 1.0);
}

/* d = L(u) - f on every cell. */
static void residual(const OLevel *L, const OModel *m, double *d)
{
    for (int k = 0; k < L->n[2]; k++)
        for (int j = 0; j < L->n[1]; j++)
            for (int i = 0; i < L->n[0]; i++) {
                double lv, dl;
                cell_op(L, m, i, j, k, &lv, &dl);
                long ci = idx3(L->n, i, j, k);
                d[ci] = lv - (L->f ? L->f[ci] : 0.0);
            }
}

/* Reading (norm unspecified in Sec. V.B.2): root-mean-square over the cells. */
static double rms_of(const double *d, long n, double *maxabs)
{
    double s = 0.0, mx = 0.0;
    for (long c = 0; c < n; c++) {
        s += d[c] * d[c];
        if (fabs(d[c]) > mx)
            mx = fabs(d[c]);
    }
    if (maxabs)
        *maxabs = mx;
    return n > 0 ? sqrt(s / (double)n) : 0.0;
}

/*
 * One Newton-Gauss-Seidel sweep, red cells ((i+j+k) even) first, then black.
 * u <- u - (L(u) - f) / (dL/du) (end of Sec. V.B.1 with the FAS right-hand side
 * of Sec. V.B.2).  Reading (the paper is silent on damping): the Newton step is
 * clamped to |du| <= cap.
 */
static void ngs_sweep(OLevel *L, const OModel *m, double cap)
{
    for (int colour = 0; colour < 2; colour++)
        for (int k = 0; k < L->n[2]; k++)
            for (int j = 0; j < L->n[1]; j++)
                for (int i = 0; i < L->n[0]; i++) {
                    if ((i + j + k) % 2 != colour)
                        continue;
                    long ci = idx3(L->n, i, j, k);
                    double lv, dl;
                    cell_op(L, m, i, j, k, &lv, &dl);
                    double du = -(lv - (L->f ? L->f[ci] : 0.0)) / dl;
                    if (du > cap)
                        du = cap;
                    if (du < -cap)
                        du = -cap;
                    L->u[ci] += du;
                }
}

/* Reading (restriction operator unspecified): average of the 8 child cells. */
static void restrict_avg(const double *fine, const int nf[3], double *coarse)
{
    int nc[3] = {nf[0] / 2, nf[1] / 2, nf[2] / 2};
    for (int K = 0; K < nc[2]; K++)
        for (int J = 0; J < nc[1]; J++)
            for (int I = 0; I < nc[0]; I++) {
                double s = 0.0;
                for (int c = 0; c < 2; c++)
                    for (int b = 0; b < 2; b++)
                        for (int a = 0; a < 2; a++)
                            s += fine[idx3(nf, 2 * I + a, 2 * J + b, 2 * K + c)];
                coarse[idx3(nc, I, J, K)] = s / 8.0;
            }
}

/* Reading of Sec. V.B.2 (coarse u_B from the matching cells of the coarser
 * level): a coarse face value is the mean of the 4 fine face values that cover it. */
static void restrict_faces(const double *ubf, const int nf[3], double *ubc)
{
    int nc[3] = {nf[0] / 2, nf[1] / 2, nf[2] / 2};
    long of[6], oc[6];
    face_offsets(nf, of);
    face_offsets(nc, oc);
    for (int f = 0; f < 6; f++) {
        int p, q;
        face_axes(f / 2, &p, &q);
        for (int Q = 0; Q < nc[q]; Q++)
            for (int P = 0; P < nc[p]; P++) {
                double s = 0.0;
                for (int b = 0; b < 2; b++)
                    for (int a = 0; a < 2; a++)
                        s += ubf[of[f] + (long)(2 * Q + b) * nf[p] + (2 * P + a)];
                ubc[oc[f] + (long)Q * nc[p] + P] = s / 4.0;
            }
    }
}

/*
 * u^h += P e^H with e^H = u^H - R u^h (Sec. V.B.3), P the trilinear operator of
 * Sec. V.A.3: the coarse cell containing the fine cell weighs 27/64, the three
 * sharing a face 9/64, the three sharing an edge 3/64, the one sharing a vertex
 * 1/64.  On a periodic grid the coarse neighbours wrap; on a patch a coarse
 * neighbour outside the patch belongs to no multigrid level of the patch, so
 * its weight is dropped (the others are not renormalised).
 */
static void prolong_add(double *uf, const int nf[3], const double *e, int dirichlet)
{
    int nc[3] = {nf[0] / 2, nf[1] / 2, nf[2] / 2};
    for (int k = 0; k < nf[2]; k++)
        for (int j = 0; j < nf[1]; j++)
            for (int i = 0; i < nf[0]; i++) {
                int c[3] = {i, j, k};
                int par[3], oth[3];
                for (int d = 0; d < 3; d++) {
                    par[d] = c[d] / 2;
                    oth[d] = par[d] + ((c[d] % 2 == 0) ? -1 : 1);
                }
                double s = 0.0;
                for (int sel = 0; sel < 8; sel++) {
                    int cc[3];
                    double w = 1.0;
                    int valid = 1;
                    for (int d = 0; d < 3; d++) {
                        int use_other = (sel >> d) & 1;
                        cc[d] = use_other ? oth[d] : par[d];
                        w *= use_other ? 1.0 : 3.0;
                        if (cc[d] < 0 || cc[d] >= nc[d]) {
                            if (dirichlet)
                                valid = 0;
                            cc[d] = (cc[d] + nc[d]) % nc[d];
                        }
                    }
                    if (valid)
                        s += (w / 64.0) * e[idx3(nc, cc[0], cc[1], cc[2])];
                }
                uf[idx3(nf, i, j, k)] += s;
            }
}

/* Reading (level count unspecified): halve while every next size is even and >= 4. */
static int count_levels(const int n[3])
{
    int m[3] = {n[0], n[1], n[2]};
    int nl = 1;
    for (;;) {
        int ok = 1;
        for (int d = 0; d < 3; d++) {
            if (m[d] % 2 != 0)
                ok = 0;
            else {
                int nx = m[d] / 2;
                if (nx < 4 || nx % 2 != 0)
                    ok = 0;
            }
        }
        if (!ok)
            break;
        for (int d = 0; d < 3; d++)
            m[d] /= 2;
        nl++;
    }
    return nl;
}

typedef struct {
    OModel m;
    int nl;
    OLevel *lev;
    double tol, cap;
    int pre_sw, post_sw;
} OHier;

static void hier_free(OHier *H)
{
    if (!H->lev)
        return;
    for (int l = 0; l < H->nl; l++) {
        OLevel *L = &H->lev[l];
        if (l > 0) {
            free(L->u);
            free(L->rho);
        }
        free(L->f);
        free(L->uR);
        free(L->d);
        free(L->ub);
    }
    free(H->lev);
    H->lev = NULL;
}

/* Builds the level series below one grid; level 0 aliases the caller's u and rho. */
static int hier_build(OHier *H, double *u, const double *rho, const int n[3], double h,
                      int dirichlet, const double *ub0)
{
    H->nl = count_levels(n);
    H->lev = (OLevel *)calloc((size_t)H->nl, sizeof(OLevel));
    if (!H->lev)
        return ORC_ENOMEM;
    int m[3] = {n[0], n[1], n[2]};
    double hh = h;
    for (int l = 0; l < H->nl; l++) {
        OLevel *L = &H->lev[l];
        for (int d = 0; d < 3; d++)
            L->n[d] = m[d];
        L->ncell = (long)m[0] * m[1] * m[2];
        L->h = hh;
        L->pre = H->m.ct * H->m.ct / (2.0 * hh * hh);
        L->dirichlet = dirichlet;
        face_offsets(L->n, L->foff);
        if (l == 0) {
            L->u = u;
            L->rho = (double *)rho;
            L->f = NULL;
        } else {
            L->u = (double *)calloc((size_t)L->ncell, sizeof(double));
            L->rho = (double *)calloc((size_t)L->ncell, sizeof(double));
            L->f = (double *)calloc((size_t)L->ncell, sizeof(double));
            if (!L->u || !L->rho || !L->f)
                return ORC_ENOMEM;
            /* Reading: the coarse density is R rho; its terms cancel between
             * L^H(u^H) and L^H(R u^h) in the FAS equation but are kept as written. */
            restrict_avg(H->lev[l - 1].rho, H->lev[l - 1].n, L->rho);
        }
        L->uR = (double *)calloc((size_t)L->ncell, sizeof(double));
        L->d = (double *)calloc((size_t)L->ncell, sizeof(double));
        if (!L->uR || !L->d)
            return ORC_ENOMEM;
        if (dirichlet) {
            long nfs = face_size_total(L->n);
            L->ub = (double *)calloc((size_t)nfs, sizeof(double));
            if (!L->ub)
                return ORC_ENOMEM;
            if (l == 0)
                memcpy(L->ub, ub0, (size_t)nfs * sizeof(double));
            else
                restrict_faces(H->lev[l - 1].ub, H->lev[l - 1].n, L->ub);
        }
        for (int d = 0; d < 3; d++)
            m[d] /= 2;
        hh *= 2.0;
    }
    return ORC_OK;
}

/*
 * Reading (coarsest solve unspecified): Newton-Gauss-Seidel sweeps until the
 * coarse residual rms is at most max(1e-3 * initial rms, 0.1 * tol), at least
 * one sweep, at most 500.
 */
static void coarsest_solve(OHier *H, OLevel *L)
{
    residual(L, &H->m, L->d);
    double r0 = rms_of(L->d, L->ncell, NULL);
    double thr = fmax(1e-3 * r0, 0.1 * H->tol);
    for (int it = 0; it < 500; it++) {
        ngs_sweep(L, &H->m, H->cap);
        residual(L, &H->m, L->d);
        if (rms_of(L->d, L->ncell, NULL) <= thr)
            break;
    }
}

/* One FAS V-cycle starting at level l (Sec. V.B.2). */
static void vcycle(OHier *H, int l)
{
    OLevel *L = &H->lev[l];
    if (l == H->nl - 1) {
        coarsest_solve(H, L);
        return;
    }
    OLevel *C = &H->lev[l + 1];
    for (int s = 0; s < H->pre_sw; s++)
        ngs_sweep(L, &H->m, H->cap);
    /* d^h = L^h(u^h) - f^h */
    residual(L, &H->m, L->d);
    /* R u^h and R d^h */
    restrict_avg(L->u, L->n, C->uR);
    restrict_avg(L->d, L->n, C->d);
    memcpy(C->u, C->uR, (size_t)C->ncell * sizeof(double));
    /* f^H = L^H(R u^h) - R d^h  (C->f must not be read while evaluating L^H) */
    double *rd = (double *)malloc((size_t)C->ncell * sizeof(double));
    memcpy(rd, C->d, (size_t)C->ncell * sizeof(double));
    double *fsave = C->f;
    C->f = NULL;
    residual(C, &H->m, C->d); /* = L^H(R u^h) */
    C->f = fsave;
    for (long c = 0; c < C->ncell; c++)
        C->f[c] = C->d[c] - rd[c];
    free(rd);
    vcycle(H, l + 1);
    /* u^h += P (u^H - R u^h) */
    double *e = (double *)malloc((size_t)C->ncell * sizeof(double));
    for (long c = 0; c < C->ncell; c++)
        e[c] = C->u[c] - C->uR[c];
    prolong_add(L->u, L->n, e, L->dirichlet);
    free(e);
    for (int s = 0; s < H->post_sw; s++)
        ngs_sweep(L, &H->m, H->cap);
}

/* ------------------------------------------------------------------------- */
/* Public entry points (shifted variable u = u~ - ubar)                       */
/* ------------------------------------------------------------------------- */

/* Model constants in the form the tests compare against:
 * out = {c~, xi, ubar, src, bkg, dens, pre(h = 1/n0)}. */
int orc_model(double box, int n0, double a, double om, double fr0, double *out)
{
    OModel m;
    if (box <= 0 || n0 <= 0 || a <= 0 || fr0 <= 0 || om <= 0 || om >= 1)
        return ORC_EINVAL;
    model_init(&m, box, a, om, fr0, 1.0);
    double h = 1.0 / n0;
    out[0] = m.ct;
    out[1] = m.xi;
    out[2] = m.ubar;
    out[3] = m.src;
    out[4] = m.bkg;
    out[5] = m.dens;
    out[6] = m.ct * m.ct / (2.0 * h * h);
    return ORC_OK;
}

static int check_dims(const int n[3])
{
    for (int d = 0; d < 3; d++)
        if (n[d] < 2 || n[d] % 2 != 0)
            return ORC_EINVAL;
    return ORC_OK;
}

static void shift(double *u, long n, double by)
{
    for (long c = 0; c < n; c++)
        u[c] += by;
}

/* One level with caller arrays; ub (Dirichlet) given in the shifted variable. */
static int level_wrap(OLevel *L, OModel *m, double *u, const double *rho, const double *f,
                      const int n[3], double h, const double *ub, double **ubt)
{
    memset(L, 0, sizeof(*L));
    for (int d = 0; d < 3; d++)
        L->n[d] = n[d];
    L->ncell = (long)n[0] * n[1] * n[2];
    L->h = h;
    L->pre = m->ct * m->ct / (2.0 * h * h);
    L->u = u;
    L->rho = (double *)rho;
    L->f = (double *)f;
    *ubt = NULL;
    if (ub) {
        long nfs = face_size_total(n);
        *ubt = (double *)malloc((size_t)nfs * sizeof(double));
        if (!*ubt)
            return ORC_ENOMEM;
        for (long c = 0; c < nfs; c++)
            (*ubt)[c] = ub[c] + m->ubar;
        L->dirichlet = 1;
        L->ub = *ubt;
        face_offsets(n, L->foff);
    }
    return ORC_OK;
}

/* d = L(u) - f for one level (f may be NULL = 0, ub NULL = periodic). */
int orc_residual(const double *u, const double *rho, const double *f, const int n[3], double h,
                 double box, double a, double om, double fr0, const double *ub, double *d)
{
    if (check_dims(n) != ORC_OK)
        return ORC_EINVAL;
    OModel m;
    model_init(&m, box, a, om, fr0, 1.0);
    long nc = (long)n[0] * n[1] * n[2];
    double *ut = (double *)malloc((size_t)nc * sizeof(double));
    if (!ut)
        return ORC_ENOMEM;
    memcpy(ut, u, (size_t)nc * sizeof(double));
    shift(ut, nc, m.ubar);
    OLevel L;
    double *ubt;
    if (level_wrap(&L, &m, ut, rho, f, n, h, ub, &ubt) != ORC_OK) {
        free(ut);
        return ORC_ENOMEM;
    }
    residual(&L, &m, d);
    free(ubt);
    free(ut);
    return ORC_OK;
}

/* L and dL/du at one cell (for derivative checks). */
int orc_cell_op(const double *u, const double *rho, const int n[3], double h, double box,
                double a, double om, double fr0, const double *ub, int i, int j, int k,
                double *out2)
{
    if (check_dims(n) != ORC_OK)
        return ORC_EINVAL;
    OModel m;
    model_init(&m, box, a, om, fr0, 1.0);
    long nc = (long)n[0] * n[1] * n[2];
    double *ut = (double *)malloc((size_t)nc * sizeof(double));
    if (!ut)
        return ORC_ENOMEM;
    memcpy(ut, u, (size_t)nc * sizeof(double));
    shift(ut, nc, m.ubar);
    OLevel L;
    double *ubt;
    level_wrap(&L, &m, ut, rho, NULL, n, h, ub, &ubt);
    cell_op(&L, &m, i, j, k, &out2[0], &out2[1]);
    free(ubt);
    free(ut);
    return ORC_OK;
}

/* nsweeps red-black NGS sweeps on one level, in place. */
int orc_smooth(double *u, const double *rho, const double *f, const int n[3], double h,
               double box, double a, double om, double fr0, const double *ub, int nsweeps,
               double cap)
{
    if (check_dims(n) != ORC_OK)
        return ORC_EINVAL;
    OModel m;
    model_init(&m, box, a, om, fr0, 1.0);
    long nc = (long)n[0] * n[1] * n[2];
    shift(u, nc, m.ubar);
    OLevel L;
    double *ubt;
    level_wrap(&L, &m, u, rho, f, n, h, ub, &ubt);
    for (int s = 0; s < nsweeps; s++)
        ngs_sweep(&L, &m, cap);
    shift(u, nc, -m.ubar);
    free(ubt);
    return ORC_OK;
}

int orc_restrict(const double *fine, const int nf[3], double *coarse)
{
    if (check_dims(nf) != ORC_OK)
        return ORC_EINVAL;
    restrict_avg(fine, nf, coarse);
    return ORC_OK;
}

/* Coarse boundary-face values of a patch from its fine ones (restrict_faces),
 * packed as the faces of nf and of nf / 2. */
int orc_restrict_faces(const double *ubf, const int nf[3], double *ubc)
{
    if (check_dims(nf) != ORC_OK)
        return ORC_EINVAL;
    restrict_faces(ubf, nf, ubc);
    return ORC_OK;
}

/* uf += P (uH - uR) on a fine grid of size nf. */
int orc_prolong_correct(double *uf, const int nf[3], const double *uH, const double *uR,
                        int dirichlet)
{
    if (check_dims(nf) != ORC_OK)
        return ORC_EINVAL;
    long ncc = (long)(nf[0] / 2) * (nf[1] / 2) * (nf[2] / 2);
    double *e = (double *)malloc((size_t)ncc * sizeof(double));
    if (!e)
        return ORC_ENOMEM;
    for (long c = 0; c < ncc; c++)
        e[c] = uH[c] - uR[c];
    prolong_add(uf, nf, e, dirichlet);
    free(e);
    return ORC_OK;
}

int orc_num_levels(const int n[3])
{
    return count_levels(n);
}

/*
 * Solve one grid to rms(L(u)) <= tol with FAS V-cycles (pre/post NGS sweeps).
 * ub == NULL: periodic domain grid of cell size h.  Otherwise a patch with
 * the given packed boundary values (shifted variable).
 * ncycles_fixed > 0 runs exactly that many cycles with no convergence test.
 * hist (optional, length max_cycles + 1) receives the rms after each cycle,
 * hist[0] the initial one.  Returns ORC_ENOCONV if tol was not reached.
 */
int orc_solve_grid(const double *rho, const int n[3], double h, double box, double a, double om,
                   double fr0, const double *ub, double tol, int max_cycles, int pre, int post,
                   double cap, int ncycles_fixed, double *u_inout, int *cycles_out,
                   double *hist, double *res_out)
{
    if (check_dims(n) != ORC_OK || a <= 0 || fr0 <= 0 || box <= 0 || h <= 0)
        return ORC_EINVAL;
    OHier H;
    memset(&H, 0, sizeof(H));
    model_init(&H.m, box, a, om, fr0, 1.0);
    H.tol = tol;
    H.cap = cap;
    H.pre_sw = pre;
    H.post_sw = post;
    long nc = (long)n[0] * n[1] * n[2];
    shift(u_inout, nc, H.m.ubar);
    double *ubt = NULL;
    if (ub) {
        long nfs = face_size_total(n);
        ubt = (double *)malloc((size_t)nfs * sizeof(double));
        for (long c = 0; c < nfs; c++)
            ubt[c] = ub[c] + H.m.ubar;
    }
    int st = hier_build(&H, u_inout, rho, n, h, ub != NULL, ubt);
    if (st != ORC_OK) {
        hier_free(&H);
        free(ubt);
        shift(u_inout, nc, -H.m.ubar);
        return st;
    }
    OLevel *L0 = &H.lev[0];
    residual(L0, &H.m, L0->d);
    double rms = rms_of(L0->d, nc, NULL);
    if (hist)
        hist[0] = rms;
    int cyc = 0;
    if (ncycles_fixed > 0) {
        for (cyc = 0; cyc < ncycles_fixed; cyc++) {
            vcycle(&H, 0);
            residual(L0, &H.m, L0->d);
            rms = rms_of(L0->d, nc, NULL);
            if (hist)
                hist[cyc + 1] = rms;
        }
    } else {
        while (rms > tol && cyc < max_cycles) {
            vcycle(&H, 0);
            cyc++;
            residual(L0, &H.m, L0->d);
            rms = rms_of(L0->d, nc, NULL);
            if (hist)
                hist[cyc] = rms;
        }
    }
    if (cycles_out)
        *cycles_out = cyc;
    if (res_out)
        res_out[0] = rms;
    shift(u_inout, nc, -H.m.ubar);
    hier_free(&H);
    free(ubt);
    if (ncycles_fixed <= 0 && !(rms <= tol))
        return ORC_ENOCONV;
    return ORC_OK;
}

/* ------------------------------------------------------------------------- */
/* Refinement-patch boundary conditions (Sec. V.A.1, V.B.1, VI.B)             */
/* ------------------------------------------------------------------------- */

/* Trilinear value (weights 27/9/3/1 over 64) at the fine cell with index g[3]
 * (g relative to the patch's lower corner, may be -1 or n for ghosts), using
 * the parent cell containing it and the parent neighbours on its side. */
static int parent_interp(const double *up, const int np_[3], int periodic, const int org[3],
                         const int g[3], double *val)
{
    double s = 0.0;
    int par[3], oth[3];
    for (int d = 0; d < 3; d++) {
        int fg = 2 * org[d] + g[d]; /* fine index in the parent's doubled frame */
        int pc = (fg >= 0) ? fg / 2 : -((-fg + 1) / 2);
        par[d] = pc;
        oth[d] = pc + ((fg - 2 * pc == 0) ? -1 : 1);
    }
    for (int sel = 0; sel < 8; sel++) {
        int cc[3];
        double w = 1.0;
        for (int d = 0; d < 3; d++) {
            int use_other = (sel >> d) & 1;
            cc[d] = use_other ? oth[d] : par[d];
            w *= use_other ? 1.0 : 3.0;
            if (cc[d] < 0 || cc[d] >= np_[d]) {
                if (!periodic)
                    return ORC_EINVAL;
                cc[d] = ((cc[d] % np_[d]) + np_[d]) % np_[d];
            }
        }
        s += (w / 64.0) * up[idx3(np_, cc[0], cc[1], cc[2])];
    }
    *val = s;
    return ORC_OK;
}

/*
 * Boundary set-up of one patch of n[3] fine cells (refinement factor 2) whose
 * lower corner sits at parent cell org[3].  Reading of Sec. V.A.1/V.B.1 ("the
 * ghost value is computed from its father cell"): the initial patch u and every
 * ghost u are the trilinear interpolation of the parent solution; then
 * u_b = (u_ghost + u_first_interior)/2 is fixed for the solve.  All values are
 * in the shifted variable (the shift is common to parent and patch).
 * Returns ORC_EINVAL if an interpolation stencil leaves a non-periodic parent.
 */
int orc_patch_bc(const double *uparent, const int np_[3], int parent_periodic, const int org[3],
                 const int n[3], double *u_init, double *ub_out)
{
    if (check_dims(n) != ORC_OK)
        return ORC_EINVAL;
    for (int k = 0; k < n[2]; k++)
        for (int j = 0; j < n[1]; j++)
            for (int i = 0; i < n[0]; i++) {
                int g[3] = {i, j, k};
                if (parent_interp(uparent, np_, parent_periodic, org, g,
                                  &u_init[idx3(n, i, j, k)]) != ORC_OK)
                    return ORC_EINVAL;
            }
    long foff[6];
    face_offsets(n, foff);
    for (int f = 0; f < 6; f++) {
        int ax = f / 2, p, q;
        face_axes(ax, &p, &q);
        for (int Q = 0; Q < n[q]; Q++)
            for (int P = 0; P < n[p]; P++) {
                int inner[3], ghost[3];
                inner[p] = ghost[p] = P;
                inner[q] = ghost[q] = Q;
                inner[ax] = (f % 2) ? n[ax] - 1 : 0;
                ghost[ax] = (f % 2) ? n[ax] : -1;
                double ug, ui;
                if (parent_interp(uparent, np_, parent_periodic, org, ghost, &ug) != ORC_OK)
                    return ORC_EINVAL;
                ui = u_init[idx3(n, inner[0], inner[1], inner[2])];
                ub_out[foff[f] + (long)Q * n[p] + P] = 0.5 * (ug + ui);
            }
    }
    return ORC_OK;
}

/* ------------------------------------------------------------------------- */
/* Cloud-in-cell density assignment (Sec. VI.C)                               */
/* ------------------------------------------------------------------------- */

/*
 * rho~ on an n[3] periodic grid from np particles at positions pos[np][3] in
 * box units [0,1).  Each particle carries mass n0 n1 n2 / np (mean density 1,
 * Sec. III.A) and spreads it over the 8 nearest cell centres with weights
 * prod_d (1 - |x_d - x_c,d| / h_d); cell centres at (i + 1/2) h.
 */
int orc_cic(const double *pos, long np, const int n[3], double *rho)
{
    if (np <= 0 || n[0] <= 0 || n[1] <= 0 || n[2] <= 0)
        return ORC_EINVAL;
    long nc = (long)n[0] * n[1] * n[2];
    memset(rho, 0, (size_t)nc * sizeof(double));
    double mass = (double)nc / (double)np;
    for (long p = 0; p < np; p++) {
        int i0[3];
        double t[3];
        for (int d = 0; d < 3; d++) {
            double x = pos[3 * p + d] * n[d] - 0.5; /* in cell-centre units */
            double fl = floor(x);
            i0[d] = (int)fl;
            t[d] = x - fl;
        }
        for (int sel = 0; sel < 8; sel++) {
            int c[3];
            double w = mass;
            for (int d = 0; d < 3; d++) {
                int hi = (sel >> d) & 1;
                c[d] = i0[d] + hi;
                c[d] = ((c[d] % n[d]) + n[d]) % n[d];
                w *= hi ? t[d] : (1.0 - t[d]);
            }
            rho[idx3(n, c[0], c[1], c[2])] += w;
        }
    }
    return ORC_OK;
}
