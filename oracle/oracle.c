/*
 * oracle.c -- plain, slow, obviously-correct FP64 CPU oracle of the hybrid
 * Linear / CWENOZ / MUSCL finite-volume residual of Tong & Tsoutsanis,
 * "A Hybrid Finite-Volume Reconstruction Framework for Efficient High-Order
 * Shock-Capturing on Unstructured Meshes" (arXiv 2510.25906).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check and the
 * benchmark's CPU-baseline leg may load this library.  It shares no code,
 * header, table or constant with the CUDA path.
 *
 * It takes the paper's steps in the paper's order, one cell at a time, with
 * straightforward loops:
 *   Sec. 2 (eq. EulerEquationsDetails)      finite-volume residual
 *   Sec. 2.1 (eqs. AVGVariables1/2, dofMatrix and the pseudo-inverse)
 *                                            least-squares reconstruction
 *   Sec. 2.2                                MUSCL with Barth-Jespersen or
 *                                            Venkatakrishnan's limiter
 *   Sec. 2.3 (CWENOZ weights, tau, SI, OI)  CWENOZ, in conserved or
 *                                            characteristic variables
 *   Sec. 2.4 (eq. harten_jump_fix)          TVD bound, first-order fallback
 *   Sec. 2.5 (eqs. DMP, NADMUSCL, NADCWENOZ, marginm, marginw,
 *             NADDeactivatedCriteria(_2)) and the closing description of
 *             the hybrid pipeline           detector, tagging, pipeline
 *   Sec. 2 (eqs. EulerEquationsDetails, HeatConduct, viscous_jump)
 *                                            viscous flux, heat conduction
 *   SSP-RK3 (Shu-Osher) and SSP-RK(5,4) (Spiteri-Ruuth) time steps
 * Readings taken where the paper is silent or garbled are stated next to the
 * code that uses them.  Every step is pinned by the CPU tests
 * (tests/test_oracle_*.py) to closed forms, invariants, library routines,
 * brute force or the paper's own statements; none is left unpinned.
 *
 * Basis: monomials xi^a eta^b zeta^c of total degree 1..r in the reference
 * coordinates of the considered cell, made mean-free over that cell.  The
 * fitted polynomial does not depend on the basis (the least-squares problem
 * is posed on the polynomial space), so this gives the same reconstruction
 * as the paper's Legendre basis; the smoothness indicator is a property of
 * the polynomial itself and is likewise basis-free.
 *
 * Quadrature: every volume integral uses a tensor Gauss-Legendre rule with
 * r+2 points per direction on a map from the unit square / cube (collapsed
 * for triangles, tetrahedra, prisms and pyramids).  That rule is exact for
 * every integrand used here.  Face integrals use Gauss-Legendre with
 * ceil((r+1)/2) points per direction on edges and on the quadrilaterals of
 * all-hexahedral meshes; a mesh with triangular faces uses the collapsed
 * rule with ceil((r+2)/2) points per direction on them, and as many per
 * direction on its quadrilaterals.
 */
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#define OR_TRI 1
#define OR_QUAD 2
#define OR_TET 3
#define OR_HEX 4
#define OR_PRISM 5
#define OR_PYRAMID 6

#define C_LIN 0
#define C_CW 1
#define C_MU 2
#define C_FIRST 3

#define MAXNF 6
#define MAXV 8

static char g_err[512];
const char* or_last_error(void) { return g_err; }
static int fail(const char* m) { snprintf(g_err, sizeof g_err, "%s", m); return -1; }

/* ------------------------------------------------------------------------ */
/* cell-type tables (local vertex order fixed by the mesh format)            */
/* ------------------------------------------------------------------------ */
static const int TRI_F[3][2] = {{0, 1}, {1, 2}, {2, 0}};
static const int QUAD_F[4][2] = {{0, 1}, {1, 2}, {2, 3}, {3, 0}};
/* hexahedron faces listed so that (c-a) x (d-b) points outward */
static const int HEX_F[6][4] = {{0, 3, 2, 1}, {4, 5, 6, 7}, {0, 1, 5, 4},
                                {1, 2, 6, 5}, {2, 3, 7, 6}, {3, 0, 4, 7}};

/* tetrahedron (positively oriented v0 v1 v2 v3) faces, each listed so that
 * (b-a) x (c-a) points outward: the face opposite vertex k is face k */
static const int TET_F[4][3] = {{1, 2, 3}, {0, 3, 2}, {0, 1, 3}, {0, 2, 1}};

/* prism: triangles v0 v1 v2 and v3 v4 v5 (v3 over v0), then the three
 * quadrilateral sides; pyramid: the four triangles to the apex v4, then the
 * base v0 v1 v2 v3 (counter-clockwise seen from the apex).  Every face is
 * listed with its area vector pointing out. */
static const int PRISM_F[5][4] = {{0, 2, 1, -1}, {3, 4, 5, -1}, {0, 1, 4, 3}, {1, 2, 5, 4}, {2, 0, 3, 5}};
static const int PYR_F[5][4] = {{0, 1, 4, -1}, {1, 2, 4, -1}, {2, 3, 4, -1}, {3, 0, 4, -1}, {0, 3, 2, 1}};

static int t_nverts(int t)
{
    switch (t) {
    case OR_TRI: return 3;
    case OR_QUAD: case OR_TET: return 4;
    case OR_PYRAMID: return 5;
    case OR_PRISM: return 6;
    case OR_HEX: return 8;
    }
    return 0;
}
static int t_nfaces(int t)
{
    switch (t) {
    case OR_TRI: return 3;
    case OR_QUAD: case OR_TET: return 4;
    case OR_PRISM: case OR_PYRAMID: return 5;
    case OR_HEX: return 6;
    }
    return 0;
}
/* vertices of face f of a type-t cell */
static int t_fnv(int t, int f)
{
    if (t == OR_TRI || t == OR_QUAD) return 2;
    if (t == OR_TET) return 3;
    if (t == OR_PRISM) return PRISM_F[f][3] < 0 ? 3 : 4;
    if (t == OR_PYRAMID) return PYR_F[f][3] < 0 ? 3 : 4;
    return 4;
}
static int t_fv(int t, int f, int k)
{
    switch (t) {
    case OR_TRI: return TRI_F[f][k];
    case OR_QUAD: return QUAD_F[f][k];
    case OR_TET: return TET_F[f][k];
    case OR_PRISM: return PRISM_F[f][k];
    case OR_PYRAMID: return PYR_F[f][k];
    }
    return HEX_F[f][k];
}

/* ------------------------------------------------------------------------ */
/* Gauss-Legendre on [0,1] by Newton iteration on P_n                         */
/* ------------------------------------------------------------------------ */
void or_gauss_legendre(int n, double* x, double* w)
{
    for (int i = 0; i < n; ++i) {
        double z = cos(M_PI * (i + 0.75) / (n + 0.5)), dp = 0.0;
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = z; /* P_0, P_1 */
            for (int k = 2; k <= n; ++k) {
                double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
                p0 = p1; p1 = p2;
            }
            if (n == 1) { p1 = z; p0 = 1.0; }
            dp = n * (z * p1 - p0) / (z * z - 1.0);
            double dz = p1 / dp;
            z -= dz;
            if (fabs(dz) < 1e-16) break;
        }
        {   /* recompute P_n' at the converged root for the weight */
            double p0 = 1.0, p1 = z;
            for (int k = 2; k <= n; ++k) {
                double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
                p0 = p1; p1 = p2;
            }
            dp = n * (z * p1 - p0) / (z * z - 1.0);
        }
        x[n - 1 - i] = 0.5 * (z + 1.0);                 /* ascending on [0,1] */
        w[n - 1 - i] = 1.0 / ((1.0 - z * z) * dp * dp);  /* 2/((1-z^2)P'^2) / 2 */
    }
}

/* Quadrature over one cell given its vertices (row-major [nv][3]).  Points
 * and weights (Jacobian included) are appended to px (stride 3) / pw. */
static int cell_rule(int type, const double* v, int n, double* px, double* pw)
{
    double gx[16], gw[16];
    or_gauss_legendre(n, gx, gw);
    int np = 0;
    if (type == OR_TRI) {
        /* collapsed map x = p0 + s (p1-p0) + s t (p2-p1), |J| = s |det| */
        double e1x = v[3] - v[0], e1y = v[4] - v[1], e2x = v[6] - v[3], e2y = v[7] - v[4];
        double det = fabs(e1x * e2y - e1y * e2x);
        for (int i = 0; i < n; ++i)
            for (int j = 0; j < n; ++j) {
                double s = gx[i], t = gx[j];
                px[3 * np + 0] = v[0] + s * e1x + s * t * e2x;
                px[3 * np + 1] = v[1] + s * e1y + s * t * e2y;
                px[3 * np + 2] = 0.0;
                pw[np++] = gw[i] * gw[j] * s * det;
            }
    } else if (type == OR_QUAD) {
        for (int i = 0; i < n; ++i)
            for (int j = 0; j < n; ++j) {
                double s = gx[i], t = gx[j];
                double N0 = (1 - s) * (1 - t), N1 = s * (1 - t), N2 = s * t, N3 = (1 - s) * t;
                double xs[2], xt[2];
                for (int d = 0; d < 2; ++d) {
                    xs[d] = (1 - t) * (v[3 + d] - v[0 + d]) + t * (v[6 + d] - v[9 + d]);
                    xt[d] = (1 - s) * (v[9 + d] - v[0 + d]) + s * (v[6 + d] - v[3 + d]);
                    px[3 * np + d] = N0 * v[d] + N1 * v[3 + d] + N2 * v[6 + d] + N3 * v[9 + d];
                }
                px[3 * np + 2] = 0.0;
                pw[np++] = gw[i] * gw[j] * fabs(xs[0] * xt[1] - xs[1] * xt[0]);
            }
    } else if (type == OR_TET) {
        /* collapsed map x = p0 + s a + s t b + s t u c with a = p1-p0,
         * b = p2-p1, c = p3-p2: |J| = s^2 t |det(a, b, c)| */
        double a[3], b[3], cc[3];
        for (int d = 0; d < 3; ++d) { a[d] = v[3 + d] - v[d]; b[d] = v[6 + d] - v[3 + d]; cc[d] = v[9 + d] - v[6 + d]; }
        double det = fabs(a[0] * (b[1] * cc[2] - b[2] * cc[1]) - a[1] * (b[0] * cc[2] - b[2] * cc[0])
                          + a[2] * (b[0] * cc[1] - b[1] * cc[0]));
        for (int i = 0; i < n; ++i)
            for (int j = 0; j < n; ++j)
                for (int k = 0; k < n; ++k) {
                    double s1 = gx[i], t = gx[j], u = gx[k];
                    for (int d = 0; d < 3; ++d) px[3 * np + d] = v[d] + s1 * a[d] + s1 * t * b[d] + s1 * t * u * cc[d];
                    pw[np++] = gw[i] * gw[j] * gw[k] * s1 * s1 * t * det;
                }
    } else if (type == OR_PRISM) {
        /* x = (1-z) [T0 + a (T1-T0) + a b (T2-T1)] + z [same on the top
         * triangle], the bottom triangle T0 T1 T2 = v0 v1 v2 and the top
         * v3 v4 v5 in collapsed coordinates (a, b); |J| = a |det dx/d(p, q, z)|
         * with (p, q) = (a (1-b), a b) the triangle's barycentric pair */
        for (int i = 0; i < n; ++i)
            for (int j = 0; j < n; ++j)
                for (int k = 0; k < n; ++k) {
                    double a = gx[i], b = gx[j], z = gx[k];
                    double p = a * (1.0 - b), q = a * b, Jm[3][3];
                    for (int d = 0; d < 3; ++d) {
                        double lo = v[d] + p * (v[3 + d] - v[d]) + q * (v[6 + d] - v[d]);
                        double hi = v[9 + d] + p * (v[12 + d] - v[9 + d]) + q * (v[15 + d] - v[9 + d]);
                        px[3 * np + d] = lo + z * (hi - lo);
                        Jm[d][0] = (1.0 - z) * (v[3 + d] - v[d]) + z * (v[12 + d] - v[9 + d]);
                        Jm[d][1] = (1.0 - z) * (v[6 + d] - v[d]) + z * (v[15 + d] - v[9 + d]);
                        Jm[d][2] = hi - lo;
                    }
                    double det = Jm[0][0] * (Jm[1][1] * Jm[2][2] - Jm[1][2] * Jm[2][1])
                               - Jm[0][1] * (Jm[1][0] * Jm[2][2] - Jm[1][2] * Jm[2][0])
                               + Jm[0][2] * (Jm[1][0] * Jm[2][1] - Jm[1][1] * Jm[2][0]);
                    pw[np++] = gw[i] * gw[j] * gw[k] * a * fabs(det);
                }
    } else if (type == OR_PYRAMID) {
        /* the cone from the apex v4 over the bilinear base: x = B(s, t) +
         * u (v4 - B(s, t)), B(0,0) = v0, B(1,0) = v1, B(1,1) = v2, B(0,1) = v3 */
        for (int i = 0; i < n; ++i)
            for (int j = 0; j < n; ++j)
                for (int k = 0; k < n; ++k) {
                    double s = gx[i], t = gx[j], u = gx[k], Jm[3][3];
                    for (int d = 0; d < 3; ++d) {
                        double B = (1 - s) * (1 - t) * v[d] + s * (1 - t) * v[3 + d] + s * t * v[6 + d] + (1 - s) * t * v[9 + d];
                        double Bs = (1 - t) * (v[3 + d] - v[d]) + t * (v[6 + d] - v[9 + d]);
                        double Bt = (1 - s) * (v[9 + d] - v[d]) + s * (v[6 + d] - v[3 + d]);
                        px[3 * np + d] = B + u * (v[12 + d] - B);
                        Jm[d][0] = (1 - u) * Bs;
                        Jm[d][1] = (1 - u) * Bt;
                        Jm[d][2] = v[12 + d] - B;
                    }
                    double det = Jm[0][0] * (Jm[1][1] * Jm[2][2] - Jm[1][2] * Jm[2][1])
                               - Jm[0][1] * (Jm[1][0] * Jm[2][2] - Jm[1][2] * Jm[2][0])
                               + Jm[0][2] * (Jm[1][0] * Jm[2][1] - Jm[1][1] * Jm[2][0]);
                    pw[np++] = gw[i] * gw[j] * gw[k] * fabs(det);
                }
    } else if (type == OR_HEX) {
        /* trilinear map over the unit cube; vertex k sits at corner (sx,sy,sz) */
        static const int cs[8][3] = {{0, 0, 0}, {1, 0, 0}, {1, 1, 0}, {0, 1, 0},
                                     {0, 0, 1}, {1, 0, 1}, {1, 1, 1}, {0, 1, 1}};
        for (int i = 0; i < n; ++i)
            for (int j = 0; j < n; ++j)
                for (int k = 0; k < n; ++k) {
                    double u[3] = {gx[i], gx[j], gx[k]};
                    double X[3] = {0, 0, 0}, Jm[3][3] = {{0}};
                    for (int a = 0; a < 8; ++a) {
                        double f[3], df[3];
                        for (int d = 0; d < 3; ++d) {
                            f[d] = cs[a][d] ? u[d] : 1.0 - u[d];
                            df[d] = cs[a][d] ? 1.0 : -1.0;
                        }
                        double Nv = f[0] * f[1] * f[2];
                        double dN[3] = {df[0] * f[1] * f[2], f[0] * df[1] * f[2], f[0] * f[1] * df[2]};
                        for (int d = 0; d < 3; ++d) {
                            X[d] += Nv * v[3 * a + d];
                            /* differences to v0: the shape-function gradients sum to zero */
                            for (int e = 0; e < 3; ++e) Jm[d][e] += (v[3 * a + d] - v[d]) * dN[e];
                        }
                    }
                    double det = Jm[0][0] * (Jm[1][1] * Jm[2][2] - Jm[1][2] * Jm[2][1])
                               - Jm[0][1] * (Jm[1][0] * Jm[2][2] - Jm[1][2] * Jm[2][0])
                               + Jm[0][2] * (Jm[1][0] * Jm[2][1] - Jm[1][1] * Jm[2][0]);
                    for (int d = 0; d < 3; ++d) px[3 * np + d] = X[d];
                    pw[np++] = gw[i] * gw[j] * gw[k] * fabs(det);
                }
    } else {
        return -1;
    }
    return np;
}

/* ------------------------------------------------------------------------ */
/* Mesh                                                                       */
/* ------------------------------------------------------------------------ */
typedef struct {
    int dim;
    int64_t nn, nc, nface;
    double* xyz;      /* [nn][3] (z = 0 in 2D) */
    uint8_t* type;
    int64_t* cptr;
    int32_t* cidx;
    double period[3];
    /* connectivity */
    int32_t* nbr;     /* [nc][MAXNF] neighbour across local face, -1 boundary */
    int8_t* nbrf;     /* [nc][MAXNF] local face index inside the neighbour */
    int64_t* cface;   /* [nc][MAXNF] global face id */
    /* faces: owner o (smaller cell id), other side n (-1 on boundary) */
    int32_t *fo, *fn;
    int8_t *ffo, *ffn;
    double* fshift;   /* [nface][3]: x_other + shift = x in owner's frame */
    double* fnorm;    /* [nface][3] unit normal, outward from the owner */
    double* farea;    /* [nface] */
    /* geometry */
    double* vol;      /* [nc] */
    double* cen;      /* [nc][3] centroid */
    double* vmean;    /* [nc][3] vertex mean */
} or_mesh;

static void cell_verts(const or_mesh* m, int64_t c, double* v)
{
    int nv = t_nverts(m->type[c]);
    for (int k = 0; k < nv; ++k)
        for (int d = 0; d < 3; ++d) v[3 * k + d] = m->xyz[3 * (int64_t)m->cidx[m->cptr[c] + k] + d];
}

/* half-face record used for matching */
typedef struct { int64_t key[4]; int64_t cell; int face; } hface;
static int hface_cmp(const void* a, const void* b)
{
    const hface* x = (const hface*)a; const hface* y = (const hface*)b;
    for (int k = 0; k < 4; ++k) {
        if (x->key[k] < y->key[k]) return -1;
        if (x->key[k] > y->key[k]) return 1;
    }
    if (x->cell != y->cell) return x->cell < y->cell ? -1 : 1;
    return x->face - y->face;
}
static void sort4(int64_t* k, int n)
{
    for (int i = 0; i < n; ++i)
        for (int j = i + 1; j < n; ++j)
            if (k[j] < k[i]) { int64_t t = k[i]; k[i] = k[j]; k[j] = t; }
}

static void face_centre(const or_mesh* m, int64_t c, int f, double* x)
{
    int t = m->type[c], fnv = t_fnv(t, f);
    x[0] = x[1] = x[2] = 0.0;
    for (int k = 0; k < fnv; ++k)
        for (int d = 0; d < 3; ++d) x[d] += m->xyz[3 * (int64_t)m->cidx[m->cptr[c] + t_fv(t, f, k)] + d];
    for (int d = 0; d < 3; ++d) x[d] /= fnv;
}

/* area vector of a local face (outward from cell c) */
static void face_areavec(const or_mesh* m, int64_t c, int f, double* A)
{
    int t = m->type[c], fnv = t_fnv(t, f);
    double P[4][3];
    for (int k = 0; k < fnv; ++k)
        for (int d = 0; d < 3; ++d) P[k][d] = m->xyz[3 * (int64_t)m->cidx[m->cptr[c] + t_fv(t, f, k)] + d];
    if (fnv == 2) {
        /* counter-clockwise cell: outward normal of edge a->b is (dy, -dx) */
        A[0] = P[1][1] - P[0][1]; A[1] = -(P[1][0] - P[0][0]); A[2] = 0.0;
    } else if (fnv == 3) {
        double u[3], w[3];
        for (int d = 0; d < 3; ++d) { u[d] = P[1][d] - P[0][d]; w[d] = P[2][d] - P[0][d]; }
        A[0] = 0.5 * (u[1] * w[2] - u[2] * w[1]);
        A[1] = 0.5 * (u[2] * w[0] - u[0] * w[2]);
        A[2] = 0.5 * (u[0] * w[1] - u[1] * w[0]);
    } else {
        double u[3], w[3];
        for (int d = 0; d < 3; ++d) { u[d] = P[2][d] - P[0][d]; w[d] = P[3][d] - P[1][d]; }
        A[0] = 0.5 * (u[1] * w[2] - u[2] * w[1]);
        A[1] = 0.5 * (u[2] * w[0] - u[0] * w[2]);
        A[2] = 0.5 * (u[0] * w[1] - u[1] * w[0]);
    }
}

void or_mesh_free(or_mesh* m)
{
    if (!m) return;
    free(m->xyz); free(m->type); free(m->cptr); free(m->cidx);
    free(m->nbr); free(m->nbrf); free(m->cface);
    free(m->fo); free(m->fn); free(m->ffo); free(m->ffn); free(m->fshift); free(m->fnorm); free(m->farea);
    free(m->vol); free(m->cen); free(m->vmean);
    free(m);
}

or_mesh* or_mesh_create(int dim, int64_t nn, int64_t nc, const double* xyz, const uint8_t* type,
                        const int64_t* cptr, const int32_t* cidx, const double* period)
{
    if (dim != 2 && dim != 3) { fail("dim must be 2 or 3"); return NULL; }
    if (nn <= 0 || nc <= 0 || nc > (int64_t)1 << 31) { fail("bad mesh sizes"); return NULL; }
    or_mesh* m = (or_mesh*)calloc(1, sizeof(or_mesh));
    m->dim = dim; m->nn = nn; m->nc = nc;
    m->xyz = (double*)calloc(3 * nn, sizeof(double));
    for (int64_t i = 0; i < nn; ++i)
        for (int d = 0; d < dim; ++d) m->xyz[3 * i + d] = xyz[dim * i + d];
    m->type = (uint8_t*)malloc(nc);
    memcpy(m->type, type, nc);
    m->cptr = (int64_t*)malloc((nc + 1) * sizeof(int64_t));
    memcpy(m->cptr, cptr, (nc + 1) * sizeof(int64_t));
    m->cidx = (int32_t*)malloc(cptr[nc] * sizeof(int32_t));
    memcpy(m->cidx, cidx, cptr[nc] * sizeof(int32_t));
    for (int d = 0; d < 3; ++d) m->period[d] = d < dim ? period[d] : 0.0;
    for (int64_t c = 0; c < nc; ++c) {
        int t = type[c];
        if ((dim == 2 && t != OR_TRI && t != OR_QUAD) ||
            (dim == 3 && t != OR_HEX && t != OR_TET && t != OR_PRISM && t != OR_PYRAMID) ||
            cptr[c + 1] - cptr[c] != t_nverts(t)) { fail("unsupported cell type or vertex count"); or_mesh_free(m); return NULL; }
    }

    /* ---- match half-faces by their vertex sets ---- */
    int64_t nh = 0;
    for (int64_t c = 0; c < nc; ++c) nh += t_nfaces(type[c]);
    hface* H = (hface*)malloc(nh * sizeof(hface));
    int64_t h = 0;
    for (int64_t c = 0; c < nc; ++c) {
        int t = type[c];
        for (int f = 0; f < t_nfaces(t); ++f, ++h) {
            int fnv = t_fnv(t, f);
            for (int k = 0; k < 4; ++k) H[h].key[k] = k < fnv ? cidx[cptr[c] + t_fv(t, f, k)] : -1;
            sort4(H[h].key, fnv);
            H[h].cell = c; H[h].face = f;
        }
    }
    qsort(H, nh, sizeof(hface), hface_cmp);
    m->nbr = (int32_t*)malloc(nc * MAXNF * sizeof(int32_t));
    m->nbrf = (int8_t*)malloc(nc * MAXNF);
    double* nsh = (double*)calloc(nc * MAXNF * 3, sizeof(double)); /* neighbour shift per half-face */
    for (int64_t i = 0; i < nc * MAXNF; ++i) { m->nbr[i] = -1; m->nbrf[i] = -1; }
    hface* U = (hface*)malloc(nh * sizeof(hface)); /* unmatched */
    int64_t nu = 0;
    for (int64_t i = 0; i < nh;) {
        int64_t j = i + 1;
        while (j < nh && memcmp(H[j].key, H[i].key, sizeof H[i].key) == 0) ++j;
        if (j - i == 2) {
            hface *a = &H[i], *b = &H[i + 1];
            m->nbr[a->cell * MAXNF + a->face] = (int32_t)b->cell; m->nbrf[a->cell * MAXNF + a->face] = (int8_t)b->face;
            m->nbr[b->cell * MAXNF + b->face] = (int32_t)a->cell; m->nbrf[b->cell * MAXNF + b->face] = (int8_t)a->face;
        } else if (j - i == 1) {
            U[nu++] = H[i];
        } else {
            free(H); free(U); free(nsh); fail("a face is shared by more than two cells"); or_mesh_free(m); return NULL;
        }
        i = j;
    }
    /* ---- periodic pairing of the remaining faces by wrapped face centres ---- */
    int periodic = 0;
    for (int d = 0; d < dim; ++d) periodic |= m->period[d] > 0.0;
    if (periodic && nu > 0) {
        for (int64_t i = 0; i < nu; ++i) {
            double x[3];
            face_centre(m, U[i].cell, U[i].face, x);
            for (int d = 0; d < 3; ++d) {
                if (m->period[d] > 0.0) {
                    const int64_t S = (int64_t)1 << 30;
                    int64_t q = llround(x[d] / m->period[d] * (double)S);
                    q %= S; if (q < 0) q += S;
                    U[i].key[d] = q;
                } else {
                    U[i].key[d] = llround(x[d] * 1073741824.0);
                }
            }
            U[i].key[3] = 0;
        }
        qsort(U, nu, sizeof(hface), hface_cmp);
        int64_t nr = 0;
        for (int64_t i = 0; i < nu;) {
            int64_t j = i + 1;
            while (j < nu && memcmp(U[j].key, U[i].key, sizeof U[i].key) == 0) ++j;
            if (j - i == 2) {
                hface *a = &U[i], *b = &U[i + 1];
                double xa[3], xb[3];
                face_centre(m, a->cell, a->face, xa);
                face_centre(m, b->cell, b->face, xb);
                m->nbr[a->cell * MAXNF + a->face] = (int32_t)b->cell; m->nbrf[a->cell * MAXNF + a->face] = (int8_t)b->face;
                m->nbr[b->cell * MAXNF + b->face] = (int32_t)a->cell; m->nbrf[b->cell * MAXNF + b->face] = (int8_t)a->face;
                for (int d = 0; d < 3; ++d) {
                    double s = m->period[d] > 0.0 ? m->period[d] * nearbyint((xa[d] - xb[d]) / m->period[d]) : 0.0;
                    nsh[(a->cell * MAXNF + a->face) * 3 + d] = s;   /* x_b + s lies next to a */
                    nsh[(b->cell * MAXNF + b->face) * 3 + d] = -s;
                }
            } else if (j - i > 2) {
                free(H); free(U); free(nsh); fail("periodic face matched more than once"); or_mesh_free(m); return NULL;
            } else {
                ++nr;
            }
            i = j;
        }
        (void)nr;
    }
    free(H); free(U);

    /* ---- global faces: owner = smaller cell id ---- */
    m->cface = (int64_t*)malloc(nc * MAXNF * sizeof(int64_t));
    int64_t nf = 0;
    for (int64_t c = 0; c < nc; ++c)
        for (int f = 0; f < t_nfaces(type[c]); ++f) {
            int32_t o = m->nbr[c * MAXNF + f];
            if (o < 0 || o > c) ++nf;
            else if (o == c) { free(nsh); fail("cell is its own neighbour (mesh too small for its period)"); or_mesh_free(m); return NULL; }
        }
    m->nface = nf;
    m->fo = (int32_t*)malloc(nf * 4); m->fn = (int32_t*)malloc(nf * 4);
    m->ffo = (int8_t*)malloc(nf); m->ffn = (int8_t*)malloc(nf);
    m->fshift = (double*)calloc(nf * 3, sizeof(double));
    m->fnorm = (double*)calloc(nf * 3, sizeof(double));
    m->farea = (double*)calloc(nf, sizeof(double));
    int64_t g = 0;
    for (int64_t c = 0; c < nc; ++c)
        for (int f = 0; f < t_nfaces(type[c]); ++f) {
            int32_t o = m->nbr[c * MAXNF + f];
            if (o < 0 || o > c) {
                m->fo[g] = (int32_t)c; m->ffo[g] = (int8_t)f;
                m->fn[g] = o; m->ffn[g] = o < 0 ? -1 : m->nbrf[c * MAXNF + f];
                for (int d = 0; d < 3; ++d) m->fshift[3 * g + d] = nsh[(c * MAXNF + f) * 3 + d];
                double A[3];
                face_areavec(m, c, f, A);
                double a = sqrt(A[0] * A[0] + A[1] * A[1] + A[2] * A[2]);
                m->farea[g] = a;
                for (int d = 0; d < 3; ++d) m->fnorm[3 * g + d] = A[d] / a;
                m->cface[c * MAXNF + f] = g;
                if (o >= 0) m->cface[(int64_t)o * MAXNF + m->ffn[g]] = g;
                ++g;
            }
        }
    free(nsh);

    /* ---- geometry ---- */
    m->vol = (double*)malloc(nc * sizeof(double));
    m->cen = (double*)calloc(nc * 3, sizeof(double));
    m->vmean = (double*)calloc(nc * 3, sizeof(double));
    double v[3 * MAXV], px[3 * 512], pw[512];
    for (int64_t c = 0; c < nc; ++c) {
        cell_verts(m, c, v);
        int np = cell_rule(type[c], v, 3, px, pw);
        double V = 0.0, X[3] = {0, 0, 0};
        for (int p = 0; p < np; ++p) {
            V += pw[p];
            for (int d = 0; d < 3; ++d) X[d] += pw[p] * px[3 * p + d];
        }
        m->vol[c] = V;
        for (int d = 0; d < 3; ++d) m->cen[3 * c + d] = X[d] / V;
        int nv = t_nverts(type[c]);
        for (int k = 0; k < nv; ++k)
            for (int d = 0; d < 3; ++d) m->vmean[3 * c + d] += v[3 * k + d];
        for (int d = 0; d < 3; ++d) m->vmean[3 * c + d] /= nv;
    }
    return m;
}

int64_t or_mesh_nfaces(const or_mesh* m) { return m->nface; }

/* connectivity in canonical per-cell form: neighbour across each local face */
void or_mesh_connectivity(const or_mesh* m, int32_t* nbr, int8_t* nbrf)
{
    memcpy(nbr, m->nbr, m->nc * MAXNF * sizeof(int32_t));
    memcpy(nbrf, m->nbrf, m->nc * MAXNF);
}
void or_mesh_geometry(const or_mesh* m, double* vol, double* cen)
{
    memcpy(vol, m->vol, m->nc * sizeof(double));
    memcpy(cen, m->cen, m->nc * 3 * sizeof(double));
}
void or_mesh_faces(const or_mesh* m, int32_t* fo, int32_t* fn, double* normal, double* area, double* shift)
{
    memcpy(fo, m->fo, m->nface * 4); memcpy(fn, m->fn, m->nface * 4);
    memcpy(normal, m->fnorm, m->nface * 3 * sizeof(double));
    memcpy(area, m->farea, m->nface * sizeof(double));
    memcpy(shift, m->fshift, m->nface * 3 * sizeof(double));
}
/* integral of x^a y^b z^c over a physical cell (quadrature pin) */
double or_cell_monomial_integral(const or_mesh* m, int64_t c, int a, int b, int cz, int npts)
{
    double v[3 * MAXV], px[3 * 4096], pw[4096];
    cell_verts(m, c, v);
    int np = cell_rule(m->type[c], v, npts, px, pw);
    double s = 0.0;
    for (int p = 0; p < np; ++p) s += pw[p] * pow(px[3 * p], a) * pow(px[3 * p + 1], b) * pow(px[3 * p + 2], cz);
    return s;
}

/* ------------------------------------------------------------------------ */
/* Scheme                                                                     */
/* ------------------------------------------------------------------------ */
typedef struct {
    int order;       /* r + 1 */
    int flux;        /* 0 Rusanov, 1 HLLC, 2 HLL */
    int scheme;      /* 0 hybrid, 1 pure linear, 2 pure CWENOZ, 3 pure MUSCL */
    int nad_vars;    /* bit0 density, bit1 pressure, bit2 the other conserved variables */
    double gamma, alpha_m, beta_m, alpha_w, beta_w, kappa, n_exp, lambda1p, cw_eps, cw_b, harten_theta, harten_eps;
    double stencil_factor;   /* M = stencil_factor * K(r,d) */
    int limiter;             /* MUSCL limiter: 0 Barth-Jespersen, 1 Venkatakrishnan */
    int cweno_vars;          /* CWENOZ in 0 conserved, 1 characteristic variables */
    double venkat_k;         /* Venkatakrishnan threshold eps^2 = (K dx)^3 */
    /* viscous terms (Sec. 2, eq. EulerEquationsDetails): mu0 = 0 gives the
     * Euler equations; Sutherland's law (eq. sutherlandlaw) with reference
     * temperature t0 and Sutherland temperature suth_s (same units), Prandtl
     * number prandtl (eq. HeatConduct), penalty alpha of eq. viscous_jump */
    double mu0, t0, suth_s, prandtl, visc_alpha;
} or_params;

typedef struct {
    int ready;
    int32_t* sten;   /* [M] central stencil cell ids */
    double* sshift;  /* [M][3] shift added to each stencil cell's coordinates */
    double* P;       /* [N][M] a = P (U_m - U_0) */
    double* Phi;     /* [Q][N] basis values at the cell's face points */
    double* OI;      /* [N][N] */
    double* A;       /* [M][N] */
    double* Vr;      /* [M+1] reference volumes, Vr[0] = |V_0'| */
    int32_t* dir;    /* [nf][Md] local indices (0..M-1) of the directional stencils */
    int32_t* nd;     /* [nf] size of each directional stencil (<= Md) */
    double* D;       /* [nf][d][Md] directional a_s = D (U - U_0) */
    double* G;       /* [d][Md] MUSCL gradient coefficients over the first Md stencil cells */
} or_ops;

typedef struct {
    or_mesh* m;
    or_params p;
    int r, d, nv, N, M, Md, nq, nfp; /* nfp = points per face */
    int nexp; int ex[128][3];          /* monomial exponents, k = 0..N-1 */
    or_ops* ops;                       /* [nc] lazily built */
    double* fqx;                       /* [nface][nfp][3] face points, owner frame */
    double* fqw;                       /* [nface][nfp] weight * |S| */
    int64_t nops_built;
} or_scheme;

static int K_of(int r, int d)
{
    int num = 1, den = 1;
    for (int l = 1; l <= d; ++l) { num *= (r + l); den *= l; }
    return num / den;
}

void or_scheme_free(or_scheme* s)
{
    if (!s) return;
    if (s->ops) {
        for (int64_t c = 0; c < s->m->nc; ++c) {
            or_ops* o = &s->ops[c];
            free(o->sten); free(o->sshift); free(o->P); free(o->Phi); free(o->OI); free(o->A);
            free(o->Vr); free(o->dir); free(o->nd); free(o->D); free(o->G);
        }
        free(s->ops);
    }
    free(s->fqx); free(s->fqw);
    free(s);
}

or_scheme* or_scheme_create(or_mesh* m, const or_params* p)
{
    int r = p->order - 1;
    if (r < 1 || r > 6) { fail("order must be 2..7"); return NULL; }
    or_scheme* s = (or_scheme*)calloc(1, sizeof(or_scheme));
    s->m = m; s->p = *p; s->r = r; s->d = m->dim; s->nv = m->dim + 2;
    s->N = K_of(r, s->d) - 1;
    s->M = (int)llround(p->stencil_factor * K_of(r, s->d));
    s->Md = 2 * K_of(1, s->d);
    if (s->M < s->N || s->M < s->Md) { free(s); fail("stencil too small"); return NULL; }
    /* Gauss points per face direction, exact to degree >= r: ceil((r+1)/2) on
     * edges and on the quadrilaterals of all-hexahedron meshes; ceil((r+2)/2)
     * per direction of the collapsed rule on triangles, exact to degree
     * 2 nq - 2, and on every face of a 3D mesh that has any cell other than
     * a hexahedron (all faces then carry nq^2 points) */
    int all_hex = s->d == 3;
    for (int64_t c = 0; all_hex && c < m->nc; ++c) all_hex = m->type[c] == OR_HEX;
    s->nq = s->d == 3 && !all_hex ? (r + 3) / 2 : (r + 2) / 2;
    s->nfp = s->d == 2 ? s->nq : s->nq * s->nq;
    /* monomial exponents by total degree, then descending powers of xi, eta */
    int k = 0;
    for (int deg = 1; deg <= r; ++deg)
        for (int a = deg; a >= 0; --a) {
            if (s->d == 2) { s->ex[k][0] = a; s->ex[k][1] = deg - a; s->ex[k][2] = 0; ++k; }
            else for (int b = deg - a; b >= 0; --b) { s->ex[k][0] = a; s->ex[k][1] = b; s->ex[k][2] = deg - a - b; ++k; }
        }
    s->nexp = k;
    if (k != s->N) { free(s); fail("internal: basis size"); return NULL; }
    s->ops = (or_ops*)calloc(m->nc, sizeof(or_ops));
    /* face quadrature points (owner frame) and weights */
    double gx[16], gw[16];
    or_gauss_legendre(s->nq, gx, gw);
    s->fqx = (double*)malloc(m->nface * s->nfp * 3 * sizeof(double));
    s->fqw = (double*)malloc(m->nface * s->nfp * sizeof(double));
    for (int64_t g = 0; g < m->nface; ++g) {
        int64_t c = m->fo[g];
        int t = m->type[c], f = m->ffo[g];
        double P[4][3];
        for (int kk = 0; kk < t_fnv(t, f); ++kk)
            for (int dd = 0; dd < 3; ++dd) P[kk][dd] = m->xyz[3 * (int64_t)m->cidx[m->cptr[c] + t_fv(t, f, kk)] + dd];
        if (s->d == 2) {
            for (int a = 0; a < s->nq; ++a) {
                for (int dd = 0; dd < 3; ++dd) s->fqx[(g * s->nfp + a) * 3 + dd] = P[0][dd] + gx[a] * (P[1][dd] - P[0][dd]);
                s->fqw[g * s->nfp + a] = gw[a] * m->farea[g];
            }
        } else if (t_fnv(t, f) == 3) {
            /* collapsed rule on the face triangle P0 P1 P2: x = P0 + u (P1-P0)
             * + u v (P2-P1), weight w_i w_j 2 u |S| (the map's Jacobian is
             * 2 |S| u) */
            for (int j = 0; j < s->nq; ++j)
                for (int i = 0; i < s->nq; ++i) {
                    double u = gx[i], v = gx[j];
                    int a = i + s->nq * j;
                    for (int dd = 0; dd < 3; ++dd)
                        s->fqx[(g * s->nfp + a) * 3 + dd] = P[0][dd] + u * (P[1][dd] - P[0][dd]) + u * v * (P[2][dd] - P[1][dd]);
                    s->fqw[g * s->nfp + a] = gw[i] * gw[j] * 2.0 * u * m->farea[g];
                }
        } else {
            for (int j = 0; j < s->nq; ++j)
                for (int i = 0; i < s->nq; ++i) {
                    double u = gx[i], v = gx[j];
                    int a = i + s->nq * j;
                    for (int dd = 0; dd < 3; ++dd)
                        s->fqx[(g * s->nfp + a) * 3 + dd] = (1 - u) * (1 - v) * P[0][dd] + u * (1 - v) * P[1][dd]
                                                          + u * v * P[2][dd] + (1 - u) * v * P[3][dd];
                    s->fqw[g * s->nfp + a] = gw[i] * gw[j] * m->farea[g];
                }
        }
    }
    return s;
}

/* ---- stencil: face-adjacency layers, whole layers while they fit, the rest
 * of the first layer that does not fit by ascending (distance key, id).
 * Stencil order: (layer, key, id).  The paper only says that neighbouring
 * elements are included recursively (Sec. 2.1); this is the reading taken. */
typedef struct { int64_t q; int32_t id; int layer; double sh[3]; } cand;
static int cand_cmp(const void* a, const void* b)
{
    const cand* x = (const cand*)a; const cand* y = (const cand*)b;
    if (x->layer != y->layer) return x->layer - y->layer;
    if (x->q != y->q) return x->q < y->q ? -1 : 1;
    return x->id < y->id ? -1 : x->id > y->id;
}

static double hsq(const or_scheme* s, int64_t i)
{
    double V = s->m->vol[i];
    if (s->d == 2) return V;
    double h = cbrt(V);
    return h * h;
}

static int build_stencil(or_scheme* s, int64_t i, int32_t* out, double* oshift)
{
    const or_mesh* m = s->m;
    int M = s->M;
    int cap = 4096;
    cand* all = (cand*)malloc(cap * sizeof(cand));
    int nall = 0;
    all[nall].id = (int32_t)i; all[nall].layer = 0; all[nall].q = 0;
    all[nall].sh[0] = all[nall].sh[1] = all[nall].sh[2] = 0.0; ++nall;
    int lay_begin = 0, lay_end = 1, taken = 0, ntake = 0;
    cand* take = (cand*)malloc((M + 1) * sizeof(cand));
    double h2 = hsq(s, i);
    for (int L = 1; L <= 16 && taken < M; ++L) {
        int newbegin = nall;
        for (int a = lay_begin; a < lay_end; ++a) {
            int64_t c = all[a].id;
            for (int f = 0; f < t_nfaces(m->type[c]); ++f) {
                int32_t j = m->nbr[c * MAXNF + f];
                if (j < 0) continue;
                int seen = 0;
                for (int b = 0; b < nall; ++b) if (all[b].id == j) { seen = 1; break; }
                if (seen) continue;
                if (nall == cap) { cap *= 2; all = (cand*)realloc(all, cap * sizeof(cand)); }
                cand* e = &all[nall++];
                e->id = j; e->layer = L;
                double dist2 = 0.0;
                /* the shift of the neighbour accumulates the shift of the face crossed */
                int64_t g = m->cface[c * MAXNF + f];
                double fs[3];
                for (int d = 0; d < 3; ++d) fs[d] = (m->fo[g] == c) ? m->fshift[3 * g + d] : -m->fshift[3 * g + d];
                /* if c owns face g, the neighbour n satisfies x_n + fshift = x_c-frame */
                for (int d = 0; d < 3; ++d) e->sh[d] = all[a].sh[d] + fs[d];
                for (int d = 0; d < 3; ++d) {
                    double dx = m->vmean[3 * (int64_t)j + d] + e->sh[d] - m->vmean[3 * i + d];
                    dist2 += dx * dx;
                }
                e->q = llround(dist2 / h2 * 1048576.0);
            }
        }
        int nl = nall - newbegin;
        if (nl == 0) break;
        qsort(all + newbegin, nl, sizeof(cand), cand_cmp);
        int room = M - taken;
        int tk = nl <= room ? nl : room;
        for (int a = 0; a < tk; ++a) take[ntake++] = all[newbegin + a];
        taken += tk;
        lay_begin = newbegin; lay_end = nall;
    }
    int ok = taken == M;
    if (ok) {
        qsort(take, ntake, sizeof(cand), cand_cmp);
        for (int a = 0; a < M; ++a) {
            out[a] = take[a].id;
            for (int d = 0; d < 3; ++d) oshift[3 * a + d] = take[a].sh[d];
        }
    }
    free(all); free(take);
    return ok ? 0 : fail("stencil: fewer than M cells within sixteen face layers");
}

/* Householder QR least squares: X = A^+ (N x M) for A (M x N), M >= N. */
static int pinv_qr(const double* A, int M, int N, double* X)
{
    double* R = (double*)malloc(M * N * sizeof(double));
    double* Qt = (double*)calloc(M * M, sizeof(double));
    memcpy(R, A, M * N * sizeof(double));
    for (int i = 0; i < M; ++i) Qt[i * M + i] = 1.0;
    double* v = (double*)malloc(M * sizeof(double));
    double rmax = 0.0;
    for (int k = 0; k < N; ++k) {
        double nrm = 0.0;
        for (int i = k; i < M; ++i) nrm += R[i * N + k] * R[i * N + k];
        nrm = sqrt(nrm);
        if (nrm == 0.0) { free(R); free(Qt); free(v); return -1; }
        double alpha = R[k * N + k] > 0 ? -nrm : nrm;
        for (int i = 0; i < M; ++i) v[i] = 0.0;
        v[k] = R[k * N + k] - alpha;
        for (int i = k + 1; i < M; ++i) v[i] = R[i * N + k];
        double vv = 0.0;
        for (int i = k; i < M; ++i) vv += v[i] * v[i];
        if (vv > 0.0) {
            for (int j = 0; j < N; ++j) {              /* R <- (I - 2 v v^T / v^T v) R */
                double sdot = 0.0;
                for (int i = k; i < M; ++i) sdot += v[i] * R[i * N + j];
                sdot *= 2.0 / vv;
                for (int i = k; i < M; ++i) R[i * N + j] -= sdot * v[i];
            }
            for (int j = 0; j < M; ++j) {              /* Qt <- H Qt */
                double sdot = 0.0;
                for (int i = k; i < M; ++i) sdot += v[i] * Qt[i * M + j];
                sdot *= 2.0 / vv;
                for (int i = k; i < M; ++i) Qt[i * M + j] -= sdot * v[i];
            }
        }
        if (fabs(R[k * N + k]) > rmax) rmax = fabs(R[k * N + k]);
    }
    for (int k = 0; k < N; ++k)
        if (fabs(R[k * N + k]) <= 1e-12 * rmax) { free(R); free(Qt); free(v); return -1; }
    /* back substitution: R[0:N,0:N] X = Qt[0:N, :] */
    for (int j = 0; j < M; ++j)
        for (int k = N - 1; k >= 0; --k) {
            double sum = Qt[k * M + j];
            for (int l = k + 1; l < N; ++l) sum -= R[k * N + l] * X[l * M + j];
            X[k * M + j] = sum / R[k * N + k];
        }
    free(R); free(Qt); free(v);
    return 0;
}

static double ipow(double x, int e) { double r = 1.0; for (int i = 0; i < e; ++i) r *= x; return r; }

/* reference map of cell i: xi = Jinv (x - v0), from its corner simplex
 * (triangle v0 v1 v2; quadrilateral v0 v1 v3; tetrahedron and prism
 * v0 v1 v2 v3; hexahedron and pyramid v0 v1 v3 v4),
 * the reading taken for the paper's transformation (Sec. 2.1) */
static void ref_map(const or_scheme* s, int64_t i, double* x0, double Jinv[3][3], double* detJ)
{
    const or_mesh* m = s->m;
    double v[3 * MAXV];
    cell_verts(m, i, v);
    int t = m->type[i];
    int simplex_first = t == OR_TRI || t == OR_TET || t == OR_PRISM;
    int c1 = 1, c2 = simplex_first ? 2 : 3, c3 = (t == OR_TET || t == OR_PRISM) ? 3 : 4;
    double J[3][3] = {{0}};
    for (int d = 0; d < 3; ++d) {
        x0[d] = v[d];
        J[d][0] = v[3 * c1 + d] - v[d];
        J[d][1] = v[3 * c2 + d] - v[d];
        J[d][2] = (s->d == 3) ? v[3 * c3 + d] - v[d] : (d == 2 ? 1.0 : 0.0);
    }
    double det = J[0][0] * (J[1][1] * J[2][2] - J[1][2] * J[2][1]) - J[0][1] * (J[1][0] * J[2][2] - J[1][2] * J[2][0])
               + J[0][2] * (J[1][0] * J[2][1] - J[1][1] * J[2][0]);
    Jinv[0][0] = (J[1][1] * J[2][2] - J[1][2] * J[2][1]) / det;
    Jinv[0][1] = (J[0][2] * J[2][1] - J[0][1] * J[2][2]) / det;
    Jinv[0][2] = (J[0][1] * J[1][2] - J[0][2] * J[1][1]) / det;
    Jinv[1][0] = (J[1][2] * J[2][0] - J[1][0] * J[2][2]) / det;
    Jinv[1][1] = (J[0][0] * J[2][2] - J[0][2] * J[2][0]) / det;
    Jinv[1][2] = (J[0][2] * J[1][0] - J[0][0] * J[1][2]) / det;
    Jinv[2][0] = (J[1][0] * J[2][1] - J[1][1] * J[2][0]) / det;
    Jinv[2][1] = (J[0][1] * J[2][0] - J[0][0] * J[2][1]) / det;
    Jinv[2][2] = (J[0][0] * J[1][1] - J[0][1] * J[1][0]) / det;
    *detJ = fabs(det);
}
static void to_ref(const double* x0, double Jinv[3][3], const double* x, double* xi)
{
    double dx[3] = {x[0] - x0[0], x[1] - x0[1], x[2] - x0[2]};
    for (int a = 0; a < 3; ++a) xi[a] = Jinv[a][0] * dx[0] + Jinv[a][1] * dx[1] + Jinv[a][2] * dx[2];
}
static double mono(const or_scheme* s, int k, const double* xi)
{
    return ipow(xi[0], s->ex[k][0]) * ipow(xi[1], s->ex[k][1]) * ipow(xi[2], s->ex[k][2]);
}

/* integrals of psi_k over the (shifted) cell c mapped to the reference space */
static double ref_integrals(const or_scheme* s, int64_t c, const double* shift, const double* x0, double Jinv[3][3],
                            double* out /* [N] */)
{
    double v[3 * MAXV], vr[3 * MAXV], px[3 * 1024], pw[1024];
    cell_verts(s->m, c, v);
    int nvtx = t_nverts(s->m->type[c]);
    for (int k = 0; k < nvtx; ++k) {
        double x[3] = {v[3 * k] + shift[0], v[3 * k + 1] + shift[1], v[3 * k + 2] + shift[2]};
        to_ref(x0, Jinv, x, &vr[3 * k]);
        if (s->d == 2) vr[3 * k + 2] = 0.0;
    }
    int np = cell_rule(s->m->type[c], vr, s->r + 2, px, pw);
    double vol = 0.0;
    for (int k = 0; k < s->N; ++k) out[k] = 0.0;
    for (int p = 0; p < np; ++p) {
        vol += pw[p];
        for (int k = 0; k < s->N; ++k) out[k] += pw[p] * mono(s, k, &px[3 * p]);
    }
    return vol;
}

/* local-face outward normal and point list of cell i in its own frame */
static void cell_face_points(const or_scheme* s, int64_t i, int f, double* pts /* [nfp][3] */, double* nrm)
{
    const or_mesh* m = s->m;
    int64_t g = m->cface[i * MAXNF + f];
    int own = m->fo[g] == i && m->ffo[g] == f;
    for (int a = 0; a < s->nfp; ++a)
        for (int d = 0; d < 3; ++d)
            pts[3 * a + d] = s->fqx[(g * s->nfp + a) * 3 + d] - (own ? 0.0 : m->fshift[3 * g + d]);
    for (int d = 0; d < 3; ++d) nrm[d] = own ? m->fnorm[3 * g + d] : -m->fnorm[3 * g + d];
}

static or_ops* get_ops(or_scheme* s, int64_t i)
{
    or_ops* o = &s->ops[i];
    if (o->ready) return o;
    const or_mesh* m = s->m;
    int M = s->M, N = s->N, d = s->d, Md = s->Md;
    int nf = t_nfaces(m->type[i]), Q = nf * s->nfp;
    o->sten = (int32_t*)malloc(M * sizeof(int32_t));
    o->sshift = (double*)malloc(M * 3 * sizeof(double));
    if (build_stencil(s, i, o->sten, o->sshift) != 0) return NULL;
    double x0[3], Jinv[3][3], detJ;
    ref_map(s, i, x0, Jinv, &detJ);
    /* cell 0: reference volume and means of the monomials */
    double mean0[128], zero[3] = {0, 0, 0};
    o->Vr = (double*)malloc((M + 1) * sizeof(double));
    o->Vr[0] = ref_integrals(s, i, zero, x0, Jinv, mean0);
    for (int k = 0; k < N; ++k) mean0[k] /= o->Vr[0];
    /* A_mk = int_{V_m'} phi_k = int psi_k - |V_m'| mean0_k */
    o->A = (double*)malloc(M * N * sizeof(double));
    double I[128];
    for (int a = 0; a < M; ++a) {
        double vm = ref_integrals(s, o->sten[a], &o->sshift[3 * a], x0, Jinv, I);
        o->Vr[a + 1] = vm;
        for (int k = 0; k < N; ++k) o->A[a * N + k] = I[k] - vm * mean0[k];
    }
    /* pseudo-inverse and b_m = |V_m'| (U_m - U_0) folded in: P = A^+ diag(|V_m'|) */
    o->P = (double*)malloc(N * M * sizeof(double));
    if (pinv_qr(o->A, M, N, o->P) != 0) { fail("rank-deficient central stencil"); return NULL; }
    for (int k = 0; k < N; ++k)
        for (int a = 0; a < M; ++a) o->P[k * M + a] *= o->Vr[a + 1];
    /* basis at the face points */
    o->Phi = (double*)malloc(Q * N * sizeof(double));
    double pts[3 * 64], nrm[3], xi[3];
    double fnrm[MAXNF][3];
    for (int f = 0; f < nf; ++f) {
        cell_face_points(s, i, f, pts, nrm);
        for (int a = 0; a < s->nfp; ++a) {
            to_ref(x0, Jinv, &pts[3 * a], xi);
            if (d == 2) xi[2] = 0.0;
            for (int k = 0; k < N; ++k) o->Phi[(f * s->nfp + a) * N + k] = mono(s, k, xi) - mean0[k];
        }
        for (int dd = 0; dd < 3; ++dd) fnrm[f][dd] = nrm[dd];
    }
    /* oscillation-indicator matrix over cell 0 in reference space, h_c = 1 */
    o->OI = (double*)calloc(N * N, sizeof(double));
    {
        double v[3 * MAXV], vr[3 * MAXV], px[3 * 1024], pw[1024];
        cell_verts(m, i, v);
        for (int k = 0; k < t_nverts(m->type[i]); ++k) { to_ref(x0, Jinv, &v[3 * k], &vr[3 * k]); if (d == 2) vr[3 * k + 2] = 0.0; }
        int np = cell_rule(m->type[i], vr, s->r + 2, px, pw);
        /* every multi-index beta with 1 <= |beta| <= r, each counted once */
        for (int b0 = 0; b0 <= s->r; ++b0)
            for (int b1 = 0; b0 + b1 <= s->r; ++b1)
                for (int b2 = 0; b0 + b1 + b2 <= s->r; ++b2) {
                    if (d == 2 && b2 > 0) continue;
                    if (b0 + b1 + b2 == 0) continue;
                    int be[3] = {b0, b1, b2};
                    for (int p = 0; p < np; ++p) {
                        double D[128];
                        for (int k = 0; k < N; ++k) {
                            double val = 1.0;
                            for (int a = 0; a < 3; ++a) {
                                int e = s->ex[k][a];
                                if (e < be[a]) { val = 0.0; break; }
                                double cf = 1.0;
                                for (int q = 0; q < be[a]; ++q) cf *= (e - q);
                                val *= cf * ipow(px[3 * p + a], e - be[a]);
                            }
                            D[k] = val;
                        }
                        for (int k = 0; k < N; ++k)
                            for (int l = 0; l < N; ++l) o->OI[k * N + l] += pw[p] * D[k] * D[l];
                    }
                }
    }
    /* directional stencils: one per face.  Candidates are the central-stencil
     * cells lying in the half-space beyond the cell's vertex mean along the
     * face's outward normal (signed distance quantised to h / 2^20, > 0), in
     * stencil order, at most Md of them.  With at least d+1 candidates they
     * form the stencil (its size nd_f may be below Md); with fewer (a face on
     * or near the domain boundary) the stencil is the first Md cells of the
     * central stencil.  The paper only requires lower-order stencils
     * contained in the central one (Sec. 2.3); this is the reading taken. */
    o->dir = (int32_t*)malloc(nf * Md * sizeof(int32_t));
    o->nd = (int32_t*)malloc(nf * sizeof(int32_t));
    o->D = (double*)calloc(nf * d * Md, sizeof(double));
    double h = d == 2 ? sqrt(m->vol[i]) : cbrt(m->vol[i]);
    double* Ad = (double*)malloc(Md * d * sizeof(double));
    double* Xd = (double*)malloc(d * Md * sizeof(double));
    for (int f = 0; f < nf; ++f) {
        int cnt = 0;
        for (int a = 0; a < M && cnt < Md; ++a) {
            int32_t j = o->sten[a];
            double sd = 0.0;
            for (int dd = 0; dd < 3; ++dd)
                sd += (m->vmean[3 * (int64_t)j + dd] + o->sshift[3 * a + dd] - m->vmean[3 * i + dd]) * fnrm[f][dd];
            if (llround(sd / h * 1048576.0) > 0) o->dir[f * Md + cnt++] = a;
        }
        if (cnt < d + 1) {
            cnt = Md;
            for (int a = 0; a < Md; ++a) o->dir[f * Md + a] = a;
        }
        o->nd[f] = cnt;
        for (int b = cnt; b < Md; ++b) o->dir[f * Md + b] = 0;   /* padding, zero coefficients */
        for (int b = 0; b < cnt; ++b)
            for (int k = 0; k < d; ++k) Ad[b * d + k] = o->A[o->dir[f * Md + b] * N + k];
        if (pinv_qr(Ad, cnt, d, Xd) != 0) { fail("rank-deficient directional stencil"); free(Ad); free(Xd); return NULL; }
        for (int k = 0; k < d; ++k)
            for (int b = 0; b < cnt; ++b) o->D[(f * d + k) * Md + b] = Xd[k * cnt + b] * o->Vr[o->dir[f * Md + b] + 1];
    }
    /* MUSCL gradient: degree-1 least squares on the first Md stencil cells */
    o->G = (double*)malloc(d * Md * sizeof(double));
    for (int b = 0; b < Md; ++b)
        for (int k = 0; k < d; ++k) Ad[b * d + k] = o->A[b * N + k];
    if (pinv_qr(Ad, Md, d, Xd) != 0) { fail("rank-deficient MUSCL stencil"); free(Ad); free(Xd); return NULL; }
    for (int k = 0; k < d; ++k)
        for (int b = 0; b < Md; ++b) o->G[k * Md + b] = Xd[k * Md + b] * o->Vr[b + 1];
    free(Ad); free(Xd);
    o->ready = 1;
    s->nops_built++;
    return o;
}

/* ------------------------------------------------------------------------ */
/* physics (Sec. 2: perfect gas, gamma = 1.4)                                 */
/* ------------------------------------------------------------------------ */
static double pres(const double* U, int d, double g)
{
    double ke = 0.0;
    for (int k = 0; k < d; ++k) ke += U[1 + k] * U[1 + k];
    return (g - 1.0) * (U[d + 1] - 0.5 * ke / U[0]);
}
static void phys_flux(const double* U, const double* n, int d, double g, double* F)
{
    double rho = U[0], un = 0.0;
    for (int k = 0; k < d; ++k) un += U[1 + k] / rho * n[k];
    double p = pres(U, d, g);
    F[0] = rho * un;
    for (int k = 0; k < d; ++k) F[1 + k] = U[1 + k] * un + p * n[k];
    F[d + 1] = (U[d + 1] + p) * un;
}

void or_flux(int kind, int d, double g, const double* UL, const double* UR, const double* n, double* F)
{
    int nv = d + 2;
    double FL[5], FR[5];
    phys_flux(UL, n, d, g, FL);
    phys_flux(UR, n, d, g, FR);
    double rl = UL[0], rr = UR[0], unl = 0, unr = 0;
    for (int k = 0; k < d; ++k) { unl += UL[1 + k] / rl * n[k]; unr += UR[1 + k] / rr * n[k]; }
    double pl = pres(UL, d, g), pr = pres(UR, d, g);
    double cl = sqrt(g * pl / rl), cr = sqrt(g * pr / rr);
    if (kind == 0) { /* Rusanov (local Lax-Friedrichs) */
        double sl = fabs(unl) + cl, sr = fabs(unr) + cr, smax = sl > sr ? sl : sr;
        for (int v = 0; v < nv; ++v) F[v] = 0.5 * (FL[v] + FR[v]) - 0.5 * smax * (UR[v] - UL[v]);
        return;
    }
    /* Davis wave-speed estimates */
    double SL = fmin(unl - cl, unr - cr), SR = fmax(unl + cl, unr + cr);
    if (SL >= 0.0) { for (int v = 0; v < nv; ++v) F[v] = FL[v]; return; }
    if (SR <= 0.0) { for (int v = 0; v < nv; ++v) F[v] = FR[v]; return; }
    if (kind == 2) { /* HLL */
        for (int v = 0; v < nv; ++v) F[v] = (SR * FL[v] - SL * FR[v] + SL * SR * (UR[v] - UL[v])) / (SR - SL);
        return;
    }
    /* HLLC (Toro): contact speed and star states */
    double Ss = (pr - pl + rl * unl * (SL - unl) - rr * unr * (SR - unr)) / (rl * (SL - unl) - rr * (SR - unr));
    const double* UK = Ss >= 0.0 ? UL : UR;
    const double* FK = Ss >= 0.0 ? FL : FR;
    double SK = Ss >= 0.0 ? SL : SR, rk = UK[0], unk = Ss >= 0.0 ? unl : unr, pk = Ss >= 0.0 ? pl : pr;
    double fac = rk * (SK - unk) / (SK - Ss);
    double Us[5];
    Us[0] = fac;
    for (int k = 0; k < d; ++k) Us[1 + k] = fac * (UK[1 + k] / rk + (Ss - unk) * n[k]);
    Us[d + 1] = fac * (UK[d + 1] / rk + (Ss - unk) * (Ss + pk / (rk * (SK - unk))));
    for (int v = 0; v < nv; ++v) F[v] = FK[v] + SK * (Us[v] - UK[v]);
}

/* ------------------------------------------------------------------------ */
/* reconstruction steps                                                       */
/* ------------------------------------------------------------------------ */
static int n_faces_of(const or_scheme* s, int64_t c) { return t_nfaces(s->m->type[c]); }
static int Q_of(const or_scheme* s, int64_t c) { return n_faces_of(s, c) * s->nfp; }

static void get_state(const or_scheme* s, const double* U, int64_t c, double* u)
{
    for (int v = 0; v < s->nv; ++v) u[v] = U[(int64_t)v * s->m->nc + c];
}

/* linear candidate (Sec. 2.1): a = P (U_m - U_0), values U_0 + Phi a */
static void rec_linear(or_scheme* s, or_ops* o, const double* U, int64_t i, double* a /*[nv][N]*/, double* V /*[Q][nv]*/)
{
    int N = s->N, M = s->M, nv = s->nv, Q = Q_of(s, i);
    double u0[5];
    get_state(s, U, i, u0);
    for (int v = 0; v < nv; ++v)
        for (int k = 0; k < N; ++k) {
            double sum = 0.0;
            for (int mm = 0; mm < M; ++mm) sum += o->P[k * M + mm] * (U[(int64_t)v * s->m->nc + o->sten[mm]] - u0[v]);
            a[v * N + k] = sum;
        }
    for (int q = 0; q < Q; ++q)
        for (int v = 0; v < nv; ++v) {
            double sum = u0[v];
            for (int k = 0; k < N; ++k) sum += o->Phi[q * N + k] * a[v * N + k];
            V[q * nv + v] = sum;
        }
}

/* d/dxi_a of monomial k at xi */
static double dmono(const or_scheme* s, int k, int a, const double* xi)
{
    int e = s->ex[k][a];
    if (e == 0) return 0.0;
    double r = e * ipow(xi[a], e - 1);
    for (int b = 0; b < 3; ++b)
        if (b != a) r *= ipow(xi[b], s->ex[k][b]);
    return r;
}

/* Viscous gradients (Sec. 2, gradients for the viscous fluxes from the
 * constrained least-squares reconstruction): at every face point of cell i,
 * the gradient in physical coordinates of the unlimited degree-r polynomial
 * of each conserved variable (grad p = sum_k a_k J^-T grad_xi phi_k), turned
 * into the gradients of the velocity components and of T = p / rho by the
 * chain rule at the cell's face-point state W (the state U_L that also enters
 * the convective flux, eq. EulerEquationsDetails).
 * PG[q][k][j]: k < d velocity component k, k = d temperature; j = x, y, z. */
static void rec_visc_grad(or_scheme* s, or_ops* o, const double* U, int64_t i, const double* Wf, double* PG)
{
    int N = s->N, nv = s->nv, d = s->d, nfp = s->nfp, nf = n_faces_of(s, i);
    double a[5 * 128], V[5 * 64], x0[3], Ji[3][3], det, pts[3 * 64], nrm[3];
    double g = s->p.gamma;
    rec_linear(s, o, U, i, a, V);
    ref_map(s, i, x0, Ji, &det);
    for (int f = 0; f < nf; ++f) {
        cell_face_points(s, i, f, pts, nrm);
        for (int al = 0; al < nfp; ++al) {
            int q = f * nfp + al;
            double xi[3], gc[5][3];
            to_ref(x0, Ji, &pts[3 * al], xi);
            if (d == 2) xi[2] = 0.0;
            for (int v = 0; v < nv; ++v)
                for (int j = 0; j < 3; ++j) {
                    double sum = 0.0;
                    if (j < d)
                        for (int k = 0; k < N; ++k) {
                            double dk = 0.0;
                            for (int b = 0; b < d; ++b) dk += Ji[b][j] * dmono(s, k, b, xi);
                            sum += a[v * N + k] * dk;
                        }
                    gc[v][j] = sum;
                }
            const double* w = &Wf[q * nv];
            double rho = w[0], u[3] = {0, 0, 0}, u2 = 0.0;
            for (int k = 0; k < d; ++k) { u[k] = w[1 + k] / rho; u2 += u[k] * u[k]; }
            double p = (g - 1.0) * (w[d + 1] - 0.5 * rho * u2), T = p / rho;
            double* out = &PG[(size_t)q * 4 * 3];
            for (int j = 0; j < 3; ++j) {
                /* grad u_k = (grad m_k - u_k grad rho) / rho */
                for (int k = 0; k < d; ++k) out[k * 3 + j] = (gc[1 + k][j] - u[k] * gc[0][j]) / rho;
                /* grad p = (g - 1)(grad E - sum_k u_k grad m_k + |u|^2 / 2 grad rho);
                 * grad T = (grad p - T grad rho) / rho */
                double gp = gc[d + 1][j] + 0.5 * u2 * gc[0][j];
                for (int k = 0; k < d; ++k) gp -= u[k] * gc[1 + k][j];
                gp *= (g - 1.0);
                out[d * 3 + j] = (gp - T * gc[0][j]) / rho;
            }
        }
    }
}

/* Viscous flux F_v . n at one face point (Sec. 2, eqs. Terms1, Stresses,
 * HeatConduct, sutherlandlaw, viscous_jump): face state = mean of the two
 * sides' primitive velocity and temperature; gradients = mean of the two
 * sides' gradients plus the penalty (alpha / L_int)(W_R - W_L) n;
 * tau_ij = mu (d_j u_i + d_i u_j - 2/3 div u delta_ij);
 * Theta_j = sum_i u_i tau_ij + mu / Pr gamma / (gamma - 1) dT/dx_j. */
static void visc_flux(const or_scheme* s, const double* WL, const double* WR, const double* GL, const double* GR,
                      const double* n, double inv_lint, double* F)
{
    int d = s->d;
    double g = s->p.gamma, pl[4], pr[4];   /* u_0..u_{d-1}, T */
    for (int side = 0; side < 2; ++side) {
        const double* w = side ? WR : WL;
        double* q = side ? pr : pl;
        double u2 = 0.0;
        for (int k = 0; k < d; ++k) { q[k] = w[1 + k] / w[0]; u2 += q[k] * q[k]; }
        q[d] = (g - 1.0) * (w[d + 1] - 0.5 * w[0] * u2) / w[0];
    }
    double um[3] = {0, 0, 0}, Tm = 0.5 * (pl[d] + pr[d]), G[4][3];
    for (int k = 0; k < d; ++k) um[k] = 0.5 * (pl[k] + pr[k]);
    for (int k = 0; k <= d; ++k)
        for (int j = 0; j < d; ++j)
            G[k][j] = 0.5 * (GL[k * 3 + j] + GR[k * 3 + j]) + s->p.visc_alpha * inv_lint * (pr[k] - pl[k]) * n[j];
    double T0 = s->p.t0, S = s->p.suth_s;
    double mu = s->p.mu0 * pow(Tm / T0, 1.5) * (T0 + S) / (Tm + S);
    double div = 0.0;
    for (int k = 0; k < d; ++k) div += G[k][k];
    double tau[3][3];
    for (int i = 0; i < d; ++i)
        for (int j = 0; j < d; ++j) tau[i][j] = mu * (G[i][j] + G[j][i] - (i == j ? 2.0 / 3.0 * div : 0.0));
    double kap = mu / s->p.prandtl * g / (g - 1.0);
    F[0] = 0.0;
    F[d + 1] = 0.0;
    for (int i = 0; i < d; ++i) {
        double t = 0.0;
        for (int j = 0; j < d; ++j) t += tau[i][j] * n[j];
        F[1 + i] = t;
    }
    for (int j = 0; j < d; ++j) {
        double th = kap * G[d][j];
        for (int i = 0; i < d; ++i) th += um[i] * tau[i][j];
        F[d + 1] += th * n[j];
    }
}

/* directional degree-1 coefficients a_s for stencil f */
static void dir_coeffs(const or_scheme* s, const or_ops* o, const double* U, int64_t i, int f, int v, double* as)
{
    int d = s->d, Md = s->Md;
    double u0 = U[(int64_t)v * s->m->nc + i];
    for (int k = 0; k < d; ++k) {
        double sum = 0.0;
        for (int b = 0; b < Md; ++b) sum += o->D[(f * d + k) * Md + b] * (U[(int64_t)v * s->m->nc + o->sten[o->dir[f * Md + b]]] - u0);
        as[k] = sum;
    }
}

/* CWENOZ (Sec. 2.3) for variable v; also returns the weights and indicators */
/* CWENOZ weights and polynomial (Sec. 2.3) of one variable from its p_opt
 * coefficients aopt [N] and directional coefficients as [nf][d] */
static void cweno_combine(or_scheme* s, or_ops* o, int64_t i, const double* aopt, double as[MAXNF][3],
                          double* acw /*[N]*/, double* omega, double* SI);

static void rec_cweno_var(or_scheme* s, or_ops* o, const double* U, int64_t i, int v, const double* aopt,
                          double* acw /*[N]*/, double* omega, double* SI)
{
    int nf = n_faces_of(s, i);
    double as[MAXNF][3];
    for (int f = 0; f < nf; ++f) dir_coeffs(s, o, U, i, f, v, as[f]);
    cweno_combine(s, o, i, aopt, as, acw, omega, SI);
}

static void cweno_combine(or_scheme* s, or_ops* o, int64_t i, const double* aopt, double as[MAXNF][3],
                          double* acw /*[N]*/, double* omega, double* SI)
{
    int N = s->N, d = s->d, nf = n_faces_of(s, i), st = nf + 1;
    double lam1 = 1.0 - 1.0 / s->p.lambda1p, lams = (1.0 - lam1) / (st - 1);
    /* p_1 = (p_opt - sum_s lambda_s p_s) / lambda_1 */
    double a1[128];
    for (int k = 0; k < N; ++k) {
        double sub = 0.0;
        if (k < d) for (int f = 0; f < nf; ++f) sub += lams * as[f][k];
        a1[k] = (aopt[k] - sub) / lam1;
    }
    /* smoothness indicators SI_s = a^T OI a */
    SI[0] = 0.0;
    for (int k = 0; k < N; ++k)
        for (int l = 0; l < N; ++l) SI[0] += a1[k] * o->OI[k * N + l] * a1[l];
    for (int f = 0; f < nf; ++f) {
        double sum = 0.0;
        for (int k = 0; k < d; ++k)
            for (int l = 0; l < d; ++l) sum += as[f][k] * o->OI[k * N + l] * as[f][l];
        SI[1 + f] = sum;
    }
    /* universal oscillation indicator and CWENOZ weights, as printed */
    double tsum = 0.0;
    for (int f = 0; f < nf; ++f) tsum += fabs(SI[1 + f] - SI[0]);
    double tau = pow(tsum / (st - 1), s->p.cw_b);
    double wt[MAXNF + 1], wsum = 0.0;
    for (int q = 0; q < st; ++q) {
        double lam = q == 0 ? lam1 : lams;
        wt[q] = lam * (1.0 + tau / (s->p.cw_eps + SI[q]));
        wsum += wt[q];
    }
    for (int q = 0; q < st; ++q) omega[q] = wt[q] / wsum;
    for (int k = 0; k < N; ++k) {
        double sum = omega[0] * a1[k];
        if (k < d) for (int f = 0; f < nf; ++f) sum += omega[1 + f] * as[f][k];
        acw[k] = sum;
    }
}

/* Eigenvectors of the Euler flux Jacobian dF.n/dU at the state u (conserved
 * variables, unit normal n): columns of R (right) and rows of L = R^-1
 * (left), ordered acoustic (u.n - c), entropy, shear (one in 2D, two in 3D
 * along t1, t2), acoustic (u.n + c).  Tangents: 2D t = (-n_y, n_x); 3D
 * t1 = n x e_a / |n x e_a| with e_a the axis of the smallest |n_a|, t2 =
 * n x t1. */
void or_euler_eigen(int d, double gamma, const double* u, const double* n, double* L, double* R)
{
    const int nv = d + 2;
    double vel[3] = {0, 0, 0}, q2 = 0.0, qn = 0.0;
    for (int k = 0; k < d; ++k) { vel[k] = u[1 + k] / u[0]; q2 += vel[k] * vel[k]; qn += vel[k] * n[k]; }
    const double p = (gamma - 1.0) * (u[d + 1] - 0.5 * u[0] * q2);
    const double c = sqrt(gamma * p / u[0]), H = (u[d + 1] + p) / u[0];
    double t[2][3] = {{0, 0, 0}, {0, 0, 0}};
    int nt = d - 1;
    if (d == 2) { t[0][0] = -n[1]; t[0][1] = n[0]; }
    else {
        int ax = 0;
        for (int k = 1; k < 3; ++k) if (fabs(n[k]) < fabs(n[ax])) ax = k;
        double e[3] = {0, 0, 0};
        e[ax] = 1.0;
        double a[3] = {n[1] * e[2] - n[2] * e[1], n[2] * e[0] - n[0] * e[2], n[0] * e[1] - n[1] * e[0]};
        double an = sqrt(a[0] * a[0] + a[1] * a[1] + a[2] * a[2]);
        for (int k = 0; k < 3; ++k) t[0][k] = a[k] / an;
        t[1][0] = n[1] * t[0][2] - n[2] * t[0][1];
        t[1][1] = n[2] * t[0][0] - n[0] * t[0][2];
        t[1][2] = n[0] * t[0][1] - n[1] * t[0][0];
    }
    for (int k = 0; k < nv * nv; ++k) { L[k] = 0.0; R[k] = 0.0; }
    /* right eigenvectors (column j of R at R[r * nv + j]) */
    R[0 * nv + 0] = 1.0; R[0 * nv + 1] = 1.0; R[0 * nv + nv - 1] = 1.0;
    for (int k = 0; k < d; ++k) {
        R[(1 + k) * nv + 0] = vel[k] - c * n[k];
        R[(1 + k) * nv + 1] = vel[k];
        R[(1 + k) * nv + nv - 1] = vel[k] + c * n[k];
    }
    R[(d + 1) * nv + 0] = H - c * qn;
    R[(d + 1) * nv + 1] = 0.5 * q2;
    R[(d + 1) * nv + nv - 1] = H + c * qn;
    for (int j = 0; j < nt; ++j) {
        double ut = 0.0;
        for (int k = 0; k < d; ++k) { R[(1 + k) * nv + 2 + j] = t[j][k]; ut += vel[k] * t[j][k]; }
        R[(d + 1) * nv + 2 + j] = ut;
    }
    /* left eigenvectors (row i of L at L[i * nv + .]) */
    const double b1 = (gamma - 1.0) / (c * c), b2 = 0.5 * b1 * q2;
    L[0 * nv + 0] = 0.5 * (b2 + qn / c);
    L[(nv - 1) * nv + 0] = 0.5 * (b2 - qn / c);
    L[1 * nv + 0] = 1.0 - b2;
    for (int k = 0; k < d; ++k) {
        L[0 * nv + 1 + k] = 0.5 * (-b1 * vel[k] - n[k] / c);
        L[(nv - 1) * nv + 1 + k] = 0.5 * (-b1 * vel[k] + n[k] / c);
        L[1 * nv + 1 + k] = b1 * vel[k];
    }
    L[0 * nv + d + 1] = 0.5 * b1;
    L[(nv - 1) * nv + d + 1] = 0.5 * b1;
    L[1 * nv + d + 1] = -b1;
    for (int j = 0; j < nt; ++j) {
        double ut = 0.0;
        for (int k = 0; k < d; ++k) { L[(2 + j) * nv + 1 + k] = t[j][k]; ut += vel[k] * t[j][k]; }
        L[(2 + j) * nv + 0] = -ut;
    }
}

/* CWENOZ in characteristic variables: for each face f of the cell, the
 * p_opt and directional coefficients of every conserved variable are
 * projected with the left eigenvectors of the Jacobian along the face's
 * normal at the cell mean, each characteristic variable gets its own
 * weights (Sec. 2.3), and the face's points are projected back with the
 * right eigenvectors */
static void rec_cweno_char(or_scheme* s, or_ops* o, const double* U, int64_t i, const double* a, double* V)
{
    int N = s->N, nv = s->nv, d = s->d, nf = n_faces_of(s, i);
    double u0[5], as[5][MAXNF][3];
    get_state(s, U, i, u0);
    for (int v = 0; v < nv; ++v)
        for (int f = 0; f < nf; ++f) dir_coeffs(s, o, U, i, f, v, as[v][f]);
    for (int f = 0; f < nf; ++f) {
        double pts[3 * 64], nrm[3], L[25], R[25];
        cell_face_points(s, i, f, pts, nrm);
        or_euler_eigen(d, s->p.gamma, u0, nrm, L, R);
        double acw[5][128];
        for (int w = 0; w < nv; ++w) {
            double aw[128], asw[MAXNF][3], om[MAXNF + 1], SI[MAXNF + 1];
            for (int k = 0; k < N; ++k) {
                double sum = 0.0;
                for (int v = 0; v < nv; ++v) sum += L[w * nv + v] * a[v * N + k];
                aw[k] = sum;
            }
            for (int g = 0; g < nf; ++g)
                for (int k = 0; k < d; ++k) {
                    double sum = 0.0;
                    for (int v = 0; v < nv; ++v) sum += L[w * nv + v] * as[v][g][k];
                    asw[g][k] = sum;
                }
            cweno_combine(s, o, i, aw, asw, acw[w], om, SI);
        }
        for (int a0 = 0; a0 < s->nfp; ++a0) {
            const int q = f * s->nfp + a0;
            double cw[5];
            for (int w = 0; w < nv; ++w) {
                double sum = 0.0;
                for (int k = 0; k < N; ++k) sum += o->Phi[q * N + k] * acw[w][k];
                cw[w] = sum;
            }
            for (int v = 0; v < nv; ++v) {
                double sum = u0[v];
                for (int w = 0; w < nv; ++w) sum += R[v * nv + w] * cw[w];
                V[q * nv + v] = sum;
            }
        }
    }
}

static void rec_cweno(or_scheme* s, or_ops* o, const double* U, int64_t i, const double* a, double* V)
{
    int N = s->N, nv = s->nv, Q = Q_of(s, i);
    double u0[5], acw[128], om[MAXNF + 1], SI[MAXNF + 1];
    if (s->p.cweno_vars == 1) { rec_cweno_char(s, o, U, i, a, V); return; }
    get_state(s, U, i, u0);
    for (int v = 0; v < nv; ++v) {
        rec_cweno_var(s, o, U, i, v, &a[v * N], acw, om, SI);
        for (int q = 0; q < Q; ++q) {
            double sum = u0[v];
            for (int k = 0; k < N; ++k) sum += o->Phi[q * N + k] * acw[k];
            V[q * nv + v] = sum;
        }
    }
}

/* Venkatakrishnan's smooth limiter value at one face point: the unlimited
 * increment d2 = grad U . (x_q - x_c), the bound's distance d1 = U_max - U_c
 * (d2 > 0) or U_min - U_c (d2 < 0), eps2 = (K dx)^3:
 *   phi = [(d1^2 + eps2) d2 + 2 d2^2 d1] / (d2 [d1^2 + 2 d2^2 + d1 d2 + eps2]),
 * capped at 1; phi = 1 where d2 = 0 */
static double venkat_phi(double d1, double d2, double eps2)
{
    if (d2 == 0.0) return 1.0;
    double num = (d1 * d1 + eps2) * d2 + 2.0 * d2 * d2 * d1;
    double den = d2 * (d1 * d1 + 2.0 * d2 * d2 + d1 * d2 + eps2);
    return fmin(1.0, num / den);
}

/* MUSCL (Sec. 2.2): degree-1 polynomial, one limiter value per variable from
 * the min / max over the cell and its face neighbours; Barth-Jespersen by
 * default, Venkatakrishnan's limiter with limiter = 1 */
static void rec_muscl(or_scheme* s, or_ops* o, const double* U, int64_t i, double* V)
{
    const or_mesh* m = s->m;
    int N = s->N, d = s->d, Md = s->Md, nv = s->nv, nf = n_faces_of(s, i), Q = Q_of(s, i);
    const double dx = d == 2 ? sqrt(m->vol[i]) : cbrt(m->vol[i]);
    const double eps2 = pow(s->p.venkat_k * dx, 3.0);
    for (int v = 0; v < nv; ++v) {
        double u0 = U[(int64_t)v * m->nc + i];
        double ac[3];
        for (int k = 0; k < d; ++k) {
            double sum = 0.0;
            for (int b = 0; b < Md; ++b) sum += o->G[k * Md + b] * (U[(int64_t)v * m->nc + o->sten[b]] - u0);
            ac[k] = sum;
        }
        double mn = u0, mx = u0;
        for (int f = 0; f < nf; ++f) {
            int32_t j = m->nbr[i * MAXNF + f];
            if (j < 0) continue;
            double uj = U[(int64_t)v * m->nc + j];
            if (uj < mn) mn = uj;
            if (uj > mx) mx = uj;
        }
        double theta = 1.0, del[64];
        for (int q = 0; q < Q; ++q) {
            double sum = 0.0;
            for (int k = 0; k < d; ++k) sum += o->Phi[q * N + k] * ac[k];
            del[q] = sum;
            double t = 1.0;
            if (s->p.limiter == 1) {
                if (sum > 0.0) t = venkat_phi(mx - u0, sum, eps2);
                else if (sum < 0.0) t = venkat_phi(mn - u0, sum, eps2);
            } else {
                if (sum > 0.0) t = fmin(1.0, (mx - u0) / sum);
                else if (sum < 0.0) t = fmin(1.0, (mn - u0) / sum);
            }
            if (t < theta) theta = t;
        }
        for (int q = 0; q < Q; ++q) V[q * nv + v] = u0 + theta * del[q];
    }
}

/* Harten bound (eq. harten_jump_fix) on density and pressure */
static int harten_ok(const or_scheme* s, const double* U, int64_t i, const double* V)
{
    int nv = s->nv, d = s->d, Q = Q_of(s, i);
    double u0[5];
    get_state(s, U, i, u0);
    double rb = u0[0], pb = pres(u0, d, s->p.gamma);
    double th = s->p.harten_theta, ep = s->p.harten_eps;
    for (int q = 0; q < Q; ++q) {
        const double* w = &V[q * nv];
        if (!(fabs(w[0] - rb) <= th * fmax(fabs(rb), ep))) return 0;
        if (!(fabs(pres(w, d, s->p.gamma) - pb) <= th * fmax(fabs(pb), ep))) return 0;
    }
    return 1;
}

/* detector value of variable kind k (0 density, 1 pressure, 2+ conserved k-1) */
static double nad_q(const or_scheme* s, const double* u, int k)
{
    if (k == 0) return u[0];
    if (k == 1) return pres(u, s->d, s->p.gamma);
    return u[k - 1];
}

/* NAD raw class (Sec. 2.5): per checked variable and face point, with the
 * deactivation test; the cell takes the largest class found */
static int nad_raw(const or_scheme* s, const double* U, int64_t i, const double* V)
{
    const or_mesh* m = s->m;
    int nv = s->nv, nf = n_faces_of(s, i), Q = Q_of(s, i), d = s->d;
    int kinds[8], nk = 0;
    if (s->p.nad_vars & 1) kinds[nk++] = 0;
    if (s->p.nad_vars & 2) kinds[nk++] = 1;
    if (s->p.nad_vars & 4) for (int v = 1; v < nv; ++v) kinds[nk++] = v + 1;
    double ui[5], uj[5];
    get_state(s, U, i, ui);
    double dx = d == 2 ? sqrt(m->vol[i]) : cbrt(m->vol[i]);
    double thr = pow(s->p.kappa * dx, s->p.n_exp);
    int cls = C_LIN;
    for (int kk = 0; kk < nk; ++kk) {
        int k = kinds[kk];
        double qi = nad_q(s, ui, k), mn = qi, mx = qi, dmin = INFINITY, dmax = -INFINITY;
        int nn = 0;
        for (int f = 0; f < nf; ++f) {
            int32_t j = m->nbr[i * MAXNF + f];
            if (j < 0) continue;
            get_state(s, U, j, uj);
            double qj = nad_q(s, uj, k);
            if (qj < mn) mn = qj;
            if (qj > mx) mx = qj;
            double dd = fabs(qj - qi);
            if (dd < dmin) dmin = dd;
            if (dd > dmax) dmax = dd;
            ++nn;
        }
        if (nn == 0 || dmax - dmin < thr) continue; /* deactivated: treated as smooth */
        double range = mx - mn;
        double dm = fmax(s->p.alpha_m, s->p.beta_m * range);
        double sg = s->p.beta_w > 0 ? 1.0 : (s->p.beta_w < 0 ? -1.0 : 0.0);
        double dw = sg * fmax(s->p.alpha_w, fabs(s->p.beta_w * range));
        for (int q = 0; q < Q; ++q) {
            double uq = nad_q(s, &V[q * nv], k);
            int c;
            if (uq <= mn - dm || uq >= mx + dm) c = C_MU;
            else if (mn - dw < uq && uq < mx + dw) c = C_LIN;
            else c = C_CW;
            if (c > cls) cls = c;
        }
    }
    return cls;
}

/* ------------------------------------------------------------------------ */
/* residual                                                                   */
/* ------------------------------------------------------------------------ */
int or_residual(or_scheme* s, const double* U, double* R, const uint8_t* forced, uint8_t* raw_out,
                uint8_t* tag_out, uint8_t* fin_out, const int64_t* sample, int64_t nsample)
{
    const or_mesh* m = s->m;
    int64_t nc = m->nc;
    int nv = s->nv, N = s->N, maxQ = MAXNF * s->nfp;
    /* needed sets: sample S, S1 = S + face neighbours, S2 = S1 + face neighbours */
    uint8_t* need = (uint8_t*)calloc(nc, 1);  /* bit0 R, bit1 face states, bit2 raw class */
    if (sample) { for (int64_t a = 0; a < nsample; ++a) need[sample[a]] |= 7; }
    else memset(need, 7, nc);
    for (int pass = 0; pass < 2; ++pass) {
        uint8_t from = pass == 0 ? 1 : 2, to = pass == 0 ? 2 : 4;
        for (int64_t c = 0; c < nc; ++c)
            if (need[c] & from)
                for (int f = 0; f < n_faces_of(s, c); ++f) {
                    int32_t j = m->nbr[c * MAXNF + f];
                    if (j >= 0) need[j] |= to | (pass == 0 ? 4 : 0);
                }
    }
    int32_t* slot = (int32_t*)malloc(nc * sizeof(int32_t));
    int64_t ns = 0;
    for (int64_t c = 0; c < nc; ++c) slot[c] = (need[c] & 2) ? (int32_t)ns++ : -1;
    double* FS = (double*)malloc((size_t)(ns > 0 ? ns : 1) * maxQ * nv * sizeof(double));
    uint8_t* raw = (uint8_t*)calloc(nc, 1);
    uint8_t* tag = (uint8_t*)calloc(nc, 1);
    uint8_t* fin = (uint8_t*)calloc(nc, 1);
    double* a = (double*)malloc(nv * N * sizeof(double));
    double* V = (double*)malloc(maxQ * nv * sizeof(double));
    const int visc = s->p.mu0 > 0.0;
    double* PG = visc ? (double*)malloc((size_t)(ns > 0 ? ns : 1) * maxQ * 12 * sizeof(double)) : NULL;
    int err = 0;
    /* a2 + a3: linear candidate and detector */
    if (!forced) {
        for (int64_t c = 0; c < nc && !err; ++c) {
            if (!(need[c] & 4)) continue;
            or_ops* o = get_ops(s, c);
            if (!o) { err = 1; break; }
            if (s->p.scheme == 0) { rec_linear(s, o, U, c, a, V); raw[c] = (uint8_t)nad_raw(s, U, c, V); }
            else raw[c] = (uint8_t)(s->p.scheme == 1 ? C_LIN : s->p.scheme == 2 ? C_CW : C_MU);
        }
        /* a4: tag the flagged cells' face neighbourhoods */
        for (int64_t c = 0; c < nc && !err; ++c) {
            if (!(need[c] & 2)) continue;
            uint8_t t = raw[c];
            if (s->p.scheme == 0)
                for (int f = 0; f < n_faces_of(s, c); ++f) {
                    int32_t j = m->nbr[c * MAXNF + f];
                    if (j >= 0 && raw[j] > t) t = raw[j];
                }
            tag[c] = t;
        }
    } else {
        for (int64_t c = 0; c < nc; ++c) if (need[c] & 2) { tag[c] = forced[c]; raw[c] = forced[c]; }
    }
    /* a5 / a6 / a7: reconstruct by class, then the Harten bound */
    for (int64_t c = 0; c < nc && !err; ++c) {
        if (!(need[c] & 2)) continue;
        or_ops* o = get_ops(s, c);
        if (!o) { err = 1; break; }
        double* W = &FS[(size_t)slot[c] * maxQ * nv];
        int Q = Q_of(s, c);
        int cls = tag[c];
        if (cls == C_FIRST) {
            for (int q = 0; q < Q; ++q) get_state(s, U, c, &W[q * nv]);
        } else {
            rec_linear(s, o, U, c, a, W);
            if (cls == C_CW) rec_cweno(s, o, U, c, a, W);
            else if (cls == C_MU) rec_muscl(s, o, U, c, W);
            if (!harten_ok(s, U, c, W)) {
                cls = C_FIRST;
                for (int q = 0; q < Q; ++q) get_state(s, U, c, &W[q * nv]);
            }
        }
        fin[c] = (uint8_t)cls;
    }
    /* viscous gradients at the face points (Sec. 2), at the final face states */
    for (int64_t c = 0; c < nc && visc && !err; ++c) {
        if (!(need[c] & 2)) continue;
        or_ops* o = get_ops(s, c);
        if (!o) { err = 1; break; }
        rec_visc_grad(s, o, U, c, &FS[(size_t)slot[c] * maxQ * nv], &PG[(size_t)slot[c] * maxQ * 12]);
    }
    /* a8: Riemann fluxes at the face points, summed into the residual */
    if (!err) {
        for (int64_t c = 0; c < nc; ++c)
            if (need[c] & 1) for (int v = 0; v < nv; ++v) R[(int64_t)v * nc + c] = 0.0;
        double F[5];
        for (int64_t g = 0; g < m->nface; ++g) {
            int32_t co = m->fo[g], cn = m->fn[g];
            int wo = need[co] & 1, wn = cn >= 0 && (need[cn] & 1);
            if (!wo && !wn) continue;
            const double* WL = &FS[(size_t)slot[co] * maxQ * nv + (size_t)m->ffo[g] * s->nfp * nv];
            const double* WR = cn >= 0 ? &FS[(size_t)slot[cn] * maxQ * nv + (size_t)m->ffn[g] * s->nfp * nv] : WL;
            double inv_lint = 0.0;
            const double *GLp = NULL, *GRp = NULL;
            if (visc) {
                /* distance between the two cells' centres (vertex means), the
                 * neighbour's moved into the owner's frame */
                if (cn >= 0) {
                    double l2 = 0.0;
                    for (int k = 0; k < 3; ++k) {
                        double dx = m->vmean[3 * cn + k] + m->fshift[3 * g + k] - m->vmean[3 * co + k];
                        l2 += dx * dx;
                    }
                    inv_lint = 1.0 / sqrt(l2);
                }
                GLp = &PG[(size_t)slot[co] * maxQ * 12 + (size_t)m->ffo[g] * s->nfp * 12];
                GRp = cn >= 0 ? &PG[(size_t)slot[cn] * maxQ * 12 + (size_t)m->ffn[g] * s->nfp * 12] : GLp;
            }
            for (int al = 0; al < s->nfp; ++al) {
                or_flux(s->p.flux, s->d, s->p.gamma, &WL[al * nv], &WR[al * nv], &m->fnorm[3 * g], F);
                double w = s->fqw[g * s->nfp + al];
                for (int v = 0; v < nv; ++v) {
                    if (wo) R[(int64_t)v * nc + co] -= F[v] * w / m->vol[co];
                    if (wn) R[(int64_t)v * nc + cn] += F[v] * w / m->vol[cn];
                }
                if (visc) {
                    /* + (1/|V|) sum F_v w |S| (eq. EulerEquationsDetails); an open
                     * boundary's outside copies the inside state and gradient */
                    visc_flux(s, &WL[al * nv], &WR[al * nv], &GLp[al * 12], &GRp[al * 12], &m->fnorm[3 * g],
                              inv_lint, F);
                    for (int v = 0; v < nv; ++v) {
                        if (wo) R[(int64_t)v * nc + co] += F[v] * w / m->vol[co];
                        if (wn) R[(int64_t)v * nc + cn] -= F[v] * w / m->vol[cn];
                    }
                }
            }
        }
    }
    for (int64_t c = 0; c < nc; ++c) {
        if (raw_out && (need[c] & 4)) raw_out[c] = raw[c];
        if (tag_out && (need[c] & 2)) tag_out[c] = tag[c];
        if (fin_out && (need[c] & 2)) fin_out[c] = fin[c];
    }
    free(need); free(slot); free(FS); free(raw); free(tag); free(fin); free(a); free(V); free(PG);
    return err ? -1 : 0;
}

/* ------------------------------------------------------------------------ */
/* time step and SSP-RK3                                                      */
/* ------------------------------------------------------------------------ */
double or_dt(or_scheme* s, const double* U, double cfl)
{
    const or_mesh* m = s->m;
    double dt = INFINITY, u[5];
    for (int64_t c = 0; c < m->nc; ++c) {
        get_state(s, U, c, u);
        double p = pres(u, s->d, s->p.gamma), cs = sqrt(s->p.gamma * p / u[0]);
        double lam = 0.0;
        for (int f = 0; f < n_faces_of(s, c); ++f) {
            int64_t g = m->cface[c * MAXNF + f];
            double un = 0.0;
            for (int k = 0; k < s->d; ++k) un += u[1 + k] / u[0] * m->fnorm[3 * g + k];
            lam += (fabs(un) + cs) * m->farea[g];
        }
        if (s->p.mu0 > 0.0) {
            /* viscous terms: the explicit diffusion limit, 4 nu sum_f |S_f|^2 / |V|
             * with nu = max(4/3, gamma / Pr) mu / rho (momentum and heat) --
             * a reading: the paper states a convective CFL number only */
            double T = p / u[0], T0 = s->p.t0, S = s->p.suth_s, s2 = 0.0;
            double mu = s->p.mu0 * pow(T / T0, 1.5) * (T0 + S) / (T + S);
            double nu = fmax(4.0 / 3.0, s->p.gamma / s->p.prandtl) * mu / u[0];
            for (int f = 0; f < n_faces_of(s, c); ++f) {
                double a = m->farea[m->cface[c * MAXNF + f]];
                s2 += a * a;
            }
            lam += 4.0 * nu * s2 / m->vol[c];
        }
        double t = cfl * m->vol[c] / lam;
        if (t < dt) dt = t;
    }
    return dt;
}

typedef void (*or_rhs_fn)(void* ctx, const double* U, double* R);

/* Shu-Osher three-stage SSP Runge-Kutta over a generic right-hand side */
void or_rk3_generic(int64_t n, double* U, double dt, or_rhs_fn rhs, void* ctx)
{
    double* U1 = (double*)malloc(n * sizeof(double));
    double* R = (double*)malloc(n * sizeof(double));
    rhs(ctx, U, R);
    for (int64_t k = 0; k < n; ++k) U1[k] = U[k] + dt * R[k];
    rhs(ctx, U1, R);
    for (int64_t k = 0; k < n; ++k) U1[k] = 0.75 * U[k] + 0.25 * (U1[k] + dt * R[k]);
    rhs(ctx, U1, R);
    for (int64_t k = 0; k < n; ++k) U[k] = U[k] / 3.0 + 2.0 / 3.0 * (U1[k] + dt * R[k]);
    free(U1); free(R);
}

/* The five-stage, fourth-order SSP Runge-Kutta method of Spiteri and Ruuth
 * (the paper's time integrator), Shu-Osher form
 *   u_i = sum_j alpha_ij u_j + beta_ij dt L(u_j),  u_0 = u^n,  u^{n+1} = u_5 */
static const double RK54_A[6][5] = {
    {0, 0, 0, 0, 0},
    {1.0, 0, 0, 0, 0},
    {0.444370493651235, 0.555629506348765, 0, 0, 0},
    {0.620101851488403, 0, 0.379898148511597, 0, 0},
    {0.178079954393132, 0, 0, 0.821920045606868, 0},
    {0, 0, 0.517231671970585, 0.096059710526147, 0.386708617503269},
};
static const double RK54_B[6][5] = {
    {0, 0, 0, 0, 0},
    {0.391752226571890, 0, 0, 0, 0},
    {0, 0.368410593050371, 0, 0, 0},
    {0, 0, 0.251891774271694, 0, 0},
    {0, 0, 0, 0.544974750228521, 0},
    {0, 0, 0, 0.063692468666290, 0.226007483236906},
};

void or_rk54_table(double* alpha, double* beta)
{
    for (int i = 0; i < 6; ++i)
        for (int j = 0; j < 5; ++j) { alpha[i * 5 + j] = RK54_A[i][j]; beta[i * 5 + j] = RK54_B[i][j]; }
}

void or_rk54_generic(int64_t n, double* U, double dt, or_rhs_fn rhs, void* ctx)
{
    double* u[6];
    double* L[5];
    u[0] = U;
    for (int i = 1; i < 6; ++i) u[i] = (double*)malloc(n * sizeof(double));
    for (int j = 0; j < 5; ++j) L[j] = (double*)malloc(n * sizeof(double));
    for (int i = 1; i < 6; ++i) {
        rhs(ctx, u[i - 1], L[i - 1]);
        for (int64_t k = 0; k < n; ++k) {
            double x = 0.0;
            for (int j = 0; j < i; ++j) x += RK54_A[i][j] * u[j][k] + RK54_B[i][j] * dt * L[j][k];
            u[i][k] = x;
        }
    }
    for (int64_t k = 0; k < n; ++k) U[k] = u[5][k];
    for (int i = 1; i < 6; ++i) free(u[i]);
    for (int j = 0; j < 5; ++j) free(L[j]);
}

static int g_rk_err;
static void scheme_rhs(void* ctx, const double* U, double* R)
{
    if (or_residual((or_scheme*)ctx, U, R, NULL, NULL, NULL, NULL, NULL, 0) != 0) g_rk_err = 1;
}
int or_rk3_step(or_scheme* s, double* U, double dt)
{
    g_rk_err = 0;
    or_rk3_generic((int64_t)s->nv * s->m->nc, U, dt, scheme_rhs, s);
    return g_rk_err ? -1 : 0;
}
int or_rk54_step(or_scheme* s, double* U, double dt)
{
    g_rk_err = 0;
    or_rk54_generic((int64_t)s->nv * s->m->nc, U, dt, scheme_rhs, s);
    return g_rk_err ? -1 : 0;
}

/* ------------------------------------------------------------------------ */
/* introspection for the pins                                                 */
/* ------------------------------------------------------------------------ */
void or_scheme_sizes(const or_scheme* s, int* out /* N M Md nq nfp nv */)
{
    out[0] = s->N; out[1] = s->M; out[2] = s->Md; out[3] = s->nq; out[4] = s->nfp; out[5] = s->nv;
}
int or_stencil(or_scheme* s, int64_t c, int32_t* sten, int32_t* dir)
{
    or_ops* o = get_ops(s, c);
    if (!o) return -1;
    memcpy(sten, o->sten, s->M * sizeof(int32_t));
    if (dir) memcpy(dir, o->dir, n_faces_of(s, c) * s->Md * sizeof(int32_t));
    return 0;
}
/* which: 0 P [N][M], 1 Phi [Q][N], 2 OI [N][N], 3 A [M][N], 4 Vr [M+1],
 *        5 D [nf][d][Md], 6 G [d][Md], 7 stencil shifts [M][3], 8 nd [nf] */
int or_cell_operator(or_scheme* s, int64_t c, int which, double* out)
{
    or_ops* o = get_ops(s, c);
    if (!o) return -1;
    int N = s->N, M = s->M, Q = Q_of(s, c), nf = n_faces_of(s, c), d = s->d, Md = s->Md;
    switch (which) {
    case 0: memcpy(out, o->P, N * M * sizeof(double)); break;
    case 1: memcpy(out, o->Phi, Q * N * sizeof(double)); break;
    case 2: memcpy(out, o->OI, N * N * sizeof(double)); break;
    case 3: memcpy(out, o->A, M * N * sizeof(double)); break;
    case 4: memcpy(out, o->Vr, (M + 1) * sizeof(double)); break;
    case 5: memcpy(out, o->D, nf * d * Md * sizeof(double)); break;
    case 6: memcpy(out, o->G, d * Md * sizeof(double)); break;
    case 7: memcpy(out, o->sshift, M * 3 * sizeof(double)); break;
    case 8: for (int f = 0; f < nf; ++f) out[f] = o->nd[f]; break;
    default: return -1;
    }
    return 0;
}
/* face points of cell c in its own frame, [Q][3] */
int or_cell_face_points(or_scheme* s, int64_t c, double* out)
{
    double nrm[3];
    for (int f = 0; f < n_faces_of(s, c); ++f) cell_face_points(s, c, f, &out[3 * f * s->nfp], nrm);
    return 0;
}
/* face-point weights w |S| of one cell, in its face-point order */
int or_cell_face_weights(or_scheme* s, int64_t c, double* out)
{
    const or_mesh* m = s->m;
    for (int f = 0; f < n_faces_of(s, c); ++f) {
        int64_t g = m->cface[c * MAXNF + f];
        for (int a = 0; a < s->nfp; ++a) out[f * s->nfp + a] = s->fqw[g * s->nfp + a];
    }
    return 0;
}
/* reference map of cell c: x0 [3], Jinv [3][3] */
void or_cell_refmap(or_scheme* s, int64_t c, double* x0, double* Jinv)
{
    double Ji[3][3], det;
    ref_map(s, c, x0, Ji, &det);
    memcpy(Jinv, Ji, sizeof Ji);
}
/* face values of one cell for a given class, without the Harten bound */
int or_reconstruct(or_scheme* s, const double* U, int64_t c, int cls, double* Vout)
{
    or_ops* o = get_ops(s, c);
    if (!o) return -1;
    double a[5 * 128];
    rec_linear(s, o, U, c, a, Vout);
    if (cls == C_CW) rec_cweno(s, o, U, c, a, Vout);
    else if (cls == C_MU) rec_muscl(s, o, U, c, Vout);
    else if (cls == C_FIRST)
        for (int q = 0; q < Q_of(s, c); ++q) get_state(s, U, c, &Vout[q * s->nv]);
    return 0;
}
int or_harten_ok(or_scheme* s, const double* U, int64_t c, const double* V) { return harten_ok(s, U, c, V); }
int or_nad_raw_cell(or_scheme* s, const double* U, int64_t c)
{
    or_ops* o = get_ops(s, c);
    if (!o) return -1;
    double a[5 * 128], V[5 * 64];
    rec_linear(s, o, U, c, a, V);
    return nad_raw(s, U, c, V);
}
/* CWENOZ weights and indicators of one cell / variable; returns s_t */
int or_cweno_info(or_scheme* s, const double* U, int64_t c, int v, double* omega, double* SI, double* acw)
{
    or_ops* o = get_ops(s, c);
    if (!o) return -1;
    double a[5 * 128], V[5 * 64], tmp[128];
    rec_linear(s, o, U, c, a, V);
    rec_cweno_var(s, o, U, c, v, &a[v * s->N], acw ? acw : tmp, omega, SI);
    return n_faces_of(s, c) + 1;
}
int64_t or_ops_built(const or_scheme* s) { return s->nops_built; }
