// setup_math.cuh -- per-cell FP64 construction of the reconstruction
// operators (run once, Sec. 2.1: the pseudo-inverse is computed once at the
// beginning of the simulation; Sec. 2.3: the OI matrix is precomputed).
//
// For one cell i:
//   1. reference map xi = J^-1 (x - v0) from the cell's corner simplex
//      (triangle v0 v1 v2, quadrilateral v0 v1 v3, hexahedron v0 v1 v3 v4);
//   2. basis psi_k = xi^a eta^b zeta^c, 1 <= a+b+c <= r, made mean-free over
//      the cell (phi_k = psi_k - mean_{V_0'} psi_k);
//   3. A_mk = int_{V_m'} phi_k over each (periodically shifted) stencil cell;
//   4. Householder QR of A, pseudo-inverse A^+ column by column, and
//      P = A^+ diag(|V_m'|) so that the coefficients are a = P (U_m - U_0);
//   5. basis values at the cell's face points, L = Phi P (rows of candidate values
//      U_0 + L (U_m - U_0)) and the linear block Phi_lin;
//   6. OI_kq = sum_{1<=|beta|<=r} int_{V_0'} D^beta phi_k D^beta phi_q in
//      reference coordinates (h_c = 1), from exact moments of the cell;
//   7. degree-1 pseudo-inverses of the directional stencils (D) and of the
//      MUSCL stencil (G), with |V_m'| folded in the same way.
// Volume integrals: collapsed Gauss-Legendre on triangles, quadrilaterals as
// two triangles, tensor Gauss-Legendre on the trilinear hexahedron map, with
// r + 1 points per direction in 2D and r + 2 on hexahedra (exact for every
// integrand used, including the degree-2r moments behind OI).
#pragma once

#include <cmath>
#include <cstdint>

#ifdef __CUDACC__
#define HD __host__ __device__
#else
#define HD
#endif

namespace hfv {

constexpr int kNmax = 55;   // K(5, 3) - 1 (hexahedra at order 6)
constexpr int kMmax = 112;  // 2 K(5, 3)
constexpr int kGmax = 8;    // Gauss points per direction
constexpr int kMomMax = 286; // moments of total degree <= 10 in 3D: K(10, 3)

struct SetupParams {
    const double* xyz;       // [nn][3]
    const int64_t* cptr;
    const int32_t* cidx;
    const uint8_t* type;
    const int32_t* sten;     // [nc][M]
    const int8_t* sshift;    // [nc][M][3]
    const uint8_t* dir;      // [nc][6][Md]
    const uint8_t* nd;       // [nc][6]
    const int32_t* fvtx;     // [nc][6][4] owner-ordered face vertices
    const int8_t* fk;        // [nc][6][3] periods added to them for this cell's frame
    const double* farea;     // [nc][6]
    const int64_t* qoff;     // [nc+1]
    const int64_t* loff;     // [nc+1] offsets of the L blocks
    double period[3];
    int d, r, N, M, Md, nq, nfp, nvq;
    int lcw;                 // column chunk of the L blocks: 16 bytes of the kernel precision
    double gfx[kGmax], gfw[kGmax];  // face rule on [0,1]
    double gvx[kGmax], gvw[kGmax];  // volume rule on [0,1]
    int8_t ex[kNmax][3];            // monomial exponents
};

struct SetupOut {
    double* L;      // cell c at loff[c]: Q_c rows x M columns, columns in chunks of lcw (l_index)
    double* P;      // [nc][N][M]
    double* Phil;   // [qoff][d]
    double* OI;     // [nc][N(N+1)/2]
    double* D;      // [nc][6][d][Md]
    double* G;      // [nc][d][Md]
    double* W;      // [qoff]
    double* VX;     // [nc][d + d d] mean of xi, then J^-1 (viscous terms; null otherwise)
    int* err;       // first failing cell + 1 (0 = none)
    // the arrays may hold a chunk of cells only: cell c is written at c - cbase,
    // its face points at qoff[c] - qbase, its L block at loff[c] - lbase
    int64_t cbase = 0, qbase = 0, lbase = 0;
};

// position of L_qm inside a cell's block of Q rows and M columns: column
// chunks of width W (the values of 16 bytes), chunk j = [Q][W]; the last
// partial chunk of width M mod W = [Q][M mod W]
HD inline int64_t l_index(int q, int m, int Q, int M, int W)
{
    const int M4 = M / W * W;
    if (m < M4) return (int64_t)(m / W) * Q * W + q * W + m % W;
    return (int64_t)M4 * Q + q * (M - M4) + (m - M4);
}

// workspace of one thread: A [M][N], stride-interleaved between threads
struct SetupWork {
    double* base;
    int64_t stride;
    HD double& A(int m, int k, int N) const { return base[(int64_t)(m * N + k) * stride]; }
};

namespace setup_detail {

// cell types as in hfv.h: 1 triangle, 2 quadrilateral, 3 tetrahedron,
// 4 hexahedron, 5 prism, 6 pyramid
HD inline int nverts(int t) { return t == 1 ? 3 : t == 2 ? 4 : t == 3 ? 4 : t == 5 ? 6 : t == 6 ? 5 : 8; }
HD inline int nfaces(int t) { return t == 1 ? 3 : t == 2 ? 4 : t == 3 ? 4 : t == 5 || t == 6 ? 5 : 6; }
// vertices of face f (prisms list their two triangles first, pyramids their
// four triangles first)
HD inline int face_nv(int t, int f)
{
    return t == 1 || t == 2 ? 2 : t == 3 ? 3 : t == 5 ? (f < 2 ? 3 : 4) : t == 6 ? (f < 4 ? 3 : 4) : 4;
}

HD inline double ipow(double x, int e)
{
    double r = 1.0;
    for (int i = 0; i < e; ++i) r *= x;
    return r;
}

// vertices of cell c shifted by k periods, mapped to xi of the current cell
HD inline void ref_vertices(const SetupParams& S, int64_t c, const int8_t* k, const double x0[3], const double Ji[3][3],
                            double v[8][3])
{
    int nvx = nverts(S.type[c]);
    for (int a = 0; a < nvx; ++a) {
        const double* x = &S.xyz[3 * (int64_t)S.cidx[S.cptr[c] + a]];
        double dx[3];
        for (int q = 0; q < 3; ++q) dx[q] = x[q] + (k ? k[q] * S.period[q] : 0.0) - x0[q];
        for (int q = 0; q < 3; ++q) v[a][q] = Ji[q][0] * dx[0] + Ji[q][1] * dx[1] + Ji[q][2] * dx[2];
        if (S.d == 2) v[a][2] = 0.0;
    }
}

// accumulate int over the cell of every monomial of total degree <= maxdeg
// (graded order of `moment_index`) and the cell measure
HD inline int moment_count(int d, int deg)
{
    int n = 1;
    for (int l = 1; l <= d; ++l) n = n * (deg + l) / l;
    return n;
}
HD inline int moment_index(int d, int a, int b, int c)
{
    // graded lexicographic: all monomials of lower total degree first
    int deg = a + b + c;
    int base = deg == 0 ? 0 : moment_count(d, deg - 1);
    if (d == 2) return base + (deg - a);                         // a = deg .. 0
    int off = 0;
    for (int aa = deg; aa > a; --aa) off += deg - aa + 1;        // entries with larger a
    return base + off + (deg - a - b);                           // b = deg-a .. 0
}

template <class F>
HD inline void cell_rule(const SetupParams& S, int t, const double v[8][3], F&& f)
{
    const int n = S.nvq;
    if (t == 1 || t == 2) {
        int ntri = t == 1 ? 1 : 2;
        for (int s = 0; s < ntri; ++s) {
            const double* p0 = v[0];
            const double* p1 = v[s == 0 ? 1 : 2];
            const double* p2 = v[s == 0 ? 2 : 3];
            double e1x = p1[0] - p0[0], e1y = p1[1] - p0[1];
            double e2x = p2[0] - p0[0], e2y = p2[1] - p0[1];
            double det = fabs(e1x * e2y - e1y * e2x);
            // collapsed square: x = p0 + u e1 + u w (e2 - e1), |J| = u det
            for (int i = 0; i < n; ++i)
                for (int j = 0; j < n; ++j) {
                    double u = S.gvx[i], w = S.gvx[j];
                    double x[3] = {p0[0] + u * e1x + u * w * (e2x - e1x), p0[1] + u * e1y + u * w * (e2y - e1y), 0.0};
                    f(x, S.gvw[i] * S.gvw[j] * u * det);
                }
        }
        return;
    }
    if (t == 3) {
        // tetrahedron: collapsed cube x = v0 + s a + s w b + s w z c with
        // a = v1 - v0, b = v2 - v1, c = v3 - v2, |J| = s^2 w |det(a, b, c)|
        double a[3], b[3], cc[3];
        for (int q = 0; q < 3; ++q) { a[q] = v[1][q] - v[0][q]; b[q] = v[2][q] - v[1][q]; cc[q] = v[3][q] - v[2][q]; }
        double det = fabs(a[0] * (b[1] * cc[2] - b[2] * cc[1]) - a[1] * (b[0] * cc[2] - b[2] * cc[0]) +
                          a[2] * (b[0] * cc[1] - b[1] * cc[0]));
        for (int i = 0; i < n; ++i)
            for (int j = 0; j < n; ++j)
                for (int k = 0; k < n; ++k) {
                    double s1 = S.gvx[i], w = S.gvx[j], z = S.gvx[k];
                    double x[3];
                    for (int q = 0; q < 3; ++q) x[q] = v[0][q] + s1 * a[q] + s1 * w * b[q] + s1 * w * z * cc[q];
                    f(x, S.gvw[i] * S.gvw[j] * S.gvw[k] * s1 * s1 * w * det);
                }
        return;
    }
    if (t == 5) {
        // prism: the collapsed triangle (xi, eta) = (u (1 - w), u w) times
        // zeta, x = (1 - zeta) T(v0, v1, v2) + zeta T(v3, v4, v5) with T the
        // barycentric combination; weight u |det dx/d(xi, eta, zeta)|
        for (int i = 0; i < n; ++i)
            for (int j = 0; j < n; ++j)
                for (int k = 0; k < n; ++k) {
                    const double u = S.gvx[i], w = S.gvx[j], z = S.gvx[k];
                    const double xi = u * (1 - w), eta = u * w, l0 = 1 - xi - eta;
                    double x[3], J[3][3];
                    for (int q = 0; q < 3; ++q) {
                        const double bot = l0 * v[0][q] + xi * v[1][q] + eta * v[2][q];
                        const double top = l0 * v[3][q] + xi * v[4][q] + eta * v[5][q];
                        x[q] = (1 - z) * bot + z * top;
                        J[q][0] = (1 - z) * (v[1][q] - v[0][q]) + z * (v[4][q] - v[3][q]);
                        J[q][1] = (1 - z) * (v[2][q] - v[0][q]) + z * (v[5][q] - v[3][q]);
                        J[q][2] = top - bot;
                    }
                    const double det = J[0][0] * (J[1][1] * J[2][2] - J[1][2] * J[2][1]) -
                                       J[0][1] * (J[1][0] * J[2][2] - J[1][2] * J[2][0]) +
                                       J[0][2] * (J[1][0] * J[2][1] - J[1][1] * J[2][0]);
                    f(x, S.gvw[i] * S.gvw[j] * S.gvw[k] * u * fabs(det));
                }
        return;
    }
    if (t == 6) {
        // pyramid: the unit cube collapsed onto the apex, x = (1 - s) B(a, b)
        // + s v4 with B the bilinear base v0 v1 v2 v3; weight |det|, which
        // carries (1 - s)^2
        for (int i = 0; i < n; ++i)
            for (int j = 0; j < n; ++j)
                for (int k = 0; k < n; ++k) {
                    const double a = S.gvx[i], b = S.gvx[j], sz = S.gvx[k];
                    double x[3], J[3][3];
                    for (int q = 0; q < 3; ++q) {
                        const double B = (1 - a) * (1 - b) * v[0][q] + a * (1 - b) * v[1][q] + a * b * v[2][q] + (1 - a) * b * v[3][q];
                        const double Ba = (1 - b) * (v[1][q] - v[0][q]) + b * (v[2][q] - v[3][q]);
                        const double Bb = (1 - a) * (v[3][q] - v[0][q]) + a * (v[2][q] - v[1][q]);
                        x[q] = (1 - sz) * B + sz * v[4][q];
                        J[q][0] = (1 - sz) * Ba;
                        J[q][1] = (1 - sz) * Bb;
                        J[q][2] = v[4][q] - B;
                    }
                    const double det = J[0][0] * (J[1][1] * J[2][2] - J[1][2] * J[2][1]) -
                                       J[0][1] * (J[1][0] * J[2][2] - J[1][2] * J[2][0]) +
                                       J[0][2] * (J[1][0] * J[2][1] - J[1][1] * J[2][0]);
                    f(x, S.gvw[i] * S.gvw[j] * S.gvw[k] * fabs(det));
                }
        return;
    }
    // hexahedron: trilinear map of the unit cube
    const int cs[8][3] = {{0, 0, 0}, {1, 0, 0}, {1, 1, 0}, {0, 1, 0}, {0, 0, 1}, {1, 0, 1}, {1, 1, 1}, {0, 1, 1}};
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j)
            for (int k = 0; k < n; ++k) {
                double u[3] = {S.gvx[i], S.gvx[j], S.gvx[k]};
                double x[3] = {0, 0, 0}, J[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
                for (int a = 0; a < 8; ++a) {
                    double s0 = cs[a][0] ? u[0] : 1 - u[0], s1 = cs[a][1] ? u[1] : 1 - u[1], s2 = cs[a][2] ? u[2] : 1 - u[2];
                    double g0 = cs[a][0] ? 1 : -1, g1 = cs[a][1] ? 1 : -1, g2 = cs[a][2] ? 1 : -1;
                    double N0 = s0 * s1 * s2;
                    double dN[3] = {g0 * s1 * s2, s0 * g1 * s2, s0 * s1 * g2};
                    for (int q = 0; q < 3; ++q) {
                        x[q] += N0 * v[a][q];
                        for (int e = 0; e < 3; ++e) J[q][e] += v[a][q] * dN[e];
                    }
                }
                double det = J[0][0] * (J[1][1] * J[2][2] - J[1][2] * J[2][1]) -
                             J[0][1] * (J[1][0] * J[2][2] - J[1][2] * J[2][0]) +
                             J[0][2] * (J[1][0] * J[2][1] - J[1][1] * J[2][0]);
                f(x, S.gvw[i] * S.gvw[j] * S.gvw[k] * fabs(det));
            }
}

// Householder QR of the rows x cols matrix held by `at(m, k)` (rows >= cols);
// reflector m-th entries stay in the lower part, diag / beta returned.
template <class Acc>
HD inline bool householder(Acc&& at, int rows, int cols, double* diag, double* beta)
{
    double dmax = 0.0;
    for (int k = 0; k < cols; ++k) {
        double nrm2 = 0.0;
        for (int m = k; m < rows; ++m) nrm2 += at(m, k) * at(m, k);
        double nrm = sqrt(nrm2);
        if (!(nrm > 0.0)) return false;
        double x0 = at(k, k);
        double alpha = x0 > 0.0 ? -nrm : nrm;
        at(k, k) = x0 - alpha;                      // v = x - alpha e1
        double vv = nrm2 - x0 * x0 + (x0 - alpha) * (x0 - alpha);
        beta[k] = 2.0 / vv;
        diag[k] = alpha;
        for (int j = k + 1; j < cols; ++j) {
            double s = 0.0;
            for (int m = k; m < rows; ++m) s += at(m, k) * at(m, j);
            s *= beta[k];
            for (int m = k; m < rows; ++m) at(m, j) -= s * at(m, k);
        }
        if (fabs(alpha) > dmax) dmax = fabs(alpha);
    }
    for (int k = 0; k < cols; ++k)
        if (!(fabs(diag[k]) > 1e-12 * dmax)) return false;
    return true;
}

// column j of the pseudo-inverse: R x = (Q^T e_j)[0:cols]
template <class Acc>
HD inline void pinv_column(Acc&& at, int rows, int cols, const double* diag, const double* beta, int j, double* x,
                           double* y)
{
    for (int m = 0; m < rows; ++m) y[m] = m == j ? 1.0 : 0.0;
    for (int k = 0; k < cols; ++k) {
        double s = 0.0;
        for (int m = k; m < rows; ++m) s += at(m, k) * y[m];
        s *= beta[k];
        for (int m = k; m < rows; ++m) y[m] -= s * at(m, k);
    }
    for (int k = cols - 1; k >= 0; --k) {
        double s = y[k];
        for (int l = k + 1; l < cols; ++l) s -= at(k, l) * x[l];
        x[k] = s / diag[k];
    }
}

}  // namespace setup_detail

// Build every operator of cell c.  Returns false on a rank-deficient system.
HD inline bool setup_cell(const SetupParams& S, const SetupOut& O, const SetupWork& Wk, int64_t c)
{
    using namespace setup_detail;
    const int d = S.d, N = S.N, M = S.M, Md = S.Md, r = S.r;
    const int t = S.type[c];
    const int nf = nfaces(t);
    const int64_t q0 = S.qoff[c];

    // 1. reference map of cell c
    double x0[3], J[3][3], Ji[3][3];
    {
        const double* p0 = &S.xyz[3 * (int64_t)S.cidx[S.cptr[c]]];
        // corner simplex: triangle v0 v1 v2, quadrilateral v0 v1 v3,
        // tetrahedron and prism v0 v1 v2 v3, hexahedron and pyramid v0 v1 v3 v4
        int c1 = 1, c2 = (t == 1 || t == 3 || t == 5) ? 2 : 3, c3 = (t == 3 || t == 5) ? 3 : 4;
        const double* p1 = &S.xyz[3 * (int64_t)S.cidx[S.cptr[c] + c1]];
        const double* p2 = &S.xyz[3 * (int64_t)S.cidx[S.cptr[c] + c2]];
        for (int q = 0; q < 3; ++q) {
            x0[q] = p0[q];
            J[q][0] = p1[q] - p0[q];
            J[q][1] = p2[q] - p0[q];
            J[q][2] = d == 3 ? S.xyz[3 * (int64_t)S.cidx[S.cptr[c] + c3] + q] - p0[q] : (q == 2 ? 1.0 : 0.0);
        }
        double det = J[0][0] * (J[1][1] * J[2][2] - J[1][2] * J[2][1]) - J[0][1] * (J[1][0] * J[2][2] - J[1][2] * J[2][0]) +
                     J[0][2] * (J[1][0] * J[2][1] - J[1][1] * J[2][0]);
        double id = 1.0 / det;
        Ji[0][0] = (J[1][1] * J[2][2] - J[1][2] * J[2][1]) * id;
        Ji[0][1] = (J[0][2] * J[2][1] - J[0][1] * J[2][2]) * id;
        Ji[0][2] = (J[0][1] * J[1][2] - J[0][2] * J[1][1]) * id;
        Ji[1][0] = (J[1][2] * J[2][0] - J[1][0] * J[2][2]) * id;
        Ji[1][1] = (J[0][0] * J[2][2] - J[0][2] * J[2][0]) * id;
        Ji[1][2] = (J[0][2] * J[1][0] - J[0][0] * J[1][2]) * id;
        Ji[2][0] = (J[1][0] * J[2][1] - J[1][1] * J[2][0]) * id;
        Ji[2][1] = (J[0][1] * J[2][0] - J[0][0] * J[2][1]) * id;
        Ji[2][2] = (J[0][0] * J[1][1] - J[0][1] * J[1][0]) * id;
    }

    // 2. moments of cell 0 up to degree 2r (means of psi, OI)
    double v[8][3];
    double mom[kMomMax];
    const int nmom = moment_count(d, 2 * r);
    for (int a = 0; a < nmom; ++a) mom[a] = 0.0;
    ref_vertices(S, c, nullptr, x0, Ji, v);
    cell_rule(S, t, v, [&](const double* x, double w) {
        for (int deg = 0; deg <= 2 * r; ++deg)
            for (int a = deg; a >= 0; --a) {
                if (d == 2) {
                    mom[moment_index(2, a, deg - a, 0)] += w * ipow(x[0], a) * ipow(x[1], deg - a);
                } else {
                    for (int b = deg - a; b >= 0; --b)
                        mom[moment_index(3, a, b, deg - a - b)] += w * ipow(x[0], a) * ipow(x[1], b) * ipow(x[2], deg - a - b);
                }
            }
    });
    const double V0 = mom[0];
    double mean0[kNmax];
    for (int k = 0; k < N; ++k) mean0[k] = mom[moment_index(d, S.ex[k][0], S.ex[k][1], S.ex[k][2])] / V0;
    if (O.VX) {
        // the degree-1 monomials come first (xi, eta[, zeta]): their means,
        // then the reference map, for gradients at the face points
        double* vx = &O.VX[(c - O.cbase) * (int64_t)(d + d * d)];
        for (int k = 0; k < d; ++k) vx[k] = mean0[k];
        for (int b = 0; b < d; ++b)
            for (int j = 0; j < d; ++j) vx[d + b * d + j] = Ji[b][j];
    }

    // 3. A_mk over the stencil cells; reference volumes kept in Vr
    double Vr[kMmax], Alin[kMmax][3];
    for (int m = 0; m < M; ++m) {
        int64_t j = S.sten[c * M + m];
        ref_vertices(S, j, &S.sshift[(c * M + m) * 3], x0, Ji, v);
        double acc[kNmax + 1];
        for (int k = 0; k <= N; ++k) acc[k] = 0.0;
        cell_rule(S, S.type[j], v, [&](const double* x, double w) {
            acc[N] += w;
            for (int k = 0; k < N; ++k) acc[k] += w * ipow(x[0], S.ex[k][0]) * ipow(x[1], S.ex[k][1]) * ipow(x[2], S.ex[k][2]);
        });
        Vr[m] = acc[N];
        for (int k = 0; k < N; ++k) Wk.A(m, k, N) = acc[k] - acc[N] * mean0[k];
        for (int k = 0; k < d; ++k) Alin[m][k] = Wk.A(m, k, N);
    }

    // 4. QR and P = A^+ diag(Vr)
    double diag[kNmax], beta[kNmax], x[kNmax], y[kMmax];
    auto atA = [&](int m, int k) -> double& { return Wk.A(m, k, N); };
    if (!householder(atA, M, N, diag, beta)) return false;
    double* P = &O.P[(c - O.cbase) * (int64_t)N * M];
    for (int j = 0; j < M; ++j) {
        pinv_column(atA, M, N, diag, beta, j, x, y);
        for (int k = 0; k < N; ++k) P[k * M + j] = x[k] * Vr[j];
    }

    // 5. face points: basis values, L = Phi P, Phi_lin and weights
    double* L = &O.L[S.loff[c] - O.lbase];
    for (int f = 0; f < nf; ++f) {
        const int32_t* fv = &S.fvtx[(c * 6 + f) * 4];
        const int8_t* k = &S.fk[(c * 6 + f) * 3];
        double pv[4][3];
        const int nfv = face_nv(t, f);
        for (int a = 0; a < nfv; ++a)
            for (int q = 0; q < 3; ++q) pv[a][q] = S.xyz[3 * (int64_t)fv[a] + q] + k[q] * S.period[q];
        const double area = S.farea[c * 6 + f];
        for (int al = 0; al < S.nfp; ++al) {
            double xp[3], wgt;
            if (d == 2) {
                double s = S.gfx[al];
                for (int q = 0; q < 3; ++q) xp[q] = pv[0][q] + s * (pv[1][q] - pv[0][q]);
                wgt = S.gfw[al] * area;
            } else if (nfv == 3) {
                // triangle face: collapsed rule x = p0 + s (p1 - p0) + s u (p2 - p1),
                // weight w_i w_j 2 s |S|
                int i = al % S.nq, jj = al / S.nq;
                double s = S.gfx[i], u = S.gfx[jj];
                for (int q = 0; q < 3; ++q) xp[q] = pv[0][q] + s * (pv[1][q] - pv[0][q]) + s * u * (pv[2][q] - pv[1][q]);
                wgt = S.gfw[i] * S.gfw[jj] * 2.0 * s * area;
            } else {
                int i = al % S.nq, jj = al / S.nq;
                double s = S.gfx[i], u = S.gfx[jj];
                for (int q = 0; q < 3; ++q)
                    xp[q] = (1 - s) * (1 - u) * pv[0][q] + s * (1 - u) * pv[1][q] + s * u * pv[2][q] + (1 - s) * u * pv[3][q];
                wgt = S.gfw[i] * S.gfw[jj] * area;
            }
            double xi[3];
            for (int q = 0; q < 3; ++q)
                xi[q] = Ji[q][0] * (xp[0] - x0[0]) + Ji[q][1] * (xp[1] - x0[1]) + Ji[q][2] * (xp[2] - x0[2]);
            if (d == 2) xi[2] = 0.0;
            double phi[kNmax];
            for (int kk = 0; kk < N; ++kk)
                phi[kk] = ipow(xi[0], S.ex[kk][0]) * ipow(xi[1], S.ex[kk][1]) * ipow(xi[2], S.ex[kk][2]) - mean0[kk];
            const int q = f * S.nfp + al;
            for (int m = 0; m < M; ++m) {
                double s = 0.0;
                for (int kk = 0; kk < N; ++kk) s += phi[kk] * P[kk * M + m];
                L[l_index(q, m, nf * S.nfp, M, S.lcw)] = s;   // block padded to 16 bytes
            }
            for (int kk = 0; kk < d; ++kk) O.Phil[(q0 - O.qbase + q) * d + kk] = phi[kk];
            O.W[q0 - O.qbase + q] = wgt;
        }
    }

    // 6. OI from the moments: D^beta psi_k = coef * monomial
    {
        double* OI = &O.OI[(c - O.cbase) * (int64_t)(N * (N + 1) / 2)];
        for (int k = 0; k < N; ++k)
            for (int l = k; l < N; ++l) {
                double s = 0.0;
                for (int b0 = 0; b0 <= r; ++b0)
                    for (int b1 = 0; b0 + b1 <= r; ++b1)
                        for (int b2 = 0; b0 + b1 + b2 <= r; ++b2) {
                            if ((d == 2 && b2 > 0) || b0 + b1 + b2 == 0) continue;
                            int bb[3] = {b0, b1, b2};
                            double cf = 1.0;
                            int e[3];
                            bool zero = false;
                            for (int q = 0; q < 3 && !zero; ++q) {
                                int ek = S.ex[k][q], el = S.ex[l][q];
                                if (ek < bb[q] || el < bb[q]) { zero = true; break; }
                                for (int z = 0; z < bb[q]; ++z) cf *= (double)(ek - z) * (double)(el - z);
                                e[q] = ek + el - 2 * bb[q];
                            }
                            if (zero) continue;
                            s += cf * mom[moment_index(d, e[0], e[1], e[2])];
                        }
                OI[k * N - k * (k - 1) / 2 + (l - k)] = s;
            }
    }

    // 7. degree-1 pseudo-inverses: directional stencils (D) and the MUSCL
    //    stencil (G, the first Md central cells), from the saved linear block
    double Ad[8 * 3], dg[3], bt[3], xx[3], yy[8];
    for (int f = 0; f <= nf; ++f) {
        const bool muscl = f == nf;
        const int cnt = muscl ? Md : S.nd[c * 6 + f];
        const uint8_t* idx = muscl ? nullptr : &S.dir[(c * 6 + f) * Md];
        for (int b = 0; b < cnt; ++b)
            for (int k = 0; k < d; ++k) Ad[b * 3 + k] = Alin[muscl ? b : idx[b]][k];
        auto atd = [&](int m, int k) -> double& { return Ad[m * 3 + k]; };
        if (!householder(atd, cnt, d, dg, bt)) return false;
        double* out = muscl ? &O.G[(c - O.cbase) * (int64_t)d * Md] : &O.D[(((c - O.cbase) * 6 + f) * (int64_t)d) * Md];
        for (int b = 0; b < Md; ++b) {
            if (b < cnt) {
                pinv_column(atd, cnt, d, dg, bt, b, xx, yy);
                for (int k = 0; k < d; ++k) out[k * Md + b] = xx[k] * Vr[muscl ? b : idx[b]];
            } else {
                for (int k = 0; k < d; ++k) out[k * Md + b] = 0.0;
            }
        }
    }
    return true;
}

}  // namespace hfv
