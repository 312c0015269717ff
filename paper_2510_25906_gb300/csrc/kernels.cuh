// kernels.cuh -- compile-time configuration of the residual kernels and the
// parameter block they receive by value.
#pragma once

#include <cstdint>

#include "physics.cuh"

namespace hfv {

constexpr int cK(int r, int d) { return d == 2 ? (r + 1) * (r + 2) / 2 : (r + 1) * (r + 2) * (r + 3) / 6; }

// sizes fixed by (dimension, polynomial degree, element family): M =
// 2 K(r, d) central cells, N = K(r, d) - 1 coefficients, Md = 2 K(1, d),
// nq Gauss points per face direction: ceil((r+1)/2) on edges and on the
// quadrilaterals of hexahedral meshes, ceil((r+2)/2) per direction of the
// collapsed rule on triangles, and on every face of a mesh with triangular
// faces.  TET: 0 hexahedra, 1 tetrahedra (four faces), 2 any mix of
// tetrahedra, prisms, pyramids and hexahedra (up to six faces)
template <int D_, int R_, int TET_ = 0>
struct Cfg {
    static constexpr int D = D_;
    static constexpr int R = R_;
    static constexpr int TET = TET_;
    static constexpr int NV = D + 2;
    static constexpr int M = 2 * cK(R, D);
    static constexpr int N = cK(R, D) - 1;
    static constexpr int MD = 2 * cK(1, D);
    static constexpr int NQ = TET ? (R + 3) / 2 : (R + 2) / 2;
    static constexpr int NFP = D == 2 ? NQ : NQ * NQ;
    static constexpr int NFMAX = D == 2 ? 4 : TET == 1 ? 4 : 6;
    static constexpr int QMAX = NFMAX * NFP;
    static constexpr int NOI = N * (N + 1) / 2;
};

// lanes of the group that owns one cell: the face points rounded up to 8, 16 or 32
template <int Q>
struct GroupSize {
    static constexpr int value = Q <= 8 ? 8 : Q <= 16 ? 16 : 32;
};

enum : uint8_t { CLS_LIN = 0, CLS_CW = 1, CLS_MU = 2, CLS_FIRST = 3, HARTEN_FAIL = 0x80 };

template <class T>
struct KParams {
    int64_t nc;
    int scheme;       // HFV_HYBRID / pure
    int nad_vars;
    int forced;       // 1 when classes are given
    const uint8_t* forced_cls;
    // topology
    const int32_t* sten;
    const int32_t* nbr;
    const int8_t* nbrf;
    const uint8_t* nfc;
    const int64_t* qoff;
    const int64_t* loff;
    const int32_t* nfs;   // [nc][6] FS point offset of the neighbour's matching face (-1: open boundary,
                          // -2: no such face)
    int nv, nfp, qmax;
    const uint8_t* dir;
    // operators
    const T* L;
    const T* P;
    const T* Phil;
    const T* OI;
    const T* Dd;
    const T* G;
    const T* W;
    const T* nrm;
    const T* ivol;
    const T* dxthr;
    // state of the current stage, cell-major: cell c at UA[c * P], P = 4 (2D) or 8 (3D)
    const T* UA;
    // scratch
    T* FS;
    uint8_t* raw;
    uint8_t* cls;
    int32_t* queue;
    int32_t* counts;
    int* status;
    // Runge-Kutta stage fused into the flux kernel (rk_mode bit 0): for every
    // variable, out = rk_a U0 + rk_b (Us + c R) with the stage's step
    // c = rk_w dt (dt per problem), and the next stage's cell-major copy
    // into ua_next (may be null); R itself also into Rcopy when non-null.
    // The state is FP64.  FP64 schemes evaluate the line in FP64; FP32
    // schemes form the increment rk_bw dt R in FP32 (rk_bw = rk_b rk_w
    // rounded to FP32; R is an FP32 value) and add it with one FP64 FMA per
    // term: out = rk_a U0 + (rk_b Us + increment).  rk_mode bit 1: rk_a != 0.
    double rk_a, rk_b, rk_w;
    float rk_bw;
    int rk_mode;
    T* Rcopy;
    const double* U0;
    const double* Us;
    const double* dt;     // [problems] the step
    const int32_t* seg;   // problem of each cell, or null (one problem)
    double* out;
    T* ua_next;
    // constants
    T gamma, alpha_m, beta_m, alpha_w, beta_w, lam1, eps_cw, b_cw, h_theta, h_eps;
    int limiter;          // MUSCL: 0 Barth-Jespersen, 1 Venkatakrishnan
    T venk_k;
    // viscous terms (mu0 > 0): per cell the mean of xi and the reference map
    // J^-1 ([D + D D], xi = J^-1 (x - v0)), per cell-face 1 / L_int, and the
    // face-point gradients of the velocity and temperature [qoff][D + 1][D]
    const T* VX;
    const T* LINV;
    T* GS;
    ViscParams<T> vp;
    // limit of the candidate kernel's consumer waits (ns) and, for testing the
    // timeout path, a switch that makes its producer issue no bulk copy
    uint64_t wait_ns;
    int withhold_copies;
    // chained steps: the last stage's flux kernel also reduces the next
    // step's stable time step into dt_next (kDtSlots slots per problem, each
    // on its own 128-byte line, as bits of positive doubles for atomicMin, a
    // warp into slot (warp index) % kDtSlots so that no single line takes
    // every warp's atomic; null in
    // every other launch) from the new state, with the face areas areaT and
    // cfl; the first stage's tagging kernel of the following step reduces
    // dt_pending (the same array; null in every other launch) over the slots
    // into dt_cur and resets it
    unsigned long long* dt_next;
    unsigned long long* dt_pending;
    double* dt_cur;
    const T* areaT;
    T cfl;
    int nseg;
};

}  // namespace hfv
