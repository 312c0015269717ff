// hfv_internal.h -- host-side structures of libhfv shared by its translation
// units (mesh ingestion, operator setup, hot path, C ABI).
#pragma once

#include <cstdint>
#include <string>
#include <vector>

#include "../../include/hfv.h"

namespace hfv {

constexpr int kMaxFaces = 6;   // hexahedron
constexpr int kDtSlots = 64;   // atomic slots per problem of the chained time-step minimum
constexpr int kDtStride = 16;  // doubles between slots: each slot on its own 128-byte line
constexpr int kMaxFaceVerts = 4;
constexpr int kMaxOrder = 5;   // r <= 4

// local face -> local vertices, listed so that the area vector points out of
// the cell (edges of counter-clockwise polygons; hexahedron faces so that
// (v2 - v0) x (v3 - v1) is outward)
int type_nverts(int t);
int type_nfaces(int t);
int face_nverts(int t, int f);
// 0: 2D or all hexahedra, 1: all tetrahedra, 2: any other 3D mix of
// tetrahedra, prisms, pyramids and hexahedra
int element_family(const hfv_mesh* m);
int type_face_vertex(int t, int f, int k);

void set_error(const std::string& msg);

}  // namespace hfv

struct hfv_mesh {
    int dim = 0;
    int64_t nn = 0, nc = 0, nface = 0;
    std::vector<double> xyz;        // [nn][3], z = 0 in 2D
    std::vector<uint8_t> type;      // [nc]
    std::vector<int64_t> cptr;      // [nc+1]
    std::vector<int32_t> cidx;
    double period[3] = {0, 0, 0};
    // per cell-face, [nc][6]
    std::vector<int32_t> nbr;       // neighbour or -1
    std::vector<int8_t> nbrf;       // neighbour's local face or -1
    std::vector<int8_t> nshift;     // [nc][6][3] periods added to the neighbour's coordinates
    std::vector<uint8_t> own;       // 1 when this cell owns the face (smaller id, or boundary)
    std::vector<double> fnorm;      // [nc][6][3] unit normal, outward from this cell (owner's, negated on the other side)
    std::vector<double> farea;      // [nc][6]
    // per cell
    std::vector<double> vol;        // [nc]
    std::vector<double> vmean;      // [nc][3] vertex mean
    // independent problems of a batch: cells seg_off[k] .. seg_off[k+1] - 1
    // form problem k (one segment for a single mesh)
    std::vector<int64_t> seg_off;
};

// ---------------------------------------------------------------------------
// device-resident scheme (pointers into one arena), see scheme.cu
// ---------------------------------------------------------------------------
struct hfv_dev_arrays {
    // topology / geometry (always present)
    int32_t* sten;     // [nc_pad][M] (rows past nc are zero)
    int32_t* nbr;      // [nc][6]
    int8_t* nbrf;      // [nc][6]
    int32_t* nfs;      // [nc][6] FS point offset of the neighbour's matching face, -1 on open boundaries,
                       // -2 past the cell's last face
    uint8_t* nfc;      // [nc] faces per cell | (distinct face neighbours << 4)
    int64_t* qoff;     // [nc+1] offsets of face points: c * (max faces * points per face)
    int64_t* loff;     // [nc_pad+1] element offsets of the per-cell L blocks (16-byte padded)
    uint8_t* dir;      // [nc][6][Md] local stencil index of directional cells
    // per precision (T = double or float), stored as void*
    void* L;           // cell c at loff[c], layout [Q_c][M], blocks padded to 16 bytes
    void* P;           // [nc][N][M]
    void* Phil;        // cell c at d*qoff[c], layout [Q_c][d]
    void* OI;          // [nc][N*(N+1)/2] packed upper triangle, row-major
    void* D;           // [nc][6][d][Md]
    void* G;           // [nc][d][Md]
    void* W;           // [qoff]: face point weight * |S|
    void* nrm;         // [nc][6][3]: outward unit normal (owner's, negated on the other side)
    void* ivol;        // [nc]: 1/|V|
    void* dxthr;       // [nc]: deactivation threshold (kappa dx)^n
    // FP64 extras for the time step
    double* vol;       // [nc]
    double* area;      // [nc][6]
    double* nrm64;     // [nc][6][3]
    // scratch of the residual
    void* FS;          // [qoff][nv] face-point states
    uint8_t* raw;      // [nc] raw class | 0x80 when the linear candidate breaks the Harten bound
    uint8_t* cls;      // [nc] final class
    int32_t* queue;    // [2][nc] CWENOZ / MUSCL queues
    int32_t* counts;   // [2] queue lengths (CWENOZ, MUSCL)
    int* status;       // [1]
    // time stepping scratch
    double* U1;        // [nv][nc]
    double* U2;        // [nv][nc]
    void* Rs;          // [nv][nc] residual of a stage (precision T)
    void* UA;          // [nc][P] cell-major copy of the stage state in the residual precision, P = 4 (2D) / 8 (3D)
    void* UB;          // second stage copy: stages alternate UA / UB
    void* areaT;       // [nc][6] face areas in the residual precision
    double* U3;        // SSP-RK(5,4) stages u_3, u_4 and the partial sum of u_5 (else null)
    double* U4;
    double* U5;
    double* dt;        // [nseg] time step per problem
    double* dt_next;   // [nseg][kDtSlots] the next step's time step (chained steps; bits of positive doubles)
    int32_t* seg;      // [nc] problem of each cell (batched meshes; null for one problem)
    double* Uio;       // [nv][nc] device state of hfv_advance_host
    // viscous terms (mu0 > 0 only, else null)
    void* VX;          // [nc][d + d d] mean of xi over the cell, then J^-1 row by row
    void* LINV;        // [nc][6] 1 / distance between the cell's and the face neighbour's vertex means (0: none)
    void* GS;          // [qoff][d + 1][d] face-point gradients of the velocity components and of T
};

namespace hfv {
// hot-path kernel ids for the optional per-kernel timer (KID_COUNT, KID_SCAN and
// KID_SCATTER are kept for the numbering only: tagging does the queue compaction)
enum KernelId { KID_LINEAR, KID_TAG, KID_COUNT, KID_SCAN, KID_SCATTER, KID_CWENO, KID_MUSCL, KID_FLUX, KID_RK,
                KID_DT, KID_CVT, KID_GRAD, KID_VJP_FLUX, KID_VJP_RECON, KID_VJP_GATHER, KID_COUNT_ALL };
struct KernelTimer {
    bool on = false;
    std::vector<void*> ev;          // cudaEvent_t pairs
    std::vector<int> kid;           // kernel id of each pending pair
    int used = 0;
    double ms[16] = {0};
    int64_t n[16] = {0};
};
void note_launch();
}  // namespace hfv

// scratch of the residual's vector-Jacobian product (adjoint.cu), allocated
// on its first use
struct hfv_adjoint_arrays {
    void* base = nullptr;
    double* MU = nullptr;       // [qtot][nv] adjoint of the face-point states
    double* A = nullptr;        // [nc][M][nv] contributions to the stencil cells
    double* S0 = nullptr;       // [nc][nv] contributions to the cell itself
    int64_t* inv_ptr = nullptr; // [nc+1] inverse stencil map (CSR, ascending (c, m))
    int32_t* inv_idx = nullptr; // [nc*M] entries c * M + m
    // [nv][nc] each: stage states, scaled adjoint, VJP result, stage adjoint
    // (hfv_step_classes / hfv_step_vjp)
    double* X1 = nullptr;
    double* X2 = nullptr;
    double* T = nullptr;
    double* G = nullptr;
    double* L2 = nullptr;
};

struct hfv_scheme {
    hfv::KernelTimer timer;
    hfv_mesh* mesh = nullptr;
    hfv_scheme_params p{};
    int r = 0, d = 0, nv = 0, N = 0, M = 0, Md = 0, nq = 0, nfp = 0;
    int fam = 0;                    // element family (element_family)
    int nfmax = 4;                  // face slots per cell: 4 (2D, tetrahedra) or 6
    int64_t qtot = 0;
    int64_t nc_pad = 0;             // cells rounded up to a multiple of 192 (bulk-copy tiles of 8-64 or 48 cells)
    int64_t ltot = 0;               // elements of L
    std::vector<int64_t> loff;      // [nc_pad+1]
    int nblocks = 0;
    int nseg = 1;                   // independent problems in the mesh
    // launch shape of the residual's kernels (hfv_autotune): resident CTAs per
    // SM of the candidate kernel (0 = as many as fit), blocks per SM of the
    // CWENOZ / MUSCL kernel and the percentage of them on the CWENOZ queue
    int tune_linear_per_sm = 0;
    int tune_linear_tile = 0;          // 0: the default tile shape, 1: the alternative (linear_tiles = 2)
    int linear_tiles = 1;              // tile shapes built for this scheme's configuration
    int tune_nl_per_sm = 16;
    int tune_nl_cweno_pct = 75;
    int sms = 152, linear_per_sm_max = 1;   // filled at the first residual
    // chained steps (step_chain): the stage copy UA and dt_next hold the step
    // after the last hfv_step on chain_U (same mode and CFL number)
    // candidate kernel's consumer wait limit and the copy-withholding switch
    // of hfv_debug_wait
    double setup_ms[2] = {0.0, 0.0};   // stencils (host), operators (device) of hfv_scheme_create
    uint64_t wait_ns = 2000000000ull;
    int withhold_copies = 0;
    bool chain_ok = false, chain_fixed = false;
    const double* chain_U = nullptr;
    double chain_cfl = 0.0;
    // host copies kept for introspection
    std::vector<int32_t> sten;      // [nc][M]
    std::vector<int8_t> sshift;     // [nc][M][3]
    std::vector<uint8_t> dir;       // [nc][6][Md]
    std::vector<uint8_t> nd;        // [nc][6]
    std::vector<uint8_t> n1;        // [nc] distinct face neighbours = the stencil's first layer
    std::vector<int64_t> qoff;      // [nc+1]
    void* arena = nullptr;
    size_t arena_bytes = 0;
    // side stream and fork / join events of hfv_step_many
    void* side = nullptr;
    void* ev_fork = nullptr;
    void* ev_join = nullptr;
    hfv_dev_arrays a{};
    hfv_adjoint_arrays adj{};
};

namespace hfv {
int build_stencils(hfv_scheme* s);       // host, scheme.cpp
int build_operators(hfv_scheme* s, void* stream);  // device FP64 setup, setup.cu
int launch_residual(hfv_scheme* s, const void* U, void* R, const uint8_t* forced, uint8_t* cls_out, void* stream);
int launch_dt(hfv_scheme* s, const double* U, double cfl, double* dt_dev, void* stream);
int launch_step(hfv_scheme* s, double* U, double cfl, double dt, void* stream);
int launch_vjp(hfv_scheme* s, const double* U, const uint8_t* cls, const double* lam, double* g, void* stream);
int launch_step_classes(hfv_scheme* s, const double* U, double dt, uint8_t* cls, int forced, double* out, void* stream);
int launch_step_vjp(hfv_scheme* s, const double* U, const uint8_t* cls, double dt, double* lam, void* stream);
void adjoint_free(hfv_scheme* s);
}  // namespace hfv
