// Tetrahedral elements of per-element degree on quadratic geometry: host data
// of a tetrahedral handle and the device descriptors of its kernels.
//
// Element space: total degree p_K (1..4) on each tetrahedron, nodal Lagrange
// basis on the equispaced lattice; trace space of a face: total degree
// p_F = max(p_L, p_R) on the face's canonical frame (vertices in ascending
// master id); collapsed Gauss-Jacobi rules with p + 2 points per collapsed
// direction (element) and p_F + 2 (face), face points placed in the canonical
// frame; isoparametric quadratic geometry (Sec. 2.2 spaces, Sec. 4 workloads).
#pragma once

#include <cstdint>
#include <string>
#include <vector>

#include "common.h"

namespace hdg {
namespace tet {

constexpr int M = 5;            // conserved variables in 3-D
constexpr int PMAX = 4;
constexpr int NPMAX = 35;       // (PMAX+1)(PMAX+2)(PMAX+3)/6
constexpr int NQMAX = 216;      // (PMAX+2)^3
constexpr int NFPMAX = 15;      // (PMAX+1)(PMAX+2)/2
constexpr int NFQMAX = 36;      // (PMAX+2)^2
constexpr int NCODE = 24;       // 4 local faces x 6 orderings of their vertices

inline int n_tet(int p) { return (p + 1) * (p + 2) * (p + 3) / 6; }
inline int n_tri(int p) { return (p + 1) * (p + 2) / 2; }

// Reference tables (host, FP64).
struct VolTab { int p, Np, Nq; std::vector<double> xq, wq, phi, dphi; };   // phi [Nq][Np], dphi [3][Nq][Np]
struct TriTab { int p, Nfp, Nfq; std::vector<double> xs, ws, mu; };       // mu [Nfq][Nfp]
void build_vol(int p, VolTab& t);
void build_tri(int p, TriTab& t);
// element basis of degree p at the canonical points of a face of degree pF
// with face code c (= 4-face index * 6 + ordering): phif [Nfq][Np]; the
// outward reference area normal nu [3]
void build_face(int p, int pF, int code, std::vector<double>& phif, double nu[3]);
// local vertices (L0, L1, L2) of face code c
void code_vertices(int code, int L[3]);

// One element's sizes and offsets, as the kernels read them.
struct TetElem {
    int32_t p, Np, Nq, NU, t, LD, curved, sfq;   // sfq: sum of face rule points
    int32_t pf[4], code[4], tag[4], toff[4], nfp[4], nfq[4], soff[4];
    int64_t face[4];
    int64_t hoff[4];   // trace offsets of the four faces
    int64_t uoff;      // U offset (Q offset is 3 uoff)
    int64_t moff;      // bordered matrix [NU + t][LD]
    int64_t roff;      // recovery data: G [3][Np][Np], H [3][Np][sum nfp], dq0 [3][m][Np]
    int64_t goff;      // curved: volume records [Nq][10] (w |J|, J^{-1} row-major [r][k])
    int64_t gfoff;     // curved: face records [sfq][3] (w_s |J| J^{-T} nu)
    int64_t koff;      // element trace residual R_uhat^K [t] (residual evaluation)
    int32_t vtab, ftab[4], ttab[4], pad;   // table offsets: volume, face (p, pF, code), trace (pF)
    double detJ, Jinv[9];                  // affine elements
    double hinv;                           // |K|^{-1/3} (state-dependent stabilization)
};

struct Ctx {
    int64_t E = 0, F = 0, nnzb = 0;
    int64_t n_u = 0, n_trace = 0, n_vals = 0, n_mat = 0, n_rec = 0, n_curved = 0;
    std::vector<int32_t> elem_p, face_p, e2f, f2e, f2lf, frame, tags;
    std::vector<int64_t> uoff, hoff, boff;
    std::vector<int32_t> rowptr, col;
    std::vector<int32_t> cptr, centry;     // contributions of each block: (e, fl, gl) ascending e
    std::vector<int32_t> diagb;            // [F] index of the diagonal block of each block row
    std::vector<int64_t> bjoff;            // [F+1] offsets of the diagonal-block inverses (bs_F^2 each)
    int64_t n_rk = 0;                      // sum of element trace sizes
    std::vector<TetElem> el;
    std::vector<int32_t> order;            // elements by decreasing cost
    std::vector<double> tab;               // all tables
    std::vector<int32_t> vtab, ttab, ftab; // offsets: [p], [pF], [(p * 5 + pF) * 24 + code]
    std::vector<double> gvol, gface;       // curved geometry records
    bool has_tag[5] = {};
    // device
    TetElem* d_el = nullptr;
    int32_t* d_order = nullptr;
    double* d_tab = nullptr;
    float* d_tabf = nullptr;               // FP32 copy of the tables (mixed-form contraction)
    double* d_gvol = nullptr;
    double* d_gface = nullptr;
    int64_t* d_hoff = nullptr;
    int64_t* d_boff = nullptr;
    int32_t* d_rowptr = nullptr;
    int32_t* d_col = nullptr;
    int32_t* d_rw = nullptr;               // [F] block-row widths (summed column-face sizes)
    int32_t* d_cptr = nullptr;
    int32_t* d_centry = nullptr;
    int32_t* d_f2e = nullptr;
    int32_t* d_f2lf = nullptr;
    double* d_mat = nullptr;               // per-element bordered matrices
    double* d_rec = nullptr;               // per-element recovery data
    double* d_vals = nullptr;              // assembled blocks (FP64 form)
    float* d_vals32 = nullptr;             // assembled blocks of the mixed form (allocated on first use)
    float* d_bj32 = nullptr;               // block-Jacobi inverses of the mixed form
    int sys_prec = HDG_PREC_FP64;          // precision of the assembled system
    int nb = 16;                           // elimination panel width (autotuned: 16 or 8)
    int bsmax = 0, wmax = 0;               // largest block size and block-row width
    double* d_g = nullptr;                 // [n_trace]
    double* d_work = nullptr;              // per-CTA workspace
    int32_t* d_diagb = nullptr;
    int64_t* d_bjoff = nullptr;
    double* d_bj = nullptr;                // block-Jacobi inverses (allocated on first set-up)
    double* d_rk = nullptr;                // element trace residuals (allocated on first residual)
    double* d_part = nullptr;              // [E + F] partial sums of squares
    bool bj_ready = false;
    int32_t* d_next = nullptr;             // work counter of the persistent launch
    int n_slots = 0;
    int64_t work_stride = 0;
    bool have_system = false;
    // additive Schwarz on element face patches (allocated on the first set-up)
    int64_t* d_aoff = nullptr;             // [E + 1] offsets of the patch factors, [t][LDA] each, LDA = t rounded to 4
    int64_t* d_poff = nullptr;             // [E + 1] offsets of the patch vectors, t each
    double* d_asm = nullptr;               // LU factors of the patches (FP64 system)
    float* d_asm32 = nullptr;              // LU factors of the patches (mixed form)
    int32_t* d_asmperm = nullptr;          // [sum t] row permutation of each patch as a gather map
    double* d_asmz = nullptr;              // [sum t] patch corrections
    int32_t* d_asmnext = nullptr;          // work counter of the set-up
    int64_t n_asm = 0, n_patch = 0;
    int64_t* d_skoff = nullptr;            // [E + 1] offsets of the element Schur complements (t^2 each)
    int asm_prec = -1;                     // precision of the stored factors
    bool asm_ready = false;
};

// Host set-up: tables, skeleton, geometry, layout; error text in err.
int create_host(hdg_ctx* h, const hdg_tet_mesh* mesh, std::string& err);
int create_device(hdg_ctx* h, std::string& err);
void destroy(hdg_ctx* h);

// Device entry points (tet.cu).
int linearize(hdg_ctx* h, const double* U, const double* Q, const double* UH, const double* Ustar, double dt,
              double a_ii);
int matvec(hdg_ctx* h, const double* x, double* y);
int recover(hdg_ctx* h, const double* dUH, double* dQ, double* dU);
// FP64 stage residual: optional outputs Rq [3 n_u], Ru [n_u], Ruh [n_trace]; the norms
// ||F||, ||(R_q, R_u)||, ||R_uhat|| go to norms (device, 3 doubles)
int residual(hdg_ctx* h, const double* U, const double* Q, const double* UH, const double* Ustar, double dt,
             double a_ii, double* Rq, double* Ru, double* Ruh, double* norms);
int bj_setup(hdg_ctx* h);
int bj_apply(hdg_ctx* h, const double* x, double* y);
// element Schur complements to the caller's buffer (packed [t_e][t_e] at offsets sum t^2)
int set_element_block_output(hdg_ctx* h, void* SK);
// additive Schwarz on element face patches (tet_schwarz.cu)
int asm_setup(hdg_ctx* h);
int asm_apply(hdg_ctx* h, const double* x, double* y);

}  // namespace tet
}  // namespace hdg
