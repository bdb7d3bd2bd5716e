// Internal declarations of libhdg: the handle, reference-element tables,
// skeleton connectivity and the per-configuration kernel launchers.
#pragma once

#include <cstdint>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/hdg.h"

namespace hdg {

constexpr int ipow(int b, int e) { return e == 0 ? 1 : b * ipow(b, e - 1); }

// Compile-time sizes of one (dimension, degree) configuration.
template <int D_, int P_>
struct Cfg {
    static constexpr int D = D_, P = P_;
    static constexpr int M = D + 2;
    static constexpr int N1 = P + 1, Q1 = P + 2;
    static constexpr int NP = ipow(N1, D), NQ = ipow(Q1, D);
    static constexpr int NF = 2 * D;
    static constexpr int NFP = ipow(N1, D - 1), NFQ = ipow(Q1, D - 1);
    static constexpr int NU = M * NP;            // interior u unknowns
    static constexpr int NQV = D * M * NP;       // interior q unknowns
    static constexpr int NT = NF * M * NFP;      // element trace unknowns
    static constexpr int NR = NU + NT;           // rows of the bordered matrix
    static constexpr int NC = NU + NT + 1;       // columns (+ right-hand side)
    static constexpr int LD = (NC + 3) & ~3;     // padded row stride
    static constexpr int BS = M * NFP;           // BSR block size
    static constexpr int NCOEF = 1 + D + NF;     // coefficients per (a, b, r, point)
};

// Reference-element tables of one configuration (host, FP64).
struct RefTables {
    int d = 0, p = 0, Np = 0, Nq = 0, nf = 0, Nfp = 0, Nfq = 0;
    std::vector<double> nodes1, gq1, gw1;           // 1-D GLL nodes, Gauss points / weights
    std::vector<double> phi, dphi, wq;              // [Nq][Np], [d][Nq][Np], [Nq]
    std::vector<double> mu, wf;                     // [Nfq][Nfp], [Nfq]
    std::vector<int32_t> fnode;                     // [nf][Nfp]
    std::vector<int32_t> node_face;                 // [Np][d]: f*Nfp + l, or -1
    std::vector<double> mhat, mf;                   // [Np][Np], [Nfp][Nfp]
    std::vector<double> minv_c, minv_e;             // [d][Np][Np], [nf][Np][Nfp]
    std::vector<double> psi, theta;                 // [d][Nq][Np], [nf][Nq][Nfp]
    std::vector<double> psi_f, theta_f;             // [nf][d][Nfq][Np], [nf][nf][Nfq][Nfp]
    std::vector<double> b1, d1;                     // [p+2][p+1] 1-D basis values / derivatives at Gauss points
};
void build_ref_tables(int d, int p, RefTables& t);

// Skeleton connectivity (host).
struct Skeleton {
    int64_t n_faces = 0;
    std::vector<int32_t> f2e, f2lf;                 // [F][2]
    std::vector<int32_t> e2f;                       // [E][nf]
    std::vector<int32_t> perm, iperm;               // [E][nf][Nfp] local->canonical, inverse
    std::vector<int32_t> rowptr, col;               // BSR pattern
    std::vector<int32_t> blk, rank;                 // [E][nf][nf]: BSR block, contribution rank
    std::vector<int32_t> frank;                     // [E][nf]: rank of the element on the face
};
int build_skeleton(const hdg_mesh& mesh, int p, Skeleton& s, std::string& err);
int build_vertex_map(const hdg_mesh& mesh, std::vector<int32_t>& ev, std::vector<int32_t>& vrow,
                     std::vector<int32_t>& vcol, std::string& err);

// Physical and numerical parameters seen by the kernels.
struct Phys {
    double gamma, re, pr, mach, tau;
    int visc_law;
    double c1, s;
    int tau_mode = 0;     // 0: constant tau; 1: state-dependent tau(uhat) = |v.n| + c + mu / h
};

struct DeviceTables {
    double* phi;  double* dphi; double* wq;
    double* mu;   double* wf;
    int32_t* fnode; int32_t* node_face;
    double* mhat; double* mf;
    double* minv_c; double* minv_e;
    double* psi; double* theta; double* psi_f; double* theta_f;
    double* b1; double* d1;          // 1-D tables of the tensor-product basis (sum factorisation)
    float* fb1; float* fd1;
    // float copies for the mixed form's FP32 contraction
    float* fphi; float* fdphi; float* fpsi; float* ftheta; float* fpsi_f; float* ftheta_f; float* fmu; float* fmf;
};

namespace tet { struct Ctx; }
}  // namespace hdg

struct hdg_ctx {
    hdg::tet::Ctx* tet = nullptr;          // tetrahedral handles (hdg_create_tet), else NULL
    int d = 0, p = 0;
    int m = 0, Np = 0, Nq = 0, nf = 0, Nfp = 0, Nfq = 0;
    int NU = 0, NQV = 0, NT = 0, NR = 0, NC = 0, LD = 0, BS = 0, NCOEF = 0;
    int64_t E = 0, F = 0, nnzb = 0;
    bool device = false;
    hdg::Phys phys{};
    int precision = HDG_PREC_FP64;
    int prec_req = HDG_PREC_FP64;          // precision as requested through hdg_set_params
    cudaStream_t stream = nullptr;
    std::string err;

    hdg::RefTables ref;
    hdg::Skeleton sk;
    std::vector<double> detJ, Jinv, NW;    // [E], [E][d][d], [E][nf][d]
    std::vector<double> centroid;          // [E][3] vertex means (mesh partitioning)

    // device memory
    std::vector<void*> allocs;
    int64_t device_bytes = 0;
    hdg::DeviceTables tab{};
    double* d_geo = nullptr;               // [E][1 + d*d + nf*d]
    int32_t* d_e2f = nullptr;
    int32_t* d_perm = nullptr;
    int32_t* d_iperm = nullptr;
    int32_t* d_rowptr = nullptr;
    int32_t* d_col = nullptr;
    int32_t* d_blk = nullptr;
    int32_t* d_rank = nullptr;
    int32_t* d_frank = nullptr;
    double* d_vals = nullptr;              // [nnzb][BS][BS]
    double* d_g = nullptr;                 // [F][m][Nfp]
    double* d_top = nullptr;               // [E][NU][LD] bordered matrix, interior rows
    double* d_bot = nullptr;               // [chunk][NT][LD] bordered matrix, trace rows
    double* d_vcoef = nullptr;             // [chunk][m][m][d][NCOEF][Nq]
    double* d_fcoef = nullptr;             // [chunk][nf][m][m][NCOEF][Nfq]
    double* d_dq0 = nullptr;               // [E][d][m][Np]
    double* d_taup = nullptr;              // [chunk][nf][Nfq] per-point tau (state-dependent stabilization)
    void* d_skout = nullptr;               // caller's [E][t][t] buffer for the element Schur complements, or NULL
    int32_t* d_ozexp = nullptr;            // [chunk][2][NT] row / column scale exponents of the tensor-core
                                           // FP64 Schur product
    int32_t* d_status = nullptr;           // [1]
    int32_t* d_ftag = nullptr;             // [E][nf] boundary tags, NULL for fully periodic meshes
    double* d_ub = nullptr;                // [m] state of tag-1 boundary faces
    double* d_ubf = nullptr;               // [F][m][Nfp] nodal tag-1 data (hdg_set_bc_field), or NULL
    double e_wall = 0.0;                   // c_v T_w of tag-3 (isothermal wall) faces
    bool has_tag[5] = {};                  // boundary kinds present in the mesh
    bool tw_set = false;
    double* ubf_store = nullptr;           // owned copy of the nodal tag-1 data
    std::vector<int32_t> ftag;             // host copy of the tags
    bool ub_set = false;
    bool has_bnd = false;
    int32_t* d_f2e = nullptr;              // [F][2]
    int32_t* d_f2lf = nullptr;             // [F][2]
    double* d_rk = nullptr;                // [E][NT] element contributions to R_uhat
    double* d_part = nullptr;              // [E + F] partial sums of squares
    double* d_norms = nullptr;             // [3]
    // block-Jacobi factors (allocated on first set-up)
    double* d_bjlu = nullptr;              // [F][BS][BS] inverses of the diagonal blocks (column-major;
                                           // FP32 values for the mixed system)
    int bj_prec = HDG_PREC_FP64;
    bool bj_ready = false;
    // additive Schwarz factors on element face patches (allocated on first set-up)
    void* d_asmlu = nullptr;               // [E][NT][LDA] LU factors of S_r (FP64, or FP32 for the mixed form)
    int32_t* d_asmpiv = nullptr;           // [E][NT]
    double* d_asmz = nullptr;              // [E][NT] patch corrections
    int32_t* d_asmperm = nullptr;          // [E][NT] row permutation of each patch as a gather map
    void* d_asmdinv = nullptr;             // [E][NBLK][2][32][32] inverses of the diagonal blocks of L and U
    size_t asm_bytes = 0;
    int asm_prec = -1;                     // precision of the stored factors
    bool asm_ready = false;
    int pc_kind = HDG_PC_BLOCKJACOBI;      // preconditioner of GMRES and Newton
    // GMRES workspace (allocated on first use)
    double* d_V = nullptr;                 // [restart + 1][N]
    double* d_w = nullptr;                 // [N]
    double* d_red = nullptr;               // [kRedBlocks]
    double* d_mred = nullptr;              // [(restart + 8) / 8][kRedBlocks][8] Gram-Schmidt partials
    double* d_h = nullptr;                 // [restart + 2]
    int gm_cap = 0;
    double* d_nw = nullptr;                // Newton work: dU, dQ, dUH, g
    // artificial-viscosity smoothing: master vertex of every corner and vertex -> element lists
    std::vector<int32_t> av_ev, av_vrow, av_vcol;
    int32_t* d_avev = nullptr;             // [E][2^d]
    int32_t* d_avvrow = nullptr;           // [V + 1]
    int32_t* d_avvcol = nullptr;           // [E * 2^d]
    double* d_avv = nullptr;               // [V] vertex field
    double* d_ave = nullptr;               // [E] elemental field
    double* d_diag = nullptr;              // [E][4] diagnostic partial integrals, then [4] totals
    // reduced-basis initial guess: window of accepted trace corrections and their products
    double* d_rbW = nullptr;               // [rb_max][N]
    double* d_rbZ = nullptr;               // [rb_max][N]
    double* d_rbpart = nullptr;            // [kRbBlocks][256] Gram partial sums
    double* d_rbc = nullptr;               // [rb_max] coefficients
    int* d_rbhead = nullptr;               // [2]: next slot, columns stored
    int rb_max = 0;
    // synchronisation-free Newton / DIRK driver and its CUDA graph
    double* d_fx = nullptr;                // device GMRES scalars: beta, R, cs, sn, y, g
    int fx_cap = 0;
    double* d_hist = nullptr;              // [4096] residual history
    int* d_hcount = nullptr;
    double* d_dirk = nullptr;              // U^n, U*, stage states
    int dirk_cap = 0;
    cudaStream_t gstream = nullptr;
    cudaGraphExec_t gexec = nullptr;
    uint64_t gkey = 0;
    // mixed form (allocated on the first mixed linearization)
    int sys_prec = HDG_PREC_FP64;          // precision of the assembled system
    int schur_mode = 0;                    // mixed Schur product: 0 FP32 SIMT, 1 TF32, 2 3xTF32 tensor cores
    int blocks_mode = 1;                   // mixed volume contraction: 0 FP32 SIMT, 1 3xTF32 tensor cores (3-D),
                                           // 2 FP32 sum factorisation
    int blocks64_mode = 1;                 // FP64 volume contraction: 0 dense GEMM, 1 sum factorisation
    int schur64_mode = 0;                  // FP64 Schur product: 0 inside the FP64 elimination, 1 on the BF16
                                           // tensor cores by exact digit splitting (k_schur_ozaki)
    double* d_m11 = nullptr;               // [E][NU][NU] interior block / its LU factors (FP64)
    float* d_m12 = nullptr;                // [E][NU][NT] Bt, then Z = L^{-1} P Bt
    double* d_mrt = nullptr;               // [E][NU] Rt, then z
    float* d_m21 = nullptr;                // [chunk][NT][NU] Ct, then W
    float* d_m22 = nullptr;                // [chunk][NT][NT] Dt, then S^K
    double* d_mrb = nullptr;               // [chunk][NT] Rh, then -g^K
    int32_t* d_mpiv = nullptr;             // [E][NU] interchanges of the interior LU (split elimination)
    float* d_vals32 = nullptr;             // [nnzb][BS][BS] condensed blocks (FP32)
    float* d_x32 = nullptr;                // [F][BS] FP32 copy of a matvec operand
    int64_t chunk = 0;
    bool have_system = false;
    int elim_minb = 2;                     // k_elim variant: resident CTAs per SM the kernel is built for
    int elim_nb = 16;                      // k_elim variant: panel width (16 or 8)
    int elim_mixed_minb = 2;               // k_elim_mixed variant: resident CTAs per SM (2 or 3)
    int elim_mixed_split = 0;              // mixed elimination: 0 fused kernel, 1 FP64 LU + FP32 triangular solves

    // instrumentation: event pairs around kernel launches
    bool prof = false;
    std::vector<cudaEvent_t> ev_pool;
    std::vector<int> ev_kind;        // kernel class of each recorded pair
    size_t ev_used = 0;              // events in use (2 per pair)
    int64_t launches[HDG_NK] = {};
    double ms_acc[HDG_NK] = {};
};

namespace hdg {
// Records a CUDA event on the handle's stream before (begin) / after (end) a
// launch of kernel class `kind` when profiling is on; counts launches always.
void prof_begin(hdg_ctx* h, int kind);
void prof_end(hdg_ctx* h);
// Launchers, one instantiation per (d, p), defined in kern_*.cu.
struct LinArgs {
    const double* U; const double* Q; const double* UH; const double* Ustar; const double* nu;
    double dt, a_ii;
};
template <int D, int P> int run_linearize(hdg_ctx* h, const LinArgs& a);
template <int D, int P> int run_matvec(hdg_ctx* h, const double* x, double* y);
template <int D, int P> int run_recover(hdg_ctx* h, const double* dUH, double* dQ, double* dU);
template <int D, int P> int run_residual(hdg_ctx* h, const LinArgs& a, double* Rq, double* Ru, double* Ruh);
// Allocates, on first use, the per-element storage of the FP64 or the mixed
// system (BSR values, interior rows, per-chunk trace rows); no-op afterwards.
int ensure_system_storage(hdg_ctx* h, int precision);
template <int D, int P> int run_asm_setup(hdg_ctx* h);
template <int D, int P> int run_asm_apply(hdg_ctx* h, const double* x, double* y);
template <int D, int P> int run_av_field(hdg_ctx* h, const double* U, const double* Q, double c_av, double h_m,
                                         double s_max, double* nu);
template <int D, int P> int run_diagnostics(hdg_ctx* h, const double* U, const double* Q);
template <int D, int P> int run_lift(hdg_ctx* h, const double* U, const double* UH, double* Q);
template <int D, int P> int run_linearize_mixed(hdg_ctx* h, const LinArgs& a);
template <int D, int P> int run_bj_setup(hdg_ctx* h);
template <int D, int P> int run_bj_apply(hdg_ctx* h, const double* x, double* y);
}  // namespace hdg
