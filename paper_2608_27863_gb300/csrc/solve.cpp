// Host side of the trace-space solve: FP64 stage residual, Newton update,
// block-Jacobi and additive Schwarz preconditioners, the reduced-basis guess,
// and restarted, left-preconditioned GMRES with FP64 Arnoldi (classical
// Gram-Schmidt with one reorthogonalisation; Sec. 3.2).  The Krylov
// coefficients live on the device; the host-driven solver reads back only the
// Hessenberg column of each iteration for the Givens rotations, the
// synchronisation-free one does those on the device as well.
#include <cmath>
#include <cstring>
#include <initializer_list>
#include <vector>

#include "solve.cuh"
#include "tet.h"

using namespace hdg;

namespace {

int fail(hdg_ctx* h, int code, const std::string& m) {
    h->err = m;
    return code;
}

// vector lengths of the state and trace unknowns (packed layouts on tetrahedral handles)
int64_t len_u(const hdg_ctx* h) { return h->tet ? h->tet->n_u : h->E * h->NU; }
int64_t len_q(const hdg_ctx* h) { return h->tet ? 3 * h->tet->n_u : h->E * h->NQV; }
int64_t len_t(const hdg_ctx* h) { return h->tet ? h->tet->n_trace : h->F * h->BS; }

#define CKS(call)                                                                         \
    do {                                                                                  \
        cudaError_t e_ = (call);                                                          \
        if (e_ != cudaSuccess)                                                            \
            return fail(h, e_ == cudaErrorMemoryAllocation ? HDG_ENOMEM : HDG_ECUDA,       \
                        std::string(#call) + ": " + cudaGetErrorString(e_));              \
    } while (0)

#define DISPATCH_S(FN, ...)                                                     \
    switch (h->d * 10 + h->p) {                                                  \
        case 21: rc = FN<2, 1>(__VA_ARGS__); break;                              \
        case 22: rc = FN<2, 2>(__VA_ARGS__); break;                              \
        case 23: rc = FN<2, 3>(__VA_ARGS__); break;                              \
        case 31: rc = FN<3, 1>(__VA_ARGS__); break;                              \
        case 32: rc = FN<3, 2>(__VA_ARGS__); break;                              \
        case 33: rc = FN<3, 3>(__VA_ARGS__); break;                              \
        default: rc = fail(h, HDG_EUNSUPPORTED, "unsupported (d, p)");          \
    }

int alloc(hdg_ctx* h, void** p, size_t bytes) {
    cudaError_t e = cudaMalloc(p, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(h, HDG_ENOMEM, "cudaMalloc of " + std::to_string(bytes) + " bytes failed");
    }
    h->allocs.push_back(*p);
    h->device_bytes += (int64_t)bytes;
    return HDG_OK;
}

unsigned grid_for(int64_t n) { return (unsigned)std::min<int64_t>(kRedBlocks * 4, (n + 255) / 256); }

int ensure_residual_storage(hdg_ctx* h) {
    if (h->tet) return h->d_norms ? HDG_OK : alloc(h, (void**)&h->d_norms, sizeof(double) * 4);
    if (h->d_rk) return HDG_OK;
    int rc;
    if ((rc = alloc(h, (void**)&h->d_rk, sizeof(double) * h->E * h->NT))) return rc;
    if ((rc = alloc(h, (void**)&h->d_part, sizeof(double) * (h->E + h->F)))) return rc;
    if ((rc = alloc(h, (void**)&h->d_norms, sizeof(double) * 4))) return rc;
    if ((rc = alloc(h, (void**)&h->d_f2e, sizeof(int32_t) * 2 * h->F))) return rc;
    if ((rc = alloc(h, (void**)&h->d_f2lf, sizeof(int32_t) * 2 * h->F))) return rc;
    CKS(cudaMemcpy(h->d_f2e, h->sk.f2e.data(), sizeof(int32_t) * 2 * h->F, cudaMemcpyHostToDevice));
    CKS(cudaMemcpy(h->d_f2lf, h->sk.f2lf.data(), sizeof(int32_t) * 2 * h->F, cudaMemcpyHostToDevice));
    return HDG_OK;
}

// out = ||x||_2 or x.y into the device scalar `out`
void dev_dot(hdg_ctx* h, const double* x, const double* y, int64_t n, double* out, bool sqrt_) {
    k_dot_part<<<kRedBlocks, 256, 0, h->stream>>>(x, y, n, h->d_red);
    k_dot_final<<<1, 32, 0, h->stream>>>(h->d_red, kRedBlocks, out, sqrt_ ? 1 : 0);
}

int precond_apply(hdg_ctx* h, const double* x, double* y) {
    if (h->tet) return h->pc_kind == HDG_PC_SCHWARZ ? hdg::tet::asm_apply(h, x, y) : hdg::tet::bj_apply(h, x, y);
    int rc;
    if (h->pc_kind == HDG_PC_SCHWARZ) {
        DISPATCH_S(run_asm_apply, h, x, y);
    } else {
        DISPATCH_S(run_bj_apply, h, x, y);
    }
    return rc;
}

bool precond_ready(const hdg_ctx* h) {
    if (h->tet) return h->pc_kind == HDG_PC_SCHWARZ ? h->tet->asm_ready : h->tet->bj_ready;
    return h->pc_kind == HDG_PC_SCHWARZ ? h->asm_ready : h->bj_ready;
}

int schwarz_setup(hdg_ctx* h) {
    if (h->tet) return hdg::tet::asm_setup(h);
    const int prec = h->sys_prec == HDG_PREC_MIXED ? HDG_PREC_MIXED : HDG_PREC_FP64;
    const int lda = (h->NT + 3) & ~3;
    const size_t need = (prec == HDG_PREC_MIXED ? sizeof(float) : sizeof(double)) * (size_t)h->E * h->NT * lda;
    int rc;
    const size_t nblk = (h->NT + 31) / 32;
    const size_t need_d = (prec == HDG_PREC_MIXED ? sizeof(float) : sizeof(double)) * (size_t)h->E * nblk * 2048;
    if (h->asm_bytes < need) {
        if ((rc = alloc(h, &h->d_asmlu, need))) return rc;
        if ((rc = alloc(h, &h->d_asmdinv, need_d))) return rc;
        h->asm_bytes = need;
    }
    if (!h->d_asmpiv) {
        if ((rc = alloc(h, (void**)&h->d_asmpiv, sizeof(int32_t) * h->E * h->NT))) return rc;
        if ((rc = alloc(h, (void**)&h->d_asmperm, sizeof(int32_t) * h->E * h->NT))) return rc;
        if ((rc = alloc(h, (void**)&h->d_asmz, sizeof(double) * h->E * h->NT))) return rc;
    }
    if ((rc = ensure_residual_storage(h))) return rc;       // face-to-element maps
    DISPATCH_S(run_asm_setup, h);
    if (rc) return rc;
    h->asm_prec = prec;
    h->asm_ready = true;
    return HDG_OK;
}

int precond_setup(hdg_ctx* h);
int matvec(hdg_ctx* h, const double* x, double* y);

// dUhat_0 = W c with c = argmin ||g - Z c|| over the window (eq. rb-min)
int rb_guess(hdg_ctx* h, const double* g, double* x0) {
    const int64_t N = len_t(h);
    k_rb_gram_part<<<kRbBlocks, 256, 0, h->stream>>>(h->d_rbZ, h->rb_max, g, N, h->d_rbpart);
    k_rb_solve<<<1, 256, 0, h->stream>>>(h->d_rbpart, kRbBlocks, h->rb_max, h->d_rbc);
    CKS(cudaMemsetAsync(x0, 0, sizeof(double) * N, h->stream));
    k_combine<<<grid_for(N), 256, 0, h->stream>>>(h->d_rbW, N, h->d_rbc, h->rb_max, x0, N);
    CKS(cudaGetLastError());
    return HDG_OK;
}

// insert an accepted correction w with z = S w (one trace matvec), dropping the oldest column when full
int rb_push(hdg_ctx* h, const double* w) {
    const int64_t N = len_t(h);
    int rc;
    if ((rc = matvec(h, w, h->d_w))) return rc;
    k_rb_store<<<grid_for(N), 256, 0, h->stream>>>(w, h->d_w, h->d_rbW, h->d_rbZ, h->d_rbhead, N);
    k_rb_advance<<<1, 32, 0, h->stream>>>(h->d_rbhead, h->rb_max);
    CKS(cudaGetLastError());
    return HDG_OK;
}

int matvec(hdg_ctx* h, const double* x, double* y) {
    if (h->tet) return hdg::tet::matvec(h, x, y);
    int rc;
    DISPATCH_S(run_matvec, h, x, y);
    return rc;
}

// Classical Gram-Schmidt with one reorthogonalisation (CGS2) of vn against
// V_0 .. V_j: hcol[0..j] = the projection coefficients (FP64, fixed-order
// reductions), vn orthogonalised in place.  All k dot products of a pass in one
// launch (eight basis vectors per block row of the grid) instead of one kernel
// pair per basis vector as modified Gram-Schmidt needs.
void cgs2(hdg_ctx* h, const double* V, int64_t N, int j, double* vn, double* hcol, double* htmp) {
    const int k = j + 1;
    for (int pass = 0; pass < 2; ++pass) {
        double* hp = pass == 0 ? hcol : htmp;
        k_mdot_part<<<dim3(kRedBlocks, (k + 7) / 8), 256, 0, h->stream>>>(V, N, k, vn, N, h->d_mred);
        k_mdot_final<<<(k + 3) / 4, 128, 0, h->stream>>>(h->d_mred, kRedBlocks, k, hp);
        k_msub<<<grid_for(N), 256, 0, h->stream>>>(V, N, hp, k, vn, N);
    }
    k_vadd<<<1, 64, 0, h->stream>>>(hcol, htmp, k);
}

// workspace of the synchronisation-free solver: Krylov basis, Newton work, device scalars
int ensure_fixed_workspace(hdg_ctx* h, int m) {
    const int64_t N = len_t(h);
    int rc;
    if (h->gm_cap < m) {
        if ((rc = alloc(h, (void**)&h->d_V, sizeof(double) * (size_t)(m + 1) * N))) return rc;
        if ((rc = alloc(h, (void**)&h->d_w, sizeof(double) * N))) return rc;
        if (!h->d_red && (rc = alloc(h, (void**)&h->d_red, sizeof(double) * kRedBlocks * 8))) return rc;
        if ((rc = alloc(h, (void**)&h->d_mred, sizeof(double) * kRedBlocks * 8 * ((m + 8) / 8)))) return rc;
        if ((rc = alloc(h, (void**)&h->d_h, sizeof(double) * 2 * (m + 2)))) return rc;
        h->gm_cap = m;
    }
    if (h->fx_cap < m) {
        const size_t n = 1 + (size_t)m * m + 3 * (size_t)m + 1 + (m + 1);
        if ((rc = alloc(h, (void**)&h->d_fx, sizeof(double) * n))) return rc;
        h->fx_cap = m;
    }
    if (!h->d_nw) {
        size_t n = (size_t)(len_u(h) + len_q(h) + 2 * len_t(h));
        if ((rc = alloc(h, (void**)&h->d_nw, sizeof(double) * n))) return rc;
    }
    if (!h->d_hist) {
        if ((rc = alloc(h, (void**)&h->d_hist, sizeof(double) * 4096))) return rc;
        if ((rc = alloc(h, (void**)&h->d_hcount, sizeof(int)))) return rc;
    }
    return ensure_residual_storage(h);
}

// GMRES(m) from x = 0, exactly m iterations, no host synchronisation: the Givens
// rotations and the triangular solve run on the device.
int gmres_fixed_async(hdg_ctx* h, const double* b, double* x, int m, bool use_x0) {
    const int64_t N = len_t(h);
    double* V = h->d_V;
    double* w = h->d_w;
    double* beta = h->d_fx;
    double* R = beta + 1;
    double* cs = R + (size_t)m * m;
    double* sn = cs + m;
    double* y = sn + m;
    double* gv = y + m;
    double* hc = h->d_h;
    int rc;
    if (use_x0) {                               // r0 = b - S x0
        if ((rc = matvec(h, x, w))) return rc;
        k_axpby<<<grid_for(N), 256, 0, h->stream>>>(1.0, b, -1.0, w, N);
        if ((rc = precond_apply(h, w, V))) return rc;
    } else if ((rc = precond_apply(h, b, V))) {
        return rc;
    }
    dev_dot(h, V, V, N, beta, true);
    k_set_first<<<1, 64, 0, h->stream>>>(beta, gv, m);
    k_scale_safe<<<grid_for(N), 256, 0, h->stream>>>(V, beta, V, N);
    for (int j = 0; j < m; ++j) {
        double* vj = V + (size_t)j * N;
        double* vn = V + (size_t)(j + 1) * N;
        if ((rc = matvec(h, vj, w))) return rc;
        if ((rc = precond_apply(h, w, vn))) return rc;
        cgs2(h, V, N, j, vn, hc, hc + m + 2);
        dev_dot(h, vn, vn, N, hc + j + 1, true);
        k_scale_safe<<<grid_for(N), 256, 0, h->stream>>>(vn, hc + j + 1, vn, N);
        k_givens_step<<<1, 1, 0, h->stream>>>(hc, j, m, R, cs, sn, gv);
    }
    k_backsolve<<<1, 1, 0, h->stream>>>(R, gv, m, m, y);
    if (!use_x0) CKS(cudaMemsetAsync(x, 0, sizeof(double) * N, h->stream));
    k_combine<<<grid_for(N), 256, 0, h->stream>>>(V, N, y, m, x, N);
    CKS(cudaGetLastError());
    return HDG_OK;
}

// one Newton iteration of the stage equations, asynchronous on the handle's stream;
// the residual norm before the update is appended to the device history
int newton_iteration_async(hdg_ctx* h, double* U, double* Q, double* UH, const double* Ustar, const double* nu,
                           double dt, double a_ii, int m);

}  // namespace

extern "C" {

int hdg_residual(hdg_handle h, const double* U, const double* Q, const double* UH, const double* Ustar,
                 const double* nu, double dt, double a_ii, double* Rq, double* Ru, double* Ruh, double* norms) {
    if (!h) return HDG_EINVAL;
    if (!h->device) return fail(h, HDG_EINVAL, "handle has no device storage");
    if (!U || !Q || !UH || !Ustar) return fail(h, HDG_EINVAL, "U, Q, UH and Ustar are required");
    if (!(dt > 0.0) || !(a_ii > 0.0)) return fail(h, HDG_EINVAL, "dt and a_ii must be positive");
    int rc = ensure_residual_storage(h);
    if (rc) return rc;
    if (h->tet) {
        if (nu) return fail(h, HDG_EUNSUPPORTED, "artificial viscosity is not available on tetrahedral handles");
        if ((rc = hdg::tet::residual(h, U, Q, UH, Ustar, dt, a_ii, Rq, Ru, Ruh, h->d_norms))) return rc;
    } else {
        LinArgs a{U, Q, UH, Ustar, nu, dt, a_ii};
        DISPATCH_S(run_residual, h, a, Rq, Ru, Ruh);
        if (rc) return rc;
        k_sum_parts<<<1, 256, 0, h->stream>>>(h->d_part, h->E, h->d_part + h->E, h->F, h->d_norms);
    }
    CKS(cudaGetLastError());
    if (norms) {
        double tmp[3];
        CKS(cudaMemcpyAsync(tmp, h->d_norms, sizeof(tmp), cudaMemcpyDeviceToHost, h->stream));
        CKS(cudaStreamSynchronize(h->stream));
        norms[0] = tmp[0]; norms[1] = tmp[1]; norms[2] = tmp[2];
    }
    return HDG_OK;
}

int hdg_lift_gradient(hdg_handle h, const double* U, const double* UH, double* Q) {
    if (h && h->tet) return fail(h, HDG_EUNSUPPORTED, "not available for tetrahedral handles");
    if (!h) return HDG_EINVAL;
    if (!h->device) return fail(h, HDG_EINVAL, "handle has no device storage");
    if (!U || !UH || !Q) return fail(h, HDG_EINVAL, "U, UH and Q are required");
    int rc;
    DISPATCH_S(run_lift, h, U, UH, Q);
    return rc;
}

int hdg_update_state(hdg_handle h, double* U, double* Q, double* UH, const double* dU, const double* dQ,
                     const double* dUH, double alpha) {
    if (!h) return HDG_EINVAL;
    if (!h->device) return fail(h, HDG_EINVAL, "handle has no device storage");
    if (!U || !Q || !UH || !dU || !dQ || !dUH) return fail(h, HDG_EINVAL, "NULL argument");
    const int64_t nU = len_u(h), nQ = len_q(h), nH = len_t(h);
    k_axpby<<<grid_for(nU), 256, 0, h->stream>>>(alpha, dU, 1.0, U, nU);
    k_axpby<<<grid_for(nQ), 256, 0, h->stream>>>(alpha, dQ, 1.0, Q, nQ);
    k_axpby<<<grid_for(nH), 256, 0, h->stream>>>(alpha, dUH, 1.0, UH, nH);
    CKS(cudaGetLastError());
    return HDG_OK;
}

int hdg_blockjacobi_setup(hdg_handle h) {
    if (!h) return HDG_EINVAL;
    if (!h->device || !h->have_system) return fail(h, HDG_EINVAL, "no assembled trace system");
    if (h->tet) return hdg::tet::bj_setup(h);
    int rc;
    if (!h->d_bjlu) {
        if ((rc = alloc(h, (void**)&h->d_bjlu, sizeof(double) * h->F * h->BS * h->BS))) return rc;
    }
    DISPATCH_S(run_bj_setup, h);
    if (rc) return rc;
    h->bj_ready = true;
    return HDG_OK;
}

int hdg_set_preconditioner(hdg_handle h, int kind) {
    if (!h) return HDG_EINVAL;
    if (kind != HDG_PC_BLOCKJACOBI && kind != HDG_PC_SCHWARZ)
        return fail(h, HDG_EINVAL, "preconditioner must be HDG_PC_BLOCKJACOBI or HDG_PC_SCHWARZ");
    h->pc_kind = kind;
    return HDG_OK;
}

int hdg_schwarz_setup(hdg_handle h) {
    if (!h) return HDG_EINVAL;
    if (!h->device || !h->have_system) return fail(h, HDG_EINVAL, "no assembled trace system");
    return schwarz_setup(h);
}

int hdg_schwarz_apply(hdg_handle h, const double* x, double* y) {
    if (!h) return HDG_EINVAL;
    if (!(h->tet ? h->tet->asm_ready : h->asm_ready)) return fail(h, HDG_EINVAL, "additive Schwarz factors not set up");
    if (!x || !y || x == y) return fail(h, HDG_EINVAL, "x and y must be distinct device arrays");
    if (h->tet) return hdg::tet::asm_apply(h, x, y);
    int rc;
    DISPATCH_S(run_asm_apply, h, x, y);
    return rc;
}

int hdg_av_field(hdg_handle h, const double* U, const double* Q, double c_av, double h_m, double s_max, double* nu) {
    if (h && h->tet) return fail(h, HDG_EUNSUPPORTED, "not available for tetrahedral handles");
    if (!h) return HDG_EINVAL;
    if (!h->device) return fail(h, HDG_EINVAL, "handle has no device storage");
    if (!U || !Q || !nu) return fail(h, HDG_EINVAL, "U, Q and nu are required");
    if (!(c_av >= 0.0) || !(h_m > 0.0) || !(s_max >= 0.0)) return fail(h, HDG_EINVAL, "c_av >= 0, h_m > 0, s_max >= 0 required");
    int rc;
    if (!h->d_avev) {
        const int64_t V = (int64_t)h->av_vrow.size() - 1;
        if ((rc = alloc(h, (void**)&h->d_avev, sizeof(int32_t) * h->av_ev.size()))) return rc;
        if ((rc = alloc(h, (void**)&h->d_avvrow, sizeof(int32_t) * h->av_vrow.size()))) return rc;
        if ((rc = alloc(h, (void**)&h->d_avvcol, sizeof(int32_t) * h->av_vcol.size()))) return rc;
        if ((rc = alloc(h, (void**)&h->d_avv, sizeof(double) * std::max<int64_t>(V, 1)))) return rc;
        if ((rc = alloc(h, (void**)&h->d_ave, sizeof(double) * h->E))) return rc;
        CKS(cudaMemcpy(h->d_avev, h->av_ev.data(), sizeof(int32_t) * h->av_ev.size(), cudaMemcpyHostToDevice));
        CKS(cudaMemcpy(h->d_avvrow, h->av_vrow.data(), sizeof(int32_t) * h->av_vrow.size(), cudaMemcpyHostToDevice));
        CKS(cudaMemcpy(h->d_avvcol, h->av_vcol.data(), sizeof(int32_t) * h->av_vcol.size(), cudaMemcpyHostToDevice));
    }
    DISPATCH_S(run_av_field, h, U, Q, c_av, h_m, s_max, nu);
    return rc;
}

int hdg_tgv_diagnostics(hdg_handle h, const double* U, const double* Q, double* out) {
    if (h && h->tet) return fail(h, HDG_EUNSUPPORTED, "not available for tetrahedral handles");
    if (!h) return HDG_EINVAL;
    if (!h->device) return fail(h, HDG_EINVAL, "handle has no device storage");
    if (!U || !Q || !out) return fail(h, HDG_EINVAL, "U, Q and out are required");
    int rc;
    if (!h->d_diag && (rc = alloc(h, (void**)&h->d_diag, sizeof(double) * (4 * h->E + 4)))) return rc;
    DISPATCH_S(run_diagnostics, h, U, Q);
    if (rc) return rc;
    double t[4];
    CKS(cudaMemcpyAsync(t, h->d_diag + 4 * h->E, sizeof(t), cudaMemcpyDeviceToHost, h->stream));
    CKS(cudaStreamSynchronize(h->stream));
    const double vol = t[3], re = h->phys.re;
    out[0] = t[0] / (2.0 * vol);
    out[1] = t[1] / (re * vol);
    out[2] = 4.0 * t[2] / (3.0 * re * vol);
    out[3] = vol;
    return HDG_OK;
}

int hdg_rb_setup(hdg_handle h, int nb_max) {
    if (!h) return HDG_EINVAL;
    if (!h->device) return fail(h, HDG_EINVAL, "handle has no device storage");
    if (nb_max < 0 || nb_max > kRbMax) return fail(h, HDG_EINVAL, "nb_max must be in 0..20");
    h->rb_max = 0;
    if (nb_max == 0) return HDG_OK;
    const int64_t N = len_t(h);
    int rc;
    if ((rc = alloc(h, (void**)&h->d_rbW, sizeof(double) * (size_t)nb_max * N))) return rc;
    if ((rc = alloc(h, (void**)&h->d_rbZ, sizeof(double) * (size_t)nb_max * N))) return rc;
    if (!h->d_rbpart) {
        if ((rc = alloc(h, (void**)&h->d_rbpart, sizeof(double) * kRbBlocks * 256))) return rc;
        if ((rc = alloc(h, (void**)&h->d_rbc, sizeof(double) * kRbMax))) return rc;
        if ((rc = alloc(h, (void**)&h->d_rbhead, sizeof(int) * 2))) return rc;
    }
    if (!h->d_w && (rc = alloc(h, (void**)&h->d_w, sizeof(double) * N))) return rc;
    CKS(cudaMemsetAsync(h->d_rbW, 0, sizeof(double) * (size_t)nb_max * N, h->stream));
    CKS(cudaMemsetAsync(h->d_rbZ, 0, sizeof(double) * (size_t)nb_max * N, h->stream));
    CKS(cudaMemsetAsync(h->d_rbhead, 0, sizeof(int) * 2, h->stream));
    h->rb_max = nb_max;
    return HDG_OK;
}

int hdg_rb_push(hdg_handle h, const double* w) {
    if (!h) return HDG_EINVAL;
    if (h->rb_max <= 0) return fail(h, HDG_EINVAL, "reduced basis not set up (hdg_rb_setup)");
    if (!h->have_system) return fail(h, HDG_EINVAL, "no assembled trace system");
    if (!w) return fail(h, HDG_EINVAL, "w is NULL");
    return rb_push(h, w);
}

int hdg_rb_guess(hdg_handle h, const double* g, double* x0) {
    if (!h) return HDG_EINVAL;
    if (h->rb_max <= 0) return fail(h, HDG_EINVAL, "reduced basis not set up (hdg_rb_setup)");
    if (!g || !x0 || g == x0) return fail(h, HDG_EINVAL, "g and x0 must be distinct device arrays");
    return rb_guess(h, g, x0);
}

int hdg_blockjacobi_apply(hdg_handle h, const double* x, double* y) {
    if (!h) return HDG_EINVAL;
    if (!(h->tet ? h->tet->bj_ready : h->bj_ready)) return fail(h, HDG_EINVAL, "block-Jacobi factors not set up");
    if (!x || !y || x == y) return fail(h, HDG_EINVAL, "x and y must be distinct device arrays");
    if (h->tet) return hdg::tet::bj_apply(h, x, y);
    int rc;
    DISPATCH_S(run_bj_apply, h, x, y);
    return rc;
}

int hdg_gmres(hdg_handle h, const double* b, double* x, int restart, int max_iter, double rtol, int precond,
              int* iters_out, double* relres_out) {
    if (!h) return HDG_EINVAL;
    if (!h->device || !h->have_system) return fail(h, HDG_EINVAL, "no assembled trace system");
    if (!b || !x || b == x) return fail(h, HDG_EINVAL, "b and x must be distinct device arrays");
    if (restart < 1 || restart > 500 || max_iter < 1 || !(rtol > 0.0))
        return fail(h, HDG_EINVAL, "restart in 1..500, max_iter >= 1, rtol > 0 required");
    if (precond && !precond_ready(h))
        return fail(h, HDG_EINVAL, "precond = 1 needs the selected preconditioner set up (hdg_blockjacobi_setup / hdg_schwarz_setup)");
    const int64_t N = len_t(h);
    int rc;
    if (h->gm_cap < restart) {
        // workspace grows to the largest restart length requested; kept until destroy
        if ((rc = alloc(h, (void**)&h->d_V, sizeof(double) * (size_t)(restart + 1) * N))) return rc;
        if ((rc = alloc(h, (void**)&h->d_w, sizeof(double) * N))) return rc;
        if (!h->d_red && (rc = alloc(h, (void**)&h->d_red, sizeof(double) * kRedBlocks * 8))) return rc;
        if ((rc = alloc(h, (void**)&h->d_mred, sizeof(double) * kRedBlocks * 8 * ((restart + 8) / 8)))) return rc;
        if ((rc = alloc(h, (void**)&h->d_h, sizeof(double) * 2 * (restart + 2)))) return rc;
        h->gm_cap = restart;
    }
    double* V = h->d_V;
    double* w = h->d_w;
    double* dh = h->d_h;
    const int m = restart;
    std::vector<double> H((size_t)(m + 1) * m, 0.0), cs(m), sn(m), g(m + 1), hc(m + 2), y(m);
    int it = 0;
    double beta0 = -1.0, res = 0.0;
    bool done = false;
    {   // reference norm ||M^{-1} b||: the tolerance does not depend on the initial guess
        if (precond) { if ((rc = precond_apply(h, b, V))) return rc; }
        else CKS(cudaMemcpyAsync(V, b, sizeof(double) * N, cudaMemcpyDeviceToDevice, h->stream));
        dev_dot(h, V, V, N, dh, true);
        CKS(cudaMemcpyAsync(&beta0, dh, sizeof(double), cudaMemcpyDeviceToHost, h->stream));
        CKS(cudaStreamSynchronize(h->stream));
        if (!std::isfinite(beta0)) return fail(h, HDG_ENONFINITE, "non-finite right-hand side in GMRES");
    }
    while (!done) {
        // r = M^{-1} (b - S x) into V_0
        if ((rc = matvec(h, x, w))) return rc;
        k_axpby<<<grid_for(N), 256, 0, h->stream>>>(1.0, b, -1.0, w, N);
        if (precond) { if ((rc = precond_apply(h, w, V))) return rc; }
        else CKS(cudaMemcpyAsync(V, w, sizeof(double) * N, cudaMemcpyDeviceToDevice, h->stream));
        dev_dot(h, V, V, N, dh, true);
        double beta;
        CKS(cudaMemcpyAsync(&beta, dh, sizeof(double), cudaMemcpyDeviceToHost, h->stream));
        CKS(cudaStreamSynchronize(h->stream));
        if (!std::isfinite(beta)) return fail(h, HDG_ENONFINITE, "non-finite residual in GMRES");
        res = beta;
        if (beta == 0.0 || beta <= rtol * beta0 || it >= max_iter) break;
        k_scale_dev<<<grid_for(N), 256, 0, h->stream>>>(V, dh, V, N);
        std::fill(g.begin(), g.end(), 0.0);
        g[0] = beta;
        int j = 0;
        for (; j < m; ++j) {
            double* vj = V + (size_t)j * N;
            double* vn = V + (size_t)(j + 1) * N;
            if (precond) {
                if ((rc = matvec(h, vj, w))) return rc;
                if ((rc = precond_apply(h, w, vn))) return rc;
            } else if ((rc = matvec(h, vj, vn))) {
                return rc;
            }
            cgs2(h, V, N, j, vn, dh, dh + m + 2);   // Gram-Schmidt with reorthogonalisation
            dev_dot(h, vn, vn, N, dh + j + 1, true);
            k_scale_dev<<<grid_for(N), 256, 0, h->stream>>>(vn, dh + j + 1, vn, N);
            CKS(cudaMemcpyAsync(hc.data(), dh, sizeof(double) * (j + 2), cudaMemcpyDeviceToHost, h->stream));
            CKS(cudaStreamSynchronize(h->stream));
            for (int i = 0; i < j; ++i) {       // previous rotations
                double t = cs[i] * hc[i] + sn[i] * hc[i + 1];
                hc[i + 1] = -sn[i] * hc[i] + cs[i] * hc[i + 1];
                hc[i] = t;
            }
            double den = std::hypot(hc[j], hc[j + 1]);
            if (!std::isfinite(den)) return fail(h, HDG_ENONFINITE, "non-finite Hessenberg entry in GMRES");
            cs[j] = den > 0.0 ? hc[j] / den : 1.0;
            sn[j] = den > 0.0 ? hc[j + 1] / den : 0.0;
            hc[j] = den;
            hc[j + 1] = 0.0;
            g[j + 1] = -sn[j] * g[j];
            g[j] = cs[j] * g[j];
            for (int i = 0; i <= j; ++i) H[(size_t)i * m + j] = hc[i];
            ++it;
            res = std::fabs(g[j + 1]);
            if (res <= rtol * beta0 || it >= max_iter) { ++j; break; }
        }
        // back substitution and update x += V y
        const int k = j;
        for (int i = k - 1; i >= 0; --i) {
            double s = g[i];
            for (int l = i + 1; l < k; ++l) s -= H[(size_t)i * m + l] * y[l];
            y[i] = s / H[(size_t)i * m + i];
        }
        CKS(cudaMemcpyAsync(dh, y.data(), sizeof(double) * k, cudaMemcpyHostToDevice, h->stream));
        k_combine<<<grid_for(N), 256, 0, h->stream>>>(V, N, dh, k, x, N);
        CKS(cudaGetLastError());
        if (res <= rtol * beta0 || it >= max_iter) done = true;
    }
    CKS(cudaStreamSynchronize(h->stream));
    if (iters_out) *iters_out = it;
    double rel = beta0 > 0.0 ? res / beta0 : 0.0;
    if (relres_out) *relres_out = rel;
    if (rel > rtol) return fail(h, HDG_ENOCONV, "GMRES reached max_iter with relative residual " + std::to_string(rel));
    return HDG_OK;
}

int hdg_newton(hdg_handle h, double* U, double* Q, double* UH, const double* Ustar, const double* nu, double dt,
               double a_ii, double tol, int max_newton, int restart, int max_gmres, double gmres_rtol,
               double* hist, int* newton_iters, int* gmres_iters) {
    if (!h) return HDG_EINVAL;
    if (!h->device) return fail(h, HDG_EINVAL, "handle has no device storage");
    if (!U || !Q || !UH || !Ustar) return fail(h, HDG_EINVAL, "U, Q, UH and Ustar are required");
    if (!(tol > 0.0) || max_newton < 0) return fail(h, HDG_EINVAL, "tol > 0 and max_newton >= 0 required");
    int rc;
    if (!h->d_nw) {
        size_t n = (size_t)(len_u(h) + len_q(h) + 2 * len_t(h));
        if ((rc = alloc(h, (void**)&h->d_nw, sizeof(double) * n))) return rc;
    }
    double* dU = h->d_nw;
    double* dQ = dU + (size_t)len_u(h);
    double* dUH = dQ + (size_t)len_q(h);
    double* g = dUH + (size_t)len_t(h);
    int total = 0, k = 0;
    double nrm[3];
    for (;; ++k) {
        if ((rc = hdg_residual(h, U, Q, UH, Ustar, nu, dt, a_ii, nullptr, nullptr, nullptr, nrm))) return rc;
        if (hist) hist[k] = nrm[0];
        if (!std::isfinite(nrm[0])) return fail(h, HDG_ENONFINITE, "non-finite residual in Newton");
        if (nrm[0] <= tol || k >= max_newton) break;
        if ((rc = hdg_linearize_condense(h, U, Q, UH, Ustar, nu, dt, a_ii, nullptr))) return rc;
        if ((rc = hdg_trace_rhs(h, g))) return rc;
        if ((rc = precond_setup(h))) return rc;
        if (h->rb_max > 0) {
            if ((rc = rb_guess(h, g, dUH))) return rc;
        } else {
            CKS(cudaMemsetAsync(dUH, 0, sizeof(double) * len_t(h), h->stream));
        }
        int it = 0;
        double rel = 0.0;
        rc = hdg_gmres(h, g, dUH, restart, max_gmres, gmres_rtol, 1, &it, &rel);
        total += it;
        if (rc && rc != HDG_ENOCONV) return rc;
        if (h->rb_max > 0 && (rc = rb_push(h, dUH))) return rc;
        if ((rc = hdg_recover_interior(h, dUH, dQ, dU))) return rc;
        if ((rc = hdg_update_state(h, U, Q, UH, dU, dQ, dUH, 1.0))) return rc;
    }
    if (newton_iters) *newton_iters = k;
    if (gmres_iters) *gmres_iters = total;
    if (nrm[0] > tol) return fail(h, HDG_ENOCONV, "Newton stopped at ||F|| = " + std::to_string(nrm[0]));
    return HDG_OK;
}

}  // extern "C"

namespace {

int precond_setup(hdg_ctx* h) { return h->pc_kind == HDG_PC_SCHWARZ ? schwarz_setup(h) : hdg_blockjacobi_setup(h); }

int newton_iteration_async(hdg_ctx* h, double* U, double* Q, double* UH, const double* Ustar, const double* nu,
                           double dt, double a_ii, int m) {
    double* dU = h->d_nw;
    double* dQ = dU + (size_t)len_u(h);
    double* dUH = dQ + (size_t)len_q(h);
    double* g = dUH + (size_t)len_t(h);
    int rc;
    if ((rc = hdg_residual(h, U, Q, UH, Ustar, nu, dt, a_ii, nullptr, nullptr, nullptr, nullptr))) return rc;
    k_hist_push<<<1, 32, 0, h->stream>>>(h->d_norms, h->d_hist, h->d_hcount, 4096);
    if ((rc = hdg_linearize_condense(h, U, Q, UH, Ustar, nu, dt, a_ii, nullptr))) return rc;
    if ((rc = hdg_trace_rhs(h, g))) return rc;
    if ((rc = precond_setup(h))) return rc;
    if (h->rb_max > 0) {
        if ((rc = rb_guess(h, g, dUH))) return rc;
        if ((rc = gmres_fixed_async(h, g, dUH, m, true))) return rc;
        if ((rc = rb_push(h, dUH))) return rc;
    } else if ((rc = gmres_fixed_async(h, g, dUH, m, false))) {
        return rc;
    }
    if ((rc = hdg_recover_interior(h, dUH, dQ, dU))) return rc;
    return hdg_update_state(h, U, Q, UH, dU, dQ, dUH, 1.0);
}

// run `body` either directly or as a CUDA graph captured once and replayed
template <class Body>
int run_maybe_graph(hdg_ctx* h, bool use_graph, uint64_t key, Body body) {
    if (!use_graph) return body();
    if (!h->gstream) CKS(cudaStreamCreateWithFlags(&h->gstream, cudaStreamNonBlocking));
    if (!h->gexec || h->gkey != key) {
        if (h->gexec) { cudaGraphExecDestroy(h->gexec); h->gexec = nullptr; }
        cudaStream_t user = h->stream;
        const bool prof = h->prof;
        h->prof = false;
        h->stream = h->gstream;
        cudaGraph_t graph = nullptr;
        CKS(cudaStreamBeginCapture(h->gstream, cudaStreamCaptureModeThreadLocal));
        int rc = body();
        cudaError_t ce = cudaStreamEndCapture(h->gstream, &graph);
        h->stream = user;
        h->prof = prof;
        if (rc) { if (graph) cudaGraphDestroy(graph); return rc; }
        if (ce != cudaSuccess) return fail(h, HDG_ECUDA, std::string("stream capture: ") + cudaGetErrorString(ce));
        ce = cudaGraphInstantiate(&h->gexec, graph, 0);
        cudaGraphDestroy(graph);
        if (ce != cudaSuccess) { h->gexec = nullptr; return fail(h, HDG_ECUDA, std::string("graph instantiate: ") + cudaGetErrorString(ce)); }
        h->gkey = key;
    }
    CKS(cudaGraphLaunch(h->gexec, h->stream));
    return HDG_OK;
}

uint64_t mix_key(std::initializer_list<uint64_t> v) {
    uint64_t k = 1469598103934665603ull;
    for (uint64_t x : v) { k ^= x; k *= 1099511628211ull; }
    return k;
}

uint64_t dbits(double d) { uint64_t u; std::memcpy(&u, &d, 8); return u; }

// device stage states of a DIRK step
int ensure_dirk_storage(hdg_ctx* h, int s) {
    if (h->dirk_cap >= s) return HDG_OK;
    int rc;
    const size_t n = (size_t)len_u(h);
    if ((rc = alloc(h, (void**)&h->d_dirk, sizeof(double) * n * (s + 2)))) return rc;
    h->dirk_cap = s;
    return HDG_OK;
}

}  // namespace

extern "C" {

int hdg_newton_fixed(hdg_handle h, double* U, double* Q, double* UH, const double* Ustar, const double* nu,
                     double dt, double a_ii, int n_newton, int m, int use_graph, double* hist) {
    if (!h) return HDG_EINVAL;
    if (!h->device) return fail(h, HDG_EINVAL, "handle has no device storage");
    if (!U || !Q || !UH || !Ustar) return fail(h, HDG_EINVAL, "U, Q, UH and Ustar are required");
    if (n_newton < 1 || n_newton > 1000 || m < 1 || m > 256) return fail(h, HDG_EINVAL, "1 <= n_newton <= 1000, 1 <= m <= 256");
    if (!(dt > 0.0) || !(a_ii > 0.0)) return fail(h, HDG_EINVAL, "dt and a_ii must be positive");
    int rc;
    if ((rc = ensure_fixed_workspace(h, m))) return rc;
    const uint64_t key = mix_key({1, (uint64_t)U, (uint64_t)Q, (uint64_t)UH, (uint64_t)Ustar, (uint64_t)nu, dbits(dt),
                                  dbits(a_ii), (uint64_t)m, (uint64_t)h->precision, (uint64_t)h->schur_mode,
                                  (uint64_t)h->d_V, (uint64_t)h->d_fx, (uint64_t)h->rb_max, (uint64_t)h->d_rbW,
                                  (uint64_t)h->pc_kind});
    if (use_graph && (!h->gexec || h->gkey != key)) {
        // one linearization outside the capture: every lazily allocated buffer exists before it
        if ((rc = hdg_linearize_condense(h, U, Q, UH, Ustar, nu, dt, a_ii, nullptr))) return rc;
        if ((rc = precond_setup(h))) return rc;
    }
    CKS(cudaMemsetAsync(h->d_hcount, 0, sizeof(int), h->stream));
    for (int k = 0; k < n_newton; ++k) {
        rc = run_maybe_graph(h, use_graph != 0, key,
                             [&]() { return newton_iteration_async(h, U, Q, UH, Ustar, nu, dt, a_ii, m); });
        if (rc) return rc;
    }
    if ((rc = hdg_residual(h, U, Q, UH, Ustar, nu, dt, a_ii, nullptr, nullptr, nullptr, nullptr))) return rc;
    k_hist_push<<<1, 32, 0, h->stream>>>(h->d_norms, h->d_hist, h->d_hcount, 4096);
    if (hist) {
        CKS(cudaMemcpyAsync(hist, h->d_hist, sizeof(double) * (n_newton + 1), cudaMemcpyDeviceToHost, h->stream));
    }
    CKS(cudaStreamSynchronize(h->stream));
    return HDG_OK;
}

int hdg_sdirk3_tableau(double* A, double* b) {
    if (!A || !b) return HDG_EINVAL;
    // gamma: the root in (1/3, 1/2) of gamma^3 - 3 gamma^2 + 3 gamma / 2 - 1/6 = 0, the condition
    // under which the three-stage, third-order SDIRK is L-stable; Newton from 0.44 converges to it
    double g = 0.44;
    for (int it = 0; it < 50; ++it) {
        const double f = ((g - 3.0) * g + 1.5) * g - 1.0 / 6.0;
        const double df = (3.0 * g - 6.0) * g + 1.5;
        const double dg = f / df;
        g -= dg;
        if (std::fabs(dg) <= 1e-17) break;
    }
    const double b1 = -(6.0 * g * g - 16.0 * g + 1.0) / 4.0;
    const double b2 = (6.0 * g * g - 20.0 * g + 5.0) / 4.0;
    const double tab[9] = {g, 0.0, 0.0, (1.0 - g) / 2.0, g, 0.0, b1, b2, g};
    for (int i = 0; i < 9; ++i) A[i] = tab[i];
    b[0] = b1; b[1] = b2; b[2] = g;       // stiffly accurate: b is the last row of A
    return HDG_OK;
}

int hdg_dirk_step(hdg_handle h, double* U, double* Q, double* UH, const double* nu, double dt, int s,
                  const double* A, const double* b, int n_newton, int m, int use_graph, double* hist) {
    if (!h) return HDG_EINVAL;
    if (!h->device) return fail(h, HDG_EINVAL, "handle has no device storage");
    double A3[9], b3[3];
    if (!A && !b) {                           // NULL tableau: Alexander's SDIRK3
        if (s != 3) return fail(h, HDG_EINVAL, "a NULL tableau means the three-stage SDIRK3 (s = 3)");
        hdg_sdirk3_tableau(A3, b3);
        A = A3;
        b = b3;
    }
    if (!U || !Q || !UH || !A || !b) return fail(h, HDG_EINVAL, "NULL argument");
    if (s < 1 || s > 8 || n_newton < 1 || n_newton > 100 || m < 1 || m > 256)
        return fail(h, HDG_EINVAL, "1 <= s <= 8, 1 <= n_newton <= 100, 1 <= m <= 256");
    if (!(dt > 0.0)) return fail(h, HDG_EINVAL, "dt must be positive");
    // Butcher matrix: lower triangular with a positive diagonal; d = A^{-1}; e_j = sum_i b_i d_ij
    double d[8][8] = {};
    for (int i = 0; i < s; ++i) {
        if (!(A[i * s + i] > 0.0)) return fail(h, HDG_EINVAL, "DIRK diagonal must be positive");
        for (int j = i + 1; j < s; ++j)
            if (A[i * s + j] != 0.0) return fail(h, HDG_EINVAL, "Butcher matrix must be lower triangular");
    }
    for (int j = 0; j < s; ++j) {            // forward substitution column by column
        for (int i = 0; i < s; ++i) {
            double r = (i == j) ? 1.0 : 0.0;
            for (int k = 0; k < i; ++k) r -= A[i * s + k] * d[k][j];
            d[i][j] = r / A[i * s + i];
        }
    }
    double e[8] = {};
    for (int j = 0; j < s; ++j)
        for (int i = 0; i < s; ++i) e[j] += b[i] * d[i][j];
    for (int j = 0; j < s - 1; ++j)
        if (std::fabs(e[j]) > 1e-12) return fail(h, HDG_EUNSUPPORTED, "only stiffly accurate tableaus (b = last row of A)");
    int rc;
    if ((rc = ensure_fixed_workspace(h, m))) return rc;
    if ((rc = ensure_dirk_storage(h, s))) return rc;
    const int64_t n = len_u(h);
    double* Un = h->d_dirk;                  // U^n
    double* Us = Un + n;                     // U* of the current stage
    double* St = Us + n;                     // stage states U^{n,1..s}
    uint64_t key = mix_key({2, (uint64_t)U, (uint64_t)Q, (uint64_t)UH, (uint64_t)nu, dbits(dt), (uint64_t)s,
                            (uint64_t)n_newton, (uint64_t)m, (uint64_t)h->precision, (uint64_t)h->schur_mode,
                            (uint64_t)h->d_V, (uint64_t)h->d_fx, (uint64_t)h->d_dirk, (uint64_t)h->rb_max,
                            (uint64_t)h->d_rbW, (uint64_t)h->pc_kind});
    for (int i = 0; i < s * s; ++i) key = mix_key({key, dbits(A[i])});
    if (use_graph && (!h->gexec || h->gkey != key)) {
        // one linearization outside the capture: every lazily allocated buffer exists before it
        CKS(cudaMemcpyAsync(Us, U, sizeof(double) * n, cudaMemcpyDeviceToDevice, h->stream));
        if ((rc = hdg_linearize_condense(h, U, Q, UH, Us, nu, dt, A[0], nullptr))) return rc;
        if ((rc = precond_setup(h))) return rc;
    }
    CKS(cudaMemsetAsync(h->d_hcount, 0, sizeof(int), h->stream));
    auto body = [&]() -> int {
        int r;
        if (cudaMemcpyAsync(Un, U, sizeof(double) * n, cudaMemcpyDeviceToDevice, h->stream) != cudaSuccess)
            return fail(h, HDG_ECUDA, "copy of U^n failed");
        for (int i = 0; i < s; ++i) {
            const double aii = A[i * s + i];
            // U* = U^n - a_ii sum_{j<i} d_ij (U^{n,j} - U^n)   (eq. dirk-stage, d_ii = 1/a_ii)
            cudaMemcpyAsync(Us, Un, sizeof(double) * n, cudaMemcpyDeviceToDevice, h->stream);
            for (int j = 0; j < i; ++j)
                k_lincomb3<<<grid_for(n), 256, 0, h->stream>>>(-aii * d[i][j], St + (size_t)j * n, aii * d[i][j], Un,
                                                               1.0, Us, n);
            for (int k = 0; k < n_newton; ++k)
                if ((r = newton_iteration_async(h, U, Q, UH, Us, nu, dt, aii, m))) return r;
            if ((r = hdg_residual(h, U, Q, UH, Us, nu, dt, aii, nullptr, nullptr, nullptr, nullptr))) return r;
            k_hist_push<<<1, 32, 0, h->stream>>>(h->d_norms, h->d_hist, h->d_hcount, 4096);
            cudaMemcpyAsync(St + (size_t)i * n, U, sizeof(double) * n, cudaMemcpyDeviceToDevice, h->stream);
        }
        // stiffly accurate: U^{n+1} = U^{n,s} (eq. dirk-update with e = (0, .., 0, 1)); Q, UH of the last stage
        return cudaGetLastError() == cudaSuccess ? HDG_OK : fail(h, HDG_ECUDA, "launch failed in DIRK step");
    };
    if ((rc = run_maybe_graph(h, use_graph != 0, key, body))) return rc;
    if (hist) CKS(cudaMemcpyAsync(hist, h->d_hist, sizeof(double) * s * (n_newton + 1), cudaMemcpyDeviceToHost, h->stream));
    CKS(cudaStreamSynchronize(h->stream));
    return HDG_OK;
}

}  // extern "C"
