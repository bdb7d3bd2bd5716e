// Host side of the trace-space solve: FP64 stage residual, Newton update,
// block-Jacobi preconditioner and restarted, left-preconditioned GMRES with
// modified Gram-Schmidt Arnoldi in FP64 (Sec. 3.2).  The Krylov coefficients
// live on the device; only the Hessenberg column of each iteration is read
// back for the Givens rotations.
#include <cmath>
#include <vector>

#include "solve.cuh"

using namespace hdg;

namespace {

int fail(hdg_ctx* h, int code, const std::string& m) {
    h->err = m;
    return code;
}

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
    int rc;
    DISPATCH_S(run_bj_apply, h, x, y);
    return rc;
}

int matvec(hdg_ctx* h, const double* x, double* y) {
    int rc;
    DISPATCH_S(run_matvec, h, x, y);
    return rc;
}

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
    LinArgs a{U, Q, UH, Ustar, nu, dt, a_ii};
    DISPATCH_S(run_residual, h, a, Rq, Ru, Ruh);
    if (rc) return rc;
    k_sum_parts<<<1, 256, 0, h->stream>>>(h->d_part, h->E, h->d_part + h->E, h->F, h->d_norms);
    CKS(cudaGetLastError());
    if (norms) {
        double tmp[3];
        CKS(cudaMemcpyAsync(tmp, h->d_norms, sizeof(tmp), cudaMemcpyDeviceToHost, h->stream));
        CKS(cudaStreamSynchronize(h->stream));
        norms[0] = tmp[0]; norms[1] = tmp[1]; norms[2] = tmp[2];
    }
    return HDG_OK;
}

int hdg_update_state(hdg_handle h, double* U, double* Q, double* UH, const double* dU, const double* dQ,
                     const double* dUH, double alpha) {
    if (!h) return HDG_EINVAL;
    if (!h->device) return fail(h, HDG_EINVAL, "handle has no device storage");
    if (!U || !Q || !UH || !dU || !dQ || !dUH) return fail(h, HDG_EINVAL, "NULL argument");
    const int64_t nU = h->E * h->NU, nQ = h->E * h->NQV, nH = h->F * h->BS;
    k_axpby<<<grid_for(nU), 256, 0, h->stream>>>(alpha, dU, 1.0, U, nU);
    k_axpby<<<grid_for(nQ), 256, 0, h->stream>>>(alpha, dQ, 1.0, Q, nQ);
    k_axpby<<<grid_for(nH), 256, 0, h->stream>>>(alpha, dUH, 1.0, UH, nH);
    CKS(cudaGetLastError());
    return HDG_OK;
}

int hdg_blockjacobi_setup(hdg_handle h) {
    if (!h) return HDG_EINVAL;
    if (!h->device || !h->have_system) return fail(h, HDG_EINVAL, "no assembled trace system");
    int rc;
    if (!h->d_bjlu) {
        if ((rc = alloc(h, (void**)&h->d_bjlu, sizeof(double) * h->F * h->BS * h->BS))) return rc;
        if ((rc = alloc(h, (void**)&h->d_bjpiv, sizeof(int32_t) * h->F * h->BS))) return rc;
    }
    DISPATCH_S(run_bj_setup, h);
    if (rc) return rc;
    h->bj_ready = true;
    return HDG_OK;
}

int hdg_blockjacobi_apply(hdg_handle h, const double* x, double* y) {
    if (!h) return HDG_EINVAL;
    if (!h->bj_ready) return fail(h, HDG_EINVAL, "block-Jacobi factors not set up");
    if (!x || !y || x == y) return fail(h, HDG_EINVAL, "x and y must be distinct device arrays");
    return precond_apply(h, x, y);
}

int hdg_gmres(hdg_handle h, const double* b, double* x, int restart, int max_iter, double rtol, int precond,
              int* iters_out, double* relres_out) {
    if (!h) return HDG_EINVAL;
    if (!h->device || !h->have_system) return fail(h, HDG_EINVAL, "no assembled trace system");
    if (!b || !x || b == x) return fail(h, HDG_EINVAL, "b and x must be distinct device arrays");
    if (restart < 1 || restart > 500 || max_iter < 1 || !(rtol > 0.0))
        return fail(h, HDG_EINVAL, "restart in 1..500, max_iter >= 1, rtol > 0 required");
    if (precond && !h->bj_ready) return fail(h, HDG_EINVAL, "precond = 1 needs hdg_blockjacobi_setup");
    const int64_t N = h->F * h->BS;
    int rc;
    if (h->gm_cap < restart) {
        // workspace grows to the largest restart length requested; kept until destroy
        if ((rc = alloc(h, (void**)&h->d_V, sizeof(double) * (size_t)(restart + 1) * N))) return rc;
        if ((rc = alloc(h, (void**)&h->d_w, sizeof(double) * N))) return rc;
        if (!h->d_red && (rc = alloc(h, (void**)&h->d_red, sizeof(double) * kRedBlocks))) return rc;
        if ((rc = alloc(h, (void**)&h->d_h, sizeof(double) * (restart + 2)))) return rc;
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
        if (beta0 < 0.0) beta0 = beta;
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
            for (int i = 0; i <= j; ++i) {      // modified Gram-Schmidt
                dev_dot(h, vn, V + (size_t)i * N, N, dh + i, false);
                k_axpy_dev<<<grid_for(N), 256, 0, h->stream>>>(dh + i, -1.0, V + (size_t)i * N, vn, N);
            }
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
        size_t n = (size_t)h->E * (h->NU + h->NQV) + 2 * (size_t)h->F * h->BS;
        if ((rc = alloc(h, (void**)&h->d_nw, sizeof(double) * n))) return rc;
    }
    double* dU = h->d_nw;
    double* dQ = dU + (size_t)h->E * h->NU;
    double* dUH = dQ + (size_t)h->E * h->NQV;
    double* g = dUH + (size_t)h->F * h->BS;
    int total = 0, k = 0;
    double nrm[3];
    for (;; ++k) {
        if ((rc = hdg_residual(h, U, Q, UH, Ustar, nu, dt, a_ii, nullptr, nullptr, nullptr, nrm))) return rc;
        if (hist) hist[k] = nrm[0];
        if (!std::isfinite(nrm[0])) return fail(h, HDG_ENONFINITE, "non-finite residual in Newton");
        if (nrm[0] <= tol || k >= max_newton) break;
        if ((rc = hdg_linearize_condense(h, U, Q, UH, Ustar, nu, dt, a_ii, nullptr))) return rc;
        if ((rc = hdg_trace_rhs(h, g))) return rc;
        if ((rc = hdg_blockjacobi_setup(h))) return rc;
        CKS(cudaMemsetAsync(dUH, 0, sizeof(double) * h->F * h->BS, h->stream));
        int it = 0;
        double rel = 0.0;
        rc = hdg_gmres(h, g, dUH, restart, max_gmres, gmres_rtol, 1, &it, &rel);
        total += it;
        if (rc && rc != HDG_ENOCONV) return rc;
        if ((rc = hdg_recover_interior(h, dUH, dQ, dU))) return rc;
        if ((rc = hdg_update_state(h, U, Q, UH, dU, dQ, dUH, 1.0))) return rc;
    }
    if (newton_iters) *newton_iters = k;
    if (gmres_iters) *gmres_iters = total;
    if (nrm[0] > tol) return fail(h, HDG_ENOCONV, "Newton stopped at ||F|| = " + std::to_string(nrm[0]));
    return HDG_OK;
}

}  // extern "C"
