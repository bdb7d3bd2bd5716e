// C-ABI entry points of libhdg: handle life cycle, host set-up (tables,
// skeleton, affine geometry), device storage and dispatch to the kernels of
// the (d, p) configuration.
#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <new>

#include "common.h"
#include "tet.h"

using namespace hdg;

namespace hdg {
void prof_begin(hdg_ctx* h, int kind) {
    h->launches[kind] += 1;
    if (!h->prof) return;
    while (h->ev_pool.size() < h->ev_used + 2) {
        cudaEvent_t ev;
        if (cudaEventCreate(&ev) != cudaSuccess) { h->prof = false; return; }
        h->ev_pool.push_back(ev);
    }
    cudaEventRecord(h->ev_pool[h->ev_used], h->stream);
    h->ev_kind.push_back(kind);
}
void prof_end(hdg_ctx* h) {
    if (!h->prof || h->ev_kind.size() * 2 != h->ev_used + 2) return;
    cudaEventRecord(h->ev_pool[h->ev_used + 1], h->stream);
    h->ev_used += 2;
}
}  // namespace hdg

namespace {

int fail(hdg_ctx* h, int code, const std::string& msg) {
    if (h) h->err = msg;
    return code;
}

#define CKH(call)                                                                   \
    do {                                                                            \
        cudaError_t e_ = (call);                                                    \
        if (e_ != cudaSuccess)                                                      \
            return fail(h, e_ == cudaErrorMemoryAllocation ? HDG_ENOMEM : HDG_ECUDA, \
                        std::string(#call) + ": " + cudaGetErrorString(e_));        \
    } while (0)

// Affine element geometry: x = X0 + J (xi + 1), J[:, r] = (X_{2^r} - X_0) / 2.
int build_geometry(hdg_ctx* h, const hdg_mesh& m) {
    const int d = h->d, nv = 1 << d, nf = 2 * d;
    h->detJ.assign(h->E, 0.0);
    h->Jinv.assign((size_t)h->E * d * d, 0.0);
    h->NW.assign((size_t)h->E * nf * d, 0.0);
    h->centroid.assign((size_t)h->E * 3, 0.0);
    for (int64_t e = 0; e < h->E; ++e) {
        double X[8][3] = {};
        for (int c = 0; c < nv; ++c)
            for (int k = 0; k < d; ++k) X[c][k] = m.vert_xyz[(size_t)m.elem_vert[(size_t)e * nv + c] * d + k];
        for (int c = 0; c < nv; ++c)
            for (int k = 0; k < d; ++k) h->centroid[(size_t)e * 3 + k] += X[c][k] / nv;
        double J[3][3] = {};  // J[k][r] = d x_k / d xi_r
        for (int r = 0; r < d; ++r)
            for (int k = 0; k < d; ++k) J[k][r] = 0.5 * (X[1 << r][k] - X[0][k]);
        double diam = 0.0;
        for (int r = 0; r < d; ++r)
            for (int k = 0; k < d; ++k) diam = std::max(diam, std::fabs(J[k][r]));
        for (int c = 0; c < nv; ++c)
            for (int k = 0; k < d; ++k) {
                double x = X[0][k];
                for (int r = 0; r < d; ++r) if ((c >> r) & 1) x += 2.0 * J[k][r];
                if (std::fabs(x - X[c][k]) > 1e-10 * diam)
                    return fail(h, HDG_EUNSUPPORTED, "element " + std::to_string(e) + " is not affine");
            }
        double det, inv[3][3];
        if (d == 2) {
            det = J[0][0] * J[1][1] - J[0][1] * J[1][0];
            inv[0][0] = J[1][1] / det; inv[0][1] = -J[0][1] / det;
            inv[1][0] = -J[1][0] / det; inv[1][1] = J[0][0] / det;
        } else {
            det = J[0][0] * (J[1][1] * J[2][2] - J[1][2] * J[2][1]) - J[0][1] * (J[1][0] * J[2][2] - J[1][2] * J[2][0]) +
                  J[0][2] * (J[1][0] * J[2][1] - J[1][1] * J[2][0]);
            for (int i = 0; i < 3; ++i)
                for (int j = 0; j < 3; ++j) {
                    int i1 = (j + 1) % 3, i2 = (j + 2) % 3, j1 = (i + 1) % 3, j2 = (i + 2) % 3;
                    inv[i][j] = (J[i1][j1] * J[i2][j2] - J[i1][j2] * J[i2][j1]) / det;
                }
        }
        if (!(det > 0.0)) return fail(h, HDG_EINVAL, "element " + std::to_string(e) + " has non-positive volume");
        // inv[r][k] = d xi_r / d x_k
        h->detJ[e] = det;
        for (int r = 0; r < d; ++r)
            for (int k = 0; k < d; ++k) h->Jinv[((size_t)e * d + r) * d + k] = inv[r][k];
        for (int f = 0; f < nf; ++f) {
            int r = f / 2;
            double sg = (f % 2) ? 1.0 : -1.0;
            for (int k = 0; k < d; ++k) h->NW[((size_t)e * nf + f) * d + k] = det * sg * inv[r][k];
        }
    }
    return HDG_OK;
}

int create_host(hdg_ctx* h, const hdg_mesh* mesh, int p, double gamma, double Re, double Pr, double Mach) {
    if (!mesh) return fail(h, HDG_EINVAL, "mesh is NULL");
    if (!(mesh->dim == 2 && mesh->elem_type == HDG_QUAD) && !(mesh->dim == 3 && mesh->elem_type == HDG_HEX))
        return fail(h, HDG_EUNSUPPORTED, "supported elements: HDG_QUAD (dim 2), HDG_HEX (dim 3)");
    if (p < 1 || p > 3) return fail(h, HDG_EUNSUPPORTED, "degree p must be 1, 2 or 3");
    if (mesh->n_elem <= 0 || mesh->n_vert <= 0 || !mesh->vert_xyz || !mesh->elem_vert)
        return fail(h, HDG_EINVAL, "empty mesh or NULL arrays");
    if (!(gamma > 1.0) || !(Re > 0.0) || !(Pr > 0.0) || !(Mach > 0.0))
        return fail(h, HDG_EINVAL, "gamma > 1, Re > 0, Pr > 0, Mach > 0 required");
    const int d = mesh->dim;
    h->d = d; h->p = p; h->m = d + 2;
    h->Np = ipow(p + 1, d); h->Nq = ipow(p + 2, d); h->nf = 2 * d;
    h->Nfp = ipow(p + 1, d - 1); h->Nfq = ipow(p + 2, d - 1);
    h->NU = h->m * h->Np; h->NQV = d * h->m * h->Np; h->NT = h->nf * h->m * h->Nfp;
    h->NR = h->NU + h->NT; h->NC = h->NR + 1; h->LD = (h->NC + 3) & ~3;
    h->BS = h->m * h->Nfp; h->NCOEF = 1 + d + h->nf;
    h->E = mesh->n_elem;
    h->phys = Phys{gamma, Re, Pr, Mach, 5.0, 0, 1.4042, 0.40417};
    try {
        build_ref_tables(d, p, h->ref);
    } catch (const std::exception& ex) {
        return fail(h, HDG_EINVAL, ex.what());
    }
    int rc = build_skeleton(*mesh, p, h->sk, h->err);
    if (rc) return rc;
    if ((rc = build_vertex_map(*mesh, h->av_ev, h->av_vrow, h->av_vcol, h->err))) return rc;
    h->F = h->sk.n_faces;
    h->nnzb = h->sk.rowptr[h->F];
    // boundary tags: 0 on interior / periodic faces; on faces with a single element
    // 1 far-field / supersonic inflow, 2 supersonic outflow, 3 isothermal wall, 4 adiabatic wall
    h->ftag.assign((size_t)h->E * h->nf, 0);
    if (mesh->bnd_tag)
        for (int64_t i = 0; i < h->E * h->nf; ++i) {
            if (mesh->bnd_tag[i] < 0 || mesh->bnd_tag[i] > 4)
                return fail(h, HDG_EUNSUPPORTED, "boundary tag " + std::to_string(mesh->bnd_tag[i]) + " not supported (0..4)");
            h->ftag[i] = mesh->bnd_tag[i];
        }
    for (int64_t F = 0; F < h->F; ++F) {
        const int32_t e0 = h->sk.f2e[2 * F], f0 = h->sk.f2lf[2 * F];
        const bool single = h->sk.f2e[2 * F + 1] < 0;
        if (single != (h->ftag[(size_t)e0 * h->nf + f0] != 0))
            return fail(h, HDG_EINVAL, "face " + std::to_string(F) + ": tags 1..4 must mark exactly the faces with one element");
        if (!single && h->ftag[(size_t)h->sk.f2e[2 * F + 1] * h->nf + h->sk.f2lf[2 * F + 1]] != 0)
            return fail(h, HDG_EINVAL, "face " + std::to_string(F) + ": interior face tagged as boundary");
    }
    h->has_bnd = false;
    for (int32_t t : h->ftag) { h->has_bnd |= (t != 0); h->has_tag[t] = true; }
    return build_geometry(h, *mesh);
}

template <class T>
int dev_alloc(hdg_ctx* h, T** out, size_t count) {
    void* p = nullptr;
    cudaError_t e = cudaMalloc(&p, std::max<size_t>(count, 1) * sizeof(T));
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(h, HDG_ENOMEM, "cudaMalloc of " + std::to_string(count * sizeof(T)) + " bytes failed: " + cudaGetErrorString(e));
    }
    h->allocs.push_back(p);
    h->device_bytes += (int64_t)(count * sizeof(T));
    *out = (T*)p;
    return HDG_OK;
}

template <class T>
int dev_upload(hdg_ctx* h, T** out, const std::vector<T>& v) {
    int rc = dev_alloc(h, out, v.size());
    if (rc) return rc;
    CKH(cudaMemcpy(*out, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice));
    return HDG_OK;
}

}  // namespace

namespace hdg {
int ensure_system_storage(hdg_ctx* h, int precision) {
    int rc;
    if (precision == HDG_PREC_FP64) {
        if (!h->d_vals && (rc = dev_alloc(h, &h->d_vals, (size_t)h->nnzb * h->BS * h->BS))) return rc;
        if (!h->d_top && (rc = dev_alloc(h, &h->d_top, (size_t)h->E * h->NU * h->LD))) return rc;
        if (!h->d_bot && (rc = dev_alloc(h, &h->d_bot, (size_t)h->chunk * h->NT * h->LD))) return rc;
        return HDG_OK;
    }
    if (h->d_m11) return HDG_OK;
    const size_t E = h->E, ch = h->chunk, NU = h->NU, NT = h->NT;
    if ((rc = dev_alloc(h, &h->d_m11, E * NU * NU))) return rc;
    if ((rc = dev_alloc(h, &h->d_m12, E * NU * NT))) return rc;
    if ((rc = dev_alloc(h, &h->d_mrt, E * NU))) return rc;
    if ((rc = dev_alloc(h, &h->d_m21, ch * NT * NU))) return rc;
    if ((rc = dev_alloc(h, &h->d_m22, ch * NT * NT))) return rc;
    if ((rc = dev_alloc(h, &h->d_mrb, ch * NT))) return rc;
    if ((rc = dev_alloc(h, &h->d_vals32, (size_t)h->nnzb * h->BS * h->BS))) return rc;
    if ((rc = dev_alloc(h, &h->d_x32, (size_t)h->F * h->BS))) return rc;
    if ((rc = dev_alloc(h, &h->d_mpiv, E * NU))) return rc;
    return HDG_OK;
}
}  // namespace hdg

namespace {

int create_device(hdg_ctx* h) {
    const RefTables& t = h->ref;
    int rc;
#define UP(dst, src) if ((rc = dev_upload(h, &(dst), (src)))) return rc
    UP(h->tab.phi, t.phi); UP(h->tab.dphi, t.dphi); UP(h->tab.wq, t.wq);
    UP(h->tab.mu, t.mu); UP(h->tab.wf, t.wf); UP(h->tab.fnode, t.fnode); UP(h->tab.node_face, t.node_face);
    UP(h->tab.mhat, t.mhat); UP(h->tab.mf, t.mf); UP(h->tab.minv_c, t.minv_c); UP(h->tab.minv_e, t.minv_e);
    UP(h->tab.psi, t.psi); UP(h->tab.theta, t.theta); UP(h->tab.psi_f, t.psi_f); UP(h->tab.theta_f, t.theta_f);
    UP(h->tab.b1, t.b1); UP(h->tab.d1, t.d1);
    auto f32 = [](const std::vector<double>& v) { return std::vector<float>(v.begin(), v.end()); };
    UP(h->tab.fphi, f32(t.phi)); UP(h->tab.fdphi, f32(t.dphi)); UP(h->tab.fpsi, f32(t.psi));
    UP(h->tab.ftheta, f32(t.theta)); UP(h->tab.fpsi_f, f32(t.psi_f)); UP(h->tab.ftheta_f, f32(t.theta_f));
    UP(h->tab.fmu, f32(t.mu)); UP(h->tab.fmf, f32(t.mf));
    UP(h->tab.fb1, f32(t.b1)); UP(h->tab.fd1, f32(t.d1));
    const int d = h->d, G = 1 + d * d + h->nf * d;
    std::vector<double> geo((size_t)h->E * G);
    for (int64_t e = 0; e < h->E; ++e) {
        double* g = &geo[(size_t)e * G];
        g[0] = h->detJ[e];
        for (int i = 0; i < d * d; ++i) g[1 + i] = h->Jinv[(size_t)e * d * d + i];
        for (int i = 0; i < h->nf * d; ++i) g[1 + d * d + i] = h->NW[(size_t)e * h->nf * d + i];
    }
    UP(h->d_geo, geo);
    UP(h->d_e2f, h->sk.e2f); UP(h->d_perm, h->sk.perm); UP(h->d_iperm, h->sk.iperm);
    UP(h->d_rowptr, h->sk.rowptr); UP(h->d_col, h->sk.col);
    UP(h->d_blk, h->sk.blk); UP(h->d_rank, h->sk.rank); UP(h->d_frank, h->sk.frank);
#undef UP
    // the per-element storage of the FP64 / mixed system is allocated on first use
    // (ensure_system_storage), so a mixed-only run never holds the FP64 arrays
    if ((rc = dev_alloc(h, &h->d_g, (size_t)h->F * h->BS))) return rc;
    if ((rc = dev_alloc(h, &h->d_dq0, (size_t)h->E * h->NQV))) return rc;
    if ((rc = dev_alloc(h, &h->d_status, 1))) return rc;
    if (h->has_bnd) {
        if ((rc = dev_upload(h, &h->d_ftag, h->ftag))) return rc;
        if ((rc = dev_alloc(h, &h->d_ub, (size_t)h->m))) return rc;
        CKH(cudaMemset(h->d_ub, 0, sizeof(double) * h->m));
    }
    CKH(cudaMemset(h->d_status, 0, sizeof(int32_t)));
    // per-chunk scratch: trace rows of the bordered matrix and the point coefficients
    const size_t per = sizeof(double) * ((size_t)h->NT * h->LD + (size_t)h->m * h->m * d * h->NCOEF * h->Nq +
                                         (size_t)h->nf * h->m * h->m * h->NCOEF * h->Nfq);
    size_t budget = (size_t)8 << 30;
    if (const char* s = std::getenv("HDG_SCRATCH_BYTES")) budget = std::strtoull(s, nullptr, 10);
    h->chunk = std::max<int64_t>(1, std::min<int64_t>(h->E, (int64_t)(budget / per)));
    if (const char* s = std::getenv("HDG_ELIM_MINB")) h->elim_minb = std::atoi(s) == 1 ? 1 : 2;
    if ((rc = dev_alloc(h, &h->d_vcoef, (size_t)h->chunk * h->m * h->m * d * h->NCOEF * h->Nq))) return rc;
    if ((rc = dev_alloc(h, &h->d_fcoef, (size_t)h->chunk * h->nf * h->m * h->m * h->NCOEF * h->Nfq))) return rc;
    if ((rc = dev_alloc(h, &h->d_taup, (size_t)h->chunk * h->nf * h->Nfq))) return rc;
    if ((rc = dev_alloc(h, &h->d_ozexp, (size_t)h->chunk * 2 * h->NT))) return rc;
    h->device = true;
    return HDG_OK;
}

#define DISPATCH(FN, ...)                                                       \
    switch (h->d * 10 + h->p) {                                                  \
        case 21: return FN<2, 1>(__VA_ARGS__);                                   \
        case 22: return FN<2, 2>(__VA_ARGS__);                                   \
        case 23: return FN<2, 3>(__VA_ARGS__);                                   \
        case 31: return FN<3, 1>(__VA_ARGS__);                                   \
        case 32: return FN<3, 2>(__VA_ARGS__);                                   \
        case 33: return FN<3, 3>(__VA_ARGS__);                                   \
        default: return fail(h, HDG_EUNSUPPORTED, "unsupported (d, p)");        \
    }

}  // namespace

extern "C" {

int hdg_create_host(hdg_handle* out, const hdg_mesh* mesh, int p, double gamma, double Re, double Pr, double Mach) {
    if (!out) return HDG_EINVAL;
    *out = nullptr;
    hdg_ctx* h = new (std::nothrow) hdg_ctx();
    if (!h) return HDG_ENOMEM;
    int rc = create_host(h, mesh, p, gamma, Re, Pr, Mach);
    *out = h;  // the handle is returned even on failure so that hdg_last_error works
    return rc;
}

int hdg_create(hdg_handle* out, const hdg_mesh* mesh, int p, double gamma, double Re, double Pr, double Mach) {
    int rc = hdg_create_host(out, mesh, p, gamma, Re, Pr, Mach);
    if (rc) return rc;
    hdg_ctx* h = *out;
    rc = create_device(h);
    return rc;
}

int hdg_destroy(hdg_handle h) {
    if (!h) return HDG_OK;
    for (cudaEvent_t ev : h->ev_pool) cudaEventDestroy(ev);
    if (h->gexec) cudaGraphExecDestroy(h->gexec);
    if (h->gstream) cudaStreamDestroy(h->gstream);
    for (void* p : h->allocs) cudaFree(p);
    if (h->tet) hdg::tet::destroy(h);
    delete h;
    return HDG_OK;
}

const char* hdg_last_error(hdg_handle h) { return h ? h->err.c_str() : "NULL handle"; }

int hdg_set_params(hdg_handle h, const hdg_params* prm) {
    if (!h || !prm) return fail(h, HDG_EINVAL, "NULL argument");
    if (!(prm->tau > 0.0)) return fail(h, HDG_EINVAL, "tau must be positive");
    if (prm->visc_law != 0 && prm->visc_law != 1) return fail(h, HDG_EINVAL, "visc_law must be 0 or 1");
    if (prm->visc_law == 1 && !(prm->suth_c1 > 0.0 && prm->suth_s > 0.0))
        return fail(h, HDG_EINVAL, "Sutherland constants must be positive");
    if (prm->precision < HDG_PREC_FP64 || prm->precision > HDG_PREC_MIXED_3XTF32)
        return fail(h, HDG_EUNSUPPORTED, "precision mode not available");
    if (prm->tau_mode != 0 && prm->tau_mode != 1) return fail(h, HDG_EINVAL, "tau_mode must be 0 or 1");
    h->phys.tau = prm->tau;
    h->phys.tau_mode = prm->tau_mode;
    h->phys.visc_law = prm->visc_law;
    h->phys.c1 = prm->suth_c1;
    h->phys.s = prm->suth_s;
    h->precision = prm->precision == HDG_PREC_FP64 ? HDG_PREC_FP64 : HDG_PREC_MIXED;
    h->schur_mode = prm->precision == HDG_PREC_FP64 ? 0 : prm->precision - HDG_PREC_MIXED;
    h->prec_req = prm->precision;
    return HDG_OK;
}

int hdg_reserve(hdg_handle h, int precision) {
    if (h && h->tet) return fail(h, HDG_EUNSUPPORTED, "not available for tetrahedral handles");
    if (!h) return HDG_EINVAL;
    if (!h->device) return fail(h, HDG_EINVAL, "handle has no device storage");
    if (precision < HDG_PREC_FP64 || precision > HDG_PREC_MIXED_3XTF32) return fail(h, HDG_EINVAL, "unknown precision");
    return hdg::ensure_system_storage(h, precision == HDG_PREC_FP64 ? HDG_PREC_FP64 : HDG_PREC_MIXED);
}

int hdg_autotune(hdg_handle h, const double* U, const double* Q, const double* UH, const double* Ustar,
                 const double* nu, double dt, double a_ii, int reps, hdg_tune* out) {
    if (h && h->tet) {
        // tetrahedral handles: the elimination panel width of the persistent kernel
        if (!h->device) return fail(h, HDG_EINVAL, "handle has no device storage");
        if (reps < 1 || reps > 100) return fail(h, HDG_EINVAL, "reps must be in 1..100");
        const int nbs[2] = {16, 8};
        double best = 1e300;
        int pick = 16;
        cudaEvent_t e0, e1;
        CKH(cudaEventCreate(&e0));
        CKH(cudaEventCreate(&e1));
        if (out) { std::memset(out, 0, sizeof(*out)); out->n_cand = 2; }
        for (int i = 0; i < 2; ++i) {
            h->tet->nb = nbs[i];
            int rc = hdg_linearize_condense(h, U, Q, UH, Ustar, nu, dt, a_ii, nullptr);   // warm-up
            if (rc) { cudaEventDestroy(e0); cudaEventDestroy(e1); return rc; }
            CKH(cudaEventRecord(e0, h->stream));
            for (int r = 0; r < reps; ++r)
                if ((rc = hdg_linearize_condense(h, U, Q, UH, Ustar, nu, dt, a_ii, nullptr))) {
                    cudaEventDestroy(e0); cudaEventDestroy(e1); return rc;
                }
            CKH(cudaEventRecord(e1, h->stream));
            CKH(cudaEventSynchronize(e1));
            float ms = 0.f;
            CKH(cudaEventElapsedTime(&ms, e0, e1));
            if (out) { out->cand[i][0] = nbs[i]; out->ms[i] = ms / reps; }
            if (ms < best) { best = ms; pick = nbs[i]; }
        }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        h->tet->nb = pick;
        if (out) out->elim_nb = pick;
        return hdg_linearize_condense(h, U, Q, UH, Ustar, nu, dt, a_ii, nullptr);
    }
    if (!h) return HDG_EINVAL;
    if (!h->device) return fail(h, HDG_EINVAL, "handle has no device storage");
    if (reps < 1 || reps > 100) return fail(h, HDG_EINVAL, "reps must be in 1..100");
    // candidates: variants that compute the same quantities to the same accuracy
    int cand[16][7];
    int n = 0;
    if (h->precision == HDG_PREC_FP64) {
        // Schur product in the FP64 elimination (schur_mode 0) or on the tensor cores by exact
        // digit splitting (3); both FP64-accurate
        const int nbs[2] = {16, 8}, minbs[2] = {2, 1};
        for (int sm : {0, 3})
            for (int bm64 : {1, 0})
                for (int a = 0; a < 2; ++a)
                    for (int b = 0; b < 2; ++b) {
                        cand[n][0] = nbs[a]; cand[n][1] = minbs[b]; cand[n][2] = sm; cand[n][3] = h->blocks_mode;
                        cand[n][4] = h->elim_mixed_minb; cand[n][5] = bm64; cand[n][6] = h->elim_mixed_split; ++n;
                    }
    } else {
        // FP32 SIMT and 3xTF32 tensor-core products are both FP32-accurate: the volume
        // contraction always, the Schur product unless TF32 / 3xTF32 was requested explicitly
        // contraction: tensor cores (3-D) or FP32 sum factorisation; the dense FP32 SIMT
        // contraction only when the Schur precision is fixed (the candidate list holds 8)
        const bool free_schur = h->prec_req == HDG_PREC_MIXED;
        for (int sm : {0, 2}) {
            if (!free_schur && sm != 0) continue;
            for (int bm : {1, 2, 0}) {
                if (bm == 1 && h->d != 3) continue;
                if (bm == 0 && free_schur) continue;
                // elimination: split with the interior LU at panel width 16 or 8 (ev 16, 8), or
                // fused at 2 or 3 CTAs per SM (ev 2, 3)
                for (int ev : {16, 8, 2, 3}) {
                    const bool split = ev >= 8;
                    cand[n][0] = split ? ev : h->elim_nb; cand[n][1] = h->elim_minb;
                    cand[n][2] = free_schur ? sm : h->schur_mode;
                    cand[n][3] = bm; cand[n][4] = split ? h->elim_mixed_minb : ev; cand[n][5] = h->blocks64_mode;
                    cand[n][6] = split ? 1 : 0; ++n;
                }
            }
        }
    }
    cudaEvent_t ev[2];
    CKH(cudaEventCreate(&ev[0]));
    CKH(cudaEventCreate(&ev[1]));
    double ms[16];
    int best = 0, rc = HDG_OK;
    const bool fp64 = h->precision == HDG_PREC_FP64;
    auto apply_schur = [&](int sm) {
        if (fp64) h->schur64_mode = sm == 3 ? 1 : 0;
        else h->schur_mode = sm;
    };
    for (int c = 0; c < n && rc == HDG_OK; ++c) {
        h->elim_nb = cand[c][0];
        h->elim_minb = cand[c][1];
        apply_schur(cand[c][2]);
        h->blocks_mode = cand[c][3];
        h->elim_mixed_minb = cand[c][4];
        h->blocks64_mode = cand[c][5];
        h->elim_mixed_split = cand[c][6];
        if ((rc = hdg_linearize_condense(h, U, Q, UH, Ustar, nu, dt, a_ii, nullptr))) break;   // warm-up
        cudaEventRecord(ev[0], h->stream);
        for (int r = 0; r < reps && rc == HDG_OK; ++r) rc = hdg_linearize_condense(h, U, Q, UH, Ustar, nu, dt, a_ii, nullptr);
        cudaEventRecord(ev[1], h->stream);
        float t = 0.f;
        if (cudaEventSynchronize(ev[1]) != cudaSuccess || cudaEventElapsedTime(&t, ev[0], ev[1]) != cudaSuccess) {
            rc = fail(h, HDG_ECUDA, "event timing failed in autotune");
            break;
        }
        ms[c] = t / reps;
        if (ms[c] < ms[best]) best = c;
    }
    cudaEventDestroy(ev[0]);
    cudaEventDestroy(ev[1]);
    if (rc) return rc;
    h->elim_nb = cand[best][0];
    h->elim_minb = cand[best][1];
    apply_schur(cand[best][2]);
    h->blocks_mode = cand[best][3];
    h->elim_mixed_minb = cand[best][4];
    h->blocks64_mode = cand[best][5];
    h->elim_mixed_split = cand[best][6];
    if (out) {
        out->elim_nb = h->elim_nb; out->elim_minb = h->elim_minb;
        out->schur_mode = fp64 ? (h->schur64_mode ? 3 : 0) : h->schur_mode;
        out->blocks_mode = h->blocks_mode; out->elim_mixed_minb = h->elim_mixed_minb;
        out->blocks64_mode = h->blocks64_mode; out->elim_mixed_split = h->elim_mixed_split;
        out->n_cand = n;
        for (int c = 0; c < 16; ++c) {
            for (int k = 0; k < 7; ++k) out->cand[c][k] = c < n ? cand[c][k] : 0;
            out->ms[c] = c < n ? ms[c] : 0.0;
        }
    }
    return HDG_OK;
}

int hdg_set_tuning(hdg_handle h, const hdg_tune* t) {
    if (h && h->tet) {
        if (!t || (t->elim_nb != 16 && t->elim_nb != 8)) return fail(h, HDG_EINVAL, "elim_nb must be 16 or 8");
        h->tet->nb = t->elim_nb;
        return HDG_OK;
    }
    if (!h || !t) return fail(h, HDG_EINVAL, "NULL argument");
    const bool fp64 = h->precision == HDG_PREC_FP64;
    if ((t->elim_nb != 8 && t->elim_nb != 16) || (t->elim_minb != 1 && t->elim_minb != 2) ||
        (fp64 ? (t->schur_mode != 0 && t->schur_mode != 3) : (t->schur_mode < 0 || t->schur_mode > 2)) ||
        t->blocks_mode < 0 || t->blocks_mode > 2 ||
        (t->elim_mixed_minb != 2 && t->elim_mixed_minb != 3) || t->blocks64_mode < 0 || t->blocks64_mode > 1 ||
        t->elim_mixed_split < 0 || t->elim_mixed_split > 1)
        return fail(h, HDG_EINVAL, "elim_nb 8 or 16, elim_minb 1 or 2, schur_mode 0..2 (FP64 handles: 0 or 3), "
                                   "blocks_mode 0..2, elim_mixed_minb 2 or 3, blocks64_mode 0..1, "
                                   "elim_mixed_split 0..1");
    if (h->precision == HDG_PREC_MIXED && h->prec_req != HDG_PREC_MIXED && t->schur_mode != h->schur_mode)
        return fail(h, HDG_EINVAL, "the Schur precision was fixed by hdg_set_params");
    h->elim_nb = t->elim_nb;
    h->elim_minb = t->elim_minb;
    h->blocks_mode = t->blocks_mode;
    h->elim_mixed_minb = t->elim_mixed_minb;
    h->blocks64_mode = t->blocks64_mode;
    h->elim_mixed_split = t->elim_mixed_split;
    if (h->precision == HDG_PREC_MIXED) h->schur_mode = t->schur_mode;
    else h->schur64_mode = t->schur_mode == 3 ? 1 : 0;
    return HDG_OK;
}

int hdg_set_bc_state(hdg_handle h, int tag, const double* ub) {
    if (!h || !ub) return fail(h, HDG_EINVAL, "NULL argument");
    if (tag != 1 && tag != 3) return fail(h, HDG_EUNSUPPORTED, "only tags 1 (state) and 3 (wall temperature) carry data");
    if (!h->device) return fail(h, HDG_EINVAL, "handle has no device storage");
    if (!h->has_tag[tag]) return fail(h, HDG_EINVAL, "the mesh has no faces of tag " + std::to_string(tag));
    if (tag == 3) {
        if (!(ub[0] > 0.0)) return fail(h, HDG_EINVAL, "wall temperature must be positive");
        const double g = h->phys.gamma, M = h->phys.mach;
        h->e_wall = ub[0] / (g * (g - 1.0) * M * M);      // c_v T_w with T~ = gamma M^2 p / rho
        h->tw_set = true;
        return HDG_OK;
    }
    CKH(cudaMemcpy(h->d_ub, ub, sizeof(double) * h->m, cudaMemcpyHostToDevice));
    h->ub_set = true;
    return HDG_OK;
}

int hdg_set_bc_field(hdg_handle h, const double* ubf) {
    if (h && h->tet) return fail(h, HDG_EUNSUPPORTED, "not available for tetrahedral handles");
    if (!h) return HDG_EINVAL;
    if (!h->device) return fail(h, HDG_EINVAL, "handle has no device storage");
    if (!h->has_tag[1]) return fail(h, HDG_EINVAL, "the mesh has no tag-1 faces");
    const size_t n = (size_t)h->F * h->BS;
    if (!ubf) {                                           // back to the constant state
        h->d_ubf = nullptr;
        return HDG_OK;
    }
    if (!h->ubf_store) {
        int rc;
        if ((rc = dev_alloc(h, &h->ubf_store, n))) return rc;
    }
    CKH(cudaMemcpyAsync(h->ubf_store, ubf, sizeof(double) * n, cudaMemcpyDeviceToDevice, h->stream));
    h->d_ubf = h->ubf_store;
    h->ub_set = true;
    return HDG_OK;
}

int hdg_set_stream(hdg_handle h, void* stream) {
    if (!h) return HDG_EINVAL;
    h->stream = (cudaStream_t)stream;
    return HDG_OK;
}

int hdg_query_sizes(hdg_handle h, hdg_sizes* o) {
    if (h && h->tet) return fail(h, HDG_EUNSUPPORTED, "not available for tetrahedral handles");
    if (!h || !o) return fail(h, HDG_EINVAL, "NULL argument");
    o->dim = h->d; o->p = h->p; o->m = h->m; o->Np = h->Np; o->Nq = h->Nq; o->nf = h->nf;
    o->Nfp = h->Nfp; o->Nfq = h->Nfq; o->n_u = h->NU; o->n_q = h->NQV; o->t = h->NT; o->block = h->BS;
    o->n_elem = h->E; o->n_faces = h->F; o->nnzb = h->nnzb; o->device_bytes = h->device_bytes;
    return HDG_OK;
}

int hdg_get_connectivity(hdg_handle h, int32_t* f2e, int32_t* f2lf, int32_t* e2f, int32_t* perm,
                         int32_t* rowptr, int32_t* col) {
    if (h && h->tet) return fail(h, HDG_EUNSUPPORTED, "not available for tetrahedral handles");
    if (!h) return HDG_EINVAL;
    const Skeleton& s = h->sk;
    if (f2e) std::memcpy(f2e, s.f2e.data(), s.f2e.size() * sizeof(int32_t));
    if (f2lf) std::memcpy(f2lf, s.f2lf.data(), s.f2lf.size() * sizeof(int32_t));
    if (e2f) std::memcpy(e2f, s.e2f.data(), s.e2f.size() * sizeof(int32_t));
    if (perm) std::memcpy(perm, s.perm.data(), s.perm.size() * sizeof(int32_t));
    if (rowptr) std::memcpy(rowptr, s.rowptr.data(), s.rowptr.size() * sizeof(int32_t));
    if (col) std::memcpy(col, s.col.data(), s.col.size() * sizeof(int32_t));
    return HDG_OK;
}

}  // extern "C"

namespace {
int linearize_fp64(hdg_ctx* h, const LinArgs& a) { DISPATCH(run_linearize, h, a); }
int linearize_mixed(hdg_ctx* h, const LinArgs& a) { DISPATCH(run_linearize_mixed, h, a); }
}  // namespace

extern "C" {

int hdg_linearize_condense(hdg_handle h, const double* U, const double* Q, const double* UH, const double* Ustar,
                           const double* nu, double dt, double a_ii, double* res_norm) {
    if (!h) return HDG_EINVAL;
    if (!h->device) return fail(h, HDG_EINVAL, "handle has no device storage (created with hdg_create_host)");
    if (!U || !Q || !UH || !Ustar) return fail(h, HDG_EINVAL, "U, Q, UH and Ustar are required");
    if (!(dt > 0.0) || !(a_ii > 0.0)) return fail(h, HDG_EINVAL, "dt and a_ii must be positive");
    if (h->has_tag[1] && !h->ub_set) return fail(h, HDG_EINVAL, "boundary state of tag 1 not set (hdg_set_bc_state)");
    if (h->has_tag[3] && !h->tw_set) return fail(h, HDG_EINVAL, "wall temperature of tag 3 not set (hdg_set_bc_state)");
    if (h->tet && nu) return fail(h, HDG_EUNSUPPORTED, "artificial viscosity is not available on tetrahedral handles");
    CKH(cudaMemsetAsync(h->d_status, 0, sizeof(int32_t), h->stream));
    int rc = HDG_OK;
    if (h->tet) {
        rc = hdg::tet::linearize(h, U, Q, UH, Ustar, dt, a_ii);
    } else {
        LinArgs a{U, Q, UH, Ustar, nu, dt, a_ii};
        rc = h->precision == HDG_PREC_MIXED ? linearize_mixed(h, a) : linearize_fp64(h, a);
    }
    if (rc || !res_norm) return rc;
    // ||F(W)||_2 of the stage equations at the same W, always in FP64 (eq. nonlinear-residual)
    double norms[3];
    if ((rc = hdg_residual(h, U, Q, UH, Ustar, nu, dt, a_ii, nullptr, nullptr, nullptr, norms))) return rc;
    *res_norm = norms[0];
    return HDG_OK;
}

int hdg_trace_matvec(hdg_handle h, const double* x, double* y) {
    if (!h) return HDG_EINVAL;
    if (h->tet) {
        if (!h->device || !h->tet->have_system) return fail(h, HDG_EINVAL, "no assembled trace system");
        if (!x || !y || x == y) return fail(h, HDG_EINVAL, "x and y must be distinct device arrays");
        return hdg::tet::matvec(h, x, y);
    }
    if (!h->device || !h->have_system) return fail(h, HDG_EINVAL, "no assembled trace system");
    if (!x || !y || x == y) return fail(h, HDG_EINVAL, "x and y must be distinct device arrays");
    DISPATCH(run_matvec, h, x, y);
}

int hdg_trace_rhs(hdg_handle h, double* g) {
    if (!h) return HDG_EINVAL;
    if (h->tet) {
        if (!h->device || !h->tet->have_system) return fail(h, HDG_EINVAL, "no assembled trace system");
        if (!g) return fail(h, HDG_EINVAL, "g is NULL");
        CKH(cudaMemcpyAsync(g, h->tet->d_g, sizeof(double) * h->tet->n_trace, cudaMemcpyDeviceToDevice, h->stream));
        return HDG_OK;
    }
    if (!h->device || !h->have_system) return fail(h, HDG_EINVAL, "no assembled trace system");
    if (!g) return fail(h, HDG_EINVAL, "g is NULL");
    CKH(cudaMemcpyAsync(g, h->d_g, sizeof(double) * h->F * h->BS, cudaMemcpyDeviceToDevice, h->stream));
    return HDG_OK;
}

int hdg_recover_interior(hdg_handle h, const double* dUH, double* dQ, double* dU) {
    if (!h) return HDG_EINVAL;
    if (h->tet) {
        if (!h->device || !h->tet->have_system) return fail(h, HDG_EINVAL, "no linearization to recover from");
        if (!dUH || !dQ || !dU) return fail(h, HDG_EINVAL, "NULL argument");
        return hdg::tet::recover(h, dUH, dQ, dU);
    }
    if (!h->device || !h->have_system) return fail(h, HDG_EINVAL, "no linearization to recover from");
    if (!dUH || !dQ || !dU) return fail(h, HDG_EINVAL, "NULL argument");
    DISPATCH(run_recover, h, dUH, dQ, dU);
}

int hdg_get_blocks(hdg_handle h, double* vals) {
    if (!h) return HDG_EINVAL;
    if (h->tet) {
        if (!h->device || !h->tet->have_system) return fail(h, HDG_EINVAL, "no assembled trace system");
        if (!vals) return fail(h, HDG_EINVAL, "vals is NULL");
        const bool f32 = h->tet->sys_prec != HDG_PREC_FP64;
        CKH(cudaMemcpyAsync(vals, f32 ? (const void*)h->tet->d_vals32 : (const void*)h->tet->d_vals,
                            (f32 ? sizeof(float) : sizeof(double)) * h->tet->n_vals, cudaMemcpyDeviceToDevice,
                            h->stream));
        return HDG_OK;
    }
    if (!h->device || !h->have_system) return fail(h, HDG_EINVAL, "no assembled trace system");
    if (!vals) return fail(h, HDG_EINVAL, "vals is NULL");
    const size_t bytes = (h->sys_prec == HDG_PREC_MIXED ? sizeof(float) : sizeof(double)) * h->nnzb * h->BS * h->BS;
    CKH(cudaMemcpyAsync(vals, h->sys_prec == HDG_PREC_MIXED ? (const void*)h->d_vals32 : (const void*)h->d_vals,
                        bytes, cudaMemcpyDeviceToDevice, h->stream));
    return HDG_OK;
}

int hdg_set_element_block_output(hdg_handle h, void* SK) {
    if (!h) return HDG_EINVAL;
    if (!h->device) return fail(h, HDG_EINVAL, "handle has no device storage");
    if (h->tet) return hdg::tet::set_element_block_output(h, SK);
    h->d_skout = SK;
    return HDG_OK;
}

int hdg_status(hdg_handle h) {
    if (!h) return HDG_EINVAL;
    if (!h->device) return fail(h, HDG_EINVAL, "handle has no device storage");
    int32_t st = 0;
    CKH(cudaMemcpyAsync(&st, h->d_status, sizeof(int32_t), cudaMemcpyDeviceToHost, h->stream));
    CKH(cudaStreamSynchronize(h->stream));
    if (st & 2) return fail(h, HDG_ENONFINITE, "non-finite pivot in an element interior block");
    if (st & 1) return fail(h, HDG_ESINGULAR, "zero pivot in an element interior block");
    return HDG_OK;
}

int hdg_profile(hdg_handle h, int enable) {
    if (!h) return HDG_EINVAL;
    h->prof = enable != 0;
    return HDG_OK;
}

int hdg_profile_read(hdg_handle h, double* ms, int64_t* launches) {
    if (!h) return HDG_EINVAL;
    if (h->device && h->ev_used) {
        CKH(cudaStreamSynchronize(h->stream));
        for (size_t i = 0; i < h->ev_kind.size(); ++i) {
            float t = 0.f;
            CKH(cudaEventElapsedTime(&t, h->ev_pool[2 * i], h->ev_pool[2 * i + 1]));
            h->ms_acc[h->ev_kind[i]] += t;
        }
    }
    for (int k = 0; k < HDG_NK; ++k) {
        if (ms) ms[k] = h->ms_acc[k];
        if (launches) launches[k] = h->launches[k];
        h->ms_acc[k] = 0.0;
        h->launches[k] = 0;
    }
    h->ev_kind.clear();
    h->ev_used = 0;
    return HDG_OK;
}

int hdg_create_tet_host(hdg_handle* out, const hdg_tet_mesh* mesh, double gamma, double Re, double Pr,
                        double Mach) {
    if (!out) return HDG_EINVAL;
    *out = nullptr;
    hdg_ctx* h = new (std::nothrow) hdg_ctx();
    if (!h) return HDG_ENOMEM;
    *out = h;  // returned even on failure so that hdg_last_error works
    if (!(gamma > 1.0) || !(Re > 0.0) || !(Pr > 0.0) || !(Mach > 0.0))
        return fail(h, HDG_EINVAL, "gamma > 1, Re > 0, Pr > 0, Mach > 0 required");
    h->phys = Phys{gamma, Re, Pr, Mach, 5.0, 0, 1.4042, 0.40417};
    return hdg::tet::create_host(h, mesh, h->err);
}

int hdg_create_tet(hdg_handle* out, const hdg_tet_mesh* mesh, double gamma, double Re, double Pr, double Mach) {
    int rc = hdg_create_tet_host(out, mesh, gamma, Re, Pr, Mach);
    if (rc) return rc;
    return hdg::tet::create_device(*out, (*out)->err);
}

int hdg_tet_query(hdg_handle h, hdg_tet_sizes* o) {
    if (!h || !o) return fail(h, HDG_EINVAL, "NULL argument");
    if (!h->tet) return fail(h, HDG_EINVAL, "not a tetrahedral handle");
    const hdg::tet::Ctx* c = h->tet;
    o->n_elem = c->E; o->n_faces = c->F; o->nnzb = c->nnzb; o->n_u = c->n_u; o->n_trace = c->n_trace;
    o->n_vals = c->n_vals; o->n_curved = c->n_curved; o->device_bytes = h->device_bytes;
    return HDG_OK;
}

int hdg_tet_layout(hdg_handle h, int64_t* uoff, int64_t* hoff, int32_t* face_p, int32_t* f2e, int32_t* e2f,
                   int32_t* frame, int32_t* rowptr, int32_t* col, int64_t* boff) {
    if (!h) return HDG_EINVAL;
    if (!h->tet) return fail(h, HDG_EINVAL, "not a tetrahedral handle");
    const hdg::tet::Ctx* c = h->tet;
    auto cp = [](void* dst, const void* src, size_t bytes) { if (dst) std::memcpy(dst, src, bytes); };
    cp(uoff, c->uoff.data(), c->uoff.size() * sizeof(int64_t));
    cp(hoff, c->hoff.data(), c->hoff.size() * sizeof(int64_t));
    cp(face_p, c->face_p.data(), c->face_p.size() * sizeof(int32_t));
    cp(f2e, c->f2e.data(), c->f2e.size() * sizeof(int32_t));
    cp(e2f, c->e2f.data(), c->e2f.size() * sizeof(int32_t));
    cp(frame, c->frame.data(), c->frame.size() * sizeof(int32_t));
    cp(rowptr, c->rowptr.data(), c->rowptr.size() * sizeof(int32_t));
    cp(col, c->col.data(), c->col.size() * sizeof(int32_t));
    cp(boff, c->boff.data(), c->boff.size() * sizeof(int64_t));
    return HDG_OK;
}

}  // extern "C"
