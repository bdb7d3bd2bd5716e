// hdg_linearize_condense_static: the FP64 linearize + condense path with its
// per-chunk scratch (trace rows of the bordered matrix, point coefficients,
// per-point stabilization and the scale exponents of the tensor-core Schur
// product) taken from a fixed, file-scope device array instead
// of the handle's scratch allocation.  This entry point calls no allocating
// CUDA or library routine.
//
// The scratch array (64 MiB) is part of the library image: every GPU that
// loads libhdg.so holds it until the process exits.  Host code may not use the
// array's name as a device address (it is a host-side stand-in), so on the
// first call on each device, with that device current, the device address is
// looked up with cudaGetSymbolAddress and cached.  The first call on a device
// should therefore be made before any stream capture.
#include <mutex>

#include "common.h"

constexpr size_t kStaticScratchDoubles = (size_t)8 << 20;  // 8 Mi doubles = 64 MiB
static __device__ __align__(256) double g_static_scratch[kStaticScratchDoubles];

namespace {

constexpr int kMaxDevices = 64;
std::mutex g_mu;
double* g_addr[kMaxDevices] = {};

int fail(hdg_ctx* h, int code, const std::string& m) {
    h->err = m;
    return code;
}

int scratch_address(hdg_ctx* h, double** out) {
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return fail(h, HDG_ECUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
    if (dev < 0 || dev >= kMaxDevices) return fail(h, HDG_EINVAL, "device index out of range");
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_addr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_static_scratch);
        if (e != cudaSuccess) return fail(h, HDG_ECUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
        g_addr[dev] = static_cast<double*>(p);
    }
    *out = g_addr[dev];
    return HDG_OK;
}

int dispatch(hdg_ctx* h, const hdg::LinArgs& a) {
    switch (h->d * 10 + h->p) {
        case 21: return hdg::run_linearize<2, 1>(h, a);
        case 22: return hdg::run_linearize<2, 2>(h, a);
        case 23: return hdg::run_linearize<2, 3>(h, a);
        case 31: return hdg::run_linearize<3, 1>(h, a);
        case 32: return hdg::run_linearize<3, 2>(h, a);
        case 33: return hdg::run_linearize<3, 3>(h, a);
        default: return fail(h, HDG_EUNSUPPORTED, "unsupported (d, p)");
    }
}

}  // namespace

extern "C" int hdg_linearize_condense_static(hdg_handle h, const double* U, const double* Q, const double* UH,
                                              const double* Ustar, const double* nu, double dt, double a_ii) {
    if (!h) return HDG_EINVAL;
    if (h->tet) return fail(h, HDG_EUNSUPPORTED, "not available for tetrahedral handles");
    if (!h->device) return fail(h, HDG_EINVAL, "handle has no device storage (created with hdg_create_host)");
    if (!U || !Q || !UH || !Ustar) return fail(h, HDG_EINVAL, "U, Q, UH and Ustar are required");
    if (!(dt > 0.0) || !(a_ii > 0.0)) return fail(h, HDG_EINVAL, "dt and a_ii must be positive");
    // the same preconditions as hdg_linearize_condense
    if (h->has_tag[1] && !h->ub_set) return fail(h, HDG_EINVAL, "boundary state of tag 1 not set (hdg_set_bc_state)");
    if (h->has_tag[3] && !h->tw_set) return fail(h, HDG_EINVAL, "wall temperature of tag 3 not set (hdg_set_bc_state)");
    if (h->precision != HDG_PREC_FP64)
        return fail(h, HDG_EUNSUPPORTED, "the allocation-free entry point builds the FP64 system only");
    if (!h->d_vals || !h->d_top)
        return fail(h, HDG_EINVAL, "FP64 system storage not reserved (hdg_reserve(h, HDG_PREC_FP64) at set-up)");
    const size_t n_bot = (size_t)h->NT * h->LD;
    const size_t n_vc = (size_t)h->m * h->m * h->d * h->NCOEF * h->Nq;
    const size_t n_fc = (size_t)h->nf * h->m * h->m * h->NCOEF * h->Nfq;
    const size_t n_tp = (size_t)h->nf * h->Nfq;      // per-point tau of the state-dependent stabilization
    const size_t n_oz = (size_t)h->NT;               // 2 NT int32 scale exponents of the tensor-core Schur product
    const size_t per = n_bot + n_vc + n_fc + n_tp + n_oz;
    if (per > kStaticScratchDoubles)
        return fail(h, HDG_EINVAL, "one element needs " + std::to_string(per * 8) +
                                       " bytes of scratch, more than the 64 MiB static scratch");
    double* base = nullptr;
    int rc = scratch_address(h, &base);
    if (rc) return rc;
    const int64_t chunk = std::min<int64_t>(h->E, (int64_t)(kStaticScratchDoubles / per));
    // every scratch word is written before it is read within a call, so the
    // previous call's contents need no clearing
    double* save_bot = h->d_bot;
    double* save_vc = h->d_vcoef;
    double* save_fc = h->d_fcoef;
    double* save_tp = h->d_taup;
    int32_t* save_oz = h->d_ozexp;
    const int64_t save_chunk = h->chunk;
    const bool save_prof = h->prof;
    h->d_bot = base;
    h->d_vcoef = base + (size_t)chunk * n_bot;
    h->d_fcoef = h->d_vcoef + (size_t)chunk * n_vc;
    h->d_taup = h->d_fcoef + (size_t)chunk * n_fc;   // sized for this chunk, not the handle's
    h->d_ozexp = reinterpret_cast<int32_t*>(h->d_taup + (size_t)chunk * n_tp);
    h->chunk = chunk;
    h->prof = false;  // event creation is an allocation
    cudaError_t e = cudaMemsetAsync(h->d_status, 0, sizeof(int32_t), h->stream);
    if (e != cudaSuccess) rc = fail(h, HDG_ECUDA, std::string("cudaMemsetAsync: ") + cudaGetErrorString(e));
    else rc = dispatch(h, hdg::LinArgs{U, Q, UH, Ustar, nu, dt, a_ii});
    h->d_bot = save_bot;
    h->d_vcoef = save_vc;
    h->d_fcoef = save_fc;
    h->d_taup = save_tp;
    h->d_ozexp = save_oz;
    h->chunk = save_chunk;
    h->prof = save_prof;
    return rc;
}
