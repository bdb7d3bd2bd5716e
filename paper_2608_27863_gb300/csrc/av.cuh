// Artificial viscosity (Sec. 2.2, eq. av-coeffs) and the volume-integrated
// TGV diagnostics (Sec. 5.1, eqs. tgv-kinetic-energy, tgv-total-dissipation).
//
// Sensor at every solution node from the nodal U and gradient Q:
//   s = sqrt(h_m / p) L(-div v) / c* * L(-div v)^2 / (L(-div v)^2 + |curl v|^2 + 1e-12),
//   nu_raw = c_av min(max(s, 0), s_max),  c* = sqrt(gamma p / rho),
// with L the clamp to non-negative values (the sensor responds to
// compression); the raw elemental value is the maximum over the element's
// nodes.  Smoothing: the elemental field is averaged to the master vertices,
// each element takes the mean of its vertices, the result is averaged to
// the vertices again, and the vertex field is interpolated multilinearly to
// the solution nodes.  Every average runs over a fixed list in ascending
// order, so the field is bitwise reproducible.
#pragma once

namespace hdg {

template <int D>
__device__ __forceinline__ void velocity_gradient(const double* u, const double (*q)[D + 2], double (&v)[D],
                                                  double (&G)[D][D]) {
    const double rho = u[0];
    for (int i = 0; i < D; ++i) v[i] = u[1 + i] / rho;
    for (int i = 0; i < D; ++i)
        for (int j = 0; j < D; ++j) G[i][j] = (q[j][1 + i] - v[i] * q[j][0]) / rho;
}

template <int D>
__device__ __forceinline__ double vorticity_sq(const double (&G)[D][D]) {
    if (D == 2) {
        const double w = G[1][0] - G[0][1];
        return w * w;
    }
    const double a = G[2 % D][1] - G[1][2 % D], b = G[0][2 % D] - G[2 % D][0], c = G[1][0] - G[0][1];
    return a * a + b * b + c * c;
}

template <class C, int NTH>
__global__ void __launch_bounds__(NTH) k_av_raw(const double* __restrict__ U, const double* __restrict__ Q,
                                                double gamma, double c_av, double sq_hk, double s_max,
                                                double* __restrict__ raw) {
    constexpr int D = C::D, M = C::M, NP = C::NP;
    __shared__ double red[NTH / 32];
    const int tid = threadIdx.x;
    const int64_t e = blockIdx.x;
    double best = 0.0;
    for (int i = tid; i < NP; i += NTH) {
        double u[M], q[D][M];
        for (int a = 0; a < M; ++a) {
            u[a] = U[(e * M + a) * NP + i];
            for (int j = 0; j < D; ++j) q[j][a] = Q[((e * D + j) * M + a) * NP + i];
        }
        double v[D], G[D][D];
        velocity_gradient<D>(u, q, v, G);
        double div = 0.0, vv = 0.0;
        for (int j = 0; j < D; ++j) { div += G[j][j]; vv += v[j] * v[j]; }
        const double pr = (gamma - 1.0) * (u[M - 1] - 0.5 * u[0] * vv);
        const double c = sqrt(gamma * pr / u[0]);
        const double lc = fmax(-div, 0.0), om2 = vorticity_sq<D>(G);
        const double s = sq_hk * lc / c * (lc * lc) / (lc * lc + om2 + 1e-12);
        best = fmax(best, c_av * fmin(fmax(s, 0.0), s_max));
    }
    for (int off = 16; off > 0; off >>= 1) best = fmax(best, __shfl_down_sync(0xffffffffu, best, off));
    if ((tid & 31) == 0) red[tid >> 5] = best;
    __syncthreads();
    if (tid == 0) {
        double b = red[0];
        for (int w = 1; w < NTH / 32; ++w) b = fmax(b, red[w]);
        raw[e] = b;
    }
}

// vertex average of an elemental field (ascending element order)
__global__ void k_av_vertex(const double* __restrict__ fe, const int32_t* __restrict__ vrow,
                            const int32_t* __restrict__ vcol, double* __restrict__ fv, int64_t V);
// element mean of its corner values
__global__ void k_av_emean(const double* __restrict__ fv, const int32_t* __restrict__ ev, int nc,
                           double* __restrict__ fe, int64_t E);

struct Nodes1 { double t[4]; };            // 1-D GLL nodes mapped to [0, 1]

template <class C>
__global__ void k_av_interp(const double* __restrict__ fv, const int32_t* __restrict__ ev, Nodes1 nd,
                            double* __restrict__ nu, int64_t E) {
    constexpr int D = C::D, NP = C::NP, N1 = C::P + 1, NC = 1 << D;
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= E * NP) return;
    const int64_t e = idx / NP;
    const int i = (int)(idx - e * NP);
    int ii[D];
    int rem = i;
    for (int r = 0; r < D; ++r) { ii[r] = rem % N1; rem /= N1; }
    double s = 0.0;
    for (int c = 0; c < NC; ++c) {
        double w = 1.0;
        for (int r = 0; r < D; ++r) w *= ((c >> r) & 1) ? nd.t[ii[r]] : 1.0 - nd.t[ii[r]];
        s += w * fv[ev[e * NC + c]];
    }
    nu[idx] = s;
}

// per element: int rho v.v, int mu~ |curl v|^2, int mu~ (div v)^2, int 1 (volume quadrature)
template <class C, int NTH>
__global__ void __launch_bounds__(NTH) k_diag(const double* __restrict__ U, const double* __restrict__ Q,
                                              DeviceTables T, const double* __restrict__ geog, PhysT<double> ph,
                                              double* __restrict__ part) {
    constexpr int D = C::D, M = C::M, NP = C::NP, NQ = C::NQ;
    constexpr int GEO = Geo<D>::N;
    __shared__ double sU[C::NU], sQ[C::NQV];
    __shared__ double red[4][NTH / 32];
    const int tid = threadIdx.x;
    const int64_t e = blockIdx.x;
    for (int i = tid; i < C::NU; i += NTH) sU[i] = U[e * C::NU + i];
    for (int i = tid; i < C::NQV; i += NTH) sQ[i] = Q[e * C::NQV + i];
    __syncthreads();
    const double detJ = geog[e * GEO];
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
    for (int g = tid; g < NQ; g += NTH) {
        double u[M], q[D][M];
        for (int a = 0; a < M; ++a) {
            u[a] = 0.0;
            for (int j = 0; j < D; ++j) q[j][a] = 0.0;
        }
        for (int n = 0; n < NP; ++n) {
            const double w = T.phi[g * NP + n];
            for (int a = 0; a < M; ++a) {
                u[a] += w * sU[a * NP + n];
                for (int j = 0; j < D; ++j) q[j][a] += w * sQ[(j * M + a) * NP + n];
            }
        }
        double v[D], G[D][D];
        velocity_gradient<D>(u, q, v, G);
        double div = 0.0, vv = 0.0;
        for (int j = 0; j < D; ++j) { div += G[j][j]; vv += v[j] * v[j]; }
        const double eint = u[M - 1] / u[0] - 0.5 * vv;
        const double mu = viscosity<double, double>(eint, ph) / ph.re_inv;   // mu~
        const double wJ = T.wq[g] * detJ;
        acc[0] += wJ * u[0] * vv;
        acc[1] += wJ * mu * vorticity_sq<D>(G);
        acc[2] += wJ * mu * div * div;
        acc[3] += wJ;
    }
    for (int k = 0; k < 4; ++k) {
        double s = acc[k];
        for (int off = 16; off > 0; off >>= 1) s += __shfl_down_sync(0xffffffffu, s, off);
        if ((tid & 31) == 0) red[k][tid >> 5] = s;
    }
    __syncthreads();
    if (tid < 4) {
        double s = 0.0;
        for (int w = 0; w < NTH / 32; ++w) s += red[tid][w];
        part[e * 4 + tid] = s;
    }
}

// totals of the [E][4] partials in a fixed order (one block)
__global__ void k_diag_sum(const double* __restrict__ part, int64_t E, double* __restrict__ out);

template <int D, int P>
int run_av_field(hdg_ctx* h, const double* U, const double* Q, double c_av, double h_m, double s_max, double* nu) {
    using C = Cfg<D, P>;
    const int64_t V = (int64_t)h->av_vrow.size() - 1;
    const int nc = 1 << D;
    k_av_raw<C, 128><<<(unsigned)h->E, 128, 0, h->stream>>>(U, Q, h->phys.gamma, c_av, sqrt(h_m / P), s_max,
                                                           h->d_ave);
    for (int pass = 0; pass < 2; ++pass) {
        k_av_vertex<<<(unsigned)((V + 255) / 256), 256, 0, h->stream>>>(h->d_ave, h->d_avvrow, h->d_avvcol,
                                                                        h->d_avv, V);
        if (pass == 0)
            k_av_emean<<<(unsigned)((h->E + 255) / 256), 256, 0, h->stream>>>(h->d_avv, h->d_avev, nc, h->d_ave,
                                                                              h->E);
    }
    Nodes1 nd{};
    for (int i = 0; i <= P; ++i) nd.t[i] = 0.5 * (h->ref.nodes1[i] + 1.0);
    const int64_t n = h->E * C::NP;
    k_av_interp<C><<<(unsigned)((n + 255) / 256), 256, 0, h->stream>>>(h->d_avv, h->d_avev, nd, nu, h->E);
    HDG_CK(cudaGetLastError());
    return HDG_OK;
}

template <int D, int P>
int run_diagnostics(hdg_ctx* h, const double* U, const double* Q) {
    using C = Cfg<D, P>;
    k_diag<C, 128><<<(unsigned)h->E, 128, 0, h->stream>>>(U, Q, h->tab, h->d_geo, phys_t<double>(h->phys),
                                                         h->d_diag);
    k_diag_sum<<<1, 256, 0, h->stream>>>(h->d_diag, h->E, h->d_diag + 4 * h->E);
    HDG_CK(cudaGetLastError());
    return HDG_OK;
}

}  // namespace hdg
