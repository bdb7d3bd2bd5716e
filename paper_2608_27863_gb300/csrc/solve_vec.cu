// FP64 vector kernels for the trace-space Krylov solver.  Reductions use a
// fixed grid and a fixed combination order, so results are bitwise
// reproducible from run to run.
#include "solve.cuh"

namespace hdg {

__global__ void k_dot_part(const double* x, const double* y, int64_t n, double* part) {
    __shared__ double red[32];
    double s = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        s = fma(x[i], y[i], s);
    for (int off = 16; off > 0; off >>= 1) s += __shfl_down_sync(0xffffffffu, s, off);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
        part[blockIdx.x] = t;
    }
}

// sum of part[0 .. nparts) by one warp: lane l adds parts l, l + 32, ... in
// order, then a fixed shuffle tree (stride-8 parts for the Gram-Schmidt partials)
__device__ __forceinline__ double warp_sum_parts(const double* part, int nparts, int stride) {
    const int lane = threadIdx.x & 31;
    double t = 0.0;
    for (int b = lane; b < nparts; b += 32) t += part[(size_t)b * stride];
    for (int off = 16; off > 0; off >>= 1) t += __shfl_down_sync(0xffffffffu, t, off);
    return t;
}

__global__ void k_dot_final(const double* part, int nparts, double* out, int take_sqrt) {
    if (blockIdx.x == 0 && threadIdx.x < 32) {
        const double t = warp_sum_parts(part, nparts, 1);
        if (threadIdx.x == 0) *out = take_sqrt ? sqrt(t) : t;
    }
}

// Partial sums of the dot products of w with vectors 8 y .. 8 y + 7 of V
// (y = blockIdx.y; fewer in the last group), one set per block x:
// part[y][block x][8].  All groups run in one launch.
__global__ void k_mdot_part(const double* V, int64_t ldv, int k, const double* w, int64_t n, double* part) {
    __shared__ double red[8][8];
    const int j0 = 8 * blockIdx.y;
    const int nv = min(8, k - j0);
    double acc[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) acc[q] = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double wi = w[i];
#pragma unroll
        for (int q = 0; q < 8; ++q)
            if (q < nv) acc[q] = fma(V[(size_t)(j0 + q) * ldv + i], wi, acc[q]);
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        double s = acc[q];
        for (int off = 16; off > 0; off >>= 1) s += __shfl_down_sync(0xffffffffu, s, off);
        if (lane == 0) red[q][warp] = s;
    }
    __syncthreads();
    if (threadIdx.x < 8) {
        double t = 0.0;
        for (int w2 = 0; w2 < (int)(blockDim.x >> 5); ++w2) t += red[threadIdx.x][w2];
        part[((size_t)blockIdx.y * gridDim.x + blockIdx.x) * 8 + threadIdx.x] = t;
    }
}

// out[j] = sum over blocks of the partials of vector j, one warp per j < k
__global__ void k_mdot_final(const double* part, int nparts, int k, double* out) {
    const int j = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    if (j < k) {
        const double t = warp_sum_parts(part + (size_t)(j >> 3) * nparts * 8 + (j & 7), nparts, 8);
        if ((threadIdx.x & 31) == 0) out[j] = t;
    }
}

// w -= sum_j coef[j] V_j (j ascending; eight basis vectors loaded ahead)
__global__ void k_msub(const double* V, int64_t ldv, const double* coef, int k, double* w, int64_t n) {
    __shared__ double cf[kMaxBasis];
    for (int j = threadIdx.x; j < k; j += blockDim.x) cf[j] = coef[j];
    __syncthreads();
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        double s = w[i];
        int j = 0;
        for (; j + 8 <= k; j += 8) {
            double v[8];
#pragma unroll
            for (int q = 0; q < 8; ++q) v[q] = V[(size_t)(j + q) * ldv + i];
#pragma unroll
            for (int q = 0; q < 8; ++q) s = fma(-cf[j + q], v[q], s);
        }
        for (; j < k; ++j) s = fma(-cf[j], V[(size_t)j * ldv + i], s);
        w[i] = s;
    }
}

// a[i] += b[i], i < k (small vectors)
__global__ void k_vadd(double* a, const double* b, int k) {
    for (int i = threadIdx.x; i < k; i += blockDim.x) a[i] += b[i];
}

__global__ void k_axpy_dev(const double* coef, double sign, const double* x, double* y, int64_t n) {
    const double a = sign * (*coef);
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        y[i] = fma(a, x[i], y[i]);
}

__global__ void k_scale_dev(const double* x, const double* div, double* y, int64_t n) {
    const double s = 1.0 / (*div);
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        y[i] = x[i] * s;
}

__global__ void k_axpby(double a, const double* x, double b, double* y, int64_t n) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        y[i] = a * x[i] + b * y[i];
}

__global__ void k_combine(const double* V, int64_t ldv, const double* coef, int k, double* x, int64_t n) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        double s = x[i];
        for (int j = 0; j < k; ++j) s = fma(coef[j], V[(size_t)j * ldv + i], s);
        x[i] = s;
    }
}

__global__ void k_sum_parts(const double* p1, int64_t n1, const double* p2, int64_t n2, double* out) {
    __shared__ double red[2][32];
    double a = 0.0, b = 0.0;
    for (int64_t i = threadIdx.x; i < n1; i += blockDim.x) a += p1[i];
    for (int64_t i = threadIdx.x; i < n2; i += blockDim.x) b += p2[i];
    for (int off = 16; off > 0; off >>= 1) {
        a += __shfl_down_sync(0xffffffffu, a, off);
        b += __shfl_down_sync(0xffffffffu, b, off);
    }
    if ((threadIdx.x & 31) == 0) { red[0][threadIdx.x >> 5] = a; red[1][threadIdx.x >> 5] = b; }
    __syncthreads();
    if (threadIdx.x == 0) {
        double s1 = 0.0, s2 = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) { s1 += red[0][w]; s2 += red[1][w]; }
        out[0] = sqrt(s1 + s2);
        out[1] = sqrt(s1);
        out[2] = sqrt(s2);
    }
}

// y = x / div, or 0 when div is zero (lucky breakdown of the Arnoldi process)
__global__ void k_scale_safe(const double* x, const double* div, double* y, int64_t n) {
    const double d = *div;
    const double s = d != 0.0 ? 1.0 / d : 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        y[i] = x[i] * s;
}

// Device-side Givens QR of the Hessenberg matrix, one column per call (single thread):
// hcol[0..j+1] is column j of H; R [m][m] upper triangle, cs/sn rotations, gv the rotated rhs.
__global__ void k_givens_step(const double* hcol, int j, int m, double* R, double* cs, double* sn, double* gv) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    double h[2];
    double col[512];
    for (int i = 0; i <= j + 1 && i < 512; ++i) col[i] = hcol[i];
    for (int i = 0; i < j; ++i) {
        double t = cs[i] * col[i] + sn[i] * col[i + 1];
        col[i + 1] = -sn[i] * col[i] + cs[i] * col[i + 1];
        col[i] = t;
    }
    h[0] = col[j];
    h[1] = col[j + 1];
    const double den = hypot(h[0], h[1]);
    cs[j] = den > 0.0 ? h[0] / den : 1.0;
    sn[j] = den > 0.0 ? h[1] / den : 0.0;
    col[j] = den;
    for (int i = 0; i <= j; ++i) R[(size_t)i * m + j] = col[i];
    gv[j + 1] = -sn[j] * gv[j];
    gv[j] = cs[j] * gv[j];
}

// y = R^{-1} gv (k x k upper triangle, zero diagonals skipped)
__global__ void k_backsolve(const double* R, const double* gv, int k, int m, double* y) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    for (int i = k - 1; i >= 0; --i) {
        double s = gv[i];
        for (int l = i + 1; l < k; ++l) s -= R[(size_t)i * m + l] * y[l];
        const double d = R[(size_t)i * m + i];
        y[i] = d != 0.0 ? s / d : 0.0;
    }
}

__global__ void k_set_first(const double* beta, double* gv, int m) {
    for (int i = threadIdx.x; i <= m; i += blockDim.x) gv[i] = (i == 0) ? *beta : 0.0;
}

// append the residual norm to a device-side history
__global__ void k_hist_push(const double* norms, double* hist, int* counter, int cap) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        int k = *counter;
        if (k < cap) hist[k] = norms[0];
        *counter = k + 1;
    }
}

// z = a x + b y + c z
__global__ void k_lincomb3(double a, const double* x, double b, const double* y, double c, double* z, int64_t n) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        z[i] = a * x[i] + b * y[i] + c * z[i];
}

// Reduced-basis window: partial sums of the Gram matrix Z^T Z (pairs k <= l)
// and of Z^T g over row tiles; thread t of a block owns quantity t.
__global__ void k_rb_gram_part(const double* Z, int nb, const double* g, int64_t n, double* part) {
    constexpr int TR = 128;
    __shared__ double zs[kRbMax][TR];
    __shared__ double gs[TR];
    const int t = threadIdx.x;
    const int npair = nb * (nb + 1) / 2;
    int k = -1, l = -1;                     // quantity t: pair (k, l) with k <= l, or (k, g) when l == nb
    if (t < npair) {
        int r = t;
        k = 0;
        while (r >= nb - k) { r -= nb - k; ++k; }
        l = k + r;
    } else if (t < npair + nb) {
        k = t - npair;
        l = nb;
    }
    double acc = 0.0;
    for (int64_t r0 = (int64_t)blockIdx.x * TR; r0 < n; r0 += (int64_t)gridDim.x * TR) {
        __syncthreads();
        for (int idx = t; idx < (nb + 1) * TR; idx += blockDim.x) {
            const int c = idx / TR, i = idx - c * TR;
            const int64_t row = r0 + i;
            const double v = row < n ? (c < nb ? Z[(size_t)c * n + row] : g[row]) : 0.0;
            if (c < nb) zs[c][i] = v; else gs[i] = v;
        }
        __syncthreads();
        if (k >= 0) {
            const double* b = (l < nb) ? zs[l] : gs;
            for (int i = 0; i < TR; ++i) acc = fma(zs[k][i], b[i], acc);
        }
    }
    part[(size_t)blockIdx.x * blockDim.x + t] = acc;
}

// Sums the partials in block order, then solves the normal equations
// (Z^T Z) c = Z^T g by Cholesky with diagonal pivoting; pivots below
// 1e-13 of the largest diagonal are dropped (their coefficients are zero), so
// an empty or rank-deficient window gives a finite least-squares solution.
__global__ void k_rb_solve(const double* part, int nparts, int nb, double* c) {
    __shared__ double q[kRbMax * (kRbMax + 1) / 2 + kRbMax];
    const int t = threadIdx.x;
    const int nq = nb * (nb + 1) / 2 + nb;
    if (t < nq) {
        double s = 0.0;
        for (int b = 0; b < nparts; ++b) s += part[(size_t)b * blockDim.x + t];
        q[t] = s;
    }
    __syncthreads();
    if (t != 0) return;
    double G[kRbMax][kRbMax], rhs[kRbMax], y[kRbMax];
    int pidx[kRbMax];
    int idx = 0;
    for (int k = 0; k < nb; ++k)
        for (int l = k; l < nb; ++l) { G[k][l] = q[idx]; G[l][k] = q[idx]; ++idx; }
    for (int k = 0; k < nb; ++k) { rhs[k] = q[idx + k]; pidx[k] = k; c[k] = 0.0; }
    double dmax = 0.0;
    for (int k = 0; k < nb; ++k) dmax = fmax(dmax, G[k][k]);
    int r = 0;                               // accepted pivots
    for (; r < nb; ++r) {
        int best = r;
        for (int i = r + 1; i < nb; ++i)
            if (G[pidx[i]][pidx[i]] > G[pidx[best]][pidx[best]]) best = i;
        const int tmp = pidx[r]; pidx[r] = pidx[best]; pidx[best] = tmp;
        const int pr = pidx[r];
        const double d = G[pr][pr];
        if (!(d > 1e-13 * dmax)) break;
        const double ld = sqrt(d);
        G[pr][pr] = ld;
        for (int i = r + 1; i < nb; ++i) G[pidx[i]][pr] /= ld;     // column r of L, stored at (pidx[i], pr)
        for (int i = r + 1; i < nb; ++i)
            for (int j = r + 1; j <= i; ++j) {
                const double v = G[pidx[i]][pidx[j]] - G[pidx[i]][pr] * G[pidx[j]][pr];
                G[pidx[i]][pidx[j]] = v;
                G[pidx[j]][pidx[i]] = v;
            }
    }
    for (int i = 0; i < r; ++i) {            // L y = P rhs
        double s = rhs[pidx[i]];
        for (int j = 0; j < i; ++j) s -= G[pidx[i]][pidx[j]] * y[j];
        y[i] = s / G[pidx[i]][pidx[i]];
    }
    for (int i = r - 1; i >= 0; --i) {       // L^T x = y
        double s = y[i];
        for (int j = i + 1; j < r; ++j) s -= G[pidx[j]][pidx[i]] * y[j];
        y[i] = s / G[pidx[i]][pidx[i]];
    }
    for (int i = 0; i < r; ++i) c[pidx[i]] = y[i];
}

// insert (w, z) into slot head[0] of the window
__global__ void k_rb_store(const double* w, const double* z, double* W, double* Z, const int* head, int64_t n) {
    const int slot = head[0];
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        W[(size_t)slot * n + i] = w[i];
        Z[(size_t)slot * n + i] = z[i];
    }
}

__global__ void k_rb_advance(int* head, int nb) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        head[0] = (head[0] + 1) % nb;
        head[1] = min(head[1] + 1, nb);
    }
}

__global__ void k_av_vertex(const double* __restrict__ fe, const int32_t* __restrict__ vrow,
                            const int32_t* __restrict__ vcol, double* __restrict__ fv, int64_t V) {
    const int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= V) return;
    double s = 0.0;
    for (int32_t k = vrow[v]; k < vrow[v + 1]; ++k) s += fe[vcol[k]];
    const int32_t n = vrow[v + 1] - vrow[v];
    fv[v] = n > 0 ? s / n : 0.0;
}

__global__ void k_av_emean(const double* __restrict__ fv, const int32_t* __restrict__ ev, int nc,
                           double* __restrict__ fe, int64_t E) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= E) return;
    double s = 0.0;
    for (int c = 0; c < nc; ++c) s += fv[ev[e * nc + c]];
    fe[e] = s / nc;
}

__global__ void k_diag_sum(const double* __restrict__ part, int64_t E, double* __restrict__ out) {
    __shared__ double red[4][256];
    const int t = threadIdx.x;
    double a[4] = {0.0, 0.0, 0.0, 0.0};
    for (int64_t e = t; e < E; e += blockDim.x)
        for (int k = 0; k < 4; ++k) a[k] += part[e * 4 + k];
    for (int k = 0; k < 4; ++k) red[k][t] = a[k];
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (t < w)
            for (int k = 0; k < 4; ++k) red[k][t] += red[k][t + w];
        __syncthreads();
    }
    if (t < 4) out[t] = red[t][0];
}

__global__ void k_to_f32(const double* x, float* y, int64_t n) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        y[i] = (float)x[i];
}

}  // namespace hdg
