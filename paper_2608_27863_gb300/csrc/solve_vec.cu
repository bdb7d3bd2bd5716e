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

__global__ void k_dot_final(const double* part, int nparts, double* out, int take_sqrt) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        double t = 0.0;
        for (int i = 0; i < nparts; ++i) t += part[i];
        *out = take_sqrt ? sqrt(t) : t;
    }
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

}  // namespace hdg
