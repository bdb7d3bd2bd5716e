// Compressible Navier-Stokes fluxes on the device (Sec. 2.1), generic in the
// scalar type so that one code path gives values (double) and directional
// derivatives with respect to the state (Dir: value + one tangent).
#pragma once

#include "common.h"

namespace hdg {

struct Dir {
    double v, t;  // value, tangent
};
__device__ __forceinline__ Dir operator+(Dir a, Dir b) { return {a.v + b.v, a.t + b.t}; }
__device__ __forceinline__ Dir operator-(Dir a, Dir b) { return {a.v - b.v, a.t - b.t}; }
__device__ __forceinline__ Dir operator*(Dir a, Dir b) { return {a.v * b.v, a.t * b.v + a.v * b.t}; }
__device__ __forceinline__ Dir operator+(Dir a, double b) { return {a.v + b, a.t}; }
__device__ __forceinline__ Dir operator-(Dir a, double b) { return {a.v - b, a.t}; }
__device__ __forceinline__ Dir operator*(Dir a, double b) { return {a.v * b, a.t * b}; }
__device__ __forceinline__ Dir operator*(double b, Dir a) { return {a.v * b, a.t * b}; }
__device__ __forceinline__ Dir recip(Dir a) { double r = 1.0 / a.v; return {r, -a.t * r * r}; }
__device__ __forceinline__ double recip(double a) { return 1.0 / a; }
__device__ __forceinline__ Dir dsqrt(Dir a) { double s = sqrt(a.v); return {s, 0.5 * a.t / s}; }
__device__ __forceinline__ double dsqrt(double a) { return sqrt(a); }
__device__ __forceinline__ Dir zero_like(Dir) { return {0.0, 0.0}; }
__device__ __forceinline__ double zero_like(double) { return 0.0; }

// Effective viscosity mu~(T~)/Re with T~ = gamma (gamma - 1) M^2 e
// (eq. sutherland in the nondimensional form of eq. tgv-sutherland).
template <class T>
__device__ __forceinline__ T viscosity(T e, const Phys& ph) {
    if (ph.visc_law == 0) return zero_like(e) + 1.0 / ph.re;
    T Tt = e * (ph.gamma * (ph.gamma - 1.0) * ph.mach * ph.mach);
    return (ph.c1 / ph.re) * Tt * dsqrt(Tt) * recip(Tt + ph.s);
}

// Convective flux f^c_j (eq. convective-flux), component a in direction k.
template <int D, class T>
__device__ __forceinline__ void conv_flux(const T* u, const Phys& ph, T (*F)[D]) {
    constexpr int M = D + 2;
    T irho = recip(u[0]);
    T v[D];
    T kin = zero_like(u[0]);
    for (int i = 0; i < D; ++i) { v[i] = u[1 + i] * irho; kin = kin + v[i] * u[1 + i]; }
    T p = (u[M - 1] - kin * 0.5) * (ph.gamma - 1.0);
    for (int k = 0; k < D; ++k) {
        F[0][k] = u[1 + k];
        for (int i = 0; i < D; ++i) {
            F[1 + i][k] = u[1 + i] * v[k];
            if (i == k) F[1 + i][k] = F[1 + i][k] + p;
        }
        F[M - 1][k] = (u[M - 1] + p) * v[k];
    }
}

// Viscous plus artificial-viscosity flux f^v_j + nu q_j (eqs. viscous-flux,
// stress-heat, thermal-conductivity, av-total); linear in q.
template <int D, class T>
__device__ __forceinline__ void visc_flux(const T* u, const double (*q)[D], double nu, const Phys& ph,
                                          T (*F)[D]) {
    constexpr int M = D + 2;
    T irho = recip(u[0]);
    T v[D];
    T kin = zero_like(u[0]);
    for (int i = 0; i < D; ++i) { v[i] = u[1 + i] * irho; kin = kin + v[i] * v[i]; }
    T E = u[M - 1] * irho;
    T e = E - kin * 0.5;
    T mu = viscosity(e, ph);
    T dv[D][D];
    T dE[D];
    for (int j = 0; j < D; ++j) {
        for (int i = 0; i < D; ++i) dv[i][j] = (v[i] * (-q[0][j]) + q[1 + i][j]) * irho;
        dE[j] = (E * (-q[0][j]) + q[M - 1][j]) * irho;
    }
    T div = dv[0][0];
    for (int i = 1; i < D; ++i) div = div + dv[i][i];
    const double kap = ph.gamma / ph.pr;
    for (int j = 0; j < D; ++j) {
        T de = dE[j];
        for (int i = 0; i < D; ++i) de = de - v[i] * dv[i][j];
        T fe = de * mu * kap;
        F[0][j] = zero_like(u[0]) + nu * q[0][j];
        for (int i = 0; i < D; ++i) {
            T tij = (dv[i][j] + dv[j][i]) * mu;
            if (i == j) tij = tij - div * mu * (2.0 / 3.0);
            F[1 + i][j] = tij + nu * q[1 + i][j];
            fe = fe + v[i] * tij;
        }
        F[M - 1][j] = fe + nu * q[M - 1][j];
    }
}

}  // namespace hdg
