// Compressible Navier-Stokes fluxes on the device (Sec. 2.1), generic in the
// scalar type: S = double or float for values, DirT<S> (value + one tangent)
// for directional derivatives with respect to the state.  All constants come
// from PhysT<S>, so a float evaluation never promotes to double.
#pragma once

#include "common.h"

namespace hdg {

template <class S>
struct DirT {
    S v, t;  // value, tangent
};
template <class S> __device__ __forceinline__ DirT<S> operator+(DirT<S> a, DirT<S> b) { return {a.v + b.v, a.t + b.t}; }
template <class S> __device__ __forceinline__ DirT<S> operator-(DirT<S> a, DirT<S> b) { return {a.v - b.v, a.t - b.t}; }
template <class S> __device__ __forceinline__ DirT<S> operator*(DirT<S> a, DirT<S> b) { return {a.v * b.v, a.t * b.v + a.v * b.t}; }
template <class S> __device__ __forceinline__ DirT<S> operator+(DirT<S> a, S b) { return {a.v + b, a.t}; }
template <class S> __device__ __forceinline__ DirT<S> operator-(DirT<S> a, S b) { return {a.v - b, a.t}; }
template <class S> __device__ __forceinline__ DirT<S> operator*(DirT<S> a, S b) { return {a.v * b, a.t * b}; }
template <class S> __device__ __forceinline__ DirT<S> operator*(S b, DirT<S> a) { return {a.v * b, a.t * b}; }
template <class S> __device__ __forceinline__ DirT<S> recip(DirT<S> a) { S r = S(1) / a.v; return {r, -a.t * r * r}; }
__device__ __forceinline__ double recip(double a) { return 1.0 / a; }
__device__ __forceinline__ float recip(float a) { return 1.0f / a; }
template <class S> __device__ __forceinline__ DirT<S> dsqrt(DirT<S> a) { S s = sqrt(a.v); return {s, S(0.5) * a.t / s}; }
__device__ __forceinline__ double dsqrt(double a) { return sqrt(a); }
__device__ __forceinline__ float dsqrt(float a) { return sqrtf(a); }
template <class S> __device__ __forceinline__ DirT<S> zero_like(DirT<S>) { return {S(0), S(0)}; }
__device__ __forceinline__ double zero_like(double) { return 0.0; }
__device__ __forceinline__ float zero_like(float) { return 0.0f; }

template <class S> __device__ __forceinline__ DirT<S> dabs(DirT<S> a) { return a.v < S(0) ? DirT<S>{-a.v, -a.t} : a; }
__device__ __forceinline__ double dabs(double a) { return fabs(a); }
__device__ __forceinline__ float dabs(float a) { return fabsf(a); }

using Dir = DirT<double>;

// Physical constants in the evaluation type.
template <class S>
struct PhysT {
    S gm1;          // gamma - 1
    S re_inv;       // 1 / Re
    S kap;          // gamma / Pr (heat flux (gamma mu / Pr) d e)
    S c1_re;        // C1 / Re (Sutherland)
    S suth_s;       // S~
    S tmul;         // gamma (gamma - 1) M^2: T~ = tmul e
    S half, two_thirds;
    int visc_law;
};

template <class S>
inline PhysT<S> phys_t(const Phys& p) {
    PhysT<S> q;
    q.gm1 = (S)(p.gamma - 1.0);
    q.re_inv = (S)(1.0 / p.re);
    q.kap = (S)(p.gamma / p.pr);
    q.c1_re = (S)(p.c1 / p.re);
    q.suth_s = (S)p.s;
    q.tmul = (S)(p.gamma * (p.gamma - 1.0) * p.mach * p.mach);
    q.half = (S)0.5;
    q.two_thirds = (S)(2.0 / 3.0);
    q.visc_law = p.visc_law;
    return q;
}

// Effective viscosity mu~(T~)/Re (eq. sutherland in the nondimensional form of
// eq. tgv-sutherland), T~ = gamma (gamma - 1) M^2 e.
template <class T, class S>
__device__ __forceinline__ T viscosity(T e, const PhysT<S>& ph) {
    if (ph.visc_law == 0) return zero_like(e) + ph.re_inv;
    T Tt = e * ph.tmul;
    return ph.c1_re * Tt * dsqrt(Tt) * recip(Tt + ph.suth_s);
}

// Convective flux f^c_j (eq. convective-flux), component a in direction k.
template <int D, class T, class S>
__device__ __forceinline__ void conv_flux(const T* u, const PhysT<S>& ph, T (*F)[D]) {
    constexpr int M = D + 2;
    T irho = recip(u[0]);
    T v[D];
    T kin = zero_like(u[0]);
    for (int i = 0; i < D; ++i) { v[i] = u[1 + i] * irho; kin = kin + v[i] * u[1 + i]; }
    T p = (u[M - 1] - kin * ph.half) * ph.gm1;
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
template <int D, class T, class S>
__device__ __forceinline__ void visc_flux(const T* u, const S (*q)[D], S nu, const PhysT<S>& ph, T (*F)[D]) {
    constexpr int M = D + 2;
    T irho = recip(u[0]);
    T v[D];
    T kin = zero_like(u[0]);
    for (int i = 0; i < D; ++i) { v[i] = u[1 + i] * irho; kin = kin + v[i] * v[i]; }
    T E = u[M - 1] * irho;
    T e = E - kin * ph.half;
    T mu = viscosity(e, ph);
    T dv[D][D];
    T dE[D];
    for (int j = 0; j < D; ++j) {
        for (int i = 0; i < D; ++i) dv[i][j] = (v[i] * (-q[0][j]) + q[1 + i][j]) * irho;
        dE[j] = (E * (-q[0][j]) + q[M - 1][j]) * irho;
    }
    T div = dv[0][0];
    for (int i = 1; i < D; ++i) div = div + dv[i][i];
    for (int j = 0; j < D; ++j) {
        T de = dE[j];
        for (int i = 0; i < D; ++i) de = de - v[i] * dv[i][j];
        T fe = de * mu * ph.kap;
        F[0][j] = zero_like(u[0]) + nu * q[0][j];
        for (int i = 0; i < D; ++i) {
            T tij = (dv[i][j] + dv[j][i]) * mu;
            if (i == j) tij = tij - div * mu * ph.two_thirds;
            F[1 + i][j] = tij + nu * q[1 + i][j];
            fe = fe + v[i] * tij;
        }
        F[M - 1][j] = fe + nu * q[M - 1][j];
    }
}

// State-dependent stabilization (an option of the face stabilization of eq.
// num-flux-hdg): tau = |vhat . n| + chat + mu(That) / h, with n the unit normal
// and h_inv = 1 / h the inverse element length scale |K|^{-1/d}; T = DirT gives
// its directional derivative with respect to uhat.
template <int D, class T, class S>
__device__ __forceinline__ T stab_tau(const T* uh, const S* nh, S h_inv, const PhysT<S>& ph) {
    constexpr int M = D + 2;
    T irho = recip(uh[0]);
    T vn = zero_like(uh[0]);
    T kin = zero_like(uh[0]);
    for (int k = 0; k < D; ++k) {
        T v = uh[1 + k] * irho;
        vn = vn + v * nh[k];
        kin = kin + v * uh[1 + k];
    }
    T rhoe = uh[M - 1] - kin * ph.half;            // rho e = rho E - rho |v|^2 / 2
    T c = dsqrt(rhoe * ph.gm1 * (ph.gm1 + S(1)) * irho);
    return dabs(vn) + c + viscosity(rhoe * irho, ph) * h_inv;
}

}  // namespace hdg
