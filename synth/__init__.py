"""Seeded synthetic inputs for the HDG linearize + condense path.

This module produces meshes (structured boxes of quadrilaterals or hexahedra),
conserved-variable states and random draws.  It holds none of the method's
arithmetic: no quadrature, no fluxes, no face connectivity, no condensation.
Both the FP64 oracle tests and the CUDA library consume exactly what it returns,
so the two sides share inputs and nothing else.

Conventions (the data interface of the library, ``include/hdg.h``):

* element vertices in tensor order, vertex ``c = c1 + 2 c2 + 4 c3`` sits at
  reference corner ``xi_r = -1`` for ``c_r = 0`` and ``+1`` for ``c_r = 1``;
* element nodes are the tensor Gauss-Lobatto points of degree p, node
  ``j = j1 + (p+1) j2 + (p+1)^2 j3`` (x fastest), placed by the multilinear
  map of the vertices;
* conserved state ``u = [rho, rho v_1..rho v_d, rho E]`` (Sec. 2.1, state vector);
* ``U[E][m][Np]``, ``Q[E][d][m][Np]`` with ``Q[e][k][a] = d u_a / d x_k``,
  trace ``UH[F][m][Nfp]``, artificial viscosity ``nu[E][Np]`` (nodal).

Random numbers come from SplitMix64 (Steele, Lea, Flood 2014), used as a
counter-based generator: draw ``i`` of stream ``seed`` is the SplitMix64 output
mix of ``seed + (i + 1) * 0x9E3779B97F4A7C15``.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)


# ----------------------------------------------------------------------------
# SplitMix64 counter-based stream
# ----------------------------------------------------------------------------
def splitmix64(seed: int, n: int, offset: int = 0) -> np.ndarray:
    """Draws ``offset .. offset+n-1`` of the SplitMix64 stream ``seed`` (uint64)."""
    with np.errstate(over="ignore"):
        i = np.arange(offset + 1, offset + n + 1, dtype=np.uint64)
        z = np.uint64(seed) + i * _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        z = z ^ (z >> np.uint64(31))
    return z


def uniform(seed: int, n: int, offset: int = 0) -> np.ndarray:
    """Uniform doubles in [0, 1) from the top 53 bits of each draw."""
    return (splitmix64(seed, n, offset) >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


def normal(seed: int, n: int) -> np.ndarray:
    """Standard normal draws by Box-Muller on consecutive uniform pairs."""
    k = (n + 1) // 2
    u = uniform(seed, 2 * k)
    u1 = 1.0 - u[0::2]  # (0, 1]
    u2 = u[1::2]
    r = np.sqrt(-2.0 * np.log(u1))
    z = np.concatenate([r * np.cos(2 * np.pi * u2), r * np.sin(2 * np.pi * u2)])
    return z[:n]


# ----------------------------------------------------------------------------
# Gauss-Lobatto points (node placement only)
# ----------------------------------------------------------------------------
def gll_points(p: int) -> np.ndarray:
    """Gauss-Lobatto points of degree p on [-1, 1] (closed forms, p <= 4)."""
    if p == 1:
        return np.array([-1.0, 1.0])
    if p == 2:
        return np.array([-1.0, 0.0, 1.0])
    if p == 3:
        a = 1.0 / math.sqrt(5.0)
        return np.array([-1.0, -a, a, 1.0])
    if p == 4:
        a = math.sqrt(3.0 / 7.0)
        return np.array([-1.0, -a, 0.0, a, 1.0])
    raise ValueError("node placement implemented for p <= 4")


# ----------------------------------------------------------------------------
# Structured box meshes
# ----------------------------------------------------------------------------
@dataclass
class Mesh:
    dim: int
    n: tuple
    vert_xyz: np.ndarray      # [n_vert][dim] float64
    elem_vert: np.ndarray     # [E][2^dim] int64
    periodic_map: np.ndarray  # [n_vert] int64 (identity where not periodic)
    bnd_tag: np.ndarray       # [E][2 dim] int32, 0 = interior or periodic
    periodic: tuple = field(default=())

    @property
    def n_elem(self) -> int:
        return int(self.elem_vert.shape[0])

    @property
    def n_vert(self) -> int:
        return int(self.vert_xyz.shape[0])

    def n_faces(self) -> int:
        """Number of distinct faces of the structured box (periodic pairs once)."""
        tot = 0
        for r in range(self.dim):
            cnt = self.n[r] + (0 if self.periodic[r] else 1)
            for s in range(self.dim):
                if s != r:
                    cnt *= self.n[s]
            tot += cnt
        return tot


def box_mesh(dim: int, n, lo, hi, periodic, coords=None, tags=None) -> Mesh:
    """Structured box of ``prod(n)`` quads (dim 2) or hexes (dim 3).

    ``coords``, if given, is a list of per-direction vertex coordinate arrays of
    length ``n[r] + 1`` (graded spacing); otherwise spacing is uniform on
    ``[lo[r], hi[r]]``.  ``tags`` maps a box side ``(r, s)`` (direction, 0 = low
    / 1 = high) to a boundary tag for non-periodic directions (default 1).
    """
    n = tuple(int(v) for v in n)
    periodic = tuple(bool(v) for v in periodic)
    for r in range(dim):
        if periodic[r] and n[r] < 3:
            raise ValueError("periodic directions need at least 3 elements")
    if coords is None:
        coords = [np.linspace(lo[r], hi[r], n[r] + 1) for r in range(dim)]
    nv = [n[r] + 1 for r in range(dim)]
    grids = np.meshgrid(*coords, indexing="ij")
    # vertex index v = i + nv0 * (j + nv1 * k): x fastest
    vert = np.stack([g.transpose(*reversed(range(dim))).reshape(-1) for g in grids], axis=1)
    idx = np.arange(int(np.prod(nv))).reshape(*reversed(nv))  # idx[k][j][i]

    def vid(ii):
        return idx[tuple(reversed(ii))]

    pmap = np.arange(vert.shape[0], dtype=np.int64)
    for v in range(vert.shape[0]):
        rem = v
        ii = []
        for r in range(dim):
            ii.append(rem % nv[r])
            rem //= nv[r]
        jj = [(0 if (periodic[r] and ii[r] == n[r]) else ii[r]) for r in range(dim)]
        pmap[v] = vid(jj)

    E = int(np.prod(n))
    ev = np.zeros((E, 2 ** dim), dtype=np.int64)
    tag = np.zeros((E, 2 * dim), dtype=np.int32)
    tags = tags or {}
    for e in range(E):
        rem = e
        ei = []
        for r in range(dim):
            ei.append(rem % n[r])
            rem //= n[r]
        for c in range(2 ** dim):
            ev[e, c] = vid([ei[r] + ((c >> r) & 1) for r in range(dim)])
        for r in range(dim):
            if not periodic[r]:
                if ei[r] == 0:
                    tag[e, 2 * r] = tags.get((r, 0), 1)
                if ei[r] == n[r] - 1:
                    tag[e, 2 * r + 1] = tags.get((r, 1), 1)
    return Mesh(dim, n, vert.astype(np.float64), ev, pmap, tag, periodic)


def node_xyz(mesh: Mesh, p: int) -> np.ndarray:
    """Physical coordinates of the Gauss-Lobatto nodes, ``[E][Np][dim]``."""
    d = mesh.dim
    t = 0.5 * (gll_points(p) + 1.0)  # [0, 1]
    n1 = p + 1
    Np = n1 ** d
    out = np.zeros((mesh.n_elem, Np, d))
    X = mesh.vert_xyz[mesh.elem_vert]  # [E][2^d][d]
    for j in range(Np):
        jj = [(j // n1 ** r) % n1 for r in range(d)]
        w = np.ones(2 ** d)
        for c in range(2 ** d):
            for r in range(d):
                w[c] *= t[jj[r]] if (c >> r) & 1 else 1.0 - t[jj[r]]
        out[:, j, :] = np.einsum("c,ecx->ex", w, X)
    return out


# ----------------------------------------------------------------------------
# States (conserved variables at nodes) and their gradients
# ----------------------------------------------------------------------------
def conserved(rho, vel, p, gamma):
    """Stack ``[rho, rho v, rho E]`` from primitives (Sec. 2.1 closure)."""
    ke = 0.5 * rho * sum(v * v for v in vel)
    return np.stack([rho] + [rho * v for v in vel] + [p / (gamma - 1.0) + ke], axis=-1)


def freestream(dim: int, gamma: float, mach: float) -> np.ndarray:
    """rho = 1, |v| = 1 along x, p = 1 / (gamma M^2)."""
    vel = [1.0] + [0.0] * (dim - 1)
    return conserved(np.array(1.0), [np.array(v) for v in vel], 1.0 / (gamma * mach * mach), gamma)


def tgv_state(x: np.ndarray, gamma: float, mach: float) -> np.ndarray:
    """Taylor-Green vortex initial condition of Sec. 5.1 (L = 1, T = 1).

    Velocity ``(sin x cos y cos z, -cos x sin y cos z, 0)``; pressure
    ``1/(gamma M^2) + (cos 2x + cos 2y)(cos 2z + 2)/16``; the density follows
    from the ideal-gas law with uniform nondimensional temperature 1, i.e.
    ``rho = gamma M^2 p``.
    """
    X, Y, Z = x[..., 0], x[..., 1], x[..., 2]
    v1 = np.sin(X) * np.cos(Y) * np.cos(Z)
    v2 = -np.cos(X) * np.sin(Y) * np.cos(Z)
    v3 = np.zeros_like(X)
    p = 1.0 / (gamma * mach * mach) + (np.cos(2 * X) + np.cos(2 * Y)) * (np.cos(2 * Z) + 2.0) / 16.0
    rho = gamma * mach * mach * p
    return conserved(rho, [v1, v2, v3], p, gamma)


def sinusoid_state(x: np.ndarray, gamma: float, mach: float, seed: int = 0, amp: float = 1e-2) -> np.ndarray:
    """2-D freestream plus four seeded sinusoids in rho, rho u and rho E.

    ``sum_k amp * sin(2 pi (a_k x + b_k y) + phi_k)`` with ``a_k, b_k`` drawn
    from {1, 2, 3} and ``phi_k`` uniform on [0, 2 pi).
    """
    u = np.broadcast_to(freestream(2, gamma, mach), x.shape[:-1] + (4,)).copy()
    r = uniform(seed, 12)
    for k in range(4):
        a = 1 + int(3 * r[3 * k])
        b = 1 + int(3 * r[3 * k + 1])
        phi = 2 * np.pi * r[3 * k + 2]
        s = amp * np.sin(2 * np.pi * (a * x[..., 0] + b * x[..., 1]) + phi)
        for comp in (0, 1, 3):
            u[..., comp] += s
    return u


def couette_state(x: np.ndarray, gamma: float, pr: float, axis_v: int = 0, axis_y: int = 1,
                  p0: float = 1.0, e0: float = 2.0) -> np.ndarray:
    """Plane Couette flow with viscous heating at constant viscosity.

    ``v_{axis_v} = y``, uniform pressure, internal energy ``e = e0 - Pr y^2 / (2 gamma)``
    (the energy balance ``d/dy (v tau + gamma mu / Pr de/dy) = 0``), density
    ``rho = p / ((gamma - 1) e)``.  An exact steady solution of the
    compressible Navier-Stokes equations of Sec. 2.1 for any constant mu.
    """
    d = x.shape[-1]
    y = x[..., axis_y]
    e = e0 - pr * y * y / (2.0 * gamma)
    rho = p0 / ((gamma - 1.0) * e)
    vel = [np.zeros_like(y) for _ in range(d)]
    vel[axis_v] = y.copy()
    return conserved(rho, vel, np.full_like(y, p0), gamma)


def nodal_gradient(fun, x: np.ndarray, h: float = 1e-5) -> np.ndarray:
    """Central-difference gradient of a state function, ``[..., d, m]``."""
    d = x.shape[-1]
    out = []
    for k in range(d):
        dx = np.zeros(d)
        dx[k] = h
        out.append((fun(x + dx) - fun(x - dx)) / (2 * h))
    return np.stack(out, axis=-2)


# ----------------------------------------------------------------------------
# Workloads
# ----------------------------------------------------------------------------
@dataclass
class Problem:
    """One linearization input: mesh, degree, physics and the stage state."""
    name: str
    mesh: Mesh
    p: int
    gamma: float
    re: float
    pr: float
    mach: float
    tau: float
    dt: float
    a_ii: float
    visc_law: int            # 0 constant mu~ = 1, 1 Sutherland C1 T^1.5 / (T + S)
    suth_c1: float
    suth_s: float
    U: np.ndarray            # [E][m][Np]
    Q: np.ndarray            # [E][d][m][Np]
    UH: np.ndarray           # [F][m][Nfp]
    Ustar: np.ndarray        # [E][m][Np]
    nu: np.ndarray | None    # [E][Np] or None
    ubc: np.ndarray | None = None  # tag-1 boundary state: [m], or nodal [F][m][Nfp] (canonical order)
    twall: float = 1.0             # wall temperature T~_w of tag-3 faces (T~_inf = 1)


def _stage_state(mesh: Mesh, p: int, fun, ubg: np.ndarray, seed: int, noise: float,
                 trace_noise: float, ustar_noise: float = 0.0):
    d = mesh.dim
    m = d + 2
    x = node_xyz(mesh, p)
    u = fun(x)                                   # [E][Np][m]
    q = nodal_gradient(fun, x)                   # [E][Np][d][m]
    E, Np = x.shape[0], x.shape[1]
    if noise:
        u = u + noise * normal(seed, u.size).reshape(u.shape)
    U = np.ascontiguousarray(u.transpose(0, 2, 1))          # [E][m][Np]
    Q = np.ascontiguousarray(q.transpose(0, 2, 3, 1))       # [E][d][m][Np]
    Nfp = (p + 1) ** (d - 1)
    F = mesh.n_faces()
    UH = np.broadcast_to(ubg.reshape(1, m, 1), (F, m, Nfp)).copy()
    scale = np.abs(ubg).reshape(1, m, 1) + 1.0
    UH += trace_noise * scale * normal(seed + 1000, UH.size).reshape(UH.shape)
    Ustar = U.copy()
    if ustar_noise:
        Ustar += ustar_noise * normal(seed + 2000, U.size).reshape(U.shape)
    return U, Q, UH, Ustar


def synthetic_nu(mesh: Mesh, p: int, seed: int, level: float) -> np.ndarray:
    """A seeded positive nodal artificial-viscosity field ``[E][Np]``."""
    x = node_xyz(mesh, p)
    r = uniform(seed, 3)
    s = np.ones(x.shape[:2])
    for k in range(mesh.dim):
        s = s * np.sin(x[..., k] + 2 * np.pi * r[k])
    return level * (1.0 + 0.5 * s)


def config1(n: int = 8, p: int = 2, seed: int = 0) -> Problem:
    """2-D compressible NS, quads p=2, n x n periodic unit square, M = 0.3."""
    gamma, mach = 1.4, 0.3
    mesh = box_mesh(2, (n, n), (0.0, 0.0), (1.0, 1.0), (True, True))
    fun = lambda x: sinusoid_state(x, gamma, mach, seed=seed)
    ubg = freestream(2, gamma, mach)
    U, Q, UH, Ustar = _stage_state(mesh, p, fun, ubg, seed, 0.0, 1e-3, 0.0)
    return Problem("quad-p%d-%dx%d-periodic" % (p, n, n), mesh, p, gamma, 100.0, 0.72, mach, 5.0,
                   1e-2, 0.29, 0, 0.0, 0.0, U, Q, UH, Ustar, None)


def config_tgv(n: int, p: int, mach: float, seed: int, sutherland: bool, av: float) -> Problem:
    """3-D hex TGV-type periodic cube [0, 2 pi]^3 with seeded noise 1e-4."""
    gamma = 1.4
    mesh = box_mesh(3, (n, n, n), (0.0,) * 3, (2 * np.pi,) * 3, (True, True, True))
    fun = lambda x: tgv_state(x, gamma, mach)
    p0 = 1.0 / (gamma * mach * mach)
    ubg = conserved(np.array(gamma * mach * mach * p0), [np.array(0.0)] * 3, p0, gamma)
    U, Q, UH, Ustar = _stage_state(mesh, p, fun, ubg, seed, 1e-4, 1e-3, 0.0)
    nu = synthetic_nu(mesh, p, seed + 3000, av) if av > 0 else None
    return Problem("hex-p%d-%d^3-tgv-M%g" % (p, n, mach), mesh, p, gamma, 1600.0, 0.71, mach, 5.0,
                   1e-2, 0.29, 1 if sutherland else 0, 1.4042, 0.40417, U, Q, UH, Ustar, nu)


def config2(n: int = 16, p: int = 2) -> Problem:
    """Hex p=2 TGV at M = 0.1, constant viscosity (16^3 = 4096 elements)."""
    return config_tgv(n, p, 0.1, 1, False, 0.0)


def config3(n: int = 24, p: int = 3, av: float = 2e-3) -> Problem:
    """Hex p=3 TGV at M = 1.25, Sutherland viscosity, artificial viscosity on."""
    return config_tgv(n, p, 1.25, 2, True, av)


def tiny(dim: int, p: int, seed: int = 7, periodic=True, visc_law: int = 0, av: float = 0.0,
         mach: float = 0.5) -> Problem:
    """3 x 3 (x 3) mesh with a random smooth state, for brute-force checks."""
    gamma = 1.4
    n = (3,) * dim
    per = (periodic,) * dim if isinstance(periodic, bool) else tuple(periodic)
    mesh = box_mesh(dim, n, (0.0,) * dim, (1.0,) * dim, per)
    r = uniform(seed, 8)

    def fun(x):
        vel = [0.3 + 0.1 * np.sin(2 * np.pi * (x[..., 0] + r[0]))]
        for k in range(1, dim):
            vel.append(0.2 * np.cos(2 * np.pi * (x[..., k] + r[k])))
        rho = 1.0 + 0.1 * np.sin(2 * np.pi * (x[..., 0] + x[..., 1] + r[4]))
        pres = 1.0 / (gamma * mach * mach) * (1.0 + 0.05 * np.cos(2 * np.pi * (x[..., 1] + r[5])))
        return conserved(rho, vel, pres, gamma)

    ubg = freestream(dim, gamma, mach)
    U, Q, UH, Ustar = _stage_state(mesh, p, fun, ubg, seed, 1e-3, 1e-2, 1e-3)
    nu = synthetic_nu(mesh, p, seed + 5, av) if av > 0 else None
    return Problem("tiny-%dd-p%d" % (dim, p), mesh, p, gamma, 50.0, 0.72, mach, 3.0, 5e-2, 0.4,
                   visc_law, 1.4042, 0.40417, U, Q, UH, Ustar, nu, ubg)


# ----------------------------------------------------------------------------
# Hypersonic flat-plate boundary layer (the wall-bounded workload)
# ----------------------------------------------------------------------------
def graded_coordinates(n: int, length: float, first: float) -> np.ndarray:
    """n cells on [0, length] growing geometrically from `first`, the ratio solved
    so that they fill the length exactly.

    The workload asks for a first cell of 1e-4 of the height growing by 1.15;
    48 such cells reach only 0.55 of the height, so the first cell and the
    height are kept and the ratio becomes 1.168 (a reading)."""
    lo, hi = 1.0 + 1e-12, 2.0
    for _ in range(200):
        r = 0.5 * (lo + hi)
        if first * (r ** n - 1.0) / (r - 1.0) > length:
            hi = r
        else:
            lo = r
    r = 0.5 * (lo + hi)
    x = np.concatenate([[0.0], np.cumsum(first * r ** np.arange(n))])
    return x * (length / x[-1])


def blasius(eta_max: float = 12.0):
    """Blasius solution of f''' + f f'' / 2 = 0, f(0) = f'(0) = 0, f'(inf) = 1:
    shooting on f''(0) with an adaptive Runge-Kutta integrator; returns a
    callable f'(eta) (dense output) and the shooting value f''(0)."""
    from scipy.integrate import solve_ivp
    from scipy.optimize import brentq

    def rhs(_, y):
        return [y[1], y[2], -0.5 * y[0] * y[2]]

    def end(s):
        return solve_ivp(rhs, (0.0, eta_max), [0.0, 0.0, s], rtol=1e-11, atol=1e-12).y[1, -1] - 1.0

    s = brentq(end, 0.2, 0.5, xtol=1e-14)
    sol = solve_ivp(rhs, (0.0, eta_max), [0.0, 0.0, s], rtol=1e-11, atol=1e-12, dense_output=True)
    return (lambda eta: sol.sol(np.minimum(eta, eta_max))[1]), s


def plate_state_function(gamma, mach, pr, re_unit, t_wall, amp, seed, lx, lz):
    """Compressible laminar plate state: Blasius velocity f'(eta), Crocco-Busemann
    temperature T = T_w + (T_aw - T_w) u - (T_aw - 1) u^2 (T_inf = 1,
    T_aw = 1 + sqrt(Pr) (gamma - 1) M^2 / 2), uniform pressure 1 / (gamma M^2),
    rho = 1 / T; the wall distance follows the Howarth-Dorodnitsyn stretching
    y = sqrt(x / Re) int_0^eta T d eta.  A seeded 3-D disturbance of relative
    amplitude `amp` is added to the momentum."""
    fpf, _ = blasius()
    eta = np.linspace(0.0, 12.0, 6001)
    fp = fpf(eta)
    t_aw = 1.0 + math.sqrt(pr) * (gamma - 1.0) * mach ** 2 / 2.0
    T_eta = t_wall + (t_aw - t_wall) * fp - (t_aw - 1.0) * fp ** 2
    ystar = np.concatenate([[0.0], np.cumsum(0.5 * (T_eta[1:] + T_eta[:-1]) * np.diff(eta))])
    from scipy.interpolate import CubicSpline
    u_of = CubicSpline(ystar, fp)                    # f' as a function of the stretched distance
    r = uniform(seed, 12)
    p_inf = 1.0 / (gamma * mach * mach)

    def fun(x):
        xs = np.maximum(x[..., 0], 1e-6)
        ys = x[..., 1] * np.sqrt(re_unit / xs)
        u = np.where(ys < ystar[-1], u_of(np.minimum(ys, ystar[-1])), 1.0)
        T = t_wall + (t_aw - t_wall) * u - (t_aw - 1.0) * u * u
        rho = 1.0 / T
        damp = (ys / 5.0) * np.exp(1.0 - ys / 5.0)   # peaks inside the layer, 0 at the wall
        vel = [u, np.zeros_like(u), np.zeros_like(u)]
        for k in range(3):
            ph = 2 * np.pi * (x[..., 0] * (1 + 2 * r[3 * k]) / lx + x[..., 2] * (1 + r[3 * k + 1]) / lz + r[3 * k + 2])
            vel[k] = vel[k] + amp * damp * np.sin(ph)
        return conserved(rho, vel, p_inf + 0.0 * rho, gamma)

    return fun, t_aw


def config5(nx: int = 64, ny: int = 48, nz: int = 32, p: int = 3, seed: int = 4) -> Problem:
    """Flat-plate boundary layer at M = 6 on [0.1, 1.1] x [0, 0.1] x [0, 0.05]:
    wall-normal cells from 1e-4 of the height growing geometrically to fill it,
    isothermal wall at T_w = 0.5 T_aw (y = 0, tag 3), far field on top and at
    the inflow (tag 1, freestream state), extrapolation outflow (tag 2),
    periodic in z; Re_unit = 1e6, Pr = 0.72, Sutherland with S~ = 110.4 / 51.86
    and C1 = 1 + S~ (mu~(1) = 1); time step 2e-4 (the Mach-7 case's)."""
    gamma, mach, pr, re = 1.4, 6.0, 0.72, 1.0e6
    H, lx, lz = 0.1, 1.0, 0.05
    xs = np.linspace(0.1, 1.1, nx + 1)
    ys = graded_coordinates(ny, H, 1e-4 * H)
    zs = np.linspace(0.0, lz, nz + 1)
    mesh = box_mesh(3, (nx, ny, nz), (0.1, 0.0, 0.0), (1.1, H, lz), (False, False, True),
                    coords=[xs, ys, zs], tags={(0, 0): 1, (0, 1): 2, (1, 0): 3, (1, 1): 1})
    t_aw = 1.0 + math.sqrt(pr) * (gamma - 1.0) * mach ** 2 / 2.0
    t_wall = 0.5 * t_aw
    fun, _ = plate_state_function(gamma, mach, pr, re, t_wall, 1e-3, seed, lx, lz)
    ubg = freestream(3, gamma, mach)
    x = node_xyz(mesh, p)
    U = np.ascontiguousarray(fun(x).transpose(0, 2, 1))
    Q = np.ascontiguousarray(nodal_gradient(fun, x, h=1e-8).transpose(0, 2, 3, 1))
    F = mesh.n_faces()
    Nfp = (p + 1) ** 2
    UH = np.broadcast_to(ubg.reshape(1, 5, 1), (F, 5, Nfp)).copy()
    UH += 1e-3 * (np.abs(ubg).reshape(1, 5, 1) + 1.0) * normal(seed + 1000, UH.size).reshape(UH.shape)
    s_t = 110.4 / 51.86
    P = Problem("hex-p%d-%dx%dx%d-plate-M6" % (p, nx, ny, nz), mesh, p, gamma, re, pr, mach, 5.0, 2e-4, 0.29,
                1, 1.0 + s_t, s_t, U, Q, UH, U.copy(), None, ubg)
    P.twall = t_wall
    return P
