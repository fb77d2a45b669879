"""Plain FP64 CPU oracle of the P3M space-charge force evaluation and leapfrog push.

TEST INFRASTRUCTURE ONLY. Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline
leg of ``bench.py`` may import this module. The product path (the CUDA library and its
binding) never imports it, and this module never imports the product path: the two share
no code. Their only common input is the seeded bunch generator, which holds no P3M
arithmetic.

Every function follows one step of the method of Wyssling & Adelmann (arXiv 2103.02046),
in double precision, in the paper's order:

* charge assignment to the mesh, eq. (rho_L) with W = W^L (Sec. 2.4.2)   -> C ``oracle_deposit``
* long-range potential, eq. (phi_L), as a discrete convolution with G^L = erf(a r)/r of
  eq. (ewald_split), and, for the grounded planar cathode, the image Green's function
  eq. (GreenFunc_planar_cathode) -- evaluated as a cyclic convolution on a doubled mesh with
  ``numpy``/``scipy`` FFTs (a library primitive used as one step)          -> ``solve``
* long-range force, first term of eq. (eom_p3m_coord), analytic dW/dxi    -> C ``oracle_interp``
* short-range force, eq. (summation_short) with G^S = erfc(a r)/r          -> C ``oracle_pp``
* leapfrog, eq. (leapfrog) with the Stoermer form of eq. (eom_p3m_coord)   -> ``push``

Readings of points the paper leaves open (stated here and in the design notes):
* alpha = kappa / r_c, kappa = 3 by default; r_c = rc_over_h * max_d h_d.
* mesh: node g at lo + g h; the automatic mesh puts two spacings of margin on either side of
  the particle bounding box: h_d = (b_d - a_d)/(n_d - 5), lo_d = a_d - 2 h_d.
* leapfrog start-up: kick-drift-kick with an initial half kick.
* emittance objective: J = eps_x + eps_y + eps_z (normalised rms emittance).
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
from dataclasses import dataclass, replace

import numpy as np

try:
    import scipy.fft as _sfft
    import scipy.special as _sspecial
except Exception:  # pragma: no cover - scipy is present in every image used here
    _sfft = None
    _sspecial = None

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liboracle.so")
_SRC = os.path.join(_HERE, "p3m_oracle.c")

EPS0 = 8.8541878128e-12
ELEMENTARY_CHARGE = 1.602176634e-19
ELECTRON_MASS = 9.1093837015e-31
SPEED_OF_LIGHT = 299792458.0


def coulomb_k() -> float:
    return 1.0 / (4.0 * math.pi * EPS0)


# ------------------------------------------------------------------------------------------
# build / load
# ------------------------------------------------------------------------------------------
def build(force: bool = False) -> str:
    """Compile the C part of the oracle (gcc, OpenMP) into oracle/_build/liboracle.so."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c11",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        P = ctypes.c_void_p
        I64 = ctypes.c_int64
        D = ctypes.c_double
        I = ctypes.c_int
        _lib.oracle_coulomb_constant.restype = D
        _lib.oracle_deposit.argtypes = [I64, P, D, P, P, P, I, P]
        _lib.oracle_deposit.restype = I64
        _lib.oracle_dipole_deposit.argtypes = [I64, P, P, P, P, P, I, P]
        _lib.oracle_dipole_deposit.restype = I64
        _lib.oracle_interp.argtypes = [I64, P, D, P, P, P, P, I, P, P]
        _lib.oracle_interp.restype = I64
        _lib.oracle_interp_vjp.argtypes = [I64, P, D, P, P, P, P, P, P, I, P]
        _lib.oracle_interp_vjp.restype = I64
        _lib.oracle_pp.argtypes = [I64, P, D, D, D, I, D, I64, P, P, P, P]
        _lib.oracle_pp.restype = None
        _lib.oracle_pp_brute.argtypes = [I64, P, D, D, D, I, D, P, P, P]
        _lib.oracle_pp_brute.restype = None
        _lib.oracle_pp_vjp.argtypes = [I64, P, D, D, D, I, D, P, P]
        _lib.oracle_pp_vjp.restype = None
        _lib.oracle_coulomb_brute.argtypes = [I64, P, D, I, D, P, P]
        _lib.oracle_coulomb_brute.restype = None
        _lib.oracle_mesh_direct.argtypes = [P, P, P, D, I, D, P, P]
        _lib.oracle_mesh_direct.restype = None
    return _lib


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p) if a is not None else None


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


# ------------------------------------------------------------------------------------------
# parameters and mesh geometry
# ------------------------------------------------------------------------------------------
@dataclass(frozen=True)
class Params:
    n: tuple = (16, 16, 16)          # mesh nodes per axis
    lo: tuple = (0.0, 0.0, 0.0)      # position of node 0 [m]
    h: tuple = (1.0, 1.0, 1.0)       # mesh spacing [m]
    rc_over_h: float = 2.0           # r_c = rc_over_h * max(h)
    kappa: float = 3.0               # alpha = kappa / r_c unless alpha > 0
    alpha: float = 0.0
    assign_order: int = 2            # 1 = CIC, 2 = TSC
    pm_bc: int = 0                   # 1 = grounded cathode plane, 2 = grounded box (long range)
    pp_bc: int = 0                   # 1 = cathode images in the short-range sum as well
    z_cathode: float = 0.0
    influence: int = 0               # 1 = principal-alias optimal factor 1/U^2, 2 = alias sum
    force_diff: int = 0              # 1 = central-difference mesh gradient (not the W derivative)
    q: float = 1e-15
    mass: float = 1e-15 / ELEMENTARY_CHARGE * ELECTRON_MASS

    @property
    def rc(self) -> float:
        return self.rc_over_h * max(self.h)

    @property
    def a(self) -> float:
        return self.alpha if self.alpha > 0 else self.kappa / self.rc


def auto_mesh(x: np.ndarray, n, **kw) -> Params:
    """Mesh over the particle bounding box with two spacings of margin on every side."""
    n = tuple(int(v) for v in np.broadcast_to(np.asarray(n), (3,)))
    a = x.min(axis=0)
    b = x.max(axis=0)
    h = tuple(float((b[d] - a[d]) / (n[d] - 5)) for d in range(3))
    lo = tuple(float(a[d] - 2.0 * h[d]) for d in range(3))
    return Params(n=n, lo=lo, h=h, **kw)


def _mesh_args(P: Params):
    return (np.asarray(P.n, dtype=np.int32), np.asarray(P.lo, dtype=np.float64),
            np.asarray(P.h, dtype=np.float64))


# ------------------------------------------------------------------------------------------
# mesh steps
# ------------------------------------------------------------------------------------------
def deposit(x, P: Params):
    """Node charges Q[gz, gy, gx] = q sum_i W(x_g - xi_i) (eq. (rho_L)); returns (Q, n_bad)."""
    x = _f64(x)
    n, lo, h = _mesh_args(P)
    Q = np.zeros((P.n[2], P.n[1], P.n[0]))
    bad = lib().oracle_deposit(len(x), _p(x), P.q, _p(n), _p(lo), _p(h), P.assign_order, _p(Q))
    return Q, int(bad)


def dipole_deposit(x, w, P: Params):
    """psi_g = sum_i grad W(x_g - xi_i) . w_i (adjoint of the deposit feeding the solve)."""
    x = _f64(x)
    w = _f64(w)
    n, lo, h = _mesh_args(P)
    psi = np.zeros((P.n[2], P.n[1], P.n[0]))
    lib().oracle_dipole_deposit(len(x), _p(x), _p(w), _p(n), _p(lo), _p(h), P.assign_order,
                                _p(psi))
    return psi


def _g_long(r, alpha):
    """G^L(r) = erf(alpha r)/r with its limit 2 alpha/sqrt(pi) at r = 0 (eq. (ewald_split))."""
    out = np.empty_like(r)
    nz = r > 0
    out[nz] = _sspecial.erf(alpha * r[nz]) / r[nz]
    out[~nz] = 2.0 * alpha / math.sqrt(math.pi)
    return out


def _signed_offsets(n, M):
    """offset m for storage index 0..M-1 of a cyclic array of length M = 2n: m in
    [-(n-1), n-1]; the unused entry (index n) is flagged."""
    idx = np.arange(M)
    m = np.where(idx < n, idx, idx - M).astype(np.float64)
    return m, idx == n


def green_kernels(P: Params):
    """Spectra of the free and image long-range kernels on the doubled mesh, times k_e.

    K_f[m] = G^L(|m h|) and K_i[m] = G^L(|(m_x h_x, m_y h_y, 2d + (m_z + n_z - 1) h_z)|),
    d = lo_z - z_cathode, for m_d in [-(n_d - 1), n_d - 1] stored at m_d mod 2 n_d (the
    single unused offset n_d holds 0). K_i is the image kernel of eq. (GreenFunc_planar_cathode)
    written as a convolution with the z-reversed charge (the image of node j_z sits at
    z-offset 2d + (i_z + j_z) h_z from node i_z), which is the shifted Green's function idea
    of Sec. 3.1 on the charge domain only.
    """
    nx, ny, nz = P.n
    Mx, My, Mz = 2 * nx, 2 * ny, 2 * nz
    mx, ux = _signed_offsets(nx, Mx)
    my, uy = _signed_offsets(ny, My)
    mz, uz = _signed_offsets(nz, Mz)
    X = (mx * P.h[0])[None, None, :]
    Y = (my * P.h[1])[None, :, None]
    unused = uz[:, None, None] | uy[None, :, None] | ux[None, None, :]
    alpha = P.a
    ke = coulomb_k()
    Zf = (mz * P.h[2])[:, None, None]
    r = np.sqrt(X * X + Y * Y + Zf * Zf)
    Kf = _g_long(r, alpha)
    Kf[unused] = 0.0
    Kf_hat = _rfftn(Kf) * ke
    Ki_hat = None
    if P.pm_bc == 1:
        d = P.lo[2] - P.z_cathode
        Zi = (2.0 * d + (mz + nz - 1) * P.h[2])[:, None, None]
        r = np.sqrt(X * X + Y * Y + Zi * Zi)
        Ki = _g_long(r, alpha)
        Ki[unused] = 0.0
        Ki_hat = _rfftn(Ki) * ke
    if P.influence:
        F = 1.0 / _assignment_spectrum_sq(P) if P.influence == 1 else alias_influence_factor(P)
        Kf_hat = Kf_hat * F
        if Ki_hat is not None:
            Ki_hat = Ki_hat * F
    return Kf_hat, Ki_hat


def alias_u2_sum(t, p1: int, mmax: int = 2):
    """sum_{|m| <= mmax} sinc(t + m)^(2 p1): one axis of the alias sum of U^2 (t = k h / 2 pi,
    p1 = assignment order + 1); the denominator of eq. (Ghfinal) is the product over axes."""
    return sum(np.sinc(t + m) ** (2 * p1) for m in range(-mmax, mmax + 1))


def alias_influence_factor(P: Params, mmax: int = 2):
    """Optimal influence function of eq. (Ghfinal) with its alias sums, as a factor on the
    sampled kernel spectra, on the rfft layout of the doubled mesh:

        F(k) = sum_m U^2(k_m) R(k_m) / [ R(k) (sum_m U^2(k_m))^2 ],   k_m = k + 2 pi m / h,

    |m_d| <= mmax, U(k) = prod_d sinc(k_d h_d / 2)^(p+1) the assignment function (point
    particles) and R(k) = exp(-|k|^2 / (4 alpha^2)) / |k|^2 the long-range reference kernel (its
    constant factor cancels). Keeping only m = 0 gives 1/U^2 (influence = 1); F(0) = 1."""
    nx, ny, nz = P.n
    Mx, My, Mz = 2 * nx, 2 * ny, 2 * nz
    p1 = P.assign_order + 1
    alpha = P.a
    t = [np.arange(Mx // 2 + 1) / Mx, np.fft.fftfreq(My, 1.0 / My) / My,
         np.fft.fftfreq(Mz, 1.0 / Mz) / Mz]            # k_d h_d / (2 pi), signed
    shape = [(1, 1, Mx // 2 + 1), (1, My, 1), (Mz, 1, 1)]
    num = np.zeros((Mz, My, Mx // 2 + 1))
    den = np.ones((Mz, My, Mx // 2 + 1))
    u2 = []   # per axis and alias: U_d^2, exp(-q_d^2 / 4 alpha^2), q_d^2
    for d in range(3):
        rows = []
        for m in range(-mmax, mmax + 1):
            tm = t[d] + m
            q = 2.0 * np.pi * tm / P.h[d]
            rows.append((np.sinc(tm) ** (2 * p1), np.exp(-q * q / (4.0 * alpha * alpha)), q * q))
        u2.append(rows)
        den = den * alias_u2_sum(t[d], p1, mmax).reshape(shape[d])
    for mz in u2[2]:
        for my in u2[1]:
            for mx in u2[0]:
                w = (mx[0] * mx[1]).reshape(shape[0]) * (my[0] * my[1]).reshape(shape[1]) * \
                    (mz[0] * mz[1]).reshape(shape[2])
                q2 = mx[2].reshape(shape[0]) + my[2].reshape(shape[1]) + mz[2].reshape(shape[2])
                with np.errstate(divide="ignore", invalid="ignore"):
                    num = num + np.where(q2 > 0.0, w / q2, 0.0)
    q2 = sum(u2[d][mmax][2].reshape(shape[d]) for d in range(3))
    rk = np.exp(-q2 / (4.0 * alpha * alpha))
    with np.errstate(divide="ignore", invalid="ignore"):
        F = num * q2 / (rk * den * den)
    F[0, 0, 0] = 1.0   # limit k -> 0: the m = 0 term dominates, every other U(k_m) vanishes
    return F


def _assignment_spectrum_sq(P: Params):
    """U(k)^2 with U = prod_d sinc(k_d h_d / 2)^(p+1), k_d = 2 pi kappa_d / (M_d h_d), on the
    rfft layout of the doubled mesh (principal-alias optimal influence function, Sec. 3.1.2)."""
    nx, ny, nz = P.n
    Mx, My, Mz = 2 * nx, 2 * ny, 2 * nz
    p1 = P.assign_order + 1
    kx = np.arange(Mx // 2 + 1)
    ky = np.fft.fftfreq(My, 1.0 / My)
    kz = np.fft.fftfreq(Mz, 1.0 / Mz)
    ux = np.sinc(kx / Mx) ** p1
    uy = np.sinc(ky / My) ** p1
    uz = np.sinc(kz / Mz) ** p1
    U = uz[:, None, None] * uy[None, :, None] * ux[None, None, :]
    return U * U


def _workers():
    return os.cpu_count() or 1


def _rfftn(a):
    return _sfft.rfftn(a, workers=_workers())


def _irfftn(a, shape):
    return _sfft.irfftn(a, s=shape, workers=_workers())


def solve(Q, P: Params, kernels=None):
    """Mesh potential phi = k_e [K_f (*) Q - K_i (*) Q_rev] restricted to the n^3 block
    (eq. (phi_L); image part only with the cathode). Q_rev[.,.,j] = Q[.,.,n_z - 1 - j].
    With the grounded box (pm_bc = 2), the discrete-Laplacian solve of ``box_solve``."""
    if P.pm_bc == 2:
        return box_solve(Q, P)
    nx, ny, nz = P.n
    shape = (2 * nz, 2 * ny, 2 * nx)
    Kf_hat, Ki_hat = kernels if kernels is not None else green_kernels(P)
    pad = np.zeros(shape)
    pad[:nz, :ny, :nx] = Q
    phi = _irfftn(_rfftn(pad) * Kf_hat, shape)[:nz, :ny, :nx]
    if P.pm_bc == 1:
        pad[:nz, :ny, :nx] = Q[::-1, :, :]
        phi = phi - _irfftn(_rfftn(pad) * Ki_hat, shape)[:nz, :ny, :nx]
    return np.ascontiguousarray(phi)


def box_laplacian_eigenvalues(P: Params):
    """Eigenvalues of the discrete Laplacian D_xyz of eq. (3dim_second_order_fin_diff) on the
    interior nodes of a box with phi = 0 on its faces (nodes 0 and n_d - 1): for the sine mode
    j_d = 1 .. N_d (N_d = n_d - 2), sum_d (2 cos(pi j_d / (N_d + 1)) - 2) / h_d^2, as [z, y, x]."""
    lam = 0.0
    shape = [(1, 1, -1), (1, -1, 1), (-1, 1, 1)]
    for d in range(3):
        N = P.n[d] - 2
        j = np.arange(1, N + 1)
        lam = lam + ((2.0 * np.cos(np.pi * j / (N + 1)) - 2.0) / P.h[d] ** 2).reshape(shape[d])
    return lam


def box_solve(Q, P: Params):
    """Long-range potential in a grounded box (Sec. 3.1, fig. boundary_gauss_seidel_results):
    the discrete Poisson equation D_xyz phi = -rho_L / eps0 of eq. (def_G_L) on the interior
    nodes, phi = 0 on the six faces, rho_L = Q / (h_x h_y h_z) screened by the Gaussian of the
    charge splitting, applied in the sine basis as gamma^(k) = exp(-|k|^2 / (4 alpha^2)),
    k_d = pi j_d / ((N_d + 1) h_d). Solved with type-1 sine transforms (each diagonalises D_xyz
    with these boundary values)."""
    from scipy.fft import dstn, idstn
    nx, ny, nz = P.n
    lam = box_laplacian_eigenvalues(P)
    k2 = 0.0
    shape = [(1, 1, -1), (1, -1, 1), (-1, 1, 1)]
    for d in range(3):
        N = P.n[d] - 2
        k = np.pi * np.arange(1, N + 1) / ((N + 1) * P.h[d])
        k2 = k2 + (k * k).reshape(shape[d])
    gam = np.exp(-k2 / (4.0 * P.a * P.a))
    vol = P.h[0] * P.h[1] * P.h[2]
    rho = _f64(Q)[1:-1, 1:-1, 1:-1] / vol          # Q holds charges (q included)
    phi_hat = -gam * dstn(rho, type=1) / (EPS0 * lam)
    phi = np.zeros((nz, ny, nx))
    phi[1:-1, 1:-1, 1:-1] = idstn(phi_hat, type=1)
    return phi


def box_valid(x, P: Params):
    """Every particle's assignment support on nodes 1 .. n - 2 (the grounded box's interior, and
    the nodes where central differences of phi exist): TSC nearest node in [2, n - 3], CIC
    lower node in [1, n - 3]."""
    s = (_f64(x) - np.asarray(P.lo)) / np.asarray(P.h)
    n = np.asarray(P.n)
    if P.assign_order == 2:
        c = np.floor(s + 0.5)
        return np.all((c >= 2) & (c <= n - 3), axis=1)
    c = np.floor(s)
    return np.all((c >= 1) & (c <= n - 3), axis=1)


def mesh_direct(Q, P: Params):
    """phi by O(M^2) direct summation over node pairs (pin for ``solve``)."""
    n, lo, h = _mesh_args(P)
    Q = _f64(Q)
    phi = np.zeros_like(Q)
    lib().oracle_mesh_direct(_p(n), _p(lo), _p(h), P.a, int(P.pm_bc), P.z_cathode, _p(Q), _p(phi))
    return phi


def interp(x, phi, P: Params):
    """F^L_i = -q sum_g phi_g grad W(x_g - xi_i); also phi(xi_i). Returns (F, phi_at, n_bad)."""
    x = _f64(x)
    phi = _f64(phi)
    n, lo, h = _mesh_args(P)
    F = np.zeros_like(x)
    pa = np.zeros(len(x))
    bad = lib().oracle_interp(len(x), _p(x), P.q, _p(phi), _p(n), _p(lo), _p(h), P.assign_order,
                              _p(F), _p(pa))
    return F, pa, int(bad)


def _weights_1d(s, order):
    """Nodes and weights of one axis: TSC (nearest node c, offsets c-1..c+1) or CIC (c, c+1)."""
    if order == 2:
        c = np.floor(s + 0.5)
        u = s - c
        return c - 1, np.stack([0.5 * (0.5 - u) ** 2, 0.75 - u * u, 0.5 * (0.5 + u) ** 2], -1)
    c = np.floor(s)
    f = s - c
    return c, np.stack([1.0 - f, f], -1)


def interp_central(x, phi, P: Params):
    """Alternative long-range force: the mesh field by central differences,
    E_d(g) = -(phi_{g + e_d} - phi_{g - e_d}) / (2 h_d), interpolated with the assignment
    function, F_i = q sum_g W(x_g - xi_i) E(g). The support must keep one node off the mesh
    edge (``box_valid``)."""
    x = _f64(x)
    phi = _f64(phi)
    s = (x - np.asarray(P.lo)) / np.asarray(P.h)
    F = np.zeros_like(x)
    base, w = [], []
    for d in range(3):
        b, wd = _weights_1d(s[:, d], P.assign_order)
        base.append(b.astype(np.int64))
        w.append(wd)
    S = w[0].shape[1]
    for c in range(S):
        for b in range(S):
            for a in range(S):
                gx, gy, gz = base[0] + a, base[1] + b, base[2] + c
                W = w[0][:, a] * w[1][:, b] * w[2][:, c]
                E = [-(phi[gz, gy, gx + 1] - phi[gz, gy, gx - 1]) / (2 * P.h[0]),
                     -(phi[gz, gy + 1, gx] - phi[gz, gy - 1, gx]) / (2 * P.h[1]),
                     -(phi[gz + 1, gy, gx] - phi[gz - 1, gy, gx]) / (2 * P.h[2])]
                for d in range(3):
                    F[:, d] += P.q * W * E[d]
    return F


# ------------------------------------------------------------------------------------------
# short range
# ------------------------------------------------------------------------------------------
def pp(x, P: Params, sample=None):
    """Short-range forces (cell list) on all particles or on `sample` (indices).
    Returns (F, phi_S, counts) with counts = (pairs, image_pairs, coincident)."""
    x = _f64(x)
    if sample is not None:
        sample = np.ascontiguousarray(sample, dtype=np.int64)
    n_out = len(x) if sample is None else len(sample)
    F = np.zeros((n_out, 3))
    phi = np.zeros(n_out)
    counts = np.zeros(3, dtype=np.int64)
    lib().oracle_pp(len(x), _p(x), P.q, P.a, P.rc, int(P.pp_bc), P.z_cathode, n_out,
                    _p(sample), _p(F), _p(phi), _p(counts))
    return F, phi, tuple(int(c) for c in counts)


def pp_brute(x, P: Params):
    x = _f64(x)
    F = np.zeros_like(x)
    phi = np.zeros(len(x))
    counts = np.zeros(3, dtype=np.int64)
    lib().oracle_pp_brute(len(x), _p(x), P.q, P.a, P.rc, int(P.pp_bc), P.z_cathode, _p(F),
                          _p(phi), _p(counts))
    return F, phi, tuple(int(c) for c in counts)


def coulomb_brute(x, P: Params, bc=None):
    """Exact Coulomb forces (+ cathode images if bc) by O(N^2) summation."""
    x = _f64(x)
    bc = P.pm_bc if bc is None else bc
    F = np.zeros_like(x)
    phi = np.zeros(len(x))
    lib().oracle_coulomb_brute(len(x), _p(x), P.q, int(bc), P.z_cathode, _p(F), _p(phi))
    return F, phi


# ------------------------------------------------------------------------------------------
# full force evaluation
# ------------------------------------------------------------------------------------------
@dataclass
class ForceResult:
    F: np.ndarray          # total force [n_out, 3]
    F_pp: np.ndarray       # short-range part
    F_pm: np.ndarray       # long-range part
    phi_pp: np.ndarray     # short-range potential at the particles [V]
    phi_pm: np.ndarray     # interpolated long-range potential [V]
    Q: np.ndarray          # node charges
    phi_mesh: np.ndarray   # mesh potential
    pairs: int
    image_pairs: int
    n_bad: int
    U_pp: float            # 1/2 q sum phi_S (over the output particles)
    U_pm: float            # 1/2 sum_g Q_g phi_g


def forces(x, P: Params, sample=None, kernels=None, parts=3):
    """One P3M force evaluation (eq. (eom_p3m_coord) right-hand side, both terms):
    deposit -> solve -> interpolate (long range) plus the short-range sum."""
    x = _f64(x)
    xs = x if sample is None else x[np.asarray(sample)]
    n_out = len(xs)
    F_pm = np.zeros((n_out, 3))
    phi_pm = np.zeros(n_out)
    Q = phi_m = None
    bad = 0
    U_pm = 0.0
    if (P.pm_bc == 2 or P.force_diff) and not np.all(box_valid(x, P)):
        raise ValueError("a particle's assignment support reaches the mesh's edge nodes")
    if parts & 2:
        Q, bad = deposit(x, P)
        phi_m = solve(Q, P, kernels)
        F_pm, phi_pm, _ = interp(xs, phi_m, P)
        if P.force_diff:
            F_pm = interp_central(xs, phi_m, P)
        U_pm = 0.5 * float(np.sum(Q * phi_m))
    F_pp = np.zeros((n_out, 3))
    phi_pp = np.zeros(n_out)
    counts = (0, 0, 0)
    if parts & 1:
        F_pp, phi_pp, counts = pp(x, P, sample)
    return ForceResult(F=F_pp + F_pm, F_pp=F_pp, F_pm=F_pm, phi_pp=phi_pp, phi_pm=phi_pm, Q=Q,
                       phi_mesh=phi_m, pairs=counts[0], image_pairs=counts[1], n_bad=bad,
                       U_pp=0.5 * P.q * float(np.sum(phi_pp)), U_pm=U_pm)


def self_energy(N: int, P: Params) -> float:
    """Ewald self-energy N k_e q^2 alpha / sqrt(pi) contained in the long-range energy."""
    return N * coulomb_k() * P.q * P.q * P.a / math.sqrt(math.pi)


def total_energy(x, p, P: Params, res: ForceResult | None = None) -> float:
    """Kinetic + short-range + long-range - self energy."""
    res = forces(x, P) if res is None else res
    ke = float(np.sum(p * p)) / (2.0 * P.mass)
    return ke + res.U_pp + res.U_pm - self_energy(len(x), P)


def discrete_action(X, dt, P: Params, kernels=None) -> float:
    """Discrete action of eq. (full_p3m_lagrangian) with the left-point patch of eq. (leapfrog):
    S_d = dt sum_n [ sum_i M |x^{n+1}_i - x^n_i|^2 / (2 dt^2) - U(x^n) ] over the states
    X = [x^0, ..., x^K], with U = U_pp + U_pm the split P3M potential energy (eq. (pot_split)).
    The self term is a constant of the motion and is left in U."""
    tot = 0.0
    for n in range(len(X) - 1):
        R = forces(X[n], P, kernels=kernels)
        kin = 0.5 * P.mass * float(((_f64(X[n + 1]) - _f64(X[n])) ** 2).sum()) / dt ** 2
        tot += kin - (R.U_pp + R.U_pm)
    return tot * dt


# ------------------------------------------------------------------------------------------
# leapfrog push (eq. (leapfrog); kick-drift-kick with an initial half kick)
# ------------------------------------------------------------------------------------------
def push(x, p, dt, nsteps, P: Params, force=None, F0=None, states=None):
    """p^{n+1/2} = p^n + dt/2 F(x^n); x^{n+1} = x^n + dt p^{n+1/2}/M; p^{n+1} = p^{n+1/2} +
    dt/2 F(x^{n+1}). `force(x)` defaults to the P3M force. If `states` is a list, (x, p) of
    every step (including step 0) is appended. Returns (x, p, F(x_end))."""
    force = force or (lambda y: forces(y, P).F)
    x = _f64(x).copy()
    p = _f64(p).copy()
    F = force(x) if F0 is None else F0
    if states is not None:
        states.append((x.copy(), p.copy()))
    for _ in range(nsteps):
        p = p + 0.5 * dt * F
        x = x + dt * p / P.mass
        F = force(x)
        p = p + 0.5 * dt * F
        if states is not None:
            states.append((x.copy(), p.copy()))
    return x, p, F


# ------------------------------------------------------------------------------------------
# objective: rms emittance
# ------------------------------------------------------------------------------------------
def emittance(x, p, P: Params):
    """eps_u = sqrt(<du^2><dp^2> - <du dp>^2) / (M c) for u = x, y, z (centred moments)."""
    x = _f64(x)
    p = _f64(p)
    dx = x - x.mean(axis=0)
    dp = p - p.mean(axis=0)
    a = np.mean(dx * dx, axis=0)
    b = np.mean(dp * dp, axis=0)
    c = np.mean(dx * dp, axis=0)
    return np.sqrt(a * b - c * c) / (P.mass * SPEED_OF_LIGHT)


def emittance_grad(x, p, P: Params):
    """Gradient of J = sum_u eps_u with respect to x and p (closed form)."""
    x = _f64(x)
    p = _f64(p)
    N = len(x)
    dx = x - x.mean(axis=0)
    dp = p - p.mean(axis=0)
    a = np.mean(dx * dx, axis=0)
    b = np.mean(dp * dp, axis=0)
    c = np.mean(dx * dp, axis=0)
    mc = P.mass * SPEED_OF_LIGHT
    eps = np.sqrt(a * b - c * c) / mc
    den = N * mc * mc * eps
    gx = (dx * b - dp * c) / den
    gp = (dp * a - dx * c) / den
    return gx, gp


# ------------------------------------------------------------------------------------------
# adjoint
# ------------------------------------------------------------------------------------------
def force_vjp(x, w, P: Params, kernels=None):
    """(dF/dx)^T w for the P3M force map (short range + long range)."""
    x = _f64(x)
    w = _f64(w)
    out = np.zeros_like(x)
    lib().oracle_pp_vjp(len(x), _p(x), P.q, P.a, P.rc, int(P.pp_bc), P.z_cathode, _p(w),
                        _p(out))
    kernels = kernels if kernels is not None else green_kernels(P)
    Q, _ = deposit(x, P)
    phi = solve(Q, P, kernels)
    psi = dipole_deposit(x, w, P)
    chi = solve(psi, P, kernels)
    n, lo, h = _mesh_args(P)
    pm = np.zeros_like(x)
    lib().oracle_interp_vjp(len(x), _p(x), P.q, _p(phi), _p(chi), _p(w), _p(n), _p(lo), _p(h),
                            P.assign_order, _p(pm))
    return out + pm


def backward(x0, p0, dt, nsteps, gxT, gpT, P: Params, kernels=None):
    """Gradient with respect to (x0, p0) of a function of the final state (x_T, p_T) of the
    kick-drift-kick leapfrog, given its gradient (gxT, gpT) at the final state.

    Reverse of one step (x_n, p_n) -> (x_{n+1}, p_{n+1}):
      lx += J(x_{n+1})^T (dt/2 lp);  lp += (dt/M) lx;  lx += J(x_n)^T (dt/2 lp),
    where J = dF/dx. All states are kept (no checkpointing: small cases only)."""
    kernels = kernels if kernels is not None else green_kernels(P)
    states = []
    force = lambda y: forces(y, P, kernels=kernels).F
    push(x0, p0, dt, nsteps, P, force=force, states=states)
    lx = _f64(gxT).copy()
    lp = _f64(gpT).copy()
    for n in range(nsteps - 1, -1, -1):
        x_next = states[n + 1][0]
        x_now = states[n][0]
        lx = lx + force_vjp(x_next, 0.5 * dt * lp, P, kernels)
        lp = lp + (dt / P.mass) * lx
        lx = lx + force_vjp(x_now, 0.5 * dt * lp, P, kernels)
    return lx, lp


def rel_l2(a, b):
    """||a - b||_2 / ||b||_2 over all components."""
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    nb = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / nb) if nb > 0 else float(np.linalg.norm(a - b))


__all__ = [n for n in dir() if not n.startswith("_")] + ["replace"]
