"""GPU tests of the paper's two diagnostic quantities, through the C ABI, against the FP64
oracle and the closed forms:

* the error measure of eq. (error_measure) (Sec. 3.1.1): the short-range boundary term that the
  paper's prescription leaves out, for one particle at several heights above the grounded
  cathode;
* the discrete action of eq. (full_p3m_lagrangian) with the leapfrog patch of eq. (leapfrog),
  evaluated along a trajectory the GPU pushed.
"""
import math

import numpy as np
import pytest
import torch
from scipy.special import erfc

from oracle import oracle as O
from paper_2103_02046_gb300 import bunches as B

pytestmark = pytest.mark.gpu

KE = O.coulomb_k()


def p3m():
    from paper_2103_02046_gb300 import p3m as m
    return m


def cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


# ------------------------------------------------------------------------------------------
# error measure (eq. (error_measure))
# ------------------------------------------------------------------------------------------
RC = 1e-4
KAPPA = 3.0


def _error_measure_params(pp_bc):
    h = RC / 2
    n = int(math.ceil(3.0 * RC / h)) + 5
    lo = (-1.5 * RC - 2 * h, -1.5 * RC - 2 * h, -2 * h)
    return O.Params(n=(n, n, n), lo=lo, h=(h, h, h), rc_over_h=2.0, kappa=KAPPA, pm_bc=1,
                    pp_bc=pp_bc, z_cathode=0.0, q=B.macro_charge(), mass=B.macro_mass())


def _probes(z_src):
    step = RC / 3
    g = np.arange(-2, 3) * step
    gz = (np.arange(0, 5) + 0.5) * step
    pts = np.stack(np.meshgrid(g, g, gz, indexing="ij"), -1).reshape(-1, 3)
    src = np.array([0.0, 0.0, z_src])
    pts = pts[np.linalg.norm(pts - src, axis=1) > 0.25 * RC]   # off the source
    return src, pts


def _potential_from_energies(energy, src, probes, q):
    """phi of the source at each probe, read off the (linear in the charges) P3M energy:
    (U(source + probe) - U(source) - U(probe)) / q."""
    us = energy(src[None, :])
    return np.array([(energy(np.stack([src, x])) - us - energy(x[None, :])) / q for x in probes])


@pytest.mark.parametrize("z_over_rc", [0.1, 0.3, 0.45, 1.0, 1.25])
def test_error_measure_short_range_boundary_term(z_over_rc):
    m = p3m()
    q = B.macro_charge()
    src, probes = _probes(z_over_rc * RC)
    phi_gpu, phi_or, img_pairs = {}, {}, {}
    for pp_bc in (0, 1):
        P = _error_measure_params(pp_bc)
        ctx = m.Context(m.Params(n=P.n, lo=P.lo, h=P.h, rc_over_h=P.rc_over_h, kappa=KAPPA,
                                 pm_bc=1, pp_bc=pp_bc, z_cathode=0.0, precision=m.FP64, q=q,
                                 mass=P.mass), 2)

        def e_gpu(pts):
            _, e = ctx.forces(cuda(pts), energy=True)
            return float(e.sum())

        def e_or(pts):
            r = O.forces(pts, P)
            return r.U_pp + r.U_pm

        phi_gpu[pp_bc] = _potential_from_energies(e_gpu, src, probes, q)
        phi_or[pp_bc] = _potential_from_energies(e_or, src, probes, q)
        ctx.forces(cuda(src[None, :]))
        img_pairs[pp_bc] = ctx.pair_count()[1]
        ctx.close()
    # the neglected term: the image's screened potential wherever the image is within r_c
    ri = np.linalg.norm(probes - src * np.array([1.0, 1.0, -1.0]), axis=1)
    closed = np.where(ri < RC, KE * q * erfc(KAPPA / RC * ri) / ri, 0.0)
    d_gpu = phi_gpu[0] - phi_gpu[1]
    d_or = phi_or[0] - phi_or[1]
    scale = np.abs(phi_gpu[1]).max()
    dV = (RC / 3) ** 3
    E_gpu = float((d_gpu ** 2).sum() * dV)
    E_closed = float((closed ** 2).sum() * dV)
    # GPU against the oracle, and both against the closed form (to the rounding of the energy
    # differences the potential is read from)
    np.testing.assert_allclose(phi_gpu[1], phi_or[1], rtol=0, atol=1e-11 * scale)
    np.testing.assert_allclose(d_gpu, d_or, rtol=0, atol=1e-11 * scale)
    np.testing.assert_allclose(d_gpu, closed, rtol=0, atol=1e-10 * scale)
    if z_over_rc >= 1.0:
        # no probe's image distance is below r_c: the boundary term vanishes (closed form exactly)
        assert E_closed == 0.0
        assert E_gpu <= 1e-20 * (scale ** 2) * dV * len(probes)
    else:
        assert E_gpu == pytest.approx(E_closed, rel=1e-8)
        assert E_closed > 0.0
    # the particle's own image enters the short range only below r_c / 2
    assert img_pairs[0] == 0
    assert img_pairs[1] == (1 if z_over_rc < 0.5 else 0)


# ------------------------------------------------------------------------------------------
# discrete action (eq. (full_p3m_lagrangian)) along a GPU trajectory
# ------------------------------------------------------------------------------------------
def test_discrete_action_along_gpu_trajectory():
    m = p3m()
    x0 = B.gaussian(300, (1e-3, 1e-3, 1e-3), 41)
    P = O.auto_mesh(x0 * 1.5, 8, rc_over_h=2.0)
    a = np.abs(O.forces(x0, P).F).max() / P.mass
    dt = math.sqrt(1e-7 / a)
    ctx = m.Context(m.Params(n=P.n, lo=P.lo, h=P.h, rc_over_h=P.rc_over_h, precision=m.FP64,
                             q=P.q, mass=P.mass), len(x0))
    x = cuda(x0)
    p = torch.zeros_like(x)
    f = ctx.forces(x)
    X = [x.clone()]
    for _ in range(6):
        f = ctx.push(x, p, dt, 1, f)
        X.append(x.clone())
    ctx.sync()
    Xh = [t.cpu().numpy() for t in X]

    def U_gpu(y):
        _, e = ctx.forces(y, energy=True)
        return float(e.sum())

    def S_gpu(Xs):
        tot = 0.0
        for n in range(len(Xs) - 1):
            kin = 0.5 * P.mass * float(((Xs[n + 1] - Xs[n]) ** 2).sum()) / dt ** 2
            tot += kin - U_gpu(Xs[n])
        return tot * dt

    # the energies along the trajectory, and the action, against the oracle
    for n in range(len(X) - 1):
        R = O.forces(Xh[n], P)
        assert U_gpu(X[n]) == pytest.approx(R.U_pp + R.U_pm, rel=1e-12)
    S_or = O.discrete_action(Xh, dt, P)
    kin_scale = dt * sum(0.5 * P.mass * float(((Xh[n + 1] - Xh[n]) ** 2).sum()) / dt ** 2
                         for n in range(len(Xh) - 1))
    U_scale = dt * sum(abs(U_gpu(X[n])) for n in range(len(X) - 1))
    assert abs(S_gpu(X) - S_or) <= 1e-12 * (kin_scale + U_scale)
    # Hamilton's principle, discrete: S_d is stationary on the GPU trajectory along a variation
    # of the interior points, and not off it
    gen = torch.Generator(device="cuda").manual_seed(3)
    V = [torch.zeros_like(x)] + [torch.randn(x.shape, dtype=x.dtype, device="cuda",
                                             generator=gen) for _ in X[1:-1]] + \
        [torch.zeros_like(x)]
    kin = dt * sum(abs(float((P.mass * (X[n] - X[n - 1]) / dt ** 2 * V[n]).sum()))
                   for n in range(1, len(X) - 1))
    eps = 1e-9

    def dS(Xs):
        return (S_gpu([u + eps * v for u, v in zip(Xs, V)]) -
                S_gpu([u - eps * v for u, v in zip(Xs, V)])) / (2 * eps)

    assert abs(dS(X)) <= 1e-6 * kin
    assert abs(dS([u + 1e-7 * v for u, v in zip(X, V)])) >= 1e-2 * kin
    ctx.close()
