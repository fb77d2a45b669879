"""Workload runs that report the paper's physics quantities on the GPU path.

  python -m paper_2103_02046_gb300.experiments boundary   # cathode BC in the short range vs mesh error
  python -m paper_2103_02046_gb300.experiments energy     # leapfrog energy drift and momentum
  python -m paper_2103_02046_gb300.experiments gradient   # adjoint gradient vs finite differences
  python -m paper_2103_02046_gb300.experiments gradient_coords --fp64  # ... on single coordinates
  python -m paper_2103_02046_gb300.experiments influence  # P3M error vs exact Coulomb per kernel
  python -m paper_2103_02046_gb300.experiments error_measure --fp64  # eq. (error_measure) vs height
  python -m paper_2103_02046_gb300.experiments action     # discrete EL residual, action stationarity
  python -m paper_2103_02046_gb300.experiments box_potentials [--save f.npz]  # grounded-box figure

Each prints one JSON line. Everything runs through the C ABI (``p3m``); no oracle is used.

* boundary (Sec. 3.1.1, the paper's claim that neglecting the cathode in the short range costs an
  error tied to the mesh discretisation error): 4,194,304 particles, 95% Gaussian core
  (sigma = 1 mm) + 5% uniform halo shell at 4-6 sigma, lifted so the lowest particle sits one mesh
  spacing above the grounded cathode; r_c = 3h; long range with the cathode. Reports
  ||F(pp_bc=1) - F(pp_bc=0)|| / ||F|| against the refinement error ||F_h - F_{h/2}|| / ||F||
  at n = 128 and n = 256, and the locality of the short-range boundary effect.
* energy: 1,048,576-particle Gaussian bunch (sigma = 1, 1, 3 mm), thermal momenta 1e-4 m_e c rms,
  64^3 mesh, r_c = 2h, dt = 1e-12 s, 100 kick-drift-kick steps: relative energy drift and the
  total momentum.
* gradient: the same bunch, 200 steps of dt = 2.5e-13 s (the bunch, about 1 nC in a few mm^3,
  expands by millimetres within 1e-10 s, so 200 steps of 1e-12 s would leave any fixed mesh)
  with checkpoints every 20: gradient of the final rms
  emittance J = eps_x + eps_y + eps_z with respect to (x0, p0) by the reverse pass, checked by
  central finite differences along two directions that change J at first order (dilations of
  x0 and of p0 about their means), relative step 1e-6 in FP64 and 1e-3 in FP32 (the evaluation
  order of the FP32 force sums is not fixed, which leaves J reproducible to about 1e-7).
* gradient_coords: the same bunch and schedule at 16,384 particles, FP64: the reverse pass
  against central finite differences on 64 randomly chosen single coordinates (positions and
  momenta), step 1e-6 times that component's rms spread. A single coordinate moves only its own
  pairs, so within the step no pair crosses the hard cutoff r_c (where the short-range force
  jumps) and the difference quotient measures the derivative the reverse pass computes. Also
  the FP32 mixed reverse pass against the FP64 one over all 6N coordinates.
"""
from __future__ import annotations

import json
import math
import sys
import time

import numpy as np
import torch

from . import bunches as B
from . import p3m as m


def _cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


def _rel(a, b):
    return float(torch.linalg.norm(a - b) / torch.linalg.norm(b))


def boundary(precision: int = m.FP32_MIXED, n_particles: int = 4_194_304):
    spec = dict(B.WORKLOADS["halo4m"])
    x0 = B.positions(spec, n_particles)
    # lift by one spacing of the coarse mesh (h does not depend on the translation)
    h128 = m.auto_mesh(_cuda(x0), m.Params(n=(128,) * 3)).h[2]
    xg = _cuda(B.lift_to_plane(x0, 0.0, h128))
    z = xg[:, 2]
    out = {"experiment": "boundary", "n": n_particles, "precision": precision, "levels": []}
    F_bc = {}
    for n in (128, 256):
        base = m.auto_mesh(xg, m.Params(n=(n,) * 3, rc_over_h=3.0, pm_bc=1, z_cathode=0.0,
                                        precision=precision))
        rc = base.rc_over_h * max(base.h)
        res, img = {}, 0
        for pp_bc in (0, 1):
            ctx = m.Context(m.Params(**{**base.__dict__, "pp_bc": pp_bc}), n_particles)
            res[pp_bc] = ctx.forces(xg)
            if pp_bc == 0:
                # the same evaluation again: the summation order inside cells is not fixed, so
                # this measures the rounding floor under which force differences mean nothing
                again = ctx.forces(xg)
            ctx.sync()
            if pp_bc:
                img = ctx.pair_count()[1]
            ctx.close()
        floor = torch.linalg.norm(again - res[0], dim=1)
        dF = res[1] - res[0]
        changed = torch.linalg.norm(dF, dim=1) > 10.0 * floor.max() + 1e-300
        out["levels"].append({
            "mesh": n, "h": list(base.h), "rc": rc,
            "bc_rel_l2": _rel(res[0], res[1]),
            "rounding_floor_rel_l2": _rel(again, res[0]),
            "image_pairs": img,
            "particles_within_rc_of_cathode": int((z < rc).sum()),
            "particles_changed": int(changed.sum()),
            "max_height_changed_over_rc": float(z[changed].max() / rc) if changed.any() else 0.0,
        })
        F_bc[n] = res[1]
        del res, dF, again
    out["refinement_rel_l2_128_vs_256"] = _rel(F_bc[128], F_bc[256])
    out["ratio_bc_over_refinement_at_128"] = (out["levels"][0]["bc_rel_l2"]
                                              / out["refinement_rel_l2_128_vs_256"])
    return out


def _grad_bunch(n):
    spec = dict(B.WORKLOADS["gauss1m"])
    x = B.positions(spec, n)
    p = B.momenta(spec, n)
    return x, p


def energy(precision: int = m.FP32_MIXED, n_particles: int = 1_048_576, steps: int = 100):
    x, p = _grad_bunch(n_particles)
    xg, pg = _cuda(x), _cuda(p)
    # a mesh with room for the bunch to move: the bounding box of the initial bunch, widened
    prm = m.auto_mesh(_cuda(x * 1.05), m.Params(n=(64,) * 3, rc_over_h=2.0, precision=precision))
    ctx = m.Context(prm, n_particles)
    mass = prm.mass
    k_e = 8.9875517923e9
    self_e = n_particles * k_e * prm.q ** 2 * (prm.kappa / (prm.rc_over_h * max(prm.h))) / math.sqrt(math.pi)

    def total_energy():
        f, e = ctx.forces(xg, energy=True)
        ke = float((pg * pg).sum()) / (2 * mass)
        return ke + float(e.sum()) - self_e, f

    E0, f = total_energy()
    P0 = pg.sum(dim=0).clone()
    # the short range conserves momentum pair by pair: sum_i F^S_i against sum_i |F^S_i|
    fs = ctx.forces(xg, parts=1)
    sum_fs_rel = float(torch.linalg.norm(fs.sum(dim=0))) / float(torch.linalg.norm(fs, dim=1).sum())
    t0 = time.time()
    energies = [E0]
    for _ in range(steps // 10):
        f = ctx.push(xg, pg, 1e-12, 10, f)
        energies.append(total_energy()[0])
    ctx.sync()
    elapsed = time.time() - t0
    P1 = pg.sum(dim=0)
    scale = float(torch.linalg.norm(pg, dim=1).sum())
    return {"experiment": "energy", "n": n_particles, "steps": steps, "precision": precision,
            "E0": E0, "rel_drift_final": (energies[-1] - E0) / abs(E0),
            "rel_drift_max": max(abs(e - E0) for e in energies) / abs(E0),
            "momentum_change_rel": float(torch.linalg.norm(P1 - P0)) / scale,
            "short_range_force_sum_rel": sum_fs_rel, "seconds": elapsed}


def gradient(precision: int = m.FP32_MIXED, n_particles: int = 1_048_576, steps: int = 200,
             every: int = 20, directions: int = 2, dt: float = 2.5e-13):
    x, p = _grad_bunch(n_particles)
    spec_mesh = m.auto_mesh(_cuda(x * 1.05), m.Params(n=(64,) * 3, rc_over_h=2.0,
                                                       precision=precision,
                                                       adj_slots=(steps + every - 1) // every,
                                                       adj_segment=every))
    ctx = m.Context(spec_mesh, n_particles)
    x0, p0 = _cuda(x), _cuda(p)

    def J(xa, pa):
        xx, pp = xa.clone(), pa.clone()
        ctx.push(xx, pp, dt, steps)
        return float(ctx.emittance(xx, pp).sum()), xx, pp

    t0 = time.time()
    J0, xT, pT = J(x0, p0)
    _, gxT, gpT = ctx.emittance(xT, pT, grad=True)
    gx0, gp0 = ctx.backward(x0, p0, dt, steps, gxT, gpT)
    ctx.sync()
    t_grad = time.time() - t0
    # directions that change the emittance at first order: dilations of the positions and of the
    # momenta about their means (a random direction's first-order change nearly cancels over
    # a million particles and drowns in the rounding of the FP32 force sums)
    dirs = [("dilate_x", x0 - x0.mean(dim=0), torch.zeros_like(p0)),
            ("dilate_p", torch.zeros_like(x0), p0 - p0.mean(dim=0))]
    res = []
    for name, vx, vp in dirs[:directions]:
        eps = 1e-6 if precision == m.FP64 else 1e-3
        Jp, _, _ = J(x0 + eps * vx, p0 + eps * vp)
        Jm, _, _ = J(x0 - eps * vx, p0 - eps * vp)
        fd = (Jp - Jm) / (2 * eps)
        ad = float((gx0 * vx).sum() + (gp0 * vp).sum())
        res.append({"direction": name, "fd": fd, "adjoint": ad, "rel_diff": abs(fd - ad) / abs(fd)})
    return {"experiment": "gradient", "n": n_particles, "steps": steps, "dt": dt,
            "checkpoint_every": every,
            "precision": precision, "J": J0, "directions": res, "seconds_gradient": t_grad}


def gradient_coords(precision: int = m.FP64, n_particles: int = 16_384, steps: int = 200,
                    every: int = 20, coords: int = 64, dt: float = 2.5e-13, eps_rel: float = 1e-6,
                    seed: int = 0, deterministic: int = 0, compare_fp32: bool = True):
    """Reverse-pass gradient of J against central finite differences on randomly chosen single
    coordinates (positions and momenta), step eps_rel times that component's rms spread; and the
    FP32 mixed path's reverse pass against the FP64 one on every coordinate. deterministic = 1
    (FP64) makes every trajectory bitwise reproducible, so the differences carry no summation
    noise."""
    x, p = _grad_bunch(n_particles)
    base = dict(n=(64,) * 3, rc_over_h=2.0, adj_slots=(steps + every - 1) // every,
                adj_segment=every)
    prm = m.auto_mesh(_cuda(x * 1.05), m.Params(precision=precision, deterministic=deterministic,
                                                **base))
    ctx = m.Context(prm, n_particles)
    x0, p0 = _cuda(x), _cuda(p)

    def J(c, xa, pa):
        xx, pp = xa.clone(), pa.clone()
        c.push(xx, pp, dt, steps)
        return float(c.emittance(xx, pp).sum()), xx, pp

    def adjoint(c):
        _, xT, pT = J(c, x0, p0)
        _, gxT, gpT = c.emittance(xT, pT, grad=True)
        gx, gp = c.backward(x0, p0, dt, steps, gxT, gpT)
        c.sync()
        return torch.cat([gx.reshape(-1), gp.reshape(-1)])

    t0 = time.time()
    g = adjoint(ctx)
    t_grad = time.time() - t0
    rng = np.random.default_rng(seed)
    picks = rng.choice(6 * n_particles, size=coords, replace=False)
    scale = np.concatenate([x.std(axis=0), p.std(axis=0)])
    fd, ad = [], []
    t0 = time.time()
    for k in picks:
        half, r = divmod(int(k), 3 * n_particles)  # half 0: positions, 1: momenta
        i, d = divmod(r, 3)
        h = eps_rel * float(scale[3 * half + d])
        vals = []
        for sgn in (1.0, -1.0):
            xx, pp = x0.clone(), p0.clone()
            (xx if half == 0 else pp)[i, d] += sgn * h
            vals.append(J(ctx, xx, pp)[0])
        fd.append((vals[0] - vals[1]) / (2 * h))
        ad.append(float(g[k]))
    t_fd = time.time() - t0
    fd, ad = np.array(fd), np.array(ad)
    rel = np.abs(fd - ad) / np.maximum(np.abs(fd), 1e-300)
    out = {"experiment": "gradient_coords", "n": n_particles, "steps": steps, "dt": dt,
           "checkpoint_every": every, "precision": precision, "deterministic": deterministic,
           "coords": coords,
           "eps_rel": eps_rel, "rel_l2_over_coords": float(np.linalg.norm(fd - ad)
                                                          / np.linalg.norm(fd)),
           "max_rel": float(rel.max()), "median_rel": float(np.median(rel)),
           "coords_above_1e-4": int((rel > 1e-4).sum()),
           "seconds_gradient": t_grad, "seconds_fd": t_fd}
    out["fd"] = fd.tolist()
    out["adjoint"] = ad.tolist()
    if precision == m.FP64 and compare_fp32:
        ctx.close()
        c32 = m.Context(m.auto_mesh(_cuda(x * 1.05), m.Params(precision=m.FP32_MIXED, **base)),
                        n_particles)
        g32 = adjoint(c32)
        out["fp32_adjoint_vs_fp64_rel_l2"] = float((g32 - g).norm() / g.norm())
    return out


def _coulomb_direct(x, targets, q, z_cathode=None, chunk=8):
    """Exact Coulomb force on the particles `targets` from all of x (FP64, torch on the GPU), with
    the grounded-plane images (charge -q at the mirror point) when z_cathode is given."""
    k_e = 8.9875517923e9
    out = torch.zeros((len(targets), 3), dtype=torch.float64, device=x.device)
    for a in range(0, len(targets), chunk):
        t = x[targets[a:a + chunk]]
        d = t[:, None, :] - x[None, :, :]
        r2 = (d * d).sum(-1)
        r2[r2 == 0] = float("inf")            # the particle itself
        out[a:a + chunk] = k_e * q * q * (d / r2[..., None] ** 1.5).sum(1)
        if z_cathode is not None:
            xi = x.clone()
            xi[:, 2] = 2.0 * z_cathode - xi[:, 2]
            d = t[:, None, :] - xi[None, :, :]
            r2 = (d * d).sum(-1)
            out[a:a + chunk] -= k_e * q * q * (d / r2[..., None] ** 1.5).sum(1)
    return out


def influence(precision: int = m.FP64, n_particles: int = 0):
    """P3M force error against the exact Coulomb force (with images) for the plain sampled
    kernel (influence 0), the principal-alias optimal factor (1) and the alias sums of
    eq. (Ghfinal) (2): the 4096-particle Gaussian above the cathode (16^3 mesh, all particles)
    and the 4,194,304-particle core + halo bunch (128^3, r_c = 3h, 2048 sampled targets)."""
    out = {"experiment": "influence", "precision": precision, "cases": []}
    g4 = B.lift_to_plane(B.gaussian(4096, (1e-3, 1e-3, 1e-3), 0), 0.0, 0.15e-3)
    halo = dict(B.WORKLOADS["halo4m"])
    x5 = B.positions(halo, 4_194_304)
    h128 = m.auto_mesh(_cuda(x5), m.Params(n=(128,) * 3)).h[2]
    x5 = B.lift_to_plane(x5, 0.0, h128)
    for name, x, n, rc, sample in (("gauss4096_cathode_16", g4, 16, 2.0, None),
                                   ("halo4m_cathode_128", x5, 128, 3.0, 2048)):
        xg = _cuda(x)
        targets = (torch.arange(len(x), device="cuda") if sample is None else
                   torch.from_numpy(B.subsample(len(x), sample, seed=12345)).cuda())
        case = {"case": name, "n": len(x), "mesh": n, "targets": len(targets), "rel_l2": {}}
        exact = None
        for infl in (0, 1, 2):
            prm = m.auto_mesh(xg, m.Params(n=(n,) * 3, rc_over_h=rc, pm_bc=1, z_cathode=0.0,
                                           influence=infl, precision=precision))
            t0 = time.time()
            ctx = m.Context(prm, len(x))
            ctx.sync()
            t_create = time.time() - t0
            f = ctx.forces(xg)
            ctx.sync()
            ctx.close()
            if exact is None:
                exact = _coulomb_direct(xg, targets, prm.q, z_cathode=0.0)
            case["rel_l2"][infl] = _rel(f[targets], exact)
            case[f"create_s_{infl}"] = t_create
        out["cases"].append(case)
    return out


def error_measure(precision: int = m.FP64, n_particles: int = 0):
    """Error measure of eq. (error_measure) for one particle at height z above the grounded
    cathode (Sec. 3.1.1), on the GPU path. The potential of the source at a probe point x is
    read from energies, P3M being linear in the charges: phi(x) = (U(source + probe) -
    U(source) - U(probe)) / q. Over a grid of probe points in the domain above the cathode:
      E_bc(z)      = sum_x |phi(pp_bc = 0) - phi(pp_bc = 1)|^2 dV  (the short-range boundary
                     term the paper neglects), against the paper's closed form: the image's
                     screened potential k_e q erfc(alpha r)/r, r = |x - S(xi)| < r_c;
      E_mesh(z, h) = sum_x |phi(pp_bc = 1) - Phi(x)|^2 dV, Phi the exact potential with image,
                     for h = r_c/2, r_c/4, r_c/8 (r_c fixed).
    The paper's claim: E_bc vanishes once no probe's image is within r_c (z >= r_c), and the
    particle's own image acts only below r_c/2."""
    from scipy.special import erfc as _erfc
    k_e = 8.9875517923e9
    q = B.macro_charge()
    rc = 1e-4
    kappa = 3.0
    alpha = kappa / rc
    heights = [0.05, 0.1, 0.2, 0.3, 0.45, 0.55, 0.75, 1.0, 1.25]
    step = rc / 3
    gx = np.arange(-3, 4) * step
    gz = (np.arange(0, 8) + 0.5) * step
    probes_all = np.stack(np.meshgrid(gx, gx, gz, indexing="ij"), -1).reshape(-1, 3)
    dV = step ** 3
    out = {"experiment": "error_measure", "precision": precision, "r_c": rc, "kappa": kappa,
           "probe_step_over_rc": 1 / 3, "rows": []}
    meshes = [("h=rc/2", 2.0), ("h=rc/4", 4.0), ("h=rc/8", 8.0)]
    ctxs = {}
    for name, rch in meshes:
        h = rc / rch
        n = int(math.ceil(3.0 * rc / h)) + 5
        lo = (-1.5 * rc - 2 * h, -1.5 * rc - 2 * h, -2 * h)
        for pp_bc in (0, 1):
            prm = m.Params(n=(n, n, n), lo=lo, h=(h, h, h), rc_over_h=rch, kappa=kappa,
                           pm_bc=1, pp_bc=pp_bc, z_cathode=0.0, precision=precision, q=q)
            ctxs[(name, pp_bc)] = m.Context(prm, 2)
    cache = {}

    def energy(ctx_key, pts):
        key = (ctx_key, tuple(np.round(np.asarray(pts).ravel() / rc, 9)))
        if key not in cache:
            _, e = ctxs[ctx_key].forces(_cuda(np.asarray(pts)), energy=True)
            cache[key] = float(e.sum())
        return cache[key]

    for zs in heights:
        xi = np.array([0.0, 0.0, zs * rc])
        probes = probes_all[probes_all[:, 2] <= xi[2] + rc]
        probes = probes[np.linalg.norm(probes - xi, axis=1) > 0.25 * rc]  # off the source
        d = probes - xi
        di = probes - xi * np.array([1, 1, -1])
        r, ri = np.linalg.norm(d, axis=1), np.linalg.norm(di, axis=1)
        exact = k_e * q * (1 / r - 1 / ri)
        img = np.where(ri < rc, k_e * q * _erfc(alpha * ri) / ri, 0.0)
        row = {"z_over_rc": zs, "probes": len(probes),
               "E_bc_closed": float((img ** 2).sum() * dV), "E_mesh": {}, "E_total_pp_bc0": {}}
        for name, _ in meshes:
            phi = {}
            for pp_bc in (0, 1):
                key = (name, pp_bc)
                us = energy(key, [xi])
                phi[pp_bc] = np.array([(energy(key, [xi, x]) - us - energy(key, [x])) / q
                                       for x in probes])
            if name == meshes[0][0]:
                row["E_bc_gpu"] = float(((phi[0] - phi[1]) ** 2).sum() * dV)
            else:
                row.setdefault("E_bc_gpu_other_meshes", []).append(
                    float(((phi[0] - phi[1]) ** 2).sum() * dV))
            row["E_mesh"][name] = float(((phi[1] - exact) ** 2).sum() * dV)
            row["E_total_pp_bc0"][name] = float(((phi[0] - exact) ** 2).sum() * dV)
        out["rows"].append(row)
    for c in ctxs.values():
        c.close()
    return out


def action(precision: int = m.FP32_MIXED, n_particles: int = 1_048_576, steps: int = 20):
    """Discrete-action diagnostics (eq. (full_p3m_lagrangian) with the leapfrog patch of
    eq. (leapfrog)) along a trajectory of the 1,048,576-particle Gaussian bunch (64^3, r_c = 2h,
    dt = 1e-12 s): the discrete Euler-Lagrange residual M (x^{n+1} - 2x^n + x^{n-1})/dt^2 - F(x^n)
    (F the force the step used), relative to max |F|; the discrete action
    S_d = dt sum_n [sum_i M |x^{n+1}_i - x^n_i|^2 / (2 dt^2) - U(x^n)], U the P3M energy; and its
    central difference along a random variation of the interior points, relative to the kinetic
    part's, on the trajectory and off it."""
    x, p = _grad_bunch(n_particles)
    xg, pg = _cuda(x), _cuda(p)
    prm = m.auto_mesh(_cuda(x * 1.05), m.Params(n=(64,) * 3, rc_over_h=2.0, precision=precision))
    ctx = m.Context(prm, n_particles)
    dt, M = 1e-12, prm.mass
    f = ctx.forces(xg)
    X, F = [xg.clone()], [f.clone()]
    for _ in range(steps):
        f = ctx.push(xg, pg, dt, 1, f)
        X.append(xg.clone())
        F.append(f.clone())
    res = max(float((M * (X[k + 1] - 2 * X[k] + X[k - 1]) / dt ** 2 - F[k]).abs().max()) /
              float(F[k].abs().max()) for k in range(1, steps))

    def U(y):
        _, e = ctx.forces(y, energy=True)
        return float(e.sum())

    def S(Xs):
        return dt * sum(0.5 * M * float(((Xs[k + 1] - Xs[k]) ** 2).sum()) / dt ** 2 - U(Xs[k])
                        for k in range(len(Xs) - 1))

    gen = torch.Generator(device="cuda").manual_seed(5)
    V = [torch.zeros_like(xg)] + [torch.randn(xg.shape, dtype=xg.dtype, device="cuda",
                                              generator=gen) for _ in range(steps - 1)] + \
        [torch.zeros_like(xg)]
    kin = dt * sum(abs(float((M * (X[k] - X[k - 1]) / dt ** 2 * V[k]).sum()))
                   for k in range(1, steps))
    eps = 1e-9

    def dS(Xs):
        return (S([a + eps * v for a, v in zip(Xs, V)]) -
                S([a - eps * v for a, v in zip(Xs, V)])) / (2 * eps)

    on = dS(X)
    off = dS([a + 1e-7 * v for a, v in zip(X, V)])
    S0 = S(X)
    ctx.sync()
    return {"experiment": "action", "n": n_particles, "steps": steps, "precision": precision,
            "el_residual_max_rel": res, "S_d": S0, "dS_on_trajectory_rel": on / kin,
            "dS_off_trajectory_rel": off / kin}


def box_potentials(precision: int = m.FP64, n_particles: int = 0, save: str = ""):
    """The three potentials of the paper's grounded-box figure (fig. boundary_gauss_seidel_results)
    for two opposite charges in a grounded box of 50^3 nodes (h = 0.1 mm, r_c = 2h, kappa = 3):
    phi^L from the box solve (pm_bc = 2), phi^S = k_e q erfc(alpha r)/r, and phi^tot, the discrete
    Poisson solution of the unscreened assigned charges (the same solve with the screening
    switched off). The API carries one charge value, so +q at A and -q at B come from two
    single-charge solves (P3M is linear in the charges). Reports, on the nodes farther than 2 r_c
    from both charges, the relative L2 difference between phi^S + phi^L and phi^tot, and the
    reach of phi^S; saves the mid-plane slices to `save` (.npz) when given."""
    from scipy.special import erfc as _erfc
    k_e = 8.9875517923e9
    n, h = 50, 1e-4
    q = B.macro_charge()
    lo = (0.0, 0.0, 0.0)
    centre = np.array([24.5, 24.5, 24.5]) * h
    A = centre + np.array([-6.0, 0.0, 0.0]) * h + np.array([0.0, 0.5, 0.5]) * h
    Bp = centre + np.array([6.0, 0.0, 0.0]) * h + np.array([0.0, 0.5, 0.5]) * h

    def potential(pos, screened=True):
        prm = m.Params(n=(n, n, n), lo=lo, h=(h, h, h), rc_over_h=2.0, pm_bc=2, precision=m.FP64,
                       q=q, alpha=0.0 if screened else 1e14)
        ctx = m.Context(prm, 1)
        ctx.deposit(_cuda(pos[None, :]))
        ctx.solve()
        phi = ctx.get_mesh(1).cpu().numpy()      # [z, y, x]
        ctx.sync()
        ctx.close()
        return phi

    phiL = potential(A) - potential(Bp)
    phiT = potential(A, False) - potential(Bp, False)
    g = np.arange(n) * h
    Z, Y, X = np.meshgrid(g, g, g, indexing="ij")
    nodes = np.stack([X, Y, Z], -1)
    rc = 2 * h
    alpha = 3.0 / rc

    def short(c):
        r = np.linalg.norm(nodes - c, axis=-1)
        return np.where(r > 0, k_e * q * _erfc(alpha * r) / np.maximum(r, 1e-30), 0.0)

    phiS = short(A) - short(Bp)
    far = (np.linalg.norm(nodes - A, axis=-1) > 2 * rc) & (np.linalg.norm(nodes - Bp, axis=-1) > 2 * rc)
    inner = np.zeros_like(far)
    inner[1:-1, 1:-1, 1:-1] = True
    mask = far & inner
    diff = (phiS + phiL - phiT)[mask]
    out = {"experiment": "box_potentials", "n": n, "h": h, "r_c": rc,
           "rel_l2_phiS_plus_phiL_vs_phiTot_far": float(np.linalg.norm(diff) /
                                                        np.linalg.norm(phiT[mask])),
           "max_abs_phiS_beyond_rc_over_max_phiL": float(
               np.abs(phiS[~((np.linalg.norm(nodes - A, axis=-1) <= rc) |
                             (np.linalg.norm(nodes - Bp, axis=-1) <= rc))]).max() /
               np.abs(phiL).max()),
           "faces_max_abs_phiL": float(max(np.abs(phiL[0]).max(), np.abs(phiL[-1]).max(),
                                           np.abs(phiL[:, 0]).max(), np.abs(phiL[:, -1]).max(),
                                           np.abs(phiL[:, :, 0]).max(), np.abs(phiL[:, :, -1]).max())),
           "max_abs": {"phiL": float(np.abs(phiL).max()), "phiS": float(np.abs(phiS).max()),
                       "phiTot": float(np.abs(phiT).max())}}
    if save:
        zc = 24
        np.savez(save, phiL=phiL[zc], phiS=phiS[zc], phiTot=phiT[zc], h=h)
    return out


def main(argv):
    which = argv[1] if len(argv) > 1 else "boundary"
    kw = {"precision": m.FP64 if "--fp64" in argv else m.FP32_MIXED}
    if "--n" in argv:
        kw["n_particles"] = int(argv[argv.index("--n") + 1])
    if "--save" in argv:
        kw["save"] = argv[argv.index("--save") + 1]
    if "--det" in argv:
        kw["deterministic"] = 1
    if "--coords" in argv:
        kw["coords"] = int(argv[argv.index("--coords") + 1])
    if "--steps" in argv:
        kw["steps"] = int(argv[argv.index("--steps") + 1])
    fn = {"boundary": boundary, "energy": energy, "gradient": gradient,
          "gradient_coords": gradient_coords,
          "influence": influence, "error_measure": error_measure, "action": action,
          "box_potentials": box_potentials}[which]
    print(json.dumps(fn(**kw)), flush=True)


if __name__ == "__main__":
    main(sys.argv)
