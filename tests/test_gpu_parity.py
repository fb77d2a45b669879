"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle, element by element,
on the same seeded inputs.

Tolerances (relative L2 over all components): FP64 path 1e-12, FP32 mixed path 1e-5; the
in-cutoff pair count is an integer decided in FP64 on both sides and must match exactly.
"""
import dataclasses
import math

import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2103_02046_gb300 import bunches as B

pytestmark = pytest.mark.gpu

TOL = {0: 1e-12, 1: 1e-5}


def p3m():
    from paper_2103_02046_gb300 import p3m as m
    return m


def gpu_params(P: O.Params, precision: int, **kw):
    m = p3m()
    return m.Params(n=P.n, lo=P.lo, h=P.h, rc_over_h=P.rc_over_h, kappa=P.kappa, alpha=P.alpha,
                    assign_order=P.assign_order, pm_bc=P.pm_bc, pp_bc=P.pp_bc,
                    z_cathode=P.z_cathode, influence=P.influence, precision=precision,
                    q=P.q, mass=P.mass, **kw)


def cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


def rel(a, b):
    return O.rel_l2(a.cpu().numpy() if torch.is_tensor(a) else a, b)


def bunch_4k(cathode: bool):
    x = B.gaussian(4096, (1e-3, 1e-3, 1e-3), 0)
    if cathode:
        x = B.lift_to_plane(x, 0.0, 0.15e-3)
    return x


CASES = [
    # (name, n, pm_bc, pp_bc, order, influence)
    ("open_tsc", 16, 0, 0, 2, 0),
    ("cathode_tsc", 16, 1, 0, 2, 0),
    ("cathode_pp_bc", 16, 1, 1, 2, 0),
    ("open_cic", 16, 0, 0, 1, 0),
    ("cathode_influence", 16, 1, 0, 2, 1),
    ("aniso_ragged", (16, 20, 24), 1, 1, 2, 0),
    # doubled z length a power of two >= 64: the FP32 path's fused z solve
    ("open_tsc_32", 32, 0, 0, 2, 0),
    ("cathode_pp_bc_aniso_z64", (20, 24, 64), 1, 1, 2, 0),
    ("cathode_cic_influence_32", 32, 1, 0, 1, 1),
    # optimal influence function with its alias sums, on the cuFFT and the fused z solve
    ("cathode_alias_influence", 16, 1, 0, 2, 2),
    ("open_alias_influence_32", 32, 0, 0, 2, 2),
]


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_forces_parity(case, precision):
    name, n, pm_bc, pp_bc, order, infl = case
    x = bunch_4k(pm_bc == 1)
    if name == "aniso_ragged":
        x = x[:3001] * np.array([1.0, 1.3, 0.7])
    P = O.auto_mesh(x, n, rc_over_h=2.0, pm_bc=pm_bc, pp_bc=pp_bc, assign_order=order,
                    influence=infl, z_cathode=0.0)
    ref = O.forces(x, P)
    ctx = p3m().Context(gpu_params(P, precision), len(x))
    xg = cuda(x)
    f_pp = ctx.forces(xg, parts=1)
    np_gpu, ni_gpu = ctx.pair_count()
    # every unordered in-cutoff pair was among the candidates the search handed out
    assert ref.pairs // 2 <= ctx.candidate_count() <= 2 * len(x) * len(x)
    f_pm = ctx.forces(xg, parts=2)
    f, e = ctx.forces(xg, energy=True)
    ctx.sync()
    tol = TOL[precision]
    assert rel(f_pp, ref.F_pp) <= tol
    assert rel(f_pm, ref.F_pm) <= tol
    assert rel(f, ref.F) <= tol
    if precision == 0:
        assert (np_gpu, ni_gpu) == (ref.pairs, ref.image_pairs)
    else:
        assert abs(np_gpu - ref.pairs) <= max(2, 1e-5 * ref.pairs)
    e = e.cpu().numpy()
    assert e[0] == pytest.approx(ref.U_pp, rel=10 * tol)
    assert e[1] == pytest.approx(ref.U_pm, rel=10 * tol)


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("kappa", [1.5, 6.0, 7.0])
def test_short_range_kappa(kappa, precision):
    # the pair function's fits depend on kappa = alpha r_c: the FP64 path evaluates it in
    # double-float arithmetic up to kappa = 6.5 (intervals of erfc(x) e^{x^2}, an exact ln2/16
    # reduction of e^{-x^2}) and in FP64 above; the FP32 path fits t P(t - t_c),
    # t = 1/(1 + 0.47 x), to its FP32 floor for any kappa. Forces, energy, pair count and the
    # force VJP (the Hessian terms) against the oracle, with images (pp_bc = 1) above a cathode.
    x = bunch_4k(True)
    P = O.auto_mesh(x, 16, rc_over_h=2.0, kappa=kappa, pm_bc=1, pp_bc=1, z_cathode=0.0)
    ref = O.forces(x, P, parts=1)
    ctx = p3m().Context(gpu_params(P, precision), len(x))
    xg = cuda(x)
    f, e = ctx.forces(xg, energy=True, parts=1)
    npairs, nimg = ctx.pair_count()
    w = np.random.default_rng(31).standard_normal(x.shape)
    g = ctx.force_vjp(xg, cuda(w))
    ctx.sync()
    tol = TOL[precision]
    assert rel(f, ref.F_pp) <= tol
    assert e.cpu().numpy()[0] == pytest.approx(ref.U_pp, rel=10 * tol)
    if precision == 0:
        assert (npairs, nimg) == (ref.pairs, ref.image_pairs)
        assert rel(g, O.force_vjp(x, w, P)) <= 1e-11
    else:
        assert rel(g, O.force_vjp(x, w, P)) <= 2e-5


@pytest.mark.parametrize("precision", [0, 1])
def test_mesh_charge_and_potential(precision):
    x = bunch_4k(True)
    P = O.auto_mesh(x, 16, pm_bc=1, z_cathode=0.0)
    Q, _ = O.deposit(x, P)
    phi = O.solve(Q, P)
    ctx = p3m().Context(gpu_params(P, precision), len(x))
    ctx.deposit(cuda(x))
    Qg = ctx.get_mesh(0)
    ctx.solve()
    phig = ctx.get_mesh(1)
    ctx.sync()
    assert rel(Qg, Q) <= (1e-14 if precision == 0 else 1e-6)
    assert rel(phig, phi) <= (1e-13 if precision == 0 else 1e-5)
    assert float(Qg.sum()) == pytest.approx(len(x) * P.q, rel=1e-12 if precision == 0 else 1e-6)


DIFF_CASES = [("open_32_fused", 32, 0), ("cathode_20x24x64_fused", (20, 24, 64), 1),
              ("cathode_16_cufft", 16, 1)]


@pytest.mark.parametrize("case", DIFF_CASES, ids=[c[0] for c in DIFF_CASES])
def test_fp32_difference_fields(case):
    # the FP32 path's long range convolves the charge with forward-difference kernels (the fused
    # z solve for a doubled z length of 64 or more, cuFFT and the Green's multiply otherwise):
    # D_d phi(g) = phi(g + e_d) - phi(g) against the differences of the oracle's FP64 potential,
    # on every node whose neighbour g + e_d is on the mesh
    _, n, pm_bc = case
    x = bunch_4k(pm_bc == 1)
    P = O.auto_mesh(x, n, pm_bc=pm_bc, z_cathode=0.0)
    phi = O.solve(O.deposit(x, P)[0], P)
    ctx = p3m().Context(gpu_params(P, 1), len(x))
    with pytest.raises(p3m().P3MError):
        ctx.get_mesh(2)          # nothing computed yet
    ctx.forces(cuda(x))
    D = [ctx.get_mesh(2 + d).cpu().numpy() for d in range(3)]
    ctx.sync()
    ref = [phi[:, :, 1:] - phi[:, :, :-1], phi[:, 1:, :] - phi[:, :-1, :],
           phi[1:, :, :] - phi[:-1, :, :]]
    got = [D[0][:, :, :-1], D[1][:, :-1, :], D[2][:-1, :, :]]
    for d in range(3):
        assert rel(got[d], ref[d]) <= 1e-5, d
    ctx.close()


@pytest.mark.parametrize("order", [1, 2])
def test_deposit_dense_clump(order):
    # 3072 coincident particles on one mesh node: a deposit block (1024 particles) puts its
    # largest possible weight (1 for CIC, 27/64 for TSC) on one node, the edge of the FP32
    # fixed-point tile's range
    base = bunch_4k(False)
    P = O.auto_mesh(base, 16, assign_order=order)
    node = np.array([P.lo[d] + 8 * P.h[d] for d in range(3)])
    x = np.concatenate([base, np.repeat(node[None, :], 3072, axis=0)])
    Q, _ = O.deposit(x, P)
    for precision in (0, 1):
        ctx = p3m().Context(gpu_params(P, precision), len(x))
        ctx.deposit(cuda(x))
        Qg = ctx.get_mesh(0)
        ctx.sync()
        ctx.close()
        # one node sums 3072 equal weights, in another order than the oracle's: FP64 rounding
        # up to about 3072 * 2^-53 = 3.4e-13 of that node, which dominates the L2 norm
        assert rel(Qg, Q) <= (1e-12 if precision == 0 else 1e-6)
        assert float(Qg.max()) == pytest.approx(float(Q.max()),
                                                rel=1e-12 if precision == 0 else 1e-6)


@pytest.mark.parametrize("precision", [0, 1])
def test_lattice_pairs_at_cutoff(precision):
    # a 16^3 cubic lattice (spacing a) whose second neighbours along the axes sit just inside the
    # cutoff (by 1e-10 relative for FP64, 1e-5 for FP32, where the cutoff test runs in FP32);
    # lattice planes fall at every offset from the short-range row boundaries, so every pair has
    # to be found across rows whatever the rounding of the binning
    a = 1e-4
    g = np.arange(16) * a
    x = np.stack(np.meshgrid(g, g, g, indexing="ij"), axis=-1).reshape(-1, 3) + 3e-3
    inside = 1e-10 if precision == 0 else 1e-5
    h = 15 * a / 11   # auto_mesh spacing for n = 16 over a 15a box
    P = O.auto_mesh(x, 16, rc_over_h=2 * a * (1 + inside) / h)
    ref = O.forces(x, P)
    # ordered pairs: each lattice offset d with |d|^2 <= 4 (in units of a) taken both ways
    offsets = [(i, j, k) for i in range(-2, 3) for j in range(-2, 3) for k in range(-2, 3)]
    assert ref.pairs == sum(2 * (16 - abs(i)) * (16 - abs(j)) * (16 - abs(k))
                            for i, j, k in offsets
                            if 0 < i * i + j * j + k * k <= 4 and (i, j, k) > (0, 0, 0))
    ctx = p3m().Context(gpu_params(P, precision), len(x))
    f_pp = ctx.forces(cuda(x), parts=1)
    npairs, _ = ctx.pair_count()
    ncand = ctx.candidate_count()
    ctx.sync()
    assert npairs == ref.pairs
    assert rel(f_pp, ref.F_pp) <= TOL[precision]
    # the row search looks at about 8 r_c^3 per particle, the cutoff sphere is 4.19 r_c^3
    assert npairs // 2 <= ncand <= 8 * npairs


@pytest.mark.parametrize("layout", ["counts", "sparse_rows"])
def test_fp32_short_range_lane_pairs(layout):
    # the FP32 short range holds two adjacent sorted particles per lane: odd counts (a lane
    # whose second particle does not exist), a single particle, and neighbours that the sort put
    # in different cell rows (each particle then walks its own runs) must all give every pair
    # exactly once
    if layout == "counts":
        x4 = bunch_4k(False)
        P = O.auto_mesh(x4, 16, rc_over_h=2.0)
        core = x4[np.argsort(np.linalg.norm(x4, axis=1))]  # densest first: many pairs
        sets = [core[:n] for n in (1, 2, 3, 255, 256, 257, 513)]
    else:
        # about one particle per cell row, so most lanes straddle a row boundary
        x = np.random.default_rng(7).uniform(-1e-3, 1e-3, size=(301, 3))
        P = O.auto_mesh(x, 16, rc_over_h=1.0)
        sets = [x, x[:300]]
    ctx = p3m().Context(gpu_params(P, 1), max(len(s) for s in sets))
    for x in sets:
        ref = O.forces(x, P)
        f_pp = ctx.forces(cuda(x), parts=1).cpu().numpy()
        npairs, _ = ctx.pair_count()
        ctx.sync()
        err = np.linalg.norm(f_pp - ref.F_pp)
        assert err <= TOL[1] * np.linalg.norm(ref.F_pp) or (ref.pairs == 0 and err == 0.0)
        assert abs(npairs - ref.pairs) <= max(2, 1e-5 * ref.pairs)
        if layout == "counts" and len(x) >= 255:
            assert ref.pairs > 0
    # an empty evaluation leaves nothing counted
    ctx.forces(torch.zeros((0, 3), dtype=torch.float64, device="cuda"))
    assert ctx.pair_count() == (0, 0) and ctx.candidate_count() == 0


def test_fp32_short_range_compensated_sums():
    """The FP32 short range sums each particle's terms in compensated form: coarse parts on a
    grid where FP32 sums are exact, the small remainders, and the rare big terms apart. A dense
    Gaussian (400,000 particles, about 40,000 neighbours in the core) with one planted pair
    1e-4 cutoff lengths apart, whose pair force is about 1e8 times the force at a cutoff length:
    the sampled forces and the planted pair's own forces match the oracle to 1e-6 relative.
    Plain FP32 sums of that many terms lose a few 1e-6 of the largest partial sum, which for
    the planted pair is its own force."""
    m = p3m()
    x = B.gaussian(400_000, (1e-3, 1e-3, 1e-3), 61)
    P = O.auto_mesh(x, 32, rc_over_h=2.0)
    rc = P.rc_over_h * max(P.h)
    order = np.argsort((x ** 2).sum(1))
    k0, k1 = int(order[0]), int(order[1])
    x[k1] = x[k0] + np.array([0.8e-4, 0.5e-4, -0.3e-4]) * rc
    assert O.auto_mesh(x, 32, rc_over_h=2.0) == P
    idx = np.union1d(B.subsample(len(x), 512, seed=12345), [k0, k1])
    ref = O.forces(x, P, sample=idx)
    ctx = m.Context(gpu_params(P, 1), len(x))
    f = ctx.forces(cuda(x))
    ctx.sync()
    fs = f[torch.from_numpy(idx).cuda()].cpu().numpy()
    pos = np.searchsorted(idx, [k0, k1])
    err_pair = np.linalg.norm(fs[pos] - ref.F[pos], axis=1) / np.linalg.norm(ref.F[pos], axis=1)
    rest = np.setdiff1d(np.arange(len(idx)), pos)
    err_rest = rel(fs[rest], ref.F[rest])
    print(f"planted pair {err_pair}, other sampled particles {err_rest:.3e}, "
          f"pairs per particle {ctx.pair_count()[0] / len(x):.0f}")
    assert np.all(err_pair <= 1e-6)
    assert err_rest <= 1e-6
    ctx.close()


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("bc", [(0, 0), (1, 1)])
def test_short_range_wide_rows(precision, bc):
    # 20,000 particles in a 32^3 mesh at r_c = 0.6h: about 52 cutoff lengths per axis, where the
    # cell budget no longer allows rows r_c / 2 wide with x cells r_c / 4, so the search uses
    # rows r_c wide (the 5 half-shell rows of a 3 x 3 block): forces, pair counts, images and
    # the force VJP through that layout
    pm_bc, pp_bc = bc
    x = np.random.default_rng(31).uniform(-1e-3, 1e-3, size=(20000, 3))
    if pm_bc:
        x = B.lift_to_plane(x, 0.0, 0.005e-3)
    P = O.auto_mesh(x, 32, rc_over_h=0.6, pm_bc=pm_bc, pp_bc=pp_bc, z_cathode=0.0)
    ref = O.forces(x, P)
    ctx = p3m().Context(gpu_params(P, precision), len(x))
    xg = cuda(x)
    f_pp = ctx.forces(xg, parts=1)
    npairs, nimg = ctx.pair_count()
    ncand = ctx.candidate_count()
    f = ctx.forces(xg)
    w = np.random.default_rng(32).standard_normal(x.shape)
    g = ctx.force_vjp(xg, cuda(w))
    ctx.sync()
    tol = TOL[precision]
    assert ref.pairs > 10000 and (pp_bc == 0 or ref.image_pairs > 0)
    assert rel(f_pp, ref.F_pp) <= tol
    assert rel(f, ref.F) <= tol
    if precision == 0:
        assert (npairs, nimg) == (ref.pairs, ref.image_pairs)
    else:
        assert abs(npairs - ref.pairs) <= 2 and abs(nimg - ref.image_pairs) <= 2
    assert ref.pairs // 2 <= ncand
    assert rel(g, O.force_vjp(x, w, P)) <= (1e-11 if precision == 0 else 2e-5)


LAYOUTS = [(1, 4), (2, 4), (2, 16), (3, 4), (3, 16), (3, 32)]


@pytest.mark.parametrize("layout", LAYOUTS, ids=[f"rows{r}_x{c}" for r, c in LAYOUTS])
@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("bc", [(0, 0), (1, 1)])
def test_short_range_search_layouts(layout, precision, bc):
    # every search layout (cell rows per cutoff in y and z, x cells per cutoff) gives the same
    # pairs: a Gaussian bunch (open, or above the cathode with images), forces, pair counts,
    # images and the force VJP against the oracle; and (FP32) a sparse set where most lanes'
    # two particles sit in different cell rows, which with 3 rows walks b's runs after a's
    rows, xcells = layout
    pm_bc, pp_bc = bc
    x = B.gaussian(3000, (0.4e-3, 0.5e-3, 0.6e-3), 71)
    if pm_bc:
        x = B.lift_to_plane(x, 0.0, 0.02e-3)
    P = O.auto_mesh(x, 16, rc_over_h=2.0, pm_bc=pm_bc, pp_bc=pp_bc, z_cathode=0.0)
    ref = O.forces(x, P)
    ctx = p3m().Context(gpu_params(P, precision, search_rows=rows, search_xcells=xcells), len(x))
    xg = cuda(x)
    f = ctx.forces(xg)
    npairs, nimg = ctx.pair_count()
    ncand = ctx.candidate_count() if precision == 1 else None
    w = np.random.default_rng(72).standard_normal(x.shape)
    g = ctx.force_vjp(xg, cuda(w))
    ctx.sync()
    tol = TOL[precision]
    assert ref.pairs > 100000 and (pp_bc == 0 or ref.image_pairs > 0)
    assert rel(f, ref.F) <= tol
    if precision == 0:
        assert (npairs, nimg) == (ref.pairs, ref.image_pairs)
    else:
        assert abs(npairs - ref.pairs) <= 2 and abs(nimg - ref.image_pairs) <= 2
        assert ref.pairs // 2 <= ncand
    assert rel(g, O.force_vjp(x, w, P)) <= (1e-11 if precision == 0 else 2e-5)
    ctx.close()
    if precision == 1 and pm_bc == 0:
        xs = np.random.default_rng(73).uniform(-1e-3, 1e-3, size=(301, 3))
        Ps = O.auto_mesh(xs, 16, rc_over_h=1.0)
        ctx = p3m().Context(gpu_params(Ps, 1, search_rows=rows, search_xcells=xcells), len(xs))
        for xx in (xs, xs[:300]):
            r = O.forces(xx, Ps)
            f_pp = ctx.forces(cuda(xx), parts=1).cpu().numpy()
            n_pp, _ = ctx.pair_count()
            ctx.sync()
            assert r.pairs > 0
            assert np.linalg.norm(f_pp - r.F_pp) <= TOL[1] * np.linalg.norm(r.F_pp)
            assert abs(n_pp - r.pairs) <= 2
        ctx.close()


def test_dense_bunch_picks_three_rows():
    # the 1,048,576-particle Gaussian's context chooses the dense search layout by itself, and
    # an explicit layout reproduces its pair count
    m = p3m()
    spec = dict(B.WORKLOADS["gauss1m"])
    x = B.positions(spec)
    P = O.auto_mesh(x, 64, rc_over_h=2.0)
    xg = cuda(x)
    counts = {}
    for rows in (0, 2, 3):
        ctx = m.Context(gpu_params(P, 0, search_rows=rows), len(x))
        ctx.forces(xg, parts=1)
        counts[rows] = ctx.pair_count()
        if rows == 0:
            assert ctx.search_layout()[0] == 3
        ctx.close()
    assert counts[0] == counts[2] == counts[3]


def _box_case():
    # a bunch inside a grounded box of 20 x 24 x 28 nodes (h = 0.1 mm), supports off the faces
    x = B.gaussian(3000, (0.2e-3, 0.25e-3, 0.3e-3), 51)
    h = 1e-4
    n = (20, 24, 28)
    lo = tuple(-(nd - 1) * h / 2 for nd in n)
    P = O.Params(n=n, lo=lo, h=(h, h, h), pm_bc=2, rc_over_h=2.0)
    return x[O.box_valid(x, P)], P


def test_grounded_box_parity():
    x, P = _box_case()
    ref = O.forces(x, P)
    ctx = p3m().Context(gpu_params(P, 0), len(x))
    xg = cuda(x)
    f_pm = ctx.forces(xg, parts=2)
    f, e = ctx.forces(xg, energy=True)
    phi = ctx.get_mesh(1)
    ctx.sync()
    assert rel(f_pm, ref.F_pm) <= 1e-12
    assert rel(f, ref.F) <= 1e-12
    assert rel(phi, ref.phi_mesh) <= 1e-12
    e = e.cpu().numpy()
    assert e[1] == pytest.approx(ref.U_pm, rel=1e-11)
    w = np.random.default_rng(52).standard_normal(x.shape)
    v = ctx.force_vjp(xg, cuda(w))
    ctx.sync()
    assert rel(v, O.force_vjp(x, w, P)) <= 1e-11


def test_grounded_box_refusals_and_faces():
    m = p3m()
    x, P = _box_case()
    for bad in (dict(precision=1), dict(pp_bc=1), dict(influence=1)):
        kw = dict(n=P.n, lo=P.lo, h=P.h, rc_over_h=P.rc_over_h, pm_bc=2, precision=0)
        kw.update(bad)
        with pytest.raises(m.P3MError) as ei:
            m.Context(m.Params(**kw), 10)
        assert ei.value.status == m.P3M_EINVAL
    ctx = m.Context(gpu_params(P, 0), len(x))
    # TSC support reaching the face nodes: the nearest node is 1
    xb = x[:20].copy()
    xb[3, 2] = P.lo[2] + 1.2 * P.h[2]
    fb = ctx.forces(cuda(xb))
    with pytest.raises(m.P3MError) as ei:
        ctx.sync()
    assert ei.value.status == m.P3M_ERANGE
    assert torch.all(fb[3] == 0)
    f = ctx.forces(cuda(x[:20]))
    ctx.sync()
    assert rel(f, O.forces(x[:20], P).F) <= 1e-12


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("n,order,pm_bc", [(16, 2, 1), (32, 2, 0), (32, 1, 0)],
                         ids=["cathode16", "open32_tsc", "open32_cic"])
def test_central_difference_force_parity(precision, n, order, pm_bc):
    x = bunch_4k(pm_bc == 1)
    P = O.auto_mesh(x, n, rc_over_h=2.0, pm_bc=pm_bc, z_cathode=0.0, assign_order=order,
                    force_diff=1)
    ref = O.forces(x, P)
    ctx = p3m().Context(gpu_params(P, precision, force_diff=1), len(x))
    xg = cuda(x)
    f_pm = ctx.forces(xg, parts=2)
    f = ctx.forces(xg)
    ctx.sync()
    assert rel(f_pm, ref.F_pm) <= TOL[precision]
    assert rel(f, ref.F) <= TOL[precision]
    # momentum: with open boundaries sum_i F^L_i = 0 for central differences (up to rounding of
    # the path); the cathode's image attraction is an external force
    if pm_bc == 0:
        s = float(f_pm.sum(0).abs().max()) / float(f_pm.abs().max())
        assert s <= (1e-10 if precision == 0 else 1e-4)
    with pytest.raises(p3m().P3MError) as ei:
        ctx.force_vjp(xg, torch.ones_like(xg))
    assert ei.value.status == p3m().P3M_ESTATE


def test_central_difference_force_in_the_grounded_box():
    x, P = _box_case()
    P = dataclasses.replace(P, force_diff=1)
    ref = O.forces(x, P)
    ctx = p3m().Context(gpu_params(P, 0, force_diff=1), len(x))
    f = ctx.forces(cuda(x))
    ctx.sync()
    assert rel(f, ref.F) <= 1e-12


def test_auto_mesh_matches_oracle():
    m = p3m()
    x = B.gaussian(5000, (1e-3, 2e-3, 3e-3), 21)
    for n in (16, (16, 24, 32)):
        P = O.auto_mesh(x, n)
        g = m.auto_mesh(cuda(x), m.Params(n=P.n))
        assert tuple(g.h) == P.h and tuple(g.lo) == P.lo


def test_edge_cases():
    m = p3m()
    x = bunch_4k(True)
    P = O.auto_mesh(x, 16, pm_bc=1, z_cathode=0.0)
    ctx = m.Context(gpu_params(P, 0), 100)
    # empty input
    f0 = ctx.forces(torch.zeros((0, 3), dtype=torch.float64, device="cuda"))
    assert f0.shape == (0, 3)
    # a single particle: no pairs; long-range self force only
    x1 = x[:1]
    f1 = ctx.forces(cuda(x1))
    ref = O.forces(x1, P)
    assert rel(f1, ref.F) <= 1e-12
    # n > n_max is refused on the host
    with pytest.raises(m.P3MError) as ei:
        ctx.forces(cuda(x[:101]))
    assert ei.value.status == m.P3M_EINVAL
    # a particle outside the mesh: its force is zero and the error surfaces on sync
    xb = x[:50].copy()
    xb[7, 0] = P.lo[0] - 1e-3
    fb = ctx.forces(cuda(xb))
    with pytest.raises(m.P3MError) as ei:
        ctx.sync()
    assert ei.value.status == m.P3M_ERANGE
    assert torch.all(fb[7] == 0)
    good = np.delete(xb, 7, axis=0)
    ref = O.forces(good, P)
    assert rel(torch.cat([fb[:7], fb[8:]]), ref.F) <= 1e-12
    # the context stays usable
    f2 = ctx.forces(cuda(x[:64]))
    ctx.sync()
    assert rel(f2, O.forces(x[:64], P).F) <= 1e-12
    # a particle below the cathode plane is out of range too
    xc = x[:10].copy()
    xc[3, 2] = -0.01e-3
    ctx.forces(cuda(xc))
    with pytest.raises(m.P3MError):
        ctx.sync()
    # NaN positions
    xn = x[:10].copy()
    xn[2, 1] = np.nan
    ctx.forces(cuda(xn))
    with pytest.raises(m.P3MError) as ei:
        ctx.sync()
    assert ei.value.status == m.P3M_EINVAL


def test_invalid_params_refused():
    m = p3m()
    for bad in (dict(n=(4, 16, 16)), dict(assign_order=3), dict(h=(0.0, 1e-5, 1e-5)),
                dict(precision=7), dict(q=0.0), dict(rc_over_h=0.2),
                dict(influence=3)):
        with pytest.raises(m.P3MError) as ei:
            m.Context(m.Params(**bad), 10)
        assert ei.value.status == m.P3M_EINVAL


@pytest.mark.parametrize("precision", [0, 1])
def test_push_parity(precision):
    x = B.gaussian(2048, (1e-3, 1e-3, 2e-3), 22)
    p = B.thermal_momenta(2048, 1e-4 * B.macro_mass() * B.SPEED_OF_LIGHT, 23)
    P = O.auto_mesh(x * 1.2, 16, rc_over_h=2.0)
    kern = O.green_kernels(P)
    xT, pT, fT = O.push(x, p, 1e-12, 10, P, force=lambda y: O.forces(y, P, kernels=kern).F)
    ctx = p3m().Context(gpu_params(P, precision), len(x))
    xg, pg = cuda(x), cuda(p)
    fg = ctx.push(xg, pg, 1e-12, 10)
    ctx.sync()
    tol = TOL[precision]
    assert rel(xg - cuda(x), xT - x) <= 10 * tol
    assert rel(pg, pT) <= 10 * tol
    assert rel(fg, fT) <= 10 * tol
    # the C-ABI push with f = NULL: the forces stay in the context, the trajectory is the same
    import ctypes
    xn, pn = cuda(x), cuda(p)
    st = p3m().lib().p3m_push(ctx._h, ctypes.c_void_p(xn.data_ptr()),
                              ctypes.c_void_p(pn.data_ptr()), len(x), 1e-12, 10, None)
    assert st == 0
    ctx.sync()
    assert rel(xn - cuda(x), xT - x) <= 10 * tol
    assert rel(pn, pT) <= 10 * tol


@pytest.mark.parametrize("precision", [0, 1])
def test_push_satisfies_discrete_euler_lagrange(precision):
    # eq. (disc_euler_lagrange_eqn) with the leapfrog patch of eq. (leapfrog): the GPU
    # trajectory satisfies M (x^{n+1} - 2 x^n + x^{n-1}) / dt^2 = F(x^n) up to the rounding of
    # the FP64 positions, with F(x^n) the force the step used (returned by the push); in FP64 a
    # fresh evaluation at x^n gives the same force
    x0 = B.gaussian(2048, (1e-3, 1e-3, 1e-3), 41)
    P = O.auto_mesh(x0 * 1.5, 16, rc_over_h=2.0)
    ctx = p3m().Context(gpu_params(P, precision), len(x0))
    xg, pg = cuda(x0), torch.zeros_like(cuda(x0))
    f = ctx.forces(xg)
    dt = math.sqrt(1e-7 / (float(f.abs().max()) / P.mass))
    X, F = [xg.clone()], [f.clone()]
    for _ in range(6):
        f = ctx.push(xg, pg, dt, 1, f)
        X.append(xg.clone())
        F.append(f.clone())
    for n in range(1, 6):
        r = P.mass * (X[n + 1] - 2 * X[n] + X[n - 1]) / dt ** 2 - F[n]
        assert float(r.abs().max()) <= 1e-9 * float(F[n].abs().max())
        if precision == 0:
            assert rel(ctx.forces(X[n]), F[n].cpu().numpy()) <= 1e-13
    ctx.sync()


def test_emittance_parity():
    x = B.gaussian(3000, (1e-3, 2e-3, 3e-3), 24)
    p = B.thermal_momenta(3000, 1e-24, 25) + 1e-21 * x
    P = O.Params()
    ctx = p3m().Context(p3m().Params(n=(8, 8, 8), h=(1e-3,) * 3), 3000)
    eps, gx, gp = ctx.emittance(cuda(x), cuda(p), grad=True)
    ogx, ogp = O.emittance_grad(x, p, P)
    assert rel(eps, O.emittance(x, p, P)) <= 1e-12
    assert rel(gx, ogx) <= 1e-11
    assert rel(gp, ogp) <= 1e-11


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("bc", [(0, 0), (1, 1)])
def test_force_vjp_parity(precision, bc):
    pm_bc, pp_bc = bc
    x = B.lift_to_plane(B.gaussian(1024, (1e-3, 1e-3, 1e-3), 26), 0.0, 0.1e-3)
    P = O.auto_mesh(x, 16, rc_over_h=2.0, pm_bc=pm_bc, pp_bc=pp_bc, z_cathode=0.0)
    w = np.random.default_rng(27).standard_normal(x.shape)
    ref = O.force_vjp(x, w, P)
    ctx = p3m().Context(gpu_params(P, precision), len(x))
    g = ctx.force_vjp(cuda(x), cuda(w))
    ctx.sync()
    assert rel(g, ref) <= (1e-11 if precision == 0 else 2e-5)


@pytest.mark.parametrize("precision", [0, 1])
def test_backward_parity(precision):
    x0 = B.gaussian(512, (1e-3, 1e-3, 2e-3), 28)
    p0 = B.thermal_momenta(512, 1e-4 * B.macro_mass() * B.SPEED_OF_LIGHT, 29)
    P = O.auto_mesh(x0 * 1.3, 16, rc_over_h=2.0)
    kern = O.green_kernels(P)
    dt, T = 2e-12, 7
    xT, pT, _ = O.push(x0, p0, dt, T, P, force=lambda y: O.forces(y, P, kernels=kern).F)
    gxT, gpT = O.emittance_grad(xT, pT, P)
    ogx, ogp = O.backward(x0, p0, dt, T, gxT, gpT, P, kern)
    ctx = p3m().Context(gpu_params(P, precision, adj_slots=4, adj_segment=3), len(x0))
    tol = 1e-10 if precision == 0 else 1e-4
    # checkpoints every adj_segment (3) steps, and every 2 steps (ckpt_every of the call)
    for every in (0, 2):
        gx0, gp0 = ctx.backward(cuda(x0), cuda(p0), dt, T, cuda(gxT), cuda(gpT),
                                ckpt_every=every)
        ctx.sync()
        assert rel(gx0, ogx) <= tol
        assert rel(gp0, ogp) <= tol
    # a checkpoint interval the segment buffer cannot hold, or too few slots for nsteps
    for every, steps in ((4, T), (1, T)):
        with pytest.raises(p3m().P3MError) as ei:
            ctx.backward(cuda(x0), cuda(p0), dt, steps, cuda(gxT), cuda(gpT), ckpt_every=every)
        assert ei.value.status == p3m().P3M_EINVAL


def test_autograd_emittance_gradient():
    m = p3m()
    x0 = B.gaussian(256, (1e-3, 1e-3, 2e-3), 30)
    p0 = B.thermal_momenta(256, 1e-4 * B.macro_mass() * B.SPEED_OF_LIGHT, 31)
    P = O.auto_mesh(x0 * 1.3, 16, rc_over_h=2.0)
    kern = O.green_kernels(P)
    dt, T = 2e-12, 4
    ctx = m.Context(gpu_params(P, 0, adj_slots=2, adj_segment=2), len(x0))
    xg = cuda(x0).requires_grad_(True)
    pg = cuda(p0).requires_grad_(True)
    xT, pT = m.P3MRun.apply(xg, pg, ctx, dt, T)
    J = m.Emittance.apply(xT, pT, ctx)
    J.backward()
    xT_o, pT_o, _ = O.push(x0, p0, dt, T, P, force=lambda y: O.forces(y, P, kernels=kern).F)
    gxT, gpT = O.emittance_grad(xT_o, pT_o, P)
    ogx, ogp = O.backward(x0, p0, dt, T, gxT, gpT, P, kern)
    assert float(J.detach()) == pytest.approx(O.emittance(xT_o, pT_o, P).sum(), rel=1e-12)
    assert rel(xg.grad, ogx) <= 1e-10
    assert rel(pg.grad, ogp) <= 1e-10


@pytest.mark.slow
@pytest.mark.parametrize("rc", [1.0, 2.0, 3.0])
@pytest.mark.parametrize("precision", [1, 0])
def test_full_size_sphere_sampled(precision, rc):
    """The precision workload at full size (16,777,216-particle uniform sphere, 256^3 mesh,
    r_c = 1, 2 and 3 h, open boundaries) in the benchmark's launch configuration, checked against
    the oracle on the 65,536-particle subsample (full deposit and solve, short range and
    interpolation per sample)."""
    spec = dict(B.WORKLOADS["sphere16m"])
    x = B.positions(spec)
    P = O.auto_mesh(x, 256, rc_over_h=rc)
    idx = B.subsample(len(x), 65536, seed=12345)
    ref = O.forces(x, P, sample=idx)
    ctx = p3m().Context(gpu_params(P, precision), len(x))
    f = ctx.forces(cuda(x))
    ctx.sync()
    fs = f[torch.from_numpy(idx).cuda()]
    assert rel(fs, ref.F) <= TOL[precision]
    pairs, _ = ctx.pair_count()
    # about 67 neighbours per particle at r_c = 2h, scaling as r_c^3
    assert pairs > 0.8 * 1.128e9 * (rc / 2.0) ** 3
    ctx.close()


# ------------------------------------------------------------------------------------------
# the other workloads at their own sizes
# ------------------------------------------------------------------------------------------
@pytest.mark.parametrize("precision", [0, 1])
def test_workload_gauss4k_cathode_eval_and_10_steps(precision):
    """4096-particle Gaussian (sigma 1 mm, seed 0, cold, q = 1e-15 C), 16^3 mesh, TSC, r_c = 2h,
    grounded cathode one spacing below the lowest particle: one evaluation and 10 steps of
    1e-12 s against the oracle."""
    spec = dict(B.WORKLOADS["gauss4k"])
    x0 = B.positions(spec)
    h = O.auto_mesh(x0, 16).h[2]
    x = B.lift_to_plane(x0, 0.0, h)
    P = O.auto_mesh(x * np.array([1.0, 1.0, 1.0]), 16, rc_over_h=2.0, pm_bc=1, z_cathode=0.0)
    kern = O.green_kernels(P)
    ref = O.forces(x, P, kernels=kern)
    ctx = p3m().Context(gpu_params(P, precision), len(x))
    xg = cuda(x)
    f = ctx.forces(xg)
    ctx.sync()
    assert rel(f, ref.F) <= TOL[precision]
    p = np.zeros_like(x)
    xT, pT, _ = O.push(x, p, 1e-12, 10, P, force=lambda y: O.forces(y, P, kernels=kern).F)
    pg = cuda(p)
    ctx.push(xg, pg, 1e-12, 10)
    ctx.sync()
    assert rel(xg - cuda(x), xT - x) <= 10 * TOL[precision]
    assert rel(pg, pT) <= 10 * TOL[precision]


@pytest.mark.slow
@pytest.mark.parametrize("precision", [1, 0])
def test_workload_gauss1m_sampled(precision):
    """1,048,576-particle Gaussian (sigma 1, 1, 3 mm, thermal), 64^3 mesh, r_c = 2h (about 3e10
    in-cutoff pairs per evaluation): one evaluation on 1024 sampled particles."""
    spec = dict(B.WORKLOADS["gauss1m"])
    x = B.positions(spec)
    P = O.auto_mesh(x, 64, rc_over_h=2.0)
    idx = B.subsample(len(x), 1024, seed=12345)
    ref = O.forces(x, P, sample=idx)
    ctx = p3m().Context(gpu_params(P, precision), len(x))
    f = ctx.forces(cuda(x))
    ctx.sync()
    assert rel(f[torch.from_numpy(idx).cuda()], ref.F) <= TOL[precision]
    ctx.close()


@pytest.mark.slow
@pytest.mark.parametrize("precision", [1, 0])
@pytest.mark.parametrize("pp_bc", [0, 1])
def test_workload_halo4m_cathode_sampled(precision, pp_bc):
    """4,194,304 particles (95% Gaussian core sigma 1 mm + 5% shell at 4-6 sigma) lifted one
    spacing above the cathode, 128^3 mesh, r_c = 3h, cathode in the long range and (pp_bc = 1)
    in the short range: one evaluation on 1024 sampled particles plus every particle within
    r_c of the cathode."""
    spec = dict(B.WORKLOADS["halo4m"])
    x0 = B.positions(spec)
    h = O.auto_mesh(x0, 128).h[2]
    x = B.lift_to_plane(x0, 0.0, h)
    P = O.auto_mesh(x, 128, rc_over_h=3.0, pm_bc=1, pp_bc=pp_bc, z_cathode=0.0)
    near = np.nonzero(x[:, 2] < P.rc)[0]
    idx = np.union1d(B.subsample(len(x), 1024, seed=12345), near)
    ref = O.forces(x, P, sample=idx)
    ctx = p3m().Context(gpu_params(P, precision), len(x))
    f = ctx.forces(cuda(x))
    ctx.sync()
    assert rel(f[torch.from_numpy(idx).cuda()], ref.F) <= TOL[precision]
    if pp_bc:
        assert ref.image_pairs > 0
    ctx.close()


@pytest.mark.slow
def test_workload_gradient_4096_200_steps():
    """Reverse pass over 200 steps with checkpoints every 20 (4096-particle Gaussian, sigma 1, 1,
    3 mm, thermal, 64^3 mesh, r_c = 2h, dt = 2.5e-13 s) against the oracle's gradient of the final
    rms emittance, FP64."""
    spec = dict(B.WORKLOADS["gauss1m_grad"])
    x0 = B.positions(spec, 4096)
    p0 = B.momenta(spec, 4096)
    P = O.auto_mesh(x0 * 1.05, 64, rc_over_h=2.0)
    kern = O.green_kernels(P)
    dt, T = 2.5e-13, 200
    xT, pT, _ = O.push(x0, p0, dt, T, P, force=lambda y: O.forces(y, P, kernels=kern).F)
    gxT, gpT = O.emittance_grad(xT, pT, P)
    ogx, ogp = O.backward(x0, p0, dt, T, gxT, gpT, P, kern)
    ctx = p3m().Context(gpu_params(P, 0, adj_slots=10, adj_segment=20), len(x0))
    gx0, gp0 = ctx.backward(cuda(x0), cuda(p0), dt, T, cuda(gxT), cuda(gpT))
    ctx.sync()
    # measured 6e-15 (x0) and 3e-16 (p0)
    assert rel(gx0, ogx) <= 1e-10
    assert rel(gp0, ogp) <= 1e-10
