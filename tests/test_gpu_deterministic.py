"""The deterministic mode (deterministic = 1, FP64 path): identical inputs give bitwise identical
forces, energies, trajectories, adjoints and emittances, still at the FP64 parity bound; and the
reverse pass agrees with central finite differences coordinate by coordinate (the check the
mode exists for: the differences of J carry no summation noise).

Reading for the gradient objective: J = eps_x + eps_y + eps_z, the normalised rms emittances
(the paper names no objective)."""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2103_02046_gb300 import bunches as B

pytestmark = pytest.mark.gpu


def p3m():
    from paper_2103_02046_gb300 import p3m as m
    return m


def cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


def test_deterministic_results_are_bitwise_reproducible():
    m = p3m()
    x = B.lift_to_plane(B.gaussian(4096, (1e-3, 1e-3, 1e-3), 0), 0.0, 0.15e-3)
    P = O.auto_mesh(x, 16, rc_over_h=2.0, pm_bc=1, pp_bc=1, z_cathode=0.0)
    prm = m.Params(n=P.n, lo=P.lo, h=P.h, rc_over_h=2.0, pm_bc=1, pp_bc=1, z_cathode=0.0,
                   precision=m.FP64, deterministic=1, adj_slots=2, adj_segment=3)
    ctx = m.Context(prm, len(x))
    xg = cuda(x)
    runs, counts = [], []
    for _ in range(2):
        f, e = ctx.forces(xg, energy=True)
        counts.append(ctx.pair_count())
        w = cuda(B.gaussian(len(x), 1.0, 9))
        v = ctx.force_vjp(xg, w)
        xx, pp = xg.clone(), torch.zeros_like(xg)
        ctx.push(xx, pp, 1e-12, 5)
        eps, gx, gp = ctx.emittance(xx, pp + 1e-24 * w, grad=True)
        bx, bp = ctx.backward(xg, torch.zeros_like(xg), 1e-12, 5, gx, gp)
        ctx.sync()
        runs.append([t.clone() for t in (f, e, v, xx, pp, eps, bx, bp)])
    for a, b in zip(*runs):
        assert torch.equal(a, b)
    ref = O.forces(x, P)
    assert O.rel_l2(runs[0][0].cpu().numpy(), ref.F) <= 1e-12
    e = runs[0][1].cpu().numpy()
    assert e[0] == pytest.approx(ref.U_pp, rel=1e-12)
    assert e[1] == pytest.approx(ref.U_pm, rel=1e-12)
    # the pair counts of the evaluation above (every ordered pair found from its own side)
    assert counts[0] == counts[1] == (ref.pairs, ref.image_pairs)
    ctx.close()


@pytest.mark.slow
def test_fd_gradient_per_coordinate_deterministic():
    """Central finite differences (step 1e-6 of each component's rms spread) on 16 random single
    coordinates of a 16,384-particle Gaussian (sigma 1, 1, 3 mm, thermal momenta; the gradient
    workload at reduced size), 200 leapfrog steps of 2.5e-13 s with checkpoints every 20,
    deterministic FP64, against the reverse pass."""
    from paper_2103_02046_gb300 import experiments as X
    out = X.gradient_coords(precision=p3m().FP64, n_particles=16_384, coords=16,
                            deterministic=1, compare_fp32=False)
    fd, ad = np.array(out["fd"]), np.array(out["adjoint"])
    rel = np.abs(fd - ad) / np.abs(fd)
    assert np.median(rel) <= 1e-4
    assert np.linalg.norm(fd - ad) / np.linalg.norm(fd) <= 1e-4
