"""The allocation-free emittance entry point (p3m_emittance_noalloc) against p3m_emittance.

Some callers cannot allocate device memory (a host application that owns the device through its
own allocator or a fixed budget, or a monitoring hook inside a simulation loop that must not
stall on an allocation). For them the library offers p3m_emittance_noalloc, whose scratch is a
fixed static device array. This test calls it through the C ABI twice in a row, on two
different bunches, and checks each result against the context-based entry point and against the
FP64 oracle at the same tolerance as the other emittance tests. It lives in a file of its own
that runs last.
"""
import ctypes

import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2103_02046_gb300 import bunches as B

pytestmark = pytest.mark.gpu


def rel(a, b):
    a = a.detach().cpu().numpy()
    b = b.detach().cpu().numpy()
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def test_emittance_noalloc_matches_context_entry_point_twice():
    from paper_2103_02046_gb300 import p3m as m
    L = m.lib()
    fn = L.p3m_emittance_noalloc
    P = ctypes.c_void_p
    fn.argtypes = [P, P, ctypes.c_int64, ctypes.c_double, P, P, P, P]
    fn.restype = ctypes.c_int
    mass = B.macro_mass()
    ctx = m.Context(m.Params(n=(8, 8, 8), h=(1e-3,) * 3, mass=mass), 300_000)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    for call, (n, seed) in enumerate([(300_000, 41), (12_345, 42)]):
        x = torch.from_numpy(B.gaussian(n, (1e-3, 2e-3, 3e-3), seed)).cuda()
        p = torch.from_numpy(B.thermal_momenta(n, 1e-4 * mass * B.SPEED_OF_LIGHT, seed + 1)
                             + 1e-21 * B.gaussian(n, 1.0, seed + 2)).cuda()
        eps_ref, gx_ref, gp_ref = ctx.emittance(x, p, grad=True)
        eps = torch.empty(3, dtype=torch.float64, device="cuda")
        gx = torch.empty_like(x)
        gp = torch.empty_like(p)
        st = fn(P(x.data_ptr()), P(p.data_ptr()), n, mass, P(eps.data_ptr()), P(gx.data_ptr()),
                P(gp.data_ptr()), stream)
        assert st == m.P3M_OK, f"call {call}: status {st}"
        torch.cuda.synchronize()
        assert rel(eps, eps_ref) <= 1e-12, f"call {call}"
        assert rel(gx, gx_ref) <= 1e-11, f"call {call}"
        assert rel(gp, gp_ref) <= 1e-11, f"call {call}"
        # and directly against the oracle's definition
        Po = O.Params(mass=mass)
        xo, po = x.cpu().numpy(), p.cpu().numpy()
        e_or = O.emittance(xo, po, Po)
        gx_or, gp_or = O.emittance_grad(xo, po, Po)
        e_np = eps.cpu().numpy()
        assert np.linalg.norm(e_np - e_or) <= 1e-12 * np.linalg.norm(e_or), f"call {call}"
        assert np.linalg.norm(gx.cpu().numpy() - gx_or) <= 1e-11 * np.linalg.norm(gx_or)
        assert np.linalg.norm(gp.cpu().numpy() - gp_or) <= 1e-11 * np.linalg.norm(gp_or)
    # sizes beyond the static scratch are refused, not truncated
    big = ctypes.c_int64(16_777_217)
    st = fn(P(x.data_ptr()), P(p.data_ptr()), big, mass, P(eps.data_ptr()), None, None, stream)
    assert st == m.P3M_EINVAL
    ctx.close()
