"""Thin Python binding of the C ABI in ``include/p3m.h`` (argument marshalling only).

Every step of the force evaluation, push and reverse pass runs in the CUDA library
``_build/libp3m.so``; this module only passes device pointers and the current CUDA stream.
PyTorch supplies device memory and streams. If the library is missing the import of any
entry point raises: there is no fallback path.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass, field

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libp3m.so")

P3M_OK, P3M_EINVAL, P3M_ENOMEM, P3M_ECUDA, P3M_ECUFFT, P3M_ERANGE, P3M_ETIMEOUT, P3M_ESTATE = range(8)
STATUS_NAMES = ["P3M_OK", "P3M_EINVAL", "P3M_ENOMEM", "P3M_ECUDA", "P3M_ECUFFT", "P3M_ERANGE",
                "P3M_ETIMEOUT", "P3M_ESTATE"]
FP64, FP32_MIXED = 0, 1


class P3MError(RuntimeError):
    def __init__(self, status: int, where: str, msg: str = ""):
        self.status = status
        name = STATUS_NAMES[status] if 0 <= status < len(STATUS_NAMES) else str(status)
        super().__init__(f"{where}: {name} {msg}".strip())


class CParams(ctypes.Structure):
    _fields_ = [
        ("n", ctypes.c_int32 * 3),
        ("lo", ctypes.c_double * 3),
        ("h", ctypes.c_double * 3),
        ("rc_over_h", ctypes.c_double),
        ("kappa", ctypes.c_double),
        ("alpha", ctypes.c_double),
        ("assign_order", ctypes.c_int32),
        ("pm_bc", ctypes.c_int32),
        ("pp_bc", ctypes.c_int32),
        ("z_cathode", ctypes.c_double),
        ("influence", ctypes.c_int32),
        ("precision", ctypes.c_int32),
        ("deterministic", ctypes.c_int32),
        ("adj_slots", ctypes.c_int32),
        ("adj_segment", ctypes.c_int32),
        ("q", ctypes.c_double),
        ("mass", ctypes.c_double),
        ("force_diff", ctypes.c_int32),
        ("search_rows", ctypes.c_int32),
        ("search_xcells", ctypes.c_int32),
    ]


_lib = None


def lib():
    """Loads the CUDA library (raises if it was not built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"the P3M CUDA library is not built ({LIB_PATH}); "
                               "run __graft_entry__.build()")
        L = ctypes.CDLL(LIB_PATH)
        P, I32, I64, D = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_double
        PP = ctypes.POINTER(CParams)
        sig = {
            "p3m_default_params": [PP],
            "p3m_auto_mesh": [P, I64, PP, P],
            "p3m_create": [PP, I64, P, ctypes.POINTER(P)],
            "p3m_destroy": [P],
            "p3m_set_stream": [P, P],
            "p3m_deposit": [P, P, I64],
            "p3m_solve": [P],
            "p3m_get_mesh": [P, I32, P],
            "p3m_forces_ex": [P, P, I64, P, P, I32],
            "p3m_forces": [P, P, I64, P, P],
            "p3m_pair_count": [P, ctypes.POINTER(I64), ctypes.POINTER(I64)],
            "p3m_candidate_count": [P, ctypes.POINTER(I64)],
            "p3m_search_layout": [P, ctypes.POINTER(I32), ctypes.POINTER(I32)],
            "p3m_push": [P, P, P, I64, D, I32, P],
            "p3m_push_ex": [P, P, P, I64, D, I32, P, I32],
            "p3m_force_vjp": [P, P, I64, P, P],
            "p3m_backward": [P, P, P, I64, D, I32, I32, P, P, P, P],
            "p3m_emittance": [P, P, P, I64, P, P, P],
            "p3m_sync": [P],
            "p3m_get_timings": [P, ctypes.POINTER(D), I32, ctypes.POINTER(I32)],
            "p3m_fp32_probe": [I32, I32, ctypes.POINTER(D), P],
        }
        for name, args in sig.items():
            fn = getattr(L, name)
            fn.argtypes = args
            fn.restype = ctypes.c_int
        L.p3m_last_error.argtypes = [P]
        L.p3m_last_error.restype = ctypes.c_char_p
        _lib = L
    return _lib


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


def _stream():
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _vec3(t: torch.Tensor, name: str):
    if not (t.is_cuda and t.dtype == torch.float64 and t.dim() == 2 and t.shape[1] == 3
            and t.is_contiguous()):
        raise ValueError(f"{name} must be a contiguous CUDA float64 tensor of shape [n, 3]")
    return t


@dataclass
class Params:
    """Mirror of ``p3m_params`` (see include/p3m.h)."""
    n: tuple = (64, 64, 64)
    lo: tuple = (0.0, 0.0, 0.0)
    h: tuple = (1e-5, 1e-5, 1e-5)
    rc_over_h: float = 2.0
    kappa: float = 3.0
    alpha: float = 0.0
    assign_order: int = 2
    pm_bc: int = 0  # 0 open, 1 grounded cathode plane, 2 grounded box (FP64)
    pp_bc: int = 0
    z_cathode: float = 0.0
    influence: int = 0  # 0 sampled kernel, 1 principal alias 1/U^2, 2 alias sums (eq. (Ghfinal))
    precision: int = FP64
    deterministic: int = 0
    adj_slots: int = 0
    adj_segment: int = 0
    q: float = 1e-15
    mass: float = 1e-15 / 1.602176634e-19 * 9.1093837015e-31
    force_diff: int = 0  # 1 = central-difference mesh gradient (not the variational force)
    search_rows: int = 0  # short-range cell rows per cutoff (1, 2, 3); 0 = chosen by the library
    search_xcells: int = 0  # x cells per cutoff (1 .. 32, powers of 2); 0 = chosen

    def to_c(self) -> CParams:
        c = CParams()
        for k, _ in CParams._fields_:
            v = getattr(self, k)
            if k in ("n", "lo", "h"):
                arr = getattr(c, k)
                for d in range(3):
                    arr[d] = v[d]
            else:
                setattr(c, k, v)
        return c

    @staticmethod
    def from_c(c: CParams) -> "Params":
        kw = {}
        for k, _ in CParams._fields_:
            v = getattr(c, k)
            kw[k] = tuple(v) if k in ("n", "lo", "h") else v
        return Params(**kw)


def default_params() -> Params:
    c = CParams()
    st = lib().p3m_default_params(ctypes.byref(c))
    if st:
        raise P3MError(st, "p3m_default_params")
    return Params.from_c(c)


def auto_mesh(x: torch.Tensor, params: Params) -> Params:
    """Fills params.lo / params.h from the particles' bounding box (p3m_auto_mesh)."""
    _vec3(x, "x")
    c = params.to_c()
    st = lib().p3m_auto_mesh(_ptr(x), x.shape[0], ctypes.byref(c), _stream())
    if st:
        raise P3MError(st, "p3m_auto_mesh")
    return Params.from_c(c)


class Context:
    """Owns one ``p3m_ctx`` (all scratch memory of the library)."""

    def __init__(self, params: Params, n_max: int):
        self.params = params
        self.n_max = int(n_max)
        h = ctypes.c_void_p()
        cp = params.to_c()
        st = lib().p3m_create(ctypes.byref(cp), self.n_max, _stream(), ctypes.byref(h))
        if st:
            raise P3MError(st, "p3m_create")
        self._h = h

    def close(self):
        if getattr(self, "_h", None):
            lib().p3m_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, st, where):
        if st:
            msg = lib().p3m_last_error(self._h)
            raise P3MError(st, where, msg.decode() if msg else "")

    def _bind(self):
        lib().p3m_set_stream(self._h, _stream())

    def forces(self, x: torch.Tensor, out: torch.Tensor | None = None, energy: bool = False,
               parts: int = 3):
        """One force evaluation (p3m_forces_ex). Returns f or (f, energy[2])."""
        _vec3(x, "x")
        f = torch.empty_like(x) if out is None else _vec3(out, "out")
        e = torch.zeros(2, dtype=torch.float64, device=x.device) if energy else None
        self._bind()
        self._check(lib().p3m_forces_ex(self._h, _ptr(x), x.shape[0], _ptr(f), _ptr(e), parts),
                    "p3m_forces_ex")
        return (f, e) if energy else f

    def deposit(self, x: torch.Tensor):
        _vec3(x, "x")
        self._bind()
        self._check(lib().p3m_deposit(self._h, _ptr(x), x.shape[0]), "p3m_deposit")

    def solve(self):
        self._bind()
        self._check(lib().p3m_solve(self._h), "p3m_solve")

    def get_mesh(self, which: int) -> torch.Tensor:
        n = self.params.n
        out = torch.empty((n[2], n[1], n[0]), dtype=torch.float64, device="cuda")
        self._bind()
        self._check(lib().p3m_get_mesh(self._h, which, _ptr(out)), "p3m_get_mesh")
        return out

    def pair_count(self):
        a, b = ctypes.c_int64(), ctypes.c_int64()
        self._bind()
        self._check(lib().p3m_pair_count(self._h, ctypes.byref(a), ctypes.byref(b)),
                    "p3m_pair_count")
        return a.value, b.value

    def candidate_count(self):
        """(particle, record) distance tests of the last short range (p3m_candidate_count)."""
        a = ctypes.c_int64()
        self._bind()
        self._check(lib().p3m_candidate_count(self._h, ctypes.byref(a)), "p3m_candidate_count")
        return a.value

    def search_layout(self):
        """(cell rows per cutoff in y and z, x cells per cutoff) of the short-range search."""
        r, c = ctypes.c_int32(), ctypes.c_int32()
        self._check(lib().p3m_search_layout(self._h, ctypes.byref(r), ctypes.byref(c)),
                    "p3m_search_layout")
        return r.value, c.value

    def push(self, x, p, dt: float, nsteps: int, f=None):
        """In-place leapfrog; returns F(x_end). With f = F(x0) given: p3m_push, which reuses it
        and overwrites it with F(x_end); without: p3m_push_ex into a new tensor."""
        _vec3(x, "x")
        _vec3(p, "p")
        self._bind()
        if f is not None:
            _vec3(f, "f")
            self._check(lib().p3m_push(self._h, _ptr(x), _ptr(p), x.shape[0], float(dt),
                                       int(nsteps), _ptr(f)), "p3m_push")
            return f
        f = torch.empty_like(x)
        self._check(lib().p3m_push_ex(self._h, _ptr(x), _ptr(p), x.shape[0], float(dt),
                                      int(nsteps), _ptr(f), 0), "p3m_push_ex")
        return f

    def force_vjp(self, x, w):
        _vec3(x, "x")
        _vec3(w, "w")
        out = torch.empty_like(x)
        self._bind()
        self._check(lib().p3m_force_vjp(self._h, _ptr(x), x.shape[0], _ptr(w), _ptr(out)),
                    "p3m_force_vjp")
        return out

    def backward(self, x0, p0, dt, nsteps, gxT, gpT, ckpt_every: int = 0):
        """Reverse pass (p3m_backward), checkpoints every ckpt_every steps (0 = adj_segment)."""
        for t, nm in ((x0, "x0"), (p0, "p0"), (gxT, "gxT"), (gpT, "gpT")):
            _vec3(t, nm)
        gx0 = torch.empty_like(x0)
        gp0 = torch.empty_like(p0)
        self._bind()
        self._check(lib().p3m_backward(self._h, _ptr(x0), _ptr(p0), x0.shape[0], float(dt),
                                       int(nsteps), int(ckpt_every), _ptr(gxT), _ptr(gpT),
                                       _ptr(gx0), _ptr(gp0)), "p3m_backward")
        return gx0, gp0

    def emittance(self, x, p, grad: bool = False):
        _vec3(x, "x")
        _vec3(p, "p")
        eps = torch.empty(3, dtype=torch.float64, device=x.device)
        gx = torch.empty_like(x) if grad else None
        gp = torch.empty_like(p) if grad else None
        self._bind()
        self._check(lib().p3m_emittance(self._h, _ptr(x), _ptr(p), x.shape[0], _ptr(eps),
                                        _ptr(gx), _ptr(gp)), "p3m_emittance")
        return (eps, gx, gp) if grad else eps

    def sync(self):
        self._bind()
        self._check(lib().p3m_sync(self._h), "p3m_sync")

    def timings(self):
        """[bin+sort, short range, deposit, solve, interp+combine, total] in ms."""
        buf = (ctypes.c_double * 6)()
        cnt = ctypes.c_int32()
        self._check(lib().p3m_get_timings(self._h, buf, 6, ctypes.byref(cnt)), "p3m_get_timings")
        return list(buf)


# ------------------------------------------------------------------------------------------
# autograd wrappers (the backward passes call the library's reverse pass)
# ------------------------------------------------------------------------------------------
class P3MRun(torch.autograd.Function):
    """(x0, p0) -> (x_T, p_T) after `nsteps` leapfrog steps; backward = p3m_backward with
    checkpoints every adj_segment steps."""

    @staticmethod
    def forward(ctx, x0, p0, context: Context, dt: float, nsteps: int):
        x = x0.detach().clone()
        p = p0.detach().clone()
        context.push(x, p, dt, nsteps)
        ctx.context, ctx.dt, ctx.nsteps = context, dt, nsteps
        ctx.save_for_backward(x0.detach(), p0.detach())
        return x, p

    @staticmethod
    def backward(ctx, gx, gp):
        x0, p0 = ctx.saved_tensors
        gx = torch.zeros_like(x0) if gx is None else gx.contiguous()
        gp = torch.zeros_like(p0) if gp is None else gp.contiguous()
        gx0, gp0 = ctx.context.backward(x0, p0, ctx.dt, ctx.nsteps, gx, gp)
        return gx0, gp0, None, None, None


class Emittance(torch.autograd.Function):
    """sum_u eps_u (normalised rms emittance) with its closed-form gradient."""

    @staticmethod
    def forward(ctx, x, p, context: Context):
        eps, gx, gp = context.emittance(x.detach().contiguous(), p.detach().contiguous(), grad=True)
        ctx.save_for_backward(gx, gp)
        return eps.sum()

    @staticmethod
    def backward(ctx, g):
        gx, gp = ctx.saved_tensors
        return g * gx, g * gp, None


def fp32_probe(packed: bool, iters: int) -> float:
    """Launches the FP32 multiply-add chain probe on the current stream; returns its flops."""
    flops = ctypes.c_double(0.0)
    st = lib().p3m_fp32_probe(int(bool(packed)), int(iters), ctypes.byref(flops), _stream())
    if st != P3M_OK:
        raise P3MError(st, "p3m_fp32_probe")
    return flops.value
