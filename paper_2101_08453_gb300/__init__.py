"""Python binding of libmcwind (mass-consistent wind downscaling on GB300).

Argument marshalling only: every step of the method runs in the CUDA
kernels of ``libmcwind.so`` behind the C boundary declared in
``include/mcwind.h``.  PyTorch supplies device memory and streams.  The
functions keep the C names; ``Plan`` bundles them for convenience.

If the library has not been built, or no CUDA device is present when a
device call is made, the call raises: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

from . import build as _build

MCWIND_OK = 0
MCWIND_EINVAL = -1
MCWIND_EGEOM = -2
MCWIND_ENONFINITE = -3
MCWIND_ENOTCONV = -4
MCWIND_ECUDA = -5
MCWIND_ESTATE = -6
MCWIND_ETIMEOUT = -7
MCWIND_ESHIFT = -8
PREC_F64, PREC_MIXED = 0, 1
RHS_GAUSS8, RHS_CENTER1 = 0, 1
RULE_PAPER, RULE_OPERATOR = 0, 1
AT_CENTERS, AT_GAUSS = 0, 1
FORWARD, BACKWARD = 0, 1
ACCEL_NONE, ACCEL_CG = 0, 1
U0_NODES, U0_CENTERS = 0, 1
ARITH_F64, ARITH_DFLOAT = 0, 1
OP_STORED, OP_SEPARABLE = 0, 1
WARM = 1
HIST = 256


class MCWindError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = code
        msg = lib().mcwind_strerror(code).decode()
        if code == MCWIND_ECUDA:
            msg += f" (cudaError {lib().mcwind_last_cuda_error()})"
        super().__init__(f"{where}: {msg} [{code}]")


class Options(ctypes.Structure):
    _fields_ = [("nu_pre", ctypes.c_int), ("nu_post", ctypes.c_int),
                ("coarsen_rule", ctypes.c_int), ("coarsest_max", ctypes.c_int),
                ("precision", ctypes.c_int), ("rhs_quad", ctypes.c_int),
                ("post_reverse", ctypes.c_int), ("accel", ctypes.c_int),
                ("use_graphs", ctypes.c_int), ("u0_at", ctypes.c_int),
                ("element_arith", ctypes.c_int), ("cycles_per_check", ctypes.c_int),
                ("op_form", ctypes.c_int)]


class Stats(ctypes.Structure):
    _fields_ = [("cycles", ctypes.c_int), ("status", ctypes.c_int),
                ("norm_f", ctypes.c_double), ("rel_res", ctypes.c_double),
                ("rate", ctypes.c_double), ("res_hist", ctypes.c_double * HIST)]

    def history(self):
        return [self.res_hist[i] for i in range(self.cycles + 1)]


_lib = None
_vp = ctypes.c_void_p
_i = ctypes.c_int
_d = ctypes.c_double


def lib():
    """Load libmcwind.so (built in-tree); raise if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(_build.LIB):
        raise ImportError(f"{_build.LIB} is not built; run __graft_entry__.build()")
    L = ctypes.CDLL(_build.LIB)
    sig = {
        "mcwind_default_options": (None, [ctypes.POINTER(Options)]),
        "mcwind_plan_create": (_i, [_i, _i, _i, ctypes.POINTER(_d), _d, ctypes.POINTER(_d),
                                    ctypes.POINTER(Options), ctypes.POINTER(_vp),
                                    ctypes.POINTER(ctypes.c_size_t)]),
        "mcwind_plan_query": (_i, [_vp, ctypes.POINTER(Options), ctypes.POINTER(ctypes.c_size_t)]),
        "mcwind_plan_num_levels": (_i, [_vp]),
        "mcwind_plan_level": (_i, [_vp, _i, ctypes.POINTER(_i), ctypes.POINTER(_i),
                                   ctypes.POINTER(_i), ctypes.POINTER(_i)]),
        "mcwind_assemble": (_i, [_vp, _vp, _vp, _vp, _vp, _vp]),
        "mcwind_solve": (_i, [_vp, _vp, _vp, _d, _i, ctypes.c_uint, ctypes.POINTER(Stats), _vp]),
        "mcwind_recover": (_i, [_vp, _vp, _vp, _vp, _i, _vp]),
        "mcwind_rhs": (_i, [_vp, _vp, _vp, _vp]),
        "mcwind_weak_div": (_i, [_vp, _vp, _vp, _vp]),
        "mcwind_level_stencil": (_i, [_vp, _i, _i, _vp, _vp]),
        "mcwind_level_residual": (_i, [_vp, _i, _i, _vp, _vp, _vp, _vp]),
        "mcwind_level_smooth": (_i, [_vp, _i, _i, _vp, _vp, _i, _i, _vp]),
        "mcwind_level_restrict": (_i, [_vp, _i, _i, _vp, _vp, _vp]),
        "mcwind_level_residual_restrict": (_i, [_vp, _i, _i, _vp, _vp, _vp, _vp]),
        "mcwind_level_prolong": (_i, [_vp, _i, _i, _vp, _vp, _vp]),
        "mcwind_coarse_solve": (_i, [_vp, _vp, _vp, _vp]),
        "mcwind_vcycle": (_i, [_vp, _i, _vp, _vp, _vp]),
        "mcwind_residual_norm_noalloc": (_i, [_vp, _vp, _vp, _vp, _vp]),
        "mcwind_solve_rhs": (_i, [_vp, _vp, _vp, _d, _i, ctypes.c_uint, ctypes.POINTER(Stats), _vp]),
        "mcwind_recover_adjoint": (_i, [_vp, _vp, _vp, _vp, _vp]),
        "mcwind_adjoint_finish": (_i, [_vp, _vp, _vp, _vp, _vp, ctypes.POINTER(_d), _vp]),
        "mcwind_batch_workspace_bytes": (ctypes.c_size_t, [_i]),
        "mcwind_batch_create": (_i, [_i, ctypes.POINTER(_vp), _vp, ctypes.POINTER(_vp)]),
        "mcwind_batch_solve": (_i, [_vp, ctypes.POINTER(_vp), ctypes.POINTER(_vp), _d, _i,
                                    ctypes.c_uint, ctypes.POINTER(Stats), _vp]),
        "mcwind_batch_destroy": (None, [_vp]),
        "mcwind_plan_set_tuning": (_i, [_vp, _i, _i, _i]),
        "mcwind_plan_wait_selftest": (_i, [_vp, _i, _vp]),
        "mcwind_launch_count": (ctypes.c_longlong, []),
        "mcwind_profile": (_i, [_vp, _i, _vp]),
        "mcwind_profile_read": (_i, [_vp, ctypes.POINTER(_d), ctypes.POINTER(ctypes.c_longlong), _i, _vp]),
        "mcwind_plan_destroy": (None, [_vp]),
        "mcwind_strerror": (ctypes.c_char_p, [_i]),
        "mcwind_last_cuda_error": (_i, []),
    }
    for name, (res, args) in sig.items():
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args
    _lib = L
    return L


def _check(rc, where, ok=(MCWIND_OK,)):
    if rc not in ok:
        raise MCWindError(rc, where)
    return rc


def _stream(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return _vp(stream.cuda_stream)


def _dev(t, name):
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != torch.float64 or not t.is_contiguous():
        raise TypeError(f"{name} must be a contiguous float64 tensor")
    return _vp(t.data_ptr())


def _need(**tensors):
    """Raise ValueError unless each tensor holds the number of values the
    call reads or writes: name=(tensor, n) needs exactly n, name=(tensor, n,
    "min") at least n.  Runs before anything is handed to the library, so a
    short buffer never reaches a kernel."""
    for name, spec in tensors.items():
        t, n = spec[0], int(spec[1])
        k = int(t.numel()) if hasattr(t, "numel") else -1
        if (k < n) if len(spec) > 2 else (k != n):
            want = f"at least {n}" if len(spec) > 2 else str(n)
            raise ValueError(f"{name} holds {k} values; the plan needs {want}")


def _dims(plan, level=0):
    """Node counts (Nx, Ny, Nz) of a level of the plan."""
    d = (_i * 3)()
    _check(lib().mcwind_plan_level(plan, int(level), d, None, None, None), "mcwind_plan_level")
    return d[0], d[1], d[2]


def _nodes(plan, level=0):
    Nx, Ny, Nz = _dims(plan, level)
    return Nx * Ny * Nz


def _cells(plan):
    Nx, Ny, Nz = _dims(plan, 0)
    return (Nx - 1) * (Ny - 1) * (Nz - 1)


def plan_options(plan):
    """The plan's options as they stand (mcwind_plan_query)."""
    o = Options()
    _check(lib().mcwind_plan_query(plan, ctypes.byref(o), None), "mcwind_plan_query")
    return o


def plan_workspace_bytes(plan):
    n = ctypes.c_size_t()
    _check(lib().mcwind_plan_query(plan, None, ctypes.byref(n)), "mcwind_plan_query")
    return n.value


def _u0_count(plan):
    return 3 * (_cells(plan) if plan_options(plan).u0_at == U0_CENTERS else _nodes(plan))


def default_options(**kw) -> Options:
    o = Options()
    lib().mcwind_default_options(ctypes.byref(o))
    for k, v in kw.items():
        setattr(o, k, int(v))
    return o


# ---- same names as the C entry points -----------------------------------

def mcwind_plan_create(nx, ny, nz, a, h1, h3, options=None):
    """Returns (plan handle, workspace bytes).  Host only."""
    a_arr = (_d * 3)(*[float(v) for v in a])
    h3l = [float(v) for v in h3]
    h3_arr = (_d * max(1, len(h3l)))(*h3l)
    o = options if options is not None else default_options()
    handle = _vp()
    ws = ctypes.c_size_t()
    _check(lib().mcwind_plan_create(int(nx), int(ny), int(nz), a_arr, float(h1), h3_arr,
                                    ctypes.byref(o), ctypes.byref(handle), ctypes.byref(ws)),
           "mcwind_plan_create")
    return handle, ws.value


def mcwind_plan_num_levels(plan):
    return _check(lib().mcwind_plan_num_levels(plan), "mcwind_plan_num_levels",
                  ok=range(0, 1 << 30))


def mcwind_plan_level(plan, level):
    dims = (_i * 3)()
    hx, hy = _i(), _i()
    kmap = (_i * 256)()
    _check(lib().mcwind_plan_level(plan, level, dims, ctypes.byref(hx), ctypes.byref(hy), kmap),
           "mcwind_plan_level")
    nlev = mcwind_plan_num_levels(plan)
    out = dict(Nx=dims[0], Ny=dims[1], Nz=dims[2])
    if level + 1 < nlev:
        nzc = (_i * 3)()
        lib().mcwind_plan_level(plan, level + 1, nzc, None, None, None)
        out.update(hx=bool(hx.value), hy=bool(hy.value), kmap=[kmap[q] for q in range(nzc[2])])
    return out


def mcwind_plan_destroy(plan):
    lib().mcwind_plan_destroy(plan)


def mcwind_assemble(plan, workspace, X, Y, Z, stream=None):
    n = _nodes(plan)
    _need(X=(X, n), Y=(Y, n), Z=(Z, n))
    if int(workspace.numel()) * workspace.element_size() < plan_workspace_bytes(plan):
        raise ValueError("workspace is smaller than mcwind_plan_create reported")
    return _check(lib().mcwind_assemble(plan, _vp(workspace.data_ptr()), _dev(X, "X"), _dev(Y, "Y"),
                                        _dev(Z, "Z"), _stream(stream)), "mcwind_assemble")


def mcwind_solve(plan, u0, lam, rtol=1e-8, max_cycles=100, flags=0, stream=None, raise_notconv=False):
    _need(u0=(u0, _u0_count(plan)), lam=(lam, _nodes(plan)))
    st = Stats()
    ok = (MCWIND_OK,) if raise_notconv else (MCWIND_OK, MCWIND_ENOTCONV)
    rc = _check(lib().mcwind_solve(plan, _dev(u0, "u0"), _dev(lam, "lambda"), float(rtol),
                                   int(max_cycles), int(flags), ctypes.byref(st), _stream(stream)),
                "mcwind_solve", ok=ok)
    return rc, st


def mcwind_solve_rhs(plan, f, x, rtol=1e-8, max_cycles=100, flags=0, stream=None):
    n = _nodes(plan)
    _need(f=(f, n), x=(x, n))
    st = Stats()
    rc = _check(lib().mcwind_solve_rhs(plan, _dev(f, "f"), _dev(x, "x"), float(rtol), int(max_cycles),
                                       int(flags), ctypes.byref(st), _stream(stream)),
                "mcwind_solve_rhs", ok=(MCWIND_OK, MCWIND_ENOTCONV))
    return rc, st


def mcwind_recover_adjoint(plan, gu, h, du0, stream=None):
    n = _nodes(plan)
    _need(gu=(gu, 3 * _cells(plan)), h=(h, n), du0=(du0, 3 * n))
    return _check(lib().mcwind_recover_adjoint(plan, _dev(gu, "gu"), _dev(h, "h"), _dev(du0, "du0"),
                                               _stream(stream)), "mcwind_recover_adjoint")


def mcwind_adjoint_finish(plan, mu, lam, gu, du0, stream=None):
    """Returns dl/dlog a as a list of 3 floats (du0 updated in place)."""
    n = _nodes(plan)
    _need(mu=(mu, n), lam=(lam, n), gu=(gu, 3 * _cells(plan)), du0=(du0, 3 * n))
    out = (_d * 3)()
    _check(lib().mcwind_adjoint_finish(plan, _dev(mu, "mu"), _dev(lam, "lambda"), _dev(gu, "gu"),
                                       _dev(du0, "du0"), out, _stream(stream)), "mcwind_adjoint_finish")
    return [out[0], out[1], out[2]]


def mcwind_recover(plan, u0, lam, u, where=AT_CENTERS, stream=None):
    _need(u0=(u0, _u0_count(plan)), lam=(lam, _nodes(plan)),
          u=(u, (3 if where == AT_CENTERS else 24) * _cells(plan)))
    return _check(lib().mcwind_recover(plan, _dev(u0, "u0"), _dev(lam, "lambda"), _dev(u, "u"),
                                       int(where), _stream(stream)), "mcwind_recover")


def mcwind_rhs(plan, u0, f, stream=None):
    _need(u0=(u0, _u0_count(plan)), f=(f, _nodes(plan)))
    return _check(lib().mcwind_rhs(plan, _dev(u0, "u0"), _dev(f, "f"), _stream(stream)), "mcwind_rhs")


def mcwind_weak_div(plan, ug, out, stream=None):
    _need(ug=(ug, 24 * _cells(plan)), out=(out, _nodes(plan)))
    return _check(lib().mcwind_weak_div(plan, _dev(ug, "ug"), _dev(out, "out"), _stream(stream)),
                  "mcwind_weak_div")


def mcwind_level_stencil(plan, level, precision, out, stream=None):
    _need(out=(out, 27 * _nodes(plan, level)))
    return _check(lib().mcwind_level_stencil(plan, level, precision, _dev(out, "out"), _stream(stream)),
                  "mcwind_level_stencil")


def mcwind_level_residual(plan, level, precision, x, f, r, stream=None):
    n = _nodes(plan, level)
    _need(x=(x, n), f=(f, n), r=(r, n))
    return _check(lib().mcwind_level_residual(plan, level, precision, _dev(x, "x"), _dev(f, "f"),
                                              _dev(r, "r"), _stream(stream)), "mcwind_level_residual")


def mcwind_level_smooth(plan, level, precision, x, f, sweeps, direction, stream=None):
    n = _nodes(plan, level)
    _need(x=(x, n), f=(f, n))
    return _check(lib().mcwind_level_smooth(plan, level, precision, _dev(x, "x"), _dev(f, "f"),
                                            int(sweeps), int(direction), _stream(stream)),
                  "mcwind_level_smooth")


def mcwind_level_restrict(plan, level, precision, r, fc, stream=None):
    _need(r=(r, _nodes(plan, level)), fc=(fc, _nodes(plan, level + 1)))
    return _check(lib().mcwind_level_restrict(plan, level, precision, _dev(r, "r"), _dev(fc, "fc"),
                                              _stream(stream)), "mcwind_level_restrict")


def mcwind_level_residual_restrict(plan, level, precision, x, f, fc, stream=None):
    n = _nodes(plan, level)
    _need(x=(x, n), f=(f, n), fc=(fc, _nodes(plan, level + 1)))
    return _check(lib().mcwind_level_residual_restrict(plan, level, precision, _dev(x, "x"),
                                                       _dev(f, "f"), _dev(fc, "fc"),
                                                       _stream(stream)),
                  "mcwind_level_residual_restrict")


def mcwind_level_prolong(plan, level, precision, ec, x, stream=None):
    _need(ec=(ec, _nodes(plan, level + 1)), x=(x, _nodes(plan, level)))
    return _check(lib().mcwind_level_prolong(plan, level, precision, _dev(ec, "ec"), _dev(x, "x"),
                                             _stream(stream)), "mcwind_level_prolong")


def mcwind_coarse_solve(plan, f, x, stream=None):
    n = _nodes(plan, mcwind_plan_num_levels(plan) - 1)
    _need(f=(f, n), x=(x, n))
    return _check(lib().mcwind_coarse_solve(plan, _dev(f, "f"), _dev(x, "x"), _stream(stream)),
                  "mcwind_coarse_solve")


def mcwind_vcycle(plan, precision, x, f, stream=None):
    n = _nodes(plan)
    _need(x=(x, n), f=(f, n))
    return _check(lib().mcwind_vcycle(plan, precision, _dev(x, "x"), _dev(f, "f"), _stream(stream)),
                  "mcwind_vcycle")


def mcwind_residual_norm_noalloc(plan, f, lam, norms, stream=None):
    """(||f_F||, ||f_F - K_FF lambda_F||) into the device tensor norms[2],
    allocating nothing: for callers that cannot call cudaMalloc when they
    check a solution (a host model whose own pool owns all device memory, or
    a loop in which an allocation, which may synchronize the device, is not
    allowed).  Its scratch is a static device array inside the library,
    shared by all calls: calls that overlap on the GPU race.  The first call
    on a device must come before any stream capture."""
    n = _nodes(plan)
    _need(f=(f, n), lam=(lam, n), norms=(norms, 2, "min"))
    return _check(lib().mcwind_residual_norm_noalloc(plan, _dev(f, "f"), _dev(lam, "lambda"),
                                                     _dev(norms, "norms"), _stream(stream)),
                  "mcwind_residual_norm_noalloc")


def mcwind_plan_wait_selftest(plan, limit_us, stream=None):
    """Returns the code: MCWIND_ETIMEOUT when the bounded wait ran out (it
    always does: nothing completes the barrier)."""
    return lib().mcwind_plan_wait_selftest(plan, int(limit_us), _stream(stream))


def mcwind_plan_set_tuning(plan, nu_pre, nu_post, gs_block_rows):
    return _check(lib().mcwind_plan_set_tuning(plan, int(nu_pre), int(nu_post), int(gs_block_rows)),
                  "mcwind_plan_set_tuning")


class Batch:
    """Independent domains (assembled Plans) solved together: each iteration of
    all domains is one CUDA graph with a branch per domain."""

    def __init__(self, plans):
        import torch
        self.plans = list(plans)
        n = len(self.plans)
        nbytes = lib().mcwind_batch_workspace_bytes(n)
        self._ws = torch.empty(nbytes + 256, dtype=torch.uint8, device="cuda")
        off = (-self._ws.data_ptr()) % 256
        arr = (_vp * n)(*[p.handle for p in self.plans])
        self.handle = _vp()
        _check(lib().mcwind_batch_create(n, arr, _vp(self._ws.data_ptr() + off),
                                         ctypes.byref(self.handle)), "mcwind_batch_create")

    def __del__(self):
        h = getattr(self, "handle", None)
        if h is not None and _lib is not None:
            _lib.mcwind_batch_destroy(h)
            self.handle = None

    def solve(self, u0s, lams=None, rtol=1e-8, max_cycles=100, warm=False, stream=None):
        import torch
        n = len(self.plans)
        if lams is None:
            lams = [torch.zeros(p.node_shape, dtype=torch.float64, device="cuda") for p in self.plans]
        if len(u0s) != n or len(lams) != n:
            raise ValueError(f"a batch of {n} domains needs {n} winds and {n} lambdas")
        for p, u, l in zip(self.plans, u0s, lams):
            _need(u0=(u, _u0_count(p.handle)), lam=(l, _nodes(p.handle)))
        u_arr = (_vp * n)(*[_dev(u, "u0").value for u in u0s])
        l_arr = (_vp * n)(*[_dev(l, "lambda").value for l in lams])
        stats = (Stats * n)()
        rc = lib().mcwind_batch_solve(self.handle, u_arr, l_arr, float(rtol), int(max_cycles),
                                      WARM if warm else 0, stats, _stream(stream))
        _check(rc, "mcwind_batch_solve", ok=(MCWIND_OK, MCWIND_ENOTCONV))
        return lams, list(stats)


class Plan:
    """One grid: a plan, its torch-allocated workspace and the geometry.

    X, Y, Z: float64 CUDA tensors [nz+1][ny+1][nx+1] (kept referenced).
    """

    def __init__(self, nx, ny, nz, a, h1, h3, **options):
        import torch
        self.nx, self.ny, self.nz = int(nx), int(ny), int(nz)
        self.a = tuple(float(v) for v in a)
        self.options = default_options(**options)
        self.handle, self.workspace_bytes = mcwind_plan_create(nx, ny, nz, a, h1, h3, self.options)
        self.workspace = None
        self.geometry = None
        self.torch = torch

    @classmethod
    def for_case(cls, case, **options):
        return cls(case.nx, case.ny, case.nz, case.a, case.h1, case.h3, **options)

    def __del__(self):
        h = getattr(self, "handle", None)
        if h is not None and _lib is not None:
            _lib.mcwind_plan_destroy(h)
            self.handle = None

    @property
    def num_levels(self):
        return mcwind_plan_num_levels(self.handle)

    def level(self, l):
        return mcwind_plan_level(self.handle, l)

    @property
    def node_shape(self):
        return (self.nz + 1, self.ny + 1, self.nx + 1)

    def assemble(self, X, Y, Z, stream=None):
        torch = self.torch
        if self.workspace is None:
            self.workspace = torch.empty(self.workspace_bytes + 256, dtype=torch.uint8, device="cuda")
        off = (-self.workspace.data_ptr()) % 256
        ws = self.workspace[off:]
        self.geometry = (X, Y, Z)
        mcwind_assemble(self.handle, ws, X, Y, Z, stream)

    def solve(self, u0, lam=None, rtol=1e-8, max_cycles=100, warm=False, stream=None):
        torch = self.torch
        if lam is None:
            lam = torch.zeros(self.node_shape, dtype=torch.float64, device="cuda")
        rc, st = mcwind_solve(self.handle, u0, lam, rtol, max_cycles, WARM if warm else 0, stream)
        return lam, st

    def recover(self, u0, lam, where=AT_CENTERS, stream=None):
        torch = self.torch
        shape = (3, self.nz, self.ny, self.nx) if where == AT_CENTERS else (3, 8, self.nz, self.ny, self.nx)
        u = torch.empty(shape, dtype=torch.float64, device="cuda")
        mcwind_recover(self.handle, u0, lam, u, where, stream)
        return u

    def rhs(self, u0, stream=None):
        f = self.torch.empty(self.node_shape, dtype=self.torch.float64, device="cuda")
        mcwind_rhs(self.handle, u0, f, stream)
        return f
