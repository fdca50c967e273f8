"""Thin ctypes binding of libtg.so (include/tg.h): argument marshalling only.

Every numerical step runs in the library's CUDA kernels.  Tensors are torch tensors on
the current CUDA device (float64 / complex128 unless stated); their raw device pointers
and the current CUDA stream are passed straight through.  The library must be built
(``python -m paper_2005_03070_gb300.build``); loading fails loudly when it is missing.

Function names match the C entry points; the ``Operator`` and ``Deflation`` classes own
the opaque handles and free them on deletion.
"""
from __future__ import annotations

import ctypes as C
import os

import torch

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libtg.so")

TG_OK, TG_NOT_CONVERGED, TG_BREAKDOWN, TG_NAN, TG_BAD_ARG, TG_OOM, TG_CUDA_ERROR, TG_SYNC_TIMEOUT = range(8)
TG_CD2D, TG_CD3D, TG_U1_4D, TG_VARK2D, TG_EXP2D = 0, 1, 2, 3, 4
TG_BICGSTAB, TG_GMRES = 0, 1
TG_PROJ_MINRES, TG_PROJ_GALERKIN = 0, 1
TG_F64, TG_F32_IR = 0, 1
TG_FINE, TG_COARSE = 0, 1

KIND = {"cd2d": TG_CD2D, "cd3d": TG_CD3D, "u1_4d": TG_U1_4D, "vark2d": TG_VARK2D, "exp2d": TG_EXP2D}
METHOD = {"bicgstab": TG_BICGSTAB, "gmres": TG_GMRES}
PROJ = {"minres": TG_PROJ_MINRES, "galerkin": TG_PROJ_GALERKIN}
PREC = {"f64": TG_F64, "f32_ir": TG_F32_IR}
INTERP = {"linear": 0, "cubic": 1}

EXPORTS = [
    "tg_status_string", "tg_last_error", "tg_setup_operator", "tg_destroy_op", "tg_op_size", "tg_apply",
    "tg_prolong", "tg_restrict", "tg_op_set_interp", "tg_coarse_gmresdr", "tg_defl_from_basis", "tg_destroy_defl",
    "tg_defl_copy", "tg_project", "tg_solve_proj", "tg_solve_idr", "tg_improve_defl", "tg_adjoint_solve",
    "tg_kappa_gradient",
    "tg_harmonic_ritz", "tg_harmonic_ritz_noalloc", "tg_profile_enable", "tg_profile_read", "tg_launch_count",
    "tg_batch_create", "tg_batch_layout", "tg_batch_setup", "tg_batch_solve", "tg_destroy_batch",
    "tg_batch_tuning",
]


class TgStats(C.Structure):
    _fields_ = [
        ("mvps", C.c_int64), ("coarse_mvps", C.c_int64), ("vops", C.c_int64),
        ("cycles", C.c_int32), ("status", C.c_int32), ("relres", C.c_double),
        ("coarse_relres", C.c_double), ("kk", C.c_int32), ("eig_converged", C.c_int32),
        ("history", C.POINTER(C.c_double)), ("history_cap", C.c_int32), ("history_len", C.c_int32),
        ("fp64_cycles", C.c_int32), ("reserved", C.c_int32),
    ]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_ if f not in ("history", "reserved")}


class TgError(RuntimeError):
    def __init__(self, status, where):
        self.status = status
        super().__init__(f"{where}: {_lib.tg_status_string(status).decode()} "
                         f"({_lib.tg_last_error().decode()})")


_lib = None


def load() -> C.CDLL:
    """Load libtg.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: run `python -m paper_2005_03070_gb300.build`")
    lib = C.CDLL(LIB_PATH)
    vp, i32, i64, dbl = C.c_void_p, C.c_int, C.c_int64, C.c_double
    sig = {
        "tg_status_string": (C.c_char_p, [i32]),
        "tg_last_error": (C.c_char_p, []),
        "tg_setup_operator": (i32, [C.POINTER(vp), i32, C.POINTER(i64), i32, C.POINTER(dbl), C.POINTER(dbl), vp, i32, vp]),
        "tg_destroy_op": (i32, [vp]),
        "tg_op_size": (i64, [vp, i32]),
        "tg_apply": (i32, [vp, i32, i32, i32, vp, vp, vp]),
        "tg_prolong": (i32, [vp, vp, vp, i32, vp]),
        "tg_restrict": (i32, [vp, vp, vp, i32, vp]),
        "tg_op_set_interp": (i32, [vp, i32]),
        "tg_coarse_gmresdr": (i32, [vp, i32, vp, i32, i32, i32, dbl, dbl, i32, vp, C.POINTER(vp), i32, i32,
                                    C.POINTER(TgStats), vp]),
        "tg_defl_from_basis": (i32, [vp, i32, vp, i32, i32, i32, C.POINTER(vp), vp]),
        "tg_destroy_defl": (i32, [vp]),
        "tg_defl_copy": (i32, [vp, i32, vp, C.POINTER(i32), vp]),
        "tg_project": (i32, [vp, vp, vp, vp, vp]),
        "tg_solve_proj": (i32, [vp, vp, i32, i32, vp, vp, i32, dbl, i32, i32, i32, i64, C.POINTER(TgStats), vp]),
        "tg_solve_idr": (i32, [vp, vp, i32, vp, vp, i32, dbl, i32, i32, i32, vp, dbl, i64, C.POINTER(TgStats), vp]),
        "tg_improve_defl": (i32, [vp, vp, i32, i32, i32, i32, dbl, C.POINTER(C.c_double), C.POINTER(TgStats), vp]),
        "tg_adjoint_solve": (i32, [vp, vp, vp, vp, vp, vp, dbl, i32, i32, i32, C.POINTER(TgStats), vp]),
        "tg_kappa_gradient": (i32, [vp, vp, vp, vp, vp]),
        "tg_harmonic_ritz": (i32, [vp, i32, i32, i32, vp, vp, vp, C.POINTER(i32), vp]),
        "tg_harmonic_ritz_noalloc": (i32, [vp, i32, i32, i32, vp, vp, vp, C.POINTER(i32), vp]),
        "tg_batch_create": (i32, [C.POINTER(vp), i32, C.POINTER(i64), C.POINTER(dbl), i32, vp]),
        "tg_batch_layout": (i32, [vp, i32, C.POINTER(i64), C.POINTER(i64)]),
        "tg_batch_setup": (i32, [vp, vp, i32, i32, i32, dbl, dbl, i32, i32, i32, C.POINTER(TgStats), vp]),
        "tg_batch_solve": (i32, [vp, vp, vp, dbl, i32, i32, i64, i32, C.POINTER(TgStats), vp]),
        "tg_destroy_batch": (i32, [vp]),
        "tg_batch_tuning": (i32, [vp, C.POINTER(i32), C.POINTER(dbl), C.POINTER(i32), C.POINTER(i32),
                                  C.POINTER(dbl)]),
        "tg_profile_enable": (i32, [i32]),
        "tg_profile_read": (i32, [C.c_char_p, i32]),
        "tg_launch_count": (i64, []),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def _check(status, where, ok=(TG_OK,)):
    if status not in ok:
        raise TgError(status, where)
    return status


def _ptr(t: torch.Tensor | None):
    if t is None:
        return None
    if not t.is_cuda or not t.is_contiguous():
        raise ValueError("expected a contiguous CUDA tensor")
    return C.c_void_p(t.data_ptr())


def _stream(stream=None):
    s = torch.cuda.current_stream() if stream is None else stream
    return C.c_void_p(s.cuda_stream)


# ----------------------------------------------------------------------------- handles
class Operator:
    """tg_setup_operator: the fine operator and its coarse partner.

    kind: "cd2d" | "cd3d" | "vark2d" | "exp2d" | "u1_4d"; N: points per axis (odd) or lattice L;
    beta: convection speeds (exp2d: (beta_x, beta_y, gamma) of -exp(gamma x y) Lap u + beta . grad u);
    kappa: (N+2)^2 float64 CUDA tensor (vark2d); links: (4, L^4) complex128 CUDA tensor and mass
    (u1_4d); mass on the grid kinds: the reaction coefficient c of + c u (Helmholtz: -k^2);
    interp: "linear" (bilinear / trilinear) or "cubic" (fourth order, the stand-in for the
    paper's splines) for every prolongation of this operator (tg_op_set_interp)."""

    def __init__(self, kind, N, beta=(0.0,), kappa=None, links=None, mass=None, interp="linear", stream=None):
        lib = load()
        self.kind = KIND[kind] if isinstance(kind, str) else int(kind)
        self.N = int(N)
        h = C.c_void_p()
        dims = (C.c_int64 * 1)(self.N)
        b = (C.c_double * 3)(*(list(beta) + [0.0] * (3 - len(beta))))
        m = C.c_double(mass) if mass is not None else None
        coeffs = kappa if kappa is not None else links
        st = lib.tg_setup_operator(C.byref(h), self.kind, dims, 1, b, C.byref(m) if m is not None else None,
                                   _ptr(coeffs), 2, _stream(stream))
        _check(st, "tg_setup_operator")
        self._h = h
        if interp != "linear":
            _check(lib.tg_op_set_interp(h, INTERP[interp]), "tg_op_set_interp")
        self.interp = interp
        self.n = lib.tg_op_size(h, TG_FINE)
        self.nc = lib.tg_op_size(h, TG_COARSE)
        self.complex = self.kind == TG_U1_4D
        self.dtype = torch.complex128 if self.complex else torch.float64

    def __del__(self):
        if getattr(self, "_h", None) and _lib is not None:
            _lib.tg_destroy_op(self._h)
            self._h = None

    @property
    def handle(self):
        return self._h

    def apply(self, x, y=None, level=TG_FINE, transpose=False, precision=TG_F64, stream=None):
        if y is None:
            y = torch.empty_like(x)
        _check(_lib.tg_apply(self._h, level, int(transpose), precision, _ptr(x), _ptr(y), _stream(stream)),
               "tg_apply")
        return y

    def prolong(self, coarse, fine=None, stream=None):
        ncols = coarse.numel() // self.nc
        if fine is None:
            fine = torch.empty(ncols * self.n, dtype=coarse.dtype, device=coarse.device)
        _check(_lib.tg_prolong(self._h, _ptr(coarse), _ptr(fine), ncols, _stream(stream)), "tg_prolong")
        return fine

    def restrict(self, fine, coarse=None, stream=None):
        ncols = fine.numel() // self.n
        if coarse is None:
            coarse = torch.empty(ncols * self.nc, dtype=fine.dtype, device=fine.device)
        _check(_lib.tg_restrict(self._h, _ptr(fine), _ptr(coarse), ncols, _stream(stream)), "tg_restrict")
        return coarse

    def coarse_gmresdr(self, b, m, k, nev=None, rtolev=1e-4, rtol=1e-8, max_cycles=300, transpose=False,
                       proj="minres", precision="f64", want_xc=True, want_defl=True, stream=None):
        """tg_coarse_gmresdr: returns (x_c or None, Deflation or None, stats dict, status)."""
        nev = k if nev is None else nev
        xc = torch.empty(self.nc, dtype=self.dtype, device=b.device) if want_xc else None
        d = C.c_void_p()
        st = TgStats()
        status = _lib.tg_coarse_gmresdr(self._h, int(transpose), _ptr(b), m, k, nev, rtolev, rtol, max_cycles,
                                        _ptr(xc), C.byref(d) if want_defl else None, PROJ[proj], PREC[precision],
                                        C.byref(st), _stream(stream))
        _check(status, "tg_coarse_gmresdr", ok=(TG_OK, TG_NOT_CONVERGED))
        defl = Deflation(d, self) if want_defl and d.value else None
        return xc, defl, st.as_dict(), status

    def defl_from_basis(self, Y, k, proj="minres", precision="f64", transpose=False, stream=None):
        d = C.c_void_p()
        _check(_lib.tg_defl_from_basis(self._h, int(transpose), _ptr(Y), k, PROJ[proj], PREC[precision],
                                       C.byref(d), _stream(stream)), "tg_defl_from_basis")
        return Deflation(d, self)

    def solve(self, b, x, defl=None, method="bicgstab", precision="f64", rtol=1e-8, ncyc=0, restart_mvps=60,
              m3=20, max_mvps=10 ** 7, nrhs=1, history=0, stream=None, raise_on_fail=False):
        """tg_solve_proj on b (n x nrhs column-major); x holds x0 and receives the solution."""
        stats = (TgStats * nrhs)()
        bufs = []
        if history:
            for s in stats:
                buf = (C.c_double * (3 * history))()
                bufs.append(buf)
                s.history = C.cast(buf, C.POINTER(C.c_double))
                s.history_cap = history
        status = _lib.tg_solve_proj(self._h, defl.handle if defl is not None else None, METHOD[method],
                                    PREC[precision], _ptr(b), _ptr(x), nrhs, rtol, ncyc, restart_mvps, m3,
                                    max_mvps, stats, _stream(stream))
        if raise_on_fail:
            _check(status, "tg_solve_proj")
        elif status in (TG_BAD_ARG, TG_OOM, TG_CUDA_ERROR):
            _check(status, "tg_solve_proj")
        out = []
        for i, s in enumerate(stats):
            d = s.as_dict()
            if history:
                n = min(s.history_len, history)
                d["history"] = [tuple(bufs[i][3 * j:3 * j + 3]) for j in range(n)]
            out.append(d)
        return status, out

    def solve_idr(self, b, x, P, defl=None, rtol=1e-8, ncyc=20, restart_mvps=0, kappa=0.7, max_mvps=10 ** 7,
                  nrhs=1, history=0, precision="f64", stream=None):
        """tg_solve_idr: IDR(s)-Proj(k) with s = P's column count; P is an (s, n) tensor whose
        rows are the shadow columns (the library orthonormalises them); precision "f64" or
        "f32_ir" (float32 cycles with float64 refinement, real operators)."""
        s = P.shape[0]
        stats = (TgStats * nrhs)()
        bufs = []
        if history:
            for st in stats:
                buf = (C.c_double * (3 * history))()
                bufs.append(buf)
                st.history = C.cast(buf, C.POINTER(C.c_double))
                st.history_cap = history
        status = _lib.tg_solve_idr(self._h, defl.handle if defl is not None else None, PREC[precision], _ptr(b), _ptr(x),
                                   nrhs, rtol, ncyc, restart_mvps, s, _ptr(P.contiguous()), kappa, max_mvps, stats,
                                   _stream(stream))
        if status in (TG_BAD_ARG, TG_OOM, TG_CUDA_ERROR):
            _check(status, "tg_solve_idr")
        out = []
        for i, st in enumerate(stats):
            d = st.as_dict()
            if history:
                n = min(st.history_len, history)
                d["history"] = [tuple(bufs[i][3 * j:3 * j + 3]) for j in range(n)]
            out.append(d)
        return status, out

    def adjoint_solve(self, defl_left, g, lam, x=None, dkappa=None, rtol=1e-8, ncyc=0, restart_mvps=60,
                      precision="f64", stream=None):
        st = TgStats()
        status = _lib.tg_adjoint_solve(self._h, defl_left.handle if defl_left is not None else None, _ptr(g),
                                       _ptr(lam), _ptr(x), _ptr(dkappa), rtol, ncyc, restart_mvps,
                                       PREC[precision], C.byref(st), _stream(stream))
        return status, st.as_dict()

    def kappa_gradient(self, x, lam, dkappa=None, stream=None):
        if dkappa is None:
            dkappa = torch.empty((self.N + 2) ** 2, dtype=torch.float64, device=x.device)
        _check(_lib.tg_kappa_gradient(self._h, _ptr(x), _ptr(lam), _ptr(dkappa), _stream(stream)),
               "tg_kappa_gradient")
        return dkappa


class Deflation:
    """A tg_defl handle (Y, A Y factored, projection data)."""

    def __init__(self, handle: C.c_void_p, op: Operator):
        self._h = handle
        self.op = op
        kk = C.c_int()
        _check(_lib.tg_defl_copy(handle, 0, None, C.byref(kk), None), "tg_defl_copy")
        self.kk = kk.value

    def __del__(self):
        if getattr(self, "_h", None) and _lib is not None:
            _lib.tg_destroy_defl(self._h)
            self._h = None

    @property
    def handle(self):
        return self._h

    def copy(self, what: int, stream=None):
        """0: Y, 1: Q (MinRes) / V (Galerkin), 2: A Y, 3: R / H.  Returns a CUDA tensor
        shaped (kk, n) for bases (row c = column c) or (kk, kk) transposed storage."""
        n = self.op.n
        shape = (self.kk, self.kk) if what == 3 else (self.kk, n)
        out = torch.empty(shape, dtype=self.op.dtype, device="cuda")
        _check(_lib.tg_defl_copy(self._h, what, _ptr(out), None, _stream(stream)), "tg_defl_copy")
        return out

    def project(self, x, r, stream=None):
        _check(_lib.tg_project(self.op.handle, self._h, _ptr(x), _ptr(r), _stream(stream)), "tg_project")

    def improve(self, m, cycles, nstart, nev=0, rtolev=0.0, stream=None):
        """tg_improve_defl: Arnoldi-E(m, kk) cycles on the fine grid; returns (kept Ritz values
        as a complex numpy array, stats dict)."""
        import numpy as np
        th = (C.c_double * (2 * (self.kk + 1)))()
        st = TgStats()
        _check(_lib.tg_improve_defl(self.op.handle, self._h, m, cycles, nstart, nev, rtolev, th, C.byref(st),
                                    _stream(stream)), "tg_improve_defl")
        kk = C.c_int()
        _check(_lib.tg_defl_copy(self._h, 0, None, C.byref(kk), None), "tg_defl_copy")
        self.kk = kk.value
        a = np.array(th[:2 * self.kk]).reshape(-1, 2)
        return a[:, 0] + 1j * a[:, 1], st.as_dict()


def harmonic_ritz(Hbar_colmajor: torch.Tensor, m: int, k: int, complex_: bool = False, stream=None):
    """tg_harmonic_ritz on a (m+1) x m matrix given column-major (a (m, m+1) row-major tensor).
    Returns (theta complex tensor (m,), basis (kk, m) rows = columns of P_k, eres (kk,))."""
    load()
    dev = Hbar_colmajor.device
    theta = torch.empty(2 * m, dtype=torch.float64, device=dev)
    dt = torch.complex128 if complex_ else torch.float64
    basis = torch.empty(m * m, dtype=dt, device=dev)
    eres = torch.empty(m, dtype=torch.float64, device=dev)
    kk = C.c_int()
    st = _lib.tg_harmonic_ritz(_ptr(Hbar_colmajor), m, k, int(complex_), _ptr(theta), _ptr(basis), _ptr(eres),
                               C.byref(kk), _stream(stream))
    _check(st, "tg_harmonic_ritz")
    kk = kk.value
    th = theta.view(m, 2)
    return torch.complex(th[:, 0], th[:, 1]), basis[: kk * m].view(kk, m), eres[:kk]


def tg_profile_enable(on: bool) -> None:
    _check(load().tg_profile_enable(int(on)), "tg_profile_enable")


def tg_profile_read() -> dict:
    import json
    buf = C.create_string_buffer(1 << 16)
    _check(load().tg_profile_read(buf, len(buf)), "tg_profile_read")
    return json.loads(buf.value.decode())


def tg_launch_count() -> int:
    return int(load().tg_launch_count())


class Batch:
    """tg_batch_*: independent 2D convection-diffusion instances, 8 right-hand sides each,
    sharing one deflation basis per instance (float32 inner / float64 refinement)."""
    R = 8

    def __init__(self, Ns, betas, stream=None):
        lib = load()
        self.count = len(Ns)
        h = C.c_void_p()
        ns = (C.c_int64 * self.count)(*[int(v) for v in Ns])
        bs = (C.c_double * self.count)(*[float(v) for v in betas])
        _check(lib.tg_batch_create(C.byref(h), self.count, ns, bs, self.R, _stream(stream)), "tg_batch_create")
        self._h = h
        self.offsets, self.sizes = [], []
        for i in range(self.count):
            o, n = C.c_int64(), C.c_int64()
            _check(lib.tg_batch_layout(h, i, C.byref(o), C.byref(n)), "tg_batch_layout")
            self.offsets.append(o.value)
            self.sizes.append(n.value)
        self.total = self.offsets[-1] + self.sizes[-1] * self.R

    def __del__(self):
        if getattr(self, "_h", None) and _lib is not None:
            _lib.tg_destroy_batch(self._h)
            self._h = None

    def setup(self, rhs, m=40, k=20, nev=None, rtolev=1e-2, rtol=1e-8, max_cycles=300, proj="minres", threads=16,
              stream=None):
        nev = k if nev is None else nev
        stats = (TgStats * self.count)()
        st = _lib.tg_batch_setup(self._h, _ptr(rhs), m, k, nev, rtolev, rtol, max_cycles, PROJ[proj], threads, stats,
                                 _stream(stream))
        _check(st, "tg_batch_setup")
        return [s.as_dict() for s in stats]

    def tuning(self):
        """tg_batch_tuning: {"blocks_per_instance", "us_per_iteration", "candidates": {blocks: us}}."""
        g, us, nc = C.c_int(), C.c_double(), C.c_int()
        cb = (C.c_int * 8)()
        cu = (C.c_double * 8)()
        _check(_lib.tg_batch_tuning(self._h, C.byref(g), C.byref(us), C.byref(nc), cb, cu), "tg_batch_tuning")
        return {"blocks_per_instance": g.value, "us_per_iteration": round(us.value, 2),
                "candidates": {str(cb[i]): round(cu[i], 2) for i in range(nc.value)}}

    def solve(self, rhs, x, rtol=1e-8, ncyc=20, restart_mvps=0, max_mvps=10 ** 6, threads=16, stream=None):
        stats = (TgStats * (self.count * self.R))()
        st = _lib.tg_batch_solve(self._h, _ptr(rhs), _ptr(x), rtol, ncyc, restart_mvps, max_mvps, threads, stats,
                                 _stream(stream))
        if st in (TG_BAD_ARG, TG_OOM, TG_CUDA_ERROR, TG_SYNC_TIMEOUT):
            _check(st, "tg_batch_solve")
        return st, [s.as_dict() for s in stats]
