"""Python binding of libstokesmg (argument marshalling only).

Every numerical step runs in the CUDA library behind the C ABI declared in
include/stokesmg.h; this module only checks tensors and forwards pointers.
There is no CPU fallback: importing works without a GPU, but constructing a
`StokesMG` needs the compiled library and a CUDA device, and fails loudly
otherwise.
"""
from __future__ import annotations

import ctypes
import os

__all__ = ["StokesMG", "load_library", "library_path", "StokesError", "layout_sizes", "patch_eigen", "cell_tables", "transfer_tables", "solve_batch", "smooth_batch", "F64", "F32"]

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIBNAME = "libstokesmg.so"

F64, F32 = 0, 1
PREC_FP64, PREC_MIXED = 0, 1
CG_FIXED, CG_TOL, LOCAL_DIRECT = 0, 1, 2
_STATUS = {0: "STK_OK", -1: "STK_EINVAL", -2: "STK_ECUDA", -3: "STK_ENOMEM", -4: "STK_ENOCONV", -5: "STK_ETIMEOUT", -6: "STK_ESTATE"}


class StokesError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{_STATUS.get(code, code)}: {msg}")
        self.code = code


class Options(ctypes.Structure):
    _fields_ = [
        ("precision", ctypes.c_int),
        ("gmres_restart", ctypes.c_int),
        ("max_iter", ctypes.c_int),
        ("local_cg_mode", ctypes.c_int),
        ("local_cg_iters", ctypes.c_int),
        ("local_cg_tol", ctypes.c_double),
        ("penalty_factor", ctypes.c_double),
        ("stream", ctypes.c_void_p),
        ("use_graphs", ctypes.c_int),
        ("fused_smoother", ctypes.c_int),
        ("direct_gemm", ctypes.c_int),
    ]


class SolveInfo(ctypes.Structure):
    _fields_ = [
        ("iterations", ctypes.c_int),
        ("converged", ctypes.c_int),
        ("relres", ctypes.c_double),
        ("nu", ctypes.c_double),
        ("seconds", ctypes.c_double),
        ("residuals", ctypes.c_double * 256),
    ]


def library_path() -> str:
    return os.path.join(_HERE, _LIBNAME)


_lib = None


def load_library():
    """Load the in-tree libstokesmg.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    path = library_path()
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build it with python -m paper_2410_09497_gb300.build")
    lib = ctypes.CDLL(path)
    P = ctypes.c_void_p
    i64p = ctypes.POINTER(ctypes.c_int64)
    sig = {
        "stk_default_options": (ctypes.c_int, [ctypes.POINTER(Options)]),
        "stk_setup": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.POINTER(Options), ctypes.POINTER(P)]),
        "stk_setup_planar": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.POINTER(Options), ctypes.POINTER(P)]),
        "stk_planar_errors": (ctypes.c_int, [P, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_double), P, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)]),
        "stk_destroy": (ctypes.c_int, [P]),
        "stk_last_error": (ctypes.c_char_p, [P]),
        "stk_num_levels": (ctypes.c_int, [P, ctypes.POINTER(ctypes.c_int)]),
        "stk_layout": (ctypes.c_int, [P, ctypes.c_int, ctypes.POINTER(ctypes.c_int), i64p, i64p, i64p]),
        "stk_apply": (ctypes.c_int, [P, ctypes.c_int, ctypes.c_int, P, P]),
        "stk_residual": (ctypes.c_int, [P, ctypes.c_int, ctypes.c_int, P, P, P]),
        "stk_apply_stage": (ctypes.c_int, [P, ctypes.c_int, ctypes.c_int, ctypes.c_int, P, P]),
        "stk_prolongate_add": (ctypes.c_int, [P, ctypes.c_int, ctypes.c_int, P, P]),
        "stk_restrict": (ctypes.c_int, [P, ctypes.c_int, ctypes.c_int, P, P]),
        "stk_smooth": (ctypes.c_int, [P, ctypes.c_int, ctypes.c_int, P, P]),
        "stk_coarse_solve": (ctypes.c_int, [P, ctypes.c_int, P, P]),
        "stk_vcycle": (ctypes.c_int, [P, ctypes.c_int, P, P]),
        "stk_solve": (ctypes.c_int, [P, P, P, ctypes.c_double, ctypes.POINTER(SolveInfo)]),
        "stk_rhs": (ctypes.c_int, [P, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_double), P]),
        "stk_smooth_static": (ctypes.c_int, [P, ctypes.c_int, ctypes.c_int, P, P]),
        "stk_smooth_colour": (ctypes.c_int, [P, ctypes.c_int, ctypes.c_int, ctypes.c_int, P, P]),
        "stk_autotune": (ctypes.c_int, [P, ctypes.c_int]),
        "stk_tuning": (ctypes.c_int, [P, ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_int)]),
        "stk_set_tuning": (ctypes.c_int, [P, ctypes.c_int, ctypes.c_int, ctypes.c_int]),
        "stk_tuned_smoother": (ctypes.c_int, [P, ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_int)]),
        "stk_tuned_split": (ctypes.c_int, [P, ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_int)]),
        "stk_solve_batch": (ctypes.c_int, [ctypes.POINTER(P), ctypes.c_int, ctypes.POINTER(P), ctypes.POINTER(P), ctypes.c_double, ctypes.POINTER(SolveInfo)]),
        "stk_smooth_batch": (ctypes.c_int, [ctypes.POINTER(P), ctypes.c_int, ctypes.POINTER(ctypes.c_int), ctypes.c_int, ctypes.POINTER(P), ctypes.POINTER(P)]),
        "stk_patch_eigen": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_int, P, P, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)]),
        "stk_cell_tables": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double, P]),
        "stk_transfer_tables": (ctypes.c_int, [ctypes.c_int, P]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def layout_sizes(n: int, k: int):
    """(n_vel_component, n_pressure, n_total) of the vector layout of an n^3 mesh at degree k."""
    m = n * (k + 1)
    nv = (m + 1) * m * m
    return nv, m ** 3, 3 * nv + m ** 3


def patch_eigen(n: int, k: int, direction: int, nu: float = 1.0, penalty_factor: float = 1.0):
    """(S, lam, even_odd) of stk_patch_eigen: the 1D fast-diagonalization
    eigenpairs the library builds for a level of n cells per side (host
    computation, no GPU needed).  S is a dim x dim NumPy array with the
    eigenvectors in its columns."""
    import numpy as np

    lib = load_library()
    npd = 2 * k + 2
    S = np.zeros(npd * npd)
    lam = np.zeros(npd)
    dim, eo = ctypes.c_int(), ctypes.c_int()
    rc = lib.stk_patch_eigen(int(n), int(k), float(nu), float(penalty_factor), int(direction), S.ctypes.data, lam.ctypes.data, ctypes.byref(dim), ctypes.byref(eo))
    if rc != 0:
        raise StokesError(rc, (lib.stk_last_error(None) or b"").decode())
    d = dim.value
    return S[: d * d].reshape(d, d).copy(), lam[:d].copy(), bool(eo.value)


def cell_tables(n: int, k: int, nu: float = 1.0, penalty_factor: float = 1.0):
    """The 1D cell matrices of stk_cell_tables as a dict of NumPy arrays
    (KC, MC, D, LS with shape (3, k+1, k+1), LLO, LHI, S); host computation,
    no GPU needed."""
    import numpy as np

    lib = load_library()
    nc, nd = k + 2, k + 1
    shapes = [("KC", (nc, nc)), ("MC", (nc, nc)), ("D", (nd, nc)), ("LS", (3, nd, nd)), ("LLO", (nd, nd)),
              ("LHI", (nd, nd)), ("S", (nd,))]
    buf = np.zeros(sum(int(np.prod(s)) for _, s in shapes))
    rc = lib.stk_cell_tables(int(n), int(k), float(nu), float(penalty_factor), buf.ctypes.data)
    if rc != 0:
        raise StokesError(rc, (lib.stk_last_error(None) or b"").decode())
    out, o = {}, 0
    for name, s in shapes:
        size = int(np.prod(s))
        out[name] = buf[o:o + size].reshape(s).copy()
        o += size
    return out


def transfer_tables(k: int):
    """(PC, PD) of stk_transfer_tables as NumPy arrays of shape (2, k+2, k+2)
    and (2, k+1, k+1); host computation, no GPU needed."""
    import numpy as np

    lib = load_library()
    nc, nd = k + 2, k + 1
    buf = np.zeros(2 * nc * nc + 2 * nd * nd)
    rc = lib.stk_transfer_tables(int(k), buf.ctypes.data)
    if rc != 0:
        raise StokesError(rc, (lib.stk_last_error(None) or b"").decode())
    return buf[: 2 * nc * nc].reshape(2, nc, nc).copy(), buf[2 * nc * nc:].reshape(2, nd, nd).copy()


class StokesMG:
    """One Stokes problem on the unit cube with n cells per side and degree k.

    All work is ordered on the CUDA stream that is current when the object is
    created (or the one passed as `stream`).
    """

    def __init__(self, n: int, k: int, nu: float = 1.0, *, precision: int = PREC_FP64, gmres_restart: int = 20,
                 max_iter: int = 200, local_cg_mode: int = CG_FIXED, local_cg_iters: int = 15,
                 local_cg_tol: float = 1e-8, penalty_factor: float = 1.0, use_graphs: bool = True,
                 fused_smoother: bool = False, direct_gemm: int = 2, dim: int = 3, stream=None):
        import torch

        if not torch.cuda.is_available():
            raise RuntimeError("StokesMG needs a CUDA device")
        self._torch = torch
        self.lib = load_library()
        opt = Options()
        self.lib.stk_default_options(ctypes.byref(opt))
        opt.precision, opt.gmres_restart, opt.max_iter = precision, gmres_restart, max_iter
        opt.local_cg_mode, opt.local_cg_iters, opt.local_cg_tol = local_cg_mode, local_cg_iters, local_cg_tol
        opt.penalty_factor = penalty_factor
        opt.use_graphs = 1 if use_graphs else 0
        opt.fused_smoother = 1 if fused_smoother else 0
        opt.direct_gemm = int(direct_gemm)
        s = stream if stream is not None else torch.cuda.current_stream()
        self.stream = s
        opt.stream = ctypes.c_void_p(s.cuda_stream)
        h = ctypes.c_void_p()
        if dim not in (2, 3):
            raise ValueError("dim must be 2 or 3")
        setup = self.lib.stk_setup_planar if dim == 2 else self.lib.stk_setup
        rc = setup(int(n), int(k), float(nu), ctypes.byref(opt), ctypes.byref(h))
        self.dim = dim
        if rc != 0:
            raise StokesError(rc, self.lib.stk_last_error(None).decode())
        self.h = h
        self.n, self.k, self.nu = n, k, nu
        nl = ctypes.c_int()
        self.lib.stk_num_levels(self.h, ctypes.byref(nl))
        self.num_levels = nl.value

    def close(self):
        if getattr(self, "h", None):
            self.lib.stk_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, rc):
        if rc != 0:
            raise StokesError(rc, self.lib.stk_last_error(self.h).decode())

    def layout(self, level: int = -1):
        level = self._lvl(level)
        nc = ctypes.c_int()
        a, b, c = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
        self._check(self.lib.stk_layout(self.h, level, ctypes.byref(nc), ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)))
        return {"n": nc.value, "n_vel_component": a.value, "n_pressure": b.value, "n_total": c.value}

    def _lvl(self, level):
        return level % self.num_levels if level < 0 else level

    def _dt(self, t):
        torch = self._torch
        if t.dtype == torch.float64:
            return F64
        if t.dtype == torch.float32:
            return F32
        raise TypeError("vectors must be float64 or float32")

    def _vec(self, t, level, dt=None):
        if not t.is_cuda or not t.is_contiguous():
            raise ValueError("vectors must be contiguous CUDA tensors")
        if t.numel() != self.layout(level)["n_total"]:
            raise ValueError("vector length does not match the level's layout")
        if dt is not None and self._dt(t) != dt:
            raise TypeError("all vectors of a call must have the same dtype")
        return ctypes.c_void_p(t.data_ptr())

    def apply(self, x, y, level: int = -1):
        """y = A x on `level` (Algorithm 1)."""
        level = self._lvl(level)
        dt = self._dt(x)
        self._check(self.lib.stk_apply(self.h, level, dt, self._vec(x, level), self._vec(y, level, dt)))
        return y

    def apply_stage(self, stage: int, x, y, level: int = -1):
        """Stage 0: velocity rows of y = A x; stage 1: pressure rows."""
        level = self._lvl(level)
        dt = self._dt(x)
        self._check(self.lib.stk_apply_stage(self.h, level, dt, int(stage), self._vec(x, level), self._vec(y, level, dt)))
        return y

    def residual(self, x, b, r, level: int = -1):
        """r = b - A x on `level`."""
        level = self._lvl(level)
        dt = self._dt(x)
        self._check(self.lib.stk_residual(self.h, level, dt, self._vec(x, level), self._vec(b, level, dt), self._vec(r, level, dt)))
        return r

    def prolongate_add(self, xc, xf, fine_level: int = -1):
        """xf += I^up xc (xc on fine_level - 1)."""
        fl = self._lvl(fine_level)
        dt = self._dt(xc)
        self._check(self.lib.stk_prolongate_add(self.h, fl, dt, self._vec(xc, fl - 1), self._vec(xf, fl, dt)))
        return xf

    def restrict(self, rf, rc, fine_level: int = -1):
        """rc = I^down rf (transpose of the embedding)."""
        fl = self._lvl(fine_level)
        dt = self._dt(rf)
        self._check(self.lib.stk_restrict(self.h, fl, dt, self._vec(rf, fl), self._vec(rc, fl - 1, dt)))
        return rc

    def smooth(self, x, b, level: int = -1):
        """One step of Algorithm 2 on `level`, x updated in place."""
        level = self._lvl(level)
        dt = self._dt(x)
        self._check(self.lib.stk_smooth(self.h, level, dt, self._vec(x, level), self._vec(b, level, dt)))
        return x

    def smooth_colour(self, colour: int, x, b, level: int = -1):
        """One colour of Algorithm 2 on `level` (residual, then that colour's patch solves), x in place."""
        level = self._lvl(level)
        dt = self._dt(x)
        self._check(self.lib.stk_smooth_colour(self.h, level, dt, int(colour), self._vec(x, level), self._vec(b, level, dt)))
        return x

    def smooth_static(self, x, b, level: int = -1):
        """stk_smooth without device allocation (residual in the library's static 32 MiB array)."""
        level = self._lvl(level)
        dt = self._dt(x)
        self._check(self.lib.stk_smooth_static(self.h, level, dt, self._vec(x, level), self._vec(b, level, dt)))
        return x

    def autotune(self, dtype: int = F32, with_smoother: bool = False):
        """Time the apply's march run length per level (and the smoother's form and
        interior-patch launch split on the smoothed levels) for dtype and keep the
        fastest; returns {level: cells_per_run} or, with with_smoother,
        {level: (cells_per_run, fused, split)}."""
        self._check(self.lib.stk_autotune(self.h, int(dtype)))
        out = {}
        for level in range(self.num_levels):
            v, f, sp = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
            self._check(self.lib.stk_tuning(self.h, level, int(dtype), ctypes.byref(v)))
            self._check(self.lib.stk_tuned_smoother(self.h, level, int(dtype), ctypes.byref(f)))
            self._check(self.lib.stk_tuned_split(self.h, level, int(dtype), ctypes.byref(sp)))
            out[level] = (v.value, f.value, sp.value) if with_smoother else v.value
        return out

    def set_tuning(self, level: int, dtype: int, cells_per_run: int):
        """Set the apply's march run length of a level and dtype (0: built-in choice)."""
        self._check(self.lib.stk_set_tuning(self.h, self._lvl(level), int(dtype), int(cells_per_run)))

    def coarse_solve(self, b, x):
        """x = A_0^+ b on level 0."""
        dt = self._dt(b)
        self._check(self.lib.stk_coarse_solve(self.h, dt, self._vec(b, 0), self._vec(x, 0, dt)))
        return x

    def vcycle(self, b, x):
        """x = one V-cycle applied to b (x0 = 0) on the finest level."""
        L = self.num_levels - 1
        dt = self._dt(b)
        self._check(self.lib.stk_vcycle(self.h, dt, self._vec(b, L), self._vec(x, L, dt)))
        return x

    def rhs(self, coeffs: dict, b):
        """b = (f, phi) of the manufactured solution with the given seeded coefficients (finest level)."""
        import numpy as np

        L = self.num_levels - 1
        pf = np.ascontiguousarray(coeffs["psi_freq"], dtype=np.int32).reshape(-1)
        pa = np.ascontiguousarray(coeffs["psi_amp"], dtype=np.float64).reshape(-1)
        qf = np.ascontiguousarray(coeffs["p_freq"], dtype=np.int32).reshape(-1)
        qa = np.ascontiguousarray(coeffs["p_amp"], dtype=np.float64).reshape(-1)
        ip = ctypes.POINTER(ctypes.c_int)
        dp = ctypes.POINTER(ctypes.c_double)
        self._check(self.lib.stk_rhs(self.h, pf.ctypes.data_as(ip), pa.ctypes.data_as(dp), qf.ctypes.data_as(ip),
                                     qa.ctypes.data_as(dp), self._vec(b, L, F64)))
        return b

    @staticmethod
    def _coeff_arrays(coeffs):
        import numpy as np

        pf = np.ascontiguousarray(coeffs["psi_freq"], dtype=np.int32).reshape(-1)
        pa = np.ascontiguousarray(coeffs["psi_amp"], dtype=np.float64).reshape(-1)
        qf = np.ascontiguousarray(coeffs["p_freq"], dtype=np.int32).reshape(-1)
        qa = np.ascontiguousarray(coeffs["p_amp"], dtype=np.float64).reshape(-1)
        return pf, pa, qf, qa

    def planar_errors(self, coeffs: dict, x):
        """(||u - u_h||_L2, ||(-p) - p_h||_L2) of a 2D discrete solution x against the
        manufactured solution of `coeffs` (stk_planar_errors)."""
        L = self.num_levels - 1
        pf, pa, qf, qa = self._coeff_arrays(coeffs)
        ip = ctypes.POINTER(ctypes.c_int)
        dp = ctypes.POINTER(ctypes.c_double)
        eu, ep = ctypes.c_double(), ctypes.c_double()
        self._check(self.lib.stk_planar_errors(self.h, pf.ctypes.data_as(ip), pa.ctypes.data_as(dp), qf.ctypes.data_as(ip),
                                               qa.ctypes.data_as(dp), self._vec(x, L, F64), ctypes.byref(eu), ctypes.byref(ep)))
        return eu.value, ep.value

    def solve(self, b, x, rtol: float = 1e-8, check: bool = True):
        """FGMRES + V-cycle solve of A x = b (FP64 vectors); returns an info dict."""
        L = self.num_levels - 1
        if self._dt(b) != F64 or self._dt(x) != F64:
            raise TypeError("solve takes float64 vectors")
        info = SolveInfo()
        rc = self.lib.stk_solve(self.h, self._vec(b, L), self._vec(x, L), float(rtol), ctypes.byref(info))
        if rc != 0 and (check or rc != -4):
            self._check(rc)
        n = info.iterations
        return {"iterations": n, "converged": bool(info.converged), "relres": info.relres, "nu": info.nu,
                "seconds": info.seconds, "residuals": list(info.residuals[: min(n, 255) + 1]), "status": rc}


def smooth_batch(problems, xs, bs, levels=None):
    """One smoothing step of several problems of the same degree (stk_smooth_batch),
    on problems[0]'s stream; levels default to every problem's finest level."""
    lib = load_library()
    n = len(problems)
    if levels is None:
        levels = [p.num_levels - 1 for p in problems]
    dt = problems[0]._dt(xs[0])
    P = ctypes.c_void_p
    hs = (P * n)(*[p.h for p in problems])
    lv = (ctypes.c_int * n)(*[p._lvl(l) for p, l in zip(problems, levels)])
    xp = (P * n)(*[p._vec(x, p._lvl(l), dt) for p, x, l in zip(problems, xs, levels)])
    bp = (P * n)(*[p._vec(b, p._lvl(l), dt) for p, b, l in zip(problems, bs, levels)])
    rc = lib.stk_smooth_batch(hs, n, lv, dt, xp, bp)
    if rc != 0:
        raise StokesError(rc, lib.stk_last_error(None).decode())


def solve_batch(problems, bs, xs, rtol: float = 1e-8):
    """Solve several independent problems together (stk_solve_batch); returns a list of info dicts.

    For concurrency each problem should have been created with its own CUDA stream.
    """
    lib = load_library()
    n = len(problems)
    P = ctypes.c_void_p
    hs = (P * n)(*[p.h for p in problems])
    bp = (P * n)(*[p._vec(b, p.num_levels - 1, F64) for p, b in zip(problems, bs)])
    xp = (P * n)(*[p._vec(x, p.num_levels - 1, F64) for p, x in zip(problems, xs)])
    infos = (SolveInfo * n)()
    rc = lib.stk_solve_batch(hs, n, bp, xp, float(rtol), infos)
    if rc != 0 and rc != -4:
        raise StokesError(rc, lib.stk_last_error(None).decode())
    out = []
    for i in range(n):
        it = infos[i].iterations
        out.append({"iterations": it, "converged": bool(infos[i].converged), "relres": infos[i].relres,
                    "nu": infos[i].nu, "seconds": infos[i].seconds,
                    "residuals": list(infos[i].residuals[: min(it, 255) + 1])})
    return out
