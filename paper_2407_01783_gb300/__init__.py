"""GB300-native generalized Stokes solver (P2-P1 Taylor-Hood on Kuhn meshes).

Thin Python binding over the C ABI of ``include/stokes.h``: the functions here
have the C names and only marshal arguments (PyTorch tensors provide device
memory and streams). Every step of a solve runs in the CUDA library; importing
this package without the compiled library raises.

Method (Creff & Guermond, arXiv 2407.01783): A U - B^T P = F, B U = g with
A = M_V/dt + mu E_V (optionally augmented Lagrangian), solved by Schur-complement
CG with the Cahouet-Chabard preconditioner (Method 1) or by FGMRES with a
block preconditioner on the coupled system (Method 2).
"""

from __future__ import annotations

import ctypes as C

import numpy as np
import torch

from . import _lib
from ._lib import (KERNEL, MAT, METHOD_COUPLED, METHOD_SCHUR, OP, PRECISION_FP64,
                   PRECISION_MIXED, SCHUR_PREC_LAPLACE, SCHUR_PREC_LUMPED, StokesInfo,
                   StokesOptions)

__all__ = ["StokesError", "StokesOptions", "StokesInfo", "Stokes", "StokesBatch", "stokes_default_options",
           "stokes_solve_multi",
           "stokes_setup", "stokes_solve", "stokes_solve_host", "stokes_adjoint",
           "stokes_destroy", "stokes_apply", "stokes_apply_agamma_noalloc", "stokes_matrix_export", "stokes_sizes",
           "stokes_kernel_stats", "stokes_kernel_timing", "stokes_kernel_stats_reset", "stokes_profile_mode",
           "stokes_setup_phases", "StokesSolve", "OP", "MAT",
           "KERNEL", "METHOD_SCHUR", "METHOD_COUPLED", "SCHUR_PREC_LUMPED",
           "SCHUR_PREC_LAPLACE", "PRECISION_FP64", "PRECISION_MIXED", "library_path"]

_L = _lib.load()


def library_path() -> str:
    return _lib.LIB_PATH


class StokesError(RuntimeError):
    def __init__(self, status: int, where: str):
        msg = _L.stokes_last_error().decode() or _L.stokes_status_string(status).decode()
        super().__init__(f"{where}: {_lib.STATUS.get(status, status)}: {msg}")
        self.status = status


def _check(status: int, where: str, allow=()):
    if status != 0 and status not in allow:
        raise StokesError(status, where)
    return status


def _ptr(t):
    if t is None:
        return None
    if isinstance(t, torch.Tensor):
        if not t.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return C.c_void_p(t.data_ptr())
    if isinstance(t, np.ndarray):
        if not t.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        return C.c_void_p(t.ctypes.data)
    raise TypeError(type(t))


def stokes_default_options(**overrides) -> StokesOptions:
    o = StokesOptions()
    _L.stokes_default_options(C.byref(o))
    for k, v in overrides.items():
        if not hasattr(o, k):
            raise KeyError(k)
        setattr(o, k, v)
    return o


def stokes_setup(n: int, vertices, mu: float, dt: float, gamma: float = 0.0,
                 options: StokesOptions | None = None, stream: torch.cuda.Stream | None = None):
    """Build all operators on the current CUDA device; returns an opaque handle."""
    V = np.ascontiguousarray(np.asarray(vertices, dtype=np.float64))
    if V.shape != ((n + 1) ** 3, 3):
        raise ValueError(f"vertices must have shape {((n + 1) ** 3, 3)}")
    if options is None:
        options = stokes_default_options()
    s = stream if stream is not None else torch.cuda.current_stream()
    h = C.c_void_p()
    _check(_L.stokes_setup(n, _ptr(V), mu, dt, gamma, C.byref(options),
                           C.c_void_p(s.cuda_stream), C.byref(h)), "stokes_setup")
    return h


def stokes_solve(ctx, f: torch.Tensor, g: torch.Tensor | None, tol: float, u: torch.Tensor,
                 p: torch.Tensor, allow_not_converged: bool = False) -> StokesInfo:
    info = StokesInfo()
    _check(_L.stokes_solve(ctx, _ptr(f), _ptr(g), tol, _ptr(u), _ptr(p), C.byref(info)),
           "stokes_solve", allow=(-4,) if allow_not_converged else ())
    return info


def stokes_solve_multi(ctx, f: torch.Tensor, g: torch.Tensor | None, tol: float, u: torch.Tensor,
                       p: torch.Tensor, allow_not_converged: bool = False) -> list:
    """k systems with one operator: f [k, (2n+1)^3, 3], g [k, (n+1)^3] or None,
    u like f, p [k, (n+1)^3] (all device, FP64, contiguous). Returns k infos."""
    k = int(f.shape[0])
    infos = (StokesInfo * k)()
    _check(_L.stokes_solve_multi(ctx, k, _ptr(f), _ptr(g), tol, _ptr(u), _ptr(p), infos),
           "stokes_solve_multi", allow=(-4,) if allow_not_converged else ())
    return list(infos)


def stokes_solve_host(ctx, f: np.ndarray, g: np.ndarray | None, tol: float, u: np.ndarray,
                      p: np.ndarray) -> StokesInfo:
    info = StokesInfo()
    _check(_L.stokes_solve_host(ctx, _ptr(f), _ptr(g), tol, _ptr(u), _ptr(p), C.byref(info)),
           "stokes_solve_host")
    return info


def stokes_adjoint(ctx, dJdu, dJdp, tol, dJdf, dJdg=None):
    info = StokesInfo()
    dmu = C.c_double(0.0)
    _check(_L.stokes_adjoint(ctx, _ptr(dJdu), _ptr(dJdp), tol, _ptr(dJdf), _ptr(dJdg),
                             C.byref(dmu), C.byref(info)), "stokes_adjoint")
    return dmu.value, info


def stokes_destroy(ctx):
    if ctx:
        _L.stokes_destroy(ctx)


def stokes_apply(ctx, op: int, x: torch.Tensor, y: torch.Tensor, level: int = 0):
    _check(_L.stokes_apply(ctx, op, level, _ptr(x), _ptr(y)), "stokes_apply")
    return y


def stokes_apply_agamma_noalloc(ctx, x: torch.Tensor, y: torch.Tensor):
    """A_gamma x through the allocation-free entry point (fixed work array)."""
    _check(_L.stokes_apply_agamma_noalloc(ctx, _ptr(x), _ptr(y)), "stokes_apply_agamma_noalloc")
    return y


def stokes_sizes(ctx) -> dict:
    s = (C.c_int64 * 6)()
    _check(_L.stokes_sizes(ctx, s), "stokes_sizes")
    return dict(n=s[0], levels=s[1], n_inner=s[2], n_p1=s[3], n_p2=s[4], dofs=s[5])


def stokes_matrix_export(ctx, which: int, level: int = 0):
    """(rowptr, colidx, vals[nnz, br, bc], (rows, cols)) of an assembled matrix."""
    d = (C.c_int64 * 5)()
    _check(_L.stokes_matrix_shape(ctx, which, level, d), "stokes_matrix_shape")
    rows, cols, nnz, br, bc = (int(x) for x in d)
    if which == MAT["LUMPED"]:
        vals = np.zeros(rows)
        _check(_L.stokes_matrix_export(ctx, which, level, None, None, _ptr(vals)),
               "stokes_matrix_export")
        return None, None, vals, (rows, cols)
    rp = np.zeros(rows + 1, np.int32)
    ci = np.zeros(max(nnz, 1), np.int32)
    vals = np.zeros(max(nnz, 1) * br * bc)
    _check(_L.stokes_matrix_export(ctx, which, level, _ptr(rp), _ptr(ci), _ptr(vals)),
           "stokes_matrix_export")
    return rp, ci[:nnz], vals[: nnz * br * bc].reshape(nnz, br, bc), (rows, cols)


def stokes_kernel_stats(ctx, kernel: int):
    n = C.c_int64(0)
    ms = C.c_double(0)
    by = C.c_double(0)
    _check(_L.stokes_kernel_stats(ctx, kernel, C.byref(n), C.byref(ms), C.byref(by)),
           "stokes_kernel_stats")
    return int(n.value), float(ms.value), float(by.value)


def stokes_kernel_timing(ctx, kernel: int):
    """(timed launches, their CUDA-event ms, their algorithmic bytes)."""
    n = C.c_int64(0)
    ms = C.c_double(0)
    by = C.c_double(0)
    _check(_L.stokes_kernel_timing(ctx, kernel, C.byref(n), C.byref(ms), C.byref(by)), "stokes_kernel_timing")
    return int(n.value), float(ms.value), float(by.value)


def stokes_kernel_stats_reset(ctx):
    _check(_L.stokes_kernel_stats_reset(ctx), "stokes_kernel_stats_reset")


def stokes_profile_mode(ctx, mode: int):
    _check(_L.stokes_profile_mode(ctx, mode), "stokes_profile_mode")


def stokes_setup_phases(ctx) -> dict:
    """Milliseconds stokes_setup spent per phase (host clock)."""
    ms = (C.c_double * len(_lib.SETUP_PHASES))()
    _check(_L.stokes_setup_phases(ctx, ms), "stokes_setup_phases")
    return {name: float(ms[k]) for k, name in enumerate(_lib.SETUP_PHASES)}


class Stokes:
    """Owning wrapper: one mesh, one (mu, dt, gamma), reusable across solves."""

    def __init__(self, n: int, vertices, mu: float, dt: float, gamma: float = 0.0,
                 options: StokesOptions | None = None, device: str | torch.device = "cuda",
                 stream: torch.cuda.Stream | None = None):
        self.n, self.mu, self.dt, self.gamma = n, mu, dt, gamma
        self.device = torch.device(device)
        with torch.cuda.device(self.device):
            self.options = options if options is not None else stokes_default_options()
            self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
            self.ctx = stokes_setup(n, vertices, mu, dt, gamma, self.options, self.stream)
        self.sizes = stokes_sizes(self.ctx)

    def close(self):
        if getattr(self, "ctx", None):
            stokes_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def n_p2(self):
        return self.sizes["n_p2"]

    @property
    def n_p1(self):
        return self.sizes["n_p1"]

    def solve(self, f: torch.Tensor, g: torch.Tensor | None = None, tol: float = 1e-8,
              out=None, allow_not_converged=False):
        f = f.to(self.device, torch.float64).contiguous().reshape(self.n_p2, 3)
        if g is not None:
            g = g.to(self.device, torch.float64).contiguous()
        if out is None:
            u = torch.empty_like(f)
            p = torch.empty(self.n_p1, dtype=torch.float64, device=self.device)
        else:
            u, p = out
        info = stokes_solve(self.ctx, f, g, tol, u, p, allow_not_converged)
        return u, p, info

    def solve_multi(self, F: torch.Tensor, G: torch.Tensor | None = None, tol: float = 1e-8,
                    out=None, allow_not_converged=False):
        """k right-hand sides at once: F [k, (2n+1)^3, 3], G [k, (n+1)^3] or
        None. Returns (U [k, (2n+1)^3, 3], P [k, (n+1)^3], infos)."""
        F = F.to(self.device, torch.float64).contiguous().reshape(-1, self.n_p2, 3)
        k = F.shape[0]
        if G is not None:
            G = G.to(self.device, torch.float64).contiguous().reshape(k, self.n_p1)
        if out is None:
            U = torch.empty_like(F)
            P = torch.empty(k, self.n_p1, dtype=torch.float64, device=self.device)
        else:
            U, P = out
        infos = stokes_solve_multi(self.ctx, F, G, tol, U, P, allow_not_converged)
        return U, P, infos

    def solve_host(self, f: np.ndarray, g: np.ndarray | None = None, tol: float = 1e-8):
        f = np.ascontiguousarray(f, dtype=np.float64).reshape(self.n_p2, 3)
        u = np.empty_like(f)
        p = np.empty(self.n_p1)
        if g is not None:
            g = np.ascontiguousarray(g, dtype=np.float64)
        info = stokes_solve_host(self.ctx, f, g, tol, u, p)
        return u, p, info

    def adjoint(self, dJdu: torch.Tensor, dJdp: torch.Tensor | None = None, tol: float = 1e-10):
        dJdu = dJdu.to(self.device, torch.float64).contiguous()
        if dJdp is not None:
            dJdp = dJdp.to(self.device, torch.float64).contiguous()
        dJdf = torch.empty(self.n_p2, 3, dtype=torch.float64, device=self.device)
        dJdg = torch.empty(self.n_p1, dtype=torch.float64, device=self.device)
        dmu, info = stokes_adjoint(self.ctx, dJdu, dJdp, tol, dJdf, dJdg)
        return dJdf, dJdg, dmu, info

    def apply(self, op: str, x: torch.Tensor, out_len: int, level: int = 0) -> torch.Tensor:
        y = torch.zeros(out_len, dtype=torch.float64, device=self.device)
        stokes_apply(self.ctx, OP[op], x.contiguous(), y, level)
        return y

    def matrix(self, which: str, level: int = 0):
        return stokes_matrix_export(self.ctx, MAT[which], level)

    def kernel_stats(self, kernel: str):
        return stokes_kernel_stats(self.ctx, KERNEL[kernel])


class StokesBatch:
    """Many independent instances of uneven size solved concurrently.

    Each instance has its own context and CUDA stream; ``solve_all`` issues
    every instance's right-hand sides from its own host thread (the C calls
    release the GIL), so the kernels of all instances overlap on the GPU.
    With ``multi`` (the default) an instance's right-hand sides go through one
    ``stokes_solve_multi`` call (Method 2: four systems in lockstep, every
    matrix sweep shared); otherwise they are solved one after another.
    """

    def __init__(self, instances, options: StokesOptions | None = None,
                 device: str | torch.device = "cuda", multi: bool = True, host_wait: int | None = None):
        self.device = torch.device(device)
        self.multi = multi
        options = StokesOptions.from_buffer_copy(options) if options is not None else stokes_default_options()
        # many solver threads waiting at once: sleep on blocking-sync events
        # rather than spin (unless the caller chose)
        options.host_wait = host_wait if host_wait is not None else (1 if len(instances) > 1 else options.host_wait)
        self.solvers = []
        for (n, vertices, mu, dt, gamma) in instances:
            st = torch.cuda.Stream(self.device)
            self.solvers.append(Stokes(n, vertices, mu, dt, gamma, options, self.device, st))

    def close(self):
        for S in self.solvers:
            S.close()

    @property
    def dofs(self):
        return [S.sizes["dofs"] for S in self.solvers]

    def stack(self, forces):
        """forces[i] (a list of [(2n_i+1)^3, 3] tensors, or one [k, (2n_i+1)^3, 3]
        tensor) -> one contiguous FP64 device tensor per instance."""
        out = []
        for S, fl in zip(self.solvers, forces):
            F = fl if isinstance(fl, torch.Tensor) else torch.stack([f.reshape(S.n_p2, 3) for f in fl])
            out.append(F.to(self.device, torch.float64).contiguous())
        return out

    def solve_all(self, forces, tol: float = 1e-8, outs=None):
        """forces[i]: list of device tensors [(2n_i+1)^3, 3] (or one stacked
        [k, (2n_i+1)^3, 3] tensor) for instance i. Returns (outs, infos,
        device_ms): outs[i][k] = (u, p)."""
        import concurrent.futures as cf
        F = self.stack(forces)
        if outs is None:
            outs = []
            for S, Fi in zip(self.solvers, F):
                U = torch.empty_like(Fi)
                P = torch.empty(Fi.shape[0], S.n_p1, dtype=torch.float64, device=self.device)
                outs.append([(U[k], P[k]) for k in range(Fi.shape[0])])
        start = torch.cuda.Event(enable_timing=True)
        ends = [torch.cuda.Event(enable_timing=True) for _ in self.solvers]
        launch = torch.cuda.current_stream(self.device)
        start.record(launch)
        for S in self.solvers:
            S.stream.wait_event(start)
        infos = [None] * len(self.solvers)

        def run(i):
            S = self.solvers[i]
            u0, p0 = outs[i][0]
            k = len(outs[i])
            stacked = (all(u.data_ptr() == u0.data_ptr() + j * u0.numel() * 8 for j, (u, _) in enumerate(outs[i]))
                       and all(p.data_ptr() == p0.data_ptr() + j * p0.numel() * 8 for j, (_, p) in enumerate(outs[i])))
            if self.multi and stacked:
                U = torch.as_strided(u0, (k, S.n_p2, 3), (S.n_p2 * 3, 3, 1))
                P = torch.as_strided(p0, (k, S.n_p1), (S.n_p1, 1))
                res = [x.as_dict() for x in stokes_solve_multi(S.ctx, F[i], None, tol, U, P)]
            else:
                res = [stokes_solve(S.ctx, F[i][j], None, tol, u, p).as_dict() for j, (u, p) in enumerate(outs[i])]
            ends[i].record(S.stream)
            infos[i] = res

        with cf.ThreadPoolExecutor(max_workers=len(self.solvers)) as ex:
            list(ex.map(run, range(len(self.solvers))))
        torch.cuda.synchronize(self.device)
        ms = max(start.elapsed_time(e) for e in ends)
        return outs, infos, ms


class StokesSolve(torch.autograd.Function):
    """u, p = StokesSolve.apply(solver, f, mu_tensor, tol): forward solve, and a
    hand-written adjoint for backward giving dJ/df and dJ/dmu (the solver's mu is
    fixed at setup; mu_tensor only carries the gradient)."""

    @staticmethod
    def forward(ctx, solver: Stokes, f: torch.Tensor, mu: torch.Tensor, tol: float = 1e-10):
        u, p, info = solver.solve(f, None, tol)
        ctx.solver = solver
        ctx.tol = tol
        return u, p

    @staticmethod
    def backward(ctx, gu, gp):
        solver = ctx.solver
        gu = torch.zeros(solver.n_p2, 3, dtype=torch.float64, device=solver.device) if gu is None else gu
        dJdf, dJdg, dmu, info = solver.adjoint(gu, gp, ctx.tol)
        return None, dJdf, torch.tensor(dmu, dtype=torch.float64, device=solver.device), None
