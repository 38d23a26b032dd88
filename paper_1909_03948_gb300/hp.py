"""ctypes binding of libhp.so (include/hp.h).

Argument marshalling only: every numerical step runs in the library's CUDA
kernels.  Blocks of vectors are torch tensors of shape (s, n), float64,
contiguous, on the CUDA device -- i.e. column-major n x s with leading
dimension n, one column per row of the tensor.  A 1-D tensor of length n is a
block of one column.  PyTorch only provides device memory and streams.

There is no fallback: if libhp.so is missing or fails to load, or a tensor is
not a CUDA float64 tensor, the call raises.
"""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass

import numpy as np
import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libhp.so")

HP_OK = 0
HP_ERR_INVALID = -1
HP_ERR_NOT_CONVERGED = -2
HP_ERR_NONFINITE = -3
HP_ERR_CUDA = -4
HP_ERR_NOMEM = -5
HP_ERR_STATE = -6
HP_FP64_PLAIN = 0
HP_FP32_IR = 1
HP_MISFIT_ONLY = 0
HP_WITH_PRIOR = 1
HP_FULL_NEWTON = 2


class HPError(RuntimeError):
    def __init__(self, code, where, detail):
        super().__init__(f"{where}: {detail} (status {code})")
        self.code = code


class Desc(C.Structure):
    _fields_ = [("dim", C.c_int), ("N", C.c_int), ("gamma", C.c_double), ("delta", C.c_double),
                ("sigma", C.c_double), ("nobs", C.c_int), ("obs_xyz", C.POINTER(C.c_double)),
                ("d_obs", C.POINTER(C.c_double)), ("m_prior", C.POINTER(C.c_double)),
                ("f", C.POINTER(C.c_double)), ("u_top", C.c_double), ("u_bottom", C.c_double),
                ("precision", C.c_int), ("rtol", C.c_double), ("max_iter", C.c_int),
                ("theta", C.c_double * 6), ("robin_beta", C.c_double)]


class SolveStats(C.Structure):
    _fields_ = [("iterations", C.c_int), ("outer", C.c_int), ("solves", C.c_int), ("rel_res", C.c_double)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class Tuning(C.Structure):
    _fields_ = [("nu", C.c_int), ("nu_coarse", C.c_int), ("omega", C.c_double), ("col_chunk", C.c_int), ("max_blocks", C.c_int),
                ("smoother", C.c_int), ("cheb_alpha", C.c_double), ("fuse_transfer", C.c_int),
                ("fuse_from", C.c_int), ("tma_tiles", C.c_int), ("smem_tail", C.c_int), ("refine_df", C.c_int)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class NewtonOpts(C.Structure):
    _fields_ = [("rel_tol", C.c_double), ("abs_tol", C.c_double), ("max_iter", C.c_int),
                ("max_backtrack", C.c_int), ("c_armijo", C.c_double), ("cg_max_iter", C.c_int),
                ("full_newton", C.c_int), ("lowrank_k", C.c_int), ("lowrank_p", C.c_int),
                ("lowrank_refresh", C.c_int), ("prec_rtol", C.c_double)]


class NewtonStats(C.Structure):
    _fields_ = [("iterations", C.c_int), ("cg_iterations", C.c_int), ("converged", C.c_int),
                ("J0", C.c_double), ("J", C.c_double), ("gnorm0", C.c_double), ("gnorm", C.c_double),
                ("pde_solves", C.c_int), ("eig_solves", C.c_int)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


_lib = None
_P = C.c_void_p
_D = C.c_void_p     # device pointer
_I = C.c_int

_SIGS = {
    "hp_problem_create": (_I, [C.POINTER(Desc), C.POINTER(C.c_void_p)]),
    "hp_problem_destroy": (None, [_P]),
    "hp_set_stream": (_I, [_P, C.c_void_p]),
    "hp_set_precision": (_I, [_P, _I]),
    "hp_set_tolerance": (_I, [_P, C.c_double, _I]),
    "hp_set_data": (_I, [_P, C.POINTER(C.c_double), C.c_double]),
    "hp_get_data": (_I, [_P, C.POINTER(C.c_double)]),
    "hp_num_nodes": (_I, [_P]),
    "hp_num_elements": (_I, [_P]),
    "hp_set_point": (_I, [_P, _D, C.POINTER(C.c_double)]),
    "hp_forward": (_I, [_P, _D, _D, C.POINTER(SolveStats)]),
    "hp_observe": (_I, [_P, _D, _D]),
    "hp_gradient": (_I, [_P, _D, _D, C.POINTER(C.c_double)]),
    "hp_hessian_apply": (_I, [_P, _D, _I, _D, _I, _I, _I, C.POINTER(SolveStats)]),
    "hp_stiffness_apply": (_I, [_P, _D, _I, _D, _I, _I]),
    "hp_state_solve": (_I, [_P, _D, _I, _D, _I, _I, C.POINTER(SolveStats)]),
    "hp_C_apply": (_I, [_P, _D, _I, _D, _I, _I]),
    "hp_Ct_apply": (_I, [_P, _D, _I, _D, _I, _I]),
    "hp_prior_apply": (_I, [_P, _D, _I, _D, _I, _I]),
    "hp_mass_apply": (_I, [_P, _D, _I, _D, _I, _I]),
    "hp_prior_solve": (_I, [_P, _D, _I, _D, _I, _I, C.POINTER(SolveStats)]),
    "hp_mass_solve": (_I, [_P, _D, _I, _D, _I, _I, C.POINTER(SolveStats)]),
    "hp_mass_solve_noalloc": (_I, [_P, _D, _I, _D, _I, _I, C.POINTER(SolveStats)]),
    "hp_R_apply": (_I, [_P, _D, _I, _D, _I, _I]),
    "hp_Rinv_apply": (_I, [_P, _D, _I, _D, _I, _I]),
    "hp_mass_factor_apply": (_I, [_P, _D, _I, _D, _I, _I]),
    "hp_newton_cg_map": (_I, [_P, _D, C.POINTER(NewtonOpts), C.POINTER(NewtonStats)]),
    "hp_lowrank_eig": (_I, [_P, _D, _I, _I, _D, _I, _D, _D, _I, _I, C.POINTER(SolveStats)]),
    "hp_laplace_sample": (_I, [_P, _D, _D, _D, _I, _I, _D, _I, C.c_ulonglong, _I, _D, _D, _I,
                               C.POINTER(SolveStats)]),
    "hp_philox_normals": (_I, [C.c_ulonglong, C.c_longlong, _I, _I, _D, _I, _I, C.c_void_p]),
    "hp_pointwise_variance": (_I, [_P, _I, _D, _I, _I, _D, _D, _I, _I, _D, _D, C.POINTER(SolveStats)]),
    "hp_profile_enable": (_I, [_P, _I]),
    "hp_profile_read": (_I, [_P, _I, C.POINTER(C.c_int), C.POINTER(C.c_double)]),
    "hp_replay_kernel": (_I, [_P, _I, _I, C.c_void_p, C.c_size_t, C.POINTER(C.c_double), C.POINTER(C.c_double)]),
    "hp_replay_kernel_graph": (_I, [_P, _I, _I, C.POINTER(C.c_double)]),
    "hp_batch_create": (_I, [C.POINTER(C.c_void_p), _I, _I, C.POINTER(C.c_void_p)]),
    "hp_batch_destroy": (None, [C.c_void_p]),
    "hp_batch_set_point": (_I, [C.c_void_p, C.POINTER(C.c_void_p), C.POINTER(C.c_int)]),
    "hp_batch_map_and_eig": (_I, [C.c_void_p, C.POINTER(C.c_void_p), C.POINTER(NewtonOpts), _I, _I,
                                  C.POINTER(C.c_void_p), C.POINTER(C.c_int), C.POINTER(C.c_void_p),
                                  C.POINTER(C.c_void_p), C.POINTER(C.c_int), C.POINTER(NewtonStats),
                                  C.POINTER(C.c_int)]),
    "hp_batch_hessian_apply": (_I, [C.c_void_p, C.POINTER(C.c_void_p), C.POINTER(C.c_int), C.POINTER(C.c_void_p),
                                    C.POINTER(C.c_int), C.POINTER(C.c_int), _I, C.POINTER(C.c_int)]),
    "hp_set_tuning": (_I, [_P, C.POINTER(Tuning)]),
    "hp_get_tuning": (_I, [_P, C.POINTER(Tuning)]),
    "hp_autotune": (_I, [_P, _I, _I, C.POINTER(Tuning), C.POINTER(C.c_double)]),
    "hp_autotune_block": (_I, [_P, _D, _I, _I, _I, C.POINTER(Tuning), C.POINTER(C.c_double)]),
    "hp_unet_create": (_I, [_I, _I, _I, C.POINTER(C.c_void_p)]),
    "hp_unet_destroy": (None, [C.c_void_p]),
    "hp_unet_num_params": (C.c_long, [C.c_void_p]),
    "hp_unet_set_params": (_I, [C.c_void_p, C.POINTER(C.c_float)]),
    "hp_unet_get_params": (_I, [C.c_void_p, C.POINTER(C.c_float)]),
    "hp_unet_forward": (_I, [C.c_void_p, _D, _I, _D]),
    "hp_unet_loss_grad": (_I, [C.c_void_p, _D, _D, _I, C.POINTER(C.c_double), C.POINTER(C.c_float)]),
    "hp_unet_train": (_I, [C.c_void_p, _D, _D, _I, _I, _I, C.c_double, C.c_ulonglong, C.POINTER(C.c_double)]),
    "hp_unet_set_tensor_cores": (_I, [C.c_void_p, _I]),
    "hp_unet_get_tensor_cores": (_I, [C.c_void_p]),
    "hp_warmstart_grid": (_I, [_P, C.POINTER(C.c_int), C.POINTER(C.c_int)]),
    "hp_warmstart_attach": (_I, [_P, C.c_void_p]),
    "hp_warmstart_enable": (_I, [_P, _I]),
    "hp_warmstart_record": (_I, [_P, _D, _D, _D, _I]),
    "hp_warmstart_counts": (_I, [_P, C.POINTER(C.c_longlong), C.POINTER(C.c_longlong),
                                 C.POINTER(C.c_longlong)]),
    "hp_status_string": (C.c_char_p, [_I]),
    "hp_last_error": (C.c_char_p, []),
    "hp_kernel_launches": (C.c_ulonglong, []),
    "hp_tiled_kernel_launches": (C.c_ulonglong, []),
    "hp_algorithmic_bytes": (_I, [C.POINTER(C.c_double), _I]),
}

EXPORTED = tuple(_SIGS)


def lib():
    """Load libhp.so (raises if it is missing: there is no fallback path)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} not found: build it with `python -m paper_1909_03948_gb300.build`")
        L = C.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def kernel_launches() -> int:
    return int(lib().hp_kernel_launches())


def tiled_kernel_launches() -> int:
    """Launches of the TMA-tiled stencil kernels since the library was loaded."""
    return int(lib().hp_tiled_kernel_launches())


BYTES_FAMILIES = ("stencil_level0", "stencil_coarse", "transfer", "vector", "refine64", "C_Ct_obs")


def algorithmic_bytes() -> dict:
    """Cumulative algorithmic DRAM bytes of direct launches since load, by kernel family
    (launches inside CUDA graphs are not counted: measure with profiling on)."""
    out = (C.c_double * len(BYTES_FAMILIES))()
    _check(lib().hp_algorithmic_bytes(out, len(BYTES_FAMILIES)), "hp_algorithmic_bytes")
    return dict(zip(BYTES_FAMILIES, [float(v) for v in out]))


def _check(code, where):
    if code != HP_OK:
        L = lib()
        raise HPError(code, where, L.hp_last_error().decode() or L.hp_status_string(code).decode())


def _dptr(t: torch.Tensor):
    return C.c_void_p(t.data_ptr())


def _block(t: torch.Tensor, n: int, name: str):
    """(s, n) or (n,) CUDA float64 contiguous -> (tensor2d, s, ld)."""
    if not isinstance(t, torch.Tensor) or not t.is_cuda or t.dtype != torch.float64:
        raise TypeError(f"{name}: expected a CUDA float64 tensor")
    t2 = t.reshape(1, -1) if t.dim() == 1 else t
    if t2.dim() != 2 or t2.shape[1] != n or not t2.is_contiguous():
        raise ValueError(f"{name}: expected a contiguous (s, {n}) block")
    return t2, t2.shape[0], n


def _hptr(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


@dataclass
class Stats:
    iterations: int = 0
    outer: int = 0
    solves: int = 0
    rel_res: float = 0.0


class Problem:
    """One inverse problem instance (owns an hp_problem handle)."""

    def __init__(self, dim: int, N: int, gamma: float, delta: float, sigma: float, obs_xyz,
                 d_obs=None, m_prior=None, f=None, u_top: float = 1.0, u_bottom: float = 0.0,
                 precision: str = "fp32_ir", rtol: float = 1e-8, max_iter: int = 500,
                 theta=None, robin_beta: float = 0.0):
        """theta: the prior's s.p.d. anisotropy tensor (dim x dim; None = identity);
        robin_beta: Robin coefficient of the prior's boundary condition (0 = Neumann)."""
        L = lib()
        self._keep = []
        obs = np.ascontiguousarray(np.asarray(obs_xyz, dtype=np.float64).reshape(-1, dim))
        self._keep.append(obs)

        def opt(a, length):
            if a is None:
                return None
            a = np.ascontiguousarray(np.asarray(a, dtype=np.float64).reshape(-1))
            if a.size != length:
                raise ValueError("wrong length")
            self._keep.append(a)
            return _hptr(a)

        n = (N + 1) ** dim
        d = Desc(dim=dim, N=N, gamma=gamma, delta=delta, sigma=sigma, nobs=obs.shape[0],
                 obs_xyz=_hptr(obs) if obs.size else None, d_obs=opt(d_obs, obs.shape[0]),
                 m_prior=opt(m_prior, n), f=opt(f, n), u_top=u_top, u_bottom=u_bottom,
                 precision=HP_FP32_IR if precision == "fp32_ir" else HP_FP64_PLAIN,
                 rtol=rtol, max_iter=max_iter, robin_beta=robin_beta)
        if theta is not None:
            Th = np.asarray(theta, dtype=np.float64).reshape(dim, dim)
            t6 = [Th[0, 0], Th[1, 1], Th[2, 2] if dim == 3 else 0.0, Th[0, 1],
                  Th[0, 2] if dim == 3 else 0.0, Th[1, 2] if dim == 3 else 0.0]
            for q in range(6):
                d.theta[q] = float(t6[q])
        h = C.c_void_p()
        _check(L.hp_problem_create(C.byref(d), C.byref(h)), "hp_problem_create")
        self._h = h
        self.dim, self.N = dim, N
        self.n = L.hp_num_nodes(h)
        self.nelems = L.hp_num_elements(h)
        self.nobs = obs.shape[0]
        self.device = torch.device("cuda", torch.cuda.current_device())

    def close(self):
        if getattr(self, "_h", None):
            lib().hp_problem_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ---- configuration ----------------------------------------------------
    def set_stream(self, stream=None):
        ptr = None if stream is None else C.c_void_p(stream.cuda_stream)
        _check(lib().hp_set_stream(self._h, ptr), "hp_set_stream")

    def set_precision(self, precision: str):
        _check(lib().hp_set_precision(self._h, HP_FP32_IR if precision == "fp32_ir" else HP_FP64_PLAIN),
               "hp_set_precision")

    def set_tolerance(self, rtol: float, max_iter: int = 500):
        _check(lib().hp_set_tolerance(self._h, rtol, max_iter), "hp_set_tolerance")

    def set_data(self, d_obs, sigma: float):
        a = np.ascontiguousarray(np.asarray(d_obs, dtype=np.float64))
        _check(lib().hp_set_data(self._h, _hptr(a), sigma), "hp_set_data")

    def get_data(self):
        out = np.zeros(self.nobs)
        _check(lib().hp_get_data(self._h, _hptr(out)), "hp_get_data")
        return out

    # ---- helpers -------------------------------------------------------------
    def zeros(self, s=None):
        return torch.zeros((self.n,) if s is None else (s, self.n), dtype=torch.float64, device=self.device)

    def _vec(self, t, name):
        t2, s, _ = _block(t, self.n, name)
        if s != 1:
            raise ValueError(f"{name}: expected a single vector")
        return t2

    # ---- forward / cost / gradient -------------------------------------------
    def set_point(self, m):
        m = self._vec(m, "m")
        J = (C.c_double * 3)()
        _check(lib().hp_set_point(self._h, _dptr(m), J), "hp_set_point")
        return tuple(J)

    def forward(self, m):
        m = self._vec(m, "m")
        u = self.zeros()
        st = SolveStats()
        _check(lib().hp_forward(self._h, _dptr(m), _dptr(u), C.byref(st)), "hp_forward")
        return u, st.as_dict()

    def observe(self, u):
        u = self._vec(u, "u")
        y = torch.zeros(max(self.nobs, 1), dtype=torch.float64, device=self.device)
        _check(lib().hp_observe(self._h, _dptr(u), _dptr(y)), "hp_observe")
        return y[: self.nobs]

    def gradient(self, m):
        m = self._vec(m, "m")
        g = self.zeros()
        J = (C.c_double * 3)()
        _check(lib().hp_gradient(self._h, _dptr(m), _dptr(g), J), "hp_gradient")
        return g, tuple(J)

    # ---- learned warm start (2D) ------------------------------------------------
    def warmstart_grid(self):
        H, W = C.c_int(), C.c_int()
        _check(lib().hp_warmstart_grid(self._h, C.byref(H), C.byref(W)), "hp_warmstart_grid")
        return H.value, W.value

    def warmstart_attach(self, net):
        """Start every stiffness solve from `net`'s guess (None detaches)."""
        _check(lib().hp_warmstart_attach(self._h, net._h if net is not None else None), "hp_warmstart_attach")
        self._ws_net = net   # keeps the network alive while attached

    def warmstart_enable(self, on: bool = True):
        _check(lib().hp_warmstart_enable(self._h, 1 if on else 0), "hp_warmstart_enable")

    def warmstart_record(self, X=None, A=None, T=None):
        """Record the following stiffness solves: inputs into X (cap,3,H,W), loss data into
        A (cap,4,H,W), solutions (optional) into T (cap,1,H,W), CUDA float32; no arguments
        stops recording."""
        if X is None:
            _check(lib().hp_warmstart_record(self._h, None, None, None, 0), "hp_warmstart_record")
            self._ws_rec = None
            return
        H, W = self.warmstart_grid()
        cap = X.shape[0]
        for t, c, nm in ((X, 3, "X"), (A, 4, "A"), (T, 1, "T")):
            if nm == "T" and t is None:
                continue
            if (not t.is_cuda or t.dtype != torch.float32 or not t.is_contiguous()
                    or tuple(t.shape) != (cap, c, H, W)):
                raise ValueError(f"{nm}: expected a contiguous CUDA float32 tensor of shape {(cap, c, H, W)}")
        _check(lib().hp_warmstart_record(self._h, _dptr(X), _dptr(A), _dptr(T) if T is not None else None, cap),
               "hp_warmstart_record")
        self._ws_rec = (X, A, T)

    def warmstart_counts(self):
        r, g, f = C.c_longlong(), C.c_longlong(), C.c_longlong()
        _check(lib().hp_warmstart_counts(self._h, C.byref(r), C.byref(g), C.byref(f)), "hp_warmstart_counts")
        return {"recorded": r.value, "guesses": g.value, "fallbacks": f.value}

    # ---- Hessian / operators --------------------------------------------------
    def hessian_apply(self, X, with_prior: bool = False, out=None, full: bool = False):
        """Gauss-Newton (default) or full (full=True: with the adjoint terms) Hessian action."""
        X2, s, n = _block(X, self.n, "X")
        Y = torch.empty_like(X2) if out is None else _block(out, self.n, "out")[0]
        st = SolveStats()
        flags = (HP_WITH_PRIOR if with_prior else HP_MISFIT_ONLY) | (HP_FULL_NEWTON if full else 0)
        _check(lib().hp_hessian_apply(self._h, _dptr(X2), n, _dptr(Y), n, s, flags, C.byref(st)),
               "hp_hessian_apply")
        return (Y.reshape(X.shape) if out is None else out), st.as_dict()

    def _unary(self, fname, X, with_stats=False):
        X2, s, n = _block(X, self.n, "X")
        Y = torch.empty_like(X2)
        if with_stats:
            st = SolveStats()
            _check(getattr(lib(), fname)(self._h, _dptr(X2), n, _dptr(Y), n, s, C.byref(st)), fname)
            return Y.reshape(X.shape), st.as_dict()
        _check(getattr(lib(), fname)(self._h, _dptr(X2), n, _dptr(Y), n, s), fname)
        return Y.reshape(X.shape)

    def stiffness_apply(self, X):
        return self._unary("hp_stiffness_apply", X)

    def state_solve(self, B):
        return self._unary("hp_state_solve", B, True)

    def C_apply(self, X):
        return self._unary("hp_C_apply", X)

    def Ct_apply(self, W):
        return self._unary("hp_Ct_apply", W)

    def prior_apply(self, X):
        return self._unary("hp_prior_apply", X)

    def mass_apply(self, X):
        return self._unary("hp_mass_apply", X)

    def prior_solve(self, B):
        return self._unary("hp_prior_solve", B, True)

    def mass_solve(self, B):
        return self._unary("hp_mass_solve", B, True)

    def mass_solve_noalloc(self, B, out):
        """X = M^{-1} B without any device allocation by the library: the caller
        provides the output block and the library uses a fixed device scratch array
        (nrhs <= 64, n * nrhs <= 262144; calls must not overlap on the GPU)."""
        B2, s, n = _block(B, self.n, "B")
        X2 = _block(out, self.n, "out")[0]
        # the library writes s columns of n values into out: it must hold exactly B's block
        if X2.shape != B2.shape or X2.device != B2.device:
            raise ValueError(f"out: expected a {tuple(B2.shape)} block on {B2.device}, got "
                             f"{tuple(X2.shape)} on {X2.device}")
        st = SolveStats()
        _check(lib().hp_mass_solve_noalloc(self._h, _dptr(B2), n, _dptr(X2), n, s, C.byref(st)),
               "hp_mass_solve_noalloc")
        return out, st.as_dict()

    def R_apply(self, X):
        return self._unary("hp_R_apply", X)

    def Rinv_apply(self, X):
        return self._unary("hp_Rinv_apply", X)

    def mass_factor_apply(self, eta):
        ne = self.nelems * (self.dim + 1)
        E2, s, _ = _block(eta, ne, "eta")
        W = torch.empty((s, self.n), dtype=torch.float64, device=self.device)
        _check(lib().hp_mass_factor_apply(self._h, _dptr(E2), ne, _dptr(W), self.n, s), "hp_mass_factor_apply")
        return W if eta.dim() == 2 else W[0]

    # ---- tuning ------------------------------------------------------------------
    def get_tuning(self):
        t = Tuning()
        _check(lib().hp_get_tuning(self._h, C.byref(t)), "hp_get_tuning")
        return t.as_dict()

    def set_tuning(self, nu=3, omega=0.7, col_chunk=0, max_blocks=4096, smoother=1, cheb_alpha=10.0,
                   fuse_transfer=0, fuse_from=0, nu_coarse=0, tma_tiles=0, smem_tail=0, refine_df=1):
        t = Tuning(nu=nu, nu_coarse=nu_coarse, omega=omega, col_chunk=col_chunk, max_blocks=max_blocks,
                   smoother=smoother, cheb_alpha=cheb_alpha, fuse_transfer=fuse_transfer, fuse_from=fuse_from,
                   tma_tiles=tma_tiles, smem_tail=smem_tail, refine_df=refine_df)
        _check(lib().hp_set_tuning(self._h, C.byref(t)), "hp_set_tuning")

    def autotune(self, nrhs, reps=3, X=None):
        """Runs the autotuner at the current point, timing a random block of nrhs directions
        or, if X is given, the caller's block X (CUDA float64 (nrhs, n), as hessian_apply
        takes it); returns (settings, ms per block)."""
        t = Tuning()
        ms = C.c_double()
        if X is None:
            _check(lib().hp_autotune(self._h, nrhs, reps, C.byref(t), C.byref(ms)), "hp_autotune")
        else:
            X2, s, n = _block(X, self.n, "X")
            if s != nrhs:
                raise ValueError(f"X has {s} columns, nrhs is {nrhs}")
            _check(lib().hp_autotune_block(self._h, _dptr(X2), n, nrhs, reps, C.byref(t), C.byref(ms)),
                   "hp_autotune_block")
        return t.as_dict(), ms.value

    # ---- measurement -------------------------------------------------------------
    PROF_NAMES = ("matvec", "smooth", "resid_mg", "resid64", "cg_update", "vcycle", "presmooth")

    def profile_enable(self, on: bool = True):
        _check(lib().hp_profile_enable(self._h, 1 if on else 0), "hp_profile_enable")

    def profile_read(self):
        k = len(self.PROF_NAMES)
        cnt = (C.c_int * k)()
        ms = (C.c_double * k)()
        _check(lib().hp_profile_read(self._h, k, cnt, ms), "hp_profile_read")
        return {name: (cnt[i], ms[i]) for i, name in enumerate(self.PROF_NAMES)}

    REPLAY_FAMILIES = ("smooth", "resid_mg", "presmooth")

    def replay_kernel(self, family: str, reps: int, flush=None):
        """(us per launch back to back, us per launch from HBM or None) of a level-0
        kernel of the last FP32 block solve, replayed on its live workspace; `flush` is a
        CUDA tensor larger than L2 read before each cold launch."""
        w, c = C.c_double(), C.c_double()
        fam = self.REPLAY_FAMILIES.index(family)
        if flush is not None:
            _check(lib().hp_replay_kernel(self._h, fam, reps, _dptr(flush), flush.numel() * flush.element_size(),
                                          C.byref(w), C.byref(c)), "hp_replay_kernel")
            return w.value, c.value
        _check(lib().hp_replay_kernel(self._h, fam, reps, None, 0, C.byref(w), None), "hp_replay_kernel")
        return w.value, None

    def replay_kernel_graph(self, family: str, reps: int):
        """us per launch of the same level-0 kernel with reps launches captured in one
        CUDA graph (the way the solver's PCG loop runs it)."""
        us = C.c_double()
        _check(lib().hp_replay_kernel_graph(self._h, self.REPLAY_FAMILIES.index(family), reps, C.byref(us)),
               "hp_replay_kernel_graph")
        return us.value

    # ---- algorithms --------------------------------------------------------------
    def newton_cg_map(self, m0=None, rel_tol=1e-6, abs_tol=0.0, max_iter=50, max_backtrack=10,
                      c_armijo=1e-4, cg_max_iter=200, full=False, lowrank_k=0, lowrank_p=10, lowrank_refresh=0,
                      prec_rtol=0.0):
        """Algorithm 1.  lowrank_k > 0 preconditions the CG with R^-1 - V D V^T from the
        lowrank_k leading eigenpairs (recomputed every lowrank_refresh iterations, 0: once);
        prec_rtol > 0 solves the prior solves of that preconditioner to this tolerance."""
        m = self.zeros() if m0 is None else self._vec(m0, "m0").clone().reshape(-1)
        o = NewtonOpts(rel_tol, abs_tol, max_iter, max_backtrack, c_armijo, cg_max_iter, 1 if full else 0,
                       lowrank_k, lowrank_p, lowrank_refresh, prec_rtol)
        st = NewtonStats()
        rc = lib().hp_newton_cg_map(self._h, _dptr(m), C.byref(o), C.byref(st))
        if rc not in (HP_OK, HP_ERR_NOT_CONVERGED):
            _check(rc, "hp_newton_cg_map")
        return m, st.as_dict()

    def lowrank_eig(self, m_map, k, p, Omega, single_pass=False):
        m_map = self._vec(m_map, "m_map")
        O2, s, n = _block(Omega, self.n, "Omega")
        if s != k + p:
            raise ValueError("Omega must have k + p columns")
        lam = torch.zeros(k, dtype=torch.float64, device=self.device)
        V = torch.zeros((k, self.n), dtype=torch.float64, device=self.device)
        st = SolveStats()
        _check(lib().hp_lowrank_eig(self._h, _dptr(m_map), k, p, _dptr(O2), n, _dptr(lam), _dptr(V), n,
                                    1 if single_pass else 0, C.byref(st)), "hp_lowrank_eig")
        return lam, V, st.as_dict()

    VARIANCE_METHODS = ("randomized", "stochastic")

    def pointwise_variance(self, Z, method: str = "randomized", lam=None, V=None):
        """Section 4.4: (prior_var, post_var or None) as (n,) float64 tensors.  Z: (r, n)
        Gaussian columns (randomized eig of R^-1, eq. prior_mvar) or probe vectors
        (stochastic estimator); lam (k,), V (k, n): Hessian eigenpairs for eq. post_mvar."""
        Z2, r, n = _block(Z, self.n, "Z")
        prior = torch.empty(self.n, dtype=torch.float64, device=self.device)
        post = None
        k, lp, vp = 0, None, None
        if V is not None:
            V2, k, _ = _block(V, self.n, "V")
            lam = lam.contiguous()
            if lam.numel() != k or not lam.is_cuda or lam.dtype != torch.float64:
                raise ValueError("lam: k CUDA float64 values")
            post = torch.empty_like(prior)
            lp, vp = _dptr(lam), _dptr(V2)
        st = SolveStats()
        _check(lib().hp_pointwise_variance(self._h, self.VARIANCE_METHODS.index(method), _dptr(Z2), n, r, lp, vp,
                                           n, k, _dptr(prior), _dptr(post) if post is not None else None,
                                           C.byref(st)), "hp_pointwise_variance")
        return prior, post

    def laplace_sample(self, m_map, lam, V, eta=None, want_prior=True, want_post=True, seed=0, nsamples=None):
        """Prior and Laplace-posterior samples.  eta: (N, (dim+1)*nelems) normals, or None
        to draw them on the device from Philox4x32-10 with `seed` (then give nsamples)."""
        ne = self.nelems * (self.dim + 1)
        null = C.c_void_p(0)
        if eta is not None:
            E2, N, _ = _block(eta, ne, "eta")
            eptr = _dptr(E2)
        else:
            N, eptr = int(nsamples), null
        k = 0 if V is None else V.shape[0]
        prior = torch.empty((N, self.n), dtype=torch.float64, device=self.device) if want_prior else None
        post = torch.empty((N, self.n), dtype=torch.float64, device=self.device) if want_post else None
        st = SolveStats()
        _check(lib().hp_laplace_sample(
            self._h, _dptr(self._vec(m_map, "m_map")) if want_post else null,
            _dptr(lam) if want_post else null, _dptr(V) if want_post else null, self.n, k,
            eptr, ne, seed, N, _dptr(prior) if want_prior else null, _dptr(post) if want_post else null,
            self.n, C.byref(st)), "hp_laplace_sample")
        return prior, post, st.as_dict()


def philox_normals(seed: int, first_sample: int, nsamples: int, nper: int, raw: bool = False, device=None):
    """(nsamples, nper) float64 tensor of the sampler's Philox normals (or raw 32-bit words)."""
    dev = device or torch.device("cuda", torch.cuda.current_device())
    out = torch.empty((nsamples, nper), dtype=torch.float64, device=dev)
    _check(lib().hp_philox_normals(seed, first_sample, nsamples, nper, _dptr(out), nper, 1 if raw else 0, None),
           "hp_philox_normals")
    return out


class UNet:
    """The warm-start network (owns an hp_unet handle).  Parameters travel as one
    packed float32 numpy vector (per layer: weights (co, ci, k, k), then biases)."""

    def __init__(self, H: int, W: int, batch_cap: int = 16, tensor_cores: bool = True):
        h = C.c_void_p()
        _check(lib().hp_unet_create(H, W, batch_cap, C.byref(h)), "hp_unet_create")
        self._h, self.H, self.W, self.cap = h, H, W, batch_cap
        self.nparam = int(lib().hp_unet_num_params(h))
        self.tensor_cores = tensor_cores

    @property
    def tensor_cores(self) -> bool:
        """Whether the 3x3 convolutions run on the tensor cores (hp_unet_set_tensor_cores)."""
        return bool(lib().hp_unet_get_tensor_cores(self._h))

    @tensor_cores.setter
    def tensor_cores(self, on: bool):
        _check(lib().hp_unet_set_tensor_cores(self._h, int(bool(on))), "hp_unet_set_tensor_cores")

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            lib().hp_unet_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_params(self, p):
        p = np.ascontiguousarray(np.asarray(p, dtype=np.float32))
        if p.size != self.nparam:
            raise ValueError(f"expected {self.nparam} parameters, got {p.size}")
        _check(lib().hp_unet_set_params(self._h, p.ctypes.data_as(C.POINTER(C.c_float))), "hp_unet_set_params")

    def get_params(self):
        p = np.empty(self.nparam, dtype=np.float32)
        _check(lib().hp_unet_get_params(self._h, p.ctypes.data_as(C.POINTER(C.c_float))), "hp_unet_get_params")
        return p

    def _chk(self, t, c, name, N=None):
        if (not isinstance(t, torch.Tensor) or not t.is_cuda or t.dtype != torch.float32 or not t.is_contiguous()
                or t.dim() != 4 or tuple(t.shape[1:]) != (c, self.H, self.W) or (N is not None and t.shape[0] != N)):
            raise ValueError(f"{name}: expected a contiguous CUDA float32 tensor (N, {c}, {self.H}, {self.W})")
        return t.shape[0]

    def forward(self, x):
        N = self._chk(x, 3, "x")
        y = torch.empty((N, 1, self.H, self.W), dtype=torch.float32, device=x.device)
        _check(lib().hp_unet_forward(self._h, _dptr(x), N, _dptr(y)), "hp_unet_forward")
        return y

    def loss_grad(self, x, aux):
        """(loss, packed gradient) of the relative-residual loss for x (N,3,H,W), aux (N,4,H,W)."""
        N = self._chk(x, 3, "x")
        self._chk(aux, 4, "aux", N)
        L = C.c_double()
        g = np.empty(self.nparam, dtype=np.float32)
        _check(lib().hp_unet_loss_grad(self._h, _dptr(x), _dptr(aux), N, C.byref(L),
                                       g.ctypes.data_as(C.POINTER(C.c_float))), "hp_unet_loss_grad")
        return L.value, g

    def train(self, X, A, epochs: int, batch: int, lr: float = 1e-3, seed: int = 0):
        ns = self._chk(X, 3, "X")
        self._chk(A, 4, "A", ns)
        losses = np.zeros(epochs)
        _check(lib().hp_unet_train(self._h, _dptr(X), _dptr(A), ns, epochs, batch, lr, seed,
                                   losses.ctypes.data_as(C.POINTER(C.c_double))), "hp_unet_train")
        return losses


def _ptrs(ts):
    return (C.c_void_p * len(ts))(*[t.data_ptr() for t in ts])


def _ints(v):
    return (C.c_int * len(v))(*v)


class Batch:
    """Independent problems of uneven size run concurrently (one stream and one host
    worker per problem at a time).  Problems stay owned by the caller.  The streams
    share CUDA's hardware work queues: set CUDA_DEVICE_MAX_CONNECTIONS=32 in the
    environment before CUDA starts (8 otherwise; hp_batch_create in include/hp.h)."""

    def __init__(self, problems, nthreads: int = 0):
        self.problems = list(problems)
        hs = (C.c_void_p * len(self.problems))(*[p._h.value for p in self.problems])
        h = C.c_void_p()
        _check(lib().hp_batch_create(hs, len(self.problems), nthreads, C.byref(h)), "hp_batch_create")
        self._h = h

    def close(self):
        if getattr(self, "_h", None):
            lib().hp_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _status(self, rc, st, where):
        if rc != HP_OK:
            bad = [i for i, v in enumerate(st) if v != HP_OK]
            raise HPError(rc, where, f"problems {bad} failed with {[st[i] for i in bad]}")

    def set_point(self, ms):
        st = (C.c_int * len(self.problems))()
        rc = lib().hp_batch_set_point(self._h, _ptrs([m.reshape(-1) for m in ms]), st)
        self._status(rc, list(st), "hp_batch_set_point")

    def map_and_eig(self, m0s, k, p, Omegas, rel_tol=1e-6, max_iter=50):
        ms = [m.clone().reshape(-1) for m in m0s]
        lams = [torch.zeros(k, dtype=torch.float64, device=m.device) for m in ms]
        Vs = [torch.zeros((k, pr.n), dtype=torch.float64, device=m.device) for m, pr in zip(ms, self.problems)]
        o = NewtonOpts(rel_tol, 0.0, max_iter, 10, 1e-4, 200)
        nst = (NewtonStats * len(ms))()
        st = (C.c_int * len(ms))()
        ns = [pr.n for pr in self.problems]
        rc = lib().hp_batch_map_and_eig(self._h, _ptrs(ms), C.byref(o), k, p, _ptrs(Omegas), _ints(ns), _ptrs(lams),
                                        _ptrs(Vs), _ints(ns), nst, st)
        self._status(rc, list(st), "hp_batch_map_and_eig")
        return ms, lams, Vs, [x.as_dict() for x in nst]

    def hessian_apply(self, Xs, with_prior=False):
        Ys = [torch.empty_like(X) for X in Xs]
        ns = [pr.n for pr in self.problems]
        st = (C.c_int * len(Xs))()
        rc = lib().hp_batch_hessian_apply(self._h, _ptrs(Xs), _ints(ns), _ptrs(Ys), _ints(ns),
                                          _ints([X.shape[0] for X in Xs]), HP_WITH_PRIOR if with_prior else 0, st)
        self._status(rc, list(st), "hp_batch_hessian_apply")
        return Ys
