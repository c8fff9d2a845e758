"""Python binding of libfhmg (include/fhmg.h): argument marshalling only.

Every computation runs in the CUDA library; this module checks tensor shapes/dtypes, passes
``data_ptr()`` and the current CUDA stream, and turns status codes into exceptions.  It fails
loudly (ImportError / RuntimeError) when the library has not been built -- there is no CPU
fallback.

Grid functions are torch.float64 CUDA tensors of shape (M, N) (1D) or (M, N, N) (2D),
time-major with space contiguous, for t_1..t_M.
"""
from __future__ import annotations

import ctypes
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libfhmg.so")

FHMG_OK, FHMG_EINVAL, FHMG_ECUDA, FHMG_ENOMEM, FHMG_ENOTCONV, FHMG_ENAN, FHMG_ETIMEOUT = 0, -1, -2, -3, -4, -5, -6
FP64, MIXED_FP32, MIXED_BF16 = 0, 1, 2
_STATUS = {0: "FHMG_OK", -1: "FHMG_EINVAL", -2: "FHMG_ECUDA", -3: "FHMG_ENOMEM", -4: "FHMG_ENOTCONV",
           -5: "FHMG_ENAN", -6: "FHMG_ETIMEOUT"}

_lib = None

_c = ctypes
_P = _c.c_void_p
_D = _c.c_double
_I = _c.c_int
_LL = _c.c_longlong
_SIGS = {
    "fhmg_last_error": (_c.c_char_p, []),
    "fhmg_build_hmatrix": (_I, [_D, _D, _D, _I, _I, _I, _D, _c.POINTER(_P)]),
    "fhmg_build_hmatrix_aca": (_I, [_D, _D, _D, _I, _I, _D, _c.POINTER(_P)]),
    "fhmg_hmatrix_info": (_I, [_P, _c.POINTER(_I), _c.POINTER(_I), _c.POINTER(_I), _c.POINTER(_c.c_size_t)]),
    "fhmg_hmatrix_mesh": (_I, [_P, _P, _P]),
    "fhmg_hmatrix_dense": (_I, [_P, _P]),
    "fhmg_hmatrix_flops": (_I, [_P, _c.POINTER(_D)]),
    "fhmg_hmatrix_split_digits": (_I, [_P, _P, _c.POINTER(_LL), _P, _P]),
    "fhmg_autotune_hmatrix": (_I, [_D, _D, _D, _I, _I, _D, _c.POINTER(_I), _c.POINTER(_D), _c.POINTER(_D),
                                  _c.POINTER(_D)]),
    "fhmg_hmatrix_destroy": (_I, [_P]),
    "fhmg_sama_two_grid": (_I, [_P, _I, _I, _D, _I, _I, _c.POINTER(_D)]),
    "fhmg_problem_create": (_I, [_P, _I, _I, _D, _I, _P, _c.POINTER(_P)]),
    "fhmg_problem_destroy": (_I, [_P]),
    "fhmg_problem_autotune": (_I, [_P]),
    "fhmg_problem_profile": (_I, [_P, _I]),
    "fhmg_problem_set_inner": (_I, [_P, _I]),
    "fhmg_problem_set_mixed_storage": (_I, [_P, _I]),
    "fhmg_problem_counters": (_I, [_P, _c.POINTER(_LL), _c.POINTER(_LL), _c.POINTER(_D)]),
    "fhmg_problem_defect_timing": (_I, [_P, _c.POINTER(_LL), _c.POINTER(_D), _c.POINTER(_LL)]),
    "fhmg_line_solve": (_I, [_P, _I, _P, _P, _LL]),
    "fhmg_hmatvec": (_I, [_P, _P, _P, _LL]),
    "fhmg_line_solve_f32": (_I, [_P, _I, _P, _P, _LL, _I]),
    "fhmg_hmatvec_f32": (_I, [_P, _P, _P, _LL, _I]),
    "fhmg_line_solve_s": (_I, [_P, _I, _P, _P, _LL]),
    "fhmg_hmatvec_s": (_I, [_P, _P, _P, _LL]),
    "fhmg_smooth": (_I, [_P, _P, _P, _I]),
    "fhmg_residual": (_I, [_P, _P, _P, _P, _P]),
    "fhmg_restrict_residual": (_I, [_P, _P, _P, _P]),
    "fhmg_prolong_correct": (_I, [_P, _P, _P]),
    "fhmg_vcycle": (_I, [_P, _P, _P, _P, _I, _I]),
    "fhmg_residual_norm": (_I, [_P, _P, _P, _P, _c.POINTER(_D)]),
    "fhmg_residual_norm_noalloc": (_I, [_P, _P, _P, _c.POINTER(_D)]),
    "fhmg_solve": (_I, [_P, _P, _P, _P, _I, _I, _D, _I, _c.POINTER(_I), _c.POINTER(_D)]),
    "fhmg_solve_host": (_I, [_P, _P, _P, _P, _I, _I, _D, _I, _c.POINTER(_I), _c.POINTER(_D)]),
    "fhmg_solve_batched": (_I, [_I, _c.POINTER(_P), _c.POINTER(_P), _c.POINTER(_P), _I, _I, _D, _I,
                                _c.POINTER(_I), _c.POINTER(_D)]),
    "fhmg_autotune_leaf": (_I, [_D, _D, _D, _I, _D, _I, _I, _D, _I, _P, _c.POINTER(_I), _c.POINTER(_D)]),
    "fhmg_problem_set_rtol_reference": (_I, [_P, _I]),
    "fhmg_problem_set_coarse_direct": (_I, [_P, _I]),
    "fhmg_problem_set_tensor_cores": (_I, [_P, _I]),
    "fhmg_problem_set_defect_arith": (_I, [_P, _I]),
    "fhmg_problem_split_flops": (_I, [_P, ctypes.POINTER(ctypes.c_double)]),
    "fhmg_problem_set_cycle_index": (_I, [_P, _I]),
    "fhmg_problem_inject_timeout": (_I, [_P, _LL]),
    "fhmg_hmatvec_df": (_I, [_P, _P, _P, _LL, _I]),
    "fhmg_wsnet_create": (_I, [_I, _I, _c.c_ulonglong, _c.POINTER(_P)]),
    "fhmg_wsnet_destroy": (_I, [_P]),
    "fhmg_wsnet_num_params": (_I, [_P, _c.POINTER(_LL)]),
    "fhmg_wsnet_get_params": (_I, [_P, _P]),
    "fhmg_wsnet_set_params": (_I, [_P, _P]),
    "fhmg_wsnet_forward": (_I, [_P, _P, _I, _I, _P, _P]),
    "fhmg_wsnet_loss_grad": (_I, [_P, _P, _P, _I, _P, _P, _P]),
    "fhmg_wsnet_train": (_I, [_P, _P, _P, _LL, _I, _I, _c.c_float, _c.c_ulonglong, _c.POINTER(_c.c_float), _P]),
    "fhmg_ws_dataset": (_I, [_P, _P, _P, _D, _I, _c.c_float, _P, _P, _c.POINTER(_LL)]),
    "fhmg_ws_predict": (_I, [_P, _P, _P, _D, _I, _I, _P]),
    "fhmg_wsnet_launches": (_I, [_c.POINTER(_LL)]),
    "fhmg_ws_solve_host": (_I, [_P, _P, _P, _P, _D, _I, _I, _I, _I, _D, _I, _c.POINTER(_I), _c.POINTER(_D)]),
}


def lib():
    """The loaded library (ctypes.CDLL); raises ImportError if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"libfhmg.so not built ({LIB_PATH}); run paper_1706_07632_gb300.build.build()")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


class FhmgError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{_STATUS.get(status, status)}: {msg}")
        self.status = status


def _check(status, allow=()):
    if status != FHMG_OK and status not in allow:
        raise FhmgError(status, lib().fhmg_last_error().decode())
    return status


def _ptr(x):
    """Device (or host) pointer of a tensor/array, or None."""
    if x is None:
        return None
    if hasattr(x, "data_ptr"):
        if not x.is_contiguous():
            raise ValueError("arrays must be contiguous")
        import torch
        if x.dtype != torch.float64:
            raise TypeError("arrays must be float64")
        return x.data_ptr()
    return x.ctypes.data  # numpy (host) arrays for the *_host entry points


def _stream_ptr(stream):
    if stream is not None:
        return stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)
    import torch
    return torch.cuda.current_stream().cuda_stream


class HMatrix:
    """fhmg_build_hmatrix: mesh, L1 matrix and its H-matrix form (host, one-time)."""

    def __init__(self, alpha, gamma, T, M, leaf=64, rank=0, tol=1e-10, lowrank="taylor"):
        """lowrank "taylor": the paper's kernel expansion (Section 3); "aca": built algebraically by
        adaptive cross approximation (needs rank 0 and tol > 0)."""
        h = _P()
        if lowrank == "aca":
            _check(lib().fhmg_build_hmatrix_aca(alpha, gamma, T, M, leaf, tol, ctypes.byref(h)))
        else:
            _check(lib().fhmg_build_hmatrix(alpha, gamma, T, M, leaf, rank, tol, ctypes.byref(h)))
        self._h = h
        self.alpha, self.gamma, self.T, self.M = alpha, gamma, T, M
        self.leaf, self.rank, self.tol = leaf, rank, tol

    def info(self):
        nd, nr, mr, by = _I(), _I(), _I(), _c.c_size_t()
        _check(lib().fhmg_hmatrix_info(self._h, ctypes.byref(nd), ctypes.byref(nr), ctypes.byref(mr), ctypes.byref(by)))
        return {"n_dense": nd.value, "n_lowrank": nr.value, "max_rank": mr.value, "bytes": by.value}

    def mesh(self):
        import numpy as np
        t = np.empty(self.M + 1)
        d = np.empty(self.M)
        _check(lib().fhmg_hmatrix_mesh(self._h, t.ctypes.data, d.ctypes.data))
        return t, d

    def dense(self):
        import numpy as np
        R = np.empty((self.M, self.M))
        _check(lib().fhmg_hmatrix_dense(self._h, R.ctypes.data))
        return R

    def flops_per_column(self):
        v = _D()
        _check(lib().fhmg_hmatrix_flops(self._h, ctypes.byref(v)))
        return v.value

    def split_digits(self):
        """fhmg_hmatrix_split_digits: (tiles, pairs, rexp) -- the BF16 digit tiles of R~ as uint16 bit
        patterns (n_tiles x 8192, K-major 128-byte-swizzled 128 x 64 tiles), the per-block table
        (n_blocks x 4: digit mask, first tile, 0, 0) and the row exponents E_m."""
        import numpy as np
        n = _LL(0)
        _check(lib().fhmg_hmatrix_split_digits(self._h, None, ctypes.byref(n), None, None))
        nI = self.M // 128
        tiles = np.empty((n.value, 8192), dtype=np.uint16)
        pairs = np.empty((nI * (nI + 1), 4), dtype=np.int32)
        rexp = np.empty(self.M, dtype=np.int32)
        _check(lib().fhmg_hmatrix_split_digits(self._h, tiles.ctypes.data, ctypes.byref(n), pairs.ctypes.data,
                                               rexp.ctypes.data))
        return tiles, pairs, rexp

    def sama_two_grid(self, dim, N, Lx=1.0, nu1=0, nu2=1):
        """Two-grid convergence factor predicted by mode analysis (fhmg_sama_two_grid)."""
        v = _D()
        _check(lib().fhmg_sama_two_grid(self._h, dim, N, Lx, nu1, nu2, ctypes.byref(v)))
        return v.value

    def __del__(self):
        if getattr(self, "_h", None) and _lib is not None:
            _lib.fhmg_hmatrix_destroy(self._h)
            self._h = None


class Problem:
    """fhmg_problem_create: a dim-D grid of N^dim interior points on the current CUDA device."""

    def __init__(self, hm: HMatrix, dim, N, Lx=1.0, prec=FP64, stream=None):
        p = _P()
        _check(lib().fhmg_problem_create(hm._h, dim, N, Lx, prec, _stream_ptr(stream), ctypes.byref(p)))
        self._p = p
        self.hm, self.dim, self.N, self.Lx, self.prec = hm, dim, N, Lx, prec
        self.M = hm.M
        self.levels = (N + 1).bit_length() - 1

    def shape(self, N=None):
        N = self.N if N is None else N
        return (self.M, N) if self.dim == 1 else (self.M, N, N)

    def autotune(self):
        _check(lib().fhmg_problem_autotune(self._p))

    def set_inner(self, cycles):
        _check(lib().fhmg_problem_set_inner(self._p, cycles))

    def set_rtol_reference(self, ref):
        """0: ||r_k|| <= rtol ||r_0|| (default); 1: ||r_k|| <= rtol max|F|."""
        _check(lib().fhmg_problem_set_rtol_reference(self._p, ref))

    def set_coarse_direct(self, n):
        """Solve the coarse-grid correction exactly on the level with n points per dimension
        (n <= 1: recursion to one point, the paper's cycle)."""
        _check(lib().fhmg_problem_set_coarse_direct(self._p, n))

    def set_cycle_index(self, cycle_index):
        """Coarse-grid cycles per level: 1 V-cycle (default), 2 W-cycle."""
        _check(lib().fhmg_problem_set_cycle_index(self._p, cycle_index))

    def inject_timeout(self, consumer_spin=1024):
        """Test hook: the next walk launch withholds a chunk and its waits give up after
        consumer_spin polls; the next norm or solve then raises FHMG_ETIMEOUT."""
        _check(lib().fhmg_problem_inject_timeout(self._p, consumer_spin))

    def set_defect_arith(self, mode):
        """Outer defect of the mixed path: 2 digit splitting on the tensor cores (the default where
        available), 1 double-float walk, 0 FP64 products."""
        _check(lib().fhmg_problem_set_defect_arith(self._p, mode))

    def split_flops(self):
        """BF16 tensor-core flops per grid point of one split defect (None where unavailable)."""
        v = ctypes.c_double()
        if lib().fhmg_problem_split_flops(self._p, ctypes.byref(v)) != FHMG_OK:
            return None
        return v.value

    def hmatvec_df(self, Y, X, tile=0):
        _check(lib().fhmg_hmatvec_df(self._p, _ptr(Y), _ptr(X), X.numel() // self.M, tile))

    def set_tensor_cores(self, enable=True):
        """FP32 products on the tensor cores (3xTF32 mma.sync) where the column tile allows."""
        _check(lib().fhmg_problem_set_tensor_cores(self._p, 1 if enable else 0))

    def set_mixed_storage(self, mode):
        """0 automatic, 1 FP64 storage with FP32 products, 2 FP32 throughout (inner cycles)."""
        _check(lib().fhmg_problem_set_mixed_storage(self._p, mode))

    def profile(self, enable=True):
        _check(lib().fhmg_problem_profile(self._p, 1 if enable else 0))

    def counters(self):
        n, ns, ms = _LL(), _LL(), _D()
        _check(lib().fhmg_problem_counters(self._p, ctypes.byref(n), ctypes.byref(ns), ctypes.byref(ms)))
        return {"launches": n.value, "smooth_launches": ns.value, "smooth_ms": ms.value}

    def defect_timing(self):
        n, ms, cols = _LL(), _D(), _LL()
        _check(lib().fhmg_problem_defect_timing(self._p, ctypes.byref(n), ctypes.byref(ms), ctypes.byref(cols)))
        return {"defect_launches": n.value, "defect_ms": ms.value, "columns": cols.value}

    def line_solve(self, level, X, B):
        ncols = B.numel() // self.M
        _check(lib().fhmg_line_solve(self._p, level, _ptr(X), _ptr(B), ncols))

    def hmatvec(self, Y, X):
        _check(lib().fhmg_hmatvec(self._p, _ptr(Y), _ptr(X), X.numel() // self.M))

    def line_solve_f32(self, level, X, B, tile=0):
        """fhmg_line_solve with the mixed path's FP32 products (tile 16/32: tensor cores)."""
        _check(lib().fhmg_line_solve_f32(self._p, level, _ptr(X), _ptr(B), B.numel() // self.M, tile))

    def hmatvec_f32(self, Y, X, tile=0):
        _check(lib().fhmg_hmatvec_f32(self._p, _ptr(Y), _ptr(X), X.numel() // self.M, tile))

    def line_solve_s(self, level, X, B):
        """FP32-storage line solve (float32 tensors); BF16 problems: tcgen05 walk on wide panels."""
        _check(lib().fhmg_line_solve_s(self._p, level, _fptr(X), _fptr(B), B.numel() // self.M))

    def hmatvec_s(self, Y, X):
        """FP32-storage product Y = R~ X (float32 tensors)."""
        _check(lib().fhmg_hmatvec_s(self._p, _fptr(Y), _fptr(X), X.numel() // self.M))

    def smooth(self, u, F, nsweeps=1):
        _check(lib().fhmg_smooth(self._p, _ptr(u), _ptr(F), nsweeps))

    def residual(self, u, f, g, r):
        _check(lib().fhmg_residual(self._p, _ptr(u), _ptr(f), _ptr(g), _ptr(r)))

    def restrict_residual(self, u, F, rc):
        _check(lib().fhmg_restrict_residual(self._p, _ptr(u), _ptr(F), _ptr(rc)))

    def prolong_correct(self, u, e):
        _check(lib().fhmg_prolong_correct(self._p, _ptr(u), _ptr(e)))

    def vcycle(self, u, f, g=None, nu1=1, nu2=1):
        _check(lib().fhmg_vcycle(self._p, _ptr(u), _ptr(f), _ptr(g), nu1, nu2))

    def residual_norm(self, u, f, g=None):
        v = _D()
        _check(lib().fhmg_residual_norm(self._p, _ptr(u), _ptr(f), _ptr(g), ctypes.byref(v)))
        return v.value

    def residual_norm_noalloc(self, u, f):
        """fhmg_residual_norm_noalloc: same norm, scratch from a fixed library-owned device array."""
        v = _D()
        _check(lib().fhmg_residual_norm_noalloc(self._p, _ptr(u), _ptr(f), ctypes.byref(v)))
        return v.value

    def solve(self, u, f, g=None, nu1=1, nu2=1, rtol=1e-10, max_cycles=50, allow_notconv=False):
        k, rr = _I(), _D()
        st = lib().fhmg_solve(self._p, _ptr(u), _ptr(f), _ptr(g), nu1, nu2, rtol, max_cycles,
                              ctypes.byref(k), ctypes.byref(rr))
        _check(st, allow=(FHMG_ENOTCONV,) if allow_notconv else ())
        return k.value, rr.value

    def solve_host(self, u, f, g=None, nu1=1, nu2=1, rtol=1e-10, max_cycles=50):
        """u, f, g: C-contiguous float64 host arrays (numpy or pinned CPU tensors)."""
        k, rr = _I(), _D()
        _check(lib().fhmg_solve_host(self._p, _ptr(u), _ptr(f), _ptr(g), nu1, nu2, rtol, max_cycles,
                                     ctypes.byref(k), ctypes.byref(rr)))
        return k.value, rr.value

    def __del__(self):
        if getattr(self, "_p", None) and _lib is not None:
            _lib.fhmg_problem_destroy(self._p)
            self._p = None


def solve_batched(problems, us, fs, nu1=1, nu2=1, rtol=1e-8, max_cycles=60, allow_notconv=False):
    """fhmg_solve_batched: all problems' V-cycles in lockstep, one launch per stage, graph-replayed.
    Returns (cycles, relres) lists."""
    n = len(problems)
    P = (_P * n)(*[p._p for p in problems])
    U = (_P * n)(*[_ptr(u) for u in us])
    F = (_P * n)(*[_ptr(f) for f in fs])
    k = (_I * n)()
    rr = (_D * n)()
    st = lib().fhmg_solve_batched(n, P, U, F, nu1, nu2, rtol, max_cycles, k, rr)
    _check(st, allow=(FHMG_ENOTCONV,) if allow_notconv else ())
    return list(k), list(rr)


def _fptr(x):
    """Device pointer of a contiguous float32 tensor."""
    import torch
    if x.dtype != torch.float32 or not x.is_contiguous():
        raise TypeError("expected a contiguous float32 tensor")
    return x.data_ptr()


class WSNet:
    """fhmg_wsnet: the warm-start network (parameters on the device)."""

    def __init__(self, hidden=320, layers=3, seed=0):
        h = _P()
        _check(lib().fhmg_wsnet_create(hidden, layers, seed, ctypes.byref(h)))
        self._h = h
        self.hidden, self.layers = hidden, layers

    def num_params(self):
        n = _LL()
        _check(lib().fhmg_wsnet_num_params(self._h, ctypes.byref(n)))
        return n.value

    def get_params(self):
        import numpy as np
        p = np.empty(self.num_params(), dtype=np.float32)
        _check(lib().fhmg_wsnet_get_params(self._h, p.ctypes.data))
        return p

    def set_params(self, p):
        import numpy as np
        p = np.ascontiguousarray(p, dtype=np.float32)
        _check(lib().fhmg_wsnet_set_params(self._h, p.ctypes.data))

    def forward(self, X, Y, bf16=False, stream=None):
        _check(lib().fhmg_wsnet_forward(self._h, _fptr(X), X.shape[0], 1 if bf16 else 0, _fptr(Y), _stream_ptr(stream)))

    def loss_grad(self, X, Y, stream=None):
        import numpy as np
        loss = np.zeros(1, dtype=np.float32)
        g = np.empty(self.num_params(), dtype=np.float32)
        _check(lib().fhmg_wsnet_loss_grad(self._h, _fptr(X), _fptr(Y), X.shape[0], loss.ctypes.data, g.ctypes.data,
                                          _stream_ptr(stream)))
        return float(loss[0]), g

    def train(self, X, Y, batch=4096, steps=1000, lr=1e-3, seed=0, stream=None):
        last = _c.c_float()
        _check(lib().fhmg_wsnet_train(self._h, _fptr(X), _fptr(Y), X.shape[0], batch, steps, lr, seed,
                                      ctypes.byref(last), _stream_ptr(stream)))
        return last.value

    def predict(self, prob, f, alpha, K=24, bf16=True, u0=None):
        """Warm start u0 for source f (constant in time) on problem prob."""
        import torch
        if u0 is None:
            u0 = torch.empty_like(f)
        _check(lib().fhmg_ws_predict(self._h, prob._p, _ptr(f), alpha, K, 1 if bf16 else 0, _ptr(u0)))
        return u0

    def solve_host(self, prob, u, f, alpha, K=24, bf16=True, nu1=1, nu2=1, rtol=1e-8, max_cycles=60):
        """fhmg_ws_solve_host: f (host, constant in time) in, warm start, solve, u (host) out."""
        k, rr = _I(), _D()
        _check(lib().fhmg_ws_solve_host(self._h, prob._p, _ptr(u), _ptr(f), alpha, K, 1 if bf16 else 0, nu1, nu2,
                                        rtol, max_cycles, ctypes.byref(k), ctypes.byref(rr)))
        return k.value, rr.value

    def __del__(self):
        if getattr(self, "_h", None) and _lib is not None:
            _lib.fhmg_wsnet_destroy(self._h)
            self._h = None


def ws_dataset(prob, u, f, alpha, K=24, rel_thr=1e-6):
    """Training pairs (X, Y) from a solution u of prob for a source f constant in time."""
    import torch
    nm = K ** prob.dim
    X = torch.empty((nm * prob.M, 6), dtype=torch.float32, device=u.device)
    Y = torch.empty((nm * prob.M,), dtype=torch.float32, device=u.device)
    n = _LL()
    _check(lib().fhmg_ws_dataset(prob._p, _ptr(u), _ptr(f), alpha, K, rel_thr, X.data_ptr(), Y.data_ptr(),
                                 ctypes.byref(n)))
    return X[: n.value], Y[: n.value]


def wsnet_launches():
    """Kernel launches issued so far by the network and warm-start kernels (process-wide)."""
    n = _LL()
    _check(lib().fhmg_wsnet_launches(ctypes.byref(n)))
    return n.value


def autotune_leaf(alpha, gamma, T, M, tol, dim, N, Lx=1.0, prec=FP64, stream=None):
    """fhmg_autotune_leaf: (best leaf size, its V-cycle time in ms)."""
    leaf, ms = _I(), _D()
    _check(lib().fhmg_autotune_leaf(alpha, gamma, T, M, tol, dim, N, Lx, prec, _stream_ptr(stream),
                                    ctypes.byref(leaf), ctypes.byref(ms)))
    return leaf.value, ms.value


def autotune_hmatrix(alpha, gamma, T, M, leaf=64, err_target=1e-10):
    """fhmg_autotune_hmatrix (host only): the (rank, tol) of fhmg_build_hmatrix with the fewest
    H-matvec flops per column whose row-relative error against the exact R is <= err_target, as
    {"rank", "tol", "err", "flops_per_column"}."""
    r, t, e, f = _I(), _D(), _D(), _D()
    _check(lib().fhmg_autotune_hmatrix(alpha, gamma, T, M, leaf, err_target, ctypes.byref(r), ctypes.byref(t),
                                       ctypes.byref(e), ctypes.byref(f)))
    return {"rank": r.value, "tol": t.value, "err": e.value, "flops_per_column": f.value}
