"""ctypes binding of libbta (include/bta.h): argument marshalling only.

Every numerical step runs in the CUDA library; this module turns torch CUDA
tensors into device pointers, host arrays into C arrays, and return codes
into exceptions.  There is no CPU fallback: if libbta.so is missing or a call
fails, an exception is raised.

Function names mirror the C ABI (bta_create, bta_assemble, bta_factor,
bta_logdet, bta_solve, bta_selinv, fobj_eval, ...).  ``BtaModel`` and
``BtaContext`` own the C handles and free them when collected.
"""

from __future__ import annotations

import ctypes as C
import os

import numpy as np

_LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "libbta.so")
_lib = None

BTA_OK, BTA_ERR_ARG, BTA_ERR_OOM, BTA_ERR_NOT_PD = 0, 1, 2, 3
BTA_ERR_TIMEOUT, BTA_ERR_NONFINITE, BTA_ERR_CUDA, BTA_ERR_STATE = 4, 5, 6, 7
BTA_QP, BTA_QC = 0, 1
BTA_FP64, BTA_MIXED, BTA_MIXED_HI = 0, 1, 2
BTA_LIK_GAUSSIAN, BTA_LIK_POISSON = 0, 1
BTA_BLK_D, BTA_BLK_B, BTA_BLK_R, BTA_BLK_T = 0, 1, 2, 3
BTA_STORE_Q, BTA_STORE_L, BTA_STORE_SIGMA, BTA_STORE_LINV = 0, 1, 2, 3
BTA_PHASES = 5
BTA_CREATE_LOW_MEMORY = 1
PHASE_NAMES = ("assemble", "factor_logdet", "solve_f", "selinv", "adjoint")


class BtaError(RuntimeError):
    def __init__(self, code: int, where: str, info: int | None = None):
        self.code = code
        self.info = info
        msg = f"{where}: {lib().bta_strerror(code).decode()} (code {code})"
        if info is not None and info >= 0:
            msg += f", info={info}"
        super().__init__(msg)


class _ModelDesc(C.Structure):
    _fields_ = [
        ("nv", C.c_int), ("ns", C.c_int), ("nt", C.c_int), ("nr", C.c_int),
        ("nodes", C.POINTER(C.c_double)), ("tri", C.POINTER(C.c_int)), ("n_tri", C.c_int),
        ("m", C.c_int), ("obs_var", C.POINTER(C.c_int)), ("obs_time", C.POINTER(C.c_int)),
        ("obs_xy", C.POINTER(C.c_double)), ("obs_tri", C.POINTER(C.c_int)),
        ("X", C.POINTER(C.c_double)), ("y", C.POINTER(C.c_double)),
        ("beta_prior_prec", C.c_double), ("theta0", C.POINTER(C.c_double)),
    ]


def lib():
    """Load libbta.so (built in-tree); raise if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(_LIB_PATH):
        raise ImportError(f"libbta.so not built ({_LIB_PATH}); run paper_2507_06938_gb300._build.build()")
    L = C.CDLL(_LIB_PATH)
    vp, ip, dp = C.c_void_p, C.c_int, C.c_double
    sig = {
        "bta_model_create": (ip, [C.POINTER(_ModelDesc), C.POINTER(vp)]),
        "bta_model_destroy": (ip, [vp]),
        "bta_model_dims": (ip, [vp, C.POINTER(ip), C.POINTER(ip), C.POINTER(ip), C.POINTER(ip)]),
        "bta_create": (ip, [ip, ip, ip, ip, vp, C.POINTER(vp)]),
        "bta_create_batched": (ip, [ip, ip, ip, ip, ip, vp, C.POINTER(vp)]),
        "bta_create_ex": (ip, [ip, ip, ip, ip, ip, ip, vp, C.POINTER(vp)]),
        "bta_batch_size": (ip, [vp, C.POINTER(ip)]),
        "bta_factor_batch": (ip, [vp, ip]),
        "bta_selinv_batch": (ip, [vp, ip]),
        "bta_last_error_matrix": (ip, [vp, C.POINTER(ip)]),
        "bta_fobj_grad": (ip, [vp, vp, vp, ip, vp, vp]),
        "bta_destroy": (ip, [vp]),
        "bta_assemble": (ip, [vp, vp, vp, ip]),
        "bta_theta_to_params": (ip, [vp, vp, vp, vp]),
        "bta_factor": (ip, [vp, ip]),
        "bta_logdet": (ip, [vp, ip, vp]),
        "bta_solve": (ip, [vp, ip, vp, vp, ip, vp]),
        "bta_selinv": (ip, [vp, ip]),
        "bta_block_ptr": (ip, [vp, ip, ip, ip, ip, C.POINTER(vp), C.POINTER(ip)]),
        "bta_matvec": (ip, [vp, ip, vp, vp]),
        "fobj_eval": (ip, [vp, vp, vp, ip, vp, vp]),
        "bta_sync": (ip, [vp]),
        "bta_last_info": (ip, [vp, C.POINTER(C.c_longlong)]),
        "bta_strerror": (C.c_char_p, [ip]),
        "bta_selinv_diag": (ip, [vp, ip, vp]),
        "bta_launch_count": (C.c_longlong, []),
        "bta_profile": (ip, [vp, ip]),
        "bta_profile_read": (ip, [vp, C.POINTER(dp), C.POINTER(C.c_longlong), C.POINTER(dp)]),
        "bta_profile_phases": (ip, [vp, C.POINTER(dp), ip]),
        "bta_chol_inv_noalloc": (ip, [vp, ip, ip, vp, ip, vp, vp]),
        "bta_autotune": (ip, [vp, ip, C.POINTER(C.c_int)]),
        "bta_fobj_eval_multi": (ip, [ip, C.POINTER(vp), C.POINTER(vp), C.POINTER(vp), C.POINTER(ip),
                                     C.POINTER(vp), C.POINTER(vp), C.POINTER(vp), vp]),
        "bta_fobj_residual": (ip, [vp, vp]),
        "bta_fobj_laplace": (ip, [vp, vp, vp, ip, ip, ip, vp, vp, vp]),
        "bta_set_time_partitions": (ip, [vp, ip]),
        "bta_set_low_memory": (ip, [vp, ip]),
        "bta_fobj_grad_host": (ip, [vp, vp, vp, ip, vp, vp, vp]),
        "bta_fp64_peak": (ip, [ip, C.POINTER(dp)]),
        "bta_flops_factor": (dp, [ip, ip, ip]),
        "bta_flops_selinv": (dp, [ip, ip, ip]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _lib = L
    return L


def exported_symbols():
    """Names the binding expects libbta.so to export."""
    return ["bta_model_create", "bta_model_destroy", "bta_model_dims", "bta_create", "bta_destroy",
            "bta_assemble", "bta_theta_to_params", "bta_factor", "bta_logdet", "bta_solve",
            "bta_selinv", "bta_block_ptr", "bta_matvec", "fobj_eval", "bta_sync", "bta_last_info",
            "bta_strerror", "bta_flops_factor", "bta_flops_selinv", "bta_selinv_diag",
            "bta_launch_count", "bta_profile", "bta_profile_read", "bta_chol_inv_noalloc",
            "bta_create_batched", "bta_batch_size", "bta_factor_batch", "bta_selinv_batch",
            "bta_last_error_matrix", "bta_fobj_grad", "bta_autotune", "bta_fobj_eval_multi",
            "bta_fobj_residual", "bta_fp64_peak", "bta_fobj_grad_host", "bta_fobj_laplace",
            "bta_set_time_partitions", "bta_profile_phases", "bta_set_low_memory", "bta_create_ex"]


def _check(code: int, where: str):
    if code != BTA_OK:
        raise BtaError(code, where)


def _ptr(t) -> int:
    """Device pointer of a contiguous CUDA float64 tensor (or None -> NULL)."""
    if t is None:
        return None
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError("expected a CUDA tensor")
    if t.dtype != torch.float64 or not t.is_contiguous():
        raise TypeError("expected a contiguous float64 tensor")
    return t.data_ptr()


def _stream_handle(stream) -> int:
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return stream.cuda_stream


class _DevArray:
    """__cuda_array_interface__ view of a raw device block (zero copy)."""

    def __init__(self, ptr: int, rows: int, cols: int, ld: int):
        self.__cuda_array_interface__ = {
            "shape": (rows, cols), "typestr": "<f8", "data": (ptr, False),
            "strides": (8, 8 * ld), "version": 3,
        }


# ----------------------------------------------------------------------------- model

class BtaModel:
    """bta_model_t built from a problem description (duck-typed: nv, ns, nt,
    nr, nodes, tri, obs_var, obs_time, obs_xy, obs_tri, X, y, theta0,
    beta_prior_prec)."""

    def __init__(self, problem):
        L = lib()
        self._keep = []

        def arr(a, dt, ct):
            a = np.ascontiguousarray(a, dtype=dt)
            self._keep.append(a)
            return a.ctypes.data_as(C.POINTER(ct))

        d = _ModelDesc()
        d.nv, d.ns, d.nt, d.nr = problem.nv, problem.ns, problem.nt, problem.nr
        d.nodes = arr(problem.nodes, np.float64, C.c_double)
        d.tri = arr(problem.tri, np.int32, C.c_int)
        d.n_tri = int(problem.tri.shape[0])
        d.m = int(problem.y.shape[0])
        d.obs_var = arr(problem.obs_var, np.int32, C.c_int)
        d.obs_time = arr(problem.obs_time, np.int32, C.c_int)
        d.obs_xy = arr(problem.obs_xy, np.float64, C.c_double)
        d.obs_tri = arr(problem.obs_tri, np.int32, C.c_int)
        d.X = arr(problem.X, np.float64, C.c_double)
        d.y = arr(problem.y, np.float64, C.c_double)
        d.beta_prior_prec = float(problem.beta_prior_prec)
        d.theta0 = arr(problem.theta0, np.float64, C.c_double)
        h = C.c_void_p()
        _check(L.bta_model_create(C.byref(d), C.byref(h)), "bta_model_create")
        self._keep = []
        self.handle = h
        n, b, a, dt = C.c_int(), C.c_int(), C.c_int(), C.c_int()
        _check(L.bta_model_dims(h, C.byref(n), C.byref(b), C.byref(a), C.byref(dt)), "bta_model_dims")
        self.n, self.b, self.a, self.dim_theta = n.value, b.value, a.value, dt.value
        self.N = self.n * self.b + self.a

    def close(self):
        """Release the device copy of the model now (also done on collection)."""
        if getattr(self, "handle", None) and _lib is not None:
            _lib.bta_model_destroy(self.handle)
            self.handle = None

    __del__ = close


# ----------------------------------------------------------------------------- context

class BtaContext:
    """bta_ctx_t: device storage of Q_p and Q_c, their factors and selected
    inverses, bound to a CUDA stream."""

    def __init__(self, n: int, b: int, a: int, precision: int = BTA_FP64, stream=None, batch: int = 1,
                 low_memory: bool = False):
        L = lib()
        import torch
        # the torch stream the context runs on (the current one when none is given)
        self._stream_obj = stream if stream is not None else torch.cuda.current_stream()
        h = C.c_void_p()
        flags = BTA_CREATE_LOW_MEMORY if low_memory else 0
        _check(L.bta_create_ex(n, b, a, precision, batch, flags, C.c_void_p(_stream_handle(stream)), C.byref(h)),
               "bta_create_ex")
        self.handle = h
        self.n, self.b, self.a, self.batch = n, b, a, batch
        self.N = n * b + a

    def close(self):
        """Release the context's device storage now (also done on collection)."""
        if getattr(self, "handle", None) and _lib is not None:
            _lib.bta_destroy(self.handle)
            self.handle = None

    __del__ = close

    # -- the C ABI, one method per entry point
    def assemble(self, model: BtaModel, params, which: int):
        _check(lib().bta_assemble(self.handle, model.handle, _ptr(params), which), "bta_assemble")

    def theta_to_params(self, model: BtaModel, theta, params):
        _check(lib().bta_theta_to_params(self.handle, model.handle, _ptr(theta), _ptr(params)),
               "bta_theta_to_params")

    def factor(self, which: int):
        _check(lib().bta_factor(self.handle, which), "bta_factor")

    def logdet(self, which: int, out):
        _check(lib().bta_logdet(self.handle, which, _ptr(out)), "bta_logdet")

    def solve(self, which: int, rhs, x, refine_iters: int = 0, resid=None):
        _check(lib().bta_solve(self.handle, which, _ptr(rhs), _ptr(x), refine_iters, _ptr(resid)), "bta_solve")

    def selinv(self, which: int):
        _check(lib().bta_selinv(self.handle, which), "bta_selinv")

    def set_time_partitions(self, P: int):
        """bta_set_time_partitions: P > 1 runs factor/solve/selinv by time-domain
        partitioning (P partitions eliminated together, then the separators).
        Needs n - (P - 1) ceil((n + 1) / P) >= 1 and a <= b; keeps assembled
        matrices, drops factors."""
        _check(lib().bta_set_time_partitions(self.handle, int(P)), "bta_set_time_partitions")

    def set_low_memory(self, enable: bool):
        """bta_set_low_memory: inverse diagonal blocks in the factor's diagonal
        slots and the selected inverse over the factor (about 0.6 of the
        default memory at large n); a selected inversion consumes the factor."""
        _check(lib().bta_set_low_memory(self.handle, 1 if enable else 0), "bta_set_low_memory")

    def factor_batch(self, kind: int):
        _check(lib().bta_factor_batch(self.handle, kind), "bta_factor_batch")

    def selinv_batch(self, kind: int):
        _check(lib().bta_selinv_batch(self.handle, kind), "bta_selinv_batch")

    def matvec(self, which: int, x, y):
        _check(lib().bta_matvec(self.handle, which, _ptr(x), _ptr(y)), "bta_matvec")

    def fobj_eval(self, model: BtaModel, thetas, f_out, mu_out=None):
        n_theta = int(thetas.shape[0]) if thetas.dim() == 2 else 1
        _check(lib().fobj_eval(self.handle, model.handle, _ptr(thetas), n_theta, _ptr(f_out), _ptr(mu_out)),
               "fobj_eval")

    def selinv_diag(self, which: int, out):
        _check(lib().bta_selinv_diag(self.handle, which, _ptr(out)), "bta_selinv_diag")

    AUTOTUNE_KEYS = ("fp64_leaf", "df32_leaf", "tensor_min_dim", "split_tile", "split_waves", "fp64_ctas_per_sm",
                     "split_band_triangular", "split_band_general", "split_band_lower")

    def autotune(self, reps: int = 2):
        """bta_autotune: time the launch-shape candidates of the diagonal chain
        and of the b x b x b products on this context's storage and keep the
        fastest; returns (leaf, df_leaf, tensor threshold, split-product tile,
        split waves, FP64 CTAs per SM).  Overwrites the first diagonal block
        of every matrix."""
        out = (C.c_int * len(self.AUTOTUNE_KEYS))()
        _check(lib().bta_autotune(self.handle, int(reps), out), "bta_autotune")
        return tuple(int(v) for v in out)

    def profile(self, enable: bool):
        _check(lib().bta_profile(self.handle, 1 if enable else 0), "bta_profile")

    def profile_read(self):
        ms, n, fl = C.c_double(), C.c_longlong(), C.c_double()
        _check(lib().bta_profile_read(self.handle, C.byref(ms), C.byref(n), C.byref(fl)), "bta_profile_read")
        return ms.value, n.value, fl.value

    def profile_phases(self):
        """bta_profile_phases: ms of (assembly, factorisation + log-det, solve + f,
        selected inversion, adjoint) of the last profiled gradient group."""
        out = (C.c_double * BTA_PHASES)()
        _check(lib().bta_profile_phases(self.handle, out, BTA_PHASES), "bta_profile_phases")
        return dict(zip(PHASE_NAMES, (float(v) for v in out)))

    def fobj_grad(self, model: BtaModel, thetas, f_out, grad_out):
        n_theta = int(thetas.shape[0]) if thetas.dim() == 2 else 1
        _check(lib().bta_fobj_grad(self.handle, model.handle, _ptr(thetas), n_theta, _ptr(f_out), _ptr(grad_out)),
               "bta_fobj_grad")

    def fobj_grad_host(self, model: BtaModel, thetas, f_out, grad_out, var_out=None):
        """bta_fobj_grad_host: host (CPU) arrays in and out; contiguous float64
        numpy arrays or CPU torch tensors (pinned ones copy asynchronously)."""
        def hp(a, name):
            if a is None:
                return None
            if hasattr(a, "data_ptr"):
                if a.is_cuda or not a.is_contiguous() or str(a.dtype) != "torch.float64":
                    raise TypeError(f"{name}: expected a contiguous CPU float64 tensor")
                return a.data_ptr()
            if not (isinstance(a, np.ndarray) and a.dtype == np.float64 and a.flags.c_contiguous):
                raise TypeError(f"{name}: expected a C-contiguous float64 array")
            return a.ctypes.data
        n_theta = int(thetas.shape[0]) if len(thetas.shape) == 2 else 1
        _check(lib().bta_fobj_grad_host(self.handle, model.handle, hp(thetas, "thetas"), n_theta,
                                        hp(f_out, "f_out"), hp(grad_out, "grad_out"), hp(var_out, "var_out")),
               "bta_fobj_grad_host")

    def fobj_laplace(self, model: BtaModel, thetas, likelihood: int, newton_iters: int, f_out, x_out=None,
                     step_out=None):
        """bta_fobj_laplace: f_obj by the Laplace approximation at the Newton
        mode of the latent field (non-Gaussian likelihoods)."""
        n_theta = int(thetas.shape[0]) if thetas.dim() == 2 else 1
        _check(lib().bta_fobj_laplace(self.handle, model.handle, _ptr(thetas), n_theta, int(likelihood),
                                      int(newton_iters), _ptr(f_out), _ptr(x_out), _ptr(step_out)),
               "bta_fobj_laplace")

    def fobj_residual(self, out):
        """||b - Q_c mu|| / ||b|| of every slot's conditional mean (last group)."""
        _check(lib().bta_fobj_residual(self.handle, _ptr(out)), "bta_fobj_residual")

    def sync(self):
        code = lib().bta_sync(self.handle)
        if code != BTA_OK:
            info = C.c_longlong()
            mat = C.c_int()
            lib().bta_last_info(self.handle, C.byref(info))
            lib().bta_last_error_matrix(self.handle, C.byref(mat))
            err = BtaError(code, "bta_sync", info.value)
            err.matrix = mat.value
            raise err

    def block(self, which: int, store: int, kind: int, i: int = 0):
        """Zero-copy torch view of one stored block (rows x cols, column-major)."""
        import torch
        p = C.c_void_p()
        ld = C.c_int()
        _check(lib().bta_block_ptr(self.handle, which, store, kind, i, C.byref(p), C.byref(ld)),
               "bta_block_ptr")
        rows = self.a if kind in (BTA_BLK_R, BTA_BLK_T) else self.b
        cols = self.a if kind == BTA_BLK_T else self.b
        return torch.as_tensor(_DevArray(p.value, rows, cols, ld.value), device="cuda")


# ----------------------------------------------------------------------------- flat C-ABI names

def bta_model_create(problem) -> BtaModel:
    return BtaModel(problem)


def bta_create(n, b, a, precision=BTA_FP64, stream=None) -> BtaContext:
    return BtaContext(n, b, a, precision, stream)


def bta_create_batched(n, b, a, precision=BTA_FP64, batch=1, stream=None) -> BtaContext:
    return BtaContext(n, b, a, precision, stream, batch)


def bta_set_time_partitions(ctx: BtaContext, P: int):
    ctx.set_time_partitions(P)


def time_partitions_valid(n: int, a: int, b: int, P: int) -> bool:
    """Whether bta_set_time_partitions accepts P for blocks of this shape."""
    if P == 1:
        return True
    h = -(-(n + 1) // P)
    return P > 1 and n - (P - 1) * h >= 1 and a <= b


def bta_factor_batch(ctx: BtaContext, kind: int):
    ctx.factor_batch(kind)


def bta_selinv_batch(ctx: BtaContext, kind: int):
    ctx.selinv_batch(kind)


def bta_assemble(ctx: BtaContext, model: BtaModel, params, which: int):
    ctx.assemble(model, params, which)


def bta_theta_to_params(ctx: BtaContext, model: BtaModel, theta, params):
    ctx.theta_to_params(model, theta, params)


def bta_factor(ctx: BtaContext, which: int):
    ctx.factor(which)


def bta_logdet(ctx: BtaContext, which: int, out):
    ctx.logdet(which, out)


def bta_solve(ctx: BtaContext, which: int, rhs, x, refine_iters: int = 0, resid=None):
    ctx.solve(which, rhs, x, refine_iters, resid)


def bta_selinv(ctx: BtaContext, which: int):
    ctx.selinv(which)


def bta_matvec(ctx: BtaContext, which: int, x, y):
    ctx.matvec(which, x, y)


def fobj_eval(ctx: BtaContext, model: BtaModel, thetas, f_out, mu_out=None):
    ctx.fobj_eval(model, thetas, f_out, mu_out)


def bta_fobj_grad(ctx: BtaContext, model: BtaModel, thetas, f_out, grad_out):
    ctx.fobj_grad(model, thetas, f_out, grad_out)


def bta_fobj_eval_multi(contexts, models, thetas, f_outs, mu_outs=None, grad_outs=None, join_stream=None):
    """f_obj (and gradients where grad_outs[i] is a tensor) of independent
    problems of any shapes, one context and model per problem; each runs on its
    context's stream and `join_stream` (default: the current stream) waits for
    all.  thetas[i]: (n_theta_i, dim_i) CUDA float64; f_outs[i]: n_theta_i
    values; mu_outs[i] / grad_outs[i]: None or (n_theta_i, N_i) / (n_theta_i, dim_i)."""
    count = len(contexts)
    if not (len(models) == len(thetas) == len(f_outs) == count) or count < 1:
        raise ValueError("bta_fobj_eval_multi: one context, model, theta block and f output per problem")
    vparr = C.c_void_p * count
    ctx_arr = vparr(*[c.handle for c in contexts])
    mod_arr = vparr(*[m.handle for m in models])
    th_arr = vparr(*[_ptr(t) for t in thetas])
    nth = (C.c_int * count)(*[int(t.shape[0]) if t.dim() == 2 else 1 for t in thetas])
    f_arr = vparr(*[_ptr(f) for f in f_outs])
    mu_arr = vparr(*[_ptr(m) for m in mu_outs]) if mu_outs is not None else None
    g_arr = vparr(*[_ptr(g) for g in grad_outs]) if grad_outs is not None else None
    _check(lib().bta_fobj_eval_multi(count, ctx_arr, mod_arr, th_arr, nth, f_arr, mu_arr, g_arr,
                                     C.c_void_p(_stream_handle(join_stream))), "bta_fobj_eval_multi")
    # the problems' streams use these tensors: keep their memory from being
    # reused by torch's caching allocator before those streams are done
    for k, c in enumerate(contexts):
        for t in (thetas[k], f_outs[k], None if mu_outs is None else mu_outs[k],
                  None if grad_outs is None else grad_outs[k]):
            if t is not None:
                t.record_stream(c._stream_obj)


def bta_sync(ctx: BtaContext):
    ctx.sync()


def bta_selinv_diag(ctx: BtaContext, which: int, out):
    ctx.selinv_diag(which, out)


def bta_launch_count() -> int:
    return lib().bta_launch_count()


def bta_profile(ctx: BtaContext, enable: bool):
    ctx.profile(enable)


def bta_profile_read(ctx: BtaContext):
    return ctx.profile_read()


def bta_profile_phases(ctx: BtaContext):
    return ctx.profile_phases()


NOALLOC_MAX_B = 2048


def bta_chol_inv_noalloc(A, X, info, stream=None):
    """Allocation-free Cholesky + inverse of one SPD block (no counterpart in
    the paper): A (b x b, CUDA float64, column-major data of a symmetric
    matrix) is overwritten in its lower triangle by L, X (b x b) receives
    L^{-1}, info (at least one int64 element) receives -1 or the first failing
    row.  Nothing is allocated by the library; the workspace is a fixed
    8.5 MiB device array of the current device, so b is limited to 2048,
    every tensor must live on the current device, and concurrent calls on the
    GPU race."""
    import torch
    for t, dt in ((A, torch.float64), (X, torch.float64), (info, torch.int64)):
        if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == dt and t.is_contiguous()):
            raise TypeError("expected contiguous CUDA tensors (float64 A, X; int64 info)")
    if A.dim() != 2 or A.shape[0] != A.shape[1]:
        raise ValueError(f"bta_chol_inv_noalloc: A must be square, got {tuple(A.shape)}")
    b = int(A.shape[0])
    if tuple(X.shape) != (b, b):
        raise ValueError(f"bta_chol_inv_noalloc: X must be {b} x {b}, got {tuple(X.shape)}")
    if info.numel() < 1:
        raise ValueError("bta_chol_inv_noalloc: info needs one element")
    if b > NOALLOC_MAX_B:
        raise ValueError(f"bta_chol_inv_noalloc: block order {b} exceeds the maximum {NOALLOC_MAX_B}")
    dev = torch.cuda.current_device()
    if any(t.device.index != dev for t in (A, X, info)):
        raise ValueError("bta_chol_inv_noalloc: A, X and info must be on the current CUDA device")
    _check(lib().bta_chol_inv_noalloc(A.data_ptr(), b, b, X.data_ptr(), b, info.data_ptr(),
                                      C.c_void_p(_stream_handle(stream))), "bta_chol_inv_noalloc")


def bta_fobj_grad_host(ctx: BtaContext, model: BtaModel, thetas, f_out, grad_out, var_out=None):
    ctx.fobj_grad_host(model, thetas, f_out, grad_out, var_out)


def bta_fobj_laplace(ctx: BtaContext, model: BtaModel, thetas, likelihood, newton_iters, f_out, x_out=None,
                     step_out=None):
    ctx.fobj_laplace(model, thetas, likelihood, newton_iters, f_out, x_out, step_out)


def bta_fobj_residual(ctx: BtaContext, out):
    ctx.fobj_residual(out)


def bta_fp64_peak(use_dmma: bool = False) -> float:
    """Measured FP64 throughput of the current GPU (TFLOP/s): DFMA loop, or
    FP64 tensor-core MMA loop when use_dmma."""
    out = C.c_double()
    _check(lib().bta_fp64_peak(1 if use_dmma else 0, C.byref(out)), "bta_fp64_peak")
    return out.value


def bta_flops_factor(n: int, b: int, a: int) -> float:
    return lib().bta_flops_factor(n, b, a)


def bta_flops_selinv(n: int, b: int, a: int) -> float:
    return lib().bta_flops_selinv(n, b, a)
