"""Thin ctypes binding of the C ABI in include/rm.h (argument marshalling
only; every step of the solver runs in librm.so's CUDA kernels).

Vectors are passed as CUDA device pointers: torch tensors (float64, on the
GPU, contiguous) or raw integer addresses.  The library must have been built
in-tree (paper_2211_14284_gb300/build.py); a missing library is an error,
never a fallback.
"""

from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "librm.so")
HOST_LIB_PATH = os.path.join(HERE, "librm_host.so")

RM_HGRAD, RM_HCURL, RM_HDIV = 0, 1, 2
RM_FP64, RM_FP32 = 0, 1
RM_PAFW, RM_PH = 0, 1
RM_CHOL, RM_ICC = 0, 1
RM_COARSE_NONE, RM_COARSE_P1, RM_COARSE_GMG = 0, 1, 2
RM_NORM_L2, RM_NORM_NATURAL = 0, 1
RM_ARITH_FP64, RM_ARITH_DF64 = 0, 1
RM_BC_DIRICHLET, RM_BC_NONE = 0, 1
RM_SMOOTH_STAR, RM_SMOOTH_HIPTMAIR = 0, 1
RM_ADDITIVE, RM_HYBRID = 0, 1
STATUS = {0: "RM_OK", 1: "RM_ERR_ARG", 2: "RM_ERR_CUDA", 3: "RM_ERR_OOM",
          4: "RM_ERR_BREAKDOWN", 5: "RM_ERR_NOT_CONVERGED", 6: "RM_ERR_NAN", 7: "RM_ERR_TIMEOUT"}

EXPORTED = ["rm_default_options", "rm_setup", "rm_ndofs", "rm_layout", "rm_history", "rm_apply",
            "rm_precondition", "rm_solve", "rm_stats", "rm_destroy", "rm_last_error",
            "rm_precondition_noalloc", "rm_debug_patch_timeout", "rm_batch_setup", "rm_batch_ndofs", "rm_batch_solve",
            "rm_batch_destroy", "rm_batch_last_error", "rm_default_train_options",
            "rm_corrector_train", "rm_corrector_save", "rm_corrector_load", "rm_corrector_use",
            "rm_net_create", "rm_net_num_params", "rm_net_get_params", "rm_net_set_params",
            "rm_net_forward", "rm_net_backward", "rm_net_adam", "rm_net_destroy",
            "rm_net_last_error", "rm_hodge_setup", "rm_hodge_ndofs", "rm_hodge_intervals",
            "rm_hodge_apply", "rm_hodge_precondition", "rm_hodge_solve", "rm_hodge_destroy",
            "rm_hodge_last_error"]
RM_NOALLOC_MAX_COARSE = 8192
RM_CORRECTOR_PLAIN, RM_CORRECTOR_LEARNED, RM_CORRECTOR_OFF = 0, 1, 2


class RmMesh(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
                ("vertices", ctypes.POINTER(ctypes.c_double))]


class RmOptions(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int), ("decomposition", ctypes.c_int),
                ("static_condensation", ctypes.c_int), ("factor", ctypes.c_int),
                ("coarse", ctypes.c_int), ("flexible", ctypes.c_int),
                ("rtol", ctypes.c_double), ("max_it", ctypes.c_int),
                ("check_every", ctypes.c_int), ("profile", ctypes.c_int),
                ("norm", ctypes.c_int), ("arith", ctypes.c_int), ("boundary", ctypes.c_int),
                ("coarse_smoother", ctypes.c_int), ("composition", ctypes.c_int),
                ("hybrid_omega", ctypes.c_double), ("relaxation", ctypes.c_int),
                ("deterministic", ctypes.c_int)]


class RmInfo(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int), ("status", ctypes.c_int),
                ("rel_res_l2", ctypes.c_double), ("rel_res_natural", ctypes.c_double),
                ("iterations_natural", ctypes.c_int), ("history_len", ctypes.c_int),
                ("setup_s", ctypes.c_double), ("solve_ms", ctypes.c_double),
                ("apply_ms", ctypes.c_double), ("apply_calls", ctypes.c_int),
                ("precond_ms", ctypes.c_double), ("precond_calls", ctypes.c_int),
                ("kernel_launches", ctypes.c_longlong),
                ("learned_calls", ctypes.c_int), ("judge_calls", ctypes.c_int),
                ("fallback_at", ctypes.c_int), ("judge_eta", ctypes.c_double)]


class RmTrainOptions(ctypes.Structure):
    _fields_ = [("pairs", ctypes.c_int), ("epochs", ctypes.c_int), ("batch", ctypes.c_int),
                ("lr", ctypes.c_float), ("levels", ctypes.c_int), ("width", ctypes.c_int),
                ("seed", ctypes.c_ulonglong), ("val_fraction", ctypes.c_double),
                ("target_cycles", ctypes.c_int), ("off_fraction", ctypes.c_double),
                ("rounds", ctypes.c_int), ("round_pairs", ctypes.c_int), ("round_epochs", ctypes.c_int)]


class RmTrainInfo(ctypes.Structure):
    _fields_ = [("pairs", ctypes.c_int), ("solves", ctypes.c_int), ("params", ctypes.c_longlong),
                ("gen_s", ctypes.c_double), ("train_s", ctypes.c_double),
                ("train_loss", ctypes.c_double), ("val_loss", ctypes.c_double),
                ("val_eta", ctypes.c_double)]


class RmError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{STATUS.get(code, code)}: {msg}")
        self.code = code


_lib = None


def load():
    """Load librm.so (raises if it was not built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: run __graft_entry__.build() first")
    lib = ctypes.CDLL(LIB_PATH)
    c_dp = ctypes.POINTER(ctypes.c_double)
    vp = ctypes.c_void_p
    lib.rm_default_options.restype = RmOptions
    lib.rm_setup.argtypes = [ctypes.POINTER(vp), ctypes.c_int, ctypes.POINTER(RmMesh),
                             ctypes.c_int, c_dp, c_dp, ctypes.POINTER(RmOptions), vp]
    lib.rm_ndofs.argtypes = [vp, ctypes.POINTER(ctypes.c_longlong),
                             ctypes.POINTER(ctypes.c_longlong)]
    lib.rm_stats.argtypes = [vp, ctypes.POINTER(ctypes.c_longlong),
                             ctypes.POINTER(ctypes.c_longlong),
                             ctypes.POINTER(ctypes.c_longlong)]
    lib.rm_layout.argtypes = [vp, ctypes.c_int, ctypes.POINTER(ctypes.c_int),
                              ctypes.POINTER(ctypes.c_longlong)]
    lib.rm_history.argtypes = [vp, ctypes.c_int, c_dp, ctypes.c_int, ctypes.POINTER(ctypes.c_int)]
    lib.rm_apply.argtypes = [vp, vp, vp]
    lib.rm_precondition.argtypes = [vp, vp, vp]
    lib.rm_precondition_noalloc.argtypes = [vp, vp, vp]
    lib.rm_debug_patch_timeout.argtypes = [ctypes.c_int]
    lib.rm_solve.argtypes = [vp, vp, vp, ctypes.POINTER(RmInfo)]
    lib.rm_destroy.argtypes = [vp]
    lib.rm_destroy.restype = None
    lib.rm_last_error.argtypes = [vp]
    lib.rm_last_error.restype = ctypes.c_char_p
    lib.rm_batch_setup.argtypes = [ctypes.POINTER(vp), ctypes.c_int, ctypes.POINTER(ctypes.c_int),
                                   ctypes.POINTER(RmMesh), ctypes.POINTER(ctypes.c_int),
                                   ctypes.POINTER(c_dp), ctypes.POINTER(c_dp),
                                   ctypes.POINTER(RmOptions), vp]
    lib.rm_batch_ndofs.argtypes = [vp, ctypes.c_int, ctypes.POINTER(ctypes.c_longlong)]
    lib.rm_batch_solve.argtypes = [vp, ctypes.POINTER(vp), ctypes.POINTER(vp),
                                   ctypes.POINTER(RmInfo), vp]
    lib.rm_batch_destroy.argtypes = [vp]
    lib.rm_batch_destroy.restype = None
    lib.rm_batch_last_error.argtypes = [vp]
    lib.rm_batch_last_error.restype = ctypes.c_char_p
    lib.rm_default_train_options.restype = RmTrainOptions
    lib.rm_corrector_train.argtypes = [vp, ctypes.POINTER(RmTrainOptions), ctypes.c_int, vp,
                                       ctypes.POINTER(RmTrainInfo)]
    lib.rm_corrector_save.argtypes = [vp, ctypes.c_char_p]
    lib.rm_corrector_load.argtypes = [vp, ctypes.c_char_p]
    lib.rm_corrector_use.argtypes = [vp, ctypes.c_int, ctypes.c_int, ctypes.c_double]
    lib.rm_net_create.argtypes = [ctypes.POINTER(vp), ctypes.POINTER(ctypes.c_int), ctypes.c_int,
                                  ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_ulonglong, vp]
    lib.rm_net_num_params.argtypes = [vp]
    lib.rm_net_num_params.restype = ctypes.c_longlong
    lib.rm_net_get_params.argtypes = [vp, vp]
    lib.rm_net_set_params.argtypes = [vp, vp]
    lib.rm_net_forward.argtypes = [vp, ctypes.c_int, vp, vp]
    lib.rm_net_backward.argtypes = [vp, vp, vp, vp]
    lib.rm_net_adam.argtypes = [vp, ctypes.c_float]
    lib.rm_net_destroy.argtypes = [vp]
    lib.rm_net_destroy.restype = None
    lib.rm_net_last_error.restype = ctypes.c_char_p
    lib.rm_hodge_setup.argtypes = [ctypes.POINTER(vp), ctypes.c_int, ctypes.POINTER(RmMesh), ctypes.c_int,
                                   ctypes.POINTER(RmOptions), ctypes.c_int, vp]
    lib.rm_hodge_ndofs.argtypes = [vp, ctypes.POINTER(ctypes.c_longlong), ctypes.POINTER(ctypes.c_longlong)]
    lib.rm_hodge_intervals.argtypes = [vp, c_dp, c_dp]
    lib.rm_hodge_apply.argtypes = [vp, vp, vp]
    lib.rm_hodge_precondition.argtypes = [vp, vp, vp]
    lib.rm_hodge_solve.argtypes = [vp, vp, vp, ctypes.POINTER(RmInfo)]
    lib.rm_hodge_destroy.argtypes = [vp]
    lib.rm_hodge_destroy.restype = None
    lib.rm_hodge_last_error.argtypes = [vp]
    lib.rm_hodge_last_error.restype = ctypes.c_char_p
    _lib = lib
    return lib


def debug_patch_timeout(on):
    """rm_debug_patch_timeout: a testing aid that makes the warp-per-patch
    kernels' bounded waits give up (on=True) or restores them (on=False)."""
    lib = load()
    rc = lib.rm_debug_patch_timeout(1 if on else 0)
    if rc != 0:
        raise RmError(rc, lib.rm_last_error(None).decode())


def _ptr(t):
    if isinstance(t, int):
        return ctypes.c_void_p(t)
    if not (t.is_cuda and t.is_contiguous()):
        raise ValueError("expected a contiguous CUDA tensor")
    return ctypes.c_void_p(t.data_ptr())


def _dbl_array(a):
    if a is None:
        return None
    import numpy as np
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a, a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def options(**kw) -> RmOptions:
    o = load().rm_default_options()
    for k, v in kw.items():
        if not hasattr(o, k):
            raise KeyError(k)
        setattr(o, k, v)
    return o


class Solver:
    """One discretisation + preconditioner (rm_setup), bound to a stream."""

    def __init__(self, space: int, n, p: int, vertices=None, alpha=None, beta=None,
                 stream=None, **opts):
        lib = load()
        n = (n, n, n) if isinstance(n, int) else tuple(n)
        self._keep = []
        mesh = RmMesh(n[0], n[1], n[2], None)
        if vertices is not None:
            arr, ptr = _dbl_array(vertices)
            self._keep.append(arr)
            mesh.vertices = ptr
        al = _dbl_array(alpha)
        be = _dbl_array(beta)
        o = options(**opts)
        if stream is None:
            s = ctypes.c_void_p(0)
        elif isinstance(stream, int):
            s = ctypes.c_void_p(stream)
        else:
            s = ctypes.c_void_p(stream.cuda_stream)
        h = ctypes.c_void_p()
        rc = lib.rm_setup(ctypes.byref(h), space, ctypes.byref(mesh), p,
                          al[1] if al else None, be[1] if be else None,
                          ctypes.byref(o), s)
        if rc != 0:
            raise RmError(rc, lib.rm_last_error(None).decode())
        self.h = h
        self.lib = lib
        self.space, self.n, self.p = space, n, p
        a, f = ctypes.c_longlong(), ctypes.c_longlong()
        lib.rm_ndofs(h, ctypes.byref(a), ctypes.byref(f))
        self.size, self.nfree = a.value, f.value

    def _check(self, rc):
        if rc != 0:
            raise RmError(rc, self.lib.rm_last_error(self.h).decode())

    def apply(self, x, y):
        self._check(self.lib.rm_apply(self.h, _ptr(x), _ptr(y)))

    def precondition_noalloc(self, r, z):
        """rm_precondition_noalloc: same result for a non-condensed handle,
        scratch in the library's static device array (no allocation)."""
        self._check(self.lib.rm_precondition_noalloc(self.h, _ptr(r), _ptr(z)))

    def precondition(self, r, z):
        self._check(self.lib.rm_precondition(self.h, _ptr(r), _ptr(z)))

    def solve(self, b, x, check=True):
        info = RmInfo()
        rc = self.lib.rm_solve(self.h, _ptr(b), _ptr(x), ctypes.byref(info))
        if check and rc not in (0,):
            self._check(rc)
        return {"iterations": info.iterations, "status": STATUS.get(info.status),
                "rel_res_l2": info.rel_res_l2, "rel_res_natural": info.rel_res_natural,
                "iterations_natural": info.iterations_natural,
                "history_len": info.history_len, "setup_s": info.setup_s,
                "solve_ms": info.solve_ms,
                "apply_ms": info.apply_ms, "apply_calls": info.apply_calls,
                "precond_ms": info.precond_ms, "precond_calls": info.precond_calls,
                "kernel_launches": info.kernel_launches, "learned_calls": info.learned_calls,
                "judge_calls": info.judge_calls, "fallback_at": info.fallback_at,
                "judge_eta": info.judge_eta}

    def layout(self, comp):
        """rm_layout: (dims, offset) of lattice component comp."""
        d = (ctypes.c_int * 3)()
        off = ctypes.c_longlong()
        self._check(self.lib.rm_layout(self.h, comp, d, ctypes.byref(off)))
        return tuple(d), off.value

    def history(self, which=RM_NORM_L2, cap=None):
        """rm_history of the last solve (l2 or natural), as a numpy array."""
        import numpy as np
        cap = 100000 if cap is None else cap
        out = np.zeros(cap)
        n = ctypes.c_int()
        self._check(self.lib.rm_history(self.h, which, out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                        cap, ctypes.byref(n)))
        return out[:n.value].copy()

    def corrector_train(self, rhs, **opts):
        """rm_corrector_train: rhs is a contiguous float64 CUDA tensor holding
        nrhs right-hand sides one after another (nrhs x size)."""
        o = self.lib.rm_default_train_options()
        for k, v in opts.items():
            if not hasattr(o, k):
                raise KeyError(k)
            setattr(o, k, v)
        nrhs = rhs.numel() // self.size
        info = RmTrainInfo()
        self._check(self.lib.rm_corrector_train(self.h, ctypes.byref(o), nrhs, _ptr(rhs),
                                                ctypes.byref(info)))
        return {f: getattr(info, f) for f, _ in RmTrainInfo._fields_}

    def corrector_save(self, path):
        rc = self.lib.rm_corrector_save(self.h, os.fsencode(path))
        if rc != 0:
            raise RmError(rc, self.lib.rm_last_error(None).decode())

    def corrector_load(self, path):
        self._check(self.lib.rm_corrector_load(self.h, os.fsencode(path)))

    def corrector_use(self, mode, judge_every=8, judge_max=0.9):
        self._check(self.lib.rm_corrector_use(self.h, mode, judge_every, judge_max))

    def stats(self):
        a, b, c = ctypes.c_longlong(), ctypes.c_longlong(), ctypes.c_longlong()
        self.lib.rm_stats(self.h, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c))
        return {"patches": a.value, "slots": b.value, "factor_nnz": c.value}

    def close(self):
        if getattr(self, "h", None):
            self.lib.rm_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class HodgeSolver:
    """rm_hodge_*: the mixed Hodge Laplacian of degree k (Gamma_D empty) with
    MINRES and the Riesz-map block preconditioner."""

    def __init__(self, k, n, p, vertices=None, cheb_its=4, stream=None, **opts):
        lib = load()
        n = (n, n, n) if isinstance(n, int) else tuple(n)
        self._keep = []
        mesh = RmMesh(n[0], n[1], n[2], None)
        if vertices is not None:
            arr, ptr = _dbl_array(vertices)
            self._keep.append(arr)
            mesh.vertices = ptr
        o = options(**opts)
        s = ctypes.c_void_p(0 if stream is None else stream.cuda_stream)
        h = ctypes.c_void_p()
        rc = lib.rm_hodge_setup(ctypes.byref(h), k, ctypes.byref(mesh), p, ctypes.byref(o), cheb_its, s)
        if rc != 0:
            raise RmError(rc, lib.rm_hodge_last_error(None).decode())
        self.h, self.lib, self.k = h, lib, k
        a, b = ctypes.c_longlong(), ctypes.c_longlong()
        lib.rm_hodge_ndofs(h, ctypes.byref(a), ctypes.byref(b))
        self.n_sigma, self.n_u = a.value, b.value
        self.size = self.n_sigma + self.n_u

    def _check(self, rc):
        if rc != 0:
            raise RmError(rc, self.lib.rm_hodge_last_error(self.h).decode())

    def intervals(self):
        a, b = (ctypes.c_double * 2)(), (ctypes.c_double * 2)()
        self._check(self.lib.rm_hodge_intervals(self.h, a, b))
        return tuple(a), tuple(b)

    def apply(self, x, y):
        self._check(self.lib.rm_hodge_apply(self.h, _ptr(x), _ptr(y)))

    def precondition(self, r, z):
        self._check(self.lib.rm_hodge_precondition(self.h, _ptr(r), _ptr(z)))

    def solve(self, b, x, check=True):
        info = RmInfo()
        rc = self.lib.rm_hodge_solve(self.h, _ptr(b), _ptr(x), ctypes.byref(info))
        if check and rc != 0:
            self._check(rc)
        return {"iterations": info.iterations, "status": STATUS.get(info.status),
                "rel_res_natural": info.rel_res_natural, "solve_ms": info.solve_ms,
                "setup_s": info.setup_s}

    def close(self):
        if getattr(self, "h", None):
            self.lib.rm_hodge_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Net:
    """rm_net_*: the corrector's network on its own (FP32 tensors on the GPU,
    channels-last [batch][voxel][channel])."""

    def __init__(self, dims, levels, width, in_channels, max_batch=1, seed=1, stream=None):
        lib = load()
        d = (ctypes.c_int * 3)(*dims)
        s = ctypes.c_void_p(0 if stream is None else stream.cuda_stream)
        h = ctypes.c_void_p()
        rc = lib.rm_net_create(ctypes.byref(h), d, levels, width, in_channels, max_batch, seed, s)
        if rc != 0:
            raise RmError(rc, lib.rm_net_last_error().decode())
        self.h, self.lib = h, lib
        self.dims, self.levels, self.width, self.in_channels = tuple(dims), levels, width, in_channels
        self.nparams = lib.rm_net_num_params(h)

    def _check(self, rc):
        if rc != 0:
            raise RmError(rc, self.lib.rm_net_last_error().decode())

    def get_params(self):
        import numpy as np
        w = np.empty(self.nparams, dtype=np.float32)
        self._check(self.lib.rm_net_get_params(self.h, ctypes.c_void_p(w.ctypes.data)))
        return w

    def set_params(self, w):
        import numpy as np
        w = np.ascontiguousarray(w, dtype=np.float32)
        assert w.size == self.nparams
        self._check(self.lib.rm_net_set_params(self.h, ctypes.c_void_p(w.ctypes.data)))

    def forward(self, x, y):
        self._check(self.lib.rm_net_forward(self.h, x.shape[0], _ptr(x), _ptr(y)))

    def backward(self, dy, grad=None, dx=None):
        self._check(self.lib.rm_net_backward(self.h, _ptr(dy),
                                             _ptr(grad) if grad is not None else None,
                                             _ptr(dx) if dx is not None else None))

    def adam(self, lr):
        self._check(self.lib.rm_net_adam(self.h, lr))

    def close(self):
        if getattr(self, "h", None):
            self.lib.rm_net_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class BatchSolver:
    """rm_batch_*: independent problems (list of dicts with space, n, p and
    optional alpha, beta, vertices) solved together with shared options."""

    def __init__(self, problems, **opts):
        lib = load()
        nprob = len(problems)
        self._keep = []
        space = (ctypes.c_int * nprob)(*[pr["space"] for pr in problems])
        degs = (ctypes.c_int * nprob)(*[pr["p"] for pr in problems])
        meshes = (RmMesh * nprob)()
        c_dp = ctypes.POINTER(ctypes.c_double)
        al = (c_dp * nprob)()
        be = (c_dp * nprob)()
        for i, pr in enumerate(problems):
            n = pr["n"]
            n = (n, n, n) if isinstance(n, int) else tuple(n)
            meshes[i] = RmMesh(n[0], n[1], n[2], None)
            if pr.get("vertices") is not None:
                arr, ptr = _dbl_array(pr["vertices"])
                self._keep.append(arr)
                meshes[i].vertices = ptr
            for key, dst in (("alpha", al), ("beta", be)):
                if pr.get(key) is not None:
                    arr, ptr = _dbl_array(pr[key])
                    self._keep.append(arr)
                    dst[i] = ptr
        o = options(**opts)
        h = ctypes.c_void_p()
        rc = lib.rm_batch_setup(ctypes.byref(h), nprob, space, meshes, degs, al, be,
                                ctypes.byref(o), None)
        if rc != 0:
            raise RmError(rc, lib.rm_batch_last_error(None).decode())
        self.h, self.lib, self.nprob = h, lib, nprob
        self.sizes = []
        for i in range(nprob):
            v = ctypes.c_longlong()
            lib.rm_batch_ndofs(h, i, ctypes.byref(v))
            self.sizes.append(v.value)

    def solve(self, bs, xs, stream=None, check=True):
        n = self.nprob
        bp = (ctypes.c_void_p * n)(*[_ptr(b).value for b in bs])
        xp = (ctypes.c_void_p * n)(*[_ptr(x).value for x in xs])
        infos = (RmInfo * n)()
        s = ctypes.c_void_p(0) if stream is None else ctypes.c_void_p(
            stream if isinstance(stream, int) else stream.cuda_stream)
        rc = self.lib.rm_batch_solve(self.h, bp, xp, infos, s)
        if check and rc != 0:
            raise RmError(rc, self.lib.rm_batch_last_error(self.h).decode())
        return [{"iterations": i.iterations, "status": STATUS.get(i.status),
                 "rel_res_l2": i.rel_res_l2, "solve_ms": i.solve_ms,
                 "kernel_launches": i.kernel_launches, "graph_rounds": i.precond_calls}
                for i in infos]

    def close(self):
        if getattr(self, "h", None):
            self.lib.rm_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---------------------------------------------------------------------------
# host-only setup inspection (librm_host.so, no CUDA): used by CPU tests
# ---------------------------------------------------------------------------
class HostProbe:
    def __init__(self):
        if not os.path.exists(HOST_LIB_PATH):
            raise RuntimeError(f"{HOST_LIB_PATH} is missing: run __graft_entry__.build()")
        self.lib = ctypes.CDLL(HOST_LIB_PATH)
        self.lib.rmh_error.restype = ctypes.c_char_p

    def basis(self, p):
        import numpy as np
        S = np.zeros((p + 1, p + 1)); lam = np.zeros(p); B = np.zeros((p + 1, p + 1))
        A = np.zeros((p + 1, p + 1)); D = np.zeros((p, p + 1)); Js = np.zeros((p + 1, 2))
        P = lambda a: a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        rc = self.lib.rmh_basis(p, P(S), P(lam), P(B), P(A), P(D), P(Js))
        if rc:
            raise RuntimeError(self.lib.rmh_error().decode())
        return dict(S=S, lam=lam, Bhat=B, Ahat=A, D=D, Js=Js)

    def build(self, k, n, p, X, alpha, beta, mode, factor, coarse=True):
        import numpy as np
        n = (n, n, n) if isinstance(n, int) else tuple(n)
        narr = (ctypes.c_int * 3)(*n)
        self._keep = [np.ascontiguousarray(X, float), np.ascontiguousarray(alpha, float),
                      np.ascontiguousarray(beta, float)]
        P = lambda a: a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        rc = self.lib.rmh_build(k, narr, p, P(self._keep[0]), P(self._keep[1]),
                                P(self._keep[2]), mode, factor, int(coarse))
        if rc:
            raise RuntimeError(self.lib.rmh_error().decode())

    def csr(self, which):
        import numpy as np
        import scipy.sparse as sp
        nr, nnz = ctypes.c_int(), ctypes.c_longlong()
        self.lib.rmh_csr_size(which, ctypes.byref(nr), ctypes.byref(nnz))
        ptr = np.zeros(nr.value + 1, np.int64); col = np.zeros(nnz.value, np.int32)
        val = np.zeros(nnz.value)
        self.lib.rmh_csr_get(which, ptr.ctypes.data_as(ctypes.c_void_p),
                             col.ctypes.data_as(ctypes.c_void_p),
                             val.ctypes.data_as(ctypes.c_void_p))
        ncol = int(col.max()) + 1 if nnz.value else 0
        return ptr, col, val

    def families(self):
        import numpy as np
        out = []
        for f in range(self.lib.rmh_nfamilies()):
            ns, npch, nnz = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
            self.lib.rmh_family_size(f, ctypes.byref(ns), ctypes.byref(npch), ctypes.byref(nnz))
            sm = np.zeros(npch.value * ns.value, np.int32)
            rp = np.zeros(ns.value + 1, np.int32)
            col = np.zeros(nnz.value, np.int32)
            val = np.zeros(npch.value * nnz.value)
            v = lambda a: a.ctypes.data_as(ctypes.c_void_p)
            self.lib.rmh_family_get(f, v(sm), v(rp), v(col), v(val))
            fam = dict(nslots=ns.value, npatch=npch.value, nnz=nnz.value,
                       slotmap=sm.reshape(npch.value, ns.value), rowptr=rp, col=col,
                       val=val.reshape(npch.value, nnz.value), inverse=None)
            isinv, nb, nv = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
            self.lib.rmh_family_inverse_size(f, ctypes.byref(isinv), ctypes.byref(nb),
                                             ctypes.byref(nv))
            if isinv.value:
                bptr = np.zeros(nb.value + 1, np.int32)
                pslot = np.zeros(ns.value, np.int32)
                boff = np.zeros(nb.value + 1, np.int32)
                ival = np.zeros(npch.value * nv.value)
                self.lib.rmh_family_inverse_get(f, v(bptr), v(pslot), v(boff), v(ival))
                fam["inverse"] = dict(bptr=bptr, pos_slot=pslot, boff=boff,
                                      ival=ival.reshape(npch.value, nv.value))
            out.append(fam)
        return out

    @staticmethod
    def patch_inverse(fam, pi):
        """Dense (slots x slots) inverse of patch pi of a block-inverse family."""
        import numpy as np
        ns = fam["nslots"]
        inv = fam["inverse"]
        M = np.zeros((ns, ns))
        for b in range(len(inv["bptr"]) - 1):
            sl = inv["pos_slot"][inv["bptr"][b]:inv["bptr"][b + 1]]
            nb = len(sl)
            blk = inv["ival"][pi, inv["boff"][b]:inv["boff"][b] + nb * nb].reshape(nb, nb).T
            M[np.ix_(sl, sl)] = blk
        return M

    def coarse_inverse(self):
        import numpy as np
        nc = self.lib.rmh_coarse_size()
        A = np.zeros((nc, nc))
        self.lib.rmh_coarse_inverse(A.ctypes.data_as(ctypes.c_void_p))
        return A
