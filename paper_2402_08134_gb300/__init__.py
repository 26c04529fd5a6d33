"""GB300 (sm_103a) randomized SymNMF: Python binding of the C ABI in include/symnmf.h.

Argument marshalling only: every step of the method runs in the CUDA kernels
of `libsymnmf_gb300.so`.  Importing this package loads that library and
fails loudly (ImportError) when it has not been built; there is no CPU
fallback.  Build it with `python -c "import __graft_entry__ as g; g.build()"`
or `python -m paper_2402_08134_gb300._build`.

The functions below carry the C names.  Tensors are torch CUDA tensors; the
stream defaults to torch's current stream.  `Solver` is a small convenience
wrapper that keeps the borrowed tensors alive for the handle's lifetime.
"""

from __future__ import annotations

import ctypes as C
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libsymnmf_gb300.so")

if not os.path.exists(LIB_PATH):
    raise ImportError(
        "libsymnmf_gb300.so is not built; run `python -m paper_2402_08134_gb300._build` "
        "(nvcc, sm_103a) before importing paper_2402_08134_gb300"
    )

_lib = C.CDLL(LIB_PATH)

# ---------------------------------------------------------------- constants
OK, EINVAL, ENOMEM, ENOTSPD, ETIMEOUT, ENAN, ECUDA, ESTATE, EUNSUPPORTED = range(9)
X_DENSE_F64, X_DENSE_F32, X_DENSE_BF16, X_DENSE_FP8, X_CSR_F32 = range(5)
SRC_X, SRC_LAI, SRC_XHI, SRC_COMP = range(4)
RULE_HALS, RULE_BPP = range(2)
GEMM_AUTO, GEMM_SIMT, GEMM_TC = range(3)

STATUS_NAMES = {
    0: "OK", 1: "EINVAL", 2: "ENOMEM", 3: "ENOTSPD", 4: "ETIMEOUT", 5: "ENAN", 6: "ECUDA",
    7: "ESTATE", 8: "EUNSUPPORTED",
}


class SymNMFError(RuntimeError):
    def __init__(self, status, msg=""):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class symnmf_problem(C.Structure):
    _fields_ = [
        ("n", C.c_int64), ("k", C.c_int32), ("fmt", C.c_int32), ("x", C.c_void_p), ("ldx", C.c_int64),
        ("row_scale", C.c_void_p), ("row_ptr", C.c_void_p), ("col", C.c_void_p), ("nnz", C.c_int64),
        ("x_hi", C.c_void_p), ("ldx_hi", C.c_int64), ("alpha", C.c_double), ("seed", C.c_uint64),
    ]


class symnmf_options(C.Structure):
    _fields_ = [("gemm", C.c_int32), ("use_graph", C.c_int32), ("max_width", C.c_int32),
                ("max_samples", C.c_int32), ("lai_mode", C.c_int32), ("reserved", C.c_int32 * 3)]


class symnmf_schedule(C.Structure):
    _fields_ = [("method", C.c_int32), ("algo", C.c_int32), ("rule", C.c_int32), ("l", C.c_int32),
                ("q_max", C.c_int32), ("stop_count", C.c_int32), ("max_iters", C.c_int32), ("refine", C.c_int32),
                ("max_refine", C.c_int32), ("s_max", C.c_int32), ("ada_tol", C.c_double), ("stop_tol", C.c_double)]


class symnmf_report(C.Structure):
    _fields_ = [("checks", C.c_int32), ("passes", C.c_int32), ("iters", C.c_int32), ("refine_iters", C.c_int32),
                ("nr_phase", C.c_double), ("nr_final", C.c_double)]


_P = C.c_void_p
_I = C.c_int
_I64 = C.c_int64
_D = C.c_double
_DP = C.POINTER(C.c_double)
_IP = C.POINTER(C.c_int)

_SIGS = {
    "symnmf_create": (_I, [C.POINTER(symnmf_problem), C.POINTER(symnmf_options), _P, C.POINTER(_P)]),
    "symnmf_destroy": (None, [_P]),
    "symnmf_last_error": (C.c_char_p, [_P]),
    "symnmf_info": (_I, [_P, _DP, _DP]),
    "symnmf_set_factors": (_I, [_P, _P, _P]),
    "symnmf_init_random": (_I, [_P, _I]),
    "symnmf_get_factors": (_I, [_P, _P, _P]),
    "symnmf_lai_sketch": (_I, [_P, _I, _I, _P]),
    "symnmf_lai_sketch_ada": (_I, [_P, _I, _I, _D, _P, _IP, _IP, _DP]),
    "symnmf_get_lai": (_I, [_P, _P, _DP, _IP]),
    "symnmf_set_lai": (_I, [_P, _P, _DP, _I]),
    "symnmf_hals_sweep": (_I, [_P, _I, _I, _I, _DP]),
    "symnmf_pgncg": (_I, [_P, _I, _I, _I, _DP]),
    "symnmf_solve": (_I, [_P, C.POINTER(symnmf_schedule), C.POINTER(symnmf_report)]),
    "symnmf_leverage": (_I, [_P, _I, _P]),
    "symnmf_lvs_sample": (_I, [_P, _I, _I, _D, _I, _DP, C.POINTER(C.c_int32), C.POINTER(C.c_float), _I,
                               _IP, _IP, _DP]),
    "symnmf_lvs_update": (_I, [_P, _I, _I]),
    "symnmf_lvs_iterate": (_I, [_P, _I, _I, _D, _I, _I]),
    "symnmf_residual": (_I, [_P, _I, _DP, _DP, _DP]),
    "symnmf_sweep_to_target": (_I, [_P, _I, _I, _I, _I, _D, C.POINTER(_I), C.POINTER(_I), _DP]),
    "symnmf_dense_xf": (_I, [_I, _P, _I64, _P, _I64, _P, _I, _I, _P, _I, _I, _P]),
    "symnmf_csr_xf": (_I, [_P, _P, _P, _I64, _P, _I, _P, _P]),
    "symnmf_gram": (_I, [_P, _I64, _I, _P, _P]),
    "symnmf_gram_noalloc": (_I, [_P, _I64, _I, _P, _P]),
    "symnmf_cholesky": (_I, [_P, _I, _D, _P, _P, _P]),
    "symnmf_gaussian": (_I, [_P, _I64, _I, C.c_uint64, _P]),
    "symnmf_quantize_fp8": (_I, [_P, _I64, _I64, _P, _I64, _P, _P]),
    "symnmf_convert_bf16": (_I, [_P, _I64, _I64, _P, _I64, _P]),
    "symnmf_launch_count": (C.c_uint64, []),
    "symnmf_debug_wait_timeout": (_I, [_P, _I64]),
    "symnmf_profile": (_I, [_P, _I]),
    "symnmf_profile_read": (_I, [_P, _DP, C.POINTER(C.c_int64), _DP]),
    "symnmf_profile_read_engine": (_I, [_P, _DP, C.POINTER(C.c_int64), _DP]),
    "symnmf_profile_read_lvs": (_I, [_P, _DP, _DP, _DP, C.POINTER(C.c_int64)]),
    "symnmf_profile_standalone": (_I, [_I]),
    "symnmf_profile_standalone_read": (_I, [_DP, C.POINTER(C.c_int64), _DP, _DP]),
    "symnmf_batched_create": (_I, [C.POINTER(symnmf_problem), _I, _I, C.POINTER(symnmf_options), _P,
                                   C.POINTER(_P)]),
    "symnmf_batched_destroy": (None, [_P]),
    "symnmf_batched_last_error": (C.c_char_p, [_P]),
    "symnmf_batched_init_random": (_I, [_P, _I]),
    "symnmf_batched_set_factors": (_I, [_P, _I, _P, _P]),
    "symnmf_batched_get_factors": (_I, [_P, _I, _P, _P]),
    "symnmf_batched_sweep": (_I, [_P, _I, _DP]),
    "symnmf_batched_info": (_I, [_P, _IP, _IP, _DP]),
    "symnmf_mlp_create": (_I, [_I, _I, _I, _I, C.c_uint64, _P, C.POINTER(_P)]),
    "symnmf_mlp_destroy": (None, [_P]),
    "symnmf_mlp_get_params": (_I, [_P, _P, _I64]),
    "symnmf_mlp_set_params": (_I, [_P, _P, _I64]),
    "symnmf_mlp_param_count": (_I64, [_P]),
    "symnmf_mlp_forward": (_I, [_P, _P, _I64, _P]),
    "symnmf_mlp_loss_grad": (_I, [_P, _P, _P, _I64, _P, _DP]),
    "symnmf_mlp_adam": (_I, [_P, C.c_float, _I]),
    "symnmf_warm_start": (_I, [_P, _P, _P]),
    "symnmf_sketch_features": (_I, [_P, _P]),
}

for _name, (_res, _args) in _SIGS.items():
    _f = getattr(_lib, _name)
    _f.restype = _res
    _f.argtypes = _args
    globals()[_name] = _f

EXPORTED = sorted(_SIGS)


def _ptr(t):
    return None if t is None else C.c_void_p(t.data_ptr())


def _stream(stream=None):
    import torch

    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


def check(status, handle=None, err_fn=None):
    if status != OK:
        msg = ""
        if handle is not None:
            fn = err_fn or symnmf_last_error
            raw = fn(handle)
            msg = raw.decode() if raw else ""
        raise SymNMFError(status, msg)


def launch_count() -> int:
    return int(symnmf_launch_count())


# -------------------------------------------------------------- conveniences

_FMT_OF_DTYPE = {"torch.float64": X_DENSE_F64, "torch.float32": X_DENSE_F32, "torch.bfloat16": X_DENSE_BF16,
                 "torch.uint8": X_DENSE_FP8}


class Solver:
    """One SymNMF problem on the GPU (wraps symnmf_create / ... / symnmf_destroy).

    X is a dense (n x ldx) CUDA tensor (float64, float32, bfloat16, or uint8
    E4M3 codes with `row_scale`), or a CSR triple (row_ptr int64, col int32,
    val float32) passed as `csr=(row_ptr, col, val)`.
    """

    def __init__(self, X=None, k=10, *, csr=None, n=None, row_scale=None, x_hi=None, alpha=0.0, seed=0,
                 gemm=GEMM_AUTO, use_graph=True, max_width=0, max_samples=0, lai_mode=0, stream=None):
        import torch

        self._keep = [X, csr, row_scale, x_hi]
        p = symnmf_problem()
        p.k = k
        p.alpha = alpha
        p.seed = seed
        if csr is not None:
            row_ptr, col, val = csr
            p.n = n if n is not None else row_ptr.numel() - 1
            p.fmt = X_CSR_F32
            p.x = val.data_ptr()
            p.row_ptr = row_ptr.data_ptr()
            p.col = col.data_ptr()
            p.nnz = val.numel()
        else:
            assert X.is_cuda and X.dim() == 2
            p.n = X.shape[0]
            p.ldx = X.stride(0)
            p.fmt = _FMT_OF_DTYPE[str(X.dtype)]
            p.x = X.data_ptr()
            if p.fmt == X_DENSE_FP8:
                assert row_scale is not None
                p.row_scale = row_scale.data_ptr()
        if x_hi is not None:
            assert x_hi.dtype == torch.float32
            p.x_hi = x_hi.data_ptr()
            p.ldx_hi = x_hi.stride(0)
        o = symnmf_options()
        o.gemm = gemm
        o.use_graph = 1 if use_graph else 0
        o.max_width = max_width
        o.max_samples = max_samples
        o.lai_mode = lai_mode
        self.n, self.k = int(p.n), int(k)
        self.stream = stream
        h = C.c_void_p()
        st = symnmf_create(C.byref(p), C.byref(o), _stream(stream), C.byref(h))
        if st != OK:
            raise SymNMFError(st, "symnmf_create")
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            symnmf_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _chk(self, st):
        check(st, self.h)

    # -- factors
    def set_factors(self, H0, W0=None):
        self._chk(symnmf_set_factors(self.h, _ptr(H0), _ptr(W0)))

    def init_random(self, scaled=True):
        self._chk(symnmf_init_random(self.h, 1 if scaled else 0))

    def factors(self):
        import torch

        H = torch.empty((self.n, self.k), dtype=torch.float32, device="cuda")
        W = torch.empty_like(H)
        self._chk(symnmf_get_factors(self.h, _ptr(H), _ptr(W)))
        return H, W

    def info(self):
        a, nx = C.c_double(), C.c_double()
        self._chk(symnmf_info(self.h, C.byref(a), C.byref(nx)))
        return a.value, nx.value

    # -- LAI
    def lai_sketch(self, l, q, omega=None):
        self._chk(symnmf_lai_sketch(self.h, l, q, _ptr(omega)))

    def lai_sketch_ada(self, l, q_max, tol=1e-3, omega=None):
        """Adaptive range finder + Apx-EVD; returns dict(checks, passes, nr_hist)."""
        import numpy as np

        hist = np.zeros(max(q_max, 1))
        ch, ps = C.c_int(), C.c_int()
        self._chk(symnmf_lai_sketch_ada(self.h, l, q_max, tol, _ptr(omega), C.byref(ch), C.byref(ps),
                                        hist.ctypes.data_as(_DP)))
        return {"checks": ch.value, "passes": ps.value, "nr_hist": hist[: ch.value]}

    def set_lai(self, U, lam):
        import numpy as np

        lam = np.ascontiguousarray(lam, dtype=np.float64)
        self._chk(symnmf_set_lai(self.h, _ptr(U), lam.ctypes.data_as(_DP), int(lam.shape[0])))

    def lai(self):
        import numpy as np
        import torch

        lo = C.c_int()
        self._chk(symnmf_get_lai(self.h, None, None, C.byref(lo)))
        l = lo.value
        U = torch.empty((self.n, l), dtype=torch.float32, device="cuda")
        lam = np.zeros(l)
        self._chk(symnmf_get_lai(self.h, _ptr(U), lam.ctypes.data_as(_DP), None))
        return U, lam

    def sketch_features(self):
        import torch

        _, lam = self.lai()
        out = torch.empty((self.n, lam.shape[0]), dtype=torch.float32, device="cuda")
        self._chk(symnmf_sketch_features(self.h, _ptr(out)))
        return out

    # -- sweeps
    def sweep(self, nsweeps, source=SRC_X, rule=RULE_HALS, record=True):
        import numpy as np

        obj = np.zeros(max(nsweeps, 1)) if record else None
        self._chk(symnmf_hals_sweep(self.h, nsweeps, source, rule,
                                    obj.ctypes.data_as(_DP) if record else None))
        return obj[:nsweeps] if record else None

    def pgncg(self, iters, source=SRC_X, s_max=5, record=True):
        """PGNCG-SymNMF iterations (LAI-PGNCG with source=SRC_LAI); SymNMF objectives if recorded."""
        import numpy as np

        obj = np.zeros(max(iters, 1)) if record else None
        self._chk(symnmf_pgncg(self.h, iters, source, s_max, obj.ctypes.data_as(_DP) if record else None))
        return obj[:iters] if record else None

    def solve(self, method=SRC_LAI, rule=RULE_HALS, algo=0, l=None, q_max=10, ada_tol=1e-3, stop_tol=1e-4,
              stop_count=4, max_iters=500, refine=True, max_refine=200, s_max=5):
        """The experiments' schedule (symnmf_solve): Ada-RRF sketch, iterations to the stopping rule,
        then Iterative Refinement on X; returns the report as a dict."""
        sc = symnmf_schedule(method=method, algo=algo, rule=rule, l=l or (2 * self.k + 10), q_max=q_max,
                             stop_count=stop_count, max_iters=max_iters, refine=1 if refine else 0,
                             max_refine=max_refine, s_max=s_max, ada_tol=ada_tol, stop_tol=stop_tol)
        rep = symnmf_report()
        self._chk(symnmf_solve(self.h, C.byref(sc), C.byref(rep)))
        return {f: getattr(rep, f) for f, _ in symnmf_report._fields_}

    # -- LvS
    def leverage(self, side):
        import torch

        lev = torch.empty(self.n, dtype=torch.float64, device="cuda")
        self._chk(symnmf_leverage(self.h, side, _ptr(lev)))
        return lev

    def lvs_sample(self, side, it, tau, s, lev_in=None, cap=None):
        import numpy as np

        cap = cap if cap is not None else max(s, 1) + self.n
        cap = min(cap, self.n + s)
        idx = np.zeros(cap, dtype=np.int32)
        wt = np.zeros(cap, dtype=np.float32)
        sd, stot, th = C.c_int(), C.c_int(), C.c_double()
        lev_arr = None
        if lev_in is not None:
            lev_arr = np.ascontiguousarray(lev_in, dtype=np.float64)
        self._chk(symnmf_lvs_sample(self.h, side, it, tau, s,
                                    lev_arr.ctypes.data_as(_DP) if lev_arr is not None else None,
                                    idx.ctypes.data_as(C.POINTER(C.c_int32)),
                                    wt.ctypes.data_as(C.POINTER(C.c_float)), cap, C.byref(sd), C.byref(stot),
                                    C.byref(th)))
        return dict(idx=idx[: stot.value], wt=wt[: stot.value], s_D=sd.value, s_tot=stot.value, theta=th.value)

    def lvs_update(self, side, rule=RULE_HALS):
        self._chk(symnmf_lvs_update(self.h, side, rule))

    def lvs_iterate(self, iters, tau, s, rule=RULE_HALS, iter0=0):
        self._chk(symnmf_lvs_iterate(self.h, iter0, iters, tau, s, rule))

    # -- live kernel timing
    def profile(self, enable=True):
        self._chk(symnmf_profile(self.h, 1 if enable else 0))

    def profile_read(self):
        t, n, b = C.c_double(), C.c_int64(), C.c_double()
        self._chk(symnmf_profile_read(self.h, C.byref(t), C.byref(n), C.byref(b)))
        return t.value, n.value, b.value

    def profile_read_engine(self):
        t, n, f = C.c_double(), C.c_int64(), C.c_double()
        self._chk(symnmf_profile_read_engine(self.h, C.byref(t), C.byref(n), C.byref(f)))
        return t.value, n.value, f.value

    def profile_read_lvs(self):
        """(sampling ms, sampled-product ms, update ms, halves) of the LvS halves since the last read."""
        a, b, c, n = C.c_double(), C.c_double(), C.c_double(), C.c_int64()
        self._chk(symnmf_profile_read_lvs(self.h, C.byref(a), C.byref(b), C.byref(c), C.byref(n)))
        return a.value, b.value, c.value, n.value

    # -- residual
    def residual(self, source=SRC_X, proj_grad=False):
        nr, ob, pg = C.c_double(), C.c_double(), C.c_double()
        self._chk(symnmf_residual(self.h, source, C.byref(nr), C.byref(ob), C.byref(pg) if proj_grad else None))
        return (nr.value, ob.value, pg.value) if proj_grad else (nr.value, ob.value)

    def sweep_to_target(self, target, *, source=SRC_LAI, check=SRC_X, chunk=10, max_sweeps=200):
        """Sweeps in chunks with a residual check after each, stopping at `target` (symnmf_sweep_to_target).
        Returns dict(sweeps, checks, nr) with the last check's normalized residual."""
        sw, ch, nr = _I(), _I(), C.c_double()
        self._chk(symnmf_sweep_to_target(self.h, source, check, int(chunk), int(max_sweeps), float(target),
                                         C.byref(sw), C.byref(ch), C.byref(nr)))
        return {"sweeps": sw.value, "checks": ch.value, "nr": nr.value}


class Batch:
    """Grouped solver over many problems with stacked restarts (wraps symnmf_batched_*)."""

    def __init__(self, Xs, ks, restarts=4, *, seeds=None, alpha=0.0, stream=None):
        n = len(Xs)
        arr = (symnmf_problem * n)()
        self._keep = list(Xs)
        self.ns, self.ks, self.R = [int(X.shape[0]) for X in Xs], [int(k) for k in ks], restarts
        for p, (X, k) in enumerate(zip(Xs, ks)):
            q = arr[p]
            q.n = X.shape[0]
            q.k = k
            q.fmt = _FMT_OF_DTYPE[str(X.dtype)]
            q.x = X.data_ptr()
            q.ldx = X.stride(0)
            q.alpha = alpha
            q.seed = seeds[p] if seeds is not None else p
        o = symnmf_options()
        h = C.c_void_p()
        st = symnmf_batched_create(arr, n, restarts, C.byref(o), _stream(stream), C.byref(h))
        if st != OK:
            raise SymNMFError(st, "symnmf_batched_create")
        self.h = h
        self.nprob = n

    def close(self):
        if getattr(self, "h", None):
            symnmf_batched_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _chk(self, st):
        check(st, self.h, symnmf_batched_last_error)

    def init_random(self, scaled=True):
        self._chk(symnmf_batched_init_random(self.h, 1 if scaled else 0))

    def set_factors(self, p, H0, W0=None):
        self._chk(symnmf_batched_set_factors(self.h, p, _ptr(H0), _ptr(W0)))

    def factors(self, p):
        import torch

        H = torch.empty((self.ns[p], self.R * self.ks[p]), dtype=torch.float32, device="cuda")
        W = torch.empty_like(H)
        self._chk(symnmf_batched_get_factors(self.h, p, _ptr(H), _ptr(W)))
        return H, W

    def sweep(self, nsweeps, record=True):
        import numpy as np

        PR = self.nprob * self.R
        obj = np.zeros((max(nsweeps, 1), PR)) if record else None
        self._chk(symnmf_batched_sweep(self.h, nsweeps, obj.ctypes.data_as(_DP) if record else None))
        return obj[:nsweeps] if record else None

    def info(self):
        a, b, t = C.c_int(), C.c_int(), C.c_double()
        self._chk(symnmf_batched_info(self.h, C.byref(a), C.byref(b), C.byref(t)))
        return dict(stages=a.value, ctas_per_sm=b.value, product_ms=t.value)


class MLP:
    """Warm-start network (wraps symnmf_mlp_*): rows of normalised X Omega -> H0 rows."""

    def __init__(self, dims=(74, 256, 256, 32), seed=0, stream=None):
        h = C.c_void_p()
        st = symnmf_mlp_create(dims[0], dims[1], dims[2], dims[3], seed, _stream(stream), C.byref(h))
        if st != OK:
            raise SymNMFError(st, "symnmf_mlp_create")
        self.h, self.dims = h, tuple(dims)
        self.count = int(symnmf_mlp_param_count(h))
        self.t = 0

    def close(self):
        if getattr(self, "h", None):
            symnmf_mlp_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def params(self):
        import numpy as np

        out = np.zeros(self.count, dtype=np.float32)
        check(symnmf_mlp_get_params(self.h, out.ctypes.data_as(C.c_void_p), self.count))
        return out

    def set_params(self, flat):
        import numpy as np

        arr = np.ascontiguousarray(flat, dtype=np.float32)
        check(symnmf_mlp_set_params(self.h, arr.ctypes.data_as(C.c_void_p), self.count))

    def unflatten(self, flat):
        d = self.dims
        out, o = [], 0
        for a, b in zip(d[:-1], d[1:]):
            out.append(flat[o:o + a * b].reshape(a, b))
            o += a * b
            out.append(flat[o:o + b])
            o += b
        return out

    def forward(self, x):
        import torch

        out = torch.empty((x.shape[0], self.dims[3]), dtype=torch.float32, device=x.device)
        check(symnmf_mlp_forward(self.h, _ptr(x), x.shape[0], _ptr(out)))
        return out

    def loss_grad(self, x, Hstar, want_grads=False):
        import torch

        g = torch.empty(self.count, dtype=torch.float32, device=x.device) if want_grads else None
        loss = C.c_double()
        check(symnmf_mlp_loss_grad(self.h, _ptr(x), _ptr(Hstar), x.shape[0], _ptr(g), C.byref(loss)))
        return (loss.value, g) if want_grads else loss.value

    def adam(self, lr=1e-3):
        self.t += 1
        check(symnmf_mlp_adam(self.h, C.c_float(lr), self.t))

    def warm_start(self, solver, features=None):
        check(symnmf_warm_start(solver.h, self.h, _ptr(features)), solver.h)


def dense_xf(X, F, *, row_scale=None, gemm=GEMM_AUTO, N=None, stream=None):
    """Y = X F with the library's dense product kernels (X float64/float32/bfloat16/uint8-E4M3)."""
    import torch

    n = X.shape[0]
    N = N or F.shape[1]
    Y = torch.empty((n, N), dtype=torch.float32, device=X.device)
    fmt = _FMT_OF_DTYPE[str(X.dtype)]
    st = symnmf_dense_xf(fmt, _ptr(X), X.stride(0), _ptr(row_scale), n, _ptr(F), F.stride(0), N, _ptr(Y), N,
                         gemm, _stream(stream))
    check(st)
    return Y


def csr_xf(row_ptr, col, val, F, stream=None):
    import torch

    n = row_ptr.numel() - 1
    N = F.shape[1]
    Y = torch.empty((n, N), dtype=torch.float32, device=F.device)
    check(symnmf_csr_xf(_ptr(row_ptr), _ptr(col), _ptr(val), n, _ptr(F), N, _ptr(Y), _stream(stream)))
    return Y


def profile_standalone(enable=True):
    """Time the kernel of every standalone tensor-core product (dense_xf) with CUDA events."""
    check(symnmf_profile_standalone(1 if enable else 0))


def profile_standalone_read():
    """(total kernel ms, launches, FLOPs, algorithmic bytes) since the last read; resets the record."""
    t, n, f, b = C.c_double(), C.c_int64(), C.c_double(), C.c_double()
    check(symnmf_profile_standalone_read(C.byref(t), C.byref(n), C.byref(f), C.byref(b)))
    return t.value, n.value, f.value, b.value


def gram(F, stream=None):
    import torch

    n, N = F.shape
    G = torch.empty((N, N), dtype=torch.float64, device=F.device)
    check(symnmf_gram(_ptr(F), n, N, _ptr(G), _stream(stream)))
    return G


def cholesky(G, shift=0.0, stream=None):
    """(R, R^{-1}) of G + shift I by the library's FP64 block Cholesky (raises ENOTSPD)."""
    import torch

    k = G.shape[0]
    R = torch.empty((k, k), dtype=torch.float64, device=G.device)
    Ri = torch.empty_like(R)
    check(symnmf_cholesky(_ptr(G), k, float(shift), _ptr(R), _ptr(Ri), _stream(stream)))
    return R, Ri


def gaussian(n, l, seed, stream=None):
    import torch

    out = torch.empty((n, l), dtype=torch.float32, device="cuda")
    check(symnmf_gaussian(_ptr(out), n, l, seed, _stream(stream)))
    return out


def quantize_fp8(X, stream=None):
    import torch

    n = X.shape[0]
    ld8 = (n + 15) // 16 * 16
    x8 = torch.empty((n, ld8), dtype=torch.uint8, device=X.device)
    rs = torch.empty(n, dtype=torch.float32, device=X.device)
    check(symnmf_quantize_fp8(_ptr(X), n, X.stride(0), _ptr(x8), ld8, _ptr(rs), _stream(stream)))
    return x8, rs


def convert_bf16(X, stream=None):
    import torch

    n = X.shape[0]
    ldb = (n + 7) // 8 * 8
    xb = torch.empty((n, ldb), dtype=torch.bfloat16, device=X.device)
    check(symnmf_convert_bf16(_ptr(X), n, X.stride(0), _ptr(xb), ldb, _stream(stream)))
    return xb
