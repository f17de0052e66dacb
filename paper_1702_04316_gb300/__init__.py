"""Python binding of libnuma, the GB300 HEVI 1D-IMEX library (C ABI in include/numa.h).

Argument marshalling only: every step of the method runs in the library's CUDA kernels.
PyTorch supplies device memory and the current CUDA stream.  There is no fallback: if
``libnuma.so`` has not been built (``python -m paper_1702_04316_gb300.build``), importing
the library raises.
"""
import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libnuma.so")

NUMA_OK = 0
ERRORS = {
    1: "NUMA_ERR_ARG", 2: "NUMA_ERR_CUDA", 3: "NUMA_ERR_OOM", 4: "NUMA_ERR_NOT_FACTORED",
    5: "NUMA_ERR_PIVOT", 6: "NUMA_ERR_NONFINITE", 7: "NUMA_ERR_TIMEOUT", 8: "NUMA_ERR_SCRATCH",
}
Q_NCOL, Q_M, Q_NNODE, Q_NELEM, Q_HALF_BAND, Q_FACTOR_BYTES, Q_WORKSPACE_BYTES, Q_FACTORED, Q_N, \
    Q_PRECISION = range(10)
PRECISIONS = {"fp64": 0, "mixed": 1}

# Every symbol include/numa.h declares (checked by tests/test_abi.py).
EXPORTS = (
    "numa_init", "numa_init_ex", "numa_destroy", "numa_set_stream", "numa_rhs_explicit", "numa_factor_columns",
    "numa_solve_columns", "numa_step_imex1d", "numa_imex_stage", "numa_step_explicit_rk",
    "numa_run_host", "numa_connectivity", "numa_column_factors", "numa_reference_levels",
    "numa_count_nonfinite", "numa_status", "numa_query", "numa_last_error",
    "numa_rk35_coefficients", "numa_ark2_tableau", "numa_profile", "numa_profile_read",
    "numa_rhs_explicit_static", "numa_batch_init", "numa_batch_destroy", "numa_batch_layout",
    "numa_batch_step_imex1d", "numa_batch_set_graph", "numa_batch_tuning",
    "numa_batch_member_query", "numa_batch_reference_levels", "numa_batch_last_error",
)
K_PRESSURE, K_RHS, K_STAGE, K_SOLVE, K_FACTOR = range(5)


class Options(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int), ("refine_iters", ctypes.c_int)]


class MeshDesc(ctypes.Structure):
    _fields_ = [("nex", ctypes.c_int), ("ney", ctypes.c_int), ("nez", ctypes.c_int),
                ("Lx", ctypes.c_double), ("Ly", ctypes.c_double), ("Lz", ctypes.c_double),
                ("theta_s", ctypes.c_double), ("n_bv", ctypes.c_double)]


_lib = None


def lib():
    """Load libnuma.so (raises if it is missing)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("libnuma.so not built: run python -m paper_1702_04316_gb300.build")
        L = ctypes.CDLL(LIB_PATH)
        P, I, D, LL = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_longlong
        sig = {
            "numa_init": (I, [ctypes.POINTER(MeshDesc), I, D, P, ctypes.POINTER(P)]),
            "numa_init_ex": (I, [ctypes.POINTER(MeshDesc), I, D, ctypes.POINTER(Options), P,
                                 ctypes.POINTER(P)]),
            "numa_destroy": (None, [P]),
            "numa_set_stream": (I, [P, P]),
            "numa_rhs_explicit": (I, [P, P, P]),
            "numa_factor_columns": (I, [P, D]),
            "numa_solve_columns": (I, [P, P, P]),
            "numa_step_imex1d": (I, [P, P, P, I]),
            "numa_imex_stage": (I, [P, I, P, P, P, P, P]),
            "numa_step_explicit_rk": (I, [P, P, P, D, I]),
            "numa_run_host": (I, [P, I, P, P, I, D]),
            "numa_profile": (I, [P, I]),
            "numa_profile_read": (I, [P, I, ctypes.POINTER(D), ctypes.POINTER(LL)]),
            "numa_connectivity": (I, [P, P, P]),
            "numa_column_factors": (I, [P, LL, P]),
            "numa_reference_levels": (I, [P, P]),
            "numa_count_nonfinite": (I, [P, P, LL, ctypes.POINTER(LL)]),
            "numa_status": (I, [P, ctypes.POINTER(I)]),
            "numa_query": (I, [P, I, ctypes.POINTER(LL)]),
            "numa_last_error": (ctypes.c_char_p, [P]),
            "numa_rk35_coefficients": (None, [P, P]),
            "numa_ark2_tableau": (None, [P, P, P]),
            "numa_rhs_explicit_static": (I, [ctypes.POINTER(MeshDesc), I, P, P, P]),
            "numa_batch_init": (I, [ctypes.POINTER(MeshDesc), P, P, I, P, ctypes.POINTER(P)]),
            "numa_batch_destroy": (None, [P]),
            "numa_batch_layout": (I, [P, P]),
            "numa_batch_step_imex1d": (I, [P, P, P, I]),
            "numa_batch_set_graph": (I, [P, I]),
            "numa_batch_tuning": (I, [P, I, ctypes.POINTER(I), ctypes.POINTER(I)]),
            "numa_batch_member_query": (I, [P, I, I, ctypes.POINTER(LL)]),
            "numa_batch_reference_levels": (I, [P, I, P]),
            "numa_batch_last_error": (ctypes.c_char_p, [P]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


class NumaError(RuntimeError):
    pass


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


class Numa:
    """One mesh, one reference state, one IMEX time step size (a numa_ctx)."""

    def __init__(self, nex, ney, nez, Lx, Ly, Lz, N, dt=0.0, theta_s=300.0, n_bv=0.0,
                 stream=None, precision="fp64", refine_iters=1):
        import torch
        self._torch = torch
        L = lib()
        self._desc = MeshDesc(nex, ney, nez, Lx, Ly, Lz, theta_s, n_bv)
        s = torch.cuda.current_stream() if stream is None else stream
        self._stream = s
        h = ctypes.c_void_p()
        self._opt = Options(PRECISIONS[precision], int(refine_iters))
        rc = L.numa_init_ex(ctypes.byref(self._desc), N, float(dt), ctypes.byref(self._opt),
                            ctypes.c_void_p(s.cuda_stream), ctypes.byref(h))
        if rc != NUMA_OK:
            raise NumaError("numa_init failed: %s" % ERRORS.get(rc, rc))
        self._h = h
        self.N = N
        self.dt = float(dt)
        self.precision = precision
        self.ncol = self.query(Q_NCOL)
        self.M = self.query(Q_M)
        self.nnode = self.query(Q_NNODE)
        self.nelem = self.query(Q_NELEM)

    # -- plumbing ---------------------------------------------------------------------
    def _check(self, rc, what):
        if rc != NUMA_OK:
            msg = lib().numa_last_error(self._h).decode()
            raise NumaError("%s: %s (%s)" % (what, ERRORS.get(rc, rc), msg))

    def _state(self, t, n=None):
        n = 5 * self.nnode if n is None else n
        torch = self._torch
        if not (t.is_cuda and t.dtype == torch.float64 and t.is_contiguous() and t.numel() == n):
            raise ValueError("expected a contiguous float64 CUDA tensor of %d values" % n)
        return t

    def empty_state(self):
        return self._torch.empty(5, self.nnode, dtype=self._torch.float64, device="cuda")

    def close(self):
        if getattr(self, "_h", None):
            lib().numa_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def query(self, what):
        v = ctypes.c_longlong()
        self._check(lib().numa_query(self._h, what, ctypes.byref(v)), "numa_query")
        return v.value

    # -- the method -------------------------------------------------------------------
    def rhs_explicit(self, q, out=None):
        self._state(q)
        out = self._torch.empty_like(q) if out is None else self._state(out)
        self._check(lib().numa_rhs_explicit(self._h, _ptr(q), _ptr(out)), "numa_rhs_explicit")
        return out

    def factor_columns(self, dt):
        self._check(lib().numa_factor_columns(self._h, float(dt)), "numa_factor_columns")
        self.dt = float(dt)

    def solve_columns(self, b, x=None):
        n = self.ncol * self.M
        self._state(b, n)
        x = self._torch.empty_like(b) if x is None else self._state(x, n)
        self._check(lib().numa_solve_columns(self._h, _ptr(b), _ptr(x)), "numa_solve_columns")
        return x

    def step_imex1d(self, q_in, q_out=None, nsteps=1):
        self._state(q_in)
        q_out = q_in if q_out is None else self._state(q_out)
        self._check(lib().numa_step_imex1d(self._h, _ptr(q_in), _ptr(q_out), int(nsteps)),
                    "numa_step_imex1d")
        return q_out

    def imex_stage(self, stage, qn, R1, R2=None, q2=None, out=None):
        out = self._torch.empty_like(qn) if out is None else self._state(out)
        self._check(lib().numa_imex_stage(self._h, int(stage), _ptr(qn), _ptr(R1), _ptr(R2),
                                          _ptr(q2), _ptr(out)), "numa_imex_stage")
        return out

    def step_explicit_rk(self, q_in, dt, q_out=None, nsteps=1):
        self._state(q_in)
        q_out = q_in if q_out is None else self._state(q_out)
        self._check(lib().numa_step_explicit_rk(self._h, _ptr(q_in), _ptr(q_out), float(dt),
                                                int(nsteps)), "numa_step_explicit_rk")
        return q_out

    def run_host(self, method, q_in, nsteps, dt=0.0, q_out=None):
        """q_in, q_out: contiguous float64 CPU tensors (5, nnode), ideally pinned;
        q_out defaults to q_in (updated in place)."""
        q_out = q_in if q_out is None else q_out
        for t in (q_in, q_out):
            if t.is_cuda or not t.is_contiguous() or t.numel() != 5 * self.nnode:
                raise ValueError("expected contiguous CPU float64 tensors")
        self._check(lib().numa_run_host(self._h, int(method), ctypes.c_void_p(q_in.data_ptr()),
                                        ctypes.c_void_p(q_out.data_ptr()), int(nsteps), float(dt)),
                    "numa_run_host")
        return q_out

    def profile(self, enable):
        self._check(lib().numa_profile(self._h, 1 if enable else 0), "numa_profile")

    def profile_read(self, kind):
        t, n = ctypes.c_double(), ctypes.c_longlong()
        self._check(lib().numa_profile_read(self._h, int(kind), ctypes.byref(t), ctypes.byref(n)),
                    "numa_profile_read")
        return t.value, n.value

    # -- inspection -------------------------------------------------------------------
    def connectivity(self):
        torch = self._torch
        nq3 = (self.N + 1) ** 3
        l2g = torch.empty(self.nelem * nq3, dtype=torch.int32, device="cuda")
        g2l = torch.empty(self.nnode * 8, dtype=torch.int32, device="cuda")
        self._check(lib().numa_connectivity(self._h, _ptr(l2g), _ptr(g2l)), "numa_connectivity")
        return l2g.view(self.nelem, self.N + 1, self.N + 1, self.N + 1), g2l.view(self.nnode, 8)

    def column_factors(self, col):
        W = 4 * self.N + 1
        out = np.empty((self.M, W), dtype=np.float64)
        self._check(lib().numa_column_factors(self._h, int(col), out.ctypes.data_as(ctypes.c_void_p)),
                    "numa_column_factors")
        return out

    def reference_levels(self):
        out = np.empty((8, self.M), dtype=np.float64)
        self._check(lib().numa_reference_levels(self._h, out.ctypes.data_as(ctypes.c_void_p)),
                    "numa_reference_levels")
        keys = ("z", "rho0", "theta0", "P0", "G0", "H0", "drho0", "dtheta0")
        return dict(zip(keys, out))

    def count_nonfinite(self, x):
        c = ctypes.c_longlong()
        self._check(lib().numa_count_nonfinite(self._h, _ptr(x), x.numel(), ctypes.byref(c)),
                    "numa_count_nonfinite")
        return c.value

    def status(self):
        s = ctypes.c_int()
        self._check(lib().numa_status(self._h, ctypes.byref(s)), "numa_status")
        return s.value


class Batch:
    """An ensemble of independent members (numa_batch): meshes is a list of
    (nex, ney, nez, Lx, Ly, Lz) tuples, N and dt lists of the same length."""

    def __init__(self, meshes, N, dt, theta_s=300.0, n_bv=0.0, stream=None):
        import torch
        self._torch = torch
        n = len(meshes)
        descs = (MeshDesc * n)(*[MeshDesc(*m, theta_s, n_bv) for m in meshes])
        Ns = (ctypes.c_int * n)(*[int(v) for v in N])
        dts = (ctypes.c_double * n)(*[float(v) for v in dt])
        s = torch.cuda.current_stream() if stream is None else stream
        h = ctypes.c_void_p()
        rc = lib().numa_batch_init(descs, ctypes.cast(Ns, ctypes.c_void_p), ctypes.cast(dts, ctypes.c_void_p),
                                   n, ctypes.c_void_p(s.cuda_stream), ctypes.byref(h))
        if rc != NUMA_OK:
            raise NumaError("numa_batch_init failed: %s" % ERRORS.get(rc, rc))
        self._h = h
        self.n = n
        off = (ctypes.c_longlong * (n + 1))()
        self._check(lib().numa_batch_layout(self._h, ctypes.cast(off, ctypes.c_void_p)), "layout")
        self.offsets = list(off)
        self.total = self.offsets[-1]

    def _check(self, rc, what):
        if rc != NUMA_OK:
            raise NumaError("%s: %s (%s)" % (what, ERRORS.get(rc, rc),
                                             lib().numa_batch_last_error(self._h).decode()))

    def close(self):
        if getattr(self, "_h", None):
            lib().numa_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def empty_state(self):
        return self._torch.empty(self.total, dtype=self._torch.float64, device="cuda")

    def member(self, state, m):
        """View of member m in a packed state: (5, nnode)."""
        return state[self.offsets[m]:self.offsets[m + 1]].view(5, -1)

    def step_imex1d(self, q_in, q_out=None, nsteps=1):
        q_out = q_in if q_out is None else q_out
        self._check(lib().numa_batch_step_imex1d(self._h, _ptr(q_in), _ptr(q_out), int(nsteps)), "step")
        return q_out

    def set_graph(self, enable):
        self._check(lib().numa_batch_set_graph(self._h, 1 if enable else 0), "set_graph")

    def tuning(self):
        """{N: {"rhs_threads_per_cta", "stage_columns_per_cta"}} for the orders present."""
        out = {}
        for n in (4, 5, 6):
            a, b = ctypes.c_int(), ctypes.c_int()
            self._check(lib().numa_batch_tuning(self._h, n, ctypes.byref(a), ctypes.byref(b)), "tuning")
            if a.value:
                out[n] = {"rhs_threads_per_cta": a.value, "stage_columns_per_cta": b.value}
        return out

    def member_query(self, m, what):
        v = ctypes.c_longlong()
        self._check(lib().numa_batch_member_query(self._h, int(m), int(what), ctypes.byref(v)), "query")
        return v.value

    def reference_levels(self, m):
        M = self.member_query(m, Q_M)
        out = np.empty((8, M), dtype=np.float64)
        self._check(lib().numa_batch_reference_levels(self._h, int(m), out.ctypes.data_as(ctypes.c_void_p)),
                    "reference_levels")
        return dict(zip(("z", "rho0", "theta0", "P0", "G0", "H0", "drho0", "dtheta0"), out))


def rhs_explicit_static(nex, ney, nez, Lx, Ly, Lz, N, q, out, theta_s=300.0, n_bv=0.0,
                        stream=None):
    """numa_rhs_explicit_static: the explicit RHS without any device allocation (for
    callers that must not allocate at the point of the call); returns the NUMA_* code."""
    import torch
    s = torch.cuda.current_stream() if stream is None else stream
    d = MeshDesc(nex, ney, nez, Lx, Ly, Lz, theta_s, n_bv)
    return lib().numa_rhs_explicit_static(ctypes.byref(d), int(N), _ptr(q), _ptr(out),
                                          ctypes.c_void_p(s.cuda_stream))


def rk35_coefficients():
    a = np.empty(5)
    b = np.empty(5)
    lib().numa_rk35_coefficients(a.ctypes.data_as(ctypes.c_void_p), b.ctypes.data_as(ctypes.c_void_p))
    return a, b


def ark2_tableau():
    a, at, b = np.empty(9), np.empty(9), np.empty(3)
    lib().numa_ark2_tableau(a.ctypes.data_as(ctypes.c_void_p), at.ctypes.data_as(ctypes.c_void_p),
                            b.ctypes.data_as(ctypes.c_void_p))
    return a.reshape(3, 3), at.reshape(3, 3), b
