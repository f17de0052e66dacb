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
NUMA_ERR_ARG, NUMA_ERR_CUDA, NUMA_ERR_OOM, NUMA_ERR_NOT_FACTORED, NUMA_ERR_PIVOT, \
    NUMA_ERR_NONFINITE, NUMA_ERR_TIMEOUT, NUMA_ERR_SCRATCH = range(1, 9)
ERRORS = {
    1: "NUMA_ERR_ARG", 2: "NUMA_ERR_CUDA", 3: "NUMA_ERR_OOM", 4: "NUMA_ERR_NOT_FACTORED",
    5: "NUMA_ERR_PIVOT", 6: "NUMA_ERR_NONFINITE", 7: "NUMA_ERR_TIMEOUT", 8: "NUMA_ERR_SCRATCH",
}
Q_NCOL, Q_M, Q_NNODE, Q_NELEM, Q_HALF_BAND, Q_FACTOR_BYTES, Q_WORKSPACE_BYTES, Q_FACTORED, Q_N, \
    Q_PRECISION, Q_COLUMN_FORM, Q_SCHEME, Q_IMEX = range(13)
PRECISIONS = {"fp64": 0, "mixed": 1, "rhs32": 2, "df": 3}
COLUMN_FORMS = {"schur": 0, "standard": 1}
SCHEMES = {"ark2": 0, "ark3": 1, "ark4": 2, "ark5": 3}
MAX_STAGES = 8
IMEX = {"1d": 0, "3d": 1}
PRECONDS = {"pbno": 0, "column": 1}

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
    "numa_rhs_tlm", "numa_rhs_adjoint", "numa_solve_columns_transposed", "numa_imex_stage_adjoint",
    "numa_step_imex1d_tlm", "numa_step_imex1d_adjoint", "numa_imex1d_forward_checkpointed",
    "numa_imex1d_adjoint_checkpointed", "numa_ark3_tableau", "numa_ark_tableau", "numa_imex_stage_s",
    "numa_schur3d_apply",
    "numa_solve_schur3d", "numa_imex3d_stage", "numa_step_imex3d", "numa_imex3d_info",
    "numa_part_plan", "numa_part_columns", "numa_gather_columns", "numa_scatter_columns",
    "numa_step_phase", "numa_step_buffers", "numa_convert_f64_f32", "numa_convert_f32_f64",
    "numa_reciprocal",
)
K_PRESSURE, K_RHS, K_STAGE, K_SOLVE, K_FACTOR, K_RHS_TLM, K_RHS_ADJ, K_STAGE_ADJ, K_SCHUR3D = range(9)


class Options(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int), ("refine_iters", ctypes.c_int),
                ("column_form", ctypes.c_int), ("scheme", ctypes.c_int), ("imex", ctypes.c_int),
                ("pbno_order", ctypes.c_int), ("krylov_max_iters", ctypes.c_int),
                ("krylov_tol", ctypes.c_double), ("precond", ctypes.c_int)]


class MeshDesc(ctypes.Structure):
    _fields_ = [("nex", ctypes.c_int), ("ney", ctypes.c_int), ("nez", ctypes.c_int),
                ("Lx", ctypes.c_double), ("Ly", ctypes.c_double), ("Lz", ctypes.c_double),
                ("theta_s", ctypes.c_double), ("n_bv", ctypes.c_double)]


PART_MAX_NEIGH = 8


class PartDesc(ctypes.Structure):
    _fields_ = [("px", ctypes.c_int), ("py", ctypes.c_int), ("rank", ctypes.c_int)]


class PartInfo(ctypes.Structure):
    _fields_ = [("ex0", ctypes.c_int), ("ex1", ctypes.c_int), ("ey0", ctypes.c_int), ("ey1", ctypes.c_int),
                ("wx0", ctypes.c_int), ("wx1", ctypes.c_int), ("wy0", ctypes.c_int), ("wy1", ctypes.c_int),
                ("window", MeshDesc),
                ("own_x0", ctypes.c_int), ("own_x1", ctypes.c_int), ("own_y0", ctypes.c_int),
                ("own_y1", ctypes.c_int), ("nneigh", ctypes.c_int),
                ("neigh", ctypes.c_int * PART_MAX_NEIGH), ("nsend", ctypes.c_int * PART_MAX_NEIGH),
                ("nrecv", ctypes.c_int * PART_MAX_NEIGH)]


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
            "numa_ark3_tableau": (None, [P, P, P]),
            "numa_ark_tableau": (I, [I, P, P, P, ctypes.POINTER(I)]),
            "numa_imex_stage_s": (I, [P, I, P, P, P, P]),
            "numa_schur3d_apply": (I, [P, P, P]),
            "numa_solve_schur3d": (I, [P, P, P, ctypes.POINTER(I)]),
            "numa_imex3d_stage": (I, [P, I, P, P, P, P, P, ctypes.POINTER(I)]),
            "numa_step_imex3d": (I, [P, P, P, I]),
            "numa_imex3d_info": (I, [P, ctypes.POINTER(D), ctypes.POINTER(D), P, ctypes.POINTER(LL)]),
            "numa_rhs_explicit_static": (I, [ctypes.POINTER(MeshDesc), I, P, P, P]),
            "numa_batch_init": (I, [ctypes.POINTER(MeshDesc), P, P, I, P, ctypes.POINTER(P)]),
            "numa_batch_destroy": (None, [P]),
            "numa_batch_layout": (I, [P, P]),
            "numa_batch_step_imex1d": (I, [P, P, P, I]),
            "numa_batch_set_graph": (I, [P, I]),
            "numa_batch_tuning": (I, [P, I, ctypes.POINTER(I), ctypes.POINTER(I), ctypes.POINTER(I)]),
            "numa_batch_member_query": (I, [P, I, I, ctypes.POINTER(LL)]),
            "numa_batch_reference_levels": (I, [P, I, P]),
            "numa_batch_last_error": (ctypes.c_char_p, [P]),
            "numa_rhs_tlm": (I, [P, P, P, P]),
            "numa_rhs_adjoint": (I, [P, P, P, P]),
            "numa_solve_columns_transposed": (I, [P, P, P]),
            "numa_imex_stage_adjoint": (I, [P, I, P, P, P, P, P]),
            "numa_step_imex1d_tlm": (I, [P, P, P, P, P, I]),
            "numa_step_imex1d_adjoint": (I, [P, P, P, P]),
            "numa_imex1d_forward_checkpointed": (I, [P, P, P, I, I, P]),
            "numa_imex1d_adjoint_checkpointed": (I, [P, P, I, I, P, P, P]),
            "numa_part_plan": (I, [ctypes.POINTER(MeshDesc), I, ctypes.POINTER(PartDesc),
                                   ctypes.POINTER(PartInfo)]),
            "numa_part_columns": (I, [ctypes.POINTER(MeshDesc), I, ctypes.POINTER(PartDesc), I, P, P]),
            "numa_gather_columns": (I, [P, P, I, P, LL, P]),
            "numa_scatter_columns": (I, [P, P, I, P, LL, P]),
            "numa_step_phase": (I, [P, I, P, P]),
            "numa_step_buffers": (I, [P, ctypes.POINTER(P), ctypes.POINTER(P), ctypes.POINTER(P),
                                      ctypes.POINTER(I)]),
            "numa_convert_f64_f32": (I, [P, P, LL, P]),
            "numa_convert_f32_f64": (I, [P, P, LL, P]),
            "numa_reciprocal": (I, [P, P, LL, P]),
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
                 stream=None, precision="fp64", refine_iters=1, column_form="schur",
                 scheme="ark2", imex="1d", pbno_order=2, krylov_tol=1e-12, krylov_max_iters=500,
                 precond="pbno"):
        import torch
        self._torch = torch
        L = lib()
        self._desc = MeshDesc(nex, ney, nez, Lx, Ly, Lz, theta_s, n_bv)
        s = torch.cuda.current_stream() if stream is None else stream
        self._stream = s
        h = ctypes.c_void_p()
        self._opt = Options(PRECISIONS[precision], int(refine_iters), COLUMN_FORMS[column_form],
                            SCHEMES[scheme], IMEX[imex], int(pbno_order), int(krylov_max_iters),
                            float(krylov_tol), PRECONDS[precond])
        rc = L.numa_init_ex(ctypes.byref(self._desc), N, float(dt), ctypes.byref(self._opt),
                            ctypes.c_void_p(s.cuda_stream), ctypes.byref(h))
        if rc != NUMA_OK:
            raise NumaError("numa_init failed: %s" % ERRORS.get(rc, rc))
        self._h = h
        self.N = N
        self.dt = float(dt)
        self.precision = precision
        self.column_form = column_form
        self.scheme = scheme
        self.imex = imex
        self.pbno_order = int(pbno_order)
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

    # -- phased step and halo messages (horizontal partition over several GPUs) --------
    def step_phase(self, phase, q_n, q_out=None):
        """numa_step_phase: phase 0 (R1, stage 2), 1 (R2, stage 3) or 2 (final update into
        q_out) of one ARK2 step."""
        self._state(q_n)
        if q_out is not None:
            self._state(q_out)
        self._check(lib().numa_step_phase(self._h, int(phase), _ptr(q_n), _ptr(q_out)),
                    "numa_step_phase")
        return q_out

    def step_buffers(self):
        """numa_step_buffers: (q2, q3, P', P' fused) as tensors viewing the context's
        workspace (q2, q3 of shape (5, nnode); P' of shape (nnode,) or None)."""
        q2, q3, pp = ctypes.c_void_p(), ctypes.c_void_p(), ctypes.c_void_p()
        fused = ctypes.c_int()
        self._check(lib().numa_step_buffers(self._h, ctypes.byref(q2), ctypes.byref(q3),
                                            ctypes.byref(pp), ctypes.byref(fused)), "numa_step_buffers")
        view = lambda p, n: _device_view(self._torch, p.value, n) if p.value else None
        q2t, q3t = view(q2, 5 * self.nnode), view(q3, 5 * self.nnode)
        return (q2t.view(5, self.nnode), q3t.view(5, self.nnode), view(pp, self.nnode),
                bool(fused.value))

    def gather_columns(self, fields, cols, buf):
        """numa_gather_columns: the listed columns of `fields` (tensors of ncol*M doubles)
        into buf (len(fields) * len(cols) * M doubles); cols: CUDA int32 tensor."""
        arr = (ctypes.c_void_p * len(fields))(*[f.data_ptr() for f in fields])
        self._check(lib().numa_gather_columns(self._h, arr, len(fields), _ptr(cols), cols.numel(),
                                              _ptr(buf)), "numa_gather_columns")

    def scatter_columns(self, fields, cols, buf):
        """numa_scatter_columns: buf into the listed columns of `fields`."""
        arr = (ctypes.c_void_p * len(fields))(*[f.data_ptr() for f in fields])
        self._check(lib().numa_scatter_columns(self._h, arr, len(fields), _ptr(cols), cols.numel(),
                                               _ptr(buf)), "numa_scatter_columns")

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

    def imex_stage_s(self, stage, qn, Rs, Qs=(), out=None):
        """Stage `stage` of the context's scheme from q^n, Rs = [R(q(1)), ..., R(q(i-1))] and
        Qs = [q(2), ..., q(i-1)] (numa_imex_stage_s)."""
        for t in (qn, *Rs, *Qs):
            self._state(t)
        out = self._torch.empty_like(qn) if out is None else self._state(out)
        Ra = (ctypes.c_void_p * max(1, len(Rs)))(*[t.data_ptr() for t in Rs])
        Qa = (ctypes.c_void_p * max(1, len(Qs)))(*[t.data_ptr() for t in Qs])
        self._check(lib().numa_imex_stage_s(self._h, int(stage), _ptr(qn), Ra,
                                            Qa if len(Qs) else None, _ptr(out)),
                    "numa_imex_stage_s")
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

    # -- differentiation form -------------------------------------------------------
    def rhs_tlm(self, q, dq, out=None):
        """R'(q) dq."""
        self._state(q)
        self._state(dq)
        out = self._torch.empty_like(q) if out is None else self._state(out)
        self._check(lib().numa_rhs_tlm(self._h, _ptr(q), _ptr(dq), _ptr(out)), "numa_rhs_tlm")
        return out

    def rhs_adjoint(self, q, lam, out=None):
        """R'(q)^T lam."""
        self._state(q)
        self._state(lam)
        out = self._torch.empty_like(q) if out is None else self._state(out)
        self._check(lib().numa_rhs_adjoint(self._h, _ptr(q), _ptr(lam), _ptr(out)),
                    "numa_rhs_adjoint")
        return out

    def solve_columns_transposed(self, b, x=None):
        n = self.ncol * self.M
        self._state(b, n)
        x = self._torch.empty_like(b) if x is None else self._state(x, n)
        self._check(lib().numa_solve_columns_transposed(self._h, _ptr(b), _ptr(x)),
                    "numa_solve_columns_transposed")
        return x

    def imex_stage_adjoint(self, stage, lam, qn_adj, R1_adj, R2_adj=None, q2_adj=None):
        """Adds the adjoints of the stage's inputs to qn_adj, R1_adj (and R2_adj, q2_adj)."""
        for t in (lam, qn_adj, R1_adj, R2_adj, q2_adj):
            if t is not None:
                self._state(t)
        self._check(lib().numa_imex_stage_adjoint(self._h, int(stage), _ptr(lam), _ptr(qn_adj),
                                                  _ptr(R1_adj), _ptr(R2_adj), _ptr(q2_adj)),
                    "numa_imex_stage_adjoint")

    def step_imex1d_tlm(self, q, dq, nsteps=1, q_out=None, dq_out=None):
        """(q^{n+nsteps}, its tangent along dq)."""
        self._state(q)
        self._state(dq)
        q_out = self._torch.empty_like(q) if q_out is None else self._state(q_out)
        dq_out = self._torch.empty_like(dq) if dq_out is None else self._state(dq_out)
        self._check(lib().numa_step_imex1d_tlm(self._h, _ptr(q), _ptr(dq), _ptr(q_out),
                                               _ptr(dq_out), int(nsteps)), "numa_step_imex1d_tlm")
        return q_out, dq_out

    def step_imex1d_adjoint(self, q, lam_next, lam=None):
        """(dq^{n+1}/dq^n)^T lam_next for the step taken from q."""
        self._state(q)
        self._state(lam_next)
        lam = self._torch.empty_like(q) if lam is None else self._state(lam)
        self._check(lib().numa_step_imex1d_adjoint(self._h, _ptr(q), _ptr(lam_next), _ptr(lam)),
                    "numa_step_imex1d_adjoint")
        return lam

    def forward_checkpointed(self, q0, nsteps, every, qT=None):
        """(q^T, checkpoints) of nsteps steps, the state kept before every `every`-th step."""
        self._state(q0)
        qT = self._torch.empty_like(q0) if qT is None else self._state(qT)
        nck = (int(nsteps) + int(every) - 1) // int(every)
        ckpt = self._torch.empty(nck, 5, self.nnode, dtype=self._torch.float64, device="cuda")
        self._check(lib().numa_imex1d_forward_checkpointed(self._h, _ptr(q0), _ptr(qT), int(nsteps),
                                                           int(every), _ptr(ckpt)),
                    "numa_imex1d_forward_checkpointed")
        return qT, ckpt

    def adjoint_checkpointed(self, ckpt, nsteps, every, lamT, lam0=None):
        """(dq^T/dq^0)^T lamT from the checkpoints of forward_checkpointed."""
        self._state(lamT)
        lam0 = self._torch.empty_like(lamT) if lam0 is None else self._state(lam0)
        work = self._torch.empty(3 * int(every), 5, self.nnode, dtype=self._torch.float64,
                                 device="cuda")
        self._check(lib().numa_imex1d_adjoint_checkpointed(self._h, _ptr(ckpt), int(nsteps),
                                                           int(every), _ptr(lamT), _ptr(lam0),
                                                           _ptr(work)),
                    "numa_imex1d_adjoint_checkpointed")
        return lam0

    def rhs_autograd(self, q):
        """R(q) as a differentiable torch operation: reverse mode through the adjoint
        kernels, forward mode (torch.autograd.forward_ad) through the TLM kernels."""
        return _functions()[0].apply(q, self)

    def trajectory(self, q0, nsteps, every=5):
        """q^T after nsteps HEVI steps as a differentiable torch operation.  Reverse mode
        keeps a checkpoint every `every` steps and recomputes each segment during the
        adjoint sweep; forward mode runs the TLM alongside the trajectory."""
        return _functions()[1].apply(q0, self, int(nsteps), int(every))

    # -- 3D-IMEX (Schur form, BiCGstab + polynomial preconditioner) -----------------------
    def schur3d_apply(self, P, out=None):
        self._state(P, self.nnode)
        out = self._torch.empty_like(P) if out is None else self._state(out, self.nnode)
        self._check(lib().numa_schur3d_apply(self._h, _ptr(P), _ptr(out)), "numa_schur3d_apply")
        return out

    def solve_schur3d(self, b, x=None):
        """(x, iterations) with S(x) = b."""
        self._state(b, self.nnode)
        x = self._torch.empty_like(b) if x is None else self._state(x, self.nnode)
        it = ctypes.c_int()
        self._check(lib().numa_solve_schur3d(self._h, _ptr(b), _ptr(x), ctypes.byref(it)),
                    "numa_solve_schur3d")
        return x, it.value

    def imex3d_stage(self, stage, qn, R1, R2=None, q2=None, out=None):
        """(q(stage), BiCGstab iterations)."""
        out = self._torch.empty_like(qn) if out is None else self._state(out)
        it = ctypes.c_int()
        self._check(lib().numa_imex3d_stage(self._h, int(stage), _ptr(qn), _ptr(R1), _ptr(R2),
                                            _ptr(q2), _ptr(out), ctypes.byref(it)),
                    "numa_imex3d_stage")
        return out, it.value

    def step_imex3d(self, q_in, q_out=None, nsteps=1):
        self._state(q_in)
        q_out = q_in if q_out is None else self._state(q_out)
        self._check(lib().numa_step_imex3d(self._h, _ptr(q_in), _ptr(q_out), int(nsteps)),
                    "numa_step_imex3d")
        return q_out

    def imex3d_info(self):
        """{"l_max", "lam_bar", "coeffs", "iters_last_step"}."""
        lm, lb, it = ctypes.c_double(), ctypes.c_double(), ctypes.c_longlong()
        c = np.zeros(self.pbno_order + 1)
        self._check(lib().numa_imex3d_info(self._h, ctypes.byref(lm), ctypes.byref(lb),
                                           c.ctypes.data_as(ctypes.c_void_p), ctypes.byref(it)),
                    "numa_imex3d_info")
        return {"l_max": lm.value, "lam_bar": lb.value, "coeffs": c, "iters_last_step": it.value}

    # -- inspection -------------------------------------------------------------------
    def connectivity(self):
        torch = self._torch
        nq3 = (self.N + 1) ** 3
        l2g = torch.empty(self.nelem * nq3, dtype=torch.int32, device="cuda")
        g2l = torch.empty(self.nnode * 8, dtype=torch.int32, device="cuda")
        self._check(lib().numa_connectivity(self._h, _ptr(l2g), _ptr(g2l)), "numa_connectivity")
        return l2g.view(self.nelem, self.N + 1, self.N + 1, self.N + 1), g2l.view(self.nnode, 8)

    def column_factors(self, col):
        """Band of one column's stored factors: (M, 4N+1) for the Schur form, (3M, 6N+3)
        for the standard form (level-interleaved unknowns)."""
        hb = self.query(Q_HALF_BAND)
        n = 3 * self.M if self.column_form == "standard" else self.M
        out = np.empty((n, 2 * hb + 1), dtype=np.float64)
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


_FUNCTIONS = None


def _functions():
    """The torch.autograd.Function classes (built on first use so that importing the
    binding does not import torch)."""
    global _FUNCTIONS
    if _FUNCTIONS is not None:
        return _FUNCTIONS
    import torch

    def _c(t):
        return t.contiguous() if t.dtype == torch.float64 else t.double().contiguous()

    class RHS(torch.autograd.Function):
        @staticmethod
        def forward(ctx, q, numa):
            ctx.numa = numa
            ctx.save_for_backward(q)
            ctx.save_for_forward(q)
            return numa.rhs_explicit(_c(q))

        @staticmethod
        def backward(ctx, lam):
            q, = ctx.saved_tensors
            return ctx.numa.rhs_adjoint(_c(q), _c(lam)), None

        @staticmethod
        def jvp(ctx, dq, _numa):
            q, = ctx.saved_tensors
            return ctx.numa.rhs_tlm(_c(q), _c(dq))

    class Trajectory(torch.autograd.Function):
        @staticmethod
        def forward(ctx, q0, numa, nsteps, every):
            qT, ckpt = numa.forward_checkpointed(_c(q0), nsteps, every)
            ctx.numa, ctx.nsteps, ctx.every, ctx.ckpt = numa, nsteps, every, ckpt
            ctx.save_for_forward(q0)
            return qT

        @staticmethod
        def backward(ctx, lamT):
            lam0 = ctx.numa.adjoint_checkpointed(ctx.ckpt, ctx.nsteps, ctx.every, _c(lamT))
            return lam0, None, None, None

        @staticmethod
        def jvp(ctx, dq0, *_):
            q0, = ctx.saved_tensors
            return ctx.numa.step_imex1d_tlm(_c(q0), _c(dq0), ctx.nsteps)[1]

    _FUNCTIONS = (RHS, Trajectory)
    return _FUNCTIONS


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
        """{N: {"rhs_threads_per_cta", "stage_columns_per_cta", "stage_threads_per_cta"}} for
        the orders present."""
        out = {}
        for n in (4, 5, 6):
            a, b, c = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
            self._check(lib().numa_batch_tuning(self._h, n, ctypes.byref(a), ctypes.byref(b),
                                                ctypes.byref(c)), "tuning")
            if a.value:
                out[n] = {"rhs_threads_per_cta": a.value, "stage_columns_per_cta": b.value,
                          "stage_threads_per_cta": c.value}
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


def _device_view(torch, ptr, n):
    """A float64 CUDA tensor of n values over device memory owned by a context (no copy;
    valid while the context lives)."""
    class _Arr:
        __cuda_array_interface__ = {"shape": (n,), "typestr": "<f8", "data": (ptr, False),
                                    "version": 3, "strides": None}
    return torch.as_tensor(_Arr(), device="cuda")


def part_plan(nex, ney, nez, Lx, Ly, Lz, N, px, py, rank, theta_s=300.0, n_bv=0.0):
    """numa_part_plan + numa_part_columns (host only, no GPU needed): the rank's rectangle,
    window (a MeshDesc-like dict) and, per neighbour, its rank and the send / receive column
    lists (numpy int32, window-local column ids)."""
    g = MeshDesc(nex, ney, nez, Lx, Ly, Lz, theta_s, n_bv)
    d = PartDesc(px, py, rank)
    info = PartInfo()
    rc = lib().numa_part_plan(ctypes.byref(g), int(N), ctypes.byref(d), ctypes.byref(info))
    if rc != NUMA_OK:
        raise NumaError("numa_part_plan: %s" % ERRORS.get(rc, rc))
    w = info.window
    out = {"own_elems": (info.ex0, info.ex1, info.ey0, info.ey1),
           "window_elems": (info.wx0, info.wx1, info.wy0, info.wy1),
           "window": dict(nex=w.nex, ney=w.ney, nez=w.nez, Lx=w.Lx, Ly=w.Ly, Lz=w.Lz,
                          theta_s=w.theta_s, n_bv=w.n_bv),
           "own_cols": (info.own_x0, info.own_x1, info.own_y0, info.own_y1),
           "neighbours": []}
    for k in range(info.nneigh):
        send = np.empty(info.nsend[k], dtype=np.int32)
        recv = np.empty(info.nrecv[k], dtype=np.int32)
        rc = lib().numa_part_columns(ctypes.byref(g), int(N), ctypes.byref(d), k,
                                     send.ctypes.data_as(ctypes.c_void_p),
                                     recv.ctypes.data_as(ctypes.c_void_p))
        if rc != NUMA_OK:
            raise NumaError("numa_part_columns: %s" % ERRORS.get(rc, rc))
        out["neighbours"].append({"rank": info.neigh[k], "send": send, "recv": recv})
    return out


def rhs_explicit_static(nex, ney, nez, Lx, Ly, Lz, N, q, out, theta_s=300.0, n_bv=0.0,
                        stream=None):
    """numa_rhs_explicit_static: the explicit RHS without any device allocation (for
    callers that must not allocate at the point of the call); returns the NUMA_* code."""
    import torch
    s = torch.cuda.current_stream() if stream is None else stream
    d = MeshDesc(nex, ney, nez, Lx, Ly, Lz, theta_s, n_bv)
    return lib().numa_rhs_explicit_static(ctypes.byref(d), int(N), _ptr(q), _ptr(out),
                                          ctypes.c_void_p(s.cuda_stream))


def convert(x, stream=None):
    """numa_convert_f64_f32 (x FP64) or numa_convert_f32_f64 (x FP32) on a contiguous device
    tensor: the library's integer-pipe conversions."""
    import torch
    if not (x.is_cuda and x.is_contiguous() and x.dtype in (torch.float64, torch.float32)):
        raise ValueError("convert: x must be a contiguous FP64 or FP32 CUDA tensor")
    s = torch.cuda.current_stream() if stream is None else stream
    if x.dtype == torch.float64:
        y = torch.empty(x.shape, dtype=torch.float32, device=x.device)
        fn = lib().numa_convert_f64_f32
    else:
        y = torch.empty(x.shape, dtype=torch.float64, device=x.device)
        fn = lib().numa_convert_f32_f64
    rc = fn(_ptr(x), _ptr(y), x.numel(), ctypes.c_void_p(s.cuda_stream))
    if rc != NUMA_OK:
        raise NumaError("convert: code %d" % rc)
    return y


def reciprocal(x, stream=None):
    """numa_reciprocal on a contiguous FP64 device tensor: 1 / x as the right-hand side
    computes it."""
    import torch
    if not (x.is_cuda and x.is_contiguous() and x.dtype == torch.float64):
        raise ValueError("reciprocal: x must be a contiguous FP64 CUDA tensor")
    s = torch.cuda.current_stream() if stream is None else stream
    y = torch.empty_like(x)
    rc = lib().numa_reciprocal(_ptr(x), _ptr(y), x.numel(), ctypes.c_void_p(s.cuda_stream))
    if rc != NUMA_OK:
        raise NumaError("reciprocal: code %d" % rc)
    return y


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


def ark_tableau(scheme):
    """(a, at, b) of a scheme ("ark2" .. "ark5") as the library evaluates it."""
    a, at, b = np.empty(MAX_STAGES ** 2), np.empty(MAX_STAGES ** 2), np.empty(MAX_STAGES)
    s = ctypes.c_int(0)
    rc = lib().numa_ark_tableau(SCHEMES[scheme], a.ctypes.data_as(ctypes.c_void_p),
                                at.ctypes.data_as(ctypes.c_void_p),
                                b.ctypes.data_as(ctypes.c_void_p), ctypes.byref(s))
    if rc != 0:
        raise ValueError("numa_ark_tableau: unknown scheme")
    n = s.value
    return a[:n * n].reshape(n, n), at[:n * n].reshape(n, n), b[:n].copy()


def ark3_tableau():
    a, at, b = np.empty(16), np.empty(16), np.empty(4)
    lib().numa_ark3_tableau(a.ctypes.data_as(ctypes.c_void_p), at.ctypes.data_as(ctypes.c_void_p),
                            b.ctypes.data_as(ctypes.c_void_p))
    return a.reshape(4, 4), at.reshape(4, 4), b
