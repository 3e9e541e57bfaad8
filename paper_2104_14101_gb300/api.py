"""Python front of the sks library: torch tensors in, torch tensors out.

Only argument marshalling lives here -- every step of the computation runs in
the CUDA kernels of ``libsks.so``.  Device memory (inputs, outputs and the
scratch workspaces the C ABI asks for) is allocated with torch; the current
torch stream is passed to every call.
"""
import ctypes as C

import torch

from . import _lib as L


def _stream(device=None):
    return C.c_void_p(torch.cuda.current_stream(device).cuda_stream)


def _ptr(t):
    return C.c_void_p(t.data_ptr()) if t is not None else C.c_void_p(None)


def _workspace(nbytes, device):
    return torch.empty(max(int(nbytes), 1), dtype=torch.uint8, device=device)


def make_problem(A, b, nu, lam):
    """Build the C problem struct from device tensors.

    A: (n, d) float64 or float32, rows contiguous (stride(1) == 1).
    b: (d,) or (d, k) float64 -- k right-hand sides.
    lam: (d,) float64, entries >= 1.
    Returns (problem_struct, b2d) where b2d is the column-major d x k copy kept alive.
    """
    if not A.is_cuda:
        raise ValueError("A must be a CUDA tensor")
    if A.dim() != 2 or (A.numel() > 0 and A.stride(1) != 1):
        raise ValueError("A must be 2-D with unit column stride")
    if A.dtype not in (torch.float64, torch.float32):
        raise ValueError("A must be float64 or float32")
    n, d = A.shape
    esz = A.element_size()
    if n > 0 and ((A.stride(0) * esz) % 16 != 0 or A.data_ptr() % 16 != 0 or (n == 1 and (d * esz) % 16 != 0)):
        # The C ABI streams A with 2-D tensor copies, which need 16-byte rows:
        # pad the leading dimension (a marshalling copy, same values).
        ld = (d * esz + 15) // 16 * 16 // esz
        Ap = torch.zeros(n, ld, dtype=A.dtype, device=A.device)
        Ap[:, :d] = A
        A = Ap[:, :d]
    b = b.to(device=A.device, dtype=torch.float64)
    if b.dim() == 1:
        b = b[:, None]
    k = b.shape[1]
    bcm = b.t().contiguous()  # k x d row-major == d x k column-major
    lam = lam.to(device=A.device, dtype=torch.float64).contiguous()
    p = L.Problem()
    p.dtype = L.F64 if A.dtype == torch.float64 else L.F32
    p.n, p.d, p.lda, p.k = n, d, (A.stride(0) if n > 0 else (d * esz + 15) // 16 * 16 // esz), k
    p.A = A.data_ptr() if n > 0 else None
    p.b = bcm.data_ptr()
    p.nu = float(nu)
    p.lambda_diag = lam.data_ptr()
    return p, (A, bcm, lam)


def hess_apply(A, x, nu, lam, extended=False):
    """y = A^T (A x) + nu^2 Lambda x in one pass over A (x: (d,) or (d, k) float64)."""
    lib = L.load()
    x2 = x.to(torch.float64)
    squeeze = x2.dim() == 1
    if squeeze:
        x2 = x2[:, None]
    xcm = x2.t().contiguous()
    p, keep = make_problem(A, x2, nu, lam)  # b slot unused by the pass
    ycm = torch.empty_like(xcm)
    nb = C.c_size_t()
    L.check(lib.sks_hess_apply_workspace_size(C.byref(p), C.byref(nb)))
    ws = _workspace(nb.value, A.device)
    L.check(lib.sks_hess_apply(C.byref(p), _ptr(xcm), _ptr(ycm), int(bool(extended)), _ptr(ws), nb.value,
                               _stream(A.device)))
    y = ycm.t()
    return y[:, 0] if squeeze else y.contiguous()


class Sketch:
    """Nested sketch S_m A (Section 2.1) held on the device."""

    def __init__(self, A, nu, lam, kind="srht", m=1, m_max=0, sjlt_s=1, seed=0):
        self._lib = L.load()
        b = torch.zeros(A.shape[1], dtype=torch.float64, device=A.device)
        self.problem, self._keep = make_problem(A, b, nu, lam)
        nb = C.c_size_t()
        L.check(self._lib.sks_sketch_workspace_size(C.byref(self.problem), L.KINDS[kind], int(m_max), int(sjlt_s),
                                                    C.byref(nb)))
        self.ws = _workspace(nb.value, A.device)
        h = C.c_void_p()
        L.check(self._lib.sks_sketch_create(C.byref(h), C.byref(self.problem), L.KINDS[kind], int(m), int(m_max),
                                            int(sjlt_s), C.c_uint64(seed), _ptr(self.ws), nb.value,
                                            _stream(A.device)))
        self.handle = h
        self.device = A.device
        self.m_max = int(m_max)

    @property
    def m(self):
        v = C.c_int64()
        L.check(self._lib.sks_sketch_rows(self.handle, C.byref(v)))
        return v.value

    def grow(self, new_m):
        L.check(self._lib.sks_sketch_grow(self.handle, int(new_m), _stream(self.device)))

    def matrix(self):
        """S A (m x d float64, scaled)."""
        out = torch.empty(self.m, int(self.problem.d), dtype=torch.float64, device=self.device)
        L.check(self._lib.sks_sketch_copy_out(self.handle, _ptr(out), _stream(self.device)))
        return out

    def __del__(self):
        if getattr(self, "handle", None):
            self._lib.sks_sketch_destroy(self.handle)
            self.handle = None


class Preconditioner:
    """H_S = (SA)^T SA + nu^2 Lambda factored on the device (Section 4.1.1)."""

    def __init__(self, sketch, m_max=None, precision="plain"):
        self._lib = L.load()
        self.sketch = sketch
        p = sketch.problem
        mm = int(m_max) if m_max else max(sketch.m, 1)
        nb = C.c_size_t()
        L.check(self._lib.sks_precond_workspace_size(C.byref(p), mm, C.byref(nb)))
        # the handle is sized by the sketch's own m_max; ask for the larger
        nb2 = C.c_size_t()
        L.check(self._lib.sks_precond_workspace_size(C.byref(p), max(mm, self._sketch_mmax()), C.byref(nb2)))
        self.ws = _workspace(max(nb.value, nb2.value), sketch.device)
        h = C.c_void_p()
        prec = L.PLAIN_F64 if precision == "plain" else L.MIXED_REFINED
        L.check(self._lib.sks_precond_build_ex(C.byref(h), sketch.handle, C.byref(p), prec, _ptr(self.ws),
                                               self.ws.numel(), _stream(sketch.device)))
        self.handle = h

    def _sketch_mmax(self):
        p = self.sketch.problem
        if self.sketch.m_max > 0:
            return self.sketch.m_max
        n = int(p.n)
        npad = 1
        while npad < max(n, 1):
            npad <<= 1
        return npad

    def apply(self, z):
        z2 = z.to(torch.float64)
        squeeze = z2.dim() == 1
        if squeeze:
            z2 = z2[:, None]
        zcm = z2.t().contiguous()
        vcm = torch.empty_like(zcm)
        L.check(self._lib.sks_precond_apply(self.handle, _ptr(zcm), _ptr(vcm), zcm.shape[0], _stream(self.sketch.device)))
        v = vcm.t()
        return v[:, 0] if squeeze else v.contiguous()

    def __del__(self):
        if getattr(self, "handle", None):
            self._lib.sks_precond_destroy(self.handle)
            self.handle = None


def options(kind="srht", rho=0.125, m_init=1, m_max=0, sjlt_s=1, tol=1e-10, max_iter=1000, precision="plain",
            reuse_residual=True, seed=0, max_outer=20, inner_tol=1e-4, stop_rule="estimate", cert_delta=0.01,
            cert_de=0.0):
    lib = L.load()
    o = L.Opts()
    lib.sks_opts_default(C.byref(o))
    o.kind = L.KINDS[kind]
    o.rho, o.m_init, o.m_max, o.sjlt_s = float(rho), int(m_init), int(m_max), int(sjlt_s)
    o.tol, o.max_iter = float(tol), int(max_iter)
    o.precision = L.PLAIN_F64 if precision == "plain" else L.MIXED_REFINED
    o.reuse_residual = int(bool(reuse_residual))
    o.seed = int(seed)
    o.max_outer, o.inner_tol = int(max_outer), float(inner_tol)
    o.stop_rule = L.STOP_RULES[stop_rule]
    o.cert_delta, o.cert_de = float(cert_delta), float(cert_de)
    return o


class Solver:
    """Reusable solver: sizes and holds the workspace once, then ``solve`` can
    be called repeatedly (the hot path of a benchmark).  method: "pcg" / "ihs"
    (adaptive, Algorithms 2 and 1) or one of the non-adaptive solvers
    "fixed-pcg", "fixed-ihs", "polyak-ihs" (sketch size m_init) and "cg"."""

    def __init__(self, A, b, nu, lam, method="pcg", trace_cap=0, x_star=None, **opts):
        self._lib = L.load()
        self.method = method
        self.problem, self._keep = make_problem(A, b, nu, lam)
        self.opts = options(**opts)
        if x_star is not None:
            # traces carry delta_t = 1/2 ||x_t - x*||_H^2 (column-major d x k copy kept alive)
            xs2 = x_star.to(device=A.device, dtype=torch.float64)
            self._xstar = (xs2[:, None] if xs2.dim() == 1 else xs2).t().contiguous()
            self.opts.x_star = self._xstar.data_ptr()
        self.trace_buf = (L.TraceEvent * trace_cap)() if trace_cap else None
        if trace_cap:
            self.opts.trace = C.cast(self.trace_buf, C.POINTER(L.TraceEvent))
            self.opts.trace_cap = trace_cap
        nb = C.c_size_t()
        L.check(self._lib.sks_solve_workspace_size(C.byref(self.problem), C.byref(self.opts), C.byref(nb)))
        self.ws = _workspace(nb.value, A.device)
        self.device = A.device
        self.d, self.k = int(self.problem.d), int(self.problem.k)

    def solve(self, x0=None, check=True):
        xcm = torch.zeros(self.k, self.d, dtype=torch.float64, device=self.device)
        if x0 is not None:
            x02 = x0.to(torch.float64)
            xcm.copy_((x02[:, None] if x02.dim() == 1 else x02).t())
        st = L.Stats()
        args = (C.byref(self.problem), C.byref(self.opts), _ptr(xcm), C.byref(st), _ptr(self.ws), self.ws.numel(),
                _stream(self.device))
        if self.method in L.FIXED_METHODS:
            status = self._lib.sks_fixed_solve(L.FIXED_METHODS[self.method], *args)
        elif self.method in ("pcg", "ihs"):
            fn = self._lib.sks_adaptive_pcg_solve if self.method == "pcg" else self._lib.sks_adaptive_ihs_solve
            status = fn(*args)
        else:
            raise ValueError("unknown method %r" % self.method)
        if check and status not in (L.OK,):
            L.check(status)
        x = xcm.t()
        x = x[:, 0] if self.k == 1 else x.contiguous()
        stats = st.as_dict()
        stats["status_name"] = L.STATUS_NAMES.get(status, status)
        trace = []
        if self.trace_buf is not None:
            for i in range(st.trace_len):
                e = self.trace_buf[i]
                trace.append(dict(t=e.t, m=e.m, ratio=e.ratio, thr=e.threshold, accepted=bool(e.accepted),
                                  outer=e.outer, column=e.column, delta=e.delta, delta0=e.delta0))
        return x, stats, trace


    def adjoint(self, x, g, want_A=True):
        """Gradients for upstream g = dL/dx at the solution x of the last
        ``solve`` (same workspace, same preconditioner): returns
        (dA, db, dnu, dlam) with dA in A's precision (None if not wanted)."""
        A = self._keep[0]
        gcm = (g.to(torch.float64)[:, None] if g.dim() == 1 else g.to(torch.float64)).t().contiguous()
        xcm = (x.to(torch.float64)[:, None] if x.dim() == 1 else x.to(torch.float64)).t().contiguous()
        dbcm = torch.empty_like(gcm)
        dA = torch.empty(A.shape, dtype=A.dtype, device=self.device) if want_A else None
        dlam = torch.empty(self.d, dtype=torch.float64, device=self.device)
        dnu = C.c_double(0.0)
        st = L.Stats()
        L.check(self._lib.sks_adjoint(C.byref(self.problem), C.byref(self.opts), _ptr(xcm), _ptr(gcm), _ptr(dbcm),
                                      _ptr(dA), int(dA.stride(0)) if dA is not None else 0, C.byref(dnu),
                                      _ptr(dlam), C.byref(st), _ptr(self.ws), self.ws.numel(),
                                      _stream(self.device)))
        db = dbcm.t()
        db = db[:, 0] if self.k == 1 else db.contiguous()
        return dA, db, dnu.value, dlam


class SketchSolve(torch.autograd.Function):
    """x = argmin 1/2 <x, H x> - b^T x with H = A^T A + nu^2 diag(lam), solved by
    the adaptive sketching solver; backward is the adjoint solve with the same
    preconditioner plus the fused dA pass (``sks_adjoint``)."""

    @staticmethod
    def forward(ctx, A, b, nu, lam, opts):
        nu_val = float(nu)
        solver = Solver(A.detach(), b.detach(), nu_val, lam.detach(), **(opts or {}))
        x, stats, _ = solver.solve()
        ctx.solver = solver
        ctx.nu_is_tensor = torch.is_tensor(nu)
        ctx.save_for_backward(x)
        ctx.stats = stats
        return x

    @staticmethod
    def backward(ctx, gx):
        (x,) = ctx.saved_tensors
        dA, db, dnu, dlam = ctx.solver.adjoint(x, gx.contiguous(), want_A=ctx.needs_input_grad[0])
        gnu = torch.tensor(dnu, dtype=torch.float64, device=x.device) if ctx.nu_is_tensor else None
        return dA, db, gnu, dlam, None


def sketch_solve(A, b, nu, lam, **opts):
    """Differentiable adaptive solve (see ``SketchSolve``)."""
    return SketchSolve.apply(A, b, nu, lam, opts)


def adaptive_pcg(A, b, nu, lam, x0=None, trace_cap=0, **opts):
    """Algorithm 2 on the GPU; returns (x, stats, trace)."""
    return Solver(A, b, nu, lam, method="pcg", trace_cap=trace_cap, **opts).solve(x0)


def adaptive_ihs(A, b, nu, lam, x0=None, trace_cap=0, **opts):
    """Algorithm 1 with the IHS step (mu = 1 - rho) on the GPU; returns (x, stats, trace)."""
    return Solver(A, b, nu, lam, method="ihs", trace_cap=trace_cap, **opts).solve(x0)


class DualSolver:
    """Eq. (2): the n x n dual problem (for n < d) solved by adaptive PCG or
    IHS on the GPU and the primal x = Lambda^{-1}(b - A^T w)/nu^2 recovered;
    sizes and holds the workspace once (``sks_dual_*_solve``)."""

    def __init__(self, A, b, nu, lam, method="pcg", **opts):
        self._lib = L.load()
        if method not in ("pcg", "ihs"):
            raise ValueError("unknown method %r" % method)
        self.method = method
        self.problem, self._keep = make_problem(A, b, nu, lam)
        self.opts = options(**opts)
        nb = C.c_size_t()
        L.check(self._lib.sks_dual_workspace_size(C.byref(self.problem), C.byref(self.opts), C.byref(nb)))
        self.ws = _workspace(nb.value, A.device)
        self.device = A.device
        self.d, self.k = int(self.problem.d), int(self.problem.k)

    def solve(self, check=True):
        xcm = torch.empty(self.k, self.d, dtype=torch.float64, device=self.device)
        st = L.Stats()
        fn = self._lib.sks_dual_pcg_solve if self.method == "pcg" else self._lib.sks_dual_ihs_solve
        status = fn(C.byref(self.problem), C.byref(self.opts), _ptr(xcm), C.byref(st), _ptr(self.ws),
                    self.ws.numel(), _stream(self.device))
        if check and status != L.OK:
            L.check(status)
        x = xcm.t()
        stats = st.as_dict()
        stats["status_name"] = L.STATUS_NAMES.get(status, status)
        return (x[:, 0] if self.k == 1 else x.contiguous()), stats


def dual_solve(A, b, nu, lam, method="pcg", check=True, **opts):
    """Eq. (2) on the GPU (see ``DualSolver``); returns (x, stats of the dual solve)."""
    return DualSolver(A, b, nu, lam, method=method, **opts).solve(check=check)


def fixed_solve(A, b, nu, lam, method="fixed-pcg", x0=None, check=True, **opts):
    """Non-adaptive solvers on the GPU (sketch size m_init): "fixed-pcg",
    "fixed-ihs", "polyak-ihs" (Appendix A) or "cg" (no preconditioner);
    returns (x, stats, trace).  check=False returns NO_CONVERGENCE results
    (x = x_T after max_iter steps) instead of raising."""
    if method not in L.FIXED_METHODS:
        raise ValueError("unknown fixed-sketch method %r" % method)
    return Solver(A, b, nu, lam, method=method, **opts).solve(x0, check=check)


class BatchSolver:
    """Many independent problems (each one (A, b, nu, lam)) solved together:
    adaptive PCG per problem, every decision on the device; precision="plain"
    takes float64 A, precision="mixed" float32 A (float32 inner passes,
    double-float refinement and preconditioner).  The plan
    (``sks_batch_create``: input checks, the A-pass unit height -- timed on
    this batch when rows_per_unit=0 -- and one instantiated CUDA graph whose
    while loop repeats the round until every problem has stopped) is made
    once; every ``solve`` is one graph launch (``sks_batch_solve``)."""

    def __init__(self, problems, rows_per_unit=0, **opts):
        self._lib = L.load()
        self.plan = None
        if len(problems) < 1:
            raise ValueError("need at least one problem")
        self.items = [make_problem(A, b, nu, lam) for (A, b, nu, lam) in problems]
        self.count = len(self.items)
        self.arr = (L.Problem * self.count)(*[p for p, _ in self.items])
        self.opts = options(**opts)
        nb = C.c_size_t()
        L.check(self._lib.sks_batch_workspace_size(self.arr, self.count, C.byref(self.opts), C.byref(nb)))
        self.device = problems[0][0].device
        self.ws = _workspace(nb.value, self.device)
        self.ds = [int(p.d) for p, _ in self.items]
        h = C.c_void_p()
        L.check(self._lib.sks_batch_create(C.byref(h), self.arr, self.count, C.byref(self.opts), int(rows_per_unit),
                                           _ptr(self.ws), self.ws.numel(), _stream(self.device)))
        self.plan = h

    def solve(self, x0s=None, check=True):
        xs = [torch.zeros(d, dtype=torch.float64, device=self.device) for d in self.ds]
        if x0s is not None:
            for x, x0 in zip(xs, x0s):
                x.copy_(x0.to(torch.float64))
        ptrs = (C.c_void_p * self.count)(*[x.data_ptr() for x in xs])
        st = (L.Stats * self.count)()
        info = L.BatchInfo()
        status = self._lib.sks_batch_solve(self.plan, ptrs, st, C.byref(info), _stream(self.device))
        if check and status != L.OK:
            L.check(status)
        stats = []
        for s in st:
            dct = s.as_dict()
            dct["status_name"] = L.STATUS_NAMES.get(s.status, s.status)
            stats.append(dct)
        return xs, stats, info.as_dict()

    def __del__(self):
        if getattr(self, "plan", None):
            self._lib.sks_batch_destroy(self.plan)
            self.plan = None


def solve_batched(problems, x0s=None, rows_per_unit=0, **opts):
    """Adaptive PCG on a batch of problems [(A, b, nu, lam), ...]; returns
    (xs, per-problem stats, batch info)."""
    return BatchSolver(problems, rows_per_unit=rows_per_unit, **opts).solve(x0s)
