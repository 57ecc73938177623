"""B300-native reduced-space OPF hot path (arXiv 2110.02590): Python binding.

Argument marshalling over the C ABI of ``libopf.so`` (``include/opf.h``).
PyTorch supplies device memory and the CUDA stream; every step of the path
runs in the library's CUDA kernels.  There is no CPU fallback: if the
library is missing, building a context raises.

    from paper_2110_02590_b300 import synth, OPFContext
    net = synth.workload("large9200")
    ctx = OPFContext(net)
    x, info = ctx.powerflow(u)                 # u: cuda float64 tensor
    g = ctx.reduced_gradient(al)               # al: dict of cuda tensors
    H, hinfo = ctx.reduced_hessian(al, block_k=8)
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libopf.so")
_lib = None

OPF_STATUS = {0: "OPF_OK", 1: "OPF_EINVAL", 2: "OPF_ENOMEM", 3: "OPF_ECUDA", 4: "OPF_ENOCONV",
              5: "OPF_ESINGULAR", 6: "OPF_ENOTPD", 7: "OPF_ESTATE", 8: "OPF_ETIMEOUT"}

_dp = C.POINTER(C.c_double)
_ip = C.POINTER(C.c_int)


class NetworkDesc(C.Structure):
    _fields_ = [("n_bus", C.c_int), ("n_branch", C.c_int), ("n_gen", C.c_int), ("ref_bus", C.c_int),
                ("pd", _dp), ("qd", _dp), ("vmin", _dp), ("vmax", _dp),
                ("br_from", _ip), ("br_to", _ip),
                ("br_r", _dp), ("br_x", _dp), ("br_b", _dp), ("br_tap", _dp), ("br_rate", _dp),
                ("gen_bus", _ip),
                ("gen_c2", _dp), ("gen_c1", _dp), ("gen_c0", _dp),
                ("gen_pmin", _dp), ("gen_pmax", _dp), ("gen_qmin", _dp), ("gen_qmax", _dp),
                ("base_mva", C.c_double)]


class PfOpts(C.Structure):
    _fields_ = [("tol", C.c_double), ("max_it", C.c_int)]


class PfInfo(C.Structure):
    _fields_ = [("iterations", C.c_int), ("res2", C.c_double), ("resinf", C.c_double)]


class AlParams(C.Structure):
    _fields_ = [("sigma_f", C.c_double), ("rho", C.c_double), ("sigma_c", C.c_void_p),
                ("y", C.c_void_p), ("s", C.c_void_p), ("omega", C.c_void_p)]


class HessOpts(C.Structure):
    _fields_ = [("block_k", C.c_int), ("grid", C.c_int), ("plain", C.c_int), ("col_begin", C.c_int),
                ("col_count", C.c_int), ("threads", C.c_int), ("reuse_first_order", C.c_int),
                ("asymmetry", C.c_int), ("phase_profile", C.c_int)]


class HessInfo(C.Structure):
    _fields_ = [("block_k", C.c_int), ("grid", C.c_int), ("tiles", C.c_int), ("launches", C.c_int),
                ("ms_total", C.c_float), ("ms_hvp", C.c_float), ("asymmetry", C.c_double),
                ("phase_ms", C.c_float * 5)]


class AlState(C.Structure):
    _fields_ = [("u", C.c_void_p), ("s", C.c_void_p), ("zl_u", C.c_void_p), ("zu_u", C.c_void_p),
                ("zl_s", C.c_void_p), ("zu_s", C.c_void_p), ("u_lo", C.c_void_p), ("u_hi", C.c_void_p),
                ("s_lo", C.c_void_p), ("s_hi", C.c_void_p), ("x", C.c_void_p), ("mu", C.c_double)]


class StepOpts(C.Structure):
    _fields_ = [("block_k", C.c_int), ("max_halvings", C.c_int), ("max_inertia", C.c_int),
                ("delta_start", C.c_double), ("line_search", C.c_int)]


class StepInfo(C.Structure):
    _fields_ = [("alpha_p", C.c_double), ("alpha_d", C.c_double), ("delta", C.c_double),
                ("du_inf", C.c_double), ("ds_inf", C.c_double), ("halvings", C.c_int),
                ("inertia_tries", C.c_int), ("pf_iterations", C.c_int), ("ms_hessian", C.c_float),
                ("ms_total", C.c_float), ("ms_first_order", C.c_float), ("ms_rhs", C.c_float),
                ("ms_cholesky", C.c_float), ("ms_solve", C.c_float), ("ms_trial", C.c_float),
                ("cholesky_fp64", C.c_int), ("factorisations", C.c_int)]


class AlOpts(C.Structure):
    _fields_ = [("max_outer", C.c_int), ("max_inner", C.c_int), ("eta_primal", C.c_double),
                ("eta_dual", C.c_double), ("rho_max", C.c_double), ("block_k", C.c_int),
                ("scaling_gmax", C.c_double), ("sigma_c_used", C.c_void_p)]


class AlInfo(C.Structure):
    _fields_ = [("outer", C.c_int), ("steps", C.c_int), ("converged", C.c_int), ("primal_inf", C.c_double),
                ("dual_inf", C.c_double), ("F", C.c_double), ("rho", C.c_double), ("mu", C.c_double),
                ("ms_total", C.c_float), ("sigma_f", C.c_double)]


class QpOpts(C.Structure):
    _fields_ = [("max_it", C.c_int), ("tol", C.c_double), ("block_k", C.c_int), ("max_halvings", C.c_int),
                ("max_inertia", C.c_int), ("delta_start", C.c_double), ("inertia_only", C.c_int)]


class QpInfo(C.Structure):
    _fields_ = [("qp_iterations", C.c_int), ("halvings", C.c_int), ("pf_iterations", C.c_int),
                ("inertia_increases", C.c_int), ("delta", C.c_double), ("delta_convex", C.c_double),
                ("kkt", C.c_double), ("mu", C.c_double),
                ("alpha_p", C.c_double), ("kkt_first", C.c_double), ("alpha_p_min", C.c_double),
                ("ms_total", C.c_float), ("ms_qp", C.c_float), ("ms_hessian", C.c_float),
                ("ms_cholesky", C.c_float), ("cholesky_fp64", C.c_int)]


class BatchInfo(C.Structure):
    _fields_ = [("ms_powerflow_first_order", C.c_float), ("ms_hessians", C.c_float), ("ms_steps", C.c_float),
                ("ms_total", C.c_float), ("hessian_tiles", C.c_int), ("host_threads", C.c_int), ("failed", C.c_int)]


class OPFError(RuntimeError):
    def __init__(self, status, what):
        self.status = status
        super().__init__(f"{what}: {OPF_STATUS.get(status, status)} ({lib().opf_last_error().decode()})")


def lib():
    """Load libopf.so (built in-tree by build.py / __graft_entry__.build())."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"libopf.so not built ({LIB_PATH}); run python -m paper_2110_02590_b300.build")
        L = C.CDLL(LIB_PATH)
        L.opf_load_network.argtypes = [C.POINTER(NetworkDesc), C.c_void_p, C.POINTER(C.c_void_p)]
        L.opf_free.argtypes = [C.c_void_p]
        L.opf_free.restype = None
        L.opf_set_stream.argtypes = [C.c_void_p, C.c_void_p]
        L.opf_dims.argtypes = [C.c_void_p] + [_ip] * 5
        L.opf_symbolic_sizes.argtypes = [C.c_void_p] + [_ip] * 4
        L.opf_symbolic_export.argtypes = [C.c_void_p] + [_ip] * 6
        L.opf_powerflow.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                    C.POINTER(PfOpts), C.POINTER(PfInfo)]
        L.opf_reduced_gradient.argtypes = [C.c_void_p, C.POINTER(AlParams)] + [C.c_void_p] * 7
        L.opf_reduced_hessian.argtypes = [C.c_void_p, C.POINTER(AlParams), C.POINTER(HessOpts), C.c_void_p,
                                          C.POINTER(HessInfo)]
        L.opf_symbolic_analyze.argtypes = [C.POINTER(NetworkDesc), C.POINTER(C.c_void_p)]
        L.opf_symbolic_info.argtypes = [C.c_void_p] + [_ip] * 5
        L.opf_symbolic_get.argtypes = [C.c_void_p] + [_ip] * 6
        L.opf_symbolic_free.argtypes = [C.c_void_p]
        L.opf_symbolic_free.restype = None
        L.opf_reduced_hessian_noalloc.argtypes = [C.c_void_p, C.POINTER(AlParams), C.POINTER(HessOpts),
                                                  C.c_void_p, C.POINTER(HessInfo)]
        L.opf_al_step.argtypes = [C.c_void_p, C.POINTER(AlParams), C.POINTER(AlState), C.POINTER(StepOpts),
                                  C.POINTER(StepInfo), C.c_void_p, C.c_void_p]
        L.opf_reduced_hessian_batched.argtypes = [C.POINTER(C.c_void_p), C.c_int, C.POINTER(AlParams),
                                                  C.POINTER(C.c_void_p), C.POINTER(HessOpts), C.POINTER(HessInfo)]
        L.opf_hessian_autotune.argtypes = [C.c_void_p, C.POINTER(AlParams), C.c_void_p, C.POINTER(HessOpts),
                                           C.POINTER(C.c_float)]
        L.opf_launch_count.argtypes = [C.c_void_p, C.POINTER(C.c_longlong)]
        L.opf_set_sweep_merge.argtypes = [C.c_void_p, C.c_int, C.c_int]
        L.opf_set_cholesky_mode.argtypes = [C.c_void_p, C.c_int]
        L.opf_set_update_engine.argtypes = [C.c_void_p, C.c_int]
        L.opf_sweep_autotune.argtypes = [C.c_void_p, C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(C.c_float),
                                         C.POINTER(C.c_float)]
        L.opf_reduced_jacobian.argtypes = [C.c_void_p, C.POINTER(AlParams), C.POINTER(HessOpts), C.c_void_p,
                                           C.c_void_p, C.POINTER(HessInfo)]
        L.opf_gradient_scaling.argtypes = [C.c_void_p, C.c_double, C.c_double, C.c_void_p, C.c_void_p,
                                           C.c_void_p, C.POINTER(C.c_double)]
        L.opf_set_wait_limit.argtypes = [C.c_void_p, C.c_int]
        L.opf_set_hessian_symmetry.argtypes = [C.c_void_p, C.c_int]
        L.opf_tracking_update.argtypes = [C.c_void_p, C.POINTER(AlParams), C.c_void_p, C.POINTER(AlState),
                                          C.POINTER(QpOpts), C.POINTER(QpInfo)]
        L.opf_al_step_batched.argtypes = [C.POINTER(C.c_void_p), C.c_int, C.POINTER(AlParams), C.POINTER(AlState),
                                          C.POINTER(C.c_void_p), C.POINTER(C.c_void_p), C.POINTER(StepOpts),
                                          C.POINTER(StepInfo), C.POINTER(C.c_int), C.POINTER(BatchInfo)]
        L.opf_objective_batched.argtypes = [C.POINTER(C.c_void_p), C.c_int, C.c_int, C.POINTER(AlParams)] + \
            [C.c_void_p] * 11 + [C.POINTER(C.c_int)]
        L.opf_al_solve.argtypes = [C.c_void_p, C.POINTER(AlParams), C.c_void_p, C.POINTER(AlState),
                                   C.POINTER(AlOpts), C.POINTER(AlInfo), C.POINTER(C.c_double)]
        L.opf_fp64_peak.argtypes = [C.c_void_p, C.POINTER(C.c_double), C.POINTER(C.c_float)]
        L.opf_pivot_reciprocal.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int]
        L.opf_dense_syrk_emulated.argtypes = [C.c_void_p, C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_int,
                                              C.c_int]
        L.opf_status_str.restype = C.c_char_p
        L.opf_status_str.argtypes = [C.c_int]
        L.opf_last_error.restype = C.c_char_p
        _lib = L
    return _lib


def exported_symbols():
    """Names declared in include/opf.h (checked against the library by the tests)."""
    import re
    hdr = os.path.join(_HERE, "..", "include", "opf.h")
    with open(hdr) as fh:
        text = fh.read()
    return sorted(set(re.findall(r"^\s*(?:opf_status|void|const char\*)\s+(opf_\w+)\s*\(", text, re.M)))


def _make_desc(net):
    """NetworkDesc over contiguous host copies of the network tables (kept alive by the caller)."""
    a = lambda v: np.ascontiguousarray(v, dtype=np.float64)  # noqa: E731
    ai = lambda v: np.ascontiguousarray(v, dtype=np.int32)  # noqa: E731
    k = dict(pd=a(net.pd), qd=a(net.qd), vmin=a(net.vmin), vmax=a(net.vmax),
             f=ai(net.br_from), t=ai(net.br_to), r=a(net.br_r), x=a(net.br_x), b=a(net.br_b),
             tap=a(net.br_tap), rate=a(net.br_rate), gbus=ai(net.gen_bus), c2=a(net.gen_c2),
             c1=a(net.gen_c1), c0=a(net.gen_c0), pmin=a(net.gen_pmin), pmax=a(net.gen_pmax),
             qmin=a(net.gen_qmin), qmax=a(net.gen_qmax))
    d = lambda v: v.ctypes.data_as(_dp)  # noqa: E731
    i = lambda v: v.ctypes.data_as(_ip)  # noqa: E731
    desc = NetworkDesc(int(net.n_bus), int(net.n_branch), int(net.n_gen), int(net.ref_bus),
                       d(k["pd"]), d(k["qd"]), d(k["vmin"]), d(k["vmax"]), i(k["f"]), i(k["t"]),
                       d(k["r"]), d(k["x"]), d(k["b"]), d(k["tap"]), d(k["rate"]), i(k["gbus"]),
                       d(k["c2"]), d(k["c1"]), d(k["c0"]), d(k["pmin"]), d(k["pmax"]), d(k["qmin"]),
                       d(k["qmax"]), float(getattr(net, "base_mva", 100.0)))
    return desc, k


def symbolic_analyze(net) -> dict:
    """Host-only symbolic analysis of G_x (ordering, filled pattern, level sets); needs no GPU."""
    L = lib()
    desc, keep = _make_desc(net)
    h = C.c_void_p()
    st = L.opf_symbolic_analyze(C.byref(desc), C.byref(h))
    if st != 0:
        raise OPFError(st, "opf_symbolic_analyze")
    try:
        nx, nnz, nsb, nlf, nlb = (C.c_int() for _ in range(5))
        L.opf_symbolic_info(h, *[C.byref(v) for v in (nx, nnz, nsb, nlf, nlb)])
        out = dict(bus_order=np.zeros(nsb.value, np.int32), perm=np.zeros(nx.value, np.int32),
                   rowptr=np.zeros(nx.value + 1, np.int32), colidx=np.zeros(nnz.value, np.int32),
                   lev_f=np.zeros(nx.value, np.int32), lev_b=np.zeros(nx.value, np.int32))
        L.opf_symbolic_get(h, *[out[k].ctypes.data_as(_ip) for k in
                                ("bus_order", "perm", "rowptr", "colidx", "lev_f", "lev_b")])
        out["nlev_f"], out["nlev_b"] = nlf.value, nlb.value
        return out
    finally:
        L.opf_symbolic_free(h)


def reduced_hessian_batched(ctxs, als, block_k=8, grid=0, outs=None):
    """Hessians of several contexts (each at its converged power flow) in one persistent launch.

    Returns ([H_k], info); H_k is the n_u(k) x n_u(k) Hessian of ctxs[k] with the AL inputs als[k].
    """
    import torch
    n = len(ctxs)
    for c in ctxs:
        c._sync_stream()
    ctxs[0]._sync_stream()
    params, keep = [], []
    for c, al in zip(ctxs, als):
        p, kp = c._al(al)
        params.append(p)
        keep.append(kp)
    if outs is None:
        outs = [torch.empty((c.nu, c.nu), dtype=torch.float64, device=c.device) for c in ctxs]
    hs = (C.c_void_p * n)(*[c.h.value for c in ctxs])
    ps = (AlParams * n)(*params)
    Hp = (C.c_void_p * n)(*[o.data_ptr() for o in outs])
    info = HessInfo()
    st = lib().opf_reduced_hessian_batched(hs, n, ps, Hp, C.byref(HessOpts(int(block_k), int(grid), 0, 0, 0, 0, 0)),
                                           C.byref(info))
    if st != 0:
        raise OPFError(st, "opf_reduced_hessian_batched")
    return [o.T for o in outs], dict(block_k=info.block_k, grid=info.grid, tiles=info.tiles,
                                     launches=info.launches, ms_total=info.ms_total, ms_hvp=info.ms_hvp)


def _stream():
    import torch
    return C.c_void_p(torch.cuda.current_stream().cuda_stream)


def fp64_peak():
    """Measured FP64 FMA rate of the current device: (TFLOP/s, ms of the timed launch)."""
    tf, ms = C.c_double(), C.c_float()
    st = lib().opf_fp64_peak(_stream(), C.byref(tf), C.byref(ms))
    if st != 0:
        raise OPFError(st, "opf_fp64_peak")
    return tf.value, ms.value


def pivot_reciprocal(u):
    """1 / u as the LU refactorisation computes its pivots' reciprocals (cuda float64 tensor)."""
    import torch
    if u.dtype != torch.float64 or not u.is_cuda or not u.is_contiguous():
        raise ValueError("expected a contiguous cuda float64 tensor")
    r = torch.empty_like(u)
    st = lib().opf_pivot_reciprocal(_stream(), C.c_void_p(u.data_ptr()), C.c_void_p(r.data_ptr()), u.numel())
    if st != 0:
        raise OPFError(st, "opf_pivot_reciprocal")
    return r


def dense_syrk_emulated(A, c0, K, r0, engine=0):
    """A[r0:, r0:] (lower) -= P P^T, P = A[r0:, c0:c0+K], in place on a column-major n x n
    cuda float64 matrix given as its transpose view (A_t[j] = column j), emulated on tensor cores
    (engine 0: tcgen05 for large updates and mma.sync for small ones, 1: warp-level mma.sync,
    2: tcgen05)."""
    import torch
    if A.dtype != torch.float64 or not A.is_cuda or not A.is_contiguous() or A.dim() != 2 or \
            A.shape[0] != A.shape[1]:
        raise ValueError("expected a square contiguous cuda float64 tensor")
    st = lib().opf_dense_syrk_emulated(_stream(), C.c_void_p(A.data_ptr()), A.shape[0], int(c0), int(K), int(r0),
                                       int(engine))
    if st != 0:
        raise OPFError(st, "opf_dense_syrk_emulated")
    return A


def al_step_batched(ctxs, als, states, loads=None, block_k=0, delta_start=0.0):
    """One tracking update per snapshot (opf_al_step_batched): power flow at loads[k] = (pd, qd)
    (cuda float64 tensors; None keeps the state), then the reduced-Newton step with all Schur
    Hessians in one persistent launch.  The state tensors are updated in place.  Returns
    (per-snapshot step infos, statuses, batch info)."""
    n = len(ctxs)
    for c in ctxs:
        c._sync_stream()
    keep, ps, sts = [], [], []
    for c, al, st in zip(ctxs, als, states):
        p, kp = c._al(dict(al, s=st["s"]))
        keep.append(kp)
        ps.append(p)
        sts.append(c._state(st))
    hs = (C.c_void_p * n)(*[c.h.value for c in ctxs])
    pdp = qdp = None
    if loads is not None:
        for c, (pd, qd) in zip(ctxs, loads):
            c._dev(pd)
            c._dev(qd)
        pdp = (C.c_void_p * n)(*[pd.data_ptr() for pd, _ in loads])
        qdp = (C.c_void_p * n)(*[qd.data_ptr() for _, qd in loads])
    infos = (StepInfo * n)()
    stat = (C.c_int * n)()
    binfo = BatchInfo()
    opts = StepOpts(int(block_k), 0, 0, float(delta_start))
    rc = lib().opf_al_step_batched(hs, n, (AlParams * n)(*ps), (AlState * n)(*sts), pdp, qdp, C.byref(opts), infos,
                                   stat, C.byref(binfo))
    out = [{k: getattr(i, k) for k, _ in StepInfo._fields_} for i in infos]
    if rc != 0 and all(v == 0 for v in stat):
        raise OPFError(rc, "opf_al_step_batched")
    return out, list(stat), {k: getattr(binfo, k) for k, _ in BatchInfo._fields_}


def objective_batched(ctxs, al, u, pd, qd, s, x0, grads=False, x_out=None):
    """F (and with grads=True the adjoint gradients w.r.t. u, pd, qd, s) for the scenarios
    u [n, n_u], pd/qd [n, n_bus], s [n, m] of one network, spread over the contexts `ctxs`
    (each should own a stream: OPFContext.use_own_stream).  x_out [n, n_x] (optional)
    receives the states; passing the same tensor as x0 starts each scenario from its own row.
    Returns a dict of cuda tensors."""
    import torch
    c0 = ctxs[0]
    n = u.shape[0]
    torch.cuda.current_stream(c0.device).synchronize()  # the inputs are on torch's stream
    keep = [c0._dev(al["sigma_c"]), c0._dev(al["y"])]
    p = AlParams(float(al["sigma_f"]), float(al["rho"]), keep[0].data_ptr(), keep[1].data_ptr(), None, None)
    z = lambda *sh: torch.empty(sh, dtype=torch.float64, device=c0.device)  # noqa: E731
    out = dict(F=z(n))
    if grads:
        out.update(grad_u=z(n, c0.nu), grad_pd=z(n, c0.net.n_bus), grad_qd=z(n, c0.net.n_bus), grad_s=z(n, c0.m))
    for t in (u, pd, qd, s, x0, x_out):
        if t is not None:
            c0._dev(t)
    if x_out is not None and tuple(x_out.shape) != (n, c0.nx):
        raise ValueError(f"x_out must have shape ({n}, {c0.nx}), got {tuple(x_out.shape)}")
    if x0 is not None and x0 is not x_out and x0.numel() != c0.nx:
        raise ValueError(f"x0 must hold n_x = {c0.nx} values (or be x_out itself)")
    hs = (C.c_void_p * len(ctxs))(*[c.h.value for c in ctxs])
    stat = (C.c_int * max(1, n))()
    rc = lib().opf_objective_batched(hs, len(ctxs), n, C.byref(p), _ptr(u), _ptr(pd), _ptr(qd), _ptr(s), _ptr(x0),
                                     _ptr(x_out), _ptr(out["F"]), _ptr(out.get("grad_u")), _ptr(out.get("grad_pd")),
                                     _ptr(out.get("grad_qd")), _ptr(out.get("grad_s")), stat)
    if rc != 0:
        raise OPFError(rc, "opf_objective_batched")
    return out


def _ptr(t):
    return None if t is None else C.c_void_p(t.data_ptr())


class OPFContext:
    """One network on one GPU: symbolic analysis, factors and workspaces."""

    def __init__(self, net, device=None):
        import torch
        self.torch = torch
        self.device = torch.device("cuda", torch.cuda.current_device() if device is None else device)
        L = lib()
        self.net = net
        desc, self._keep = _make_desc(net)
        h = C.c_void_p()
        with torch.cuda.device(self.device):
            st = L.opf_load_network(C.byref(desc), C.c_void_p(torch.cuda.current_stream().cuda_stream), C.byref(h))
        if st != 0:
            raise OPFError(st, "opf_load_network")
        self.h = h
        dims = [C.c_int() for _ in range(5)]
        L.opf_dims(h, *[C.byref(v) for v in dims])
        self.nx, self.nu, self.m, self.npv, self.npq = (v.value for v in dims)

    def __del__(self):
        if getattr(self, "h", None) is not None and _lib is not None:
            _lib.opf_free(self.h)
            self.h = None

    def _sync_stream(self):
        if getattr(self, "_own_stream", None) is not None:
            return
        lib().opf_set_stream(self.h, C.c_void_p(self.torch.cuda.current_stream(self.device).cuda_stream))

    def use_own_stream(self):
        """Bind the context to a stream of its own (for scenario pools that run concurrently);
        the context's calls then no longer follow torch's current stream."""
        self._own_stream = self.torch.cuda.Stream(device=self.device)
        st = lib().opf_set_stream(self.h, C.c_void_p(self._own_stream.cuda_stream))
        if st != 0:
            raise OPFError(st, "opf_set_stream")

    def _dev(self, v):
        t = self.torch
        if isinstance(v, t.Tensor):
            if v.device != self.device or v.dtype != t.float64 or not v.is_contiguous():
                raise ValueError("expected a contiguous float64 tensor on the context's device")
            return v
        return t.as_tensor(np.ascontiguousarray(v, dtype=np.float64), device=self.device)

    def _out_hessian(self, out):
        """The n_u x n_u output buffer of a Hessian call (checked: the kernels write all of it)."""
        if out is None:
            return self.torch.empty((self.nu, self.nu), dtype=self.torch.float64, device=self.device)
        self._dev(out)
        if tuple(out.shape) != (self.nu, self.nu):
            raise ValueError(f"out must have shape ({self.nu}, {self.nu}), got {tuple(out.shape)}")
        return out

    # ---------------------------------------------------------------- symbolic
    def symbolic(self) -> dict:
        L = lib()
        nnz, nsb, nlf, nlb = (C.c_int() for _ in range(4))
        L.opf_symbolic_sizes(self.h, C.byref(nnz), C.byref(nsb), C.byref(nlf), C.byref(nlb))
        out = dict(bus_order=np.zeros(nsb.value, np.int32), perm=np.zeros(self.nx, np.int32),
                   rowptr=np.zeros(self.nx + 1, np.int32), colidx=np.zeros(nnz.value, np.int32),
                   lev_f=np.zeros(self.nx, np.int32), lev_b=np.zeros(self.nx, np.int32))
        st = L.opf_symbolic_export(self.h, *[out[k].ctypes.data_as(_ip) for k in
                                             ("bus_order", "perm", "rowptr", "colidx", "lev_f", "lev_b")])
        if st != 0:
            raise OPFError(st, "opf_symbolic_export")
        out["nlev_f"], out["nlev_b"] = nlf.value, nlb.value
        return out

    # ---------------------------------------------------------------- power flow
    def powerflow(self, u, pd=None, qd=None, x0=None, tol=1e-10, max_it=20, check=True):
        """Newton-Raphson from x0 (default flat start).  Returns (x, info)."""
        t = self.torch
        self._sync_stream()
        u = self._dev(u)
        pd = None if pd is None else self._dev(pd)
        qd = None if qd is None else self._dev(qd)
        if x0 is None:
            x = t.cat([t.zeros(self.npv + self.npq, dtype=t.float64, device=self.device),
                       t.ones(self.npq, dtype=t.float64, device=self.device)])
        else:
            x = self._dev(x0).clone()
        info = PfInfo()
        st = lib().opf_powerflow(self.h, _ptr(u), _ptr(pd), _ptr(qd), _ptr(x), C.byref(PfOpts(tol, max_it)),
                                 C.byref(info))
        res = dict(status=st, iterations=info.iterations, res2=info.res2, resinf=info.resinf)
        if check and st != 0:
            raise OPFError(st, "opf_powerflow")
        return x, res

    def _al(self, al):
        keep = [self._dev(al["sigma_c"]), self._dev(al["y"]), self._dev(al["s"])]
        om = al.get("omega")
        if om is not None:
            keep.append(self._dev(om))
        p = AlParams(float(al["sigma_f"]), float(al["rho"]), keep[0].data_ptr(), keep[1].data_ptr(),
                     keep[2].data_ptr(), keep[3].data_ptr() if om is not None else None)
        return p, keep

    def reduced_gradient(self, al) -> dict:
        """Prop. 1 gradient of the scaled AL at the last converged power flow."""
        t = self.torch
        self._sync_stream()
        p, keep = self._al(al)
        z = lambda n: t.empty(n, dtype=t.float64, device=self.device)  # noqa: E731
        out = dict(F=z(1), grad_u=z(self.nu), grad_s=z(self.m), c=z(self.m), lam=z(self.nx),
                   grad_pd=z(self.net.n_bus), grad_qd=z(self.net.n_bus))
        st = lib().opf_reduced_gradient(self.h, C.byref(p), *[_ptr(out[k]) for k in
                                                             ("F", "grad_u", "grad_s", "c", "lam", "grad_pd",
                                                              "grad_qd")])
        if st != 0:
            raise OPFError(st, "opf_reduced_gradient")
        return out

    def autotune(self, al):
        """Pick the fastest (block_k, threads) for this context; later calls with block_k=0 use it."""
        t = self.torch
        self._sync_stream()
        p, keep = self._al(al)
        H = t.empty((self.nu, self.nu), dtype=t.float64, device=self.device)
        best = HessOpts()
        ms = C.c_float()
        st = lib().opf_hessian_autotune(self.h, C.byref(p), _ptr(H), C.byref(best), C.byref(ms))
        if st != 0:
            raise OPFError(st, "opf_hessian_autotune")
        return dict(block_k=best.block_k, threads=best.threads, ms=ms.value)

    def set_wait_limit(self, spins: int) -> None:
        """Iteration limit of the context's bounded device waits (0 = the kernels' defaults)."""
        self._sync_stream()
        st = lib().opf_set_wait_limit(self.h, int(spins))
        if st != 0:
            raise OPFError(st, "opf_set_wait_limit")

    def set_hessian_symmetry(self, on: bool) -> None:
        """Full Hessians by their symmetry (opf_set_hessian_symmetry; on by default)."""
        self._sync_stream()
        st = lib().opf_set_hessian_symmetry(self.h, int(bool(on)))
        if st != 0:
            raise OPFError(st, "opf_set_hessian_symmetry")

    def launch_count(self) -> int:
        v = C.c_longlong()
        lib().opf_launch_count(self.h, C.byref(v))
        return v.value

    def reduced_hessian(self, al, block_k=8, grid=0, plain=False, out=None, col_begin=0, col_count=0,
                        threads=0, asymmetry=False, phase_profile=False):
        """Dense reduced Hessian (n_u x n_u) by adjoint-adjoint HVPs (Prop. 2).

        Returns (H, info); H is column-major in memory, i.e. H_t[j] is column j.  With
        asymmetry=True (full Hessian) info["asymmetry"] = ||H - H^T||_F / ||H||_F; with
        phase_profile=True info["phase_ms"] apportions the HVP time to the tile phases (first L
        solve, U sweep, second-order terms, U^T + L^T sweeps, assembly).
        """
        t = self.torch
        self._sync_stream()
        p, keep = self._al(al)
        H = self._out_hessian(out)
        info = HessInfo()
        opts = HessOpts(int(block_k), int(grid), int(plain), int(col_begin), int(col_count), int(threads), 0,
                        int(bool(asymmetry)), int(bool(phase_profile)))
        st = lib().opf_reduced_hessian(self.h, C.byref(p), C.byref(opts),
                                       _ptr(H), C.byref(info))
        if st != 0:
            raise OPFError(st, "opf_reduced_hessian")
        return H.T, dict(block_k=info.block_k, grid=info.grid, tiles=info.tiles, launches=info.launches,
                         ms_total=info.ms_total, ms_hvp=info.ms_hvp, asymmetry=info.asymmetry,
                         phase_ms=list(info.phase_ms))

    def reduced_jacobian(self, al=None, hessian=False, block_k=8, grid=0, col_begin=0, col_count=0, threads=0,
                         out=None, out_hessian=None):
        """Reduced constraint Jacobian J = dc/du (m x n_u) from the HVP tiles' first adjoint
        (opf_reduced_jacobian).  With hessian=True the same launch also returns the reduced Hessian
        (as reduced_hessian; `al` required), else `al` may be None.  `out`: a preallocated
        (n_u, m) float64 buffer whose row j receives column j of J.  Returns (J, H or None, info)
        with J an (m, n_u) view."""
        t = self.torch
        self._sync_stream()
        if hessian and al is None:
            raise ValueError("the Hessian needs the AL parameters")
        p, keep = self._al(al) if al is not None else (None, [])
        if out is None:
            Jt = t.empty((self.nu, self.m), dtype=t.float64, device=self.device)
        else:
            Jt = self._dev(out)
            if tuple(Jt.shape) != (self.nu, self.m):
                raise ValueError(f"out must have shape ({self.nu}, {self.m}), got {tuple(Jt.shape)}")
        H = self._out_hessian(out_hessian) if hessian else None
        info = HessInfo()
        opts = HessOpts(int(block_k), int(grid), 0, int(col_begin), int(col_count), int(threads), 0, 0, 0)
        st = lib().opf_reduced_jacobian(self.h, C.byref(p) if p is not None else None, C.byref(opts), _ptr(Jt),
                                        _ptr(H) if H is not None else None, C.byref(info))
        if st != 0:
            raise OPFError(st, "opf_reduced_jacobian")
        return Jt.T, (H.T if H is not None else None), dict(block_k=info.block_k, grid=info.grid,
                                                             tiles=info.tiles, launches=info.launches,
                                                             ms_total=info.ms_total, ms_hvp=info.ms_hvp)

    def set_cholesky_mode(self, mode):
        """Trailing updates of the dense Cholesky (opf_set_cholesky_mode): 1 emulated only (the
        default), 0 emulated with an FP64 re-check of a failed pivot, 2 FP64 only."""
        st = lib().opf_set_cholesky_mode(self.h, int(mode))
        if st != 0:
            raise OPFError(st, "opf_set_cholesky_mode")

    def set_update_engine(self, engine):
        """Tensor-core kernel of the emulated Cholesky updates (opf_set_update_engine): 0 tcgen05
        for large updates and mma.sync for small ones (the default), 1 warp-level mma.sync,
        2 tcgen05."""
        st = lib().opf_set_update_engine(self.h, int(engine))
        if st != 0:
            raise OPFError(st, "opf_set_update_engine")

    def set_sweep_merge(self, lookahead, narrow=4):
        """Level-merge schedule of the single-right-hand-side solves (opf_set_sweep_merge)."""
        self._sync_stream()
        st = lib().opf_set_sweep_merge(self.h, int(lookahead), int(narrow))
        if st != 0:
            raise OPFError(st, "opf_set_sweep_merge")

    SWEEP_MERGE_CANDIDATES = ((0, 0), (1, 4), (2, 4), (4, 4), (6, 4), (8, 4), (4, 2), (4, 8))

    def sweep_autotune(self, table=False):
        """Time the level-merge schedules of the single-RHS solve and keep the fastest
        (opf_sweep_autotune).  Returns (lookahead, narrow, ms per forward + transposed solve), and
        with table=True also {(lookahead, narrow): ms} over SWEEP_MERGE_CANDIDATES."""
        self._sync_stream()
        d, w, ms = C.c_int(0), C.c_int(0), C.c_float(0.0)
        allms = (C.c_float * 8)()
        st = lib().opf_sweep_autotune(self.h, C.byref(d), C.byref(w), C.byref(ms), allms)
        if st != 0:
            raise OPFError(st, "opf_sweep_autotune")
        if table:
            return d.value, w.value, ms.value, dict(zip(self.SWEEP_MERGE_CANDIDATES, list(allms)))
        return d.value, w.value, ms.value

    def gradient_scaling(self, g_max=100.0, s_min=1e-8, prior=None, out_jacobian=None):
        """Gradient-based scales of the AL problem (opf_gradient_scaling), with the caller's own
        constraint scales `prior` (optional, [m]): returns (sigma_c [m] on the device, sigma_f, J as an
        (m, n_u) view)."""
        t = self.torch
        self._sync_stream()
        prior = None if prior is None else self._dev(prior)
        if out_jacobian is None:
            Jt = t.empty((self.nu, self.m), dtype=t.float64, device=self.device)
        else:
            Jt = self._dev(out_jacobian)
            if tuple(Jt.shape) != (self.nu, self.m):
                raise ValueError(f"out_jacobian must have shape ({self.nu}, {self.m})")
        sig = t.empty(self.m, dtype=t.float64, device=self.device)
        sf = C.c_double(0.0)
        st = lib().opf_gradient_scaling(self.h, float(g_max), float(s_min), _ptr(prior), _ptr(Jt), _ptr(sig),
                                        C.byref(sf))
        if st != 0:
            raise OPFError(st, "opf_gradient_scaling")
        return sig, sf.value, Jt.T

    def reduced_hessian_noalloc(self, al, block_k=8, grid=0, out=None, col_begin=0, col_count=0):
        """Reduced Hessian through opf_reduced_hessian_noalloc (fixed static workspace, no allocation
        inside the call).  Callers that cannot allocate pass a preallocated n_u x n_u float64 `out`."""
        t = self.torch
        self._sync_stream()
        p, keep = self._al(al)
        H = self._out_hessian(out)
        info = HessInfo()
        opts = HessOpts(int(block_k), int(grid), 0, int(col_begin), int(col_count), 0, 0)
        st = lib().opf_reduced_hessian_noalloc(self.h, C.byref(p), C.byref(opts), _ptr(H), C.byref(info))
        if st != 0:
            raise OPFError(st, "opf_reduced_hessian_noalloc")
        return H.T, dict(block_k=info.block_k, grid=info.grid, tiles=info.tiles, launches=info.launches,
                         ms_total=info.ms_total, ms_hvp=info.ms_hvp)

    def _state(self, state):
        for k in ("u", "s", "zl_u", "zu_u", "zl_s", "zu_s", "u_lo", "u_hi", "s_lo", "s_hi", "x"):
            self._dev(state[k])
        return AlState(*[state[k].data_ptr() for k in ("u", "s", "zl_u", "zu_u", "zl_s", "zu_s", "u_lo", "u_hi",
                                                        "s_lo", "s_hi", "x")], float(state["mu"]))

    def al_solve(self, al, state, y, max_outer=20, max_inner=30, eta_primal=1e-5, eta_dual=1e-4, rho_max=1e6,
                 block_k=0, scaling_gmax=0.0):
        """Static OPF by the augmented-Lagrangian outer loop (opf_al_solve).  `al`: sigma_f, the initial
        rho and sigma_c; `y` (cuda float64 [m]) and the state tensors are updated in place, and
        state["mu"] is set to the final barrier parameter.  scaling_gmax > 0 scales the problem by its
        gradients first (sigma_c as the prior).  Returns (info dict with "sigma_c" the constraint
        scales used, history array [outer, 8]: steps, mu, rho, eta_p, E_0, F, delta, 0)."""
        t = self.torch
        self._sync_stream()
        y = self._dev(y)
        keep = [self._dev(al["sigma_c"])]
        p = AlParams(float(al["sigma_f"]), float(al["rho"]), keep[0].data_ptr(), y.data_ptr(), None, None)
        st = self._state(state)
        hist = np.zeros((max(1, int(max_outer)), 8))
        info = AlInfo()
        sig_used = t.empty(self.m, dtype=t.float64, device=self.device)
        rc = lib().opf_al_solve(self.h, C.byref(p), C.c_void_p(y.data_ptr()), C.byref(st),
                                C.byref(AlOpts(int(max_outer), int(max_inner), float(eta_primal), float(eta_dual),
                                               float(rho_max), int(block_k), float(scaling_gmax),
                                               sig_used.data_ptr())),
                                C.byref(info), hist.ctypes.data_as(_dp))
        state["mu"] = st.mu
        if rc != 0:
            raise OPFError(rc, "opf_al_solve")
        out = {k: getattr(info, k) for k, _ in AlInfo._fields_}
        out["sigma_c"] = sig_used
        return out, hist[:info.outer].copy()

    def tracking_update(self, al, state, y, max_it=50, tol=1e-6, block_k=0, max_halvings=0, max_inertia=0,
                        delta_start=0.0, inertia_only=False):
        """One real-time update (opf_tracking_update): gradient and Hessian at the current point, the
        bounded QP of eq. qp_rto by an interior-point method on the Schur complement, the power flow
        at the new controls and the multiplier update.  `al`: sigma_f, rho, sigma_c; y and the state
        tensors are updated in place, state["mu"] is set to the QP's last barrier.  Returns info."""
        self._sync_stream()
        y = self._dev(y)
        keep = [self._dev(al["sigma_c"])]
        p = AlParams(float(al["sigma_f"]), float(al["rho"]), keep[0].data_ptr(), y.data_ptr(), None, None)
        st = self._state(state)
        info = QpInfo()
        rc = lib().opf_tracking_update(self.h, C.byref(p), C.c_void_p(y.data_ptr()), C.byref(st),
                                       C.byref(QpOpts(int(max_it), float(tol), int(block_k), int(max_halvings),
                                                      int(max_inertia), float(delta_start),
                                                      int(bool(inertia_only)))), C.byref(info))
        state["mu"] = st.mu
        if rc != 0:
            raise OPFError(rc, "opf_tracking_update")
        return {k: getattr(info, k) for k, _ in QpInfo._fields_}

    def al_step(self, al, state, block_k=8, max_halvings=0, max_inertia=0, delta_start=0.0, line_search=False):
        """One reduced-Newton step (Prop. 3).  `state`: dict of cuda float64 tensors u, s, zl_u,
        zu_u, zl_s, zu_s, u_lo, u_hi, s_lo, s_hi, x and the float mu; u, s, the duals and x are
        updated in place.  Returns (du, ds, info)."""
        t = self.torch
        self._sync_stream()
        p, keep = self._al(dict(al, s=state["s"]))
        for k in ("u", "s", "zl_u", "zu_u", "zl_s", "zu_s", "u_lo", "u_hi", "s_lo", "s_hi", "x"):
            self._dev(state[k])
        st = AlState(*[state[k].data_ptr() for k in ("u", "s", "zl_u", "zu_u", "zl_s", "zu_s", "u_lo", "u_hi",
                                                      "s_lo", "s_hi", "x")], float(state["mu"]))
        du = t.empty(self.nu, dtype=t.float64, device=self.device)
        ds = t.empty(self.m, dtype=t.float64, device=self.device)
        info = StepInfo()
        rc = lib().opf_al_step(self.h, C.byref(p), C.byref(st),
                               C.byref(StepOpts(int(block_k), int(max_halvings), int(max_inertia), float(delta_start),
                                                int(bool(line_search)))),
                               C.byref(info), _ptr(du), _ptr(ds))
        if rc != 0:
            raise OPFError(rc, "opf_al_step")
        return du, ds, {k: getattr(info, k) for k, _ in StepInfo._fields_}
