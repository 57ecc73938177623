"""CPU oracle (TEST INFRASTRUCTURE ONLY).

Thin ctypes wrapper over ``opf_oracle.c``: plain FP64 C code computing the
power flow, reduced gradient (Prop. 1) and reduced Hessian (Prop. 2) of the
scaled augmented Lagrangian from their definitions.  Only the tests, the
smoke check and the CPU-baseline leg of ``bench.py`` may use it; the library
never imports it.  Networks are passed as any object with the attribute
names of the synthetic generator's ``Network`` (duck typing: this package
imports nothing from the library).

Functions without an independent pin are marked in their docstring
("parity unpinned"); at present every exported function has one.  The
Hessian's columns are shared out over OpenMP threads (OMP_NUM_THREADS; the
arithmetic of a column does not depend on the thread count).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "opf_oracle.c")
_LIB = os.path.join(_HERE, "libopf_oracle.so")
_lib = None

_dp = C.POINTER(C.c_double)
_ip = C.POINTER(C.c_int)


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (portable flags: the .so may run on another host)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < max(
            os.path.getmtime(_SRC), os.path.getmtime(os.path.join(_HERE, "opf_oracle.h"))):
        cmd = ["gcc", "-O2", "-std=c99", "-fopenmp", "-fPIC", "-shared", "-o", _LIB + ".tmp", _SRC, "-lm"]
        subprocess.check_call(cmd)
        os.replace(_LIB + ".tmp", _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        build()
        lib = C.CDLL(_LIB)
        lib.orc_net_new.restype = C.c_void_p
        lib.orc_net_new.argtypes = [C.c_int] * 4 + [_dp] * 4 + [_ip, _ip] + [_dp] * 5 + [_ip] + [_dp] * 7
        lib.orc_net_free.argtypes = [C.c_void_p]
        lib.orc_dims.argtypes = [C.c_void_p] + [_ip] * 5
        lib.orc_symbolic_sizes.argtypes = [C.c_void_p, _ip, _ip]
        lib.orc_symbolic_export.argtypes = [C.c_void_p] + [_ip] * 6
        lib.orc_powerflow.argtypes = [C.c_void_p, _dp, _dp, _dp, _dp, C.c_double, C.c_int, _ip, _dp, _dp]
        lib.orc_eval.argtypes = [C.c_void_p] + [_dp] * 9
        lib.orc_reduced_gradient.argtypes = [C.c_void_p, _dp, _dp, _dp, _dp, C.c_double, C.c_double,
                                             _dp, _dp, _dp] + [_dp] * 7
        lib.orc_reduced_hessian.argtypes = [C.c_void_p, _dp, _dp, _dp, _dp, C.c_double, C.c_double,
                                            _dp, _dp, _dp, _dp, _ip, C.c_int, _dp]
        lib.orc_hvp.argtypes = [C.c_void_p, _dp, _dp, _dp, _dp, C.c_double, C.c_double,
                                _dp, _dp, _dp, _dp, _dp, _dp]
        lib.orc_reduced_jac_prod.argtypes = [C.c_void_p] + [_dp] * 8
        lib.orc_bruteforce.argtypes = [C.c_void_p, _dp, _dp, _dp, _dp, C.c_double, C.c_double,
                                       _dp, _dp, _dp, _dp, _dp, _dp, _dp]
        _lib = lib
    return _lib


def _d(a):
    if a is None:
        return None
    return np.ascontiguousarray(a, dtype=np.float64)


def _pd(a):
    return None if a is None else a.ctypes.data_as(_dp)


def _pi(a):
    return None if a is None else a.ctypes.data_as(_ip)


class OracleError(RuntimeError):
    pass


def _check(rc, what):
    if rc != 0:
        raise OracleError(f"oracle {what} failed with code {rc}")


class OracleNet:
    """One network in the oracle.  Loads are passed per call."""

    def __init__(self, net):
        lib = _load()
        self.net = net
        self._keep = [
            _d(net.pd), _d(net.qd), _d(net.vmin), _d(net.vmax),
            np.ascontiguousarray(net.br_from, dtype=np.int32), np.ascontiguousarray(net.br_to, dtype=np.int32),
            _d(net.br_r), _d(net.br_x), _d(net.br_b), _d(net.br_tap), _d(net.br_rate),
            np.ascontiguousarray(net.gen_bus, dtype=np.int32),
            _d(net.gen_c2), _d(net.gen_c1), _d(net.gen_c0), _d(net.gen_pmin), _d(net.gen_pmax),
            _d(net.gen_qmin), _d(net.gen_qmax)]
        k = self._keep
        self.h = lib.orc_net_new(int(net.n_bus), int(net.n_branch), int(net.n_gen), int(net.ref_bus),
                                 _pd(k[0]), _pd(k[1]), _pd(k[2]), _pd(k[3]), _pi(k[4]), _pi(k[5]),
                                 _pd(k[6]), _pd(k[7]), _pd(k[8]), _pd(k[9]), _pd(k[10]), _pi(k[11]),
                                 *[_pd(a) for a in k[12:]])
        if not self.h:
            raise OracleError("invalid network")
        dims = [C.c_int() for _ in range(5)]
        lib.orc_dims(self.h, *[C.byref(d) for d in dims])
        self.nx, self.nu, self.m, self.npv, self.npq = (d.value for d in dims)

    def __del__(self):
        if getattr(self, "h", None) and _lib is not None:
            _lib.orc_net_free(self.h)
            self.h = None

    # -- symbolic (bit-exact integer work) -----------------------------------
    def symbolic(self) -> dict:
        lib = _load()
        nnz, nsb = C.c_int(), C.c_int()
        _check(lib.orc_symbolic_sizes(self.h, C.byref(nnz), C.byref(nsb)), "symbolic")
        out = dict(bus_order=np.zeros(nsb.value, np.int32), perm=np.zeros(self.nx, np.int32),
                   rowptr=np.zeros(self.nx + 1, np.int32), colidx=np.zeros(nnz.value, np.int32),
                   lev_f=np.zeros(self.nx, np.int32), lev_b=np.zeros(self.nx, np.int32))
        _check(lib.orc_symbolic_export(self.h, *[_pi(out[k]) for k in
                                                 ("bus_order", "perm", "rowptr", "colidx", "lev_f", "lev_b")]),
               "symbolic export")
        return out

    # -- power flow ------------------------------------------------------------
    def powerflow(self, u, pd=None, qd=None, x0=None, tol=1e-10, max_it=20):
        lib = _load()
        pd = _d(self.net.pd if pd is None else pd)
        qd = _d(self.net.qd if qd is None else qd)
        u = _d(u)
        if x0 is None:
            x = np.concatenate([np.zeros(self.npv + self.npq), np.ones(self.npq)])
        else:
            x = _d(x0).copy()
        it, r2, ri = C.c_int(), C.c_double(), C.c_double()
        rc = lib.orc_powerflow(self.h, _pd(u), _pd(pd), _pd(qd), _pd(x), float(tol), int(max_it),
                               C.byref(it), C.byref(r2), C.byref(ri))
        return x, dict(rc=rc, iterations=it.value, res2=r2.value, resinf=ri.value)

    def eval(self, x, u, pd=None, qd=None):
        lib = _load()
        pd = _d(self.net.pd if pd is None else pd)
        qd = _d(self.net.qd if qd is None else qd)
        g = np.zeros(self.nx)
        c = np.zeros(self.m)
        P = np.zeros(self.net.n_bus)
        Q = np.zeros(self.net.n_bus)
        fc = C.c_double()
        _check(lib.orc_eval(self.h, _pd(_d(x)), _pd(_d(u)), _pd(pd), _pd(qd), _pd(g), _pd(c), _pd(P), _pd(Q),
                            C.byref(fc)), "eval")
        return dict(g=g, c=c, P=P, Q=Q, cost=fc.value)

    def _al(self, al):
        return (float(al["sigma_f"]), float(al["rho"]), _d(al["sigma_c"]), _d(al["y"]), _d(al["s"]))

    def reduced_gradient(self, x, u, al, pd=None, qd=None) -> dict:
        lib = _load()
        pd = _d(self.net.pd if pd is None else pd)
        qd = _d(self.net.qd if qd is None else qd)
        sf, rho, sc, y, s = self._al(al)
        F = C.c_double()
        out = dict(grad_u=np.zeros(self.nu), grad_s=np.zeros(self.m), c=np.zeros(self.m),
                   lam=np.zeros(self.nx), grad_pd=np.zeros(self.net.n_bus), grad_qd=np.zeros(self.net.n_bus))
        _check(lib.orc_reduced_gradient(self.h, _pd(_d(x)), _pd(_d(u)), _pd(pd), _pd(qd), sf, rho, _pd(sc),
                                        _pd(y), _pd(s), C.byref(F), _pd(out["grad_u"]), _pd(out["grad_s"]),
                                        _pd(out["c"]), _pd(out["lam"]), _pd(out["grad_pd"]),
                                        _pd(out["grad_qd"])), "reduced_gradient")
        out["F"] = F.value
        return out

    def reduced_hessian(self, x, u, al, omega=None, cols=None, pd=None, qd=None) -> np.ndarray:
        """Columns of the reduced Hessian (n_u x len(cols)), one HVP per column (Prop. 2)."""
        lib = _load()
        pd = _d(self.net.pd if pd is None else pd)
        qd = _d(self.net.qd if qd is None else qd)
        sf, rho, sc, y, s = self._al(al)
        cols = np.arange(self.nu, dtype=np.int32) if cols is None else np.ascontiguousarray(cols, np.int32)
        H = np.zeros((len(cols), self.nu))  # row c = column cols[c] (column-major storage)
        _check(lib.orc_reduced_hessian(self.h, _pd(_d(x)), _pd(_d(u)), _pd(pd), _pd(qd), sf, rho, _pd(sc),
                                       _pd(y), _pd(s), _pd(_d(omega)), _pi(cols), len(cols), _pd(H)),
               "reduced_hessian")
        return H.T.copy()

    def hvp(self, x, u, al, w, omega=None, pd=None, qd=None) -> np.ndarray:
        lib = _load()
        pd = _d(self.net.pd if pd is None else pd)
        qd = _d(self.net.qd if qd is None else qd)
        sf, rho, sc, y, s = self._al(al)
        Hw = np.zeros(self.nu)
        _check(lib.orc_hvp(self.h, _pd(_d(x)), _pd(_d(u)), _pd(pd), _pd(qd), sf, rho, _pd(sc), _pd(y), _pd(s),
                           _pd(_d(omega)), _pd(_d(w)), _pd(Hw)), "hvp")
        return Hw

    def jac_prod(self, x, u, v=None, w=None, pd=None, qd=None):
        """Reduced constraint Jacobian products (J v, J^T w), J = dc/du on g = 0."""
        lib = _load()
        pd = _d(self.net.pd if pd is None else pd)
        qd = _d(self.net.qd if qd is None else qd)
        Jv = np.zeros(self.m) if v is not None else None
        Jtw = np.zeros(self.nu) if w is not None else None
        _check(lib.orc_reduced_jac_prod(self.h, _pd(_d(x)), _pd(_d(u)), _pd(pd), _pd(qd), _pd(_d(v)), _pd(Jv),
                                        _pd(_d(w)), _pd(Jtw)), "jac_prod")
        return Jv, Jtw

    def bruteforce(self, x, u, al, omega=None, pd=None, qd=None) -> dict:
        """Dense reduced Hessian, reduced Jacobian and gradient from hyper-dual numbers (small nets)."""
        lib = _load()
        pd = _d(self.net.pd if pd is None else pd)
        qd = _d(self.net.qd if qd is None else qd)
        sf, rho, sc, y, s = self._al(al)
        H = np.zeros((self.nu, self.nu))
        J = np.zeros((self.nu, self.m))
        gu = np.zeros(self.nu)
        _check(lib.orc_bruteforce(self.h, _pd(_d(x)), _pd(_d(u)), _pd(pd), _pd(qd), sf, rho, _pd(sc), _pd(y),
                                  _pd(s), _pd(_d(omega)), _pd(H), _pd(J), _pd(gu)), "bruteforce")
        return dict(H=H.T.copy(), J=J.T.copy(), grad_u=gu)
