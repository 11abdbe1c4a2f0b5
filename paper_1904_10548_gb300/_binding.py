"""ctypes binding of librapidnet.so (include/rapidnet.h).

Argument marshalling only: every computation runs in the CUDA library.
The module-level functions carry the C names; ``Factor`` bundles them for
numpy (host) and torch (device) arrays.  Importing this module does not
need a GPU; loading the library does need it to be built
(``__graft_entry__.build()``), and a missing library is an error, never
a fallback.
"""
from __future__ import annotations

import ctypes
import os
from ctypes import POINTER, c_double, c_int, c_longlong, c_void_p

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "librapidnet.so")

RN_OK = 0
RN_NOT_CONVERGED = 1
RN_ERR_INVAL = -1
RN_ERR_RANK = -2
RN_ERR_CUDA = -3
RN_ERR_TIMEOUT = -4
RN_ERR_NOMEM = -5
RN_ERR_UNSUPPORTED = -6
RN_ERR_DIVERGED = -7
RN_PREC_FP64 = 0
RN_NOALLOC_SCRATCH_BYTES = 8 << 20  # rapidnet.h
RN_PREC_MIXED = 1
RN_PREC_FP32 = 2
RN_FACTOR_AUTO = 0
RN_FACTOR_SHARED = 1
RN_FACTOR_PER_NODE = 2
RN_THETA_EQUALITY = 0
RN_THETA_SIMPLE = 1

STATUS_NAMES = {0: "RN_OK", 1: "RN_NOT_CONVERGED", -1: "RN_ERR_INVAL", -2: "RN_ERR_RANK",
                -3: "RN_ERR_CUDA", -4: "RN_ERR_TIMEOUT", -5: "RN_ERR_NOMEM",
                -6: "RN_ERR_UNSUPPORTED", -7: "RN_ERR_DIVERGED"}

PD = POINTER(c_double)
PI = POINTER(c_int)


class rn_network(ctypes.Structure):
    _fields_ = [("nx", c_int), ("nu", c_int), ("nd", c_int), ("ne", c_int),
                ("A", PD), ("B", PD), ("Gd", PD), ("E", PD), ("Ed", PD),
                ("xmin", PD), ("xmax", PD), ("xs", PD), ("umin", PD), ("umax", PD)]


class rn_tree(ctypes.Structure):
    _fields_ = [("N", c_int), ("n_nodes", c_int), ("stage_ptr", PI), ("anc", PI), ("prob", PD)]


class rn_cost(ctypes.Structure):
    _fields_ = [("W_alpha", c_double), ("alpha0", PD), ("Wu", PD), ("Ws", c_double),
                ("Wx", c_double)]


class rn_opts(ctypes.Structure):
    _fields_ = [("device", c_int), ("stream", c_void_p), ("precision", c_int),
                ("gamma", c_double), ("power_iters", c_int), ("check_every", c_int),
                ("refresh_every", c_int), ("max_ctas", c_int), ("block_threads", c_int),
                ("wait_us", c_int), ("theta_rule", c_int), ("batch_tune", c_int),
                ("factor_form", c_int)]


class rn_result(ctypes.Structure):
    _fields_ = [("u", PD), ("x", PD), ("y", PD), ("res_hist", PD), ("res_hist_len", c_int),
                ("compute_gap", c_int), ("iters", c_int), ("n_checks", c_int),
                ("primal_res", c_double), ("ubox_viol", c_double), ("cost", c_double),
                ("gap", c_double), ("gamma", c_double), ("apg_ms", c_double),
                ("t_begin_ns", c_longlong), ("t_end_ns", c_longlong),
                ("u_avg", PD), ("x_avg", PD)]


RESULT_SCALARS = ("iters", "n_checks", "primal_res", "ubox_viol", "cost", "gap", "gamma",
                  "apg_ms", "t_begin_ns", "t_end_ns")


class rn_solve_req(ctypes.Structure):
    _fields_ = [("x0", c_void_p), ("q", c_void_p), ("demand", c_void_p), ("alpha", c_void_p),
                ("y_warm", c_void_p), ("out", POINTER(rn_result))]


class rn_server_opts(ctypes.Structure):
    _fields_ = [("device", c_int), ("budget_bytes", c_longlong), ("max_queue", c_int),
                ("workers", c_int), ("slots_per_model", c_int)]


class rn_server_stats(ctypes.Structure):
    _fields_ = [("submitted", c_longlong), ("completed", c_longlong), ("rejected", c_longlong),
                ("slots", c_int), ("models", c_int), ("bytes_in_use", c_longlong),
                ("p50_s", c_double), ("p99_s", c_double), ("mean_s", c_double)]


class rn_tree_out(ctypes.Structure):
    _fields_ = [("max_nodes", c_int), ("n_nodes", c_int), ("stage_ptr", PI), ("anc", PI),
                ("prob", PD), ("value", PD), ("rep", PI), ("leaf_of", PI)]


class rn_factor_info(ctypes.Structure):
    _fields_ = [("nx", c_int), ("nu", c_int), ("nd", c_int), ("ne", c_int), ("N", c_int),
                ("n_nodes", c_int), ("n_chains", c_int), ("n_top", c_int),
                ("grid_ctas", c_int), ("block_threads", c_int), ("L", c_double),
                ("gamma", c_double), ("precision", c_int), ("device_bytes", c_longlong),
                ("collapse_dev", c_double), ("noalloc_bytes", c_longlong),
                ("factor_form", c_int)]


EXPORTS = {
    "rapidnet_factor": (c_int, [POINTER(rn_network), POINTER(rn_tree), POINTER(rn_cost),
                                POINTER(rn_opts), POINTER(c_void_p)]),
    "rapidnet_factor_free": (None, [c_void_p]),
    "rapidnet_factor_info": (c_int, [c_void_p, POINTER(rn_factor_info)]),
    "rapidnet_solve": (c_int, [c_void_p, PD, PD, PD, PD, c_int, c_double, PD,
                               POINTER(rn_result)]),
    "rapidnet_solve_device": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_int,
                                      c_double, c_void_p, POINTER(rn_result)]),
    "rapidnet_dual_gradient_device": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p, c_void_p,
                                              c_void_p, c_void_p, c_void_p]),
    "rapidnet_dual_gradient_noalloc": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p]),
    "rapidnet_solve_batch": (c_int, [POINTER(c_void_p), POINTER(rn_solve_req), c_int, c_int,
                                     c_double]),
    "rapidnet_server_create": (c_int, [POINTER(rn_server_opts), POINTER(c_void_p)]),
    "rapidnet_server_add_model": (c_int, [c_void_p, POINTER(rn_network), POINTER(rn_tree),
                                          POINTER(rn_cost), POINTER(rn_opts), POINTER(c_int)]),
    "rapidnet_server_submit": (c_int, [c_void_p, c_int, PD, PD, PD, PD, c_int, c_double, c_int,
                                       POINTER(c_longlong)]),
    "rapidnet_server_wait": (c_int, [c_void_p, c_longlong, c_double, POINTER(rn_result),
                                     POINTER(c_double)]),
    "rapidnet_server_stats": (c_int, [c_void_p, POINTER(rn_server_stats)]),
    "rapidnet_server_destroy": (None, [c_void_p]),
    "rapidnet_scenario_tree": (c_int, [PD, PD, c_int, c_int, c_int, PI, c_int,
                                       POINTER(rn_tree_out)]),
    "rapidnet_pernode_matrices": (c_int, [POINTER(rn_network), POINTER(rn_tree),
                                          POINTER(rn_cost), PD, PD, PD]),
    "rapidnet_last_error": (ctypes.c_char_p, []),
}

_lib = None


def load() -> ctypes.CDLL:
    """Load librapidnet.so; raises if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} is missing: build it with __graft_entry__.build()")
        lib = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in EXPORTS.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib


class RapidNetError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


def rapidnet_last_error() -> str:
    return load().rapidnet_last_error().decode()


def _check(rc: int) -> int:
    if rc < 0:
        raise RapidNetError(rc, rapidnet_last_error())
    return rc


def rapidnet_factor(net, tree, cost, opts):
    h = c_void_p()
    _check(load().rapidnet_factor(ctypes.byref(net), ctypes.byref(tree), ctypes.byref(cost),
                                  ctypes.byref(opts), ctypes.byref(h)))
    return h


def rapidnet_factor_free(h) -> None:
    load().rapidnet_factor_free(h)


def rapidnet_factor_info(h) -> rn_factor_info:
    info = rn_factor_info()
    _check(load().rapidnet_factor_info(h, ctypes.byref(info)))
    return info


def rapidnet_solve(h, x0, q, demand, alpha, max_iters, tol, y_warm, res) -> int:
    return _check(load().rapidnet_solve(h, x0, q, demand, alpha, int(max_iters), float(tol),
                                        y_warm, ctypes.byref(res)))


def rapidnet_solve_device(h, x0, q, demand, alpha, max_iters, tol, y_warm, res) -> int:
    return _check(load().rapidnet_solve_device(h, x0, q, demand, alpha, int(max_iters),
                                               float(tol), y_warm, ctypes.byref(res)))


def rapidnet_dual_gradient_device(h, x0, q, demand, alpha, w, u, x) -> int:
    return _check(load().rapidnet_dual_gradient_device(h, x0, q, demand, alpha, w, u, x))


def rapidnet_solve_batch(handles, reqs, n, max_iters, tol) -> int:
    return _check(load().rapidnet_solve_batch(handles, reqs, int(n), int(max_iters), float(tol)))


def solve_batch(factors, data, max_iters: int, tol: float = 0.0, outs=None) -> list:
    """Batched solve of several mixed-precision factors (rapidnet_solve_batch).
    data[i] = (x0, q, demand, alpha[, y_warm]) as float64 CUDA tensors;
    outs[i] = (u, x, y) CUDA tensors (allocated here when omitted)."""
    import torch
    n = len(factors)
    handles = (c_void_p * n)(*[f.h.value if isinstance(f.h, c_void_p) else f.h for f in factors])
    results = (rn_result * n)()
    reqs = (rn_solve_req * n)()
    keep = []
    for i, (f, d) in enumerate(zip(factors, data)):
        if outs is None:
            u = torch.empty((f.n_nodes, f.nu), dtype=torch.float64, device="cuda")
            x = torch.empty((f.n_nodes, f.nx), dtype=torch.float64, device="cuda")
            y = torch.empty((f.n_nodes, f.ny), dtype=torch.float64, device="cuda")
        else:
            u, x, y = outs[i]
        keep.append((u, x, y))
        results[i].u = ctypes.cast(_dev_ptr(u), PD)
        results[i].x = ctypes.cast(_dev_ptr(x), PD)
        results[i].y = ctypes.cast(_dev_ptr(y), PD)
        yw = d[4] if len(d) > 4 else None
        reqs[i] = rn_solve_req(_dev_ptr(d[0]), _dev_ptr(d[1]), _dev_ptr(d[2]), _dev_ptr(d[3]),
                               _dev_ptr(yw), ctypes.pointer(results[i]))
    rc = rapidnet_solve_batch(handles, reqs, n, max_iters, tol)
    out = []
    for i in range(n):
        r = results[i]
        out.append(dict(status=rc, iters=r.iters, n_checks=r.n_checks, primal_res=r.primal_res,
                        ubox_viol=r.ubox_viol, cost=r.cost, gamma=r.gamma, apg_ms=r.apg_ms,
                        u=keep[i][0], x=keep[i][1], y=keep[i][2]))
    return out


class Server:
    """Continuous-batching solve server (rapidnet_server_*): models are
    added once (resident factors), requests are submitted with host arrays
    and waited for by ticket."""

    def __init__(self, device: int = 0, budget_bytes: int = 0, max_queue: int = 0,
                 workers: int = 0, slots_per_model: int = 0):
        self.h = c_void_p()
        _check(load().rapidnet_server_create(
            ctypes.byref(rn_server_opts(device, budget_bytes, max_queue, workers,
                                        slots_per_model)),
            ctypes.byref(self.h)))
        self.models = {}

    def add_model(self, net, cost, tree, precision: int = RN_PREC_MIXED, gamma: float = 0.0,
                  **kw) -> int:
        spec = Factor.__new__(Factor)
        Factor._marshal(spec, net, cost, tree, precision, gamma, 0, None, **kw)
        key = c_int()
        _check(load().rapidnet_server_add_model(self.h, ctypes.byref(spec.net_c),
                                                ctypes.byref(spec.tree_c),
                                                ctypes.byref(spec.cost_c),
                                                ctypes.byref(spec.opts_c), ctypes.byref(key)))
        self.models[key.value] = spec
        return key.value

    def submit(self, key: int, x0, q, demand, alpha, max_iters: int, tol: float = 0.0,
               warm: bool = False) -> int:
        m = self.models[key]
        arrs = [_f64(x0, (m.nx,)), _f64(q, (m.nu,)), _f64(demand, (m.n_nodes, m.nd)),
                _f64(alpha, (m.n_nodes, m.nu))]
        t = c_longlong()
        _check(load().rapidnet_server_submit(self.h, key, *[_pd(a) for a in arrs], int(max_iters),
                                             float(tol), int(warm), ctypes.byref(t)))
        return t.value

    def wait(self, key: int, ticket: int, timeout_s: float = -1.0) -> dict:
        m = self.models[key]
        u = np.empty((m.n_nodes, m.nu))
        x = np.empty((m.n_nodes, m.nx))
        y = np.empty((m.n_nodes, m.ny))
        res = rn_result(_pd(u), _pd(x), _pd(y), None, 0, 0)
        lat = c_double()
        rc = _check(load().rapidnet_server_wait(self.h, ticket, float(timeout_s),
                                                ctypes.byref(res), ctypes.byref(lat)))
        out = {f: getattr(res, f) for f in RESULT_SCALARS}
        out.update(status=rc, u=u, x=x, y=y, latency_s=lat.value)
        return out

    def stats(self) -> dict:
        st = rn_server_stats()
        _check(load().rapidnet_server_stats(self.h, ctypes.byref(st)))
        return {f: getattr(st, f) for f, _ in rn_server_stats._fields_}

    def close(self) -> None:
        if getattr(self, "h", None):
            load().rapidnet_server_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def pernode_matrices(net, cost, tree) -> dict:
    """rapidnet_pernode_matrices: the per-node matrices of the general
    recursion as the per-node form's factor step computes them (FP64, on the
    host, no device work): Phi, K (n_nodes, nu, nu) and Mc (n_nodes, nu, ne)."""
    spec = Factor.__new__(Factor)
    Factor._marshal(spec, net, cost, tree, RN_PREC_FP64, 0.0, 0, None)
    n, nu, ne = spec.n_nodes, spec.nu, spec.ne
    Phi = np.zeros((n, nu, nu))
    K = np.zeros((n, nu, nu))
    Mc = np.zeros((n, nu, max(ne, 1)))
    _check(load().rapidnet_pernode_matrices(ctypes.byref(spec.net_c), ctypes.byref(spec.tree_c),
                                            ctypes.byref(spec.cost_c), _pd(Phi), _pd(K),
                                            _pd(Mc)))
    return {"Phi": Phi, "K": K, "Mc": Mc[:, :, :ne]}


def scenario_tree(paths, branching, prob=None, device: int = 0) -> dict:
    """rapidnet_scenario_tree: paths (S, N, dim) host array, branching (N,);
    returns the tree (stage_ptr, anc, prob, value, rep, leaf_of)."""
    P = _f64(paths)
    if P.ndim == 2:
        P = P[:, :, None]
    S, N, dim = P.shape
    br = np.ascontiguousarray(branching, dtype=np.int32)
    if br.shape != (N,):
        raise ValueError("branching needs one entry per stage")
    cap, level = 1, 1
    for b in br:
        level *= int(max(b, 1))
        cap += min(level, S)
    stage_ptr = np.zeros(N + 2, dtype=np.int32)
    anc = np.zeros(cap, dtype=np.int32)
    prb = np.zeros(cap)
    value = np.zeros((cap, dim))
    rep = np.zeros(cap, dtype=np.int32)
    leaf = np.zeros(S, dtype=np.int32)
    out = rn_tree_out(cap, 0, stage_ptr.ctypes.data_as(PI), anc.ctypes.data_as(PI), _pd(prb),
                      _pd(value), rep.ctypes.data_as(PI), leaf.ctypes.data_as(PI))
    p = None if prob is None else _f64(prob, (S,))
    _check(load().rapidnet_scenario_tree(_pd(P), None if p is None else _pd(p), S, N, dim,
                                         br.ctypes.data_as(PI), device, ctypes.byref(out)))
    n = out.n_nodes
    return dict(n_nodes=n, stage_ptr=stage_ptr, anc=anc[:n], prob=prb[:n], value=value[:n],
                rep=rep[:n], leaf_of=leaf)


def rapidnet_dual_gradient_noalloc(h, w, u, x) -> int:
    return _check(load().rapidnet_dual_gradient_noalloc(h, w, u, x))


# ---------------------------------------------------------------------------
# convenience wrapper
# ---------------------------------------------------------------------------
def _f64(a, shape=None) -> np.ndarray:
    a = np.ascontiguousarray(np.asarray(a, dtype=np.float64))
    if shape is not None:
        a = a.reshape(shape)
    return a


def _pd(a: np.ndarray):
    return a.ctypes.data_as(PD)


def _dev_ptr(t):
    """Device address of a contiguous float64 CUDA tensor (or None)."""
    if t is None:
        return None
    if not (t.is_cuda and t.is_contiguous()):
        raise ValueError("expected a contiguous CUDA tensor")
    import torch
    if t.dtype != torch.float64:
        raise ValueError("expected float64")
    return c_void_p(t.data_ptr())


class Factor:
    """A factor handle (paper Table 2: Engine::factorStep) with solve calls."""

    def __init__(self, net, cost, tree, precision: int = RN_PREC_FP64, gamma: float = 0.0,
                 device: int = 0, stream=None, power_iters: int = 0, check_every: int = 0,
                 refresh_every: int = 0, max_ctas: int = 0, block_threads: int = 0,
                 wait_us: int = 0, theta_rule: int = 0, batch_tune: int = 0,
                 factor_form: int = RN_FACTOR_AUTO):
        self._marshal(net, cost, tree, precision, gamma, device, stream, power_iters,
                      check_every, refresh_every, max_ctas, block_threads, wait_us, theta_rule,
                      batch_tune, factor_form)
        self.h = rapidnet_factor(self.net_c, self.tree_c, self.cost_c, self.opts_c)

    def _marshal(self, net, cost, tree, precision, gamma, device, stream, power_iters=0,
                 check_every=0, refresh_every=0, max_ctas=0, block_threads=0, wait_us=0,
                 theta_rule=0, batch_tune=0, factor_form=RN_FACTOR_AUTO):
        nx, nu, nd, ne = net.nx, net.nu, net.nd, net.ne
        self._keep = [
            _f64(net.A, (nx, nx)), _f64(net.B, (nx, nu)), _f64(net.Gd, (nx, nd)),
            _f64(net.E, (ne, nu)) if ne else np.zeros((1, nu)),
            _f64(net.Ed, (ne, nd)) if ne else np.zeros((1, nd)),
            _f64(net.xmin), _f64(net.xmax), _f64(net.xs), _f64(net.umin), _f64(net.umax),
            np.ascontiguousarray(tree.stage_ptr, dtype=np.int32),
            np.ascontiguousarray(tree.anc, dtype=np.int32), _f64(tree.prob),
            _f64(cost.alpha0), _f64(cost.Wu, (nu, nu)),
        ]
        k = self._keep
        self.net_c = rn_network(nx, nu, nd, ne, *[_pd(a) for a in k[:10]])
        self.tree_c = rn_tree(int(tree.N), int(tree.stage_ptr[-1]), k[10].ctypes.data_as(PI),
                              k[11].ctypes.data_as(PI), _pd(k[12]))
        self.cost_c = rn_cost(float(cost.W_alpha), _pd(k[13]), _pd(k[14]), float(cost.Ws),
                              float(cost.Wx))
        st = None if stream is None else c_void_p(getattr(stream, "cuda_stream", stream))
        self.opts_c = rn_opts(device, st, precision, gamma, power_iters, check_every,
                              refresh_every, max_ctas, block_threads, wait_us, theta_rule,
                              batch_tune, factor_form)
        self.nx, self.nu, self.nd, self.ne = nx, nu, nd, ne
        self.n_nodes = int(tree.stage_ptr[-1])
        self.ny = 2 * nx + nu

    def info(self) -> dict:
        i = rapidnet_factor_info(self.h)
        return {f: getattr(i, f) for f, _ in rn_factor_info._fields_}

    def solve(self, x0, q, demand, alpha, max_iters: int, tol: float = 0.0, y_warm=None,
              compute_gap: bool = False, res_hist_len: int = 0, out=None,
              average: bool = False) -> dict:
        """Host arrays in and out (rapidnet_solve).  ``out`` may supply
        contiguous float64 arrays (u, x, y), e.g. views of pinned memory.
        average: also return the averaged primal iterate (u_avg, x_avg)."""
        n = self.n_nodes
        x0 = _f64(x0, (self.nx,))
        q = _f64(q, (self.nu,))
        demand = _f64(demand, (n, self.nd))
        alpha = _f64(alpha, (n, self.nu))
        yw = None if y_warm is None else _f64(y_warm, (n, self.ny))
        if out is not None:
            u, x, y = out
            for a, shp in ((u, (n, self.nu)), (x, (n, self.nx)), (y, (n, self.ny))):
                if a.dtype != np.float64 or a.shape != shp or not a.flags.c_contiguous:
                    raise ValueError("out arrays must be C-contiguous float64 of the output shapes")
        else:
            u = np.empty((n, self.nu))
            x = np.empty((n, self.nx))
            y = np.empty((n, self.ny))
        hist = np.zeros(max(res_hist_len, 1))
        res = rn_result(_pd(u), _pd(x), _pd(y), _pd(hist) if res_hist_len else None,
                        res_hist_len, int(compute_gap))
        if average:
            ua, xa = np.empty((n, self.nu)), np.empty((n, self.nx))
            res.u_avg, res.x_avg = _pd(ua), _pd(xa)
        rc = rapidnet_solve(self.h, _pd(x0), _pd(q), _pd(demand), _pd(alpha), max_iters, tol,
                            None if yw is None else _pd(yw), res)
        out = {f: getattr(res, f) for f in RESULT_SCALARS}
        out.update(status=rc, u=u, x=x, y=y,
                   res_hist=hist[:min(res_hist_len, res.n_checks)] if res_hist_len else None)
        if average:
            out.update(u_avg=ua, x_avg=xa)
        return out

    def solve_device(self, x0, q, demand, alpha, max_iters: int, tol: float, u, x, y,
                     y_warm=None, compute_gap: bool = False, res_hist=None, u_avg=None,
                     x_avg=None) -> dict:
        """torch CUDA float64 tensors in and out (rapidnet_solve_device)."""
        res = rn_result(ctypes.cast(_dev_ptr(u), PD), ctypes.cast(_dev_ptr(x), PD),
                        ctypes.cast(_dev_ptr(y), PD),
                        ctypes.cast(_dev_ptr(res_hist), PD) if res_hist is not None else None,
                        0 if res_hist is None else res_hist.numel(), int(compute_gap))
        if u_avg is not None or x_avg is not None:
            res.u_avg = ctypes.cast(_dev_ptr(u_avg), PD)
            res.x_avg = ctypes.cast(_dev_ptr(x_avg), PD)
        rc = rapidnet_solve_device(self.h, _dev_ptr(x0), _dev_ptr(q), _dev_ptr(demand),
                                   _dev_ptr(alpha), max_iters, tol, _dev_ptr(y_warm), res)
        out = {f: getattr(res, f) for f in RESULT_SCALARS}
        out["status"] = rc
        return out

    def dual_gradient_device(self, w, u, x, x0=None, q=None, demand=None, alpha=None) -> None:
        rapidnet_dual_gradient_device(self.h, _dev_ptr(x0), _dev_ptr(q), _dev_ptr(demand),
                                      _dev_ptr(alpha), _dev_ptr(w), _dev_ptr(u), _dev_ptr(x))

    def dual_gradient_noalloc(self, w, u, x) -> None:
        """x*(w) with the library's fixed scratch array (no allocation)."""
        rapidnet_dual_gradient_noalloc(self.h, _dev_ptr(w), _dev_ptr(u), _dev_ptr(x))

    def close(self) -> None:
        if getattr(self, "h", None):
            rapidnet_factor_free(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
