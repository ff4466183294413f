"""Python binding of libzkq (argument marshalling only; every compute step runs in the CUDA library).

Accurate batched Hermitian eigensolves for MPS circuit simulation (arXiv:2402.11868, Section 2):
an FP64 Jacobi eigensolve followed by precision recovery to double-double or quad-double.

Functions mirror the C ABI in include/zkq.h and take either integers (raw pointers) or torch tensors
(their data_ptr is passed).  Streams may be a torch.cuda.Stream, an int handle, or None.
"""
from __future__ import annotations

import ctypes
import os
import threading

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libzkq.so")
_lib = None
_lock = threading.Lock()

ZKQ_OK, ZKQ_EINVAL, ZKQ_ENOMEM, ZKQ_ENOCONV, ZKQ_ETIMEOUT, ZKQ_ECUDA, ZKQ_EADMIT, ZKQ_ETOOBIG = range(8)
ZKQ_NOALLOC_SCRATCH_BYTES = 32 * 1024 * 1024
ZKQ_FP64, ZKQ_DD, ZKQ_QD = 1, 2, 4
ZKQ_PLAIN_RQI, ZKQ_OA_OZAKI, ZKQ_OA_FP64, ZKQ_SVD_OA = 0, 1, 2, 3


class ZkqError(RuntimeError):
    def __init__(self, status: int, what: str):
        msg = lib().zkq_status_string(status).decode()
        if status == ZKQ_ECUDA:
            msg += f" (cuda error {lib().zkq_last_cuda_error()})"
        super().__init__(f"{what}: {msg}")
        self.status = status


class _Config(ctypes.Structure):
    _fields_ = [("device", ctypes.c_int), ("max_sweeps", ctypes.c_int), ("rqi_max_iter", ctypes.c_int),
                ("oa_max_iter", ctypes.c_int), ("jacobi_cluster", ctypes.c_int)]


def build(force: bool = False) -> str:
    from . import buildlib as _b
    return _b.build(force=force)


def lib():
    """Load libzkq.so; raises if it has not been built (there is no fallback path)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(f"libzkq.so not built at {LIB_PATH}; run paper_2402_11868_gb300.build()")
            L = ctypes.CDLL(LIB_PATH)
            P, I, I64 = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64
            L.zkq_status_string.restype = ctypes.c_char_p
            L.zkq_status_string.argtypes = [I]
            L.zkq_last_cuda_error.restype = I
            L.zkq_ctx_create.restype = I
            L.zkq_ctx_create.argtypes = [ctypes.POINTER(P), ctypes.POINTER(_Config)]
            L.zkq_ctx_destroy.restype = I
            L.zkq_ctx_destroy.argtypes = [P]
            L.zkq_eigh_batched.restype = I
            L.zkq_eigh_batched.argtypes = [P, I, P, P, P, I, P, P, P, P]
            L.zkq_eigh_batched_noalloc.restype = I
            L.zkq_eigh_batched_noalloc.argtypes = [I, P, P, P, I, P, P, P, P]
            L.zkq_svd_batched.restype = I
            L.zkq_svd_batched.argtypes = [P, I, P, P, P, P, I, P, P, P, P, P, P, P]
            L.zkq_rqi_refine.restype = I
            L.zkq_rqi_refine.argtypes = [P, I, P, P, P, I, P, P, I, I, P, P, P, P, P]
            L.zkq_mw_gemm.restype = I
            L.zkq_mw_gemm.argtypes = [P, I, P, P, P, P, P, P, I, P, P, I, P, P, I, I, I, P]
            L.zkq_profile_classes.restype = I
            L.zkq_profile_class_name.restype = ctypes.c_char_p
            L.zkq_profile_class_name.argtypes = [I]
            L.zkq_profile_enable.restype = I
            L.zkq_profile_enable.argtypes = [I]
            L.zkq_profile_read.restype = I
            L.zkq_profile_read.argtypes = [P, P, P, I]
            for nm, args in (("zkq_mps_create", [P, I, I, I, ctypes.POINTER(P)]), ("zkq_mps_destroy", [P]),
                             ("zkq_mps_bond_dims", [P, P]), ("zkq_mps_download", [P, P, P, P]),
                             ("zkq_mps_upload", [P, P, P, P, P]), ("zkq_mps_apply1q", [P, P, I, P, P]),
                             ("zkq_mps_apply2q", [P, P, I, P, ctypes.c_double, I, P, P, P]),
                             ("zkq_mps_expect1", [P, P, I, P, P, P, P]), ("zkq_mps_sample", [P, P, I, P, P, P, P]),
                             ("zkq_mps_footprint", [P, I, I, I, I, P, P])):
                getattr(L, nm).restype = I
                getattr(L, nm).argtypes = args
            L.zkq_workspace_size.restype = I
            L.zkq_workspace_size.argtypes = [P, I, P, I, I, I, P]
            L.zkq_ctx_workspace_bytes.restype = I
            L.zkq_ctx_workspace_bytes.argtypes = [P, P]
            L.zkq_autotune_jacobi.restype = I
            L.zkq_autotune_jacobi.argtypes = [P, I, P, I, I, P]
            L.zkq_set_gemm_tile_width.restype = I
            L.zkq_set_gemm_tile_width.argtypes = [I]
            L.zkq_autotune_gemm.restype = I
            L.zkq_autotune_gemm.argtypes = [P, I, P, I, I, P]
            L.zkq_plan_create.restype = I
            L.zkq_plan_create.argtypes = [P, I, P, P, I, I, ctypes.POINTER(P)]
            for nm in ("zkq_plan_execute", "zkq_plan_execute_graph"):
                getattr(L, nm).restype = I
                getattr(L, nm).argtypes = [P, P, P, P, P, P, P, P, P, P]
            L.zkq_plan_destroy.restype = I
            L.zkq_plan_destroy.argtypes = [P]
            L.zkq_set_gemm_kernel.restype = I
            L.zkq_set_gemm_kernel.argtypes = [I]
            L.zkq_get_gemm_kernel.restype = I
            L.zkq_check_device_waits.restype = I
            L.zkq_test_grid_barrier_hook.restype = I
            L.zkq_test_grid_barrier_hook.argtypes = [I, I]
            L.zkq_mw_op.restype = I
            L.zkq_mw_op.argtypes = [I, I, I64, P, P, P, I, P]
            _lib = L
    return _lib


def _ptr(x):
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    if hasattr(x, "ctypes"):
        return x.ctypes.data
    raise TypeError(f"cannot pass {type(x)} as a pointer")


def _stream(s):
    if s is None:
        return None
    if isinstance(s, int):
        return s
    return s.cuda_stream


def _host_array(x, ctype):
    import numpy as np
    dt = np.int32 if ctype is ctypes.c_int32 else np.int64
    a = np.ascontiguousarray(x, dtype=dt)
    return a, a.ctypes.data


def _check(st, what):
    if st != ZKQ_OK:
        raise ZkqError(st, what)


class Context:
    """Owns a zkq_ctx (and its device workspace)."""

    def __init__(self, device: int = 0, max_sweeps: int = 0, rqi_max_iter: int = 0, oa_max_iter: int = 0,
                 jacobi_cluster: int = 0):
        cfg = _Config(device, max_sweeps, rqi_max_iter, oa_max_iter, jacobi_cluster)
        h = ctypes.c_void_p()
        _check(lib().zkq_ctx_create(ctypes.byref(h), ctypes.byref(cfg)), "zkq_ctx_create")
        self.handle = h.value
        self.device = device

    def autotune_jacobi(self, sizes, a_words: int = 4, reps: int = 2):
        """Measure the Jacobi cluster width per order (zkq_autotune_jacobi); returns the chosen widths."""
        import numpy as np
        sz, sp = _host_array(sizes, ctypes.c_int32)
        best = np.zeros(len(sz), dtype=np.int32)
        _check(lib().zkq_autotune_jacobi(self.handle, len(sz), sp, a_words, reps, best.ctypes.data),
               "zkq_autotune_jacobi")
        return [int(x) for x in best]

    def autotune_gemm(self, sizes, words: int = 4, reps: int = 2):
        """Measure the split-product GEMM tile width per order (zkq_autotune_gemm); returns 256 or 128 each."""
        import numpy as np
        sz, sp = _host_array(sizes, ctypes.c_int32)
        best = np.zeros(len(sz), dtype=np.int32)
        _check(lib().zkq_autotune_gemm(self.handle, len(sz), sp, words, reps, best.ctypes.data), "zkq_autotune_gemm")
        return [int(x) for x in best]

    def workspace_bytes(self) -> int:
        """Device bytes of workspace the context holds now (zkq_ctx_workspace_bytes)."""
        b = ctypes.c_size_t()
        _check(lib().zkq_ctx_workspace_bytes(self.handle, ctypes.byref(b)), "zkq_ctx_workspace_bytes")
        return b.value

    def close(self):
        if getattr(self, "handle", None):
            lib().zkq_ctx_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


def zkq_eigh_batched(ctx: Context, n, a_off, A, a_words, W, V, info, stream=None):
    n_arr, n_p = _host_array(n, ctypes.c_int32)
    o_arr, o_p = _host_array(a_off, ctypes.c_int64)
    _check(lib().zkq_eigh_batched(ctx.handle, len(n_arr), n_p, o_p, _ptr(A), a_words, _ptr(W), _ptr(V), _ptr(info),
                                  _stream(stream)), "zkq_eigh_batched")


def zkq_eigh_batched_noalloc(n, a_off, A, a_words, W, V, info, stream=None):
    """zkq_eigh_batched on the current device without any device allocation (fixed library scratch)."""
    n_arr, n_p = _host_array(n, ctypes.c_int32)
    o_arr, o_p = _host_array(a_off, ctypes.c_int64)
    _check(lib().zkq_eigh_batched_noalloc(len(n_arr), n_p, o_p, _ptr(A), a_words, _ptr(W), _ptr(V), _ptr(info),
                                          _stream(stream)), "zkq_eigh_batched_noalloc")


def zkq_svd_batched(ctx: Context, m, n, a_off, A, a_words, S, U, u_off, V, v_off, info, stream=None):
    """FP64 one-sided Jacobi SVD of a batch: A_b = U_b diag(S_b) V_b^H (thin)."""
    m_arr, m_p = _host_array(m, ctypes.c_int32)
    n_arr, n_p = _host_array(n, ctypes.c_int32)
    a_arr, a_p = _host_array(a_off, ctypes.c_int64)
    u_arr, u_p = _host_array(u_off, ctypes.c_int64)
    v_arr, v_p = _host_array(v_off, ctypes.c_int64)
    _check(lib().zkq_svd_batched(ctx.handle, len(m_arr), m_p, n_p, a_p, _ptr(A), a_words, _ptr(S), _ptr(U), u_p,
                                 _ptr(V), v_p, _ptr(info), _stream(stream)), "zkq_svd_batched")


def zkq_rqi_refine(ctx: Context, n, a_off, A, a_words, W, V, target_words, method, W_out, V_out, err_est, info,
                   stream=None):
    n_arr, n_p = _host_array(n, ctypes.c_int32)
    o_arr, o_p = _host_array(a_off, ctypes.c_int64)
    _check(lib().zkq_rqi_refine(ctx.handle, len(n_arr), n_p, o_p, _ptr(A), a_words, _ptr(W), _ptr(V), target_words,
                                method, _ptr(W_out), _ptr(V_out), _ptr(err_est), _ptr(info), _stream(stream)),
           "zkq_rqi_refine")


def zkq_workspace_size(ctx: Context, n, a_words, target_words=0, method=ZKQ_OA_OZAKI) -> int:
    """Device workspace bytes of an eigensolve (and refinement) of the batch on a fresh context."""
    n_arr, n_p = _host_array(n, ctypes.c_int32)
    b = ctypes.c_size_t()
    _check(lib().zkq_workspace_size(ctx.handle, len(n_arr), n_p, a_words, target_words, method, ctypes.byref(b)),
           "zkq_workspace_size")
    return b.value


def zkq_mw_gemm(ctx: Context, m, n, k, opA, A, a_off, wa, B, b_off, wb, C, c_off, wc, p_bits, method, stream=None):
    arrs = [_host_array(x, ctypes.c_int32) for x in (m, n, k, opA)]
    offs = [_host_array(x, ctypes.c_int64) for x in (a_off, b_off, c_off)]
    _check(lib().zkq_mw_gemm(ctx.handle, len(arrs[0][0]), arrs[0][1], arrs[1][1], arrs[2][1], arrs[3][1], _ptr(A),
                             offs[0][1], wa, _ptr(B), offs[1][1], wb, _ptr(C), offs[2][1], wc, p_bits, method,
                             _stream(stream)), "zkq_mw_gemm")


def zkq_mw_op(op: int, words: int, count: int, a, b, out, on_device: bool, stream=None):
    _check(lib().zkq_mw_op(op, words, count, _ptr(a), _ptr(b), _ptr(out), int(bool(on_device)), _stream(stream)),
           "zkq_mw_op")


def zkq_set_gemm_kernel(which: int):
    _check(lib().zkq_set_gemm_kernel(which), "zkq_set_gemm_kernel")


def zkq_set_gemm_tile_width(width: int):
    _check(lib().zkq_set_gemm_tile_width(width), "zkq_set_gemm_tile_width")


def zkq_get_gemm_kernel() -> int:
    return lib().zkq_get_gemm_kernel()


def zkq_check_device_waits():
    _check(lib().zkq_check_device_waits(), "zkq_check_device_waits")


def zkq_test_grid_barrier_hook(extra_arrivals: int, log2_poll_limit: int):
    """Test hook of the cooperative-grid Jacobi's bounded barrier (see include/zkq.h); (0, 22) = defaults."""
    _check(lib().zkq_test_grid_barrier_hook(extra_arrivals, log2_poll_limit), "zkq_test_grid_barrier_hook")


def zkq_profile_enable(on: bool):
    _check(lib().zkq_profile_enable(int(bool(on))), "zkq_profile_enable")


def zkq_profile_read():
    """{class name: (milliseconds, launches, algorithmic flops)} since the last read."""
    import numpy as np
    k = lib().zkq_profile_classes()
    ms = np.zeros(k); n = np.zeros(k, dtype=np.int64); w = np.zeros(k)
    _check(lib().zkq_profile_read(ms.ctypes.data, n.ctypes.data, w.ctypes.data, k), "zkq_profile_read")
    return {lib().zkq_profile_class_name(i).decode(): (float(ms[i]), int(n[i]), float(w[i])) for i in range(k)}


class Plan:
    """Fixed-shape batch: FP64 eigensolve, then plain RQI to `target_words` (0: eigensolve only).  execute()
    only enqueues kernels; execute_graph() replays a CUDA graph captured for the same buffers."""

    def __init__(self, ctx: Context, n, a_off, a_words: int, target_words: int = 0):
        n_arr, n_p = _host_array(n, ctypes.c_int32)
        o_arr, o_p = _host_array(a_off, ctypes.c_int64)
        h = ctypes.c_void_p()
        _check(lib().zkq_plan_create(ctx.handle, len(n_arr), n_p, o_p, a_words, target_words, ctypes.byref(h)),
               "zkq_plan_create")
        self.handle, self.ctx = h.value, ctx

    def execute(self, A, W, V, info, W_out=None, V_out=None, err_est=None, rinfo=None, stream=None):
        _check(lib().zkq_plan_execute(self.handle, _ptr(A), _ptr(W), _ptr(V), _ptr(info), _ptr(W_out), _ptr(V_out),
                                      _ptr(err_est), _ptr(rinfo), _stream(stream)), "zkq_plan_execute")

    def execute_graph(self, A, W, V, info, W_out=None, V_out=None, err_est=None, rinfo=None, stream=None):
        _check(lib().zkq_plan_execute_graph(self.handle, _ptr(A), _ptr(W), _ptr(V), _ptr(info), _ptr(W_out),
                                            _ptr(V_out), _ptr(err_est), _ptr(rinfo), _stream(stream)),
               "zkq_plan_execute_graph")

    def close(self):
        if getattr(self, "handle", None):
            lib().zkq_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class MPS:
    """Device-resident Vidal MPS (|0...0> at creation)."""

    def __init__(self, ctx: Context, n_qubits: int, r_max: int, words: int = 4):
        h = ctypes.c_void_p()
        _check(lib().zkq_mps_create(ctx.handle, n_qubits, r_max, words, ctypes.byref(h)), "zkq_mps_create")
        self.handle, self.ctx, self.n, self.words = h.value, ctx, n_qubits, words

    def close(self):
        if getattr(self, "handle", None):
            lib().zkq_mps_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def bond_dims(self):
        import numpy as np
        chi = np.zeros(self.n - 1, dtype=np.int32)
        _check(lib().zkq_mps_bond_dims(self.handle, chi.ctypes.data), "zkq_mps_bond_dims")
        return chi

    def download(self, stream=None):
        """(chi, gammas (sum 2 chi_l-1 chi_l, 2, w), lambdas (sum chi_l, w)) in the oracle's layout."""
        import numpy as np
        chi = self.bond_dims()
        dims = [1] + list(chi) + [1]
        ng = sum(2 * dims[l] * dims[l + 1] for l in range(self.n))
        g = np.zeros((ng, 2, self.words)); lam = np.zeros((max(1, int(chi.sum())), self.words))
        _check(lib().zkq_mps_download(self.handle, g.ctypes.data, lam.ctypes.data, _stream(stream)), "zkq_mps_download")
        return chi, g, lam[:int(chi.sum())]

    def upload(self, chi, gammas, lambdas, stream=None):
        import numpy as np
        chi = np.ascontiguousarray(chi, dtype=np.int32)
        g = np.ascontiguousarray(gammas, dtype=np.float64); l = np.ascontiguousarray(lambdas, dtype=np.float64)
        _check(lib().zkq_mps_upload(self.handle, chi.ctypes.data, g.ctypes.data, l.ctypes.data, _stream(stream)),
               "zkq_mps_upload")

    def apply1q(self, site, U, stream=None):
        import numpy as np
        u = np.ascontiguousarray(U, dtype=np.float64)
        _check(lib().zkq_mps_apply1q(self.ctx.handle, self.handle, site, u.ctypes.data, _stream(stream)), "zkq_mps_apply1q")

    def apply2q(self, site, G, trunc_tau=0.0, method=ZKQ_OA_OZAKI, stream=None, ctx=None):
        """Returns (new bond dimension, discarded weight).  `ctx` (default: the creating context) supplies
        the workspace; concurrent updates must use different contexts."""
        import numpy as np
        g = np.ascontiguousarray(G, dtype=np.float64)
        nb = ctypes.c_int32(0); dw = ctypes.c_double(0.0)
        c = (ctx or self.ctx).handle
        _check(lib().zkq_mps_apply2q(c, self.handle, site, g.ctypes.data, float(trunc_tau), method,
                                     ctypes.byref(nb), ctypes.byref(dw), _stream(stream)), "zkq_mps_apply2q")
        return nb.value, dw.value

    def expect1(self, sites, ops, stream=None):
        """<O_k> at sites[k] (ops: (count, 4, 2, words) row-major 2x2 operators); returns (count, 2, words)."""
        import numpy as np
        st = np.ascontiguousarray(sites, dtype=np.int32)
        o = np.ascontiguousarray(ops, dtype=np.float64)
        assert o.shape == (len(st), 4, 2, self.words)
        out = np.zeros((len(st), 2, self.words))
        _check(lib().zkq_mps_expect1(self.ctx.handle, self.handle, len(st), st.ctypes.data, o.ctypes.data,
                                     out.ctypes.data, _stream(stream)), "zkq_mps_expect1")
        return out

    def sample(self, u, stream=None):
        """Bit strings by the chain rule from uniforms u (shots, n); returns (bits (shots, n), prob (shots, words))."""
        import numpy as np
        uu = np.ascontiguousarray(u, dtype=np.float64)
        assert uu.ndim == 2 and uu.shape[1] == self.n
        bits = np.zeros(uu.shape, dtype=np.int32)
        prob = np.zeros((uu.shape[0], self.words))
        _check(lib().zkq_mps_sample(self.ctx.handle, self.handle, uu.shape[0], uu.ctypes.data, bits.ctypes.data,
                                    prob.ctypes.data, _stream(stream)), "zkq_mps_sample")
        return bits, prob


# --------------------------------------------------------------------------------------------------
# the remaining entry points under their C names (thin forms of the classes above)
def zkq_status_string(status: int) -> str:
    return lib().zkq_status_string(status).decode()


def zkq_last_cuda_error() -> int:
    return lib().zkq_last_cuda_error()


def zkq_profile_classes() -> int:
    return lib().zkq_profile_classes()


def zkq_profile_class_name(cls: int) -> str:
    return lib().zkq_profile_class_name(cls).decode()


def zkq_ctx_create(device: int = 0, **config) -> Context:
    return Context(device, **config)


def zkq_ctx_destroy(ctx: Context):
    ctx.close()


def zkq_ctx_workspace_bytes(ctx: Context) -> int:
    return ctx.workspace_bytes()


def zkq_autotune_jacobi(ctx: Context, sizes, a_words: int = 4, reps: int = 2):
    return ctx.autotune_jacobi(sizes, a_words, reps)


def zkq_autotune_gemm(ctx: Context, sizes, words: int = 4, reps: int = 2):
    return ctx.autotune_gemm(sizes, words, reps)


def zkq_plan_create(ctx: Context, n, a_off, a_words: int, target_words: int = 0) -> Plan:
    return Plan(ctx, n, a_off, a_words, target_words)


def zkq_plan_execute(plan: Plan, A, W, V, info, W_out=None, V_out=None, err_est=None, rinfo=None, stream=None):
    plan.execute(A, W, V, info, W_out, V_out, err_est, rinfo, stream)


def zkq_plan_execute_graph(plan: Plan, A, W, V, info, W_out=None, V_out=None, err_est=None, rinfo=None,
                           stream=None):
    plan.execute_graph(A, W, V, info, W_out, V_out, err_est, rinfo, stream)


def zkq_plan_destroy(plan: Plan):
    plan.close()


def zkq_mps_create(ctx: Context, n_qubits: int, r_max: int, words: int = 4) -> MPS:
    return MPS(ctx, n_qubits, r_max, words)


def zkq_mps_footprint(ctx: Context, n_qubits: int, r_max: int, words: int = 4, method=ZKQ_OA_OZAKI):
    """(state bytes, gate-update workspace bytes) of an MPS before it is created."""
    a = ctypes.c_size_t(0); b = ctypes.c_size_t(0)
    _check(lib().zkq_mps_footprint(ctx.handle, n_qubits, r_max, words, method, ctypes.byref(a), ctypes.byref(b)),
           "zkq_mps_footprint")
    return a.value, b.value


def zkq_mps_destroy(mps: MPS):
    mps.close()


def zkq_mps_bond_dims(mps: MPS):
    return mps.bond_dims()


def zkq_mps_download(mps: MPS, stream=None):
    return mps.download(stream)


def zkq_mps_upload(mps: MPS, chi, gammas, lambdas, stream=None):
    mps.upload(chi, gammas, lambdas, stream)


def zkq_mps_apply1q(ctx: Context, mps: MPS, site: int, U, stream=None):
    if ctx is not mps.ctx:
        raise ValueError("zkq_mps_apply1q: the MPS uses the context it was created with")
    mps.apply1q(site, U, stream)


def zkq_mps_apply2q(ctx: Context, mps: MPS, site: int, G, trunc_tau=0.0, method=ZKQ_OA_OZAKI, stream=None):
    return mps.apply2q(site, G, trunc_tau, method, stream, ctx=ctx)


def zkq_mps_expect1(ctx: Context, mps: MPS, sites, ops, stream=None):
    if ctx is not mps.ctx:
        raise ValueError("zkq_mps_expect1: the MPS uses the context it was created with")
    return mps.expect1(sites, ops, stream)


def zkq_mps_sample(ctx: Context, mps: MPS, u, stream=None):
    if ctx is not mps.ctx:
        raise ValueError("zkq_mps_sample: the MPS uses the context it was created with")
    return mps.sample(u, stream)


# --------------------------------------------------------------------------------------------------
# batch helpers (host-side packing; no arithmetic of the method)
def batch_offsets(ns):
    """Element offsets a_off and eigenvalue offsets w_off for a list of matrix orders."""
    a_off, w_off, a, w = [], [], 0, 0
    for n in ns:
        a_off.append(a); w_off.append(w)
        a += n * n; w += n
    return a_off, w_off, a, w


def pack(mats, words):
    """Concatenate (n*n, 2, w) word arrays (numpy) into one flat float64 array with `words` words."""
    import numpy as np
    parts = []
    for M in mats:
        M = np.asarray(M, dtype=np.float64)
        if M.shape[-1] < words:
            pad = np.zeros(M.shape[:-1] + (words - M.shape[-1],))
            M = np.concatenate([M, pad], axis=-1)
        elif M.shape[-1] > words:
            raise ValueError("matrix has more words than requested")
        parts.append(M.reshape(-1))
    return np.concatenate(parts) if parts else np.zeros(0)
