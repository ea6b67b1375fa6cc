"""Thin ctypes binding of libqst.so (include/qst.h), same call names as the C ABI.

Only argument marshalling happens here: tensors are passed as raw pointers
(``tensor.data_ptr()`` for CUDA tensors, the array address for NumPy / CPU
buffers) and every step of the computation runs inside libqst's CUDA kernels.
If the shared library is missing, every call raises: there is no fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libqst.so")

QST_OK = 0
QST_E_INVAL = -1
QST_E_INPUT = -2
QST_E_NOMEM = -3
QST_E_CUDA = -4
QST_E_TIMEOUT = -5
QST_E_STATE = -6
QST_E_UNSUPPORTED = -7
QST_W_CLAMP = 1

QST_MAP_CHOL_H = 0
QST_MAP_ABS_P = 1
QST_MAP_CHOL_DELTA = 2
QST_NET_FNN = 0
QST_NET_CNN = 1
QST_STATE_PRODUCT = 0
QST_STATE_GHZI = 1
QST_STATE_W = 2
QST_FP64 = 0
QST_FP32 = 1
QST_MIXED = 2
QST_MIXED_BF16 = 3

EXPORTED = [
    "qst_default_options", "qst_theta_size", "qst_init", "qst_set_params", "qst_get_params",
    "qst_probs", "qst_loss_grad", "qst_step", "qst_reconstruct", "qst_get_rho",
    "qst_state_bytes", "qst_get_state", "qst_set_state", "qst_iterations",
    "qst_kernel_launches", "qst_sync", "qst_strerror", "qst_destroy",
    "qst_timing_enable", "qst_timing_read", "qst_probs_static", "qst_graph_enable",
    "qst_batch_init", "qst_batch_context", "qst_batch_set_params", "qst_batch_step",
    "qst_batch_reconstruct", "qst_batch_kernel_launches", "qst_batch_sync", "qst_batch_destroy",
    "qst_classical_fidelity", "qst_test_state", "qst_sample_counts", "qst_theta_size_net",
    "qst_state_fidelity", "qst_jacobi_schedule",
]

PHASES = ["hidden", "build_T", "x_fwd", "povm_lo", "povm_hi", "povm_adj", "gt", "sym", "w2", "w1", "fused"]


class qst_options(ctypes.Structure):
    _fields_ = [
        ("mapping", ctypes.c_int),
        ("precision", ctypes.c_int),
        ("P", ctypes.c_double),
        ("lr", ctypes.c_double),
        ("eta_minus", ctypes.c_double),
        ("eta_plus", ctypes.c_double),
        ("step_min", ctypes.c_double),
        ("step_max", ctypes.c_double),
        ("leaky_slope", ctypes.c_double),
        ("eig_sweeps", ctypes.c_int),
        ("eig_warm_sweeps", ctypes.c_int),
        ("network", ctypes.c_int),
        ("device_memory_limit", ctypes.c_size_t),
        ("fused_max_qubits", ctypes.c_int),
        ("eig_refine", ctypes.c_int),
    ]


class qst_tuning(ctypes.Structure):
    _fields_ = [
        ("bulk_chunks_per_cta", ctypes.c_int),
        ("fused_ctas_per_sm", ctypes.c_int),
        ("fused_max_qubits", ctypes.c_int),
        ("batch_concurrent_runs", ctypes.c_int),
    ]


class QstError(RuntimeError):
    def __init__(self, status: int, what: str):
        self.status = status
        super().__init__(f"{what}: {strerror(status)} ({status})")


_lib = None


def load(path: str = LIB_PATH) -> ctypes.CDLL:
    """Load libqst.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"{path} not found: build it with paper_2207_05341_gb300.build.build()")
    L = ctypes.CDLL(path)
    vp, i, d, sz = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_size_t
    pd = ctypes.POINTER(ctypes.c_double)
    sig = {
        "qst_default_options": (None, [ctypes.POINTER(qst_options)]),
        "qst_theta_size": (sz, [i]),
        "qst_theta_size_net": (sz, [i, i]),
        "qst_init": (i, [ctypes.POINTER(vp), i, vp, i, ctypes.POINTER(qst_options), vp]),
        "qst_set_params": (i, [vp, vp]),
        "qst_get_params": (i, [vp, vp]),
        "qst_probs": (i, [vp, vp, vp]),
        "qst_loss_grad": (i, [vp, vp, vp, pd, vp]),
        "qst_step": (i, [vp, vp, pd]),
        "qst_reconstruct": (i, [vp, vp, i, vp, pd]),
        "qst_get_rho": (i, [vp, vp, vp, pd]),
        "qst_classical_fidelity": (i, [vp, vp, vp, ctypes.c_longlong, ctypes.c_ulonglong, pd]),
        "qst_state_fidelity": (i, [vp, vp, vp, ctypes.c_double, i, pd]),
        "qst_test_state": (i, [vp, i, d, vp]),
        "qst_sample_counts": (i, [vp, vp, ctypes.c_longlong, ctypes.c_ulonglong, vp, vp]),
        "qst_state_bytes": (sz, [vp]),
        "qst_get_state": (i, [vp, vp, sz]),
        "qst_set_state": (i, [vp, vp, sz]),
        "qst_iterations": (ctypes.c_longlong, [vp]),
        "qst_eig_counts": (i, [vp, ctypes.POINTER(ctypes.c_longlong), ctypes.POINTER(ctypes.c_longlong), pd]),
        "qst_jacobi_schedule": (i, [i, ctypes.POINTER(i), ctypes.POINTER(i), ctypes.POINTER(i), i]),
        "qst_kernel_launches": (ctypes.c_longlong, [vp]),
        "qst_sync": (i, [vp]),
        "qst_strerror": (ctypes.c_char_p, [i]),
        "qst_destroy": (None, [vp]),
        "qst_timing_enable": (i, [vp, i]),
        "qst_timing_read": (i, [vp, pd, ctypes.POINTER(ctypes.c_longlong), i]),
        "qst_probs_static": (i, [i, vp, i, vp, vp, vp]),
        "qst_graph_enable": (i, [vp, i]),
        "qst_get_tuning": (None, [ctypes.POINTER(qst_tuning)]),
        "qst_inject_wait_timeout": (i, [i, i]),
        "qst_set_tuning": (i, [ctypes.POINTER(qst_tuning)]),
        "qst_batch_init": (i, [ctypes.POINTER(vp), i, ctypes.POINTER(ctypes.c_int), vp, i,
                               ctypes.POINTER(qst_options), vp]),
        "qst_batch_context": (vp, [vp, i]),
        "qst_batch_set_params": (i, [vp, i, vp]),
        "qst_batch_step": (i, [vp, ctypes.POINTER(vp), pd]),
        "qst_batch_reconstruct": (i, [vp, ctypes.POINTER(vp), i, ctypes.POINTER(vp), pd]),
        "qst_batch_kernel_launches": (ctypes.c_longlong, [vp]),
        "qst_batch_sync": (i, [vp]),
        "qst_batch_destroy": (None, [vp]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args
    _lib = L
    return L


def ptr(x) -> int | None:
    """Raw address of a torch tensor, NumPy array, integer address or None."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if isinstance(x, np.ndarray):
        if not x.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        return x.ctypes.data
    if hasattr(x, "data_ptr"):
        if not x.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return x.data_ptr()
    raise TypeError(f"cannot take the address of {type(x)!r}")


def strerror(status: int) -> str:
    try:
        return load().qst_strerror(int(status)).decode()
    except RuntimeError:
        return f"status {status}"


def _check(status: int, what: str, allow_warn: bool = True) -> int:
    if status < 0 or (status > 0 and not allow_warn):
        raise QstError(status, what)
    return status


def qst_default_options() -> qst_options:
    o = qst_options()
    load().qst_default_options(ctypes.byref(o))
    return o


def qst_theta_size(N: int) -> int:
    return int(load().qst_theta_size(int(N)))


def tetrahedral_povm_flat() -> np.ndarray:
    """The Sec. 4.1 tetrahedral POVM as the K*2*2 interleaved complex doubles qst_init takes."""
    s = np.array([[1, 1, 1], [-1, -1, 1], [-1, 1, -1], [1, -1, -1]], dtype=float) / np.sqrt(3.0)
    out = np.empty((4, 2, 2, 2), dtype=np.float64)
    for a in range(4):
        x, y, z = s[a]
        m = np.array([[1 + z, x - 1j * y], [x + 1j * y, 1 - z]]) / 4.0
        out[a, :, :, 0] = m.real
        out[a, :, :, 1] = m.imag
    return np.ascontiguousarray(out.reshape(-1))


def qst_init(N: int, povm=None, K: int = 4, opt: qst_options | None = None, stream: int = 0) -> int:
    """Create a context; returns the opaque handle (an integer address)."""
    if povm is None:
        povm = tetrahedral_povm_flat()
    povm = np.ascontiguousarray(povm, dtype=np.float64)
    h = ctypes.c_void_p()
    st = load().qst_init(ctypes.byref(h), int(N), povm.ctypes.data, int(K),
                         ctypes.byref(opt) if opt is not None else None, stream or None)
    _check(st, "qst_init")
    return h.value


def qst_theta_size_net(N: int, network: int) -> int:
    return load().qst_theta_size_net(int(N), int(network))


def qst_set_params(ctx: int, theta) -> int:
    return _check(load().qst_set_params(ctx, ptr(theta)), "qst_set_params")


def qst_get_params(ctx: int, theta) -> int:
    return _check(load().qst_get_params(ctx, ptr(theta)), "qst_get_params")


def qst_probs(ctx: int, rho, p) -> int:
    return _check(load().qst_probs(ctx, ptr(rho), ptr(p)), "qst_probs")


def qst_loss_grad(ctx: int, theta, f, dtheta) -> tuple[float, int]:
    loss = ctypes.c_double()
    st = _check(load().qst_loss_grad(ctx, ptr(theta), ptr(f), ctypes.byref(loss), ptr(dtheta)), "qst_loss_grad")
    return loss.value, st


def qst_step(ctx: int, f, want_loss: bool = True) -> tuple[float | None, int]:
    loss = ctypes.c_double()
    st = _check(load().qst_step(ctx, ptr(f), ctypes.byref(loss) if want_loss else None), "qst_step")
    return (loss.value if want_loss else None), st


def qst_reconstruct(ctx: int, f, iters: int, rho_out=None, want_loss: bool = True) -> tuple[float | None, int]:
    loss = ctypes.c_double()
    st = _check(load().qst_reconstruct(ctx, ptr(f), int(iters), ptr(rho_out),
                                       ctypes.byref(loss) if want_loss else None), "qst_reconstruct")
    return (loss.value if want_loss else None), st


def qst_classical_fidelity(ctx: int, f, P, samples: int = 0, seed: int = 0) -> float:
    """Classical fidelity (Sec. 2.3): exact eq. F_CF for samples == 0, else eq. fc_sample."""
    out = ctypes.c_double()
    _check(load().qst_classical_fidelity(ctx, ptr(f), ptr(P), int(samples), int(seed), ctypes.byref(out)),
           "qst_classical_fidelity")
    return out.value


def qst_state_fidelity(ctx: int, f, psi, w: float = 1.0, sweeps: int = 0) -> float:
    """Quantum fidelity (Sec. 2.3 eq. F_QF via eq. fq_decom) against w |psi><psi| + (1 - w) I / d."""
    out = ctypes.c_double()
    _check(load().qst_state_fidelity(ctx, ptr(f), ptr(psi), float(w), int(sweeps), ctypes.byref(out)),
           "qst_state_fidelity")
    return out.value


def qst_test_state(ctx: int, kind: int, w: float, rho) -> int:
    """rho = w |psi><psi| + (1 - w) I / d for QST_STATE_PRODUCT / GHZI / W (device d x d complex)."""
    return _check(load().qst_test_state(ctx, int(kind), float(w), ptr(rho)), "qst_test_state")


def qst_sample_counts(ctx: int, P, shots: int, seed: int, counts, f=None) -> int:
    """Seeded multinomial counts of `shots` draws from P (device FP64) into counts (device int64)."""
    return _check(load().qst_sample_counts(ctx, ptr(P), int(shots), int(seed), ptr(counts), ptr(f) if f is not None
                                           else None), "qst_sample_counts")


def qst_get_rho(ctx: int, f, rho_out, want_loss: bool = False) -> tuple[float | None, int]:
    loss = ctypes.c_double()
    st = _check(load().qst_get_rho(ctx, ptr(f), ptr(rho_out), ctypes.byref(loss) if want_loss else None),
                "qst_get_rho")
    return (loss.value if want_loss else None), st


def qst_state_bytes(ctx: int) -> int:
    return int(load().qst_state_bytes(ctx))


def qst_get_state(ctx: int) -> bytes:
    n = qst_state_bytes(ctx)
    buf = ctypes.create_string_buffer(n)
    _check(load().qst_get_state(ctx, buf, n), "qst_get_state")
    return buf.raw


def qst_set_state(ctx: int, blob: bytes) -> int:
    buf = ctypes.create_string_buffer(blob, len(blob))
    return _check(load().qst_set_state(ctx, buf, len(blob)), "qst_set_state")


def qst_iterations(ctx: int) -> int:
    return int(load().qst_iterations(ctx))


def qst_kernel_launches(ctx: int) -> int:
    return int(load().qst_kernel_launches(ctx))


def qst_sync(ctx: int) -> int:
    return _check(load().qst_sync(ctx), "qst_sync")


def qst_destroy(ctx: int) -> None:
    if ctx:
        load().qst_destroy(ctx)


def qst_timing_enable(ctx: int, max_steps: int) -> int:
    return _check(load().qst_timing_enable(ctx, int(max_steps)), "qst_timing_enable")


def qst_timing_read(ctx: int) -> dict:
    """Per-phase (total ms, count) over the steps recorded since the last read."""
    n = len(PHASES)
    ms = (ctypes.c_double * n)()
    cnt = (ctypes.c_longlong * n)()
    _check(load().qst_timing_read(ctx, ms, cnt, n), "qst_timing_read")
    return {PHASES[p]: (ms[p], int(cnt[p])) for p in range(n)}


def qst_probs_static(N: int, rho, p, povm=None, K: int = 4, stream: int = 0) -> int:
    """Allocation-free POVM map (FP32, N <= 10): see qst_probs_static in include/qst.h."""
    if povm is None:
        povm = tetrahedral_povm_flat()
    povm = np.ascontiguousarray(povm, dtype=np.float64)
    return _check(load().qst_probs_static(int(N), povm.ctypes.data, int(K), ptr(rho), ptr(p), stream or None),
                  "qst_probs_static")


def qst_graph_enable(ctx: int, enable: bool = True) -> int:
    return _check(load().qst_graph_enable(ctx, 1 if enable else 0), "qst_graph_enable")


QST_INJECT_TC_LOADS = 1
QST_INJECT_WPASS_LOADS = 2


def qst_inject_wait_timeout(what: int, count: int = 1) -> None:
    """Testing hook: the next `count` launches of a kernel kind issue no operand copies (see qst.h)."""
    _check(load().qst_inject_wait_timeout(int(what), int(count)), "qst_inject_wait_timeout")


def qst_eig_counts(ctx: int, last: bool = False):
    """(tensor-core refinements taken, steps handed to Jacobi sweeps) of a mixed A_P context; with
    last=True also the latest refinement's (largest correction, unresolved coupling)."""
    a, b = ctypes.c_longlong(), ctypes.c_longlong()
    v = (ctypes.c_double * 2)()
    _check(load().qst_eig_counts(ctx, ctypes.byref(a), ctypes.byref(b), v), "qst_eig_counts")
    return (a.value, b.value, (v[0], v[1])) if last else (a.value, b.value)


def qst_jacobi_schedule(N: int):
    """Passes of one Jacobi sweep at N qubits (host only): a list of subspace bases (tuples of 1 to 4 ints)."""
    cnt = ctypes.c_int()
    _check(load().qst_jacobi_schedule(int(N), ctypes.byref(cnt), None, None, 0), "qst_jacobi_schedule")
    dims = (ctypes.c_int * cnt.value)()
    basis = (ctypes.c_int * (4 * cnt.value))()
    _check(load().qst_jacobi_schedule(int(N), ctypes.byref(cnt), dims, basis, cnt.value), "qst_jacobi_schedule")
    return [tuple(basis[4 * p:4 * p + dims[p]]) for p in range(cnt.value)]


def qst_get_tuning() -> dict:
    t = qst_tuning()
    load().qst_get_tuning(ctypes.byref(t))
    return {k: getattr(t, k) for k, _ in qst_tuning._fields_}


def qst_set_tuning(**kw) -> None:
    """Change some of the process-wide launch parameters (the others keep their values)."""
    t = qst_tuning()
    load().qst_get_tuning(ctypes.byref(t))
    for k, v in kw.items():
        if k not in dict(qst_tuning._fields_):
            raise KeyError(k)
        setattr(t, k, int(v))
    _check(load().qst_set_tuning(ctypes.byref(t)), "qst_set_tuning")


def _ptr_array(xs):
    arr = (ctypes.c_void_p * len(xs))()
    for k, x in enumerate(xs):
        arr[k] = ptr(x)
    return arr


def qst_batch_init(Ns, povm=None, K: int = 4, opt: qst_options | None = None, stream: int = 0) -> int:
    """Create a batch of len(Ns) independent tomographies; returns the handle."""
    if povm is None:
        povm = tetrahedral_povm_flat()
    povm = np.ascontiguousarray(povm, dtype=np.float64)
    ns = (ctypes.c_int * len(Ns))(*[int(x) for x in Ns])
    h = ctypes.c_void_p()
    st = load().qst_batch_init(ctypes.byref(h), len(Ns), ns, povm.ctypes.data, int(K),
                               ctypes.byref(opt) if opt is not None else None, stream or None)
    _check(st, "qst_batch_init")
    return h.value


def qst_batch_context(batch: int, b: int) -> int:
    return load().qst_batch_context(batch, int(b))


def qst_batch_set_params(batch: int, b: int, theta) -> int:
    return _check(load().qst_batch_set_params(batch, int(b), ptr(theta)), "qst_batch_set_params")


def qst_batch_step(batch: int, fs, want_losses: bool = False):
    arr = _ptr_array(fs)
    losses = (ctypes.c_double * len(fs))() if want_losses else None
    _check(load().qst_batch_step(batch, arr, losses), "qst_batch_step")
    return list(losses) if want_losses else None


def qst_batch_reconstruct(batch: int, fs, iters: int, rhos=None, want_losses: bool = True):
    arr = _ptr_array(fs)
    rarr = _ptr_array(rhos) if rhos is not None else None
    losses = (ctypes.c_double * len(fs))() if want_losses else None
    _check(load().qst_batch_reconstruct(batch, arr, int(iters), rarr, losses), "qst_batch_reconstruct")
    return list(losses) if want_losses else None


def qst_batch_kernel_launches(batch: int) -> int:
    return int(load().qst_batch_kernel_launches(batch))


def qst_batch_sync(batch: int) -> int:
    return _check(load().qst_batch_sync(batch), "qst_batch_sync")


def qst_batch_destroy(batch: int) -> None:
    if batch:
        load().qst_batch_destroy(batch)
