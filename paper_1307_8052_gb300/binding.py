"""ctypes binding of the C ABI in include/rpa.h (argument marshalling only).

Every function keeps the C name.  Array arguments may be numpy arrays (host
memory) or torch tensors (host or CUDA memory); complex arrays are passed as
interleaved (re, im) doubles, which is the memory layout of numpy/torch
complex128.  Errors raise ``RpaError`` carrying the status and the library's
message.  There is no fallback: if the shared library is missing or fails to
load, importing the binding raises.
"""
from __future__ import annotations

import ctypes as ct
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "librpa_gb300.so")

RPA_OK, RPA_ERR_ARG, RPA_ERR_OOM, RPA_ERR_CUDA, RPA_ERR_NOT_HPD, RPA_ERR_TIMEOUT, RPA_ERR_STATE = range(7)
RPA_FP64, RPA_FP32, RPA_BF16X2, RPA_BF16X3 = range(4)
PRECISIONS = {"fp64": RPA_FP64, "fp32": RPA_FP32, "bf16x2": RPA_BF16X2, "bf16x3": RPA_BF16X3}
STATUS_NAMES = ["RPA_OK", "RPA_ERR_ARG", "RPA_ERR_OOM", "RPA_ERR_CUDA", "RPA_ERR_NOT_HPD", "RPA_ERR_TIMEOUT",
                "RPA_ERR_STATE"]

# exported entry points and their ctypes signatures (kept in step with include/rpa.h)
_P = ct.c_void_p
_I = ct.c_int32
_D = ct.c_double
SIGNATURES = {
    "rpa_create": (_I, [_P, _P]),
    "rpa_destroy": (None, [_P]),
    "rpa_last_error": (ct.c_char_p, [_P]),
    "rpa_gauss_legendre": (_I, [_I, _D, _P, _P]),
    "rpa_set_orbitals": (_I, [_P, _I, _P, _I, _I, _P, _P, _P, _P]),
    "rpa_set_paw": (_I, [_P, _I, _I, _P, _P]),
    "rpa_set_qpoint": (_I, [_P, _I, _P, _I, _P, _P, _P, _P]),
    "rpa_gvectors": (_I, [_P, _I, _P, _P]),
    "rpa_response_sphere": (_I, [_P, _P, _D, _I, _P, _P, _P]),
    "rpa_set_paw_Q": (_I, [_P, _I, _I, _P, _P]),
    "rpa_set_optical": (_I, [_P, _I, _P, _I, _P, _P]),
    "rpa_set_orbitals_sym": (_I, [_P, _I, _I, _P, _P, _I, _I, _P, _P]),
    "rpa_chi0": (_I, [_P, _I, _I, _P, _P]),
    "rpa_epsilon_inv": (_I, [_P, _I, _I, _P, _P]),
    "rpa_energy": (_I, [_P, _I, _P, _P, _I, _P, _P, _P, _P]),
    "rpa_set_profiling": (_I, [_P, _I]),
    "rpa_get_profile": (_I, [_P, _P, _P]),
    "rpa_set_tuning": (_I, [_P, _I, ct.c_int64]),
    "rpa_logdet_noalloc": (_I, [_P, _P, _I, _I, _P, _P]),
    "rpa_energy_backward": (_I, [_P, _I, _P, _P, _I, _P, _P, _D, _P, _I, _P, _P, _P, _P]),
    "rpa_set_frequencies": (_I, [_P, _I, _P]),
    "rpa_energy_enqueue": (_I, [_P, _I, _P]),
    "rpa_energy_collect": (_I, [_P, _P, _P, _P, _P]),
    "rpa_graph_create": (_I, [_P, _I, _P, _P, _P]),
    "rpa_graph_launch": (_I, [_P]),
    "rpa_graph_destroy": (None, [_P]),
}
RPA_NSTAGES = 6  # profile stages: wf, pair densities, rank-k kernel, log-det, other, operand preparation
(RPA_TUNE_TC_FOLD, RPA_TUNE_PAIR_CHUNK, RPA_TUNE_TC_FLUSH, RPA_TUNE_PD_GRID, RPA_TUNE_OPERAND_MB, RPA_TUNE_TC_PIPE,
 RPA_TUNE_LOGDET, RPA_TUNE_PAW_TC, RPA_TUNE_TC_FUSE, RPA_TUNE_TC_WAIT_US, RPA_TUNE_TC_STALL,
 RPA_TUNE_PD_FUSE, RPA_TUNE_BATCH_PERSIST, RPA_TUNE_BATCH_MB, RPA_TUNE_GAMMA,
 RPA_TUNE_TC_PAIR, RPA_TUNE_PD_FACT, RPA_TUNE_LD_OVERLAP) = range(18)
RPA_TUNE_COUNT = 18


class RpaParams(ct.Structure):
    _fields_ = [("cell", ct.c_double * 9), ("grid", ct.c_int32 * 3), ("ecut_chi", ct.c_double),
                ("spin_factor", ct.c_double), ("nk_bz", ct.c_int32), ("precision", ct.c_int32),
                ("device", ct.c_int32), ("stream", ct.c_void_p)]


class RpaError(RuntimeError):
    def __init__(self, status: int, msg: str):
        name = STATUS_NAMES[status] if 0 <= status < len(STATUS_NAMES) else str(status)
        super().__init__(f"{name}: {msg}")
        self.status = status


def load(path: str = LIB_PATH) -> ct.CDLL:
    if not os.path.exists(path):
        raise ImportError(f"{path} is missing: run paper_1307_8052_gb300.build.build() first")
    lib = ct.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


_lib = None


def lib() -> ct.CDLL:
    global _lib
    if _lib is None:
        _lib = load()
    return _lib


# ------------------------------------------------------------------ marshalling
_TORCH_DTYPE = {np.dtype(np.complex128): "torch.complex128", np.dtype(np.float64): "torch.float64",
                np.dtype(np.int32): "torch.int32"}


def _is_tensor(x):
    return hasattr(x, "data_ptr") and hasattr(x, "is_contiguous")


def _ptr(x, dtype=None, keep=None):
    """Pointer to contiguous memory of an input (numpy array, sequence or torch
    tensor).  Host arrays are converted to ``dtype`` (a copy if needed, kept
    alive in ``keep``); a tensor, which may live on the device, is passed as
    it is and must already be contiguous and of that dtype."""
    if x is None:
        return None
    if _is_tensor(x):
        if not x.is_contiguous():
            raise ValueError("tensor must be contiguous")
        if dtype is not None and str(x.dtype) != _TORCH_DTYPE[np.dtype(dtype)]:
            raise TypeError(f"tensor of {x.dtype} where {_TORCH_DTYPE[np.dtype(dtype)]} is required")
        return ct.c_void_p(x.data_ptr())
    a = np.ascontiguousarray(x, dtype=dtype)
    if keep is not None:
        keep.append(a)
    return ct.c_void_p(a.ctypes.data)


def _host(x, dtype, shape, what):
    """A host array argument as a contiguous array of ``dtype``, checked
    against the shape that the other arguments imply: the library reads
    exactly that many elements."""
    a = np.ascontiguousarray(x, dtype=dtype)
    if a.shape != tuple(shape):
        raise ValueError(f"{what} has shape {a.shape}, expected {tuple(shape)}")
    return a


def _out_ptr(x, dtype, count=None):
    """Pointer to an output buffer that the library fills in place: a writable,
    contiguous numpy array or tensor of exactly ``dtype`` (and ``count``
    elements when the binding knows the size).  Never a converted copy, whose
    contents the caller would not see, nor a narrower type the library would
    write past."""
    dt = np.dtype(dtype)
    if _is_tensor(x):
        ok = x.is_contiguous() and str(x.dtype) == _TORCH_DTYPE[dt] and (count is None or x.numel() == count)
        ptr = x.data_ptr() if ok else 0
    else:
        ok = (isinstance(x, np.ndarray) and x.flags.c_contiguous and x.flags.writeable and x.dtype == dt
              and (count is None or x.size == count))
        ptr = x.ctypes.data if ok else 0
    if not ok:
        size = "" if count is None else f" of {count} elements"
        raise ValueError(f"output buffer must be a writable contiguous {dt} array or tensor{size}")
    return ct.c_void_p(ptr)


def _check(ctx, st):
    if st != RPA_OK:
        msg = lib().rpa_last_error(ctx).decode() if ctx else ""
        raise RpaError(st, msg)


# ------------------------------------------------------------------ API (same names as the C ABI)
def rpa_create(cell, grid, ecut_chi, spin_factor=2.0, nk_bz=1, precision="fp64", device=0, stream=0):
    p = RpaParams()
    p.cell[:] = [float(v) for v in np.asarray(cell, dtype=np.float64).reshape(9)]
    p.grid[:] = [int(v) for v in grid]
    p.ecut_chi = float(ecut_chi)
    p.spin_factor = float(spin_factor)
    p.nk_bz = int(nk_bz)
    p.precision = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
    p.device = int(device)
    p.stream = ct.c_void_p(int(stream)) if stream else None
    out = ct.c_void_p()
    st = lib().rpa_create(ct.byref(p), ct.byref(out))
    _check(None, st)
    return out


def rpa_destroy(ctx):
    lib().rpa_destroy(ctx)


def rpa_last_error(ctx) -> str:
    return lib().rpa_last_error(ctx).decode()


def rpa_gauss_legendre(n, omega0=1.0):
    om = np.zeros(n)
    W = np.zeros(n)
    _check(None, lib().rpa_gauss_legendre(int(n), float(omega0), om.ctypes.data_as(_P), W.ctypes.data_as(_P)))
    return om, W


def rpa_set_orbitals(ctx, kidx, k_red, miller, C, eps, f):
    keep = []
    nb, npw = int(C.shape[0]), int(C.shape[1])
    k_red = _host(k_red, np.float64, (3,), "k_red")
    miller = _host(miller, np.int32, (npw, 3), "miller")
    eps = _host(eps, np.float64, (nb,), "eps")
    f = _host(f, np.float64, (nb,), "f")
    st = lib().rpa_set_orbitals(ctx, int(kidx), _ptr(k_red, np.float64, keep), nb, npw,
                                _ptr(miller, np.int32, keep), _ptr(C, np.complex128, keep),
                                _ptr(eps, np.float64, keep), _ptr(f, np.float64, keep))
    _check(ctx, st)


def rpa_set_paw(ctx, kidx, nproj, P):
    keep = []
    nproj = np.asarray(nproj, dtype=np.int32)
    _check(ctx, lib().rpa_set_paw(ctx, int(kidx), len(nproj), _ptr(nproj, np.int32, keep),
                                  _ptr(P, np.complex128, keep)))


def rpa_set_qpoint(ctx, iq, q_red, k_of, kq_of, G0) -> int:
    keep = []
    ng = ct.c_int32()
    k_of = np.ascontiguousarray(k_of, dtype=np.int32).reshape(-1)
    nk = len(k_of)
    q_red = _host(q_red, np.float64, (3,), "q_red")
    kq_of = _host(kq_of, np.int32, (nk,), "kq_of")
    G0 = _host(np.asarray(G0).reshape(-1, 3), np.int32, (nk, 3), "G0")
    st = lib().rpa_set_qpoint(ctx, int(iq), _ptr(q_red, np.float64, keep), nk, _ptr(k_of, np.int32, keep),
                              _ptr(kq_of, np.int32, keep), _ptr(G0, np.int32, keep), ct.byref(ng))
    _check(ctx, st)
    return ng.value


def rpa_gvectors(ctx, iq) -> np.ndarray:
    ng = ct.c_int32()
    _check(ctx, lib().rpa_gvectors(ctx, int(iq), ct.byref(ng), None))
    out = np.zeros((ng.value, 3), dtype=np.int32)
    _check(ctx, lib().rpa_gvectors(ctx, int(iq), ct.byref(ng), out.ctypes.data_as(_P)))
    return out


def rpa_response_sphere(cell, q_red, ecut_chi):
    """Miller indices (NG, 3) int32 and Coulomb kernel (NG,) of the response
    sphere, computed by the library on the host (no context, no GPU)."""
    keep = []
    pc = _ptr(np.asarray(cell, dtype=np.float64).reshape(9), np.float64, keep)
    pq = _ptr(np.asarray(q_red, dtype=np.float64).reshape(3), np.float64, keep)
    ng = ct.c_int32()
    _check(None, lib().rpa_response_sphere(pc, pq, float(ecut_chi), 0, ct.byref(ng), None, None))
    gm = np.zeros((ng.value, 3), dtype=np.int32)
    v = np.zeros(ng.value)
    _check(None, lib().rpa_response_sphere(pc, pq, float(ecut_chi), ng.value, ct.byref(ng),
                                           gm.ctypes.data_as(_P), v.ctypes.data_as(_P)))
    return gm, v


def rpa_set_paw_Q(ctx, iq, nproj, Q):
    keep = []
    nproj = np.asarray(nproj, dtype=np.int32)
    _check(ctx, lib().rpa_set_paw_Q(ctx, int(iq), len(nproj), _ptr(nproj, np.int32, keep),
                                    _ptr(Q, np.complex128, keep)))


def rpa_set_orbitals_sym(ctx, kidx, src, M, time_reversal=False, atom_map=None, D=None, tau=None):
    """Set kidx = set src under the operation {M|tau} (M: 3x3 integers on reduced
    reciprocal coordinates, tau: reduced fractional translation or None),
    optionally time-reversed; ``D[a]`` (ni, ni) complex rotates the projections
    of atom ``atom_map[a]`` onto atom a."""
    keep = []
    Mi = np.ascontiguousarray(np.asarray(M, dtype=np.int32).reshape(9))
    tp = None if tau is None else _ptr(np.ascontiguousarray(tau, dtype=np.float64), np.float64, keep)
    if D is None:
        _check(ctx, lib().rpa_set_orbitals_sym(ctx, int(kidx), int(src), _ptr(Mi, np.int32, keep), tp,
                                               int(bool(time_reversal)), 0, None, None))
        return
    am = np.ascontiguousarray(atom_map, dtype=np.int32)
    flat = np.ascontiguousarray(np.concatenate([np.asarray(d, dtype=np.complex128).reshape(-1) for d in D]))
    _check(ctx, lib().rpa_set_orbitals_sym(ctx, int(kidx), int(src), _ptr(Mi, np.int32, keep), tp,
                                           int(bool(time_reversal)), len(am), _ptr(am, np.int32, keep),
                                           _ptr(flat, np.complex128, keep)))


def rpa_set_optical(ctx, iq, qdir, nproj=None, Qgrad=None):
    """Optical limit at q = 0 point iq along ``qdir`` (Cartesian); ``Qgrad[a]``
    complex (3, ni, ni) per atom, or None without PAW; ``qdir=None`` switches it off."""
    keep = []
    if qdir is None:
        _check(ctx, lib().rpa_set_optical(ctx, int(iq), None, 0, None, None))
        return
    qd = np.ascontiguousarray(qdir, dtype=np.float64)
    if Qgrad is None or nproj is None or len(nproj) == 0:
        _check(ctx, lib().rpa_set_optical(ctx, int(iq), _ptr(qd, np.float64, keep), 0, None, None))
        return
    nproj = np.asarray(nproj, dtype=np.int32)
    flat = np.ascontiguousarray(np.concatenate([np.asarray(q, dtype=np.complex128).reshape(-1) for q in Qgrad]))
    _check(ctx, lib().rpa_set_optical(ctx, int(iq), _ptr(qd, np.float64, keep), len(nproj),
                                      _ptr(nproj, np.int32, keep), _ptr(flat, np.complex128, keep)))


def rpa_chi0(ctx, iq, omega, out=None):
    """chi0[nw][NG][NG] complex128; ``out`` may be a preallocated numpy array or CUDA tensor."""
    keep = []
    omega = np.ascontiguousarray(omega, dtype=np.float64)
    ng = ct.c_int32()
    _check(ctx, lib().rpa_gvectors(ctx, int(iq), ct.byref(ng), None))
    if out is None:
        out = np.zeros((len(omega), ng.value, ng.value), dtype=np.complex128)
    dst = _out_ptr(out, np.complex128, len(omega) * ng.value * ng.value)
    _check(ctx, lib().rpa_chi0(ctx, int(iq), len(omega), _ptr(omega, np.float64, keep), dst))
    return out


def rpa_epsilon_inv(ctx, iq, omega, out=None):
    """(1 - v^1/2 chi0 v^1/2)^-1 [nw][NG][NG] complex128; ``out`` may be a preallocated numpy array or CUDA tensor."""
    keep = []
    omega = np.ascontiguousarray(omega, dtype=np.float64)
    ng = ct.c_int32()
    _check(ctx, lib().rpa_gvectors(ctx, int(iq), ct.byref(ng), None))
    if out is None:
        out = np.zeros((len(omega), ng.value, ng.value), dtype=np.complex128)
    dst = _out_ptr(out, np.complex128, len(omega) * ng.value * ng.value)
    _check(ctx, lib().rpa_epsilon_inv(ctx, int(iq), len(omega), _ptr(omega, np.float64, keep), dst))
    return out


def rpa_energy(ctx, iqs, wq, omega, W):
    """Returns (E_c, terms[nq][nw])."""
    keep = []
    iqs = np.ascontiguousarray(iqs, dtype=np.int32)
    omega = np.ascontiguousarray(omega, dtype=np.float64)
    wq = _host(wq, np.float64, (len(iqs),), "wq")
    W = _host(W, np.float64, (len(omega),), "W")
    terms = np.zeros((len(iqs), len(omega)))
    E = ct.c_double()
    st = lib().rpa_energy(ctx, len(iqs), _ptr(iqs, np.int32, keep), _ptr(wq, np.float64, keep), len(omega),
                          _ptr(omega, np.float64, keep), _ptr(W, np.float64, keep), ct.byref(E),
                          terms.ctypes.data_as(_P))
    _check(ctx, st)
    return E.value, terms


def rpa_energy_backward(ctx, iqs, wq, omega, W, dEc=1.0, sets=(), dC=None, dP=None, dchi=None):
    """Gradient of E_c.  ``sets`` lists orbital-set indices; ``dC[s]`` / ``dP[s]``
    are output buffers (numpy arrays or CUDA tensors, complex128, shaped like the
    set's C / P; entries may be None) and ``dchi[i]`` ([nw][NG][NG] complex128)
    per q-point.  Returns E_c."""
    keep = []
    iqs = np.ascontiguousarray(iqs, dtype=np.int32)
    omega = np.ascontiguousarray(omega, dtype=np.float64)
    sets = np.ascontiguousarray(sets, dtype=np.int32)
    wq = _host(wq, np.float64, (len(iqs),), "wq")
    W = _host(W, np.float64, (len(omega),), "W")

    def ptr_array(bufs, n, counts=None):
        if bufs is None:
            return None
        if len(bufs) > n:
            raise ValueError(f"{len(bufs)} output buffers for {n} entries")
        ptrs = [_out_ptr(x, np.complex128, None if counts is None else counts[i]).value if x is not None else None
                for i, x in enumerate(bufs)]
        arr = (ct.c_void_p * n)(*ptrs)
        keep.append(arr)
        return ct.cast(arr, ct.c_void_p)

    chi_counts = None
    if dchi is not None:
        chi_counts = []
        for iq in iqs:
            ng = ct.c_int32()
            _check(ctx, lib().rpa_gvectors(ctx, int(iq), ct.byref(ng), None))
            chi_counts.append(len(omega) * ng.value * ng.value)

    E = ct.c_double()
    st = lib().rpa_energy_backward(ctx, len(iqs), _ptr(iqs, np.int32, keep), _ptr(wq, np.float64, keep), len(omega),
                                   _ptr(omega, np.float64, keep), _ptr(W, np.float64, keep), float(dEc),
                                   ct.byref(E), len(sets), _ptr(sets, np.int32, keep) if len(sets) else None,
                                   ptr_array(dC, len(sets)), ptr_array(dP, len(sets)),
                                   ptr_array(dchi, len(iqs), chi_counts))
    _check(ctx, st)
    return E.value


def rpa_set_frequencies(ctx, omega):
    keep = []
    omega = np.ascontiguousarray(omega, dtype=np.float64)
    _check(ctx, lib().rpa_set_frequencies(ctx, len(omega), _ptr(omega, np.float64, keep)))


def rpa_energy_enqueue(ctx, iqs):
    keep = []
    iqs = np.ascontiguousarray(iqs, dtype=np.int32)
    _check(ctx, lib().rpa_energy_enqueue(ctx, len(iqs), _ptr(iqs, np.int32, keep)))


def rpa_energy_collect(ctx, wq, W, nq):
    keep = []
    W = np.ascontiguousarray(W, dtype=np.float64)
    wq = _host(wq, np.float64, (nq,), "wq")
    terms = np.zeros((nq, len(W)))
    E = ct.c_double()
    _check(ctx, lib().rpa_energy_collect(ctx, _ptr(wq, np.float64, keep), _ptr(W, np.float64, keep), ct.byref(E),
                                         terms.ctypes.data_as(_P)))
    return E.value, terms


def rpa_graph_create(ctxs, iq_lists):
    arr = (ct.c_void_p * len(ctxs))(*[c.value for c in ctxs])
    nq = np.array([len(x) for x in iq_lists], dtype=np.int32)
    flat = np.ascontiguousarray(np.concatenate([np.asarray(x, dtype=np.int32) for x in iq_lists]))
    out = ct.c_void_p()
    st = lib().rpa_graph_create(ct.cast(arr, ct.c_void_p), len(ctxs), nq.ctypes.data_as(_P), flat.ctypes.data_as(_P),
                                ct.byref(out))
    if st != RPA_OK:
        raise RpaError(st, lib().rpa_last_error(ctxs[0]).decode())
    return out


def rpa_graph_launch(g):
    _check(None, lib().rpa_graph_launch(g))


def rpa_graph_destroy(g):
    lib().rpa_graph_destroy(g)


def rpa_set_profiling(ctx, enable=True):
    _check(ctx, lib().rpa_set_profiling(ctx, 1 if enable else 0))


def rpa_set_tuning(ctx, param, value):
    _check(ctx, lib().rpa_set_tuning(ctx, int(param), int(value)))


def rpa_logdet_noalloc(chi, v, terms, stream=0):
    """Allocation-free log-det terms from device tensors chi [nw][ng][ng] (complex128),
    v [ng] and terms [nw] (float64); see include/rpa.h."""
    nw, ng = int(chi.shape[0]), int(chi.shape[1])
    _check(None, lib().rpa_logdet_noalloc(_ptr(chi, np.complex128), _ptr(v, np.float64), nw, ng,
                                          _out_ptr(terms, np.float64, nw),
                                          ct.c_void_p(int(stream)) if stream else None))


def rpa_get_profile(ctx):
    ms = np.zeros(RPA_NSTAGES)
    nl = np.zeros(RPA_NSTAGES, dtype=np.int64)
    _check(ctx, lib().rpa_get_profile(ctx, ms.ctypes.data_as(_P), nl.ctypes.data_as(_P)))
    return ms, nl


# ------------------------------------------------------------------ convenience
def load_problem(ctx, problem, qs=None, paw_Q=None):
    """Upload every orbital set, projection set and q-point of a Problem-like object.
    ``paw_Q(iq, gmiller) -> flat Q`` supplies augmentation functions per q."""
    for i, s in enumerate(problem.sets):
        rpa_set_orbitals(ctx, i, s.k_red, s.miller, s.C, s.eps, s.f)
        if s.P is not None and problem.paw is not None:
            rpa_set_paw(ctx, i, problem.paw.nproj, s.P)
    ngs = []
    for iq, qp in enumerate(problem.qpoints):
        if qs is not None and iq not in qs:
            continue
        ngs.append(rpa_set_qpoint(ctx, iq, qp.q_red, qp.k_of, qp.kq_of, qp.G0))
        if paw_Q is not None and problem.paw is not None:
            rpa_set_paw_Q(ctx, iq, problem.paw.nproj, paw_Q(iq, rpa_gvectors(ctx, iq)))
    return ngs
