"""Python binding of libz2lgt, the GB300 (sm_103a) state-vector library for
the digital adiabatic simulation of quantum Z2 lattice gauge theory
(Cui, Shi, Yang, arXiv:1910.08020).

Argument marshalling only: every step of the simulation runs in the CUDA
library behind the C ABI of include/z2lgt.h.  Functions keep the C names
(``z2_run``, ``z2_evolve``, ...).  States are CUDA tensors (complex64 or
complex128, 256-byte aligned, owned by the caller); streams are
``torch.cuda.Stream`` objects or raw ``cudaStream_t`` integers (default: the
current PyTorch stream).  There is no CPU fallback: if the library is not
built, loading fails with an error.
"""

from __future__ import annotations

import ctypes
import os

import numpy as np

__all__ = [
    "Z2Error", "RunParams", "Results", "LatticeInfo", "load", "build",
    "z2_ctx_create", "z2_ctx_destroy", "z2_last_error", "z2_version", "z2_ctx_launch_count",
    "z2_ctx_flush_plans", "z2_evolve_plan_info", "PlanInfo", "z2_plan_geometry", "GroupInfo", "z2_ctx_set_option", "z2_autotune", "TuneResult",
    "z2_lattice_create", "z2_lattice_destroy", "z2_lattice_info_get", "z2_lattice_masks", "z2_state_bytes",
    "z2_init_plus", "z2_apply_plaquettes", "z2_apply_rx_layer", "z2_apply_hadamard",
    "z2_evolve", "z2_measure", "z2_run", "GrampParams", "gramp_params", "z2_init_projected", "z2_evolve_gramp",
    "z2_measure_gramp", "z2_run_gramp", "z2_apply_gate", "z2_evolve_gramp_circuit", "QpeParams", "qpe_params",
    "z2_controlled_evolution", "z2_zsums", "z2_overlap", "z2_zsums_static", "z2_dos", "Z2_DOS_Z", "Z2_DOS_X",
    "trajectory", "finite_differences",
    "Context", "Lattice", "results_dict", "z2_sweep", "RunSpec", "run_specs", "ServeStats",
    "z2_server_create", "z2_server_submit", "z2_server_poll", "z2_server_wait", "z2_server_cancel",
    "z2_server_stats", "z2_server_request_times", "z2_server_request_device_times", "z2_server_set_option", "Z2_SERVE_OPT_LARGE_QUBITS",
    "Z2_SERVE_OPT_MAX_LARGE", "z2_server_destroy",
]

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libz2lgt.so")

Z2_OK = 0
Z2_FIRST_ORDER, Z2_SYMMETRIC = 0, 1
Z2_C64, Z2_C128 = 0, 1
Z2_SAMPLE_STD, Z2_SAMPLE_PAPER = 0, 1
Z2_MASK_PLAQ, Z2_MASK_STAR, Z2_MASK_WILSON_2X2, Z2_MASK_CONTOUR, Z2_MASK_W_MU, Z2_MASK_V_MU = range(6)
Z2_FLAG_WILSON_DEGENERATE, Z2_FLAG_CONTOUR_DEGENERATE, Z2_FLAG_NO_FIDELITY = 1, 2, 4
Z2_MAX_LINKS, Z2_MAX_PLAQ, Z2_MAX_SITES = 34, 32, 32
ERRORS = {-1: "Z2_ERR_ARG", -2: "Z2_ERR_LATTICE", -3: "Z2_ERR_OOM", -4: "Z2_ERR_BUDGET", -5: "Z2_ERR_CUDA",
          -6: "Z2_ERR_DEVICE_TIMEOUT", -7: "Z2_ERR_CANCELLED", -8: "Z2_ERR_NOT_FOUND"}


class Z2Error(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{ERRORS.get(code, code)}: {msg}")
        self.code = code


class RunParams(ctypes.Structure):
    _fields_ = [("lambda_", ctypes.c_double), ("T", ctypes.c_double), ("M", ctypes.c_int32),
                ("decomp", ctypes.c_int32), ("precision", ctypes.c_int32), ("sampling", ctypes.c_int32)]


class GrampParams(ctypes.Structure):
    _fields_ = [("g_s", ctypes.c_double), ("t_s", ctypes.c_double), ("N_s", ctypes.c_int32), ("n", ctypes.c_int32),
                ("decomp", ctypes.c_int32), ("precision", ctypes.c_int32)]


class QpeParams(ctypes.Structure):
    _fields_ = [("g", ctypes.c_double), ("t", ctypes.c_double), ("n", ctypes.c_int32), ("decomp", ctypes.c_int32),
                ("precision", ctypes.c_int32), ("reserved", ctypes.c_int32)]


Z2_GATE_CNOT, Z2_GATE_RZ, Z2_GATE_RX, Z2_GATE_H = 0, 1, 2, 3


class LatticeInfo(ctypes.Structure):
    _fields_ = [("d", ctypes.c_int32), ("L", ctypes.c_int32 * 3), ("n_links", ctypes.c_int32),
                ("n_plaq", ctypes.c_int32), ("n_sites", ctypes.c_int32)]


class PlanInfo(ctypes.Structure):
    _fields_ = [("tile_bits", ctypes.c_int32), ("n_groups", ctypes.c_int32), ("n_passes", ctypes.c_int32),
                ("n_launches", ctypes.c_int32), ("n_tables", ctypes.c_int32), ("flip", ctypes.c_int32),
                ("low_tile_bits", ctypes.c_int32)]


class GroupInfo(ctypes.Structure):
    _fields_ = [("tile_bits", ctypes.c_int32), ("c", ctypes.c_int32), ("b", ctypes.c_int32), ("k", ctypes.c_int32),
                ("k1", ctypes.c_int32), ("b2", ctypes.c_int32)]


class TuneResult(ctypes.Structure):
    _fields_ = [("tile_bits", ctypes.c_int32), ("variant", ctypes.c_int32), ("us_per_step", ctypes.c_double),
                ("n_candidates", ctypes.c_int32)]


class Results(ctypes.Structure):
    _fields_ = [("s", ctypes.c_double), ("energy", ctypes.c_double), ("norm", ctypes.c_double),
                ("mean_plaq", ctypes.c_double), ("wilson_2x2", ctypes.c_double), ("mean_star", ctypes.c_double),
                ("fidelity", ctypes.c_double), ("plaq", ctypes.c_double * Z2_MAX_PLAQ),
                ("star", ctypes.c_double * Z2_MAX_SITES), ("sigmaz", ctypes.c_double * Z2_MAX_LINKS),
                ("sigmax", ctypes.c_double * Z2_MAX_LINKS), ("wmu", ctypes.c_double * 3),
                ("vmu", ctypes.c_double * 3), ("contours", ctypes.c_double * 3), ("flags", ctypes.c_uint32),
                ("status", ctypes.c_int32)]


class RunSpec(ctypes.Structure):
    _fields_ = [("d", ctypes.c_int32), ("L", ctypes.c_int32 * 3), ("params", RunParams)]


Z2_SWEEP_PLAIN, Z2_SWEEP_STREAMS, Z2_SWEEP_GRAPHS, Z2_SWEEP_PERSISTENT = 0, 1, 2, 3


class ServeStats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_uint64), ("completed", ctypes.c_uint64), ("rejected", ctypes.c_uint64),
                ("cancelled", ctypes.c_uint64), ("active", ctypes.c_int32), ("queued", ctypes.c_int32),
                ("hbm_in_use", ctypes.c_size_t), ("hbm_peak", ctypes.c_size_t)]

_lib = None
_P = ctypes.c_void_p
_I = ctypes.c_int32
_D = ctypes.c_double

_SIGS = {
    "z2_ctx_create": [ctypes.c_int, ctypes.POINTER(_P)],
    "z2_ctx_destroy": [_P],
    "z2_ctx_launch_count": [_P, ctypes.POINTER(ctypes.c_uint64)],
    "z2_ctx_flush_plans": [_P],
    "z2_ctx_set_option": [_P, _I, _I],
    "z2_autotune": [_P, _P, _I, _P, _P, ctypes.POINTER(TuneResult)],
    "z2_evolve_plan_info": [_P, _P, ctypes.POINTER(RunParams), _I, _I, ctypes.POINTER(PlanInfo)],
    "z2_dos": [_P, _P, _I, _P, _I, ctypes.POINTER(ctypes.c_double), _I, ctypes.POINTER(ctypes.c_int32), _P],
    "z2_plan_geometry": [_I, _I, _I, _I, _I, ctypes.POINTER(GroupInfo), _I, ctypes.POINTER(ctypes.c_int32)],
    "z2_last_error": [_P],
    "z2_version": [],
    "z2_lattice_create": [_I, ctypes.POINTER(_I), ctypes.POINTER(_P)],
    "z2_lattice_destroy": [_P],
    "z2_lattice_info_get": [_P, ctypes.POINTER(LatticeInfo)],
    "z2_lattice_masks": [_P, _I, ctypes.POINTER(ctypes.c_uint64), ctypes.c_size_t, ctypes.POINTER(ctypes.c_size_t)],
    "z2_state_bytes": [_P, _I, ctypes.POINTER(ctypes.c_size_t)],
    "z2_init_plus": [_P, _P, _I, _P, _P],
    "z2_apply_plaquettes": [_P, _P, _I, _P, _D, _P],
    "z2_apply_rx_layer": [_P, _P, _I, _P, _D, _P],
    "z2_apply_hadamard": [_P, _P, _I, _P, _P],
    "z2_evolve": [_P, _P, ctypes.POINTER(RunParams), _P, _I, _I, _P],
    "z2_measure": [_P, _P, ctypes.POINTER(RunParams), _P, _D, _P, _P, ctypes.POINTER(Results)],
    "z2_run": [_P, _P, ctypes.POINTER(RunParams), _P, _P, _P, ctypes.POINTER(Results)],
    "z2_init_projected": [_P, _P, _I, ctypes.c_uint32, _P, _P],
    "z2_evolve_gramp": [_P, _P, ctypes.POINTER(GrampParams), _P, _I, _I, _P],
    "z2_measure_gramp": [_P, _P, _I, _D, _P, _P, _P, ctypes.POINTER(Results)],
    "z2_run_gramp": [_P, _P, ctypes.POINTER(GrampParams), ctypes.c_uint32, _P, _P, _P, ctypes.POINTER(Results)],
    "z2_apply_gate": [_P, _I, _I, _P, _I, _I, _I, _D, _P],
    "z2_evolve_gramp_circuit": [_P, _P, ctypes.POINTER(GrampParams), _P, _I, _I, _P, ctypes.POINTER(ctypes.c_uint64)],
    "z2_controlled_evolution": [_P, _P, ctypes.POINTER(QpeParams), _P, _P],
    "z2_zsums": [_P, _I, _I, _P, ctypes.POINTER(ctypes.c_uint64), _I, ctypes.POINTER(_D), _P],
    "z2_overlap": [_P, _I, _I, _P, _P, ctypes.POINTER(_D), _P],
    "z2_sweep": [_P, ctypes.POINTER(RunSpec), _I, _I, _I, ctypes.POINTER(Results)],
    "z2_zsums_static": [_I, _I, _P, ctypes.POINTER(ctypes.c_uint64), _I, ctypes.POINTER(_D), _P],
    "z2_server_create": [_P, ctypes.c_size_t, _I, ctypes.POINTER(_P)],
    "z2_server_submit": [_P, ctypes.POINTER(RunSpec), ctypes.POINTER(ctypes.c_uint64)],
    "z2_server_poll": [_P, ctypes.c_uint64, ctypes.POINTER(_I), ctypes.POINTER(Results)],
    "z2_server_wait": [_P, ctypes.c_uint64, _D, ctypes.POINTER(Results)],
    "z2_server_cancel": [_P, ctypes.c_uint64],
    "z2_server_stats": [_P, ctypes.POINTER(ServeStats)],
    "z2_server_request_times": [_P, ctypes.c_uint64, ctypes.POINTER(_D), ctypes.POINTER(_D)],
    "z2_server_request_device_times": [_P, ctypes.c_uint64, ctypes.POINTER(_D), ctypes.POINTER(_D)],
    "z2_server_set_option": [_P, _I, _I],
    "z2_server_destroy": [_P],
}


def build(force=False, verbose=False):
    """Compile libz2lgt.so in-tree (nvcc for sm_103a)."""
    from . import buildlib as _b
    return _b.build(force=force, verbose=verbose)


def load():
    """Load libz2lgt.so; raises if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"libz2lgt.so is not built ({LIB_PATH}); run paper_1910_08020_gb300.build() "
                          "(there is no CPU fallback)")
    L = ctypes.CDLL(LIB_PATH)
    for name, argtypes in _SIGS.items():
        f = getattr(L, name)
        f.argtypes = argtypes
        f.restype = ctypes.c_char_p if name in ("z2_last_error", "z2_version") else ctypes.c_int
    _lib = L
    return L


def _ptr(x):
    """Device pointer of a tensor, or an int / None passed through."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    return x.data_ptr()


def _stream(s):
    if s is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(s, int):
        return s
    return s.cuda_stream


def _check(rc, ctx=None):
    if rc != Z2_OK:
        raise Z2Error(rc, load().z2_last_error(ctx).decode())


# -- raw C-ABI mirrors (same names, argument marshalling only) ---------------------
def z2_version():
    return load().z2_version().decode()


def z2_last_error(ctx=None):
    return load().z2_last_error(ctx).decode()


def z2_ctx_create(device=0):
    out = _P()
    _check(load().z2_ctx_create(device, ctypes.byref(out)))
    return out.value


def z2_ctx_destroy(ctx):
    _check(load().z2_ctx_destroy(ctx))


def z2_ctx_launch_count(ctx):
    out = ctypes.c_uint64()
    _check(load().z2_ctx_launch_count(ctx, ctypes.byref(out)), ctx)
    return out.value


Z2_OPT_TILE_BITS, Z2_OPT_PASS_VARIANT, Z2_OPT_SPLIT_LOW_BITS, Z2_OPT_GANG_WAIT_POLLS = 0, 1, 2, 3
Z2_DOS_Z, Z2_DOS_X = 0, 1


def z2_ctx_set_option(ctx, option, value):
    _check(load().z2_ctx_set_option(ctx, int(option), int(value)), ctx)


def z2_autotune(ctx, lat, precision, state, stream=None):
    res = TuneResult()
    _check(load().z2_autotune(ctx, lat, int(precision), _ptr(state), _stream(stream), ctypes.byref(res)), ctx)
    return res


def z2_ctx_flush_plans(ctx):
    _check(load().z2_ctx_flush_plans(ctx), ctx)


def z2_evolve_plan_info(ctx, lat, params, j0, j1):
    info = PlanInfo()
    _check(load().z2_evolve_plan_info(ctx, lat, ctypes.byref(params), int(j0), int(j1), ctypes.byref(info)), ctx)
    return info


def z2_plan_geometry(n_qubits, precision=0, tile_bits=0, variant=0, assume_tma=True):
    """Qubit groups of a plan (host only, no GPU): list of GroupInfo, low group first."""
    out = (GroupInfo * 8)()
    n = ctypes.c_int32(0)
    _check(load().z2_plan_geometry(int(n_qubits), int(precision), int(tile_bits), int(variant), int(bool(assume_tma)),
                                   out, 8, ctypes.byref(n)))
    return [out[i] for i in range(n.value)]


def z2_lattice_create(d, L):
    arr = (_I * 3)(*(list(L) + [1] * (3 - len(L))))
    out = _P()
    _check(load().z2_lattice_create(d, arr, ctypes.byref(out)))
    return out.value


def z2_lattice_destroy(lat):
    _check(load().z2_lattice_destroy(lat))


def z2_lattice_info_get(lat):
    info = LatticeInfo()
    _check(load().z2_lattice_info_get(lat, ctypes.byref(info)))
    return info


def z2_lattice_masks(lat, kind):
    n = ctypes.c_size_t()
    buf = (ctypes.c_uint64 * 64)()
    _check(load().z2_lattice_masks(lat, kind, buf, 64, ctypes.byref(n)))
    return np.array(buf[:n.value], dtype=np.uint64)


def z2_state_bytes(lat, precision):
    n = ctypes.c_size_t()
    _check(load().z2_state_bytes(lat, precision, ctypes.byref(n)))
    return n.value


def z2_init_plus(ctx, lat, precision, state, stream=None):
    _check(load().z2_init_plus(ctx, lat, precision, _ptr(state), _stream(stream)), ctx)


def z2_apply_plaquettes(ctx, lat, precision, state, theta, stream=None):
    _check(load().z2_apply_plaquettes(ctx, lat, precision, _ptr(state), float(theta), _stream(stream)), ctx)


def z2_apply_rx_layer(ctx, lat, precision, state, dt, stream=None):
    _check(load().z2_apply_rx_layer(ctx, lat, precision, _ptr(state), float(dt), _stream(stream)), ctx)


def z2_apply_hadamard(ctx, lat, precision, state, stream=None):
    _check(load().z2_apply_hadamard(ctx, lat, precision, _ptr(state), _stream(stream)), ctx)


def z2_evolve(ctx, lat, params, state, j0, j1, stream=None):
    _check(load().z2_evolve(ctx, lat, ctypes.byref(params), _ptr(state), int(j0), int(j1), _stream(stream)), ctx)


def z2_measure(ctx, lat, params, state, s=1.0, ref=None, stream=None):
    res = Results()
    _check(load().z2_measure(ctx, lat, ctypes.byref(params), _ptr(state), float(s), _ptr(ref), _stream(stream),
                             ctypes.byref(res)), ctx)
    return res


def z2_run(ctx, lat, params, state, ref=None, stream=None):
    res = Results()
    _check(load().z2_run(ctx, lat, ctypes.byref(params), _ptr(state), _ptr(ref), _stream(stream),
                         ctypes.byref(res)), ctx)
    return res


def z2_init_projected(ctx, lat, precision, state, sectors=0, stream=None):
    _check(load().z2_init_projected(ctx, lat, int(precision), int(sectors), _ptr(state), _stream(stream)), ctx)


def z2_evolve_gramp(ctx, lat, gp, state, k0, k1, stream=None):
    _check(load().z2_evolve_gramp(ctx, lat, ctypes.byref(gp), _ptr(state), int(k0), int(k1), _stream(stream)), ctx)


def z2_measure_gramp(ctx, lat, precision, g, state, ref=None, stream=None):
    res = Results()
    _check(load().z2_measure_gramp(ctx, lat, int(precision), float(g), _ptr(state), _ptr(ref), _stream(stream),
                                   ctypes.byref(res)), ctx)
    return res


def z2_run_gramp(ctx, lat, gp, state, sectors=0, ref=None, stream=None):
    res = Results()
    _check(load().z2_run_gramp(ctx, lat, ctypes.byref(gp), int(sectors), _ptr(state), _ptr(ref), _stream(stream),
                               ctypes.byref(res)), ctx)
    return res


def z2_apply_gate(ctx, n_qubits, precision, state, kind, q0, q1=-1, angle=0.0, stream=None):
    _check(load().z2_apply_gate(ctx, int(n_qubits), int(precision), _ptr(state), int(kind), int(q0), int(q1),
                                float(angle), _stream(stream)), ctx)


def z2_evolve_gramp_circuit(ctx, lat, gp, state, k0, k1, stream=None):
    """Gate-by-gate ramp on N + 1 qubits (ancilla = top bit); returns the gate count."""
    n = ctypes.c_uint64(0)
    _check(load().z2_evolve_gramp_circuit(ctx, lat, ctypes.byref(gp), _ptr(state), int(k0), int(k1),
                                          _stream(stream), ctypes.byref(n)), ctx)
    return n.value


def z2_controlled_evolution(ctx, lat, qp, state, stream=None):
    _check(load().z2_controlled_evolution(ctx, lat, ctypes.byref(qp), _ptr(state), _stream(stream)), ctx)


def z2_zsums(ctx, n_qubits, precision, state, masks, stream=None):
    m = np.ascontiguousarray(masks, dtype=np.uint64)
    out = np.zeros(len(m), dtype=np.float64)
    _check(load().z2_zsums(ctx, n_qubits, precision, _ptr(state), m.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)),
                           len(m), out.ctypes.data_as(ctypes.POINTER(_D)), _stream(stream)), ctx)
    return out


def z2_zsums_static(n_qubits, precision, state, masks, stream=None):
    """Allocation-free z2_zsums (no context; fixed device scratch inside the library)."""
    m = np.ascontiguousarray(masks, dtype=np.uint64)
    out = np.zeros(len(m), dtype=np.float64)
    _check(load().z2_zsums_static(n_qubits, precision, _ptr(state), m.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)),
                                  len(m), out.ctypes.data_as(ctypes.POINTER(_D)), _stream(stream)))
    return out


def z2_dos(ctx, lat, precision, state, kind=Z2_DOS_Z, stream=None):
    """Density of states (Z2_DOS_Z: by plaquettes with U_p = -1; Z2_DOS_X: by
    links with sigma^x = -1) as a numpy array of n_plaq + 1 or n_links + 1 bins."""
    out = np.zeros(40, dtype=np.float64)
    nb = ctypes.c_int32(0)
    _check(load().z2_dos(ctx, lat, int(precision), _ptr(state), int(kind), out.ctypes.data_as(ctypes.POINTER(_D)),
                         len(out), ctypes.byref(nb), _stream(stream)), ctx)
    return out[:nb.value].copy()


def trajectory(ctx, lat, p, state, every, ref=None, dos=False, stream=None):
    """One adiabatic run from |+>^N, measured every `every` Trotter steps and at
    the end (Sec. 3.2: observables along the ramp, s = j / M).  Built from
    z2_init_plus, z2_evolve segments and z2_measure (plus z2_dos when `dos`),
    so every point is the state the unsegmented run has after j steps.
    `lat` is a Lattice; returns a list of dicts: step j, results (see
    results_dict) and, with dos, the "zdos" and "xdos" arrays."""
    if every < 1:
        raise ValueError("every must be >= 1")
    marks = list(range(every, p.M, every)) + [p.M]
    z2_init_plus(ctx, lat.handle, p.precision, state, stream)
    points, j = [], 0
    for j1 in marks:
        z2_evolve(ctx, lat.handle, p, state, j, j1, stream)
        j = j1
        point = {"step": j1, **results_dict(z2_measure(ctx, lat.handle, p, state, j1 / p.M, ref, stream), lat.info)}
        if dos:
            point["zdos"] = z2_dos(ctx, lat.handle, p.precision, state, Z2_DOS_Z, stream)
            point["xdos"] = z2_dos(ctx, lat.handle, p.precision, state, Z2_DOS_X, stream)
        points.append(point)
    return points


def finite_differences(x, y):
    """First and second derivatives of samples y(x) on an increasing, possibly
    uneven grid, by three-point differences (second order inside, first order
    at the two ends for the second derivative): the host step of the paper's
    critical-point estimate from d<H>/d lambda and d^2<H>/d lambda^2 (Sec. 3.2).
    Returns (dy, d2y, x at the largest |d2y| inside the grid)."""
    x = np.asarray(x, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    if x.ndim != 1 or x.shape != y.shape or len(x) < 3 or np.any(np.diff(x) <= 0):
        raise ValueError("need >= 3 samples on a strictly increasing grid")
    n = len(x)
    dy = np.empty(n)
    d2y = np.empty(n)
    for i in range(n):
        j = min(max(i, 1), n - 2)  # centre of the three points used
        h0, h1 = x[j] - x[j - 1], x[j + 1] - x[j]
        a, b, c = y[j - 1], y[j], y[j + 1]
        d2 = 2.0 * (h0 * c - (h0 + h1) * b + h1 * a) / (h0 * h1 * (h0 + h1))
        d1_mid = (h0 * h0 * c + (h1 * h1 - h0 * h0) * b - h1 * h1 * a) / (h0 * h1 * (h0 + h1))
        dy[i] = d1_mid + d2 * (x[i] - x[j])
        d2y[i] = d2
    inner = np.arange(1, n - 1)
    xc = x[inner[np.argmax(np.abs(d2y[inner]))]]
    return dy, d2y, xc


def z2_overlap(ctx, n_qubits, precision, a, b, stream=None):
    out = np.zeros(2, dtype=np.float64)
    _check(load().z2_overlap(ctx, n_qubits, precision, _ptr(a), _ptr(b), out.ctypes.data_as(ctypes.POINTER(_D)),
                             _stream(stream)), ctx)
    return complex(out[0], out[1])


def run_specs(specs):
    """List of dicts (d, L, lam, T, M, decomp[, precision, sampling]) -> RunSpec array."""
    arr = (RunSpec * len(specs))()
    for i, sp in enumerate(specs):
        L = list(sp["L"]) + [1] * (3 - len(sp["L"]))
        arr[i].d = sp["d"]
        arr[i].L[:] = L[:3]
        arr[i].params = params(sp["lam"], sp["T"], sp["M"], sp.get("decomp", Z2_SYMMETRIC),
                               sp.get("precision", Z2_C64), sp.get("sampling", Z2_SAMPLE_STD))
    return arr


def z2_sweep(ctx, specs, mode=Z2_SWEEP_GRAPHS, n_streams=8):
    """Run a batch of independent adiabatic runs; returns a list of Results."""
    arr = specs if isinstance(specs, ctypes.Array) else run_specs(specs)
    out = (Results * len(arr))()
    _check(load().z2_sweep(ctx, arr, len(arr), int(mode), int(n_streams), out), ctx)
    return list(out)


def _scheck(rc, what):
    if rc != Z2_OK:
        raise Z2Error(rc, what)


def z2_server_create(ctx, hbm_budget=0, max_slots=8):
    out = _P()
    _check(load().z2_server_create(ctx, int(hbm_budget), int(max_slots), ctypes.byref(out)), ctx)
    return out.value


def z2_server_submit(srv, spec):
    arr = run_specs([spec]) if isinstance(spec, dict) else spec
    t = ctypes.c_uint64()
    _scheck(load().z2_server_submit(srv, arr, ctypes.byref(t)), "server submit")
    return t.value


def z2_server_poll(srv, ticket):
    done = _I()
    res = Results()
    rc = load().z2_server_poll(srv, ticket, ctypes.byref(done), ctypes.byref(res))
    if rc not in (Z2_OK, -7):
        raise Z2Error(rc, "server poll")
    return bool(done.value), res


def z2_server_wait(srv, ticket, timeout_s=-1.0):
    res = Results()
    rc = load().z2_server_wait(srv, ticket, float(timeout_s), ctypes.byref(res))
    return rc, res


def z2_server_cancel(srv, ticket):
    return load().z2_server_cancel(srv, ticket)


def z2_server_stats(srv):
    st = ServeStats()
    _scheck(load().z2_server_stats(srv, ctypes.byref(st)), "server stats")
    return st


def z2_server_request_times(srv, ticket):
    q, r = _D(), _D()
    _scheck(load().z2_server_request_times(srv, ticket, ctypes.byref(q), ctypes.byref(r)), "request times")
    return q.value, r.value


def z2_server_request_device_times(srv, ticket):
    a, b = _D(), _D()
    _scheck(load().z2_server_request_device_times(srv, ticket, ctypes.byref(a), ctypes.byref(b)),
            "request device times")
    return a.value, b.value


Z2_SERVE_OPT_LARGE_QUBITS, Z2_SERVE_OPT_MAX_LARGE = 0, 1


def z2_server_set_option(srv, option, value):
    _scheck(load().z2_server_set_option(srv, int(option), int(value)), "server option")


def z2_server_destroy(srv):
    _scheck(load().z2_server_destroy(srv), "server destroy")


def results_dict(res, info):
    """Results struct -> dict of numpy arrays trimmed to the lattice."""
    d = {k: getattr(res, k) for k in ("s", "energy", "norm", "mean_plaq", "wilson_2x2", "mean_star", "fidelity",
                                      "flags", "status")}
    d["plaq"] = np.array(res.plaq[:info.n_plaq])
    d["star"] = np.array(res.star[:info.n_sites])
    d["sigmaz"] = np.array(res.sigmaz[:info.n_links])
    d["sigmax"] = np.array(res.sigmax[:info.n_links])
    d["wmu"] = np.array(res.wmu[:info.d])
    d["vmu"] = np.array(res.vmu[:info.d])
    d["contours"] = np.array(res.contours[:3])
    return d


# -- small object wrappers ---------------------------------------------------------
class Context:
    def __init__(self, device=0):
        self.handle = z2_ctx_create(device)

    def close(self):
        if self.handle:
            z2_ctx_destroy(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Lattice:
    def __init__(self, d, L):
        self.handle = z2_lattice_create(d, L)
        self.info = z2_lattice_info_get(self.handle)
        self.d = self.info.d
        self.n_links = self.info.n_links
        self.n_plaq = self.info.n_plaq
        self.n_sites = self.info.n_sites

    def masks(self, kind):
        return z2_lattice_masks(self.handle, kind)

    def state_bytes(self, precision=Z2_C64):
        return z2_state_bytes(self.handle, precision)

    def close(self):
        if self.handle:
            z2_lattice_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def gramp_params(g_s, t_s, N_s, n, decomp=Z2_SYMMETRIC, precision=Z2_C64):
    """Parameters of the paper's own ramp H(g) = Z + g X (z2_gramp_params)."""
    return GrampParams(float(g_s), float(t_s), int(N_s), int(n), int(decomp), int(precision))


def qpe_params(g, t, n, decomp=Z2_SYMMETRIC, precision=Z2_C64):
    """Parameters of the controlled evolution U(t) of phase estimation (z2_qpe_params)."""
    return QpeParams(float(g), float(t), int(n), int(decomp), int(precision), 0)


def params(lam, T, M, decomp=Z2_SYMMETRIC, precision=Z2_C64, sampling=Z2_SAMPLE_STD):
    return RunParams(float(lam), float(T), int(M), int(decomp), int(precision), int(sampling))
