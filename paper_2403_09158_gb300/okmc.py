"""ctypes binding of the C ABI in include/okmc.h (argument marshalling only).

Every function here forwards to the CUDA library ``_lib/libokmc.so``; nothing
of the method is computed in Python.  Loading fails loudly when the library is
missing: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from .workload import DEFECT_DTYPE

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, '_lib', 'libokmc.so')

OKMC_OK, OKMC_EINVAL, OKMC_ENOMEM, OKMC_ECUDA, OKMC_ETIMEOUT, OKMC_ESTATE, OKMC_ERANGE = range(7)
LOOP_111, LOOP_100, SIA_CLUSTER = 0, 1, 2
IMMOBILE, ONE_D, THREE_D = 0, 1, 2
MEAN_STRESS_ZERO, MEAN_STRAIN_ZERO = 0, 1
FP32_FIELDS, FP64_FIELDS = 0, 1
RESIDENCE, FIXED_DT = 0, 1
BATCH_AUTO, BATCH_KERNELS, BATCH_GRAPHS = 0, 1, 2

EXPORTED = [
    'okmc_grid_create', 'okmc_grid_destroy', 'okmc_last_error', 'okmc_set_stream', 'okmc_set_defects',
    'okmc_get_defects', 'okmc_set_positions', 'okmc_get_positions', 'okmc_solve_stress', 'okmc_eigenstrain',
    'okmc_interaction_energies', 'okmc_candidate_energies', 'okmc_self_terms', 'okmc_dipole_energies',
    'okmc_dipole_self_terms', 'okmc_get_stencil', 'okmc_step',
    'okmc_get_stats', 'okmc_device_bytes', 'okmc_set_profiling', 'okmc_kernel_times', 'okmc_reset_kernel_times',
    'okmc_launch_shape', 'okmc_solve_stress_static', 'okmc_set_graphs', 'okmc_batch_create', 'okmc_batch_step',
    'okmc_batch_destroy', 'okmc_batch_last_error', 'okmc_batch_set_mode', 'okmc_batch_get_mode', 'okmc_get_variants',
    'okmc_set_variant',
    'okmc_set_kinetic_state', 'okmc_estimate_field_bytes', 'okmc_server_create', 'okmc_server_add_replica',
    'okmc_server_submit', 'okmc_server_wait', 'okmc_server_get_stats', 'okmc_server_last_error', 'okmc_server_destroy',
    'okmc_isotropic_stiffness', 'okmc_set_dislocations', 'okmc_point_dipole_energies', 'okmc_shift_energies',
]


class GridDesc(C.Structure):
    _fields_ = [('n', C.c_int32 * 3), ('k0_mode', C.c_int32), ('precision', C.c_int32), ('reserved', C.c_int32),
                ('voxel_nm', C.c_double), ('C11', C.c_double), ('C12', C.c_double), ('C44', C.c_double),
                ('nu0', C.c_double), ('seed', C.c_uint64), ('stream', C.c_void_p), ('hbm_budget', C.c_size_t)]


class StepParams(C.Structure):
    _fields_ = [('T_K', C.c_double), ('mode', C.c_int32), ('reserved', C.c_int32), ('t_end', C.c_double)]


class StepStats(C.Structure):
    _fields_ = [('events', C.c_int64), ('steps', C.c_int64), ('solves', C.c_int64),
                ('negative_barriers', C.c_int64), ('clock', C.c_double), ('dt_last', C.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class ServerDesc(C.Structure):
    _fields_ = [('hbm_budget', C.c_size_t), ('lanes', C.c_int32), ('reserved', C.c_int32)]


class Request(C.Structure):
    _fields_ = [('replica', C.c_int32), ('kind', C.c_int32), ('n_events', C.c_int64), ('params', StepParams),
                ('energies', C.c_void_p), ('positions', C.c_void_p)]


class Result(C.Structure):
    _fields_ = [('status', C.c_int32), ('admitted', C.c_int32), ('t_submit', C.c_double), ('t_start', C.c_double),
                ('t_end', C.c_double), ('stats', StepStats)]


class ServerStats(C.Structure):
    _fields_ = [('submitted', C.c_int64), ('completed', C.c_int64), ('failed', C.c_int64), ('admissions', C.c_int64),
                ('evictions', C.c_int64), ('resident', C.c_int64), ('queued', C.c_int64), ('device_bytes', C.c_size_t)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class OkmcError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__('okmc error %d: %s' % (code, msg))
        self.code = code


_lib = None


def load(path=LIB_PATH):
    """Load the CUDA library (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise OkmcError(-1, 'CUDA library not built: %s (run __graft_entry__.build())' % path)
    lib = C.CDLL(path)
    vp, i32, i64, dp = C.c_void_p, C.c_int32, C.c_int64, C.c_void_p
    sig = {
        'okmc_grid_create': (C.c_int, [C.POINTER(GridDesc), C.POINTER(vp)]),
        'okmc_grid_destroy': (C.c_int, [vp]),
        'okmc_last_error': (C.c_char_p, [vp]),
        'okmc_set_stream': (C.c_int, [vp, vp]),
        'okmc_set_defects': (C.c_int, [vp, dp, i32]),
        'okmc_get_defects': (C.c_int, [vp, dp, i32]),
        'okmc_set_positions': (C.c_int, [vp, dp, i32, C.c_int]),
        'okmc_get_positions': (C.c_int, [vp, dp, i32, C.c_int]),
        'okmc_solve_stress': (C.c_int, [vp, dp, C.c_int]),
        'okmc_eigenstrain': (C.c_int, [vp, dp, C.c_int]),
        'okmc_interaction_energies': (C.c_int, [vp, dp, C.c_int]),
        'okmc_candidate_energies': (C.c_int, [vp, dp, dp, C.c_int]),
        'okmc_self_terms': (C.c_int, [vp, dp, C.c_int]),
        'okmc_set_dislocations': (C.c_int, [vp, dp, dp, dp, dp, i32, C.c_double]),
        'okmc_point_dipole_energies': (C.c_int, [vp, dp, dp, i32, dp, C.c_int]),
        'okmc_shift_energies': (C.c_int, [vp, i32, dp, i32, dp, C.c_int]),
        'okmc_dipole_energies': (C.c_int, [vp, dp, dp, C.c_int]),
        'okmc_dipole_self_terms': (C.c_int, [vp, dp, C.c_int]),
        'okmc_get_stencil': (C.c_int, [vp, i32, i32, dp, dp, i32, C.POINTER(i32), C.POINTER(C.c_double)]),
        'okmc_step': (C.c_int, [vp, C.POINTER(StepParams), i64, C.POINTER(StepStats)]),
        'okmc_get_stats': (C.c_int, [vp, C.POINTER(StepStats)]),
        'okmc_device_bytes': (C.c_size_t, [vp]),
        'okmc_set_profiling': (C.c_int, [vp, C.c_int]),
        'okmc_kernel_times': (C.c_int, [vp, C.POINTER(C.c_char_p), C.POINTER(C.c_double), C.POINTER(i64), C.c_int]),
        'okmc_reset_kernel_times': (C.c_int, [vp]),
        'okmc_launch_shape': (C.c_int, [vp, C.POINTER(i32)]),
        'okmc_solve_stress_static': (C.c_int, [dp, dp, C.POINTER(i32), C.c_double, C.c_double, C.c_double, i32,
                                              vp]),
        'okmc_set_graphs': (C.c_int, [vp, C.c_int]),
        'okmc_batch_create': (C.c_int, [C.POINTER(vp), i32, vp, C.POINTER(vp)]),
        'okmc_batch_step': (C.c_int, [vp, C.POINTER(StepParams), i64, C.POINTER(StepStats)]),
        'okmc_batch_destroy': (C.c_int, [vp]),
        'okmc_batch_last_error': (C.c_char_p, [vp]),
        'okmc_batch_set_mode': (C.c_int, [vp, i32]),
        'okmc_batch_get_mode': (C.c_int, [vp, C.POINTER(i32)]),
        'okmc_get_variants': (C.c_int, [vp, C.POINTER(i32), C.POINTER(i32)]),
        'okmc_set_kinetic_state': (C.c_int, [vp, C.POINTER(StepStats)]),
        'okmc_estimate_field_bytes': (C.c_size_t, [C.POINTER(GridDesc)]),
        'okmc_server_create': (C.c_int, [C.POINTER(ServerDesc), C.POINTER(vp)]),
        'okmc_server_add_replica': (C.c_int, [vp, C.POINTER(GridDesc), dp, i32, C.POINTER(i32)]),
        'okmc_server_submit': (C.c_int, [vp, C.POINTER(Request), C.POINTER(C.c_uint64)]),
        'okmc_server_wait': (C.c_int, [vp, C.c_uint64, i32, C.POINTER(Result)]),
        'okmc_server_get_stats': (C.c_int, [vp, C.POINTER(ServerStats)]),
        'okmc_server_last_error': (C.c_char_p, [vp]),
        'okmc_server_destroy': (C.c_int, [vp]),
        'okmc_isotropic_stiffness': (C.c_int, [C.c_double, C.c_double, C.POINTER(C.c_double)]),
        'okmc_set_variant': (C.c_int, [vp, i32, i32]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def _ptr(a):
    """(address, on_device) of a numpy array, a torch tensor or a raw int address."""
    if a is None:
        return None, 0
    if isinstance(a, np.ndarray):
        assert a.flags['C_CONTIGUOUS']
        return a.ctypes.data, 0
    if hasattr(a, 'data_ptr'):
        assert a.is_contiguous()
        return a.data_ptr(), int(a.is_cuda)
    raise TypeError('expected a numpy array or a torch tensor')


class Grid:
    """One okmc_grid handle.  Methods mirror the C calls one to one."""

    def __init__(self, n, voxel_nm, C11, C12, C44, k0_mode=MEAN_STRESS_ZERO, precision=FP32_FIELDS, nu0=0.0,
                 seed=0, stream=None, hbm_budget=0):
        self.lib = load()
        d = GridDesc()
        n = tuple(int(v) for v in (n if np.ndim(n) else (n, n, n)))
        d.n[:] = n
        d.k0_mode, d.precision, d.reserved = k0_mode, precision, 0
        d.voxel_nm, d.C11, d.C12, d.C44, d.nu0 = voxel_nm, C11, C12, C44, nu0
        d.seed = seed
        d.stream = stream
        d.hbm_budget = hbm_budget
        h = C.c_void_p()
        rc = self.lib.okmc_grid_create(C.byref(d), C.byref(h))
        if rc != OKMC_OK:
            raise OkmcError(rc, 'okmc_grid_create failed')
        self.h = h
        self.n = n
        self.precision = precision
        self.nd = 0
        self.fdtype = np.float64 if precision == FP64_FIELDS else np.float32

    def _chk(self, rc):
        if rc != OKMC_OK:
            raise OkmcError(rc, self.lib.okmc_last_error(self.h).decode())

    def close(self):
        if getattr(self, 'h', None):
            self.lib.okmc_grid_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_stream(self, stream_ptr):
        self._chk(self.lib.okmc_set_stream(self.h, stream_ptr))

    def set_defects(self, defects):
        d = np.ascontiguousarray(defects, dtype=DEFECT_DTYPE)
        self._chk(self.lib.okmc_set_defects(self.h, d.ctypes.data if len(d) else None, len(d)))
        self.nd = len(d)

    def get_defects(self):
        out = np.zeros(self.nd, dtype=DEFECT_DTYPE)
        self._chk(self.lib.okmc_get_defects(self.h, out.ctypes.data if self.nd else None, self.nd))
        return out

    def set_positions(self, pos):
        p, dev = _ptr(pos)
        self._chk(self.lib.okmc_set_positions(self.h, p, self.nd, dev))

    def get_positions(self, out=None):
        if out is None:
            out = np.zeros((self.nd, 3), dtype=np.int32)
        p, dev = _ptr(out)
        self._chk(self.lib.okmc_get_positions(self.h, p, self.nd, dev))
        return out

    def solve_stress(self, out=None, copy=True):
        if out is None and copy:
            out = np.zeros((6, self.n[2], self.n[1], self.n[0]), dtype=self.fdtype)
        p, dev = _ptr(out)
        self._chk(self.lib.okmc_solve_stress(self.h, p, dev))
        return out

    def eigenstrain(self, out=None):
        if out is None:
            out = np.zeros((6, self.n[2], self.n[1], self.n[0]), dtype=self.fdtype)
        p, dev = _ptr(out)
        self._chk(self.lib.okmc_eigenstrain(self.h, p, dev))
        return out

    def interaction_energies(self, out=None):
        if out is None:
            out = np.zeros(self.nd)
        p, dev = _ptr(out)
        self._chk(self.lib.okmc_interaction_energies(self.h, p, dev))
        return out

    def candidate_energies(self, out=None, valid=None):
        if out is None:
            out = np.zeros((self.nd, 8))
        if valid is None and isinstance(out, np.ndarray):
            valid = np.zeros((self.nd, 8), dtype=np.uint8)
        p, dev = _ptr(out)
        v, _ = _ptr(valid)
        self._chk(self.lib.okmc_candidate_energies(self.h, p, v, dev))
        return out, valid

    def set_dislocations(self, lines, ds_max_nm=0.0):
        """Immobile dislocation lines (okmc_set_dislocations): `lines` is a list of
        (points (m, 3) nm, burgers (3,) nm, closed) tuples; [] removes them."""
        pts = np.ascontiguousarray(np.concatenate([np.asarray(p, np.float64).reshape(-1, 3) for p, _, _ in lines])
                                   if lines else np.zeros((0, 3)), dtype=np.float64)
        cnt = np.ascontiguousarray([len(np.asarray(p).reshape(-1, 3)) for p, _, _ in lines], dtype=np.int32)
        cl = np.ascontiguousarray([1 if c else 0 for _, _, c in lines], dtype=np.int32)
        b = np.ascontiguousarray(np.asarray([bv for _, bv, _ in lines], np.float64).reshape(-1, 3))
        n = len(lines)
        self._chk(self.lib.okmc_set_dislocations(self.h, pts.ctypes.data if n else None, cnt.ctypes.data if n else None,
                                                 cl.ctypes.data if n else None, b.ctypes.data if n else None, n,
                                                 float(ds_max_nm)))

    def point_dipole_energies(self, pos, P):
        """okmc_point_dipole_energies on host arrays: pos (m, 3) int32 sites, P (m, 6) eV."""
        pos = np.ascontiguousarray(pos, dtype=np.int32).reshape(-1, 3)
        P = np.ascontiguousarray(np.broadcast_to(np.asarray(P, np.float64), (len(pos), 6)))
        out = np.zeros(len(pos))
        m = len(pos)
        self._chk(self.lib.okmc_point_dipole_energies(self.h, pos.ctypes.data if m else None, P.ctypes.data if m else None,
                                                      m, out.ctypes.data if m else None, 0))
        return out

    def shift_energies(self, i, X):
        """okmc_shift_energies on host arrays: defect i moved to positions X (m, 3) nm."""
        X = np.ascontiguousarray(X, dtype=np.float64).reshape(-1, 3)
        out = np.zeros(len(X))
        m = len(X)
        self._chk(self.lib.okmc_shift_energies(self.h, int(i), X.ctypes.data if m else None, m,
                                               out.ctypes.data if m else None, 0))
        return out

    def self_terms(self):
        out = np.zeros((self.nd, 2, 9))
        self._chk(self.lib.okmc_self_terms(self.h, out.ctypes.data, 0))
        return out

    def dipole_energies(self):
        """(E[n], Ec[n][8]): dipole-approximation energies at the sites and after the jumps."""
        E = np.zeros(self.nd)
        Ec = np.zeros((self.nd, 8))
        self._chk(self.lib.okmc_dipole_energies(self.h, E.ctypes.data, Ec.ctypes.data, 0))
        return E, Ec

    def dipole_self_terms(self):
        out = np.zeros((self.nd, 2, 9))
        self._chk(self.lib.okmc_dipole_self_terms(self.h, out.ctypes.data, 0))
        return out

    def stencil(self, i, c):
        k = C.c_int32()
        a = C.c_double()
        self._chk(self.lib.okmc_get_stencil(self.h, i, c, None, None, 0, C.byref(k), C.byref(a)))
        offs = np.zeros((k.value, 3), dtype=np.int32)
        cnt = np.zeros(k.value, dtype=np.int32)
        self._chk(self.lib.okmc_get_stencil(self.h, i, c, offs.ctypes.data, cnt.ctypes.data, k.value, C.byref(k),
                                            C.byref(a)))
        return offs, cnt, a.value

    def step(self, T_K, n_steps=1, mode=RESIDENCE, t_end=0.0):
        p = StepParams(T_K, mode, 0, t_end)
        s = StepStats()
        self._chk(self.lib.okmc_step(self.h, C.byref(p), n_steps, C.byref(s)))
        return s.as_dict()

    def set_kinetic_state(self, st):
        s = StepStats(**{k: st[k] for k, _ in StepStats._fields_})
        self._chk(self.lib.okmc_set_kinetic_state(self.h, C.byref(s)))

    def stats(self):
        s = StepStats()
        self._chk(self.lib.okmc_get_stats(self.h, C.byref(s)))
        return s.as_dict()

    def device_bytes(self):
        return int(self.lib.okmc_device_bytes(self.h))

    def set_profiling(self, on=True):
        self._chk(self.lib.okmc_set_profiling(self.h, int(on)))

    def kernel_times(self):
        cap = 64
        names = (C.c_char_p * cap)()
        ms = (C.c_double * cap)()
        cnt = (C.c_int64 * cap)()
        k = self.lib.okmc_kernel_times(self.h, names, ms, cnt, cap)
        return {names[i].decode(): (ms[i], cnt[i]) for i in range(min(k, cap))}

    def reset_kernel_times(self):
        self._chk(self.lib.okmc_reset_kernel_times(self.h))

    def set_graphs(self, on=True):
        self._chk(self.lib.okmc_set_graphs(self.h, int(on)))

    def variants(self):
        """(current, available): per pass (forward plane, pencil, inverse plane) the
        launch variant in use and the bit mask of variants that exist."""
        cur = (C.c_int32 * 3)()
        av = (C.c_int32 * 3)()
        self._chk(self.lib.okmc_get_variants(self.h, cur, av))
        return list(cur), list(av)

    def set_variant(self, pass_, variant):
        self._chk(self.lib.okmc_set_variant(self.h, pass_, variant))

    def launch_shape(self):
        out = (C.c_int32 * 3)()
        self._chk(self.lib.okmc_launch_shape(self.h, out))
        return list(out)


class Batch:
    """Replicas advanced together by one CUDA graph launch per step (okmc_batch_*)."""

    def __init__(self, grids, stream=None, mode=BATCH_AUTO):
        self.lib = load()
        self.grids = list(grids)
        arr = (C.c_void_p * len(self.grids))(*[g.h.value for g in self.grids])
        h = C.c_void_p()
        rc = self.lib.okmc_batch_create(arr, len(self.grids), stream, C.byref(h))
        if rc != OKMC_OK:
            raise OkmcError(rc, 'okmc_batch_create failed')
        self.h = h
        rc = self.lib.okmc_batch_set_mode(self.h, mode)
        if rc != OKMC_OK:
            raise OkmcError(rc, 'okmc_batch_set_mode failed')

    def mode(self):
        """The form the last step used (BATCH_KERNELS or BATCH_GRAPHS; 0 before the first)."""
        m = C.c_int32()
        self.lib.okmc_batch_get_mode(self.h, C.byref(m))
        return m.value

    def step(self, T_K, n_steps=1, mode=RESIDENCE):
        n = len(self.grids)
        Ts = list(T_K) if np.ndim(T_K) else [T_K] * n
        modes = list(mode) if np.ndim(mode) else [mode] * n
        params = (StepParams * n)(*[StepParams(float(t), int(m), 0, 0.0) for t, m in zip(Ts, modes)])
        stats = (StepStats * n)()
        rc = self.lib.okmc_batch_step(self.h, params, n_steps, stats)
        if rc != OKMC_OK:
            raise OkmcError(rc, self.lib.okmc_batch_last_error(self.h).decode())
        return [s.as_dict() for s in stats]

    def close(self):
        if getattr(self, 'h', None):
            self.lib.okmc_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


SOLVE, STEP = 0, 1


def _grid_desc(n, voxel_nm, C11, C12, C44, k0_mode=MEAN_STRESS_ZERO, precision=FP32_FIELDS, nu0=0.0, seed=0):
    d = GridDesc()
    d.n[:] = tuple(int(v) for v in (n if np.ndim(n) else (n, n, n)))
    d.k0_mode, d.precision, d.reserved = k0_mode, precision, 0
    d.voxel_nm, d.C11, d.C12, d.C44, d.nu0 = voxel_nm, C11, C12, C44, nu0
    d.seed = seed
    return d


def isotropic_stiffness(mu_GPa, nu):
    """(C11, C12, C44) of an isotropic solid (okmc_isotropic_stiffness)."""
    out = (C.c_double * 3)()
    rc = load().okmc_isotropic_stiffness(mu_GPa, nu, out)
    if rc != OKMC_OK:
        raise OkmcError(rc, 'okmc_isotropic_stiffness: mu must be > 0 and -1 < nu < 1/2')
    return tuple(out)


def estimate_field_bytes(n, voxel_nm, C11, C12, C44, **kw):
    return int(load().okmc_estimate_field_bytes(C.byref(_grid_desc(n, voxel_nm, C11, C12, C44, **kw))))


class Server:
    """okmc_server_*: request server over resident replicas.  submit() returns a
    ticket; the output arrays handed to the library are kept alive here until the
    ticket's result has been fetched with wait()."""

    def __init__(self, hbm_budget=0, lanes=4):
        self.lib = load()
        d = ServerDesc(hbm_budget, lanes, 0)
        h = C.c_void_p()
        rc = self.lib.okmc_server_create(C.byref(d), C.byref(h))
        if rc != OKMC_OK:
            raise OkmcError(rc, 'okmc_server_create failed')
        self.h = h
        self.nd = []
        self._keep = {}

    def _chk(self, rc):
        if rc != OKMC_OK:
            raise OkmcError(rc, self.lib.okmc_server_last_error(self.h).decode())

    def add_replica(self, n, voxel_nm, C11, C12, C44, defects, **kw):
        d = _grid_desc(n, voxel_nm, C11, C12, C44, **kw)
        defs = np.ascontiguousarray(defects, dtype=DEFECT_DTYPE)
        rid = C.c_int32()
        self._chk(self.lib.okmc_server_add_replica(self.h, C.byref(d), defs.ctypes.data if len(defs) else None,
                                                   len(defs), C.byref(rid)))
        self.nd.append(len(defs))
        return rid.value

    def submit_solve(self, replica):
        E = np.zeros(self.nd[replica], dtype=np.float64)
        r = Request(replica, SOLVE, 0, StepParams(0.0, RESIDENCE, 0, 0.0), E.ctypes.data, None)
        return self._submit(r, E)

    def submit_step(self, replica, T_K, n_events, mode=RESIDENCE, positions=True):
        P = np.zeros((self.nd[replica], 3), dtype=np.int32) if positions else None
        r = Request(replica, STEP, n_events, StepParams(float(T_K), mode, 0, 0.0), None,
                    P.ctypes.data if P is not None else None)
        return self._submit(r, P)

    def _submit(self, r, out):
        t = C.c_uint64()
        self._chk(self.lib.okmc_server_submit(self.h, C.byref(r), C.byref(t)))
        self._keep[t.value] = out
        return t.value

    def wait(self, ticket, timeout_ms=-1):
        """(result dict, output array) of a ticket; raises OkmcError on timeout."""
        res = Result()
        self._chk(self.lib.okmc_server_wait(self.h, ticket, timeout_ms, C.byref(res)))
        out = self._keep.pop(ticket)
        d = {k: getattr(res, k) for k, _ in Result._fields_ if k != 'stats'}
        d['stats'] = res.stats.as_dict()
        return d, out

    def stats(self):
        st = ServerStats()
        self._chk(self.lib.okmc_server_get_stats(self.h, C.byref(st)))
        return st.as_dict()

    def close(self):
        if getattr(self, 'h', None):
            self.lib.okmc_server_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
