"""Thin Python binding of the C ABI in include/bsmps.h (argument marshalling only).

Every computation runs in libbsmps.so; importing this module fails loudly when
the library has not been built (there is no CPU fallback).
"""

import ctypes as C
import math
import os

import numpy as np

_LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_lib", "libbsmps.so")

OK = 0
STATUS = {0: "OK", 1: "INVALID_ARG", 2: "CHARGE", 3: "OOM", 4: "RANK_CAP", 5: "NOT_SPD",
          6: "NUMERIC", 7: "TIMEOUT", 8: "CUDA"}


class BsmpsError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{STATUS.get(code, code)}: {msg}")
        self.code = code


class Precond(C.Structure):
    _fields_ = [("K", C.c_int), ("d", C.POINTER(C.c_double)), ("t_min", C.c_double),
                ("t_max", C.c_double), ("c0", C.c_double), ("alpha0", C.c_double)]


class SolverParams(C.Structure):
    _fields_ = [("c", C.c_double), ("delta", C.c_double), ("eps_num", C.c_double),
                ("t_eig", C.c_double), ("tau", C.c_double), ("r_max", C.c_int), ("u_rel", C.c_double)]


class SolverState(C.Structure):
    _fields_ = [("eta_res", C.c_double), ("n", C.c_int), ("last_tries", C.c_int),
                ("last_sum_norms", C.c_double), ("fp64_locked", C.c_int)]


class StepInfo(C.Structure):
    _fields_ = [("lambda_", C.c_double), ("rho", C.c_double), ("eta_res", C.c_double),
                ("res_norm", C.c_double), ("eta_tries", C.c_int), ("bound", C.c_double),
                ("releig_bound", C.c_double), ("lambda_star", C.c_double), ("omega", C.c_double),
                ("eta_in", C.c_double), ("delta_A", C.c_double), ("converged", C.c_int),
                ("max_rank", C.c_int), ("flops", C.c_double), ("cap_discarded", C.c_double),
                ("precision", C.c_int)]

    def as_dict(self):
        d = {name: getattr(self, name) for name, _ in self._fields_}
        d["lambda"] = d.pop("lambda_")
        return d


class OuterRecord(C.Structure):
    _fields_ = [("inner_steps", C.c_int), ("inner_converged", C.c_int), ("lambda_", C.c_double),
                ("rho", C.c_double), ("releig_bound", C.c_double), ("eta_out", C.c_double),
                ("tau_m", C.c_double), ("max_rank_before", C.c_int), ("max_rank_after", C.c_int),
                ("flops", C.c_double)]

    def as_dict(self):
        d = {name: getattr(self, name) for name, _ in self._fields_}
        d["lambda"] = d.pop("lambda_")
        return d


MAX_COLUMNS = 16


class JointStepInfo(C.Structure):
    _fields_ = [("D", C.c_int), ("lambda_", C.c_double * MAX_COLUMNS), ("rho", C.c_double * MAX_COLUMNS),
                ("res_norm", C.c_double * MAX_COLUMNS), ("lambda_star", C.c_double * MAX_COLUMNS),
                ("delta_A", C.c_double * MAX_COLUMNS), ("eta_res", C.c_double), ("eta_tries", C.c_int),
                ("bound", C.c_double), ("releig_bound", C.c_double), ("eta_in", C.c_double),
                ("converged", C.c_int), ("max_rank", C.c_int), ("flops", C.c_double),
                ("cap_discarded", C.c_double)]

    def as_dict(self):
        D = self.D
        d = {}
        for name, _ in self._fields_:
            v = getattr(self, name)
            d[name] = np.array(v[:D]) if isinstance(v, C.Array) else v
        d["lambda"] = d.pop("lambda_")
        return d


_vp = C.c_void_p
_i = C.c_int
_d = C.c_double
_i64 = C.c_int64
_pd = C.POINTER(C.c_double)
_pi = C.POINTER(C.c_int)
_pi64 = C.POINTER(C.c_int64)

_SIGS = {
    "bsmps_status_string": (C.c_char_p, [_i]),
    "bsmps_ctx_create": (_i, [_i, _vp, C.POINTER(_vp)]),
    "bsmps_ctx_destroy": (_i, [_vp]),
    "bsmps_ctx_sync": (_i, [_vp]),
    "bsmps_last_error": (C.c_char_p, [_vp]),
    "bsmps_ctx_launch_count": (_i64, [_vp]),
    "bsmps_ctx_alloc_count": (_i64, [_vp]),
    "bsmps_ctx_profile": (_i, [_vp, _i]),
    "bsmps_ctx_kernel_stats": (_i, [_vp, _i, _i, _pi64, _pd, _pd, _pd]),
    "bsmps_precond_theta": (_i, [_i, _pd, _pd, _i, _i, _d, _pd]),
    "bsmps_precond_interval": (_i, [_i, _i, _pd, _pd, _i, _i, _pd, _pd]),
    "bsmps_energy_lower_bound": (_i, [_i, _pd, _pd, _i, _i, _i, _i, _pd]),
    "bsmps_precond_alpha0": (_i, [_d, _d, _d, _d, _pd, _pd]),
    "bsmps_lowest_determinants": (_i, [_i, _pd, _i, _i, _i, _i, _i64, C.POINTER(C.c_ubyte)]),
    "bsmps_mps_random_size": (_i, [_i, _i, _i, _i, _i, _pi64]),
    "bsmps_mps_create": (_i, [_vp, _i, _i, _i, _i, _i, _i, _pd, _i64, C.POINTER(_vp)]),
    "bsmps_mps_import": (_i, [_vp, _i, _i, _i, _i, _pi, _pi, _pd, _i64, C.POINTER(_vp)]),
    "bsmps_mps_num_sites": (_i, [_vp, _pi]),
    "bsmps_mps_num_sectors": (_i, [_vp, _pi, _pi]),
    "bsmps_mps_sectors": (_i, [_vp, _pi]),
    "bsmps_mps_size": (_i, [_vp, _pi64]),
    "bsmps_mps_export": (_i, [_vp, _pd]),
    "bsmps_mps_write": (_i, [_vp, _pd, _i64]),
    "bsmps_plan_apply_zipup_batch": (_i, [_vp, _i, C.POINTER(_vp), C.POINTER(_vp), _pd, C.POINTER(_vp),
                                         C.POINTER(_vp), _pd]),
    "bsmps_ctx_set_jacobi_precond": (_i, [_vp, _i]),
    "bsmps_plan_launch": (_i, [_vp]),
    "bsmps_plan_launch_count": (_i64, [_vp]),
    "bsmps_plan_destroy": (_i, [_vp]),
    "bsmps_mps_destroy": (_i, [_vp]),
    "bsmps_mpo_from_integrals": (_i, [_vp, _i, _pd, _pd, _i, _i, _d, _d, C.POINTER(_vp)]),
    "bsmps_mpo_bond_dims": (_i, [_vp, _pi]),
    "bsmps_mpo_num_entries": (_i, [_vp, _i, _pi]),
    "bsmps_mpo_entries": (_i, [_vp, _i, _pi, _pd]),
    "bsmps_mpo_channel_charges": (_i, [_vp, _i, _pi]),
    "bsmps_mpo_destroy": (_i, [_vp]),
    "bsmps_apply_H": (_i, [_vp, _vp, _vp, _d, _d, _i, C.POINTER(_vp), _pd]),
    "bsmps_apply_zipup": (_i, [_vp, _vp, _vp, _d, C.POINTER(_vp), _pd]),
    "bsmps_apply_zipup_batch": (_i, [_vp, _i, C.POINTER(_vp), C.POINTER(_vp), _pd, C.POINTER(_vp), _pd]),
    "bsmps_truncate": (_i, [_vp, _vp, _d, _i, C.POINTER(_vp), _pd, _pd]),
    "bsmps_add": (_i, [_vp, _vp, _vp, _d, _d, C.POINTER(_vp)]),
    "bsmps_scale_sites": (_i, [_vp, _vp, _pd, _pd, C.POINTER(_vp)]),
    "bsmps_precondition": (_i, [_vp, C.POINTER(Precond), _i, _vp, C.POINTER(_vp), _pi]),
    "bsmps_dot": (_i, [_vp, _vp, _vp, _vp, _d, _pd]),
    "bsmps_dot_noalloc": (_i, [_vp, _vp, _vp, _vp, _d, _pd]),
    "bsmps_check_grid_wait": (_i, [_vp, _i, C.POINTER(C.c_int)]),
    "bsmps_eigensolve_outer": (_i, [_vp, _vp, _vp, _vp, _d, _d, _i, _i, C.POINTER(_vp), _vp,
                                    C.POINTER(C.c_int), C.POINTER(C.c_int)]),
    "bsmps_mlp_create": (_i, [_vp, _i, _pi, C.POINTER(C.c_float), _i64, C.POINTER(_vp)]),
    "bsmps_mlp_num_params": (_i, [_vp, _pi64]),
    "bsmps_mlp_get_params": (_i, [_vp, C.POINTER(C.c_float)]),
    "bsmps_mlp_forward": (_i, [_vp, C.POINTER(C.c_float), _i, C.POINTER(C.c_float)]),
    "bsmps_mlp_loss_grad": (_i, [_vp, C.POINTER(C.c_float), C.POINTER(C.c_float), _i, C.POINTER(C.c_float),
                                 C.POINTER(C.c_float)]),
    "bsmps_mlp_train_step": (_i, [_vp, C.POINTER(C.c_float), C.POINTER(C.c_float), _i, C.c_float,
                                  C.POINTER(C.c_float)]),
    "bsmps_mlp_destroy": (_i, [_vp]),
    "bsmps_eigensolve_step": (_i, [_vp, _vp, C.POINTER(Precond), C.POINTER(SolverParams),
                                   C.POINTER(SolverState), C.POINTER(_vp), C.POINTER(StepInfo)]),
    "bsmps_gemm_tf32x3": (_i, [_vp, _i, _i, _i, _vp, _i, _vp, _i, _vp, _i]),
    "bsmps_ctx_set_precision": (_i, [_vp, _i]),
    "bsmps_gemm_ozaki": (_i, [_vp, _i, _i, _i, _vp, _i, _vp, _i, _vp, _i, _i]),
    "bsmps_ctx_set_gemm_emulation": (_i, [_vp, _i]),
    "bsmps_mps_joint_random_size": (_i, [_i, _i, _i, _i, _i, _i, _pi64]),
    "bsmps_mps_create_joint": (_i, [_vp, _i, _i, _i, _i, _i, _i, C.POINTER(C.c_ubyte), _i, _pd, _i64,
                                    C.POINTER(_vp)]),
    "bsmps_mps_num_columns": (_i, [_vp, _pi]),
    "bsmps_gram": (_i, [_vp, _vp, _vp, _vp, _d, _pd]),
    "bsmps_apply_columns": (_i, [_vp, _vp, _vp, _d, _pd, C.POINTER(_vp)]),
    "bsmps_mix_columns": (_i, [_vp, _vp, _pd, _i, C.POINTER(_vp)]),
    "bsmps_eigensolve_joint_step": (_i, [_vp, _vp, C.POINTER(Precond), C.POINTER(SolverParams),
                                         C.POINTER(SolverState), C.POINTER(_vp), C.POINTER(JointStepInfo)]),
}

DECLARED = tuple(_SIGS.keys())


def load(path=None):
    path = _LIB_PATH if path is None else path
    if not os.path.exists(path):
        raise ImportError(f"{path} is missing: build it with paper_2604_16118_gb300.build.build()")
    lib = C.CDLL(path)
    for name, (res, args) in _SIGS.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = load()
    return _lib


def _check(ctx, code):
    if code != OK:
        msg = lib().bsmps_last_error(ctx.h if ctx is not None else None)
        raise BsmpsError(code, (msg or b"").decode())


def _dptr(a):
    return a.ctypes.data_as(_pd)


def _iptr(a):
    return a.ctypes.data_as(_pi)


class Context:
    """bsmps_ctx: a device and the stream all work is ordered on."""

    def __init__(self, device=0, stream=None):
        h = _vp()
        self.h = None
        _check(None, lib().bsmps_ctx_create(device, stream, C.byref(h)))
        self.h = h

    def sync(self):
        _check(self, lib().bsmps_ctx_sync(self.h))

    def launch_count(self):
        return int(lib().bsmps_ctx_launch_count(self.h))

    def set_precision(self, precision):
        """Arithmetic of the zip-up contraction stage (PREC_FP64 or PREC_TF32X3)."""
        _check(self, lib().bsmps_ctx_set_precision(self.h, int(precision)))

    def set_jacobi_precond(self, min_k):
        """Cluster Jacobi SVDs with k >= min_k start from an FP32 Jacobi (0: never)."""
        _check(self, lib().bsmps_ctx_set_jacobi_precond(self.h, int(min_k)))

    def alloc_count(self):
        """Device-memory requests served by the context's allocator so far."""
        return int(lib().bsmps_ctx_alloc_count(self.h))

    KERNELS = ("copy", "gemm", "qr", "svd", "sumsq", "apply", "apply_qr", "mlp")

    def set_gemm_emulation(self, min_log2_flops=0):
        """Block products of at least 2^min_log2_flops flops on the tensor cores
        (0: none), see bsmps_ctx_set_gemm_emulation."""
        _check(self, lib().bsmps_ctx_set_gemm_emulation(self.h, int(min_log2_flops)))

    def profile(self, enable=True):
        _check(self, lib().bsmps_ctx_profile(self.h, 1 if enable else 0))

    def kernel_stats(self, reset=True):
        """{kind: (launches, ms, flops, bytes)} of the profiled launches."""
        out = {}
        for k, name in enumerate(self.KERNELS):
            n = C.c_int64()
            ms, fl, by = C.c_double(), C.c_double(), C.c_double()
            _check(self, lib().bsmps_ctx_kernel_stats(self.h, k, 1 if (reset and k == len(self.KERNELS) - 1) else 0,
                                                      C.byref(n), C.byref(ms), C.byref(fl), C.byref(by)))
            out[name] = (n.value, ms.value, fl.value, by.value)
        return out

    def close(self):
        if self.h:
            lib().bsmps_ctx_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class MPS:
    """bsmps_mps handle."""

    def __init__(self, ctx, h):
        self.ctx = ctx
        self.h = h

    def __del__(self):
        try:
            if self.h:
                lib().bsmps_mps_destroy(self.h)
                self.h = None
        except Exception:
            pass

    @property
    def K(self):
        k = C.c_int()
        _check(self.ctx, lib().bsmps_mps_num_sites(self.h, C.byref(k)))
        return k.value

    def bonds(self):
        """Per bond: {(n0, n1): dim} in ascending sector order."""
        K = self.K
        per = np.zeros(K + 1, dtype=np.int32)
        tot = C.c_int()
        _check(self.ctx, lib().bsmps_mps_num_sectors(self.h, _iptr(per), C.byref(tot)))
        tr = np.zeros(3 * max(tot.value, 1), dtype=np.int32)
        _check(self.ctx, lib().bsmps_mps_sectors(self.h, _iptr(tr)))
        out = []
        pos = 0
        for b in range(K + 1):
            d = {}
            for _ in range(per[b]):
                d[(int(tr[3 * pos]), int(tr[3 * pos + 1]))] = int(tr[3 * pos + 2])
                pos += 1
            out.append(d)
        return out

    def ranks(self):
        return [sum(b.values()) for b in self.bonds()]

    def size(self):
        n = C.c_int64()
        _check(self.ctx, lib().bsmps_mps_size(self.h, C.byref(n)))
        return n.value

    def export(self):
        v = np.zeros(max(self.size(), 1))
        _check(self.ctx, lib().bsmps_mps_export(self.h, _dptr(v)))
        return v[:self.size()]

    def write(self, values):
        """Overwrite the blocks in place (flat layout; bsmps_mps_write)."""
        v = np.ascontiguousarray(values, dtype=np.float64)
        _check(self.ctx, lib().bsmps_mps_write(self.h, _dptr(v), len(v)))


class MPO:
    def __init__(self, ctx, h):
        self.ctx = ctx
        self.h = h

    def __del__(self):
        try:
            if self.h:
                lib().bsmps_mpo_destroy(self.h)
                self.h = None
        except Exception:
            pass

    def bond_dims(self, K):
        d = np.zeros(K + 1, dtype=np.int32)
        _check(self.ctx, lib().bsmps_mpo_bond_dims(self.h, _iptr(d)))
        return [int(v) for v in d]

    def entries(self, site):
        n = C.c_int()
        _check(self.ctx, lib().bsmps_mpo_num_entries(self.h, site, C.byref(n)))
        q = np.zeros(4 * max(n.value, 1), dtype=np.int32)
        w = np.zeros(max(n.value, 1))
        _check(self.ctx, lib().bsmps_mpo_entries(self.h, site, _iptr(q), _dptr(w)))
        return [(int(q[4 * i]), int(q[4 * i + 1]), int(q[4 * i + 2]), int(q[4 * i + 3]), float(w[i]))
                for i in range(n.value)]

    def channel_charges(self, bond, width):
        p = np.zeros(2 * max(width, 1), dtype=np.int32)
        _check(self.ctx, lib().bsmps_mpo_channel_charges(self.h, bond, _iptr(p)))
        return [(int(p[2 * i]), int(p[2 * i + 1])) for i in range(width)]


def _c64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def precond_theta(h, eri, spin, n_particles, gamma):
    """theta_i of Sec. 7.1.1 (bsmps_precond_theta)."""
    h, eri = _c64(h), _c64(eri)
    n = h.shape[0]
    th = np.zeros(2 * n if spin else n)
    _check(None, lib().bsmps_precond_theta(n, _dptr(h), _dptr(eri), int(spin), int(n_particles), float(gamma),
                                           _dptr(th)))
    return th


def precond_interval(theta, spin, n_up, n_dn, h=None):
    """[t_min, t_max] (bsmps_precond_interval); h given: the orbital-order rule."""
    theta = _c64(theta)
    n_orb = len(theta) // 2 if spin else len(theta)
    hp = None if h is None else _c64(h)
    lo, hi = C.c_double(), C.c_double()
    _check(None, lib().bsmps_precond_interval(n_orb, int(spin), _dptr(theta), None if hp is None else _dptr(hp),
                                              int(n_up), int(n_dn), C.byref(lo), C.byref(hi)))
    return lo.value, hi.value


def energy_lower_bound(h, eri, spin, n_up, n_dn, cholesky):
    """A rigorous lower bound of the ground energy (bsmps_energy_lower_bound)."""
    h = _c64(h)
    e = None if eri is None else _c64(eri)
    out = C.c_double()
    _check(None, lib().bsmps_energy_lower_bound(h.shape[0], _dptr(h), None if e is None else _dptr(e), int(spin),
                                                int(n_up), int(n_dn), int(bool(cholesky)), C.byref(out)))
    return out.value


def precond_alpha0(c0, t_min, c_lower, c_upper):
    """(alpha_0, c) of Eq. (Sdef) / Eq. (precondcdef) (bsmps_precond_alpha0)."""
    a, c = C.c_double(), C.c_double()
    _check(None, lib().bsmps_precond_alpha0(float(c0), float(t_min), float(c_lower), float(c_upper), C.byref(a),
                                            C.byref(c)))
    return a.value, c.value


def lowest_determinants(t_diag, spin, n_up, n_dn, D, max_configs=2_000_000):
    """D x K occupation strings of the lowest determinants (bsmps_lowest_determinants)."""
    t = _c64(t_diag)
    K = len(t)
    occ = np.zeros((D, K), dtype=np.uint8)
    _check(None, lib().bsmps_lowest_determinants(K, _dptr(t), int(spin), int(n_up), int(n_dn), int(D),
                                                 int(max_configs), occ.ctypes.data_as(C.POINTER(C.c_ubyte))))
    return occ


def mps_random_size(n_orb, spin, n_up, n_dn, r_max):
    n = C.c_int64()
    _check(None, lib().bsmps_mps_random_size(n_orb, spin, n_up, n_dn, r_max, C.byref(n)))
    return n.value


def mps_create(ctx, n_orb, spin, n_up, n_dn, r_max=1, values=None):
    """e_1 when values is None, else the random-rule iterate filled from values."""
    h = _vp()
    if values is None:
        _check(ctx, lib().bsmps_mps_create(ctx.h, n_orb, spin, n_up, n_dn, r_max, 0, None, 0, C.byref(h)))
    else:
        v = np.ascontiguousarray(values, dtype=np.float64)
        _check(ctx, lib().bsmps_mps_create(ctx.h, n_orb, spin, n_up, n_dn, r_max, 1, _dptr(v), len(v),
                                            C.byref(h)))
    return MPS(ctx, h)


def mps_import(ctx, n_orb, spin, n_up, n_dn, bonds, values):
    """bonds: per bond {(n0, n1): dim}; values: flat layout."""
    per = np.array([len(b) for b in bonds], dtype=np.int32)
    tr = []
    for b in bonds:
        for q in sorted(b):
            tr += [q[0], q[1], b[q]]
    tr = np.array(tr if tr else [0], dtype=np.int32)
    v = np.ascontiguousarray(values, dtype=np.float64)
    if len(v) == 0:
        v = np.zeros(1)
        n = 0
    else:
        n = len(v)
    h = _vp()
    _check(ctx, lib().bsmps_mps_import(ctx.h, n_orb, spin, n_up, n_dn, _iptr(per), _iptr(tr), _dptr(v), n,
                                        C.byref(h)))
    return MPS(ctx, h)


def mpo_from_integrals(ctx, h, eri, spin, n_particles, gamma=0.0, compress_tol=0.0):
    hh = np.ascontiguousarray(h, dtype=np.float64)
    ee = np.ascontiguousarray(eri, dtype=np.float64)
    out = _vp()
    _check(ctx, lib().bsmps_mpo_from_integrals(ctx.h, hh.shape[0], _dptr(hh), _dptr(ee), spin, n_particles,
                                                gamma, compress_tol, C.byref(out)))
    return MPO(ctx, out)


def apply_H(ctx, mpo, x, shift=0.0, tol=0.0, r_max=0):
    y = _vp()
    fl = C.c_double()
    _check(ctx, lib().bsmps_apply_H(ctx.h, mpo.h, x.h, shift, tol, r_max, C.byref(y), C.byref(fl)))
    return MPS(ctx, y), fl.value


def apply_zipup(ctx, mpo, x, shift=0.0):
    """(H_gamma + shift) x in left-orthogonal form by the zip-up application (bsmps_apply_zipup)."""
    y = _vp()
    fl = C.c_double()
    _check(ctx, lib().bsmps_apply_zipup(ctx.h, mpo.h, x.h, shift, C.byref(y), C.byref(fl)))
    return MPS(ctx, y), fl.value


def apply_zipup_batch(ctx, mpos, xs, shifts):
    """Zip-up applications of independent problems advanced together (bsmps_apply_zipup_batch)."""
    n = len(xs)
    Wa = (_vp * n)(*[w.h for w in mpos])
    Xa = (_vp * n)(*[x.h for x in xs])
    sh = np.ascontiguousarray(shifts, dtype=np.float64)
    Ya = (_vp * n)()
    fl = C.c_double()
    _check(ctx, lib().bsmps_apply_zipup_batch(ctx.h, n, Wa, Xa, _dptr(sh), Ya, C.byref(fl)))
    return [MPS(ctx, _vp(Ya[i])) for i in range(n)], fl.value


class ZipupPlan:
    """A batch of zip-up applications recorded as one CUDA graph
    (bsmps_plan_apply_zipup_batch): launch() replays it on the context's
    stream; outputs are the MPS the replays overwrite."""

    def __init__(self, ctx, mpos, xs, shifts):
        n = len(xs)
        Wa = (_vp * n)(*[w.h for w in mpos])
        Xa = (_vp * n)(*[x.h for x in xs])
        sh = np.ascontiguousarray(shifts, dtype=np.float64)
        Ya = (_vp * n)()
        fl = C.c_double()
        h = _vp()
        _check(ctx, lib().bsmps_plan_apply_zipup_batch(ctx.h, n, Wa, Xa, _dptr(sh), C.byref(h), Ya, C.byref(fl)))
        self.ctx, self.h, self.flops = ctx, h, fl.value
        self._inputs = (list(mpos), list(xs))   # the graph reads them
        self.outputs = [MPS(ctx, _vp(Ya[i])) for i in range(n)]
        for o in self.outputs:
            o._plan = self   # the outputs' blocks live in the plan's memory

    def launch(self):
        _check(self.ctx, lib().bsmps_plan_launch(self.h))

    def launch_count(self):
        return int(lib().bsmps_plan_launch_count(self.h))

    def __del__(self):
        try:
            if self.h:
                lib().bsmps_plan_destroy(self.h)
                self.h = None
        except Exception:
            pass


def truncate(ctx, x, eps, r_max=0):
    y = _vp()
    dt = C.c_double()
    dc = C.c_double()
    _check(ctx, lib().bsmps_truncate(ctx.h, x.h, eps, r_max, C.byref(y), C.byref(dt), C.byref(dc)))
    return MPS(ctx, y), dt.value, dc.value


def add(ctx, x, y, alpha=1.0, beta=1.0):
    o = _vp()
    _check(ctx, lib().bsmps_add(ctx.h, x.h, y.h, alpha, beta, C.byref(o)))
    return MPS(ctx, o)


def scale_sites(ctx, x, f0, f1):
    a = np.ascontiguousarray(f0, dtype=np.float64)
    b = np.ascontiguousarray(f1, dtype=np.float64)
    o = _vp()
    _check(ctx, lib().bsmps_scale_sites(ctx.h, x.h, _dptr(a), _dptr(b), C.byref(o)))
    return MPS(ctx, o)


def make_precond(d, t_min, t_max, c0, alpha0):
    d = np.ascontiguousarray(d, dtype=np.float64)
    p = Precond(len(d), _dptr(d), t_min, t_max, c0, alpha0)
    p._keep = d
    return p


def precondition(ctx, p, x, term=-1):
    o = _vp()
    n = C.c_int()
    _check(ctx, lib().bsmps_precondition(ctx.h, C.byref(p), term, x.h, C.byref(o), C.byref(n)))
    return MPS(ctx, o), n.value


def dot(ctx, a, b, mpo=None, shift=0.0):
    out = C.c_double()
    _check(ctx, lib().bsmps_dot(ctx.h, a.h, b.h, mpo.h if mpo is not None else None, shift, C.byref(out)))
    return out.value


def dot_noalloc(ctx, a, b, mpo=None, shift=0.0):
    """bsmps_dot without device allocation (fixed 32 MiB scratch, see include/bsmps.h)."""
    out = C.c_double()
    _check(ctx, lib().bsmps_dot_noalloc(ctx.h, a.h, b.h, mpo.h if mpo is not None else None, shift,
                                        C.byref(out)))
    return out.value


def check_grid_wait(ctx, skip_cta=-1):
    """True when a grid-wide wait gave up (bsmps_check_grid_wait)."""
    out = C.c_int()
    _check(ctx, lib().bsmps_check_grid_wait(ctx.h, skip_cta, C.byref(out)))
    return bool(out.value)


def solver_params(c, delta, eps_num=None, t_eig=0.5, tau=1e-8, r_max=0, u_rel=1e-13):
    return SolverParams(c, delta, 0.5 * (1.0 - c) if eps_num is None else eps_num, t_eig, tau, r_max, u_rel)


def solver_state():
    return SolverState(math.inf, 0, 0, 0.0, 0)


def eigensolve_step(ctx, mpo, p, params, state, x):
    """One Alg. 2 step; returns (x_next, info dict).  x's handle is consumed."""
    h = _vp(x.h.value)
    info = StepInfo()
    code = lib().bsmps_eigensolve_step(ctx.h, mpo.h, C.byref(p), C.byref(params), C.byref(state), C.byref(h),
                                       C.byref(info))
    _check(ctx, code)
    x.h = None          # destroyed by the library
    return MPS(ctx, h), info.as_dict()


def eigensolve_outer(ctx, mpo, p, params, x, tau, alpha=1.0, max_outer=20, max_inner=100):
    """Alg. 3 from x (consumed); returns (y, records, converged)."""
    h = _vp(x.h.value)
    recs = (OuterRecord * max_outer)()
    n = C.c_int()
    ok = C.c_int()
    _check(ctx, lib().bsmps_eigensolve_outer(ctx.h, mpo.h, C.byref(p), C.byref(params), alpha, tau, max_outer,
                                             max_inner, C.byref(h), recs, C.byref(n), C.byref(ok)))
    x.h = None          # destroyed by the library
    return MPS(ctx, h), [recs[i].as_dict() for i in range(n.value)], bool(ok.value)


def gemm_tf32x3(ctx, A, B, C):
    """C = A B (row-major float64 device tensors) on the tensor cores in split
    precision (3xTF32, FP32 accumulation); stream-ordered on ctx's stream."""
    M, K = A.shape
    N = B.shape[1]
    _check(ctx, lib().bsmps_gemm_tf32x3(ctx.h, M, N, K, A.data_ptr(), A.stride(0), B.data_ptr(), B.stride(0),
                                        C.data_ptr(), C.stride(0)))
    return C


PREC_FP64, PREC_TF32X3 = 0, 1


def gemm_ozaki(ctx, A, B, C, slices=8):
    """C = A B (row-major float64 device tensors, e.g. torch CUDA tensors with
    data_ptr()), emulated on the tensor cores; stream-ordered on ctx's stream."""
    M, K = A.shape
    N = B.shape[1]
    _check(ctx, lib().bsmps_gemm_ozaki(ctx.h, M, N, K, A.data_ptr(), A.stride(0), B.data_ptr(), B.stride(0),
                                       C.data_ptr(), C.stride(0), slices))
    return C


def mps_joint_random_size(n_orb, spin, n_up, n_dn, r_max, D):
    n = C.c_int64()
    _check(None, lib().bsmps_mps_joint_random_size(n_orb, spin, n_up, n_dn, r_max, D, C.byref(n)))
    return n.value


def mps_create_joint(ctx, n_orb, spin, n_up, n_dn, D, occ=None, r_max=1, values=None):
    """Joint block MPS of D columns: the unit vectors of the occupation strings
    occ (D x K of 0/1) when given, else the random-rule iterate filled from values."""
    h = _vp()
    if occ is not None:
        o = np.ascontiguousarray(occ, dtype=np.uint8)
        assert o.shape[0] == D
        _check(ctx, lib().bsmps_mps_create_joint(ctx.h, n_orb, spin, n_up, n_dn, D, 0,
                                                  o.ctypes.data_as(C.POINTER(C.c_ubyte)), 0, None, 0, C.byref(h)))
    else:
        v = np.ascontiguousarray(values, dtype=np.float64)
        _check(ctx, lib().bsmps_mps_create_joint(ctx.h, n_orb, spin, n_up, n_dn, D, 1, None, r_max, _dptr(v),
                                                  len(v), C.byref(h)))
    return MPS(ctx, h)


def num_columns(x):
    d = C.c_int()
    _check(None, lib().bsmps_mps_num_columns(x.h, C.byref(d)))
    return d.value


def gram(ctx, a, b, mpo=None, shift=0.0):
    """The columns(a) x columns(b) matrix <a_i, O b_j>."""
    out = np.zeros((num_columns(a), num_columns(b)))
    _check(ctx, lib().bsmps_gram(ctx.h, a.h, b.h, mpo.h if mpo is not None else None, shift, _dptr(out)))
    return out


def apply_columns(ctx, mpo, x, col_shift, shift=0.0):
    """Exact (H_gamma + shift) X + X diag(col_shift)."""
    cs = np.ascontiguousarray(col_shift, dtype=np.float64)
    y = _vp()
    _check(ctx, lib().bsmps_apply_columns(ctx.h, mpo.h, x.h, shift, _dptr(cs), C.byref(y)))
    return MPS(ctx, y)


def mix_columns(ctx, x, Wm):
    """X Wm (Wm: columns(x) x D_out)."""
    w = np.ascontiguousarray(Wm, dtype=np.float64)
    y = _vp()
    _check(ctx, lib().bsmps_mix_columns(ctx.h, x.h, _dptr(w), w.shape[1], C.byref(y)))
    return MPS(ctx, y)


def eigensolve_joint_step(ctx, mpo, p, params, state, x):
    """One Alg. 4 step on a joint iterate; returns (X_next, info dict).  x's handle is consumed."""
    h = _vp(x.h.value)
    info = JointStepInfo()
    code = lib().bsmps_eigensolve_joint_step(ctx.h, mpo.h, C.byref(p), C.byref(params), C.byref(state),
                                             C.byref(h), C.byref(info))
    _check(ctx, code)
    x.h = None          # destroyed by the library
    return MPS(ctx, h), info.as_dict()


def _fptr(a):
    return a.ctypes.data_as(C.POINTER(C.c_float))


class MLP:
    """bsmps_mlp handle: BF16-weight MLP with FP32 accumulation and Adam training."""

    def __init__(self, ctx, widths, params):
        self.ctx = ctx
        self.widths = [int(w) for w in widths]
        w = np.ascontiguousarray(self.widths, dtype=np.int32)
        p = np.ascontiguousarray(params, dtype=np.float32)
        h = _vp()
        _check(ctx, lib().bsmps_mlp_create(ctx.h, len(w) - 1, _iptr(w), _fptr(p), len(p), C.byref(h)))
        self.h = h

    def __del__(self):
        try:
            if self.h:
                lib().bsmps_mlp_destroy(self.h)
                self.h = None
        except Exception:
            pass

    def n_params(self):
        n = C.c_int64()
        _check(self.ctx, lib().bsmps_mlp_num_params(self.h, C.byref(n)))
        return n.value

    def params(self):
        p = np.zeros(self.n_params(), dtype=np.float32)
        _check(self.ctx, lib().bsmps_mlp_get_params(self.h, _fptr(p)))
        return p

    def forward(self, x):
        x = np.ascontiguousarray(x, dtype=np.float32)
        y = np.zeros((x.shape[0], self.widths[-1]), dtype=np.float32)
        _check(self.ctx, lib().bsmps_mlp_forward(self.h, _fptr(x), x.shape[0], _fptr(y)))
        return y

    def loss_grad(self, x, t):
        x = np.ascontiguousarray(x, dtype=np.float32)
        t = np.ascontiguousarray(t, dtype=np.float32)
        g = np.zeros(self.n_params(), dtype=np.float32)
        loss = C.c_float()
        _check(self.ctx, lib().bsmps_mlp_loss_grad(self.h, _fptr(x), _fptr(t), x.shape[0], C.byref(loss), _fptr(g)))
        return loss.value, g

    def train_step(self, x, t, lr):
        x = np.ascontiguousarray(x, dtype=np.float32)
        t = np.ascontiguousarray(t, dtype=np.float32)
        loss = C.c_float()
        _check(self.ctx, lib().bsmps_mlp_train_step(self.h, _fptr(x), _fptr(t), x.shape[0], lr, C.byref(loss)))
        return loss.value
