"""Python binding of libfnocc: frozen-natural-orbital EOM-CCSDT on one GB300.

Argument marshalling only: every step runs in the CUDA library behind the C
ABI of include/fnocc.h. Importing this package fails loudly when the compiled
library is missing; there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libfnocc.so")

IP, EA, DIP, DEA, EE = 0, 1, 2, 3, 4
VARIANTS = {"ip": IP, "ea": EA, "dip": DIP, "dea": DEA, "ee": EE}
GUESS = {"koopmans": 0, "diagonal": 1, "learned": 2}
CRITERIA = {"abs": 0, "occt": 1}
PRECISION = {"fp64": 0, "mixed": 1, "mixed_tf32": 2}  # mixed: BF16 three-slice split
STATUS = {0: "OK", 1: "NOT_CONVERGED", -1: "E_INVALID", -2: "E_NOMEM", -3: "E_CUDA",
          -4: "E_STATE", -5: "E_NUMERIC", -6: "E_TIMEOUT"}
# (holes, particles) of R1, R2, R3 per variant
EOM_SPACES = {IP: [(1, 0), (2, 1), (3, 2)], EA: [(0, 1), (1, 2), (2, 3)],
              DIP: [(2, 0), (3, 1), (4, 2)], DEA: [(0, 2), (1, 3), (2, 4)]}


class FnoccError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s: %s" % (STATUS.get(status, status), msg))
        self.status = status


class FnoOptions(ctypes.Structure):
    _fields_ = [("criterion", ctypes.c_int), ("nkeep", ctypes.c_int), ("scf_maxiter", ctypes.c_int),
                ("scf_e_tol", ctypes.c_double), ("scf_comm_tol", ctypes.c_double)]


class FnoInfo(ctypes.Structure):
    _fields_ = [("e_rhf", ctypes.c_double), ("e_mp2", ctypes.c_double), ("nkept", ctypes.c_int),
                ("nvir", ctypes.c_int), ("kept_fraction", ctypes.c_double), ("scf_iters", ctypes.c_int)]


class CcsdtOptions(ctypes.Structure):
    _fields_ = [("tol_res", ctypes.c_double), ("tol_e", ctypes.c_double), ("maxiter", ctypes.c_int),
                ("diis", ctypes.c_int), ("precision", ctypes.c_int), ("switch_tol", ctypes.c_double)]


class CcsdtInfo(ctypes.Structure):
    _fields_ = [("e_corr", ctypes.c_double), ("e_tot", ctypes.c_double), ("iters", ctypes.c_int),
                ("res_max", ctypes.c_double), ("seconds", ctypes.c_double),
                ("seconds_per_iter", ctypes.c_double), ("iters_mixed", ctypes.c_int)]


class EomOptions(ctypes.Structure):
    _fields_ = [("tol_res", ctypes.c_double), ("tol_e", ctypes.c_double), ("max_sub", ctypes.c_int),
                ("maxiter", ctypes.c_int), ("nguess", ctypes.c_int), ("precision", ctypes.c_int),
                ("switch_tol", ctypes.c_double)]


class EomInfo(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int), ("sigma_calls", ctypes.c_int), ("seconds", ctypes.c_double),
                ("seconds_per_iter", ctypes.c_double), ("complex_roots", ctypes.c_int),
                ("res_max", ctypes.c_double), ("sigma_calls_mixed", ctypes.c_int), ("guess_used", ctypes.c_int)]


class System(ctypes.Structure):
    _fields_ = [("h", ctypes.POINTER(ctypes.c_double)), ("eri", ctypes.POINTER(ctypes.c_double)),
                ("n", ctypes.c_int), ("nocc", ctypes.c_int), ("occ_threshold", ctypes.c_double),
                ("nkeep", ctypes.c_int)]


class SystemResult(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("nkept", ctypes.c_int), ("e_rhf", ctypes.c_double),
                ("e_ccsdt", ctypes.c_double), ("ccsdt_iters", ctypes.c_int), ("sigma_calls", ctypes.c_int),
                ("seconds", ctypes.c_double), ("message", ctypes.c_char * 128)]


_dp = ctypes.POINTER(ctypes.c_double)
_fp = ctypes.POINTER(ctypes.c_float)
_vp = ctypes.c_void_p
_cp = ctypes.c_void_p

# exported symbol -> (restype, argtypes)
SIGNATURES = {
    "fnocc_create": (ctypes.c_int, [ctypes.POINTER(_cp), ctypes.c_int, _vp]),
    "fnocc_destroy": (None, [_cp]),
    "fnocc_last_error": (ctypes.c_char_p, [_cp]),
    "fnocc_launch_count": (ctypes.c_uint64, [_cp]),
    "fno_truncate": (ctypes.c_int, [_cp, _dp, _dp, ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                    ctypes.POINTER(FnoOptions), ctypes.POINTER(FnoInfo), _dp]),
    "fnocc_set_mo_hamiltonian": (ctypes.c_int, [_cp, _dp, _dp, ctypes.c_int, ctypes.c_int]),
    "ccsdt_solve": (ctypes.c_int, [_cp, ctypes.POINTER(CcsdtOptions), ctypes.POINTER(CcsdtInfo)]),
    "ccsdt_residual": (ctypes.c_int, [_cp, _dp, _dp, _dp, _dp, _dp, _dp, _dp]),
    "ccsdt_residual_dev": (ctypes.c_int, [_cp, _vp, _vp, _vp, _vp, _vp, _vp, _dp]),
    "eom_ccsdt_solve": (ctypes.c_int, [_cp, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                       ctypes.POINTER(EomOptions), _dp, _dp, ctypes.POINTER(EomInfo)]),
    "eom_ccsdt_solve_left": (ctypes.c_int, [_cp, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                       ctypes.POINTER(EomOptions), _dp, _dp, ctypes.POINTER(EomInfo)]),
    "eom_sigma": (ctypes.c_int, [_cp, ctypes.c_int, _dp, _dp]),
    "eom_sigma_dev": (ctypes.c_int, [_cp, ctypes.c_int, _vp, _vp]),
    "eom_left_sigma": (ctypes.c_int, [_cp, ctypes.c_int, _dp, _dp]),
    "eom_left_sigma_dev": (ctypes.c_int, [_cp, ctypes.c_int, _vp, _vp]),
    "fnocc_eom_sizes": (ctypes.c_int, [_cp, ctypes.c_int, ctypes.POINTER(ctypes.c_size_t)]),
    "fnocc_set_amplitudes": (ctypes.c_int, [_cp, _dp, _dp, _dp]),
    "fnocc_dims": (ctypes.c_int, [_cp, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int), _dp]),
    "fnocc_get_block": (ctypes.c_int, [_cp, ctypes.c_int, ctypes.c_int, _dp, ctypes.c_size_t]),
    "xfno_extrapolate": (ctypes.c_double, [_dp, _dp, ctypes.c_int]),
    "fno_truncate_dev": (ctypes.c_int, [_cp, _vp, _vp, ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                        ctypes.POINTER(FnoOptions), ctypes.POINTER(FnoInfo), _dp]),
    "fnocc_flop_count": (ctypes.c_double, [_cp]),
    "fnocc_set_precision": (ctypes.c_int, [_cp, ctypes.c_int]),
    "fnocc_set_tile_shape": (ctypes.c_int, [_cp, ctypes.c_int]),
    "fnocc_tile_shape_count": (ctypes.c_int, []),
    "fnocc_tile_shape_first_mixed": (ctypes.c_int, []),
    "fnocc_tile_shape_kind": (ctypes.c_int, [ctypes.c_int]),
    "fnocc_set_autotune": (ctypes.c_int, [ctypes.c_int]),
    "fnocc_set_graphs": (ctypes.c_int, [_cp, ctypes.c_int]),
    "fnocc_fp64_peak": (ctypes.c_int, [ctypes.c_int, _dp, _dp]),
    "fnocc_multi_dot": (ctypes.c_int, [_cp, _vp, _vp, ctypes.c_size_t, ctypes.c_size_t, ctypes.c_int, _vp]),
    "fnocc_multi_dot_noalloc": (ctypes.c_int, [_vp, _vp, ctypes.c_size_t, ctypes.c_size_t, ctypes.c_int, _vp, _vp]),
    "fnocc_equation_text": (ctypes.c_long, [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                            ctypes.c_char_p, ctypes.c_size_t]),
    "fnocc_plan_text": (ctypes.c_long, [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                        ctypes.c_int, ctypes.c_double, ctypes.c_char_p, ctypes.c_size_t]),
    "fnocc_profile": (ctypes.c_int, [_cp, ctypes.c_int]),
    "fnocc_plan_selfcheck": (ctypes.c_long, [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                             ctypes.c_int, ctypes.c_double]),
    "fnocc_plan_stats": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                        ctypes.c_int, ctypes.POINTER(ctypes.c_double)]),
    "fnocc_mlp_create": (ctypes.c_int, [ctypes.POINTER(_cp), ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                        ctypes.c_ulonglong]),
    "fnocc_mlp_destroy": (None, [_cp]),
    "fnocc_mlp_last_error": (ctypes.c_char_p, [_cp]),
    "fnocc_mlp_param_count": (ctypes.c_size_t, [_cp]),
    "fnocc_mlp_get_params": (ctypes.c_int, [_cp, _fp, ctypes.c_size_t]),
    "fnocc_mlp_set_params": (ctypes.c_int, [_cp, _fp, ctypes.c_size_t]),
    "fnocc_mlp_forward": (ctypes.c_int, [_cp, _fp, ctypes.c_longlong, _fp, ctypes.c_int]),
    "fnocc_mlp_loss_grad": (ctypes.c_int, [_cp, _fp, _fp, _fp, ctypes.c_longlong, _dp, _fp]),
    "fnocc_mlp_train": (ctypes.c_int, [_cp, _fp, _fp, _fp, ctypes.c_longlong, ctypes.c_int, ctypes.c_int,
                                       ctypes.c_float, ctypes.c_ulonglong, _dp]),
    "fnocc_mlp_save": (ctypes.c_int, [_cp, ctypes.c_char_p]),
    "fnocc_mlp_load": (ctypes.c_int, [_cp, ctypes.c_char_p]),
    "fnocc_eom_features": (ctypes.c_int, [_cp, ctypes.c_int, _fp]),
    "fnocc_eom_diagonal": (ctypes.c_int, [_cp, ctypes.c_int, _dp]),
    "fnocc_eom_diagonal_at": (ctypes.c_int, [_cp, ctypes.c_int, ctypes.c_longlong,
                                             ctypes.POINTER(ctypes.c_longlong), _dp]),
    "fnocc_set_guess_model": (ctypes.c_int, [_cp, _cp]),
    "fnocc_batch_solve": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.POINTER(System), ctypes.c_int,
                                         ctypes.POINTER(ctypes.c_int), ctypes.c_int,
                                         ctypes.POINTER(CcsdtOptions), ctypes.POINTER(EomOptions), ctypes.c_int,
                                         _dp, ctypes.POINTER(SystemResult)]),
    "fnocc_profile_read": (ctypes.c_int, [_cp, ctypes.c_int, _dp, _dp, ctypes.POINTER(ctypes.c_uint64)]),
}

_lib = None


def load_library(path=LIB_PATH):
    """Loads libfnocc.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError("libfnocc.so not built: run `python -c 'import __graft_entry__ as g; g.build()'`")
    lib = ctypes.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _arr(x):
    a = np.ascontiguousarray(x, dtype=np.float64)
    return a, a.ctypes.data_as(_dp)


def xfno_extrapolate(kept_fraction, energy):
    """XFNO extrapolation (Sec. 2): least-squares line E(f) at f = 1 (xfno_extrapolate)."""
    lib = load_library()
    f, fp = _arr(kept_fraction)
    e, ep = _arr(energy)
    return float(lib.xfno_extrapolate(fp, ep, len(f)))


def batch_solve(systems, variants, nroots, device=0, nworkers=4, cc_tol_res=1e-10, cc_tol_e=1e-12,
                eom_tol_res=1e-8, eom_tol_e=1e-10, precision="fp64"):
    """Independent systems through the whole path, nworkers at a time (one
    context and stream each); see fnocc_batch_solve.

    systems: list of dicts with h, eri, nocc and threshold or nkeep.
    Returns (omegas[nsys, len(variants), nroots], list of per-system dicts);
    a system that failed carries its status in its dict."""
    lib = load_library()
    keep = []
    arr = (System * len(systems))()
    for i, sy in enumerate(systems):
        h, hp = _arr(sy["h"])
        e, ep = _arr(sy["eri"])
        keep += [h, e]
        arr[i] = System(hp, ep, h.shape[0], int(sy["nocc"]), float(sy.get("threshold", 0.0)),
                        int(sy.get("nkeep", 0)))
    vs = [VARIANTS.get(v, v) for v in variants]
    var = (ctypes.c_int * len(vs))(*vs)
    cc = CcsdtOptions(cc_tol_res, cc_tol_e, 200, 8, PRECISION[precision], 1e-6)
    eo = EomOptions(eom_tol_res, eom_tol_e, 0, 200, 0, PRECISION[precision], 1e-5)
    om = np.zeros((len(systems), len(vs), nroots))
    res = (SystemResult * len(systems))()
    st = lib.fnocc_batch_solve(int(device), len(systems), arr, len(vs), var, int(nroots), ctypes.byref(cc),
                               ctypes.byref(eo), int(nworkers), om.ctypes.data_as(_dp), res)
    if st == -1:
        raise FnoccError(st, "invalid batch request")
    out = [dict(status=r.status, nkept=r.nkept, e_rhf=r.e_rhf, e_ccsdt=r.e_ccsdt, ccsdt_iters=r.ccsdt_iters,
                sigma_calls=r.sigma_calls, seconds=r.seconds, message=r.message.decode(errors="replace"))
           for r in res]
    return om, out


def tile_shapes():
    """(number of tile shapes, index of the first split-product shape)."""
    lib = load_library()
    return int(lib.fnocc_tile_shape_count()), int(lib.fnocc_tile_shape_first_mixed())


def tile_shape_kind(shape):
    """0 FP64, 1 split product on mma.sync, 2 BF16x3 on tcgen05 (-1 out of range)."""
    return int(load_library().fnocc_tile_shape_kind(int(shape)))


def fp64_peak(device=0):
    """Measured FP64 throughput of the device in TFLOP/s: (FMA, mma.sync m8n8k4)."""
    lib = load_library()
    a, b = ctypes.c_double(), ctypes.c_double()
    st = lib.fnocc_fp64_peak(int(device), ctypes.byref(a), ctypes.byref(b))
    if st != 0:
        raise FnoccError(st, "fnocc_fp64_peak failed")
    return a.value, b.value


def set_autotune(enable):
    """Process-wide switch of the FP64 tile-shape timing (fnocc_set_autotune)."""
    load_library().fnocc_set_autotune(1 if enable else 0)


def equation_text(kind, variant=0, out_comp=0, in_comp=0):
    """Term list the library derived (host only); see fnocc_equation_text."""
    lib = load_library()
    var = VARIANTS.get(variant, variant)
    n = lib.fnocc_equation_text(kind, var, out_comp, in_comp, None, 0)
    if n < 0:
        raise ValueError("bad equation request")
    buf = ctypes.create_string_buffer(n + 1)
    lib.fnocc_equation_text(kind, var, out_comp, in_comp, buf, n + 1)
    return buf.value.decode()


def plan_selfcheck(kind, variant=0, out_comp=0, in_comp=0, o=4, v=6, max_work=2e6):
    """Inconsistencies of the executable plan's grouped tasks against its
    spin blocks (host only); see fnocc_plan_selfcheck."""
    lib = load_library()
    return int(lib.fnocc_plan_selfcheck(kind, VARIANTS.get(variant, variant), out_comp, in_comp, o, v, max_work))


def plan_stats(kind, variant=0, out_comp=0, in_comp=0, o=10, v=30):
    """Host-only plan statistics (fnocc_plan_stats) as a dict."""
    lib = load_library()
    out = (ctypes.c_double * 10)()
    st = lib.fnocc_plan_stats(kind, VARIANTS.get(variant, variant), out_comp, in_comp, o, v, out)
    if st != 0:
        raise ValueError("bad plan request")
    keys = ("grouped_steps", "grouped_flops", "padded_flops", "model_seconds", "small_launch_steps",
            "small_launch_flops", "other_steps", "other_flops", "scratch_doubles", "cache_doubles")
    return dict(zip(keys, list(out)))


def plan_text(kind, variant=0, out_comp=0, in_comp=0, o=10, v=30, amortize=0.0):
    """Contraction plan the library builds (host only); see fnocc_plan_text."""
    lib = load_library()
    var = VARIANTS.get(variant, variant)
    n = lib.fnocc_plan_text(kind, var, out_comp, in_comp, o, v, amortize, None, 0)
    if n < 0:
        raise ValueError("bad plan request")
    buf = ctypes.create_string_buffer(n + 1)
    lib.fnocc_plan_text(kind, var, out_comp, in_comp, o, v, amortize, buf, n + 1)
    return buf.value.decode()


def _farr(x, cols=None):
    a = np.ascontiguousarray(x, dtype=np.float32)
    if cols is not None and (a.ndim != 2 or a.shape[1] != cols):
        raise ValueError("expected an array of shape (n, %d)" % cols)
    return a, a.ctypes.data_as(_fp)


class Mlp:
    """Per-amplitude guess network (8 features -> width -> width -> 2) whose
    training and inference run in the library's kernels; see fnocc_mlp_*."""
    NIN, NOUT = 8, 2

    def __init__(self, device=0, width=256, seed=0):
        self.lib = load_library()
        self._h = _cp()
        st = self.lib.fnocc_mlp_create(ctypes.byref(self._h), int(device), self.NIN, int(width), self.NOUT,
                                       int(seed))
        if st != 0:
            raise FnoccError(st, "fnocc_mlp_create failed")
        self.width = width

    def close(self):
        """Releases the network's device memory."""
        if self._h:
            self.lib.fnocc_mlp_destroy(self._h)
            self._h = _cp()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, st):
        if st != 0:
            msg = self.lib.fnocc_mlp_last_error(self._h)
            raise FnoccError(st, msg.decode() if msg else "")

    @property
    def nparam(self):
        """Number of FP32 parameters (fnocc_mlp_param_count)."""
        return int(self.lib.fnocc_mlp_param_count(self._h))

    def get_params(self):
        """Parameters as a host FP32 array (get_params layout)."""
        p = np.zeros(self.nparam, dtype=np.float32)
        self._check(self.lib.fnocc_mlp_get_params(self._h, p.ctypes.data_as(_fp), p.size))
        return p

    def set_params(self, p):
        """Sets the parameters and resets the optimiser state."""
        p, pp = _farr(p)
        self._check(self.lib.fnocc_mlp_set_params(self._h, pp, p.size))

    def forward(self, x, bf16=False):
        """Network outputs [n x 2] for features [n x 8]; bf16=True: the tensor-core inference path."""
        x, xp = _farr(x, self.NIN)
        y = np.zeros((x.shape[0], self.NOUT), dtype=np.float32)
        self._check(self.lib.fnocc_mlp_forward(self._h, xp, x.shape[0], y.ctypes.data_as(_fp), 1 if bf16 else 0))
        return y

    def loss_grad(self, x, t, w):
        """Weighted mean-squared loss and its gradient at the current parameters."""
        x, xp = _farr(x, self.NIN)
        t, tp = _farr(t, self.NOUT)
        w, wp = _farr(w, self.NOUT)
        loss = ctypes.c_double()
        g = np.zeros(self.nparam, dtype=np.float32)
        self._check(self.lib.fnocc_mlp_loss_grad(self._h, xp, tp, wp, x.shape[0], ctypes.byref(loss),
                                                 g.ctypes.data_as(_fp)))
        return loss.value, g

    def train(self, x, t, w, epochs=20, batch=4096, lr=1e-3, seed=0):
        """Minibatch Adam on the library's kernels; returns the mean loss per epoch."""
        x, xp = _farr(x, self.NIN)
        t, tp = _farr(t, self.NOUT)
        w, wp = _farr(w, self.NOUT)
        hist = np.zeros(max(epochs, 1))
        self._check(self.lib.fnocc_mlp_train(self._h, xp, tp, wp, x.shape[0], int(epochs), int(batch),
                                             float(lr), int(seed), hist.ctypes.data_as(_dp)))
        return hist[:epochs]

    def save(self, path):
        """Write the parameters to a file (fnocc_mlp_save)."""
        self._check(self.lib.fnocc_mlp_save(self._h, os.fsencode(path)))

    def load(self, path):
        """Read parameters written by save() for a network of this shape."""
        self._check(self.lib.fnocc_mlp_load(self._h, os.fsencode(path)))


class Context:
    """One library context (device memory, stream, loaded Hamiltonian)."""

    def __init__(self, device=0, stream=None):
        self.lib = load_library()
        self._h = _cp()
        st = self.lib.fnocc_create(ctypes.byref(self._h), int(device), stream)
        if st != 0:
            raise FnoccError(st, "fnocc_create failed")

    def close(self):
        """Destroys the context and frees its device memory."""
        if self._h:
            self.lib.fnocc_destroy(self._h)
            self._h = _cp()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, st, allow=(0,)):
        if st not in allow:
            msg = self.lib.fnocc_last_error(self._h)
            raise FnoccError(st, msg.decode() if msg else "")
        return st

    @property
    def launches(self):
        """Kernel launches issued so far (fnocc_launch_count)."""
        return int(self.lib.fnocc_launch_count(self._h))

    def dims(self):
        """(o, v, E_ref): active occupied / virtual spin orbitals and the reference energy."""
        o, v, e = ctypes.c_int(), ctypes.c_int(), ctypes.c_double()
        self._check(self.lib.fnocc_dims(self._h, ctypes.byref(o), ctypes.byref(v), ctypes.byref(e)))
        return o.value, v.value, e.value

    def fno_truncate(self, h, eri, nocc, threshold, criterion="abs", nkeep=0):
        """RHF, MP2 natural orbitals, truncation and the active Hamiltonian (Sec. 1.2, Eq. 8-10)."""
        h, hp = _arr(h)
        eri, ep = _arr(eri)
        n = h.shape[0]
        opt = FnoOptions(CRITERIA[criterion], int(nkeep), 200, 1e-12, 1e-10)
        info = FnoInfo()
        occ = np.zeros(n - nocc)
        self._check(self.lib.fno_truncate(self._h, hp, ep, n, int(nocc), float(threshold), ctypes.byref(opt),
                                          ctypes.byref(info), occ.ctypes.data_as(_dp)))
        return dict(e_rhf=info.e_rhf, e_mp2=info.e_mp2, nkept=info.nkept, nvir=info.nvir,
                    kept_fraction=info.kept_fraction, scf_iters=info.scf_iters, occ=occ)

    def fno_truncate_dev(self, h_ptr, eri_ptr, n, nocc, threshold, criterion="abs", nkeep=0):
        """h_ptr, eri_ptr: device addresses (e.g. torch tensor data_ptr())."""
        opt = FnoOptions(CRITERIA[criterion], int(nkeep), 200, 1e-12, 1e-10)
        info = FnoInfo()
        occ = np.zeros(n - nocc)
        self._check(self.lib.fno_truncate_dev(self._h, h_ptr, eri_ptr, int(n), int(nocc), float(threshold),
                                              ctypes.byref(opt), ctypes.byref(info), occ.ctypes.data_as(_dp)))
        return dict(e_rhf=info.e_rhf, e_mp2=info.e_mp2, nkept=info.nkept, nvir=info.nvir,
                    kept_fraction=info.kept_fraction, scf_iters=info.scf_iters, occ=occ)

    def set_precision(self, precision):
        """Arithmetic of standalone residual / sigma calls: 'fp64', 'mixed'
        (BF16 three-slice split products) or 'mixed_tf32' (TF32 two-slice)."""
        self._check(self.lib.fnocc_set_precision(self._h, PRECISION[precision]))

    def set_graphs(self, enable):
        """Graph replay of the EOM products' launch sequences (fnocc_set_graphs)."""
        self._check(self.lib.fnocc_set_graphs(self._h, 1 if enable else 0))

    def set_tile_shape(self, shape):
        """Forces one grouped-GEMM tile shape (-1: the library's choice)."""
        self._check(self.lib.fnocc_set_tile_shape(self._h, int(shape)))

    @property
    def flops(self):
        """Algorithmic flops of the contraction steps run so far (fnocc_flop_count)."""
        return float(self.lib.fnocc_flop_count(self._h))

    def profile(self, enable=True):
        """Per-launch event timing of the contraction kernels on / off (fnocc_profile)."""
        self._check(self.lib.fnocc_profile(self._h, 1 if enable else 0))

    PROFILE_PATHS = {0: "k_ggemm", 1: "k_ggemm_split+k_greduce", 2: "k_gemm_small+k_reduce_partials",
                     3: "k_gemv_rows", 4: "k_ggemm_bf16x3", 5: "k_ggemm_bf16x3_split+k_greduce",
                     6: "k_ggemm_tf32x3", 7: "k_ggemm_tf32x3_split+k_greduce",
                     8: "k_ggemm_tc", 9: "k_ggemm_tc_split+k_greduce",
                     10: "k_tc_pack+k_ggemm_tcp", 11: "k_tc_pack+k_ggemm_tcp_split+k_greduce"}

    def profile_read(self, path=-1):
        """(device ms, algorithmic flops, launches) of one contraction kernel path
        (see PROFILE_PATHS) or of all (-1) since the last read of that path."""
        ms, fl, n = ctypes.c_double(), ctypes.c_double(), ctypes.c_uint64()
        self._check(self.lib.fnocc_profile_read(self._h, int(path), ctypes.byref(ms), ctypes.byref(fl),
                                                ctypes.byref(n)))
        return ms.value, fl.value, int(n.value)

    def set_mo_hamiltonian(self, h_mo, eri_mo, nocc):
        """Loads an MO-basis Hamiltonian directly (no RHF or FNO step)."""
        h, hp = _arr(h_mo)
        e, ep = _arr(eri_mo)
        self._check(self.lib.fnocc_set_mo_hamiltonian(self._h, hp, ep, h.shape[0], int(nocc)))

    def ccsdt_solve(self, tol_res=1e-10, tol_e=1e-12, maxiter=200, diis=8, precision="fp64", switch_tol=1e-6):
        """CCSDT ground state (Eq. 5-7) by Jacobi + DIIS iterations."""
        opt = CcsdtOptions(tol_res, tol_e, maxiter, diis, PRECISION[precision], switch_tol)
        info = CcsdtInfo()
        st = self._check(self.lib.ccsdt_solve(self._h, ctypes.byref(opt), ctypes.byref(info)), allow=(0, 1))
        return dict(e_corr=info.e_corr, e_tot=info.e_tot, iters=info.iters, res_max=info.res_max,
                    seconds=info.seconds, seconds_per_iter=info.seconds_per_iter, converged=(st == 0),
                    iters_mixed=info.iters_mixed)

    def amp_sizes(self):
        """Packed sizes of T1, T2, T3."""
        from math import comb
        o, v, _ = self.dims()
        return [comb(o, r) * comb(v, r) for r in (1, 2, 3)]

    def ccsdt_residual(self, t1, t2, t3):
        """CCSDT residuals (Eq. 6) and energy of packed host amplitudes."""
        sizes = self.amp_sizes()
        ins = [_arr(t) for t in (t1, t2, t3)]
        outs = [np.zeros(s) for s in sizes]
        e = ctypes.c_double()
        self._check(self.lib.ccsdt_residual(self._h, ins[0][1], ins[1][1], ins[2][1],
                                            *[o_.ctypes.data_as(_dp) for o_ in outs], ctypes.byref(e)))
        return outs, e.value

    def ccsdt_residual_dev(self, t1_ptr, t2_ptr, t3_ptr, r1_ptr, r2_ptr, r3_ptr):
        """ccsdt_residual on device pointers."""
        e = ctypes.c_double()
        self._check(self.lib.ccsdt_residual_dev(self._h, t1_ptr, t2_ptr, t3_ptr, r1_ptr, r2_ptr, r3_ptr,
                                                ctypes.byref(e)))
        return e.value

    def set_amplitudes(self, t1, t2, t3):
        """Stores ground-state amplitudes (packed, host) for the EOM products."""
        ins = [_arr(t) for t in (t1, t2, t3)]
        self._check(self.lib.fnocc_set_amplitudes(self._h, ins[0][1], ins[1][1], ins[2][1]))

    def multi_dot_dev(self, x_ptr, y_ptr, n, ld, nvec, dots_ptr):
        """dots[j] = x . Y[j] on the device (all device addresses)."""
        self._check(self.lib.fnocc_multi_dot(self._h, x_ptr, y_ptr, int(n), int(ld), int(nvec), dots_ptr))

    def eom_sizes(self, variant):
        """Packed sizes of the variant's three EOM components."""
        sz = (ctypes.c_size_t * 3)()
        self._check(self.lib.fnocc_eom_sizes(self._h, VARIANTS.get(variant, variant), sz))
        return [int(x) for x in sz]

    def eom_sigma(self, variant, r):
        """sigma = (H-bar R)_c of a packed host vector (Eq. 1-4)."""
        var = VARIANTS.get(variant, variant)
        r, rp = _arr(r)
        s = np.zeros_like(r)
        self._check(self.lib.eom_sigma(self._h, var, rp, s.ctypes.data_as(_dp)))
        return s

    def eom_sigma_dev(self, variant, r_ptr, s_ptr):
        """eom_sigma on device pointers."""
        self._check(self.lib.eom_sigma_dev(self._h, VARIANTS.get(variant, variant), r_ptr, s_ptr))

    def eom_left_sigma_dev(self, variant, l_ptr, lam_ptr):
        """eom_left_sigma on device pointers."""
        self._check(self.lib.eom_left_sigma_dev(self._h, VARIANTS.get(variant, variant), l_ptr, lam_ptr))

    def eom_left_sigma(self, variant, lvec):
        """lambda = L^T H-bar (eom_left_sigma)."""
        var = VARIANTS.get(variant, variant)
        lvec, lp = _arr(lvec)
        out = np.zeros_like(lvec)
        self._check(self.lib.eom_left_sigma(self._h, var, lp, out.ctypes.data_as(_dp)))
        return out

    def eom_solve(self, variant, nroots, guess="koopmans", tol_res=1e-8, tol_e=1e-10, max_sub=0,
                  maxiter=200, nguess=0, precision="fp64", switch_tol=1e-5, left=False):
        """Lowest roots (eom_ccsdt_solve); left=True solves for the left
        eigenvectors with the left product (eom_ccsdt_solve_left)."""
        var = VARIANTS.get(variant, variant)
        self._last_sizes = self.eom_sizes(var)
        opt = EomOptions(tol_res, tol_e, max_sub, maxiter, nguess, PRECISION[precision], switch_tol)
        info = EomInfo()
        en = np.zeros(nroots)
        om = np.zeros(nroots)
        solve = self.lib.eom_ccsdt_solve_left if left else self.lib.eom_ccsdt_solve
        st = self._check(solve(self._h, var, int(nroots), GUESS[guess], ctypes.byref(opt),
                               en.ctypes.data_as(_dp), om.ctypes.data_as(_dp), ctypes.byref(info)), allow=(0, 1))
        return dict(energies=en, omegas=om, iters=info.iters, sigma_calls=info.sigma_calls,
                    seconds=info.seconds, seconds_per_iter=info.seconds_per_iter,
                    complex_roots=info.complex_roots, res_max=info.res_max, converged=(st == 0),
                    sigma_calls_mixed=info.sigma_calls_mixed, guess_used=info.guess_used)

    def eom_features(self, variant):
        """Per-element features [dim x 8] of the learned guess."""
        var = VARIANTS.get(variant, variant)
        dim = sum(self.eom_sizes(var))
        f = np.zeros((dim, Mlp.NIN), dtype=np.float32)
        self._check(self.lib.fnocc_eom_features(self._h, var, f.ctypes.data_as(_fp)))
        return f

    def eom_diagonal(self, variant, idx=None):
        """Exact H-bar diagonal of the sector's elements (one product each),
        or with idx only at those packed indices (fnocc_eom_diagonal_at)."""
        var = VARIANTS.get(variant, variant)
        if idx is None:
            d = np.zeros(sum(self.eom_sizes(var)))
            self._check(self.lib.fnocc_eom_diagonal(self._h, var, d.ctypes.data_as(_dp)))
            return d
        ix = np.ascontiguousarray(idx, dtype=np.int64)
        d = np.zeros(ix.shape[0])
        self._check(self.lib.fnocc_eom_diagonal_at(self._h, var, ix.shape[0],
                                                   ix.ctypes.data_as(ctypes.POINTER(ctypes.c_longlong)),
                                                   d.ctypes.data_as(_dp)))
        return d

    def set_guess_model(self, mlp):
        """Attaches the network FNOCC_GUESS_LEARNED uses (None detaches)."""
        self._guess_model = mlp  # keep the network alive while attached
        self._check(self.lib.fnocc_set_guess_model(self._h, mlp._h if mlp is not None else None))

    def get_block(self, which, root=0):
        """which: 't1','t2','t3' or ('r', k) for component k=1..3 of EOM root `root`."""
        if isinstance(which, str):
            k = int(which[1])
            size = self.amp_sizes()[k - 1]
            code = k
        else:
            k = which[1]
            var_sizes = self._last_sizes
            size = var_sizes[k - 1]
            code = 10 + k
        buf = np.zeros(size)
        self._check(self.lib.fnocc_get_block(self._h, code, int(root), buf.ctypes.data_as(_dp), size))
        return buf
