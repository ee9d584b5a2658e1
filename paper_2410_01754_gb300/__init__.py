"""Python binding of libmahi (MAHI on GB300, sm_103a).

Argument marshalling only: every step of the evaluation runs in the CUDA
kernels of ``libmahi.so``.  Device buffers come from torch tensors (their
``data_ptr()``), streams from ``torch.cuda.Stream.cuda_stream``.  There is no
CPU path: if the library is missing the import of a compute entry point
raises.  Function names follow ``include/mahi.h``.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libmahi.so")

MAHI_FP64, MAHI_MIXED, MAHI_MIXED_SIMT = 0, 1, 2
MAHI_ERR_TIMEOUT, MAHI_ERR_SITE_OVERFLOW = -5, -8
OPTIONS = {"site_theta": 1, "site_list_cap": 2, "wait_limit_ms": 3, "watchdog_selftest": 4,
           "m2l_split_degree": 5, "m2l_single_tile": 6, "m2l_b_stages": 7, "p2p_threads": 8, "site_blocks": 9,
           "p2p_targets": 10}
PRECISIONS = {"fp64": MAHI_FP64, "mixed": MAHI_MIXED, "mixed_simt": MAHI_MIXED_SIMT}

_lib = None

_SIGS = {
    "mahi_create": (ctypes.c_int, [ctypes.c_double, ctypes.c_int64, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                   ctypes.c_int32, ctypes.c_void_p, ctypes.POINTER(ctypes.c_void_p)]),
    "mahi_destroy": (ctypes.c_int, [ctypes.c_void_p]),
    "mahi_set_stream": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    "mahi_set_charges": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "mahi_eval": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p,
                                 ctypes.c_void_p, ctypes.c_void_p]),
    "mahi_eval_host": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p,
                                      ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "mahi_get_potential": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    "mahi_backward": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                     ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p,
                                     ctypes.c_void_p, ctypes.c_void_p]),
    "mahi_backward_forms": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                           ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p,
                                           ctypes.c_void_p, ctypes.c_void_p]),
    "mahi_set_timing": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32]),
    "mahi_stage_times": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_float), ctypes.c_int32]),
    "mahi_stage_name": (ctypes.c_char_p, [ctypes.c_int32]),
    "mahi_launch_count": (ctypes.c_int, [ctypes.c_void_p]),
    "mahi_lattice_coeffs": (ctypes.c_int, [ctypes.c_int32, ctypes.c_int32, ctypes.c_void_p]),
    "mahi_lattice_eval": (ctypes.c_int, [ctypes.c_double, ctypes.c_int32, ctypes.c_int32, ctypes.c_int64,
                                         ctypes.c_void_p, ctypes.c_void_p]),
    "mahi_site_terms_static": (ctypes.c_int, [ctypes.c_double, ctypes.c_int64, ctypes.c_int32, ctypes.c_void_p,
                                              ctypes.c_void_p,
                                              ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p,
                                              ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                              ctypes.c_void_p, ctypes.c_void_p]),
    "mahi_get_status": (ctypes.c_int, [ctypes.c_void_p]),
    "mahi_update_charges": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "mahi_set_option": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_double]),
    "mahi_get_option": (ctypes.c_double, [ctypes.c_void_p, ctypes.c_int32]),
    "mahi_batch_create": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p,
                                         ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                         ctypes.c_void_p, ctypes.POINTER(ctypes.c_void_p)]),
    "mahi_batch_launch": (ctypes.c_int, [ctypes.c_void_p]),
    "mahi_batch_destroy": (ctypes.c_int, [ctypes.c_void_p]),
    "mahi_autotune": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p,
                                     ctypes.c_int32]),
    "mahi_get_tuning": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_int32),
                                       ctypes.POINTER(ctypes.c_int32)]),
    "mahi_set_forms": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                      ctypes.c_void_p]),
    "mahi_n_lambdas": (ctypes.c_int, [ctypes.c_void_p]),
    "mahi_coulomb_constant": (ctypes.c_double, []),
    "mahi_error_string": (ctypes.c_char_p, [ctypes.c_int]),
    "mahi_last_cuda_error": (ctypes.c_char_p, []),
}


class MahiError(RuntimeError):
    def __init__(self, code, where=""):
        msg = lib().mahi_error_string(code).decode()
        if code == -4:
            msg += ": " + lib().mahi_last_cuda_error().decode()
        super().__init__(f"{where}: {msg} ({code})")
        self.code = code


def lib():
    """Load libmahi.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"libmahi.so not built ({LIB_PATH}); run paper_2410_01754_gb300/build.py")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _ck(code, where):
    if code != 0:
        raise MahiError(code, where)


def _ptr(t):
    if t is None:
        return None
    if isinstance(t, np.ndarray):
        return t.ctypes.data
    return t.data_ptr()


def _stream_handle(stream):
    if stream is None:
        return None
    return getattr(stream, "cuda_stream", stream)


def mahi_create(box_L_nm, n_atoms, n_sites, order_p, depth, precision=MAHI_FP64, stream=None):
    if isinstance(precision, str):
        precision = PRECISIONS[precision]
    h = ctypes.c_void_p()
    _ck(lib().mahi_create(float(box_L_nm), int(n_atoms), int(n_sites), int(order_p), int(depth), int(precision),
                          _stream_handle(stream), ctypes.byref(h)), "mahi_create")
    return h


def mahi_destroy(h):
    _ck(lib().mahi_destroy(h), "mahi_destroy")


def mahi_set_stream(h, stream):
    _ck(lib().mahi_set_stream(h, _stream_handle(stream)), "mahi_set_stream")


def _host_or_device(a, dtype):
    """numpy arrays are passed as host memory, contiguous CUDA tensors by pointer."""
    if hasattr(a, "data_ptr") and getattr(a, "is_cuda", False):
        want = "torch.float64" if dtype == np.float64 else "torch.int32"
        if str(a.dtype) != want or not a.is_contiguous():
            raise TypeError(f"device array must be a contiguous {want} tensor")
        return a, a.data_ptr()
    arr = np.ascontiguousarray(a, dtype=dtype)
    return arr, arr.ctypes.data


def mahi_set_charges(h, qA, qB, site_of_atom):
    """qA, qB (float64) and site_of_atom (int32): numpy arrays or CUDA tensors."""
    ka, pa = _host_or_device(qA, np.float64)
    kb, pb = _host_or_device(qB, np.float64)
    ks, ps = _host_or_device(site_of_atom, np.int32)
    _ck(lib().mahi_set_charges(h, pa, pb, ps), "mahi_set_charges")


def mahi_update_charges(h, qA, qB):
    """New charges (contiguous float64 CUDA tensors) for the same site map; enqueued."""
    _ck(lib().mahi_update_charges(h, _ptr(qA), _ptr(qB)), "mahi_update_charges")


def mahi_get_status(h):
    """Synchronises the handle's stream; returns 0 or the code of a device-side failure."""
    return int(lib().mahi_get_status(h))


def mahi_set_option(h, option, value):
    opt = OPTIONS[option] if isinstance(option, str) else int(option)
    _ck(lib().mahi_set_option(h, opt, float(value)), "mahi_set_option")


def mahi_get_option(h, option):
    opt = OPTIONS[option] if isinstance(option, str) else int(option)
    return float(lib().mahi_get_option(h, opt))


def mahi_set_forms(h, q_env, site_of_atom, forms):
    """forms: list over sites of (F_s, n_s) arrays (charges of the site's atoms,
    in increasing atom index, in each of its F_s = 2^m forms)."""
    q_env = np.ascontiguousarray(q_env, dtype=np.float64)
    so = np.ascontiguousarray(site_of_atom, dtype=np.int32)
    nf = np.ascontiguousarray([np.asarray(f).shape[0] for f in forms], dtype=np.int32)
    qf = np.ascontiguousarray(np.concatenate([np.asarray(f, dtype=np.float64).ravel() for f in forms])
                              if len(forms) else np.zeros(1))
    _ck(lib().mahi_set_forms(h, q_env.ctypes.data, so.ctypes.data, nf.ctypes.data, qf.ctypes.data), "mahi_set_forms")


def mahi_n_lambdas(h):
    return int(lib().mahi_n_lambdas(h))


def mahi_eval(h, x, lam, energy=None, forces=None, dEdlambda=None):
    """x, lam, energy, forces, dEdlambda: CUDA tensors (x float32/float64 N x 3)."""
    x_is_fp64 = 1 if str(x.dtype).endswith("float64") else 0
    _ck(lib().mahi_eval(h, _ptr(x), x_is_fp64, _ptr(lam), _ptr(energy), _ptr(forces), _ptr(dEdlambda)),
        "mahi_eval")


def mahi_eval_host(h, x, lam, energy=None, forces=None, dEdlambda=None):
    """Host numpy buffers (pinned or pageable); copies happen inside the call."""
    x_is_fp64 = 1 if x.dtype == np.float64 else 0
    _ck(lib().mahi_eval_host(h, _ptr(x), x_is_fp64, _ptr(lam), _ptr(energy), _ptr(forces), _ptr(dEdlambda)),
        "mahi_eval_host")


def mahi_get_potential(h, phi):
    _ck(lib().mahi_get_potential(h, _ptr(phi)), "mahi_get_potential")


def mahi_backward(h, grad_energy, forces, dEdlambda, lam, dx=None, dlambda=None, dEdqA=None, dEdqB=None):
    """Backward of the last mahi_eval (device tensors; outputs may be None)."""
    ref = forces if forces is not None else dx
    x_is_fp64 = 1 if ref is not None and str(ref.dtype).endswith("float64") else 0
    _ck(lib().mahi_backward(h, _ptr(grad_energy), _ptr(forces), _ptr(dEdlambda), _ptr(lam), x_is_fp64, _ptr(dx),
                            _ptr(dlambda), _ptr(dEdqA), _ptr(dEdqB)), "mahi_backward")


def mahi_backward_forms(h, grad_energy, forces, dEdlambda, lam, dx=None, dlambda=None, dEdq_env=None,
                        dEdq_forms=None):
    """Backward of the last mahi_eval on a handle with 2^m-form sites (device tensors)."""
    ref = forces if forces is not None else dx
    x_is_fp64 = 1 if ref is not None and str(ref.dtype).endswith("float64") else 0
    _ck(lib().mahi_backward_forms(h, _ptr(grad_energy), _ptr(forces), _ptr(dEdlambda), _ptr(lam), x_is_fp64,
                                  _ptr(dx), _ptr(dlambda), _ptr(dEdq_env), _ptr(dEdq_forms)), "mahi_backward_forms")


def mahi_set_timing(h, on=True):
    _ck(lib().mahi_set_timing(h, 1 if on else 0), "mahi_set_timing")


def mahi_stage_times(h):
    buf = (ctypes.c_float * 32)()
    n = lib().mahi_stage_times(h, buf, 32)
    if n < 0:
        raise MahiError(n, "mahi_stage_times")
    return {lib().mahi_stage_name(i).decode(): float(buf[i]) for i in range(n)}


def mahi_launch_count(h):
    return int(lib().mahi_launch_count(h))


def mahi_lattice_coeffs(order_p, shell=1):
    out = np.zeros((2 * order_p + 1) ** 2)
    _ck(lib().mahi_lattice_coeffs(int(order_p), int(shell), out.ctypes.data), "mahi_lattice_coeffs")
    return out


def mahi_lattice_eval(box_L_nm, order_p, r, shell=1):
    r = np.ascontiguousarray(r, dtype=np.float64).reshape(-1, 3)
    out = np.zeros(r.shape[0])
    _ck(lib().mahi_lattice_eval(float(box_L_nm), int(order_p), int(shell), r.shape[0], r.ctypes.data, out.ctypes.data),
        "mahi_lattice_eval")
    return out


def mahi_site_terms_static(box_L_nm, site_ptr, site_atoms, x, qA, qB, lam, phi, dEdlambda=None,
                           energy_correction=None, forces=None, stream=None):
    """Allocation-free per-site HI terms (device tensors in, device tensors out)."""
    n_sites = int(site_ptr.numel()) - 1
    n_atoms = int(x.shape[0])
    x_is_fp64 = 1 if str(x.dtype).endswith("float64") else 0
    _ck(lib().mahi_site_terms_static(float(box_L_nm), n_atoms, n_sites, _ptr(site_ptr), _ptr(site_atoms), _ptr(x),
                                     x_is_fp64,
                                     _ptr(qA), _ptr(qB), _ptr(lam), _ptr(phi), _ptr(dEdlambda),
                                     _ptr(energy_correction), _ptr(forces), _stream_handle(stream)),
        "mahi_site_terms_static")


def mahi_autotune(h, x, lam, reps=3):
    x_is_fp64 = 1 if str(x.dtype).endswith("float64") else 0
    _ck(lib().mahi_autotune(h, _ptr(x), x_is_fp64, _ptr(lam), int(reps)), "mahi_autotune")


def mahi_get_tuning(h):
    a, b = ctypes.c_int32(), ctypes.c_int32()
    _ck(lib().mahi_get_tuning(h, ctypes.byref(a), ctypes.byref(b)), "mahi_get_tuning")
    return int(a.value), int(b.value)


class MahiBatch:
    """Replicas (handles) evaluated as one CUDA graph; tensors are captured by
    pointer, so update them in place between launch() calls."""

    def __init__(self, handles, stream, xs, lams, energies, forces, dEdls):
        n = len(handles)
        arr = lambda vals: (ctypes.c_void_p * n)(*vals)
        self._keep = (xs, lams, energies, forces, dEdls)
        is64 = (ctypes.c_int32 * n)(*[1 if str(x.dtype).endswith("float64") else 0 for x in xs])
        out = ctypes.c_void_p()
        _ck(lib().mahi_batch_create(arr([h.value if hasattr(h, "value") else h for h in handles]), n,
                                    _stream_handle(stream), arr([_ptr(x) for x in xs]), is64,
                                    arr([_ptr(v) for v in lams]), arr([_ptr(v) for v in energies]),
                                    arr([_ptr(v) for v in forces]), arr([_ptr(v) for v in dEdls]),
                                    ctypes.byref(out)), "mahi_batch_create")
        self.b = out

    def launch(self):
        _ck(lib().mahi_batch_launch(self.b), "mahi_batch_launch")

    def close(self):
        if self.b is not None:
            _ck(lib().mahi_batch_destroy(self.b), "mahi_batch_destroy")
            self.b = None


def mahi_coulomb_constant():
    return float(lib().mahi_coulomb_constant())


def mahi_error_string(code):
    return lib().mahi_error_string(int(code)).decode()


class Mahi:
    """Owning wrapper around a handle: create, set charges, evaluate (torch)."""

    def __init__(self, box_L_nm, n_atoms, n_sites, order_p, depth, precision="fp64", stream=None):
        self.h = mahi_create(box_L_nm, n_atoms, n_sites, order_p, depth, precision, stream)
        self.n_atoms, self.n_sites = int(n_atoms), int(n_sites)
        self.n_lambdas = self.n_sites

    def set_charges(self, qA, qB, site_of_atom):
        mahi_set_charges(self.h, qA, qB, site_of_atom)
        self.n_lambdas = self.n_sites

    def update_charges(self, qA, qB):
        mahi_update_charges(self.h, qA, qB)

    def set_option(self, option, value):
        mahi_set_option(self.h, option, value)

    def get_option(self, option):
        return mahi_get_option(self.h, option)

    def status(self):
        return mahi_get_status(self.h)

    def set_forms(self, q_env, site_of_atom, forms):
        mahi_set_forms(self.h, q_env, site_of_atom, forms)
        self.n_lambdas = mahi_n_lambdas(self.h)

    def eval(self, x, lam):
        import torch
        E = torch.zeros(1, dtype=torch.float64, device=x.device)
        F = torch.empty_like(x)
        g = torch.zeros(max(1, self.n_lambdas), dtype=torch.float64, device=x.device)
        mahi_eval(self.h, x, lam, E, F, g)
        return E, F, g[: self.n_lambdas]

    def potential(self, device="cuda"):
        import torch
        phi = torch.empty(self.n_atoms, dtype=torch.float64, device=device)
        mahi_get_potential(self.h, phi)
        return phi

    def close(self):
        if self.h is not None:
            mahi_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
