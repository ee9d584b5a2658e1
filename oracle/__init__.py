"""Oracle — test infrastructure only.

A plain, slow, FP64 CPU statement of what the MAHI hot path computes, written
from the paper (arxiv 2410.01754) and shared with nothing on the GPU path.
Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import it.

* ``ewald``      periodic potential, field and energy of a charge set (tin-foil
                 boundary, uniform neutralising background), by Ewald summation
                 in ``ewald.c``.
* ``pair_A``     the periodic pair kernel A(r) and its gradient; A(0) = xi.
* ``hi``         Hamiltonian-interpolation energy, lambda-derivatives and forces
                 (module ``oracle.hi``).
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "liboracle.so")
_lib = None

# Coulomb constant f = N_A e^2 / (4 pi eps0) in kJ mol^-1 nm e^-2, from the
# CODATA 2018 values of the elementary charge, Avogadro constant and eps0.
_E_CHARGE = 1.602176634e-19
_N_AVOGADRO = 6.02214076e23
_EPS0 = 8.8541878128e-12
F_COULOMB = _N_AVOGADRO * _E_CHARGE ** 2 / (4.0 * np.pi * _EPS0) * 1e6


def build(force: bool = False) -> str:
    """Compile ``ewald.c`` into ``liboracle.so`` next to it (gcc, OpenMP)."""
    src = os.path.join(_HERE, "ewald.c")
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(src):
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-o", _SO, src, "-lm"])
    return _SO


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_SO)
        dp = ctypes.POINTER(ctypes.c_double)
        L.oracle_ewald.argtypes = [ctypes.c_int64, dp, dp, ctypes.c_double, ctypes.c_double,
                                   ctypes.c_int64, ctypes.POINTER(ctypes.c_int64), dp, dp, dp]
        L.oracle_ewald.restype = ctypes.c_int
        L.oracle_ewald_parts.argtypes = L.oracle_ewald.argtypes + [ctypes.c_int]
        L.oracle_ewald_parts.restype = ctypes.c_int
        L.oracle_pair_A.argtypes = [dp, ctypes.c_double, ctypes.c_double, dp]
        L.oracle_pair_A.restype = ctypes.c_double
        L.oracle_ewald_params.argtypes = [ctypes.c_double, ctypes.c_double, dp,
                                          ctypes.POINTER(ctypes.c_int)]
        L.oracle_direct.argtypes = [ctypes.c_int64, dp, ctypes.c_int64, dp, dp, dp]
        L.oracle_ewald_energy.argtypes = [ctypes.c_int64, dp, dp, ctypes.c_double, ctypes.c_double]
        L.oracle_ewald_energy.restype = ctypes.c_double
        L.oracle_num_threads.restype = ctypes.c_int
        _lib = L
    return _lib


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def num_threads() -> int:
    return int(lib().oracle_num_threads())


def default_rc(L: float, n: int) -> float:
    """Real-space cutoff balancing the real-space and reciprocal-space work
    (alpha = 6/rc, |m| <= 11.6 L/rc), capped at L/2."""
    rho = n / L ** 3
    rcs = np.linspace(0.3, 0.5 * L, 400)
    cost = rho * (4.0 / 3.0) * np.pi * rcs ** 3 + (2.0 / 3.0) * np.pi * (11.6 * L / rcs) ** 3
    return float(rcs[int(np.argmin(cost))])


def ewald(x, q, L, rc=None, targets=None, parts=3):
    """Periodic potential phi (e/nm), its gradient and the energy (e^2/nm), f = 1.

    phi_i = sum_j q_j A(x_i - x_j) with A(0) = xi; grad excludes the j = i term.
    With ``targets`` None all atoms are targets and the energy 1/2 sum q phi is
    returned, otherwise energy is None.  ``parts`` = 1 (real space only), 2
    (reciprocal space with self and background terms only) or 3 (both)."""
    x = np.ascontiguousarray(x, dtype=np.float64)
    q = np.ascontiguousarray(q, dtype=np.float64)
    n = q.shape[0]
    if rc is None:
        rc = default_rc(L, n)
    rc = min(rc, 0.5 * L)
    if targets is None:
        nt = n
        tptr = ctypes.POINTER(ctypes.c_int64)()
    else:
        t = np.ascontiguousarray(targets, dtype=np.int64)
        nt = t.shape[0]
        tptr = t.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))
    phi = np.zeros(nt)
    grad = np.zeros((nt, 3))
    e = np.zeros(1)
    rcode = lib().oracle_ewald_parts(n, _dp(x), _dp(q), float(L), float(rc), nt, tptr, _dp(phi), _dp(grad),
                                     _dp(e), int(parts))
    if rcode != 0:
        raise RuntimeError("oracle_ewald failed")
    return phi, grad, (float(e[0]) if targets is None else None)


def ewald_energy(x, q, L, rc=None):
    """Energy 1/2 sum_i q_i phi_i (f = 1) without per-atom potentials."""
    x = np.ascontiguousarray(x, dtype=np.float64)
    q = np.ascontiguousarray(q, dtype=np.float64)
    if rc is None:
        rc = default_rc(L, q.shape[0])
    rc = min(rc, 0.5 * L)
    return float(lib().oracle_ewald_energy(q.shape[0], _dp(x), _dp(q), float(L), float(rc)))


def pair_A(r, L, rc=None):
    """A(r) and grad A(r) (f = 1) for one displacement; A(0) = xi."""
    r = np.ascontiguousarray(r, dtype=np.float64)
    if rc is None:
        rc = 0.5 * L
    g = np.zeros(3)
    v = lib().oracle_pair_A(_dp(r), float(L), float(rc), _dp(g))
    return float(v), g


def xi(L):
    """Self-image term A(0) of the periodic kernel."""
    return pair_A(np.zeros(3), L)[0]


def direct(targets, sources, qs):
    """Non-periodic direct Coulomb potential sum_j q_j/|x_i - y_j| (f = 1)."""
    xt = np.ascontiguousarray(targets, dtype=np.float64)
    ys = np.ascontiguousarray(sources, dtype=np.float64)
    qs = np.ascontiguousarray(qs, dtype=np.float64)
    phi = np.zeros(xt.shape[0])
    lib().oracle_direct(xt.shape[0], _dp(xt), ys.shape[0], _dp(ys), _dp(qs), _dp(phi))
    return phi
