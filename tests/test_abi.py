"""The C ABI library loads without a GPU and exports every symbol that
include/mahi.h declares; host-only entry points work on the CPU."""
import itertools
import os
import re

import numpy as np
import pytest

import oracle
import paper_2410_01754_gb300 as pkg
from paper_2410_01754_gb300 import build as pkg_build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module", autouse=True)
def _built():
    pkg_build.build()


def declared_symbols():
    txt = open(os.path.join(ROOT, "include", "mahi.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(mahi_[a-z_]+)\s*\(", txt)))


def test_every_declared_symbol_is_exported():
    lib = pkg.lib()
    names = declared_symbols()
    assert "mahi_create" in names and "mahi_eval" in names and len(names) >= 15
    for n in names:
        assert hasattr(lib, n), n


def test_coulomb_constant_matches_oracle():
    assert pkg.mahi_coulomb_constant() == pytest.approx(oracle.F_COULOMB, rel=1e-15)


def test_error_strings():
    for c in range(0, -9, -1):
        assert pkg.mahi_error_string(c)


def test_create_without_device_reports_no_device():
    import torch
    if torch.cuda.is_available():
        pytest.skip("a device is present")
    with pytest.raises(pkg.MahiError) as ei:
        pkg.mahi_create(2.0, 10, 0, 4, 1, "fp64")
    assert ei.value.code == -6


@pytest.mark.parametrize("args", [(-1.0, 10, 0, 4, 1), (1.0, 0, 0, 4, 1), (1.0, 10, 0, 0, 1), (1.0, 10, 0, 4, 7),
                                  (1.0, 10, -1, 4, 1), (1.0, 10, 0, 25, 1)])
def test_create_rejects_bad_arguments(args):
    with pytest.raises(pkg.MahiError) as ei:
        pkg.mahi_create(*args, "fp64")
    assert ei.value.code == -1


@pytest.mark.parametrize("shell", [1, 3])
def test_lattice_coefficients_cubic_symmetry(shell):
    p = 8
    c = pkg.mahi_lattice_coeffs(p, shell)
    for l in range(2 * p + 1):
        for m in range(l + 1):
            vals = [c[l * l]] if m == 0 else [c[l * l + 2 * m - 1], c[l * l + 2 * m]]
            allowed = (l % 2 == 0) and (m % 4 == 0) and l != 2
            if not allowed:
                assert all(v == 0.0 for v in vals)
            if m > 0:
                assert vals[1] == 0.0
    # the l = 0 term is H(0) = xi - (shell image sum), unit box
    rng_ = range(-shell, shell + 1)
    ssum = sum(1 / np.linalg.norm(n) for n in itertools.product(rng_, repeat=3) if any(n))
    assert c[0] == pytest.approx(oracle.xi(1.0) - ssum, rel=1e-13)


@pytest.mark.parametrize("shell,p,tol,span", [(1, 4, 5e-6, 0.5), (1, 8, 1e-8, 0.5), (1, 12, 5e-12, 0.5),
                                               (3, 8, 1e-10, 1.0), (3, 12, 5e-12, 1.0)])
def test_lattice_function_matches_oracle_kernel(shell, p, tol, span):
    """H_K(r) = A(r) - sum_{|n|_inf<=K} 1/|r+nL| - (2pi/3V)|r|^2 from the library's
    coefficients (degree 2p) against the Ewald oracle; |r|_inf <= span L."""
    rng = np.random.default_rng(p + 100 * shell)
    L = 3.7
    r = rng.uniform(-span, span, (25, 3)) * L
    H = pkg.mahi_lattice_eval(L, p, r, shell)
    ref = []
    shells = list(itertools.product(range(-shell, shell + 1), repeat=3))
    for ri in r:
        A, _ = oracle.pair_A(ri, L)
        near = sum(1 / np.linalg.norm(ri + np.array(n) * L) for n in shells)
        ref.append(A - near - 2 * np.pi / (3 * L ** 3) * ri @ ri)
    assert np.abs(H - np.array(ref)).max() * L < tol


def test_binding_option_names_match_the_header():
    """Every MAHI_OPT_* value of include/mahi.h is in the binding's OPTIONS
    under its lower-case name with the same number, and nothing else is."""
    txt = open(os.path.join(ROOT, "include", "mahi.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    header = {m.group(1).lower(): int(m.group(2)) for m in re.finditer(r"\bMAHI_OPT_([A-Z0-9_]+)\s*=\s*(\d+)", txt)}
    assert header, "no MAHI_OPT_* enum found"
    assert pkg.OPTIONS == header


def test_stage_names():
    """Ten intervals of the evaluation's chain, then the two side-stream intervals."""
    lib = pkg.lib()
    names = [lib.mahi_stage_name(i).decode() for i in range(12)]
    assert names == ["bin", "sort", "p2m", "m2m", "lattice", "m2l", "l2l", "near_pairs", "far_near_out", "site",
                     "side_site_pairs", "side_site_potential"]
    assert lib.mahi_stage_name(12).decode() == "?"
