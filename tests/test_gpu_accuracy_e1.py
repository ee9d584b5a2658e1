"""The paper's accuracy test on the GPU path (Sec. "Accuracy of the Random
System with Two Forms and Four Forms", Fig. "accuracy"): 1,000 + 10 random
charges, one site of 10 particles with two or four forms, clustered
("typical") or scattered ("worst") site particles, lambda = 0.345 and
(0.345, 0.721).  dE/dlambda is compared with the oracle (exact periodic HI)
and with the paper's reference, the end-state energies of the same path at
the same order and depth combined by the derivative of the multilinear
interpolation (Eqs. "ref_two_forms", "ref_four_forms", read as the
derivative of Eq. "rek_ham_lambda").  At depth 0 every interaction is direct
and both deviations sit at the lattice term's truncation; at depth 2 they fall
with the order.  Scattered sites take one traversal per atom."""
import os
import sys

import numpy as np
import pytest

from oracle import hi
import synth

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA device")]

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
from bench import e1_point  # noqa: E402


@pytest.fixture(scope="module", params=[("typical", 2), ("typical", 4), ("worst", 2), ("worst", 4)],
                ids=lambda v: f"{v[0]}-{v[1]}forms")
def e1(request):
    layout, forms = request.param
    s = synth.make_e1(layout, forms, 1)
    return s, hi.multiform_eval(s)["dEdl"]


@pytest.mark.parametrize("prec,p,tol,tol_same", [("fp64", 20, 1e-9, 1e-7), ("mixed", 15, 1e-5, 1e-2)])
def test_depth_zero_is_exact(e1, prec, p, tol, tol_same):
    """Depth 0: the whole box is one leaf, so every first-shell interaction
    is direct and only the far images go through the root multipole (its
    truncation falls like 0.866^(p+1)): at p = 20 the FP64 path reaches the
    oracle to 1e-9.  The same-order reference uses the FMM's own potential in
    its end-state energies, so it carries that truncation too, and in the
    mixed path the single-precision rounding of those energies (their
    difference is a few hundred kJ/mol out of ~1e5: 1e-3 relative)."""
    s, ref = e1
    r = e1_point(s, prec, p, 0, ref)
    assert r["status"] == 0
    assert max(r["rel_dev_vs_oracle"]) < tol, r
    assert max(r["rel_dev_vs_same_order_fmm"]) < tol_same, r


def test_fp64_deviation_falls_with_order(e1):
    s, ref = e1
    devs = [max(e1_point(s, "fp64", p, 2, ref)["rel_dev_vs_oracle"]) for p in (4, 8, 12, 16)]
    assert devs[-1] < 1e-6, devs
    for a, b in zip(devs, devs[1:]):
        assert b < a or b < 1e-9, devs


@pytest.mark.parametrize("prec,p", [("fp64", 12), ("mixed", 12)])
def test_production_order_within_bar(e1, prec, p):
    """At the 1M-atom workload's order the absolute dE/dlambda error stays
    below 1e-3 kJ/mol against the oracle for both site layouts."""
    s, ref = e1
    r = e1_point(s, prec, p, 2, ref)
    assert r["status"] == 0
    err = np.abs(np.array(r["dEdl"]) - ref).max()
    assert err < 1e-3, (err, r)
