"""Backward pass (mahi_backward, the autograd function) against the oracle and
against central finite differences of the GPU energy.

The HI energy is a quadratic polynomial in lambda and in the charges, so its
central differences there are exact up to rounding.  The GPU energy is the
FMM's, however, while dE/dlambda and dE/dq at site atoms use the refined
site-atom potential; the two differ by the FMM's truncation error of the
potential at the site atoms (a few 1e-3 kJ/mol/e at p = 12), which bounds
those tolerances.  In x the forces are likewise not the exact gradient of the
truncated FMM energy."""
import numpy as np
import pytest

import oracle
from oracle import hi
import paper_2410_01754_gb300 as pkg
import synth

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA device")]

from paper_2410_01754_gb300.autograd import MahiEnergy  # noqa: E402


def _tensors(s, xdt):
    dev = torch.device("cuda")
    x = torch.tensor(s["x"], dtype=xdt, device=dev, requires_grad=True)
    lam = torch.tensor(s["lam"], dtype=torch.float64, device=dev, requires_grad=True)
    qA = torch.tensor(s["qA"], dtype=torch.float64, device=dev, requires_grad=True)
    qB = torch.tensor(s["qB"], dtype=torch.float64, device=dev, requires_grad=True)
    return x, lam, qA, qB


@pytest.fixture(scope="module")
def sysA():
    s = synth.make("A", 1)
    ref = hi.hi_eval(s)
    return s, ref, hi.hi_charge_gradients(s, ref=ref)


@pytest.mark.parametrize("prec,xdt,tol,etol", [("fp64", torch.float64, 1e-6, 5e-7), ("mixed", torch.float32, 1e-4, 2e-5)])
def test_backward_matches_oracle(sysA, prec, xdt, tol, etol):
    """Config A (3,000 charges, 4 sites) at p = 16: every gradient against the
    oracle's closed forms, scaled by an upstream gradient of 0.7."""
    s, ref, cg = sysA
    me = MahiEnergy(s["L"], s["site_of"], len(s["lam"]), 16 if prec == "fp64" else 15, 3, prec)
    x, lam, qA, qB = _tensors(s, xdt)
    E = me.energy(x, lam, qA, qB)
    (0.7 * E).backward()
    torch.cuda.synchronize()
    me.close()
    # mixed: the tensor-core M2L accumulates toward zero (a few 1e-6 of E here)
    assert abs(E.item() - ref["E"]) < etol * abs(ref["E"])
    Fr = ref["F"]
    dx = x.grad.double().cpu().numpy()
    assert np.sqrt(((dx + 0.7 * Fr) ** 2).sum() / ((0.7 * Fr) ** 2).sum()) < 10 * tol
    np.testing.assert_allclose(lam.grad.cpu().numpy(), 0.7 * ref["dEdl"], atol=1e-3)
    for key, g in (("dqA", qA.grad), ("dqB", qB.grad)):
        got = g.cpu().numpy()
        want = 0.7 * cg[key]
        scale = np.abs(want).max()
        assert np.abs(got - want).max() < tol * scale, (key, np.abs(got - want).max() / scale)


@pytest.fixture(scope="module")
def sysD():
    return synth.make("D", 1)


def test_autograd_finite_differences_fp64(sysD):
    """200,001 atoms, 128 sites, p = 12, FP64 path: autograd gradients against
    central differences of the GPU energy on 64 random coordinates (h = 1e-4 nm),
    8 lambdas (h = 1e-4) and 8 charges of each set."""
    s = sysD
    N, S = len(s["qA"]), len(s["lam"])
    me = MahiEnergy(s["L"], s["site_of"], S, 12, 4, "fp64")
    x, lam, qA, qB = _tensors(s, torch.float64)
    E = me.energy(x, lam, qA, qB)
    E.backward()
    gx, gl, gA, gB = (t.grad.clone() for t in (x, lam, qA, qB))
    rng = np.random.default_rng(5)

    def energy(xx=None, ll=None, a=None, b=None):
        with torch.no_grad():
            return me.energy(x if xx is None else xx, lam if ll is None else ll, qA if a is None else a,
                             qB if b is None else b).item()

    # positions: 64 random (atom, axis) pairs
    h = 1e-4
    Fscale = gx.abs().max().item()
    errs = []
    for k in rng.choice(N, 64, replace=False):
        ax = int(rng.integers(3))
        xp = x.detach().clone(); xp[k, ax] += h
        xm = x.detach().clone(); xm[k, ax] -= h
        fd = (energy(xx=xp) - energy(xx=xm)) / (2 * h)
        errs.append(abs(fd - gx[k, ax].item()))
    # FMM truncation at p = 12: the forces differ from the gradient of the
    # truncated energy by ~1e-6 of the largest force
    assert max(errs) < 2e-5 * Fscale, (max(errs), Fscale)
    # lambda and charges: exact central differences of a quadratic
    for k in rng.choice(S, 8, replace=False):
        lp = lam.detach().clone(); lp[k] += 1e-4
        lm = lam.detach().clone(); lm[k] -= 1e-4
        fd = (energy(ll=lp) - energy(ll=lm)) / 2e-4
        assert fd == pytest.approx(gl[k].item(), abs=1e-2)
    site_atoms = np.where(s["site_of"] >= 0)[0]
    for key, t, g in (("qA", qA, gA), ("qB", qB, gB)):
        for k in list(rng.choice(site_atoms, 6, replace=False)) + list(rng.choice(N, 2, replace=False)):
            hq = 1e-3
            tp = t.detach().clone(); tm = t.detach().clone()
            tp[k] += hq; tm[k] -= hq
            if s["site_of"][k] < 0:  # environment atoms carry one charge (qA == qB)
                other = qB if key == "qA" else qA
                op = other.detach().clone(); om = other.detach().clone()
                op[k] += hq; om[k] -= hq
                args_p = dict(a=tp, b=op) if key == "qA" else dict(a=op, b=tp)
                args_m = dict(a=tm, b=om) if key == "qA" else dict(a=om, b=tm)
                fd = (energy(**args_p) - energy(**args_m)) / (2 * hq)
                assert fd == pytest.approx((gA[k] + gB[k]).item(), abs=1e-2)
            else:
                fd = (energy(**{"a" if key == "qA" else "b": tp}) - energy(**{"a" if key == "qA" else "b": tm})) / (2 * hq)
                assert fd == pytest.approx(g[k].item(), abs=1e-2)
    me.close()


def test_autograd_finite_differences_mixed(sysD):
    """200,001 atoms, 128 sites, p = 12, mixed path (float32 positions, FP32
    FMM with the FP64 site terms): autograd gradients against central
    differences of the same path's energy.  The energy is an FP64 sum of
    single-precision potentials, whose rounding changes with any perturbation
    (about 1e-2 kJ/mol over 200k atoms), so the steps are chosen where that
    noise is small next to the difference: 2e-3 nm in x (the truncation error
    of the central difference there is below 2 kJ/mol/nm even for the
    closest pairs), and 0.25 in lambda and 0.05 e in the charges, where the
    energy is exactly quadratic and central differences are exact for any
    step.  dE/dlambda and dE/dq use the refined site-atom potential, the
    energy the FMM's, whose truncation and, in the mixed path, tensor-core
    accumulation bias (about 7e-4 of the far-field locals, mostly in their
    constant term, so in the potential and not in the forces) put the energy's
    potential at a site atom up to ~1 kJ/mol/e (1e-3 relative) away from the
    refined one: differences of a few tenths per unit lambda (measured 0.23).
    A central difference in a charge measures the symmetrised potential
    (A + A^T) q / 2 of the FMM's approximate operator A, which single
    precision and the tensor-core rounding make asymmetric at ~1e-3: up to
    ~1.6 kJ/mol/e on a 450 kJ/mol/e potential.
    In x the check is bounded by the single-precision near-field sums: moving
    one atom re-rounds the ~800 potentials it enters (each a sum of terms up
    to ~1e3 kJ/mol/e), which shifts the energy by ~1e-2 kJ/mol, so central
    differences over 4e-3 nm scatter by ~10 kJ/mol/nm (measured median 9,
    largest 41, against forces up to 1.1e4): the check catches sign, scale
    and leaf-boundary errors, not rounding."""
    s = sysD
    N, S = len(s["qA"]), len(s["lam"])
    me = MahiEnergy(s["L"], s["site_of"], S, 12, 4, "mixed")
    x, lam, qA, qB = _tensors(s, torch.float32)
    E = me.energy(x, lam, qA, qB)
    E.backward()
    gx, gl, gA, gB = (t.grad.clone() for t in (x, lam, qA, qB))
    rng = np.random.default_rng(6)

    def energy(xx=None, ll=None, a=None, b=None):
        with torch.no_grad():
            return me.energy(x if xx is None else xx, lam if ll is None else ll, qA if a is None else a,
                             qB if b is None else b).item()

    Fscale = gx.abs().max().item()
    errs = []
    for k in rng.choice(N, 64, replace=False):
        ax = int(rng.integers(3))
        xp = x.detach().clone(); xp[k, ax] += 2e-3
        xm = x.detach().clone(); xm[k, ax] -= 2e-3
        h2 = (xp[k, ax] - xm[k, ax]).item()        # the step as stored in float32
        fd = (energy(xx=xp) - energy(xx=xm)) / h2
        errs.append(abs(fd - gx[k, ax].item()))
    print(f"mixed finite differences in x: max {max(errs):.3g}, median {np.median(errs):.3g} kJ/mol/nm "
          f"(largest force {Fscale:.4g})")
    assert max(errs) < 5e-3 * Fscale, (max(errs), np.median(errs), Fscale)
    assert np.median(errs) < 1.5e-3 * Fscale, (max(errs), np.median(errs), Fscale)
    for k in rng.choice(S, 8, replace=False):
        lp = lam.detach().clone(); lp[k] += 0.25
        lm = lam.detach().clone(); lm[k] -= 0.25
        fd = (energy(ll=lp) - energy(ll=lm)) / 0.5
        assert fd == pytest.approx(gl[k].item(), abs=0.5)
    site_atoms = np.where(s["site_of"] >= 0)[0]
    for key, t, g in (("qA", qA, gA), ("qB", qB, gB)):
        for k in rng.choice(site_atoms, 6, replace=False):
            tp = t.detach().clone(); tm = t.detach().clone()
            tp[k] += 0.05; tm[k] -= 0.05
            arg = "a" if key == "qA" else "b"
            fd = (energy(**{arg: tp}) - energy(**{arg: tm})) / 0.1
            assert fd == pytest.approx(g[k].item(), abs=1.0, rel=5e-3)
    me.close()


def test_autograd_mixed_matches_fp64(sysD):
    """The mixed path's gradients (single precision with FP64 site terms)
    against the FP64 path's on the same 200,001-atom system."""
    s = sysD
    S = len(s["lam"])
    out = {}
    for prec, xdt in (("fp64", torch.float64), ("mixed", torch.float32)):
        me = MahiEnergy(s["L"], s["site_of"], S, 12, 4, prec)
        x, lam, qA, qB = _tensors(s, xdt)
        me.energy(x, lam, qA, qB).backward()
        torch.cuda.synchronize()
        out[prec] = [t.grad.double().cpu().numpy() for t in (x, lam, qA, qB)]
        me.close()
    a, b = out["fp64"], out["mixed"]
    assert np.sqrt(((a[0] - b[0]) ** 2).sum() / (a[0] ** 2).sum()) < 1e-4
    assert np.abs(a[1] - b[1]).max() < 1e-3
    # charge gradients are potentials: at environment atoms the mixed path's
    # carries the tensor-core accumulation bias of its far field
    for k in (2, 3):
        assert np.abs(a[k] - b[k]).max() < 3e-4 * np.abs(a[k]).max()


def test_backward_before_charges_is_an_error():
    m = pkg.Mahi(2.0, 10, 1, 4, 1, "fp64")
    g = torch.ones(1, dtype=torch.float64, device="cuda")
    with pytest.raises(pkg.MahiError) as ei:
        pkg.mahi_backward(m.h, g, None, None, None)
    assert ei.value.code == -7
    m.close()
