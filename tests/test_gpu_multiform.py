"""Sites with 2^m forms (mahi_set_forms) against the multi-form oracle, and
the two-form case against the two-form path."""
import numpy as np
import pytest

from oracle import hi
import paper_2410_01754_gb300 as pkg
import synth

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA device")]


def _multiform_system(nforms=(4, 2, 8, 16), seed=12):
    """3,000 charges in L = 3.2 nm (the paper's random-system shape) with sites
    of four atoms having 2^m forms: every form perturbs the atoms' charges."""
    s = synth.make_charges(n=3000, L=3.2, n_sites=len(nforms), atoms_per_site=4, seed=seed, depth=3, order=12,
                           dmin=0.1)
    rng = np.random.default_rng(seed)
    sites = hi.site_lists(s["site_of"], len(nforms))
    forms = [s["qA"][at][None, :] + rng.uniform(-0.4, 0.4, (F, len(at))) for F, at in zip(nforms, sites)]
    lams = [rng.uniform(0, 1, int(np.log2(F))) for F in nforms]
    return dict(x=s["x"], q_env=s["qA"], site_of=s["site_of"], forms=forms, lams=lams, L=s["L"])


@pytest.fixture(scope="module")
def mf():
    s = _multiform_system()
    return s, hi.multiform_eval(s)


@pytest.mark.parametrize("prec,p,tolE,tolF", [("fp64", 16, 5e-7, 3e-6), ("mixed", 12, 2e-5, 1e-4)])
def test_multiform_matches_oracle(mf, prec, p, tolE, tolF):
    s, ref = mf
    N, S = len(s["q_env"]), len(s["forms"])
    m = pkg.Mahi(s["L"], N, S, p, 3, prec)
    m.set_forms(s["q_env"], s["site_of"], s["forms"])
    assert m.n_lambdas == sum(len(l) for l in s["lams"])
    xdt = torch.float64 if prec == "fp64" else torch.float32
    x = torch.tensor(s["x"], dtype=xdt, device="cuda")
    lam = torch.tensor(np.concatenate(s["lams"]), dtype=torch.float64, device="cuda")
    E, F, g = m.eval(x, lam)
    torch.cuda.synchronize()
    m.close()
    assert abs(E.item() - ref["E"]) < tolE * abs(ref["E"])
    Fg, Fr = F.double().cpu().numpy(), ref["F"]
    assert np.sqrt(((Fg - Fr) ** 2).sum() / (Fr ** 2).sum()) < tolF
    assert np.abs(g.cpu().numpy() - ref["dEdl"]).max() < 1e-3


def test_two_forms_equal_two_form_path():
    s = synth.make_water(n_water=3000, grid=16, L=4.5, n_sites=6, seed=9, depth=3, order=10)
    N, S = len(s["qA"]), 6
    sites = hi.site_lists(s["site_of"], S)
    x = torch.tensor(s["x"], dtype=torch.float64, device="cuda")
    lam = torch.tensor(s["lam"], dtype=torch.float64, device="cuda")
    a = pkg.Mahi(s["L"], N, S, 10, 3, "fp64")
    a.set_charges(s["qA"], s["qB"], s["site_of"])
    Ea, Fa, ga = a.eval(x, lam)
    b = pkg.Mahi(s["L"], N, S, 10, 3, "fp64")
    b.set_forms(s["qA"], s["site_of"], [np.stack([s["qA"][at], s["qB"][at]]) for at in sites])
    Eb, Fb, gb = b.eval(x, lam)
    torch.cuda.synchronize()
    a.close()
    b.close()
    assert abs(Ea.item() - Eb.item()) < 1e-12 * abs(Ea.item())
    assert np.abs(ga.cpu().numpy() - gb.cpu().numpy()).max() < 1e-8
    assert np.abs(Fa.cpu().numpy() - Fb.cpu().numpy()).max() < 1e-8 * np.abs(Fa.cpu().numpy()).max()


def test_set_forms_rejects_bad_form_counts():
    m = pkg.Mahi(2.0, 10, 1, 4, 1, "fp64")
    so = np.full(10, -1, dtype=np.int32)
    so[:3] = 0
    with pytest.raises(pkg.MahiError) as ei:
        m.set_forms(np.zeros(10), so, [np.zeros((3, 3))])
    assert ei.value.code == -1
    m.close()


@pytest.mark.parametrize("prec,p,tol", [("fp64", 16, 1e-6), ("mixed", 12, 3e-4)])
def test_multiform_backward_matches_oracle(mf, prec, p, tol):
    """mahi_backward_forms against the oracle's charge gradients of the
    multi-form energy (and dx = -g F, dlambda = g dE/dlambda), upstream
    gradient 0.7.  Mixed: environment potentials carry the tensor-core M2L's
    accumulation bias, so they are held to 3e-4 of the largest gradient."""
    s, ref = mf
    cg = hi.multiform_charge_gradients(s, ref=ref)
    N, S = len(s["q_env"]), len(s["forms"])
    m = pkg.Mahi(s["L"], N, S, p, 3, prec)
    m.set_forms(s["q_env"], s["site_of"], s["forms"])
    xdt = torch.float64 if prec == "fp64" else torch.float32
    dev = torch.device("cuda")
    x = torch.tensor(s["x"], dtype=xdt, device=dev)
    lam = torch.tensor(np.concatenate(s["lams"]), dtype=torch.float64, device=dev)
    E, F, g = m.eval(x, lam)
    ge = torch.tensor([0.7], dtype=torch.float64, device=dev)
    nform = sum(np.asarray(f).size for f in s["forms"])
    dx = torch.empty_like(F)
    dl = torch.empty_like(g)
    dq_env = torch.full((N,), 9.0, dtype=torch.float64, device=dev)
    dq_forms = torch.full((nform,), 9.0, dtype=torch.float64, device=dev)
    pkg.mahi_backward_forms(m.h, ge, F, g, lam, dx, dl, dq_env, dq_forms)
    with pytest.raises(pkg.MahiError) as ei:   # the two-form entry point refuses these sites
        pkg.mahi_backward(m.h, ge, F, g, lam, dx)
    assert ei.value.code == -1
    torch.cuda.synchronize()
    m.close()
    assert torch.equal(dx, -0.7 * F)
    assert torch.allclose(dl, 0.7 * g, rtol=0, atol=0)
    want_env = 0.7 * cg["dq_env"]
    want_forms = 0.7 * np.concatenate([np.asarray(f).ravel() for f in cg["dq_forms"]])
    got_env, got_forms = dq_env.cpu().numpy(), dq_forms.cpu().numpy()
    scale = max(np.abs(want_env).max(), np.abs(want_forms).max())
    assert np.abs(got_forms - want_forms).max() < tol * scale, np.abs(got_forms - want_forms).max() / scale
    assert np.abs(got_env - want_env).max() < tol * scale, np.abs(got_env - want_env).max() / scale
