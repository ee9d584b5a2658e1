"""Device-side failure reporting and solver options, through the C ABI.

Two failures are detected inside the kernels and reported through the
handle's status word: a bounded wait of the tensor-core M2L that runs out
(MAHI_ERR_TIMEOUT) and a site traversal whose per-level lists outgrow their
capacity (MAHI_ERR_SITE_OVERFLOW).  Both are provoked here without any fault:
the watchdog self-test option makes the M2L wait on a barrier that nothing
completes (with a 20 ms wait limit), and a list capacity of 64 is below the
343 root images every traversal starts from.  After each failure the same
handle must evaluate normally again, bit for bit as before.  Also here:
charges from device memory (mahi_set_charges) and the asynchronous charge
update (mahi_update_charges)."""
import numpy as np
import pytest

import paper_2410_01754_gb300 as pkg
import synth

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA device")]


@pytest.fixture(scope="module")
def small():
    return synth.make_water(n_water=3000, grid=16, L=4.5, n_sites=6, seed=9, depth=3, order=8)


def _solver(s, prec="mixed"):
    m = pkg.Mahi(s["L"], len(s["qA"]), len(s["lam"]), s["order"], s["depth"], prec)
    m.set_charges(s["qA"], s["qB"], s["site_of"])
    x = torch.tensor(s["x"], dtype=torch.float32, device="cuda")
    lam = torch.tensor(s["lam"], dtype=torch.float64, device="cuda")
    return m, x, lam


def _host(r):
    E, F, g = r
    torch.cuda.synchronize()
    return E.item(), F.cpu().numpy(), g.cpu().numpy()


def _same(a, b):
    return a[0] == b[0] and np.array_equal(a[1], b[1]) and np.array_equal(a[2], b[2])


def test_watchdog_timeout_is_reported_and_the_handle_recovers(small):
    m, x, lam = _solver(small)
    try:
        ref = _host(m.eval(x, lam))
        assert m.status() == 0
        m.set_option("wait_limit_ms", 20)
        m.set_option("watchdog_selftest", 1)
        m.eval(x, lam)                       # enqueued; the M2L's wait runs out on the device
        assert m.status() == pkg.MAHI_ERR_TIMEOUT
        assert m.status() == 0               # reporting cleared the word
        m.eval(x, lam)
        torch.cuda.synchronize()
        with pytest.raises(pkg.MahiError) as ei:   # reported by the next evaluation ...
            m.eval(x, lam)
        assert ei.value.code == pkg.MAHI_ERR_TIMEOUT
        torch.cuda.synchronize()
        m.set_option("watchdog_selftest", 0)
        m.set_option("wait_limit_ms", 0)
        assert m.status() == 0               # ... which enqueued nothing
        again = _host(m.eval(x, lam))
        assert m.status() == 0
        assert _same(again, ref)
    finally:
        m.close()


def test_watchdog_timeout_through_eval_host(small):
    m, _, _ = _solver(small)
    try:
        m.set_option("wait_limit_ms", 20)
        m.set_option("watchdog_selftest", 1)
        N, S = len(small["qA"]), len(small["lam"])
        E, F, g = np.zeros(1), np.zeros((N, 3), np.float32), np.zeros(S)
        with pytest.raises(pkg.MahiError) as ei:
            pkg.mahi_eval_host(m.h, np.ascontiguousarray(small["x"], dtype=np.float32),
                               np.ascontiguousarray(small["lam"]), E, F, g)
        assert ei.value.code == pkg.MAHI_ERR_TIMEOUT
        m.set_option("watchdog_selftest", 0)
        pkg.mahi_eval_host(m.h, np.ascontiguousarray(small["x"], dtype=np.float32),
                           np.ascontiguousarray(small["lam"]), E, F, g)
        assert np.isfinite(E[0])
    finally:
        m.close()


@pytest.mark.parametrize("prec", ["mixed", "fp64"])
def test_site_list_overflow_is_reported_and_the_handle_recovers(small, prec):
    m, x, lam = _solver(small, prec)
    try:
        ref = _host(m.eval(x, lam))
        m.set_option("site_list_cap", 64)
        assert m.get_option("site_list_cap") == 64
        m.eval(x, lam)
        assert m.status() == pkg.MAHI_ERR_SITE_OVERFLOW
        m.set_option("site_list_cap", 0)
        again = _host(m.eval(x, lam))
        assert m.status() == 0
        assert _same(again, ref)
    finally:
        m.close()


def test_option_defaults_and_range():
    for p, theta in [(4, 0.25), (8, 0.4 ** (13 / 9)), (10, 0.4 ** (13 / 11)), (12, 0.4), (14, 0.4)]:
        m = pkg.Mahi(3.0, 100, 2, p, 2, "fp64")
        try:
            assert m.get_option("site_theta") == pytest.approx(theta, rel=1e-6)
            cap = m.get_option("site_list_cap")
            assert cap >= 1536 and cap % 256 == 0
            assert m.get_option("wait_limit_ms") == pytest.approx(2000.0)
            m.set_option("site_theta", 0.3)
            assert m.get_option("site_theta") == pytest.approx(0.3)
            m.set_option("site_theta", 0)
            assert m.get_option("site_theta") == pytest.approx(theta, rel=1e-6)
            assert m.get_option("m2l_split_degree") == 2
            m.set_option("m2l_split_degree", p)
            assert m.get_option("m2l_split_degree") == p
            for opt, bad in [("site_theta", 0.8), ("site_theta", -0.1), ("site_list_cap", 10),
                             ("site_list_cap", 20000), ("wait_limit_ms", 0.5), ("watchdog_selftest", 2),
                             ("m2l_split_degree", -2), ("m2l_split_degree", p + 1), ("m2l_split_degree", 1.5),
                             ("m2l_single_tile", 2), ("m2l_b_stages", 1), ("m2l_b_stages", 5), ("p2p_threads", 100),
                             ("site_blocks", 17), ("p2p_targets", 3), ("p2p_targets", 16), (99, 1)]:
                with pytest.raises(pkg.MahiError) as ei:
                    m.set_option(opt, bad)
                assert ei.value.code == -1
        finally:
            m.close()


def test_charges_from_device_memory(small):
    m1, x, lam = _solver(small, "mixed_simt")
    m2 = pkg.Mahi(small["L"], len(small["qA"]), len(small["lam"]), small["order"], small["depth"], "mixed_simt")
    try:
        dev = torch.device("cuda")
        m2.set_charges(torch.tensor(small["qA"], device=dev), torch.tensor(small["qB"], device=dev),
                       torch.tensor(small["site_of"], dtype=torch.int32, device=dev))
        assert _same(_host(m1.eval(x, lam)), _host(m2.eval(x, lam)))
        bad = small["site_of"].copy()
        bad[0] = len(small["lam"])           # site index out of range, from device memory
        with pytest.raises(pkg.MahiError) as ei:
            m2.set_charges(torch.tensor(small["qA"], device=dev), torch.tensor(small["qB"], device=dev),
                           torch.tensor(bad, dtype=torch.int32, device=dev))
        assert ei.value.code == -2
    finally:
        m1.close()
        m2.close()


def test_update_charges_matches_set_charges(small):
    """New charges through the enqueued update equal a fresh mahi_set_charges."""
    s = small
    rng = np.random.default_rng(5)
    qA2 = s["qA"] * (1.0 + 0.1 * rng.standard_normal(len(s["qA"])))
    qB2 = np.where(s["site_of"] >= 0, s["qB"] + 0.05, qA2)
    m1, x, lam = _solver(s, "mixed")
    m2, _, _ = _solver(s, "mixed")
    try:
        dev = torch.device("cuda")
        m1.eval(x, lam)
        m1.update_charges(torch.tensor(qA2, device=dev), torch.tensor(qB2, device=dev))
        a = _host(m1.eval(x, lam))
        m2.set_charges(qA2, qB2, s["site_of"])
        b = _host(m2.eval(x, lam))
        assert _same(a, b)
    finally:
        m1.close()
        m2.close()
