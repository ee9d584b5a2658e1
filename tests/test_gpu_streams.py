"""Stream semantics of mahi_eval with its internal side stream: evaluations
queued back to back on the caller's stream, outputs copied out in stream
order with a single synchronisation at the end, give bitwise the results of
the same evaluations run one at a time with a full device synchronisation
in between (the side-stream work of an evaluation is joined before anything
that reads it, and never overlaps the next evaluation's writes)."""
import numpy as np
import pytest

import paper_2410_01754_gb300 as pkg
import synth

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA device")]


def _inputs(s, dev, k):
    rng = np.random.default_rng(100 + k)
    x = np.asarray(s["x"], dtype=np.float64) + rng.uniform(-0.02, 0.02, size=(len(s["qA"]), 3))
    lam = rng.uniform(0.0, 1.0, size=len(s["lam"]))
    return (torch.tensor(x, dtype=torch.float32, device=dev), torch.tensor(lam, dtype=torch.float64, device=dev))


@pytest.mark.parametrize("prec", ["mixed", "fp64"])
def test_back_to_back_evaluations_on_a_user_stream(prec):
    s = synth.make_water(n_water=10000, grid=22, L=6.76, n_sites=7, seed=41, depth=3, order=10)
    N, S = len(s["qA"]), len(s["lam"])
    dev = torch.device("cuda")
    h = pkg.mahi_create(s["L"], N, S, 10, 3, prec)
    try:
        pkg.mahi_set_charges(h, s["qA"], s["qB"], s["site_of"])
        inputs = [_inputs(s, dev, k) for k in range(3)]
        # reference: one evaluation at a time, device synchronised around each
        ref = []
        for x, lam in inputs:
            E = torch.zeros(1, dtype=torch.float64, device=dev)
            F = torch.zeros_like(x)
            g = torch.zeros(S, dtype=torch.float64, device=dev)
            torch.cuda.synchronize()
            pkg.mahi_eval(h, x, lam, E, F, g)
            torch.cuda.synchronize()
            ref.append((E.cpu().numpy(), F.cpu().numpy(), g.cpu().numpy()))
        # the same evaluations queued on a user stream into shared output
        # buffers, each result copied to pinned host memory in stream order
        stream = torch.cuda.Stream()
        pkg.mahi_set_stream(h, stream)
        E = torch.zeros(1, dtype=torch.float64, device=dev)
        F = torch.zeros_like(inputs[0][0])
        g = torch.zeros(S, dtype=torch.float64, device=dev)
        host = [(torch.empty(1, dtype=torch.float64, pin_memory=True), torch.empty(F.shape, dtype=F.dtype, pin_memory=True),
                 torch.empty(S, dtype=torch.float64, pin_memory=True)) for _ in inputs]
        torch.cuda.synchronize()
        with torch.cuda.stream(stream):
            for (x, lam), (hE, hF, hg) in zip(inputs, host):
                pkg.mahi_eval(h, x, lam, E, F, g)
                hE.copy_(E, non_blocking=True)
                hF.copy_(F, non_blocking=True)
                hg.copy_(g, non_blocking=True)
        stream.synchronize()
        for (E0, F0, g0), (hE, hF, hg) in zip(ref, host):
            assert np.array_equal(hE.numpy(), E0)
            assert np.array_equal(hF.numpy(), F0)
            assert np.array_equal(hg.numpy(), g0)
        # the three inputs differ, so a stale output would have shown
        assert not np.array_equal(ref[0][2], ref[1][2])
    finally:
        pkg.mahi_destroy(h)
