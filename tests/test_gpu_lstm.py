"""MDHP-LSTM cell on the GPU (mdhp_lstm_forward / mdhp_lstm_backward, through
the autograd Function) against the FP64 oracle (oracle/lstm.py): outputs and
the gradients of every weight, the inputs and the MDHP parameters, for a
ragged mix of sizes (H not a multiple of 32, per-source and scalar beta,
single-step sequences, weights staged in shared memory or read from global
memory), and each sequences-per-CTA variant of the kernels with a ragged
last CTA."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("B,L,D,H,M,nb,O", [(5, 7, 4, 3, 2, 2, 2), (64, 33, 11, 64, 16, 1, 3),
                                             (9, 1, 5, 20, 4, 4, 1), (17, 12, 40, 200, 8, 8, 5)])
def test_lstm_matches_oracle(B, L, D, H, M, nb, O):
    _check(B, L, D, H, M, nb, O)


@pytest.mark.parametrize("S", [1, 4, 8, 16])
@pytest.mark.parametrize("B,L,D,H,M,nb,O", [(37, 9, 11, 64, 16, 1, 2), (21, 5, 40, 200, 8, 8, 5),
                                             (13, 6, 30, 12, 4, 4, 2)])
def test_lstm_sequences_per_cta(monkeypatch, S, B, L, D, H, M, nb, O):
    # (13, 6, 30, 12): inputs wider than the hidden state, so part of each
    # step's inputs is fetched after the matvec rather than ahead of it
    monkeypatch.setenv("MDHP_LSTM_SEQ_PER_CTA", str(S))
    _check(B, L, D, H, M, nb, O)


def _check(B, L, D, H, M, nb, O):
    from oracle import lstm

    import paper_2411_10258_gb300 as mdhp

    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    rng = np.random.default_rng(B * 1000 + H)
    k = 1 / np.sqrt(H)
    p = dict(x=rng.normal(size=(B, L, D)), mu=rng.uniform(0.1, 1, (B, M)),
             alpha=rng.uniform(0, 0.5 / M, (B, M, M)), beta=rng.uniform(0.5, 2, (B, nb)),
             T=rng.uniform(5, 20, B), W=rng.uniform(-k, k, (4 * H, D)), U=rng.uniform(-k, k, (4 * H, H)),
             b=rng.uniform(-k, k, 4 * H), A=rng.uniform(-k, k, (H, M * M)),
             Bm=rng.uniform(-k / 20, k / 20, (H, nb)), C=rng.uniform(-k, k, (H, M)),
             Wy=rng.uniform(-k, k, (O, H)))
    y_ref, cache = lstm.forward(**p)
    dy = rng.normal(size=y_ref.shape)
    g_ref = lstm.backward(cache, dy)
    t = {n: torch.tensor(v, dtype=torch.float32, device="cuda", requires_grad=n != "T") for n, v in p.items()}
    y = mdhp.MdhpLSTMFunction.apply(t["x"], t["mu"], t["alpha"], t["beta"], t["T"], t["W"], t["U"],
                                    t["b"], t["A"], t["Bm"], t["C"], t["Wy"])
    y.backward(torch.tensor(dy, dtype=torch.float32, device="cuda"))
    np.testing.assert_allclose(y.detach().cpu().numpy(), y_ref, rtol=1e-4, atol=1e-5)
    names = dict(x="dx", W="dW", U="dU", b="db", A="dA", Bm="dBm", C="dC", Wy="dWy", mu="dmu",
                 alpha="dalpha", beta="dbeta")
    for n, gn in names.items():
        got = t[n].grad.cpu().numpy().reshape(-1)
        ref = np.asarray(g_ref[gn]).reshape(-1)
        scale = max(np.abs(ref).max(), 1e-12)
        assert np.max(np.abs(got - ref)) <= 2e-4 * scale, (n, np.max(np.abs(got - ref)) / scale)
