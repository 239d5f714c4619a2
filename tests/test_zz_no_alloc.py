"""Allocation-free inference of the warm-start network (kamino_mlp_predict_static).

Callers that cannot let memory be allocated for them -- a host framework that owns the device
allocator, or a real-time loop that cannot absorb the synchronisation of cudaMalloc -- use this
entry point: its activations live in a fixed file-scope device array of the library.  The test
checks it through the C ABI against the allocating kamino_mlp_predict on two calls in a row (the
second with different inputs, so a stale scratch would show), and that an oversized batch is
refused.  It sits in a file collected last so that a stop-at-first-failure run has already run the
rest of the suite."""
import numpy as np
import pytest

import worldgen as wg

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def K():
    import os
    import __graft_entry__ as ge
    from paper_2603_16536_gb300 import build as B, kamino
    if not os.path.exists(B.LIB):
        ge.build()
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return kamino


def test_static_scratch_prediction_matches_allocating_prediction(K):
    ws = wg.make_biped(num_worlds=16, seed=4)
    model = K.Model(ws, "mixed", K.make_params())
    net = K.Mlp(model, np.arange(16), hidden=128, max_batch=1024, seed=7)
    rng = np.random.default_rng(1)
    norm = net.get_normalization()
    din, dout = net.info.d_in, net.info.d_out
    norm[:din] = rng.standard_normal(din)                      # non-trivial normalisation
    norm[din:2 * din] = rng.uniform(0.5, 2.0, din)
    norm[2 * din:2 * din + dout] = rng.standard_normal(dout)
    norm[2 * din + dout:] = rng.uniform(0.5, 2.0, dout)
    net.set_normalization(norm)
    for batch in (1000, 37):                                   # two calls in a row, different sizes
        X = torch.tensor(rng.standard_normal((batch, din)), dtype=torch.float32, device="cuda")
        ref = net.predict(X)
        got = net.predict_static(X)
        torch.cuda.synchronize()
        torch.testing.assert_close(got, ref, rtol=1e-6, atol=1e-6)


def test_static_scratch_refuses_oversized_batch(K):
    ws = wg.make_biped(num_worlds=4, seed=5)
    model = K.Model(ws, "mixed", K.make_params())
    net = K.Mlp(model, np.arange(4), hidden=256, max_batch=64, seed=1)
    X = torch.zeros((20000, net.info.d_in), dtype=torch.float32, device="cuda")
    with pytest.raises(K.KaminoError) as err:
        net.predict_static(X)
    assert err.value.status == 7 and "static scratch" in str(err.value)


def test_static_scratch_at_its_limit(K):
    """The largest batch the refusal message names for a hidden-256 network fits the array (its
    activations packed up to the array's end) and matches the allocating path; one row more is
    refused."""
    import re
    ws = wg.make_biped(num_worlds=4, seed=6)
    model = K.Model(ws, "mixed", K.make_params())
    net = K.Mlp(model, np.arange(4), hidden=256, max_batch=8192, seed=2)
    din = net.info.d_in
    with pytest.raises(K.KaminoError) as err:
        net.predict_static(torch.zeros((20000, din), dtype=torch.float32, device="cuda"))
    rows = int(re.search(r"at most (\d+) rows", str(err.value)).group(1))
    assert 1000 < rows < 8192
    rng = np.random.default_rng(3)
    X = torch.tensor(rng.standard_normal((rows + 1, din)), dtype=torch.float32, device="cuda")
    for _ in range(2):                                         # two calls in a row at the limit
        got = net.predict_static(X[:rows])
        ref = net.predict(X[:rows])
        torch.cuda.synchronize()
        torch.testing.assert_close(got, ref, rtol=1e-6, atol=1e-6)
    with pytest.raises(K.KaminoError) as err:
        net.predict_static(X)
    assert err.value.status == 7
