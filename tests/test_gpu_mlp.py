"""GPU tests of the learned warm start: the BF16 tensor-core forward and backward kernels against
the FP64 MLP reference (oracle/mlp.py), and what a trained network gains over the cold start."""
import numpy as np
import pytest

import worldgen as wg
from oracle import mlp as OM

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


def _bf16(a):
    return torch.tensor(a, dtype=torch.float32).to(torch.bfloat16).to(torch.float64).numpy()


def test_mlp_forward_and_gradients_match_fp64_reference(K):
    """Identity normalisation, random inputs: the GPU forward and every parameter gradient agree
    with the FP64 reference evaluated at the same BF16-rounded weights and inputs, within the error
    that BF16 activations leave (relative 3e-2 on each tensor)."""
    ws = wg.make_biped(num_worlds=8, seed=1)
    model = K.Model(ws, "fp32", K.make_params())
    net = K.Mlp(model, np.arange(8), hidden=64, max_batch=256, seed=3)
    din, dout = net.info.d_in, net.info.d_out
    assert (din, dout) == (13 * 31 + 1 + 12 + 4 * 16 + (180 + 3 * 16), 180 + 3 * 16)   # ... + the impulse cache
    rng = np.random.default_rng(0)
    B = 96
    X = rng.standard_normal((B, din)).astype(np.float32)
    Y = rng.standard_normal((B, dout)).astype(np.float32)
    Xd, Yd = torch.tensor(X, device="cuda"), torch.tensor(Y, device="cuda")
    g, loss = net.gradients(Xd, Yd)
    pred = net.predict(Xd)
    torch.cuda.synchronize()
    Ws, bs = net.layer_params()
    Wr = [_bf16(w) for w in Ws]
    br = [b.astype(np.float64) for b in bs]
    xr = _bf16(X)
    y_ref, _ = OM.forward(Wr, br, xr)
    p = pred.cpu().numpy()
    assert np.linalg.norm(p - y_ref) / np.linalg.norm(y_ref) < 3e-2
    gW, gb = OM.backward(Wr, br, xr, Y.astype(np.float64))
    gl_W, gl_b = net.layer_params(g.cpu().numpy())
    for k in range(len(gW)):
        assert np.linalg.norm(gl_W[k] - gW[k]) / np.linalg.norm(gW[k]) < 3e-2, k
        assert np.linalg.norm(gl_b[k] - gb[k]) / np.linalg.norm(gb[k]) < 3e-2, k
    assert abs(loss.item() - OM.loss(Wr, br, xr, Y.astype(np.float64))) / OM.loss(Wr, br, xr, Y) < 3e-2


def test_trained_warm_start_cuts_iterations(K):
    """Solver-generated data (cold solves, 256 bipeds x 120 steps), a short training run, then on
    held-out steps the learned warm start needs fewer PADMM iterations to tol 1e-5 than the cold
    start and converges in more worlds; where both starts converged the solutions agree to the
    accuracy that tol 1e-5 gives on these mechanisms (the solver, not the network, decides)."""
    W, steps, dt, tol, iters = 256, 120, 2e-3, 1e-5, 400
    ws = wg.make_biped(num_worlds=W, seed=11)
    model = K.Model(ws, "fp32", K.make_params(rho=0.1))
    st = K.State(model)
    net = K.Mlp(model, np.arange(W), hidden=256, max_batch=4096, seed=0)
    X = torch.empty((steps * W, net.info.d_in), device="cuda")
    Y = torch.empty((steps * W, net.info.d_out), device="cuda")
    taus = [torch.tensor(wg.actuation(ws, 11, k), dtype=torch.float32, device="cuda") for k in range(steps + 20)]
    for k in range(steps):
        net.features(st, taus[k], out=X[k * W:(k + 1) * W])
        st.step(dt, iters, 1e-6, taus[k])
        net.targets(st, out=Y[k * W:(k + 1) * W])
    net.fit_normalization(X, Y)
    gen = torch.Generator(device="cuda").manual_seed(0)
    loss = torch.zeros(1, device="cuda")
    losses = []
    for it in range(1500):
        rows = torch.randint(0, steps * W, (1024,), device="cuda", generator=gen, dtype=torch.int32)
        loss.zero_()
        net.train_step(X, Y, rows, lr=1e-3 if it < 1000 else 3e-4, loss=loss)
        if it % 100 == 0:
            losses.append(loss.item())
    assert losses[-1] < 0.5 * losses[0]
    # held-out steps: same state trajectory continued, compare cold and learned warm starts
    q0, u0 = st.body_q.clone(), st.body_u.clone()
    cold, learned, diffs, conv_c, conv_l = [], [], [], [], []
    for k in range(steps, steps + 10):
        st.body_q.copy_(q0); st.body_u.copy_(u0)
        model.set_params(K.make_params(rho=0.1, warm_mode=K.WARM_COLD))
        st.step(dt, iters, tol, taus[k])
        rc = st.residuals(); uc = st.body_u.clone()
        st.body_q.copy_(q0); st.body_u.copy_(u0)
        net.warm_start(st, taus[k])
        model.set_params(K.make_params(rho=0.1, warm_mode=K.WARM_EXTERNAL))
        st.step(dt, iters, tol, taus[k])
        rl = st.residuals()
        cold.append(rc["iterations"].mean()); learned.append(rl["iterations"].mean())
        conv_c.append(np.mean(rc["status"] == 0)); conv_l.append(np.mean(rl["status"] == 0))
        both = np.nonzero((rc["status"] == 0) & (rl["status"] == 0))[0]
        ul, ucn = st.body_u.double().cpu().numpy(), uc.double().cpu().numpy()
        for w in both:
            b0, b1 = int(ws.world_body_offset[w]), int(ws.world_body_offset[w + 1])
            diffs.append(np.abs(ul[b0:b1] - ucn[b0:b1]).max() / max(np.abs(ucn[b0:b1]).max(), 9.81 * dt))
        q0, u0 = st.body_q.clone(), st.body_u.clone()
    assert np.mean(learned) < np.mean(cold), (np.mean(learned), np.mean(cold))
    assert np.mean(conv_l) >= np.mean(conv_c) - 0.02, (np.mean(conv_l), np.mean(conv_c))
    assert diffs and np.median(diffs) < 1e-2, (np.median(diffs), max(diffs))
