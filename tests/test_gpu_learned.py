"""Learned candidate proposal on the GPU against the FP64 oracle.

The GEMM building block is checked against numpy on the same BF16 inputs; the network's
forward pass and its batch gradient against the oracle's FP64 network (BF16 operands and
activations on the GPU, hence the 2^-7-level tolerances); the AdamW update against the oracle's
formula given the GPU's gradient; the fused top-m against the top-m of the GPU's own logits;
and the learned assignment against the exact method's labels (the certificate makes them equal).
"""
import numpy as np
import pytest
import torch

from oracle import mlp as omlp
from paper_1502_04265_gb300 import synth

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def bf(a):
    return torch.from_numpy(np.ascontiguousarray(a, np.float32)).to(DEV).to(torch.bfloat16)


def as64(t):
    torch.cuda.synchronize()
    return t.float().cpu().numpy().astype(np.float64)


@pytest.mark.parametrize("M,N,K", [(300, 64, 64), (129, 400, 256), (1000, 16, 8)])
@pytest.mark.parametrize("act,out_bf16", [(0, False), (1, True)])
def test_gemm_bf16_epilogue(gb, M, N, K, act, out_bf16):
    rng = np.random.default_rng(M + N + K)
    A, Bm = bf(rng.normal(size=(M, K))), bf(rng.normal(size=(N, K)))
    bias = torch.from_numpy(rng.normal(size=N).astype(np.float32)).to(DEV)
    Y = gb.kmeans_gemm_bf16(A, Bm, bias=bias, act=act, out_bf16=out_bf16)
    ref = as64(A) @ as64(Bm).T + bias.cpu().numpy().astype(np.float64)
    if act == 1:
        ref = omlp.gelu(ref)
    tol = (2.0 ** -8 if out_bf16 else 0.0) * np.abs(ref) + K * 2.0 ** -22 * np.sqrt(K) * 4 + 1e-5
    assert np.all(np.abs(as64(Y) - ref) <= tol)


def _net(gb, d, h, k, seed=0):
    from paper_1502_04265_gb300.learned import ProposalNet

    return ProposalNet(d, h, k, seed=seed, device=DEV)


def test_mlp_forward_matches_oracle(gb):
    d, h, k, n = 64, 64, 160, 300
    net = _net(gb, d, h, k)
    X = np.random.default_rng(1).normal(size=(n, d)).astype(np.float32)
    Xh = bf(X)
    logits = torch.empty((n, k), dtype=torch.float32, device=DEV)
    gb.kmeans_mlp_forward(net, Xh, logits=logits)
    ref = omlp.forward(net.params_bf16.float().cpu().numpy(), as64(Xh), d, h, k)["z"]
    err = np.abs(as64(logits) - ref)
    assert err.max() <= 2.0 ** -6 * (np.abs(ref).max() + 1.0)


def test_topm_epilogue_equals_topm_of_logits(gb):
    d, h, k, n, m = 64, 64, 2048, 513, 32
    net = _net(gb, d, h, k, seed=3)
    Xh = bf(np.random.default_rng(2).normal(size=(n, d)) * 2)
    logits = torch.empty((n, k), dtype=torch.float32, device=DEV)
    top = torch.empty((n, m), dtype=torch.int32, device=DEV)
    gb.kmeans_mlp_forward(net, Xh, logits=logits, top_idx=top, topm=m)
    Z, T = logits.cpu().numpy(), top.cpu().numpy()
    for i in range(n):
        sel = T[i]
        assert len(set(sel.tolist())) == m and sel.min() >= 0
        thr = np.sort(Z[i])[-m]
        assert np.all(Z[i, sel] >= thr)


def test_train_step_gradient_and_adamw_match_oracle(gb):
    d, h, k, Bn = 64, 64, 160, 128
    net = _net(gb, d, h, k, seed=5)
    rng = np.random.default_rng(4)
    Xh = bf(rng.normal(size=(Bn, d)))
    y = rng.integers(0, k, size=Bn).astype(np.int32)
    p_before = net.params.cpu().numpy().astype(np.float64)
    pb = net.params_bf16.float().cpu().numpy().astype(np.float64)
    grad = torch.empty_like(net.params)
    loss = torch.empty(Bn, dtype=torch.float32, device=DEV)
    lr, wd = 1e-3, 0.01
    gb.kmeans_mlp_train_step(net, Xh, torch.from_numpy(y).to(DEV), lr, wd, loss_rows=loss, grad_out=grad)
    L, g_ref = omlp.loss_and_grad(pb, as64(Xh), y, d, h, k)
    assert float(loss.double().mean()) == pytest.approx(L, rel=2e-2)
    g = grad.cpu().numpy().astype(np.float64)
    lay, _ = omlp.layout(d, h, k)
    for name, (o, shp) in lay.items():
        sz = int(np.prod(shp))
        a, b = g[o:o + sz], g_ref[o:o + sz]
        assert np.linalg.norm(a - b) <= 5e-2 * np.linalg.norm(b) + 1e-6, name
    # AdamW: the oracle's update applied to the GPU's own gradient
    mask = omlp.wd_mask(d, h, k)
    p_ref, _, _ = omlp.adamw_step(p_before, g, np.zeros_like(g), np.zeros_like(g), 1, lr, wd, mask)
    np.testing.assert_allclose(net.params.cpu().numpy(), p_ref, rtol=1e-5, atol=1e-7)
    assert net.step == 1


def _clustered(n, d, k, seed):
    X, z, prm = synth.gaussian_mixture(n, d, k, seed=seed, return_params=True)
    return X, z, prm["mu"]


def test_training_lowers_the_loss(gb):
    d, h, k = 64, 64, 32
    X, z, mu = _clustered(8192, d, k, seed=11)
    Xh = bf(X)
    lab = torch.from_numpy(z.astype(np.int32)).to(DEV)
    net = _net(gb, d, h, k, seed=1)
    losses = net.train(Xh, lab, epochs=4, batch=1024, lr=3e-3)
    assert losses[-1] < 0.5 * losses[0]


def test_learned_assign_labels_are_exact(gb):
    d, h, k = 64, 64, 64
    # one mixture: the first 20,000 points are assigned, the last 8,192 (held out) train the net
    Xall, z, mu = _clustered(28192, d, k, seed=12)
    X, Xt = Xall[:20000], Xall[20000:]
    C = torch.from_numpy(mu.astype(np.float32)).to(DEV)
    Xg = torch.from_numpy(np.ascontiguousarray(X)).to(DEV)
    Xh = Xg.to(torch.bfloat16)
    exact = gb.kmeans_assign(Xg, C, compute="f32")
    Xtg = torch.from_numpy(np.ascontiguousarray(Xt)).to(DEV)
    lt = gb.kmeans_assign(Xtg, C, compute="f32")
    net = _net(gb, d, h, k, seed=2)
    net.train(Xtg.to(torch.bfloat16), lt, epochs=6, batch=1024, lr=3e-3)
    s2 = gb.kmeans_center_separation(C)
    labels, nf = gb.kmeans_learned_assign(net, Xg, Xh, C, s2, topm=8)
    gb.gbkm_sync()
    assert torch.equal(labels, exact)
    assert int(nf.item()) < 20000 // 10


def test_topm_order_is_rank_order(gb):
    """The top-m indices come in decreasing logit order (equal logits by increasing index)."""
    d, h, k, n, m = 64, 64, 1024, 257, 32
    net = _net(gb, d, h, k, seed=7)
    Xh = bf(np.random.default_rng(8).normal(size=(n, d)))
    logits = torch.empty((n, k), dtype=torch.float32, device=DEV)
    top = torch.empty((n, m), dtype=torch.int32, device=DEV)
    gb.kmeans_mlp_forward(net, Xh, logits=logits, top_idx=top, topm=m)
    Z, T = logits.cpu().numpy(), top.cpu().numpy()
    for i in range(n):
        ref = np.lexsort((np.arange(k), -Z[i]))[:m]
        assert np.array_equal(T[i], ref)


def test_grouped_proposal_is_best_of_top_groups(gb):
    """group 16: the best center of each aligned 16-center group competes; the m best offers come
    back in decreasing logit order (ties by lower index), checked against the GPU's own logits."""
    d, h, k, n, m = 64, 64, 2048 + 48, 300, 32
    net = _net(gb, d, h, k, seed=9)
    Xh = bf(np.random.default_rng(10).normal(size=(n, d)))
    logits = torch.empty((n, k), dtype=torch.float32, device=DEV)
    top = torch.empty((n, m), dtype=torch.int32, device=DEV)
    gb.kmeans_mlp_forward(net, Xh, logits=logits, top_idx=top, topm=m, group=16)
    Z, T = logits.cpu().numpy(), top.cpu().numpy()
    for i in range(n):
        G = Z[i].reshape(-1, 16)
        best = G.argmax(1) + 16 * np.arange(G.shape[0])   # argmax: first index of the maximum
        vals = Z[i][best]
        ref = best[np.lexsort((best, -vals))][:m]
        assert np.array_equal(T[i], ref)
