"""Learned candidate proposal: a small MLP trained on the exact method's labels proposes the
top-m centers of every point; the library checks the proposals exactly and certifies each
accepted label (see include/gbkm.h, kmeans_learned_assign).  This module holds the network's
device buffers and sequences the library's training and inference calls.
"""
from __future__ import annotations

import torch

from . import _binding as B
from . import synth


class ProposalNet:
    """Parameters (FP32 master + BF16 copy) and AdamW state of the d_in -> h -> h -> k network."""

    def __init__(self, d_in, hidden, k, seed=0, device="cuda:0", train=True):
        self.d_in, self.hidden, self.k = d_in, hidden, k
        self.step = 0
        p = torch.from_numpy(synth.mlp_init(d_in, hidden, k, seed)).to(device)
        assert p.numel() == B.kmeans_mlp_param_count(d_in, hidden, k)
        self.params = p
        self.params_bf16 = p.to(torch.bfloat16)
        self.adam_m = torch.zeros_like(p) if train else None
        self.adam_v = torch.zeros_like(p) if train else None
        mask = torch.zeros(p.numel(), dtype=torch.uint8, device=device)
        o = 0
        for rows, cols in ((hidden, d_in), (hidden, hidden), (k, hidden)):
            mask[o:o + rows * cols] = 1
            o += rows * cols + rows
        self.wd_mask = mask

    def load_params(self, p):
        self.params.copy_(p)
        self.params_bf16.copy_(p.to(torch.bfloat16))

    def train(self, Xh, labels, epochs=3, batch=4096, lr=2e-3, wd=1e-4, seed=0, ctx=None):
        """Mini-batch AdamW over (Xh, labels); returns the mean loss of every epoch (host floats)."""
        n = Xh.shape[0]
        g = torch.Generator(device="cpu").manual_seed(seed)
        losses = []
        loss_rows = torch.empty(batch, dtype=torch.float32, device=Xh.device)
        for _ in range(epochs):
            order = torch.randperm(n, generator=g).to(Xh.device)
            tot, cnt = torch.zeros((), dtype=torch.float64, device=Xh.device), 0
            for b0 in range(0, n - batch + 1, batch):
                idx = order[b0:b0 + batch]
                B.kmeans_mlp_train_step(self, Xh[idx].contiguous(), labels[idx].contiguous(), lr, wd,
                                        loss_rows=loss_rows, ctx=ctx)
                tot += loss_rows.double().sum()
                cnt += batch
            losses.append(float(tot.item()) / max(cnt, 1))
        return losses
