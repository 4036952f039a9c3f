"""Argument checks of the Python binding: a mis-shaped operand is refused on the host, before the
library is loaded or any pointer is passed (a narrower operand than the sizes say would otherwise
be read out of bounds on the device).  CPU only: every case below fails in the checks."""
from types import SimpleNamespace

import pytest
import torch

from paper_1502_04265_gb300 import _binding as B

f32, f64, i32, i64, bf16 = torch.float32, torch.float64, torch.int32, torch.int64, torch.bfloat16
n, d, k = 40, 8, 5


def z(*shape, dtype=f32):
    return torch.zeros(shape, dtype=dtype)


def net(d_in=d, hidden=16, kk=k):
    return SimpleNamespace(d_in=d_in, hidden=hidden, k=kk, params=z(100), params_bf16=z(100, dtype=bf16),
                           adam_m=None, adam_v=None, wd_mask=None, step=0)


CASES = [
    ("row_norms: xnorm length", lambda: B.kmeans_row_norms(z(n, d), xnorm=z(n - 1))),
    ("quantize: Xq shape", lambda: B.kmeans_quantize(z(n, d), "bf16", Xq=z(n, d + 1, dtype=bf16))),
    ("quantize: fp8 scales shape", lambda: B.kmeans_quantize(z(n, d), "fp8", scales=z(n, 2))),
    ("ingest: xnorm length", lambda: B.kmeans_ingest(z(n, d), xnorm=z(n + 1), copy=False, quantize=False,
                                                     device="cuda:0")),
    ("rsvd: V shape", lambda: B.kmeans_rsvd(z(n, d), z(d, 6), 4, V=z(d, 5))),
    ("rsvd: Omega rows", lambda: B.kmeans_rsvd(z(n, d), z(d + 1, 6), 4)),
    ("project: Y shape", lambda: B.kmeans_project_block(z(n, d), z(d, 3), Y=z(n, 4))),
    ("project: X_lift shape", lambda: B.kmeans_project_block(z(n, d), z(d, 3), Y=z(n, 3), X_lift=z(n, d - 1))),
    ("assign: C width", lambda: B.kmeans_assign(z(n, d), z(k, d - 1))),
    ("update: C_old width", lambda: B.kmeans_update(z(n, d), z(n, dtype=i32), z(k, d + 1))),
    ("update_noalloc: counts length", lambda: B.kmeans_update_noalloc(z(n, d), z(n, dtype=i32), z(k, d),
                                                                        counts=z(k + 1, dtype=f64))),
    ("cost: C width", lambda: B.kmeans_cost(z(n, d), z(k, d - 1))),
    ("cost: w length", lambda: B.kmeans_cost(z(n, d), z(k, d), w=z(n - 1))),
    ("cost: cost dtype", lambda: B.kmeans_cost(z(n, d), z(k, d), cost=z(1))),
    ("batch: C_out shape", lambda: B.kmeans_batch_run([{"X": z(n, d), "k": k, "u": z(2, k, dtype=f64),
                                                        "C_out": z(2, k, d - 1)}], 2, 1)),
    ("gemm: B width", lambda: B.kmeans_gemm_bf16(z(16, 32, dtype=bf16), z(16, 24, dtype=bf16))),
    ("gemm: Y rows", lambda: B.kmeans_gemm_bf16(z(16, 32, dtype=bf16), z(16, 32, dtype=bf16), Y=z(8, 16))),
    ("mlp_forward: Xh width", lambda: B.kmeans_mlp_forward(net(), z(n, d + 1, dtype=bf16))),
    ("mlp_forward: top_idx shape", lambda: B.kmeans_mlp_forward(net(), z(n, d, dtype=bf16),
                                                                top_idx=z(n, 4, dtype=i32), topm=8)),
    ("mlp_train: labels length", lambda: B.kmeans_mlp_train_step(net(), z(n, d, dtype=bf16), z(n - 8, dtype=i32),
                                                                 1e-3)),
    ("mlp_train: grad_out length", lambda: B.kmeans_mlp_train_step(net(), z(n, d, dtype=bf16), z(n, dtype=i32),
                                                                   1e-3, grad_out=z(99))),
    ("separation: s2 length", lambda: B.kmeans_center_separation(z(k, d), s2=z(k + 1))),
    ("learned: C shape", lambda: B.kmeans_learned_assign(net(), z(n, d), z(n, d, dtype=bf16), z(k + 1, d), z(k + 1))),
    ("learned: Xh shape", lambda: B.kmeans_learned_assign(net(), z(n, d), z(n - 1, d, dtype=bf16), z(k, d), z(k))),
    ("learned: X width", lambda: B.kmeans_learned_assign(net(), z(n, d + 1), z(n, d + 1, dtype=bf16), z(k, d + 1),
                                                         z(k))),
    ("bico: S shape", lambda: B.kmeans_bico_query(z(n, d), z(k, d), z(k, dtype=f64), z(k, d - 1, dtype=f64),
                                                  z(k, dtype=f64), 1.0)),
]


@pytest.mark.parametrize("name,call", CASES, ids=[c[0] for c in CASES])
def test_mis_shaped_operand_is_refused(name, call):
    with pytest.raises((ValueError, TypeError)):
        call()


def test_cross_device_operands_are_refused():
    class Fake:
        device = torch.device("cuda", 1)

    with pytest.raises(ValueError, match="is on"):
        B._same_device(z(2), C=Fake())
