"""GB300 (sm_103a) k-means hot path: block projection, k-means++ seeding, Lloyd assign/update
and cost, behind the C ABI of include/gbkm.h.

``synth`` (seeded inputs) imports without CUDA.  The binding functions load
libgbkm.so on first use and raise if it is not built; there is no CPU path.
"""
from __future__ import annotations

__all__ = [
    "kmeans_row_norms", "kmeans_quantize", "kmeans_project_block", "kmeans_seed_pp",
    "kmeans_assign", "kmeans_update", "kmeans_cost", "gbkm_sync", "gbkm_version",
    "Context", "default_context", "GbkmError", "lloyd", "kmeans_batch_run", "kmeans_batch_replay", "kmeans_autotune",
    "kmeans_autotune_assign",
    "kmeans_update_noalloc", "kmeans_update_scratch_bytes", "kmeans_ingest", "HostBlock", "kmeans_rsvd",
    "kmeans_piecy_lift", "kmeans_bico_query", "kmeans_center_separation", "kmeans_gemm_bf16",
    "kmeans_learned_assign", "kmeans_mlp_forward", "kmeans_mlp_param_count", "kmeans_mlp_train_step",
]


def __getattr__(name):
    if name in __all__:
        if name == "lloyd":
            from . import driver

            return driver.lloyd
        from . import _binding

        return getattr(_binding, name)
    raise AttributeError(name)
