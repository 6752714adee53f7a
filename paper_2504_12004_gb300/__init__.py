"""GB300-native Scaled Block Vecchia (arxiv 2504.12004): the likelihood hot path.

The computation lives in libsbv.so (CUDA kernels for sm_103a behind the C
ABI of include/sbv.h); this package only builds it and marshals arguments.

    from paper_2504_12004_gb300 import Context
    ctx = Context(0)
    b = ctx.sbv_blocking(X, beta_scale, bc, kmeans_iters, seed)
    nbr, cnt = ctx.sbv_knn(X, beta_scale, b["ptr"], b["pts"], b["rank"], b["centres"], m)
    ll = ctx.sbv_loglik(X, y, b["ptr"], b["pts"], nbr, cnt, theta, nu2=5, precision="mixed")
    ll, grad = ctx.sbv_loglik_grad(X, y, b["ptr"], b["pts"], nbr, cnt, theta, nu2=5)  # FP64

One evaluation split over ranks (contiguous block ranges, rank-ordered sum):
paper_2504_12004_gb300.shard.
"""
from ._lib import (SBV_F32, SBV_F64, SBV_PREC_FP64, SBV_PREC_MIXED, Context, LoglikGraph,  # noqa: F401
                   Mlp, SBVError, load)

__all__ = ["Context", "LoglikGraph", "Mlp", "SBVError", "load", "SBV_F32", "SBV_F64", "SBV_PREC_FP64",
           "SBV_PREC_MIXED"]
