"""GB300-native GW iteration (QAssemble, arXiv 2604.22223): CUDA kernels behind a C ABI.

    from paper_2604_22223_gb300 import qa
    ctx = qa.Context(model, precision="mixed")   # model: workloads.Model
    G, mu, n, stats = ctx.step()                  # one G -> P -> W -> Sigma -> G iteration
"""
from .builder import build  # noqa: F401
