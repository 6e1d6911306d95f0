"""GB300-native adaptive hypergraph learning (Karantaidis, Sarridis and Kotropoulos,
"Block randomized optimization for adaptive hypergraph learning").

The compute path is libhgl.so, a C-ABI CUDA library for sm_103a (include/hgl.h);
``hgl`` is its Python binding (argument marshalling only) and ``build`` compiles it.
"""
from . import hgl  # noqa: F401
from .hgl import (HglError, adaptive_step, adjoint_grad, apply_theta, block_rsvd, build_incidence,  # noqa: F401
                  cg_solve, degrees, graph_export, padded_panel, precond_apply, precond_export,
                  project_simplex, weight_grad)
