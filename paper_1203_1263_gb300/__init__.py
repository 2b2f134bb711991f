"""GB300-native RK4 integrator for the NLSE / Gross-Pitaevskii equation
(CD and 2SHOC Laplacians, Dirichlet, MSD and Laplacian-zero boundaries), after
arXiv 1203.1263.

The compute path is the CUDA library libnlse.so (C ABI in include/nlse.h);
this package only marshals arguments and owns device memory through torch.
"""
from . import workloads  # noqa: F401


def __getattr__(name):
    if name in ("Integrator", "max_dt", "workspace_bytes"):
        from . import integrator
        return getattr(integrator, name)
    raise AttributeError(name)
