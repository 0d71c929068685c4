"""GB300-native Iterative Perturbation Theory (IPT) eigensolver.

IPT (Kenmoe, Kriemann, Smerlak, Zadorin, "A fast iterative algorithm for
near-diagonal eigenvalue problems", 2020) finds eigenpairs of M = D + Delta,
D = diag(theta), as fixed points of the quadratic map of Eq. (dyn):

    F(Z) = I + G o (Z D(Delta Z) - Delta Z),   G_jk = 1/(theta_j - theta_k).

The compute path lives in the CUDA library ``libipt.so`` behind the C ABI of
``include/ipt.h``; :mod:`paper_2012_14702_gb300.ipt` is its Python binding.
:mod:`paper_2012_14702_gb300.workloads` holds the seeded input generators.

Importing this package does not load the native library; importing
:mod:`paper_2012_14702_gb300.ipt` does, and raises if it is missing.
"""

__all__ = ["workloads"]
