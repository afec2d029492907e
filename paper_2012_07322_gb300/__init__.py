"""GB300-native non-linear cell-centred multigrid (FAS) solver for the xCFC
metric equations and elliptic divergence cleaning of Gmunu
(arXiv:2012.07322, Secs. 2.2, 2.6 and 2.7).

The compute path is the CUDA library ``libgmunu_mg.so`` behind the C ABI of
``include/mg.h``; :mod:`paper_2012_07322_gb300.mg` is its ctypes binding.
:mod:`paper_2012_07322_gb300.inputs` holds the seeded synthetic inputs.
"""
__all__ = ["inputs", "mg"]
