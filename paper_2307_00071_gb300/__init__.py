"""GB300-native EM fitting of Gaussian mixture models to point clouds (GIRA,
arXiv 2307.00071, Sec. V).

Modules:
  gira       ctypes binding of the C ABI (include/gira.h): fits (single, batched,
             4D), log-likelihoods and their gradient, intensity regression,
             sampling, mode seeking; importing it loads (or builds) libgira.so
  autograd   torch.autograd binding of the log-likelihood gradient, SE(3) helpers
  model_io   the compact binary32 storage of a fitted model and its size
  synth      seeded synthetic inputs (GMM clouds, depth frames, intensity)
  build_lib  nvcc build of libgira.so for sm_103a
  fit_once   fixed-length runs for profiling
"""
