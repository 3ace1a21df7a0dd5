"""Multi-view differentiable Gaussian splatting on GB300 (sm_103a).

The compute path is libmvgs (CUDA kernels behind the C ABI in include/mvgs.h);
`mvgs` is its ctypes binding, `autograd` wraps it in torch.autograd.Function.
Importing `mvgs` fails loudly when the library has not been built.
"""
