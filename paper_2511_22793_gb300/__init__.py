"""GB300-native equirectangular Gaussian splatting for RF spectra (GSpaRC hot path).

The compute path is the C-ABI library libgsparc.so (hand-written sm_103a
CUDA, declared in include/gsparc.h).  `gsparc` is its thin Python binding;
`autograd` wraps the forward/backward chain in a torch.autograd.Function.
`synth` holds the seeded input generators.
"""
__all__ = ["gsparc", "autograd", "synth"]
