"""GB300-native equirectangular Gaussian splatting for RF spectra (GSpaRC hot path).

The compute path is the C-ABI library libgsparc.so (hand-written sm_103a
CUDA, declared in include/gsparc.h).  `gsparc` is its thin Python binding;
`pipeline` owns the buffers of one view / band / scene size; `autograd` wraps
the forward/backward chain in a torch.autograd.Function; `train` is the
training loop, `serve` the continuous-batching query server, `replicas` the
host logic of the multi-GPU form; `synth` holds the seeded input generators
and `build` compiles the library.
"""
__all__ = ["gsparc", "pipeline", "autograd", "train", "serve", "replicas", "synth", "build"]
