"""FP64 CPU oracle for the equirectangular Gaussian-splatting path.

TEST INFRASTRUCTURE.  Only the test suite, the smoke check and the CPU
baseline leg of the benchmark may import, call or link anything in this
package.  The library path never routes through it and shares no code with
it: the two meet only on the seeded arrays produced by the input generator.

Contents, each following the passage of the paper it cites:
  projection.py   receiver-centric transform, equirectangular map and the 2D
                  covariance J V Sigma V^T J^T (Sec. 4.2 "Directional
                  Projection and Splatting"; Sec. 3.2 for Sigma = R S S^T R^T)
  attributes.py   attribute network with the log-distance feature (Eq. 1)
  emission.py     the per-Gaussian emission network R^3 -> R^2 of Eq. 1 with its
                  element-wise sigmoid (Sec. 4.1, per Gaussian) and the 1/d toggle
  binsort.py      tile binning and front-to-back (receiver distance) ordering
                  (Algorithm 1, IntersectGaussians / Sort by depth)
  render_oracle.c per-pixel compositing of complex contributions across
                  subcarriers and its analytic gradient (Sec. 4.2 compositing
                  rule; Algorithm 1 inner loop)
  render.py       ctypes wrapper of render_oracle.c
  csi.py          spatial-mean CSI head (Eq. 2), channel loss (Eq. 3), NMSE
  spectrum_loss.py  magnitude-spectrum loss L1 + SSIM (Eq. 4) and its gradient
  confidence.py   confidence-weighted objective C L_task - alpha log C (Eq. 5)
  densify.py      adaptive density control: clone, split, prune, opacity reset
                  (Algorithm 1, densification branch)
  pipeline.py     the whole forward pass, the L2 or channel loss and the full
                  gradient
  adam.py         the Adam update (Algorithm 1, Adam step)

Readings of points the paper leaves open are listed in each module header.
"""
