"""FP64 CPU oracle for Variable Basis Mapping (VBM) -- TEST INFRASTRUCTURE ONLY.

This package is a plain, slow, obviously-correct restatement of what the VBM
path computes, written from the paper (arXiv 2601.09417) and from the 3D
Gaussian Splatting conventions the paper defers to for its fine-tuning loss
(Sec. 4.4).  It exists to check the CUDA path; it is never part of it.

Only the tests, `__graft_entry__.smoke()` and the CPU-baseline leg of
`bench.py` may import, call, link or execute anything under `oracle/`.  It
shares no code with the CUDA library and never imports it.

Modules (each function cites the passage it follows):
  filters   bior4.4 (CDF 9/7) and Haar filter banks              (Sec. 4.2, Sec. 5.2)
  dwt       periodised separable 3D DWT / IDWT, Mallat layout    (Sec. 3, Sec. 4.3)
  tf        piecewise-linear transfer function                    (Sec. 3)
  bank      wavelet-to-Gaussian transition bank                  (Sec. 4.2, Eq. 8-14)
  select    adaptive filtering: budget, MAD threshold, top-K     (Supp. Sec. 1)
  mapping   coefficient -> Gaussian construction                 (Sec. 4.3, Eq. 16-18)
  dvr       emission-absorption ray marching (targets)            (Sec. 4.4)
  raster    EWA projection, tile binning, compositing, backward   (Sec. 4.4, via 3DGS)
  loss      L1 + D-SSIM image loss and its gradient               (Sec. 4.4, via 3DGS)
  adam      Adam update                                           (Sec. 5.2)
  step      one fine-tuning step composed from the above          (Sec. 4.4)

Parity status: every function is pinned by a `-m "not gpu"` test against
something other than itself (closed forms, brute force, finite differences,
library routines, published filter values); none is "parity unpinned".
"""
