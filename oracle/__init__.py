"""FP64 CPU oracle for the image pipelines the fused GPU kernels compute.

TEST INFRASTRUCTURE ONLY. Nothing on the product path may import, call or
execute this package: only the test suite, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` use it.

Every function here is a plain, whole-image, stage-by-stage restatement of a
definition, in float64 (or exact integers), with no tiling, fusion or
reordering.  It shares no code with the CUDA path.  The workloads come from the
imaging apps the paper evaluates (Sec. 6: stencil chain, Harris corner
detection, local Laplacian, unsharp mask, histogram equalize, max filter,
interpolate, bilateral grid).  The paper names
them but does not define their arithmetic, so each module states the reading it
implements; those readings are listed again in the design notes.

Modules:
  stencil          clamp-to-edge 2-D stencils and stencil chains (Sec. 2, Fig. 1)
  harris           Harris corner response
  pyramid          binomial downsample / upsample, Gaussian & Laplacian pyramids
  local_laplacian  local Laplacian filter (remap, per-level interpolation, collapse)
  unsharp          unsharp mask
  histeq           256-bin histogram, CDF lookup table, equalization (exact ints)
  maxfilter        clamp-to-edge window maximum (exact)
  interpolate      premultiplied pyramid fill of a partially covered RGBA image
  bilateral_grid   splat / blur / slice bilateral filter of a gray image

Parity status: every function is pinned by tests in ``tests/test_oracle_*.py``
against closed forms, library routines (scipy.ndimage, numpy.bincount),
invariants and hand-worked examples; none is "parity unpinned".
"""

from . import stencil, harris, pyramid, local_laplacian, unsharp, histeq, maxfilter, interpolate, bilateral_grid  # noqa: F401
