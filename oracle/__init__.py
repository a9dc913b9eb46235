"""FP64 CPU oracle of V3DG's online path (selection + splatting).

TEST INFRASTRUCTURE ONLY: this package exists to check the CUDA library.  Only the tests,
``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may import it; the
library and its Python binding never do, and the two share no code.

Parity status per function (what pins it lives in tests/test_oracle_*.py):
  compose, footprint ........ pinned (ray-cast pixel area, hand-worked values, composition)
  select, cover_counts ...... pinned (hand-worked tree, tau->0 / tau->inf, exact cover)
  sh_basis, sh_color ........ pinned (orthonormality by quadrature, parity, degree 0)
  project ................... pinned (isotropic closed forms, clamp, rotation invariance,
                              instance = world Gaussian)
  sorted_pairs, blend_order . pinned (brute-force sort on small inputs)
  render_pixels, render_image pinned (one-Gaussian closed form, two layers, stop rule,
                              pixelwise == Gaussian-wise)
"""
from .core import *  # noqa: F401,F403
