"""FP64 CPU oracle for the nested-mesh convolution method (Vorobyov et al., 2023).

This package is TEST INFRASTRUCTURE.  Only ``tests/``, ``__graft_entry__.smoke()``
and the ``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import it.
The CUDA library never calls it, links it or falls back to it, and it imports
nothing from the CUDA package: the two share no code.

It is a plain, slow, step-by-step restatement of the method in float64 numpy:

* ``fft``         -- its own recursive radix-2 FFT (no library FFT on the path).
* ``green``       -- the inverse-distance kernel of Eq. 10 with the self-cell
                     term of Eq. 13, laid out on the doubled domain of Fig. 4.
* ``convolution`` -- the zero-padded (isolated) convolution of Sect. 3 and the
                     O(M^2) direct sum of Eq. 10.
* ``nested``      -- restriction, hole grids, trilinear interpolation and the
                     assembly of Eq. 14 (Sect. 4), plus the pairwise-dipole
                     variant of Eqs. 15 and B.1-B.2 (Sect. 7, Appendix B).
* ``acceleration``-- g = -grad Phi with the six-point stencil of Eq. 8 and the
                     interface rules of Sect. 2 / Appendix A (methods A, B).
* ``direct``      -- a second route to the same nested potential at sampled
                     cells using direct summation only (no FFT), for checks at
                     sizes where the FFT oracle is too slow.

Equation numbers follow the paper's LaTeX source as numbered by the A&A class
(main text 1-15, appendices A.x and B.x).  Readings of points where the paper is
silent or garbled are listed beside the functions that take them.
"""
from .fft import fft_axis, fft3, ifft3
from .green import SELF_TERM_C, green_kernel, green_spectrum
from .convolution import isolated_convolution, direct_sum
from .nested import (Geometry, restrict, level_masses, solve, trilinear_to_level,
                     solve_components)
from .direct import nested_potential_at
from .acceleration import acceleration

__all__ = [
    "fft_axis", "fft3", "ifft3", "SELF_TERM_C", "green_kernel", "green_spectrum",
    "isolated_convolution", "direct_sum", "Geometry", "restrict", "level_masses",
    "solve", "solve_components", "trilinear_to_level", "nested_potential_at", "acceleration",
]
