"""CPU oracle for the Universal Beta Splatting rasterizer (arXiv 2510.03312).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
the CPU-baseline leg of ``bench.py`` may import or run anything in this
package.  The CUDA path never imports it and it never imports the CUDA path;
the two share only the seeded input generator
(``paper_2510_03312_gb300.scenes``), which holds none of the method's
arithmetic.

Modules
-------
``fp32_spec``  the FP32 decision stage: every integer the rasterizer derives
               from floating point (culls, depth sort keys, tile rectangles)
               written as individually rounded IEEE float32 operations with
               project-written exp/log (Cody-Waite reduction + Taylor
               polynomial; atanh series), so that an independent
               implementation of the same written rules reproduces it bit for
               bit.
``binning``    the sorted (tile, primitive) instance list and per-tile ranges,
               by their plain definition (a lexicographic sort).
``render64``   the method itself in float64 PyTorch CPU ops: spatial-
               orthogonal Cholesky covariance (Sec. 4.2), Beta-modulated
               conditioning and opacity (Sec. 4.3), EWA projection and the
               Beta kernel (Sec. 3), front-to-back compositing (Sec. 3);
               gradients by autograd of that float64 forward.
``train64``    the training step around the rasterizer (Sec. 4.5 loss,
               Sec. 5.1 optimiser): L1 + (1 - SSIM) image loss with its
               float64 autograd gradient, and the Adam step on raw
               parameters with the activation chain, the opacity and scale
               penalties and the spatial noise.
``mcmc64``     MCMC relocation (Sec. 4.5 primitive management): dead
               primitives moved onto live ones drawn by opacity with exact
               integer weights, cloned opacity 1 - (1 - o)^(1/N).

Every function names the passage it follows.  Parity status of each function
is given in its module header.
"""
