"""FP64 CPU oracle for the grouped Fourier transform and its solvers.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import, call, link or run anything in this
package.  The library under ``paper_2010_10199_gb300`` never imports it, and
this package never imports the library: the two share no code.  The only
shared module is the input generator ``paper_2010_10199_gb300.inputs``, which
holds no arithmetic of the method.

Contents (each function cites the passage of the paper it follows):

* ``anova``   -- term sets U_{d_s}, grouped index sets I_N(U), coefficient layout
* ``ndft``    -- direct NDFT summation of F and F^H in FP64 (C, via ctypes)
* ``solvers`` -- LSQR (Tikhonov), the group-lasso prox, FISTA, KKT check,
                 direct normal-equation solve, sensitivity indices
* ``mlp``     -- FP64 forward/backward of the group-screening MLP
* ``ndct``    -- direct FP64 sums of the grouped half-period cosine transform
                 (the orthonormal system of Sec. 5, grouped as in the Remark on
                 other systems in Sec. 3)
"""
